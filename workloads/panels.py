"""Gauss-Legendre boundary panels ("chunks", paper Sec. 2.2).

A closed curve is split into ``n_panels`` equal parameter ranges; each carries
``order`` Gauss-Legendre nodes.  The boundary quadrature weight of a node is
|gamma'(t)| * (dt/2) * w_GL, so sum_j g(x_j) w_j approximates the arc-length
integral of g.  Panels are stored consecutively in the direction of travel,
so panel i is adjacent to panels i-1 and i+1 (cyclically).
"""
from __future__ import annotations

import numpy as np

from .quadrature import gauss_legendre


def make_panels(curve, n_panels, order=16, t0=0.0):
    x, wgl = gauss_legendre(order)
    dt = 2 * np.pi / n_panels
    starts = t0 + dt * np.arange(n_panels)
    t = (starts[:, None] + (x[None, :] + 1.0) * dt / 2).reshape(-1)
    xy = curve.point(t)
    sp = curve.speed(t)
    w = (sp.reshape(n_panels, order) * wgl[None, :] * dt / 2).reshape(-1)
    nrm = curve.outward_normal(t)
    return {
        "n_panels": int(n_panels),
        "order": int(order),
        "t": t,
        "xy": np.ascontiguousarray(xy),
        "w": np.ascontiguousarray(w),
        "normal": np.ascontiguousarray(nrm),
    }


def make_square_panels(half, panels_per_side, order=16):
    """Straight panels on the boundary of [-half, half]^2, counter-clockwise."""
    x, wgl = gauss_legendre(order)
    h = float(half)
    corners = np.array([[-h, -h], [h, -h], [h, h], [-h, h]])
    xy, w, nrm = [], [], []
    outward = np.array([[0.0, -1.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])
    for s in range(4):
        a, b = corners[s], corners[(s + 1) % 4]
        for p in range(panels_per_side):
            pa = a + (b - a) * p / panels_per_side
            pb = a + (b - a) * (p + 1) / panels_per_side
            u = (x + 1.0) / 2
            xy.append(pa[None, :] + u[:, None] * (pb - pa)[None, :])
            w.append(wgl * np.linalg.norm(pb - pa) / 2)
            nrm.append(np.repeat(outward[s][None, :], order, axis=0))
    return {
        "n_panels": 4 * panels_per_side,
        "order": int(order),
        "xy": np.ascontiguousarray(np.concatenate(xy)),
        "w": np.ascontiguousarray(np.concatenate(w)),
        "normal": np.ascontiguousarray(np.concatenate(nrm)),
    }
