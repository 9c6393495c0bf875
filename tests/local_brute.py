"""Brute-force local heat integrals and exact tangent-frame derivatives, used to
pin the oracle's asymptotic expansions (Sec. 4).

Independent of the oracle: the local integrals are computed by adaptive
quadrature of their definitions (eq. sheatloc, eq. dheatloc and the local
term of eq. heatdecompdefs, time-integrated with eq. eiformula), and the
frame derivatives by sampling the curve as a graph over its tangent line and
fitting a Chebyshev polynomial.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, special


def closest_param(curve, x, t_guess=None):
    """Parameter of the closest point of an analytic curve to x."""
    if t_guess is None:
        ts = np.linspace(0, 2 * np.pi, 4096, endpoint=False)
        d = np.sum((curve.point(ts) - x) ** 2, axis=1)
        t = ts[np.argmin(d)]
    else:
        t = t_guess
    for _ in range(50):
        g = curve.deriv(np.array([t]), 0)[0] - x
        g1 = curve.deriv(np.array([t]), 1)[0]
        g2 = curve.deriv(np.array([t]), 2)[0]
        f = g @ g1
        fp = g1 @ g1 + g @ g2
        dt = f / fp
        t -= dt
        if abs(dt) < 1e-15:
            break
    return t


def tangent_frame_jet(curve, tb, dens_funcs=(), h=0.04, deg=14):
    """kappa = gamma'', gamma''', gamma'''' and density xi-derivatives (orders
    0..4) at curve(tb), in the frame (T, N_inward), by a Chebyshev fit of the
    curve written as a graph over its tangent line."""
    b = curve.point(tb)[0]
    d1 = curve.deriv(np.array([tb]), 1)[0]
    T = d1 / np.linalg.norm(d1)
    N = np.array([-T[1], T[0]])
    j = np.arange(deg + 1)
    xi = h * np.cos(np.pi * (j + 0.5) / (deg + 1))
    ts = np.empty_like(xi)
    for i, x in enumerate(xi):
        t = tb + x / np.linalg.norm(d1)
        for _ in range(60):
            p = curve.deriv(np.array([t]), 0)[0]
            g1 = curve.deriv(np.array([t]), 1)[0]
            r = (p - b) @ T - x
            dt = r / (g1 @ T)
            t -= dt
            if abs(dt) < 1e-16:
                break
        ts[i] = t
    eta = (curve.point(ts) - b) @ N
    cheb = np.polynomial.chebyshev.Chebyshev.fit(xi, eta, deg, domain=[-h, h])
    out = {"b": b, "T": T, "N": N,
           "kappa": cheb.deriv(2)(0.0), "g3": cheb.deriv(3)(0.0), "g4": cheb.deriv(4)(0.0)}
    dens = []
    for f in dens_funcs:
        c = np.polynomial.chebyshev.Chebyshev.fit(xi, f(ts), deg, domain=[-h, h])
        dens.append([c(0.0)] + [c.deriv(k)(0.0) for k in range(1, 5)])
    out["dens"] = dens
    return out


def _window(curve, tb, x, delta, reach=14.0):
    """Parameter interval around tb covering the part of the curve within
    reach*sqrt(delta) of x."""
    sp = np.linalg.norm(curve.deriv(np.array([tb]), 1)[0])
    R = reach * math.sqrt(delta) + np.linalg.norm(curve.point(tb)[0] - x)
    return tb - 1.5 * R / sp, tb + 1.5 * R / sp


def brute_single(curve, sigma, x, delta, tb):
    """S_L(x) = int_Gamma E1(|x-y|^2/(4 delta))/(4 pi) sigma ds (eq. sheatloc, eq. eiformula)."""
    a, b = _window(curve, tb, x, delta)

    def f(t):
        y = curve.point(t)[0]
        r2 = float(np.sum((x - y) ** 2))
        sp = np.linalg.norm(curve.deriv(np.array([t]), 1)[0])
        z = r2 / (4 * delta)
        return (special.exp1(z) if z > 0 else 0.0) / (4 * math.pi) * sigma(t) * sp

    v1, _ = integrate.quad(f, a, tb, limit=400, epsabs=1e-15, epsrel=1e-13)
    v2, _ = integrate.quad(f, tb, b, limit=400, epsabs=1e-15, epsrel=1e-13)
    return v1 + v2


def brute_double(curve, mu, x, delta, tb):
    """D_L(x) = int_Gamma exp(-r^2/(4 delta)) nu_y.(x-y)/(2 pi r^2) mu ds,
    the source-point normal derivative of E1(r^2/(4 delta))/(4 pi)."""
    a, b = _window(curve, tb, x, delta)

    def f(t):
        y = curve.point(t)[0]
        nu = curve.outward_normal(t)[0]
        d = x - y
        r2 = float(d @ d)
        sp = np.linalg.norm(curve.deriv(np.array([t]), 1)[0])
        if r2 == 0.0:
            return 0.0
        return math.exp(-r2 / (4 * delta)) * float(nu @ d) / (2 * math.pi * r2) * mu(t) * sp

    v1, _ = integrate.quad(f, a, tb, limit=400, epsabs=1e-15, epsrel=1e-13)
    v2, _ = integrate.quad(f, tb, b, limit=400, epsabs=1e-15, epsrel=1e-13)
    return v1 + v2


def brute_volume(curve_exit, f, x, delta, n_phi=512, reach=14.0):
    """V_L(x) = int_Omega E1(|x-y|^2/(4 delta))/(4 pi) f(y) dy for x inside a
    convex domain: polar coordinates around x, ray length to the boundary
    given by curve_exit(x, phi); trapezoid rule in phi (periodic, smooth),
    adaptive quadrature in rho."""
    Rcap = reach * math.sqrt(delta)
    phis = 2 * math.pi * np.arange(n_phi) / n_phi
    total = 0.0
    for ph in phis:
        e = np.array([math.cos(ph), math.sin(ph)])
        rmax = min(curve_exit(x, e), Rcap)

        def g(rho):
            if rho == 0.0:
                return 0.0
            y = x + rho * e
            return special.exp1(rho * rho / (4 * delta)) / (4 * math.pi) * f(y[None, :])[0] * rho

        v, _ = integrate.quad(g, 0.0, rmax, limit=200, epsabs=1e-16, epsrel=1e-12)
        total += v
    return total * 2 * math.pi / n_phi


def ellipse_exit(a, b):
    def exit_len(x, e):
        # solve ((x0 + r e0)/a)^2 + ((x1 + r e1)/b)^2 = 1 for r > 0
        A = (e[0] / a) ** 2 + (e[1] / b) ** 2
        B = 2 * (x[0] * e[0] / a ** 2 + x[1] * e[1] / b ** 2)
        C = (x[0] / a) ** 2 + (x[1] / b) ** 2 - 1.0
        return (-B + math.sqrt(B * B - 4 * A * C)) / (2 * A)
    return exit_len
