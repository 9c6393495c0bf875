"""f-jets at targets estimated from node values (test infrastructure only).

The volume expansion of Sec. 4 needs, at each target, the value and the
first and second derivatives of f (eq. vplocO5; the far form delta f +
delta^2/2 lap f).  The paper computes them analytically (Sec. 6.1); a
caller that has only f at the quadrature nodes needs an estimate.  This is
the plain statement of the estimator the CUDA path implements (the reading
is the library's own, the paper gives none):

  * neighbours: the nodes y_j with |y_j - x| < rho, rho = sqrt(3 delta_1)
    (three mean node spacings when delta_1 = 3 x mean weight, Sec. 6);
  * weights (1 - |y_j - x|^2 / rho^2)^2;
  * weighted least squares of f_j on the quadratic basis
    1, u, v, u^2, u v, v^2 in (u, v) = (y_j - x) / rho when there are at
    least 10 neighbours, on 1, u, v with 4 to 9, the weighted mean with 1
    to 3, and a zero jet with none (a target away from every node, e.g.
    outside the domain);
  * the value is replaced by f at a node within 1e-12 x (box side) of the
    target.

The jet is (f, f_x, f_y, f_xx, f_xy, f_yy) = (c0, c1/rho, c2/rho,
2 c3/rho^2, c4/rho^2, 2 c5/rho^2).
"""
from __future__ import annotations

import numpy as np


def jet_radius(delta):
    return float(np.sqrt(3.0 * delta))


def _cholesky_solve(A, b):
    """Solution of A c = b by Cholesky factorisation, or None when a pivot is
    not above 1e-12 A[0, 0]."""
    n = len(b)
    L = np.zeros((n, n))
    for j in range(n):
        d = A[j, j] - np.dot(L[j, :j], L[j, :j])
        if not d > 1e-12 * A[0, 0]:
            return None
        L[j, j] = np.sqrt(d)
        for i in range(j + 1, n):
            L[i, j] = (A[i, j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    y = np.zeros(n)
    for i in range(n):
        y[i] = (b[i] - np.dot(L[i, :i], y[:i])) / L[i, i]
    c = np.zeros(n)
    for i in range(n - 1, -1, -1):
        c[i] = (y[i] - np.dot(L[i + 1:, i], c[i + 1:])) / L[i, i]
    return c


def estimate_jets(src_xy, src_f, tgt_xy, delta, box_side):
    from scipy.spatial import cKDTree
    src_xy = np.asarray(src_xy, dtype=np.float64)
    src_f = np.asarray(src_f, dtype=np.float64)
    tgt_xy = np.atleast_2d(np.asarray(tgt_xy, dtype=np.float64))
    rho = jet_radius(delta)
    on_tol = 1e-12 * box_side
    tree = cKDTree(src_xy)
    out = np.zeros((len(tgt_xy), 6))
    for i, x in enumerate(tgt_xy):
        idx = np.array(tree.query_ball_point(x, rho), dtype=np.int64)
        if idx.size:
            d = (src_xy[idx] - x) / rho
            r2 = np.sum(d * d, axis=1)
            keep = r2 < 1.0
            idx, d, r2 = idx[keep], d[keep], r2[keep]
        n = idx.size
        if n == 0:
            continue
        w = (1.0 - r2) ** 2
        fj = src_f[idx]
        u, v = d[:, 0], d[:, 1]
        B = np.stack([np.ones(n), u, v, u * u, u * v, v * v], axis=1)
        A = B.T @ (w[:, None] * B)
        b = B.T @ (w * fj)
        c = _cholesky_solve(A, b) if n >= 10 else None
        if c is None and n >= 4:
            c = _cholesky_solve(A[:3, :3], b[:3])
        if c is None:
            c = np.array([b[0] / A[0, 0]])
        jet = np.zeros(6)
        jet[0] = c[0]
        if c.size >= 3:
            jet[1], jet[2] = c[1] / rho, c[2] / rho
        if c.size == 6:
            jet[3], jet[4], jet[5] = 2 * c[3] / rho ** 2, c[4] / rho ** 2, 2 * c[5] / rho ** 2
        k = int(np.argmin(np.sum((src_xy[idx] - x) ** 2, axis=1)))
        if np.hypot(*(src_xy[idx[k]] - x)) <= on_tol:
            jet[0] = fj[k]
        out[i] = jet
    return out
