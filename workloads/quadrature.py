"""Quadrature rules used to discretise the domain and its boundary.

* Gauss-Legendre nodes/weights on [-1, 1] (numpy's implementation).
* A fully symmetric 6-node triangle rule of polynomial degree 4.  It is
  obtained here by solving its moment equations with Newton's method; no
  tabulated values are used.  The paper discretises each triangle with a
  6-node rule (Sec. 6); any smooth rule serves the method equally.
"""
from __future__ import annotations

import functools
import math
import numpy as np


def gauss_legendre(p):
    x, w = np.polynomial.legendre.leggauss(int(p))
    return x, w


def _orbit_invariants(a):
    """Values of e2, e3, e2^2 at the barycentric point (a, a, 1-2a)."""
    l3 = 1.0 - 2.0 * a
    e2 = a * a + 2.0 * a * l3
    e3 = a * a * l3
    return np.array([e2, e3, e2 * e2])


# Area-averaged invariants over a triangle, from the Dirichlet moment formula
# avg(l1^i l2^j l3^k) = 2 i! j! k! / (i+j+k+2)!.
_AVG = np.array([3 * 2 / math.factorial(4),                       # e2
                 2 / math.factorial(5),                           # e3
                 3 * 2 * 4 / math.factorial(6) + 2 * 2 / math.factorial(5)])  # e2^2


def _residual(v):
    a1, a2, w1, w2 = v
    r = np.empty(4)
    r[0] = 3 * w1 + 3 * w2 - 1.0
    r[1:] = 3 * w1 * _orbit_invariants(a1) + 3 * w2 * _orbit_invariants(a2) - _AVG
    return r


@functools.lru_cache(maxsize=1)
def triangle_rule6():
    """Return (bary[6,3], weights[6]) with weights summing to 1 (i.e. area-
    normalised).  Exact for all polynomials of degree <= 4."""
    v = np.array([0.1, 0.4, 1 / 6, 1 / 6])
    for _ in range(60):
        r = _residual(v)
        if np.max(np.abs(r)) < 1e-15:
            break
        J = np.empty((4, 4))
        h = 1e-7
        for j in range(4):
            dv = np.zeros(4)
            dv[j] = h
            J[:, j] = (_residual(v + dv) - _residual(v - dv)) / (2 * h)
        v = v - np.linalg.solve(J, r)
    a1, a2, w1, w2 = v
    bary = []
    wts = []
    for a, w in ((a1, w1), (a2, w2)):
        b = 1.0 - 2.0 * a
        bary += [(b, a, a), (a, b, a), (a, a, b)]
        wts += [w, w, w]
    return np.array(bary), np.array(wts)
