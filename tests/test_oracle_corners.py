"""Pin of the oracle's local volume part at the corners of a polygonal
boundary (the configuration of the 12M-node square).

The paper's expansions (Sec. 4, eq. vplocO5) assume a smooth boundary.  The
readings used at corners: a target within 12 sqrt(delta) of only one edge
takes the perpendicular foot on that edge, with kappa = 0 and no higher
derivatives of the curve, i.e. the local integral over the half-plane of
that edge; a target within 12 sqrt(delta) of both edges of a convex
right-angle corner takes the exact local integral over the quadrant (order
5).  For a straight edge and a quadratic f the printed expansion with every
term is that half-plane integral exactly, so the oracle must reproduce it to
rounding:

  V_half(eta) = int_0^delta [(f + t f_xixi) M0 + f_eta M1 + f_etaeta M2 / 2] dt,

with the 1D heat kernel g_t(s) = exp(-s^2/4t)/sqrt(4 pi t), eta the distance to
the edge and M_k = int_{-eta}^inf s^k g_t(s) ds:
M0 = 1 - erfc(eta/(2 sqrt t))/2, M1 = sqrt(t/pi) exp(-eta^2/4t),
M2 = 2t M0 - 2t eta g_t(eta).  Here the tangential moments of the Gaussian are
0 and 2t, and the two directions separate.

For a right-angle corner the exact local integral runs over the quadrant and
separates into the moments of both edges; the oracle must match it (here by
scipy's adaptive quadrature in t) to rounding.  The test also measures what
the nearest-edge reading alone would miss there: for constant f,
f int_0^delta M0(a) (1 - M0(b)) dt, at most delta f / 4, at the corner.
"""
import math

import numpy as np
from scipy import integrate, special

from workloads.panels import make_square_panels

DELTA = 1e-3


def _moments(eta, t):
    g = math.exp(-eta * eta / (4 * t)) / math.sqrt(4 * math.pi * t)
    m0 = 1.0 - 0.5 * special.erfc(eta / (2 * math.sqrt(t)))
    m1 = math.sqrt(t / math.pi) * math.exp(-eta * eta / (4 * t))
    m2 = 2 * t * m0 - 2 * t * eta * g
    return m0, m1, m2


def _half_plane(jet, eta, N, T, delta=DELTA):
    f, grad, H = jet[0], jet[1:3], np.array([[jet[3], jet[4]], [jet[4], jet[5]]])
    f_eta, f_ee, f_xx = grad @ N, N @ H @ N, T @ H @ T

    def integrand(t):
        if t <= 0.0:
            return 0.0
        m0, m1, m2 = _moments(eta, t)
        return (f + t * f_xx) * m0 + f_eta * m1 + 0.5 * f_ee * m2

    v, _ = integrate.quad(integrand, 0.0, delta, epsabs=1e-18, epsrel=1e-13, limit=200)
    return v


def _quadrant(jet, a, b, N1, N2, delta=DELTA):
    """Exact local integral over the quadrant bounded by two perpendicular
    edges at distances a (inward normal N1) and b (inward normal N2)."""
    f, grad, H = jet[0], jet[1:3], np.array([[jet[3], jet[4]], [jet[4], jet[5]]])
    fu, fv = grad @ N1, grad @ N2
    fuu, fvv, fuv = N1 @ H @ N1, N2 @ H @ N2, N1 @ H @ N2

    def integrand(t):
        if t <= 0.0:
            return 0.0
        A0, A1, A2 = _moments(a, t)
        B0, B1, B2 = _moments(b, t)
        return (f * A0 * B0 + fu * A1 * B0 + fv * A0 * B1 + 0.5 * fuu * A2 * B0 + fuv * A1 * B1
                + 0.5 * fvv * A0 * B2)

    v, _ = integrate.quad(integrand, 0.0, delta, epsabs=1e-18, epsrel=1e-13, limit=200)
    return v


def _targets():
    """Points near the corner (1, 1) of [-1, 1]^2 at distances (a, b) from the
    edges x = 1 and y = 1, plus mirrored copies near the other corners."""
    ab = [(0.02, 0.05), (0.05, 0.02), (0.1, 0.3), (0.3, 0.1), (0.004, 0.011), (0.2, 0.21), (0.06, 0.5),
          (0.03, 0.45), (0.45, 0.01), (0.2, 0.6), (0.0, 0.1), (0.1, 0.0), (0.0, 0.0)]
    pts, dist = [], []
    for sx, sy in [(1, 1), (-1, 1), (-1, -1), (1, -1)]:
        for a, b in ab:
            pts.append([sx * (1 - a), sy * (1 - b)])
            dist.append((a, b, sx, sy))
    return np.array(pts), dist


def test_nearest_edge_reading_is_the_half_plane_integral(oracle_lib):
    bnd = make_square_panels(1.0, 8, 16)
    txy, dist = _targets()
    rng = np.random.default_rng(12)
    jet = np.column_stack([rng.uniform(0.5, 2.0, len(txy)), rng.uniform(-1, 1, (len(txy), 5))])
    VL, _, _, info, st = oracle_lib.local(bnd, None, None, txy, jet, DELTA, order=5, on_tol=1e-12)
    assert st == 0
    band = 12 * math.sqrt(DELTA)
    checked = 0
    for i, (a, b, sx, sy) in enumerate(dist):
        if max(a, b) < band:
            continue  # both edges in the band: the quadrant reading (next test)
        checked += 1
        if a <= b:  # nearest edge x = sx: inward normal (-sx, 0), tangent along y
            eta, N, T = a, np.array([-sx, 0.0]), np.array([0.0, 1.0])
        else:       # nearest edge y = sy
            eta, N, T = b, np.array([0.0, -sy]), np.array([1.0, 0.0])
        ref = _half_plane(jet[i], eta, N, T)
        assert abs(VL[i] - ref) <= 1e-12 * DELTA * np.max(np.abs(jet[i])), (i, VL[i], ref)
    assert checked == 16


def test_quadrant_reading_at_right_angle_corners(oracle_lib):
    """Targets within 12 sqrt(delta) of both edges of a corner of the square
    (including the corner and points on either edge): the oracle's V_L is the
    exact quadrant integral of the target's quadratic f."""
    bnd = make_square_panels(1.0, 8, 16)
    txy, dist = _targets()
    rng = np.random.default_rng(13)
    jet = np.column_stack([rng.uniform(0.5, 2.0, len(txy)), rng.uniform(-1, 1, (len(txy), 5))])
    VL = oracle_lib.local(bnd, None, None, txy, jet, DELTA, order=5, on_tol=1e-12)[0]
    band = 12 * math.sqrt(DELTA)
    checked = 0
    for i, (a, b, sx, sy) in enumerate(dist):
        if max(a, b) >= band:
            continue
        checked += 1
        # inward normals of the edges x = sx and y = sy
        ref = _quadrant(jet[i], a, b, np.array([-sx, 0.0]), np.array([0.0, -sy]))
        assert abs(VL[i] - ref) <= 1e-13 * np.max(np.abs(jet[i])), (i, a, b, VL[i], ref)
    assert checked == 36


def test_corner_gap_of_the_reading(oracle_lib):
    """The reading's error against the exact quadrant integral: at most
    delta f / 4 for constant f (at the corner), and nothing once the farther
    edge is outside the band."""
    jet = np.array([1.3, 0, 0, 0, 0, 0])
    N1, N2 = np.array([-1.0, 0.0]), np.array([0.0, -1.0])
    T1 = np.array([0.0, 1.0])
    band = 12 * math.sqrt(DELTA)
    gaps = []
    for a, b in [(1e-9, 1e-9), (0.01, 0.01), (0.01, 0.05), (0.05, 0.2), (0.1, band + 1e-3)]:
        gaps.append(_half_plane(jet, a, N1, T1) - _quadrant(jet, a, b, N1, N2))
    gaps = np.array(gaps) / (DELTA * jet[0])
    assert abs(gaps[0] - 0.25) < 1e-6          # at the corner: half of the half-plane's delta f / 2
    assert np.all(np.diff(gaps) < 0) and np.all(gaps[:-1] > 0)
    assert abs(gaps[-1]) < 1e-12               # second edge beyond 12 sqrt(delta): no gap
    # the oracle takes the quadrant there, closing the gap
    bnd = make_square_panels(1.0, 8, 16)
    x = np.array([[1 - 0.01, 1 - 0.01]])
    VL = oracle_lib.local(bnd, None, None, x, jet[None, :], DELTA, order=5, on_tol=1e-12)[0][0]
    assert abs(VL - _quadrant(jet, 0.01, 0.01, N1, N2)) < 1e-13 * jet[0]
    # order 4 keeps the nearest-edge reading (no quadrant form is truncated)
    VL4 = oracle_lib.local(bnd, None, None, x, jet[None, :], DELTA, order=4, on_tol=1e-12)[0][0]
    assert abs(VL4 - _half_plane(jet, 0.01, N1, T1)) < 1e-12 * DELTA
