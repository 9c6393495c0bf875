"""Pins of the oracle's asymptotic local part (Sec. 4) against brute-force
quadrature of the local heat integrals and against closed forms.

Rates: with all printed terms (p = 5) the absolute error is O(delta^{5/2}),
i.e. relative O(delta^2) for S_L (which is O(sqrt delta)), O(delta^{5/2}) for
D_L off the surface (O(1) there) and O(delta^{3/2}) for V_L (O(delta)).
Quartering delta must therefore cut the relative error by about 16, 32 and
8.  A sign slip in any leading term stalls the error at O(1) or
O(delta^{1/2}); a dropped higher term halves the rate.  Geometry enters
through exact tangent-frame derivatives computed by a Chebyshev fit.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from local_brute import (brute_double, brute_single, brute_volume, closest_param, ellipse_exit,
                         tangent_frame_jet)
from workloads.curves import Ellipse
from workloads.fields import GaussianSum, PolyField

DELTAS = (4e-3, 1e-3, 2.5e-4)
CURVE = Ellipse(1.0, 0.6)
SIG = lambda t: 1 + 0.5 * np.sin(2 * t) + 0.3 * np.cos(3 * t)
MU = lambda t: 0.7 + 0.4 * np.cos(t) - 0.3 * np.sin(3 * t)


def _geom(fr, r, sgn):
    s, m = fr["dens"]
    return dict(r=r, sgn=float(sgn), kappa=fr["kappa"], g3=fr["g3"], g4=fr["g4"],
                s0=s[0], s1=s[1], s2=s[2], m0=m[0], m1=m[1], m2=m[2], m4=m[4],
                Tx=fr["T"][0], Ty=fr["T"][1])


@pytest.mark.parametrize("tb,c,side", [(0.4, 1.5, -1), (1.3, 0.7, 1), (1.3, 2.5, 1), (0.4, 0.0, 0)])
def test_layer_local_rates_on_ellipse(oracle_lib, tb, c, side):
    fr = tangent_frame_jet(CURVE, tb, (SIG, MU))
    es, ed = [], []
    for delta in DELTAS:
        r = c * math.sqrt(delta)
        x = fr["b"] + side * fr["N"] * r if side != 0 else fr["b"].copy()
        asym = oracle_lib.local_formulas(_geom(fr, r, side), None, delta, order=5)
        bs = brute_single(CURVE, SIG, x, delta, tb)
        bd = brute_double(CURVE, MU, x, delta, tb)
        es.append(abs(asym["S"] - bs) / abs(bs))
        ed.append(abs(asym["D"] - bd) / abs(bd))
    es, ed = np.array(es), np.array(ed)
    # S: relative delta^2 (ratio 16); D: delta^{5/2} off-surface (32), delta^2 on it
    assert es[-1] < 5e-6 and np.all(es[1:] < es[:-1])
    assert es[-2] / es[-1] > 11.0
    want_d = 11.0 if side == 0 else 22.0
    assert ed[-2] / ed[-1] > want_d
    assert ed[-1] < 1e-5


@pytest.mark.parametrize("field,c", [("poly", 0.8), ("gauss", 2.0)])
def test_volume_local_rate_on_ellipse(oracle_lib, field, c):
    fld = {"poly": PolyField(1.0, 0.5, -0.3, 0.3, 0.2, 0.4),
           "gauss": GaussianSum([[0.5, 0.1]], [0.4], background=0.3)}[field]
    fr = tangent_frame_jet(CURVE, 0.4)
    ex = ellipse_exit(1.0, 0.6)
    errs = []
    for delta in DELTAS:
        r = c * math.sqrt(delta)
        x = fr["b"] + fr["N"] * r
        geom = dict(r=r, sgn=1.0, kappa=fr["kappa"], Tx=fr["T"][0], Ty=fr["T"][1])
        asym = oracle_lib.local_formulas(geom, fld.jet(x[None, :])[0], delta, order=5)["V"]
        bv = brute_volume(ex, fld.value, x, delta, n_phi=192)
        errs.append(abs(asym - bv) / abs(bv))
    errs = np.array(errs)
    assert errs[-1] < 5e-5
    assert errs[0] / errs[1] > 6.0 and errs[1] / errs[2] > 6.0  # delta^{3/2}: 8


def test_flat_boundary_closed_forms(oracle_lib):
    """Straight boundary, constant densities: S_L = sqrt(d) s (e^{-c^2/4}/sqrt(pi)
    - (c/2) erfc(c/2)), D_L = -sgn m/2 erfc(c/2), V_L = f int_0^d (1 + erf(r/(2 sqrt t)))/2 dt."""
    delta = 1e-3
    for c in [0.0, 0.3, 1.0, 2.2, 5.0]:
        r = c * math.sqrt(delta)
        for sgn in ([0.0] if c == 0 else [1.0, -1.0]):
            g = dict(r=r, sgn=sgn, s0=1.7, m0=-0.4, Tx=1.0, Ty=0.0)
            jet = np.array([2.5, 0, 0, 0, 0, 0])
            out = oracle_lib.local_formulas(g, jet, delta, order=5)
            S = math.sqrt(delta) * 1.7 * (math.exp(-c * c / 4) / math.sqrt(math.pi) - c / 2 * math.erfc(c / 2))
            assert abs(out["S"] - S) < 1e-15
            D = -sgn * (-0.4) / 2 * math.erfc(c / 2)
            assert abs(out["D"] - D) < 1e-15
            if sgn >= 0:
                V, _ = integrate.quad(lambda t: 0.5 * (1 + math.erf(r / (2 * math.sqrt(t)))) if t > 0 else 0.5 + 0.5 * (r > 0),
                                      0, delta, epsabs=1e-17, epsrel=1e-13)
                assert abs(out["V"] - 2.5 * V) < 1e-14


def test_on_surface_corollaries(oracle_lib):
    """c = 0, sgn = 0 reproduces the printed on-surface corollaries (S and D
    negated, see module docstring of the oracle; V as printed)."""
    d = 2e-3
    g = dict(r=0.0, sgn=0.0, kappa=1.3, g3=-0.7, g4=2.1, s0=0.9, s1=0.4, s2=-1.1,
             m0=1.2, m1=-0.6, m2=0.8, m4=3.0, Tx=0.6, Ty=0.8)
    T = np.array([0.6, 0.8])
    N = np.array([-0.8, 0.6])
    jet = np.array([1.1, 0.3, -0.5, 0.7, 0.2, -0.4])
    H = np.array([[0.7, 0.2], [0.2, -0.4]])
    feta = jet[1:3] @ N
    lap = 0.7 - 0.4
    out = oracle_lib.local_formulas(g, jet, d, order=5)
    sp = math.sqrt(math.pi)
    S = -(-math.sqrt(d) * 0.9 / sp - d ** 1.5 / (3 * sp) * (1.3 ** 2 * 0.9 / 4 + (-1.1)))
    D = -(math.sqrt(d) * 1.3 * 1.2 / (2 * sp) + d ** 1.5 * (-5 * 1.3 ** 3 * 1.2 / (8 * sp)
          + 1.3 * 0.8 / (2 * sp) + 2 * (-0.6) * (-0.7) / (3 * sp) + 1.2 * 2.1 / (4 * sp)))
    V = d / 2 * 1.1 + d ** 1.5 / (3 * sp) * (2 * feta - 1.3 * 1.1) + d * d / 4 * lap
    assert abs(out["S"] - S) < 1e-15
    assert abs(out["D"] - D) < 1e-15
    assert abs(out["V"] - V) < 1e-15
    del H, T


def test_double_layer_jump(oracle_lib):
    """D_L(b -/+ r nu) -> D_L(b) -/+ mu/2 as r -> 0 (remark after the on-surface
    corollary, read with eq. dlpjump)."""
    d = 1e-3
    base = dict(kappa=0.9, g3=0.3, g4=1.0, m0=1.5, m1=0.2, m2=-0.7, m4=0.4, Tx=1.0, Ty=0.0)
    on = oracle_lib.local_formulas({**base, "r": 0.0, "sgn": 0.0}, None, d)["D"]
    inside = oracle_lib.local_formulas({**base, "r": 1e-12, "sgn": 1.0}, None, d)["D"]
    outside = oracle_lib.local_formulas({**base, "r": 1e-12, "sgn": -1.0}, None, d)["D"]
    assert abs(inside - (on - 0.75)) < 1e-10
    assert abs(outside - (on + 0.75)) < 1e-10


def test_far_interior_volume_formula(oracle_lib):
    """Far from the boundary V_L = delta f + delta^2/2 (f_xx + f_yy)
    (Sec. 4, after eq. vplocO5).  For a quadratic f this is exact over the
    whole plane (the heat semigroup gives f + t lap f), so brute force over a
    disk far larger than the kernel must agree to quadrature accuracy."""
    d = 1e-3
    fld = PolyField(0.4, 0.3, -0.2, 1.5, 0.7, -0.6)
    x = np.array([0.1, -0.05])
    exit_far = lambda x, e: 10.0
    bv = brute_volume(exit_far, fld.value, x, d, n_phi=64)
    far = oracle_lib.local(None, None, None, x[None, :], fld.jet(x[None, :]), d, order=5)[0][0]
    assert abs(far - bv) / abs(bv) < 1e-10


def test_flat_boundary_polynomial_densities(oracle_lib):
    """Straight boundary, polynomial densities in the tangent coordinate xi
    (sigma of degree 3, mu of degree 4): the heat kernel separates, the
    tangential Gaussian moments are 1, 0, 2t, 0, 12t^2, and the local
    integrals (eq. sheatloc, eq. dheatloc) reduce to
      S_L = int_0^d g_t(r) (s0 + s2 t) dt,
      D_L = -sgn int_0^d r/(2t) g_t(r) (m0 + m2 t + m4 t^2/2) dt,
    g_t the 1D heat kernel.  The printed expansions, all terms kept, give
    these exactly (S's next term, s4 t^2/2, is O(delta^{5/2}))."""
    delta = 2e-3
    s0, s1, s2 = 1.3, -0.4, 0.9      # s1, m1 enter only with curvature terms
    m0, m1, m2, m4 = -0.6, 0.5, 1.1, 2.3
    for c in [0.0, 0.2, 0.9, 2.0, 4.5]:
        r = c * math.sqrt(delta)
        for sgn in ([0.0] if c == 0 else [1.0, -1.0]):
            g = dict(r=r, sgn=sgn, s0=s0, s1=s1, s2=s2, m0=m0, m1=m1, m2=m2, m4=m4, Tx=0.0, Ty=1.0)
            out = oracle_lib.local_formulas(g, None, delta, order=5)

            def gt(t):
                return math.exp(-r * r / (4 * t)) / math.sqrt(4 * math.pi * t)

            S, _ = integrate.quad(lambda t: gt(t) * (s0 + s2 * t) if t > 0 else 0.0, 0, delta,
                                  epsabs=1e-18, epsrel=1e-13, limit=200)
            assert abs(out["S"] - S) < 1e-13 * math.sqrt(delta), (c, sgn, out["S"], S)
            if c == 0:
                continue  # on the surface D is the principal value (pinned by the corollary test)
            D, _ = integrate.quad(lambda t: r / (2 * t) * gt(t) * (m0 + m2 * t + m4 * t * t / 2) if t > 0 else 0.0,
                                  0, delta, epsabs=1e-18, epsrel=1e-13, limit=200)
            assert abs(out["D"] - (-sgn * D)) < 1e-13, (c, sgn, out["D"], -sgn * D)
