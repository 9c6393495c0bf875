"""Pins of the oracle's dyadic refinement of the local layer potentials
(Sec. 4.4): S_L[delta] = S_L[delta / 4^J] + sum_j of direct sums of the
difference kernels G_H[delta_j] - G_H[delta_{j-1}] (and their normal
derivatives for D) on refined panels.

* Against the closed forms on the unit circle (S[cos nt] = r^n cos(nt)/(2n),
  D[cos nt] = -r^n cos(nt)/2 inside, 0 on the curve): each refinement level
  divides delta by 4 in the expansion, so the error falls by 4^{p/2} per
  level for expansion order p (8 at p = 3, 32 at p = 5), and J levels at
  delta reproduce zero levels at delta / 4^J.
* The difference sums against an independent quadrature: S_H[delta_J] -
  S_H[delta] (and D) summed over a fine panel discretisation with the
  generator's own weights.
"""
import numpy as np
import pytest

from workloads import configs


def _exact(tgt, n):
    r = np.hypot(tgt[:, 0], tgt[:, 1])
    th = np.arctan2(tgt[:, 1], tgt[:, 0])
    on = np.abs(r - 1.0) < 1e-12
    S = np.where(r <= 1, r ** n, r ** (-n)) * np.cos(n * th) / (2 * n)
    D = np.where(on, 0.0, np.where(r < 1, -r ** n, r ** (-n)) * np.cos(n * th) / 2)
    return S, D


def _errors(oracle_lib, delta, order, levels, n=3):
    p = configs.circle_layer_problem(n_panels=64, order=16, n_targets=60, delta=delta, mode=n,
                                     radii=(0.9, 0.97, 0.99, 1.0, 1.01, 1.05), seed=3)
    b, t = p["bnd"], p["tgt_xy"]
    SH = oracle_lib.smooth_charge(b["xy"], p["sigma"] * b["w"], t, delta)
    DH = oracle_lib.smooth_dipole(b["xy"], b["normal"], p["mu"] * b["w"], t, delta)
    Se, De = _exact(t, n)
    out = []
    for J in levels:
        SL, DL = oracle_lib.local_dyadic(b, p["sigma"], p["mu"], t, delta, J, order=order)
        out.append((np.max(np.abs(SH + SL - Se)), np.max(np.abs(DH + DL - De))))
    return np.array(out)


@pytest.mark.parametrize("order,rate", [(3, 8.0), (5, 32.0)])
def test_refinement_rate_against_closed_forms(oracle_lib, order, rate):
    e = _errors(oracle_lib, 4e-3, order, [0, 1, 2, 3])
    for k in range(3):
        for c in range(2):
            ratio = e[k, c] / e[k + 1, c]
            assert 0.8 * rate < ratio < 1.25 * rate, (order, k, c, ratio)


def test_levels_equal_smaller_delta(oracle_lib):
    """J levels at delta give the unrefined result at delta / 4^J (the error
    against the closed form is that of the expansion at delta / 4^J)."""
    refined = _errors(oracle_lib, 4e-3, 3, [2])[0]
    plain = _errors(oracle_lib, 4e-3 / 16, 3, [0])[0]
    assert np.allclose(refined, plain, rtol=1e-2)


def test_difference_sums_match_smooth_parts(oracle_lib):
    """sum_j (difference kernel sums) = S_H[delta_J] - S_H[delta], with the
    right-hand side from the smooth-part sums over a finer discretisation
    (1024 panels, the generator's weights) -- an independent quadrature of
    the same integrals."""
    delta, J, n = 1e-3, 3, 4
    coarse = configs.circle_layer_problem(n_panels=64, order=16, n_targets=40, delta=delta, mode=n,
                                          radii=(0.9, 0.97, 0.99, 1.0, 1.02), seed=5)
    fine = configs.circle_layer_problem(n_panels=1024, order=16, n_targets=40, delta=delta, mode=n,
                                        radii=(0.9, 0.97, 0.99, 1.0, 1.02), seed=5)
    t = coarse["tgt_xy"]
    assert np.array_equal(t, fine["tgt_xy"])
    bc, bf = coarse["bnd"], fine["bnd"]
    SL0, DL0 = oracle_lib.local_dyadic(bc, coarse["sigma"], coarse["mu"], t, delta / 4 ** J, 0, order=5)
    SLJ, DLJ = oracle_lib.local_dyadic(bc, coarse["sigma"], coarse["mu"], t, delta, J, order=5)
    sums_S, sums_D = SLJ - SL0, DLJ - DL0
    dS = (oracle_lib.smooth_charge(bf["xy"], fine["sigma"] * bf["w"], t, delta / 4 ** J)
          - oracle_lib.smooth_charge(bf["xy"], fine["sigma"] * bf["w"], t, delta))
    dD = (oracle_lib.smooth_dipole(bf["xy"], bf["normal"], fine["mu"] * bf["w"], t, delta / 4 ** J)
          - oracle_lib.smooth_dipole(bf["xy"], bf["normal"], fine["mu"] * bf["w"], t, delta))
    assert np.max(np.abs(sums_S - dS)) < 1e-10
    assert np.max(np.abs(sums_D - dD)) < 1e-9


def test_zero_levels_is_plain_local(oracle_lib):
    p = configs.circle_layer_problem(n_panels=64, order=16, n_targets=30, delta=2e-3, mode=2, seed=9)
    b, t = p["bnd"], p["tgt_xy"]
    SL, DL = oracle_lib.local_dyadic(b, p["sigma"], p["mu"], t, 2e-3, 0, order=4)
    _, SL2, DL2, _, _ = oracle_lib.local(b, p["sigma"], p["mu"], t, None, 2e-3, order=4)
    assert np.array_equal(SL, SL2) and np.array_equal(DL, DL2)
