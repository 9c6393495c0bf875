"""Pins of the oracle's smooth kernel against mathematics and library routines.

* E1 against scipy.special.exp1 (an independent implementation).
* G_H[delta] = G - G_L (eq. splitting2) where G_L is the time integral of
  the heat kernel over [0, delta] (eq. eiformula), computed here by adaptive
  quadrature of the heat kernel itself.
* G_H(0) = (gamma - ln(4 delta)) / (4 pi) (limit of eq. splitting2).
* The dipole kernel equals the finite-difference normal derivative of the
  charge kernel with respect to the source point (eq. dlpot convention).
* The Fourier representation of the history part (Lemmas of Sec. 2:
  eq. vnearkspace with eq. Wdef) inverts to G_H[delta_1]: this pins the
  multiplier formulas the CUDA path uses against the oracle's real-space
  kernel.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special


@pytest.mark.parametrize("z", [1e-12, 1e-6, 0.01, 0.3, 0.999, 1.0, 1.001, 2.5, 7.0, 30.0, 120.0])
def test_e1_matches_scipy(oracle_lib, z):
    ref = special.exp1(z)
    assert abs(oracle_lib.e1(z) / ref - 1.0) < 1e-14


def test_ein_entire_part(oracle_lib):
    for z in [1e-3, 0.2, 0.7, 1.0]:
        ein = oracle_lib.ein(z)
        ref = special.exp1(z) + np.euler_gamma + math.log(z)
        assert abs(ein - ref) < 5e-16 * max(1.0, abs(ref))


def _heat_time_integral(r, delta):
    """G_L via eq. eiformula's left-hand side: int_0^delta exp(-r^2/4t)/(4 pi t) dt."""
    f = lambda t: math.exp(-r * r / (4 * t)) / (4 * math.pi * t) if t > 0 else 0.0
    val, err = integrate.quad(f, 0.0, delta, epsabs=1e-15, epsrel=1e-13, limit=200)
    return val


@pytest.mark.parametrize("delta", [1e-4, 3e-3])
@pytest.mark.parametrize("c", [0.05, 0.5, 1.0, 2.0, 4.0, 9.0])
def test_green_smooth_is_green_minus_heat_integral(oracle_lib, delta, c):
    r = c * math.sqrt(delta)
    G = -math.log(r) / (2 * math.pi)
    GL = _heat_time_integral(r, delta)
    GH = oracle_lib.green_smooth(r, delta)[0]
    assert abs(GH - (G - GL)) < 1e-13 * max(1.0, abs(G))


@pytest.mark.parametrize("delta", [1e-6, 1e-3, 0.5])
def test_green_smooth_limit_at_zero(oracle_lib, delta):
    lim = (np.euler_gamma - math.log(4 * delta)) / (4 * math.pi)
    assert abs(oracle_lib.green_smooth(0.0, delta)[0] - lim) < 1e-15 * abs(lim) + 1e-16
    # continuity into r > 0
    r = 1e-6 * math.sqrt(delta)
    assert abs(oracle_lib.green_smooth(r, delta)[0] - lim) < 1e-12


def test_green_smooth_continuous_across_branch(oracle_lib):
    delta = 2e-4
    dz = 1e-9
    rs = np.sqrt(4 * delta * np.array([1 - dz, 1 + dz]))
    v = oracle_lib.green_smooth(rs, delta)
    # dG_H/dz = -(1 - e^{-z}) / (4 pi z) at z = 1 (derivative of -Ein(z)/(4 pi))
    expected = (1 - math.exp(-1.0)) / (4 * math.pi) * 2 * dz
    assert abs((v[0] - v[1]) - expected) < 1e-14


def test_dipole_is_source_normal_derivative(oracle_lib):
    rng = np.random.default_rng(5)
    delta = 1e-3
    y = np.array([[0.1, -0.2]])
    nu = np.array([[0.6, 0.8]])
    tgt = y + rng.normal(scale=0.08, size=(12, 2))
    tgt = np.concatenate([tgt, y])  # includes r = 0
    h = 1e-5
    gp = oracle_lib.smooth_charge(y + h * nu, np.ones(1), tgt, delta)
    gm = oracle_lib.smooth_charge(y - h * nu, np.ones(1), tgt, delta)
    fd = (gp - gm) / (2 * h)
    dip = oracle_lib.smooth_dipole(y, nu, np.ones(1), tgt, delta)
    assert np.max(np.abs(fd - dip)) < 1e-7
    assert dip[-1] == 0.0
    # sign convention of eq. dlpot: derivative in the source point, so a
    # target on the inward side (x - y = -t nu) sees a negative kernel
    assert oracle_lib.smooth_dipole(y, nu, np.ones(1), y - 0.3 * nu, delta)[0] < 0


def _fourier_inverse_radial(M, r, kmax):
    """(1/(2 pi)^2) int_{R^2} M(|k|) e^{ik.x} dk = (1/2pi) int_0^inf M(k) J0(kr) k dk."""
    f = lambda k: M(k) * special.j0(k * r) * k
    val, _ = integrate.quad(f, 0.0, kmax, limit=4000, epsabs=1e-14, epsrel=1e-12)
    return val / (2 * math.pi)


def test_fourier_multipliers_invert_to_smooth_kernel(oracle_lib):
    d1 = 2e-3
    d2 = 32 * d1
    D = 2.0                                  # box side
    R = math.sqrt(4 * d2 * math.log(1e14))   # Gaussian reach of the far kernel
    L = math.sqrt(2) * D + R                 # truncation radius of eq. Wdef (generalised)

    def W(k):
        if k < 1e-6:
            return L * L * (1 - 2 * math.log(L)) / 4 + k * k * 0.0
        return (1 - special.j0(L * k)) / (k * k) - L * math.log(L) * special.j1(L * k) / k

    MNH = lambda k: (math.expm1(-k * k * d1) - math.expm1(-k * k * d2)) / (k * k) if k > 1e-8 else d2 - d1
    MFH = lambda k: math.exp(-k * k * d2) * W(k)
    kmax_nh = math.sqrt(40 / d1)
    kmax_fh = math.sqrt(40 / d2)
    for r in [0.0, 0.01, 0.07, 0.3, 1.0, math.sqrt(2) * D * 0.99]:
        u = _fourier_inverse_radial(MNH, r, kmax_nh) + _fourier_inverse_radial(MFH, r, kmax_fh)
        ref = oracle_lib.green_smooth(r, d1)[0]
        assert abs(u - ref) < 1e-9, (r, u, ref)


def test_far_multiplier_limit():
    """W(k) -> L^2 (1 - 2 ln L)/4 as k -> 0 (Lemma after eq. Wdef), L = 2 sqrt 2."""
    L = 2 * math.sqrt(2)
    k = 1e-4
    W = (1 - special.j0(L * k)) / (k * k) - L * math.log(L) * special.j1(L * k) / k
    lim = L * L * (1 - 2 * math.log(L)) / 4
    assert abs(W - lim) < 1e-6
    assert abs(lim - (-2.158883)) < 1e-6


def test_single_level_multiplier_inverts_to_smooth_kernel(oracle_lib):
    """The one-level alternative of Sec. 3 (delta_2 = delta_1, so the near
    history vanishes): e^{-k^2 delta_1} W(k), W the transform of the log
    kernel truncated at L = sqrt 2 D + R with R = sqrt(4 delta_1 ln(1/eps)),
    inverts to G_H[delta_1] at every separation inside the box."""
    d1 = 2e-3
    D = 2.0
    R = math.sqrt(4 * d1 * math.log(1e14))
    L = math.sqrt(2) * D + R

    def W(k):
        if k < 1e-6:
            return L * L * (1 - 2 * math.log(L)) / 4
        return (1 - special.j0(L * k)) / (k * k) - L * math.log(L) * special.j1(L * k) / k

    M = lambda k: math.exp(-k * k * d1) * W(k)
    kmax = math.sqrt(40 / d1)
    for r in [0.0, 0.02, 0.2, 1.0, math.sqrt(2) * D * 0.99]:
        u = _fourier_inverse_radial(M, r, kmax)
        ref = oracle_lib.green_smooth(r, d1)[0]
        assert abs(u - ref) < 1e-9, (r, u, ref)
