"""Pins of the oracle's boundary geometry: closest point (Sec. 2.2: nearest node
plus Newton), side classification (Sec. 4: sgn = 1, 0, -1 in Omega, on the
boundary, outside) and tangent-frame derivatives (eq. tanparams) against an
analytic ellipse."""
import math

import numpy as np

from local_brute import closest_param, tangent_frame_jet
from workloads.curves import Ellipse
from workloads.panels import make_panels

A, B = 1.0, 0.6


def _setup(n_panels=64, n=80, seed=3):
    curve = Ellipse(A, B)
    bnd = make_panels(curve, n_panels, 16)
    rng = np.random.default_rng(seed)
    t = rng.uniform(0, 2 * np.pi, n)
    s = rng.uniform(-0.08, 0.08, n)
    tgt = curve.point(t) + s[:, None] * curve.outward_normal(t)
    return curve, bnd, tgt, s


def test_closest_point_and_side(oracle_lib):
    curve, bnd, tgt, s = _setup()
    delta = 1e-4  # band 12 sqrt(delta) = 0.12 covers every target
    _, _, _, info, st = oracle_lib.local(bnd, None, np.ones(len(bnd["xy"])), tgt, None, delta)
    assert st == 0
    for i, x in enumerate(tgt):
        panel, t, r, sgn = info[i]
        assert panel >= 0
        fr = oracle_lib.frame(bnd, None, None, int(panel), t)
        tb = closest_param(curve, x)
        bx = curve.point(tb)[0]
        assert np.hypot(fr["bx"] - bx[0], fr["by"] - bx[1]) < 1e-11
        assert abs(r - np.hypot(*(x - bx))) < 1e-11
        assert sgn == (1.0 if s[i] < 0 else -1.0)


def test_on_surface_classification(oracle_lib):
    curve, bnd, _, _ = _setup()
    tgt = bnd["xy"][::7]
    _, _, _, info, _ = oracle_lib.local(bnd, None, np.ones(len(bnd["xy"])), tgt, None, 1e-4,
                                        on_tol=1e-12)
    assert np.all(info[:, 3] == 0.0)
    assert np.all(info[:, 2] < 1e-12)


def test_far_targets_skip_newton(oracle_lib):
    curve, bnd, _, _ = _setup()
    tgt = np.array([[0.0, 0.0], [0.2, -0.1], [3.0, 0.0]])
    _, _, _, info, _ = oracle_lib.local(bnd, None, np.ones(len(bnd["xy"])), tgt, None, 1e-4)
    assert np.all(info[:, 0] == -1)


def test_frame_derivatives_match_analytic(oracle_lib):
    curve, bnd, _, _ = _setup()
    sig = lambda t: 1 + 0.5 * np.sin(2 * t) + 0.3 * np.cos(3 * t)
    tn = bnd["t"]
    dens = sig(tn)
    for panel in [3, 17, 40]:
        for t in [-0.6, 0.1, 0.55]:
            fr = oracle_lib.frame(bnd, dens, dens, panel, t)
            tb = closest_param(curve, np.array([fr["bx"], fr["by"]]))
            ex = tangent_frame_jet(curve, tb, (sig,))
            kap = A * B / (A * A * math.sin(tb) ** 2 + B * B * math.cos(tb) ** 2) ** 1.5
            assert abs(fr["kappa"] - kap) < 1e-9
            assert abs(fr["kappa"] - ex["kappa"]) < 1e-8
            assert abs(fr["g3"] - ex["g3"]) < 1e-5 * max(1, abs(ex["g3"]))
            assert abs(fr["g4"] - ex["g4"]) < 1e-4 * max(1, abs(ex["g4"]))
            d = ex["dens"][0]
            assert abs(fr["s0"] - d[0]) < 1e-12
            assert abs(fr["s1"] - d[1]) < 1e-8
            assert abs(fr["s2"] - d[2]) < 1e-6
            assert abs(fr["m4"] - d[4]) < 1e-3 * max(1, abs(d[4]))
