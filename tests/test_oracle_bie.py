"""Pins of the oracle's interior Dirichlet solve (Sec. 5, eq. dir_inteq):
mu solves -mu/2 + D[mu] = g - V[f] at the boundary nodes, and
u = V[f] + D[mu] inside.

* Unit circle, g = cos 3t: the principal-value double layer of cos nt
  vanishes on the unit circle, so mu = -2 g exactly; the discrete solve
  reaches it to the expansion's accuracy, and three levels of dyadic
  refinement (Sec. 4.4) bring it at least 100x closer.
* Ellipse, g = e^x cos y (harmonic): u = D[mu] at interior points equals
  e^x cos y.
"""
import numpy as np

from workloads.curves import Circle, Ellipse
from workloads.panels import make_panels


def _inside_u(oracle_lib, bnd, mu, tgt, delta, order=5):
    DH = oracle_lib.smooth_dipole(bnd["xy"], bnd["normal"], mu * bnd["w"], tgt, delta)
    _, _, DL, _, _ = oracle_lib.local(bnd, None, mu, tgt, None, delta, order)
    return DH + DL


def test_circle_density_closed_form(oracle_lib):
    bnd = make_panels(Circle(1.0), 32, 16)
    g = np.cos(3 * bnd["t"])
    e = []
    for J in (0, 3):
        mu = oracle_lib.solve_dirichlet(bnd, g, 1e-3, order=5, refine_levels=J)
        e.append(np.max(np.abs(mu + 2 * g)))
    assert e[0] < 5e-6, e
    assert e[1] < e[0] / 100, e


def test_circle_interior_solution(oracle_lib):
    bnd = make_panels(Circle(1.0), 32, 16)
    g = np.cos(3 * bnd["t"])
    mu = oracle_lib.solve_dirichlet(bnd, g, 1e-3, order=5)
    rng = np.random.default_rng(2)
    r, th = np.sqrt(rng.uniform(0.0, 0.9, 200)), rng.uniform(0, 2 * np.pi, 200)
    tgt = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    u = _inside_u(oracle_lib, bnd, mu, tgt, 1e-3)
    assert np.max(np.abs(u - r ** 3 * np.cos(3 * th))) < 5e-6


def test_ellipse_harmonic_data(oracle_lib):
    bnd = make_panels(Ellipse(1.0, 0.6), 48, 16)
    x, y = bnd["xy"][:, 0], bnd["xy"][:, 1]
    g = np.exp(x) * np.cos(y)
    mu = oracle_lib.solve_dirichlet(bnd, g, 5e-4, order=5)
    rng = np.random.default_rng(3)
    s, th = np.sqrt(rng.uniform(0.0, 0.85, 200)), rng.uniform(0, 2 * np.pi, 200)
    tgt = np.stack([s * np.cos(th), 0.6 * s * np.sin(th)], 1)
    u = _inside_u(oracle_lib, bnd, mu, tgt, 5e-4)
    exact = np.exp(tgt[:, 0]) * np.cos(tgt[:, 1])
    assert np.max(np.abs(u - exact)) < 1e-5, np.max(np.abs(u - exact))


def test_neumann_circle_closed_form(oracle_lib):
    """u = r^3 cos 3t: g = du/dr = 3 cos 3t on the unit circle; the boundary
    values cos 3t have zero mean, so the solve returns them (S[cos nt] =
    cos(nt)/(2n) and the principal-value D[cos nt] = 0 on the circle)."""
    bnd = make_panels(Circle(1.0), 32, 16)
    t = bnd["t"]
    e = []
    for J in (0, 3):
        u = oracle_lib.solve_neumann(bnd, 3 * np.cos(3 * t), 1e-3, order=5, refine_levels=J)
        e.append(np.max(np.abs(u - np.cos(3 * t))))
    assert e[0] < 5e-6 and e[1] < e[0] / 100, e


def test_neumann_ellipse_harmonic(oracle_lib):
    """u = e^x cos y on an ellipse: g = grad u . nu; the solve gives u minus
    its boundary mean, and the interior representation u = S[g] - D[u]
    reproduces e^x cos y up to that constant."""
    bnd = make_panels(Ellipse(1.0, 0.6), 48, 16)
    x, y = bnd["xy"][:, 0], bnd["xy"][:, 1]
    ux, uy = np.exp(x) * np.cos(y), -np.exp(x) * np.sin(y)
    g = ux * bnd["normal"][:, 0] + uy * bnd["normal"][:, 1]
    u = oracle_lib.solve_neumann(bnd, g, 5e-4, order=5)
    exact = np.exp(x) * np.cos(y)
    shift = np.sum(bnd["w"] * exact) / np.sum(bnd["w"])
    assert np.max(np.abs(u - (exact - shift))) < 1e-5
    rng = np.random.default_rng(4)
    s, th = np.sqrt(rng.uniform(0.0, 0.85, 100)), rng.uniform(0, 2 * np.pi, 100)
    tgt = np.stack([s * np.cos(th), 0.6 * s * np.sin(th)], 1)
    SH = oracle_lib.smooth_charge(bnd["xy"], g * bnd["w"], tgt, 5e-4)
    _, SL, _, _, _ = oracle_lib.local(bnd, g, None, tgt, None, 5e-4, 5)
    inside = SH + SL - _inside_u(oracle_lib, bnd, u, tgt, 5e-4)
    ref = np.exp(tgt[:, 0]) * np.cos(tgt[:, 1]) - shift
    assert np.max(np.abs(inside - ref)) < 1e-5, np.max(np.abs(inside - ref))
