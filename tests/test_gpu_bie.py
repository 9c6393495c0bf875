"""Interior Dirichlet solve on the GPU (Sec. 5, eq. dir_inteq): GMRES with D
applied by the evaluator at the boundary nodes, against the oracle's dense
direct solve of the same discrete equation, and against closed forms."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lp():
    from paper_2409_11998_gb300 import build
    build.build()
    import paper_2409_11998_gb300 as lp
    return lp


def _layer_problem(curve, n_panels, delta, tol=1e-11):
    """Boundary-only problem on `curve` (no volume sources) in the dict
    layout of the workload generators."""
    from workloads.panels import make_panels
    bnd = make_panels(curve, n_panels, 16)
    lo, hi = bnd["xy"].min(0) - 0.1, bnd["xy"].max(0) + 0.1
    return {"bnd": bnd, "delta": delta, "tol": tol, "precision": "fp64", "box_lo": lo.tolist(),
            "box_hi": hi.tolist(), "src_xy": np.zeros((0, 2)), "src_w": np.zeros(0), "src_f": np.zeros(0)}


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("levels", [0, 3])
def test_circle_matches_oracle_and_closed_form(lp, oracle_lib, levels):
    from workloads.curves import Circle
    p = _layer_problem(Circle(1.0), 32, 1e-3)
    b = p["bnd"]
    g = np.cos(3 * b["t"])
    ev = lp.Evaluator(p, precision="fp64", refine_levels=levels).bind()
    mu, it, res = ev.solve_dirichlet(g, tol=1e-12)
    mu = mu.cpu().numpy()
    assert res < 1e-11 and 0 < it < 30, (it, res)
    ref = oracle_lib.solve_dirichlet(b, g, 1e-3, order=5, refine_levels=levels)
    assert _rel(mu, ref) < 1e-9, _rel(mu, ref)
    # mu = -2 g exactly for the continuous problem; the discrete error is
    # that of the expansions (refinement: 32x per level at order 5)
    err = np.max(np.abs(mu + 2 * g))
    assert err < (5e-6 if levels == 0 else 1e-9), err
    ev.close()


def test_ellipse_harmonic_interior_solution(lp, oracle_lib):
    from workloads.curves import Ellipse
    p = _layer_problem(Ellipse(1.0, 0.6), 48, 5e-4)
    b = p["bnd"]
    g = np.exp(b["xy"][:, 0]) * np.cos(b["xy"][:, 1])
    ev = lp.Evaluator(p, precision="fp64").bind()
    mu, it, res = ev.solve_dirichlet(g, tol=1e-12)
    assert res < 1e-11
    ref = oracle_lib.solve_dirichlet(b, g, 5e-4, order=5)
    assert _rel(mu.cpu().numpy(), ref) < 1e-9
    rng = np.random.default_rng(3)
    s, th = np.sqrt(rng.uniform(0.0, 0.85, 300)), rng.uniform(0, 2 * np.pi, 300)
    tgt = np.stack([s * np.cos(th), 0.6 * s * np.sin(th)], 1)
    u = ev.evaluate(tgt_xy=tgt, tgt_jet=np.zeros((300, 6)), want=("D",))["D"].cpu().numpy()
    assert np.max(np.abs(u - np.exp(tgt[:, 0]) * np.cos(tgt[:, 1]))) < 1e-5
    ev.close()


def test_poisson_on_the_disk(lp, oracle_lib):
    """u = x^2 + y^2 on the unit disk: f = -lap u = -4, g = 1; u = V[f] +
    D[mu] with mu from the solve (V[f] at the boundary nodes from the
    f-jet there)."""
    from workloads import configs
    p = dict(configs.disk())
    p["src_f"] = np.full(len(p["src_w"]), -4.0)
    b = p["bnd"]
    nb = len(b["w"])
    jet_b = np.zeros((nb, 6))
    jet_b[:, 0] = -4.0
    g = np.ones(nb)
    ev = lp.Evaluator(p, precision="fp64").bind()
    mu, it, res = ev.solve_dirichlet(g, f_jet_b=jet_b, tol=1e-12)
    assert res < 1e-11
    # the oracle: V[f] at the boundary nodes, then the dense solve
    q = dict(p)
    q["tgt_xy"], q["tgt_jet"] = b["xy"], jet_b
    vb = oracle_lib.evaluate(q, want=("V",))["V"]
    ref = oracle_lib.solve_dirichlet(b, g, p["delta"], order=5, on_tol=oracle_lib.on_tolerance(p), v_boundary=vb)
    assert _rel(mu.cpu().numpy(), ref) < 1e-9
    # interior: u = V[f] + D[mu] against x^2 + y^2
    P = p["tgt_xy"]
    inside = np.hypot(P[:, 0], P[:, 1]) < 0.9
    tgt = P[inside]
    jet = np.zeros((len(tgt), 6))
    jet[:, 0] = -4.0
    out = ev.evaluate(tgt_xy=tgt, tgt_jet=jet, want=("V", "D"))
    u = out["V"].cpu().numpy() + out["D"].cpu().numpy()
    assert np.max(np.abs(u - (tgt[:, 0] ** 2 + tgt[:, 1] ** 2))) < 5e-5  # volume discretisation: 1.5e-5
    ev.close()


def test_fp32_plan_and_host_buffers(lp):
    from workloads.curves import Circle
    p = _layer_problem(Circle(1.0), 32, 1e-3, tol=1e-5)
    g = np.cos(3 * p["bnd"]["t"])
    ev = lp.Evaluator(p, precision="fp32", tol=1e-5).bind()
    mu, it, res = ev.solve_dirichlet(g, tol=1e-5)
    assert res < 1e-5 and np.max(np.abs(mu.cpu().numpy() + 2 * g)) < 1e-4
    ev.close()
    ev = lp.Evaluator(p, precision="fp64", host=True).bind()
    mu, it, res = ev.solve_dirichlet(g, tol=1e-12)
    assert isinstance(mu, np.ndarray) and res < 1e-11 and np.max(np.abs(mu + 2 * g)) < 5e-6
    ev.close()


@pytest.mark.parametrize("levels", [0, 3])
def test_neumann_circle_matches_oracle_and_closed_form(lp, oracle_lib, levels):
    from workloads.curves import Circle
    p = _layer_problem(Circle(1.0), 32, 1e-3)
    t = p["bnd"]["t"]
    g = 3 * np.cos(3 * t)
    ev = lp.Evaluator(p, precision="fp64", refine_levels=levels).bind()
    u, it, res = ev.solve_neumann(g, tol=1e-12)
    u = u.cpu().numpy()
    assert res < 1e-11 and 0 < it < 40, (it, res)
    ref = oracle_lib.solve_neumann(p["bnd"], g, 1e-3, order=5, refine_levels=levels)
    assert _rel(u, ref) < 1e-9, _rel(u, ref)
    assert np.max(np.abs(u - np.cos(3 * t))) < (5e-6 if levels == 0 else 1e-9)
    ev.close()


def test_neumann_poisson_interior(lp, oracle_lib):
    """u = exp(x) cos(y) + (x^2 + y^2) on the unit disk: f = -lap u = -4,
    g = du/dr; u = V[f] + S[g] - D[u] inside, up to the constant fixed by
    the zero boundary mean."""
    from workloads import configs
    p = dict(configs.disk())
    p["src_f"] = np.full(len(p["src_w"]), -4.0)
    b = p["bnd"]
    nb = len(b["w"])
    x, y = b["xy"][:, 0], b["xy"][:, 1]
    ux = np.exp(x) * np.cos(y) + 2 * x
    uy = -np.exp(x) * np.sin(y) + 2 * y
    g = ux * b["normal"][:, 0] + uy * b["normal"][:, 1]
    jet_b = np.zeros((nb, 6))
    jet_b[:, 0] = -4.0
    # the smooth part at 1e-11: the Neumann operator (singular up to its
    # rank-one term) amplifies the evaluator's tolerance more than the
    # Dirichlet one, and the comparison is with the oracle's exact sums
    ev = lp.Evaluator(p, precision="fp64", tol=1e-11).bind()
    u, it, res = ev.solve_neumann(g, f_jet_b=jet_b, tol=1e-12)
    assert res < 1e-10
    q = dict(p)
    q["tgt_xy"], q["tgt_jet"] = b["xy"], jet_b
    vb = oracle_lib.evaluate(q, want=("V",))["V"]
    ref = oracle_lib.solve_neumann(b, g, p["delta"], order=5, on_tol=oracle_lib.on_tolerance(p), v_boundary=vb)
    assert _rel(u.cpu().numpy(), ref) < 1e-9
    exact_b = np.exp(x) * np.cos(y) + x ** 2 + y ** 2
    shift = np.sum(b["w"] * exact_b) / np.sum(b["w"])
    P = p["tgt_xy"]
    tgt = P[np.hypot(P[:, 0], P[:, 1]) < 0.9]
    jet = np.zeros((len(tgt), 6))
    jet[:, 0] = -4.0
    out = ev.evaluate(tgt_xy=tgt, tgt_jet=jet)
    u_in = out["V"].cpu().numpy() + out["S"].cpu().numpy() - out["D"].cpu().numpy()
    exact = np.exp(tgt[:, 0]) * np.cos(tgt[:, 1]) + tgt[:, 0] ** 2 + tgt[:, 1] ** 2 - shift
    assert np.max(np.abs(u_in - exact)) < 5e-5
    ev.close()
