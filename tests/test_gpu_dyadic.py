"""Dyadic refinement of the local layer potentials on the GPU (Sec. 4.4):
the expansions at delta / 4^J plus the difference-kernel sums of J levels on
refined panels, against the oracle's refinement (plain direct sums of the
literal difference G_H[delta_j] - G_H[delta_{j-1}] over Lagrange-interpolated
subnodes) and against the closed forms on the unit circle."""
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


def _circle(delta=2e-3, n_targets=400, seed=3, mode=3):
    from workloads import configs
    return configs.circle_layer_problem(n_panels=64, order=16, n_targets=n_targets, delta=delta, mode=mode,
                                        radii=(0.9, 0.97, 0.99, 1.0, 1.01, 1.05), seed=seed, tol=1e-10)


def _exact(tgt, n):
    r = np.hypot(tgt[:, 0], tgt[:, 1])
    th = np.arctan2(tgt[:, 1], tgt[:, 0])
    on = np.abs(r - 1.0) < 1e-12
    S = np.where(r <= 1, r ** n, r ** (-n)) * np.cos(n * th) / (2 * n)
    D = np.where(on, 0.0, np.where(r < 1, -r ** n, r ** (-n)) * np.cos(n * th) / 2)
    return S, D


def _run(lp, p, precision, tol, order, levels):
    ev = lp.Evaluator(p, precision=precision, tol=tol, order=order, refine_levels=levels)
    ev.bind()
    out = ev.evaluate(want=("S", "D"))
    res = {k: out[k].cpu().numpy() for k in ("S", "D")}
    info = ev.info()
    ev.close()
    return res, info


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-10, 1e-9), ("fp32", 1e-5, 1e-5)])
@pytest.mark.parametrize("levels", [1, 3])
def test_refined_layers_match_oracle(lp, oracle_lib, precision, tol, bound, levels):
    p = _circle()
    ref = oracle_lib.evaluate(p, order=3, want=("S", "D"), refine_levels=levels)
    got, info = _run(lp, p, precision, tol, 3, levels)
    assert info["refine_levels"] == levels
    assert info["refine_subnodes"] == 64 * 16 * sum(2 ** j for j in range(1, levels + 1))
    # c4..c15 of each piece are stored in single precision: ~5e-12 of H <= 0.75
    assert info["refine_table_err"] < 1e-11
    for k in ("S", "D"):
        assert _rel_l2(got[k], ref[k]) < bound, (k, _rel_l2(got[k], ref[k]))
        scale = np.max(np.abs(ref[k]))
        assert np.max(np.abs(got[k] - ref[k])) < 5 * bound * scale, k


def test_refinement_reduces_error_against_closed_forms(lp):
    """Order 3 at delta = 4e-3: each level divides the expansion error by
    about 4^{3/2} = 8; three levels reach the closed forms ~500x closer."""
    p = _circle(delta=4e-3, n_targets=300, seed=11)
    Se, De = _exact(p["tgt_xy"], 3)
    errs = []
    for J in (0, 3):
        got, _ = _run(lp, p, "fp64", 1e-12, 3, J)
        errs.append((np.max(np.abs(got["S"] - Se)), np.max(np.abs(got["D"] - De))))
    for c in range(2):
        assert errs[0][c] / errs[1][c] > 200, (c, errs)


def test_levels_match_unrefined_at_smaller_delta(lp):
    """J levels at delta reach the closed forms as closely as no refinement
    at delta / 4^J: the expansion error is that of delta / 4^J."""
    delta, J = 4e-3, 2
    p = _circle(delta=delta, n_targets=300, seed=21)
    Se, De = _exact(p["tgt_xy"], 3)
    refined, _ = _run(lp, p, "fp64", 1e-12, 3, J)
    q = dict(p)
    q["delta"] = delta / 4 ** J
    plain, _ = _run(lp, q, "fp64", 1e-12, 3, 0)
    for k, ex in (("S", Se), ("D", De)):
        e1 = np.max(np.abs(refined[k] - ex))
        e0 = np.max(np.abs(plain[k] - ex))
        assert abs(e1 - e0) < 0.05 * e0, (k, e1, e0)


def test_volume_unchanged_and_layers_refined_on_starfish(lp, oracle_lib):
    from workloads import configs
    p = configs.starfish(seed=2002, n_interior=2600, n_boundary_vertices=200, n_panels=128)
    idx = np.random.default_rng(1).choice(len(p["tgt_xy"]), 600, replace=False)
    txy, jet = p["tgt_xy"][idx], p["tgt_jet"][idx]
    outs = {}
    for J in (0, 2):
        ev = lp.Evaluator(p, precision="fp64", refine_levels=J).bind()
        o = ev.evaluate(tgt_xy=txy, tgt_jet=jet)
        outs[J] = {k: o[k].cpu().numpy() for k in "VSD"}
        ev.close()
    # V takes no refinement: the same arithmetic (atomics may reorder sums)
    assert np.max(np.abs(outs[2]["V"] - outs[0]["V"])) <= 1e-12 * np.max(np.abs(outs[0]["V"]))
    ref = oracle_lib.evaluate(p, targets=idx, want=("S", "D"), refine_levels=2)
    for k in ("S", "D"):
        assert _rel_l2(outs[2][k], ref[k]) < 1e-9, k


def test_refined_plan_rejected_by_batch_and_served_by_noalloc(lp):
    p = _circle(n_targets=100)
    ev = lp.Evaluator(p, precision="fp64", refine_levels=2).bind()
    ref = {k: v.cpu().numpy() for k, v in ev.evaluate(want=("S", "D")).items()}
    txy, _ = ev._tgt
    n = len(p["tgt_xy"])
    L = lp.library()
    outs = [torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    rc = L.lp_execute_noalloc(ev.plan, n, txy.data_ptr(), None, None, outs[0].data_ptr(), outs[1].data_ptr())
    assert rc == 0 and L.lp_sync(ev.plan) == 0
    for k, o in zip("SD", outs):
        assert _rel_l2(o.cpu().numpy(), ref[k]) < 1e-13, k
    b = lp.lp_batch_create(0)
    t = torch.as_tensor(p["tgt_xy"], device="cuda")
    j = torch.zeros((n, 6), dtype=torch.float64, device="cuda")
    o = [torch.empty(n, dtype=torch.float64, device="cuda")]
    with pytest.raises(lp.LpError):
        lp.lp_batch_execute(b, [ev.plan], [n], [t], [j], [None], o, [None])
    lp.lp_batch_destroy(b)
    ev.close()


@pytest.mark.parametrize("order,tol,delta,want", [(3, 1e-8, 4e-3, 5), (5, 1e-9, 8e-6, 0), (3, 1e-9, 8e-6, 2),
                                                  (3, 1e-12, 4e-3, 6)])
def test_automatic_levels(lp, order, tol, delta, want):
    """refine_levels="auto": the smallest J with (delta/4^J)^(order/2) <= tol,
    at most 6 (the selection rule of Sec. 4.4)."""
    p = _circle(delta=delta, n_targets=10)
    ev = lp.Evaluator(p, precision="fp64", tol=tol, order=order, refine_levels="auto")
    assert ev.info()["refine_levels"] == want
    J = 0
    while J < 6 and (delta / 4 ** J) ** (order / 2) > tol:
        J += 1
    assert J == want
    ev.close()
