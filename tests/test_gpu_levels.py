"""Single-level plans and other grid upsampling factors (Sec. 3): the smooth
part from one grid carrying the truncated-kernel representation of G_H[delta]
(delta_2 = delta_1), or from grids at upsampling 1.25 / 2, matches the oracle
within the plan tolerance, as the default two-level plan does."""
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


@pytest.fixture(scope="module")
def disk():
    from workloads import configs
    return configs.disk()


@pytest.fixture(scope="module")
def disk_ref(disk, oracle_lib):
    return oracle_lib.evaluate(disk)


def _check(out, ref, tol):
    for k in ("V", "S", "D"):
        got = out[k].cpu().numpy()
        l2 = np.linalg.norm(got - ref[k]) / np.linalg.norm(ref[k])
        mx = np.max(np.abs(got - ref[k])) / np.max(np.abs(ref[k]))
        assert l2 < tol and mx < 5 * tol, (k, l2, mx)


@pytest.mark.parametrize("precision,tol,levels,ups", [
    ("fp64", 1e-9, 1, 0.0), ("fp32", 1e-5, 1, 0.0),
    ("fp64", 1e-9, 2, 1.25), ("fp64", 1e-9, 2, 2.0), ("fp32", 1e-5, 2, 1.25),
    ("fp64", 1e-9, 1, 2.0)])
def test_variants_match_oracle(lp, disk, disk_ref, precision, tol, levels, ups):
    ev = lp.Evaluator(disk, precision=precision, tol=tol, levels=levels, upsampling=ups).bind()
    info = ev.info()
    assert info["levels"] == levels
    if levels == 1:
        assert info["g_nh"] == 0 and info["delta2"] == info["delta1"]
    if ups:
        assert info["sigma"] == ups and info["sigma_eff"] >= ups
    _check(ev.evaluate(), disk_ref, tol)
    ev.close()


def test_single_level_starfish_and_layers_on_surface(lp, oracle_lib):
    from workloads import configs
    p = configs.starfish(seed=2001, n_interior=2600, n_boundary_vertices=200, n_panels=256)
    idx = np.random.default_rng(4).choice(len(p["tgt_xy"]), 1200, replace=False)
    ref = oracle_lib.evaluate(p, targets=idx)
    ev = lp.Evaluator(p, precision="fp64", levels=1).bind()
    out = ev.evaluate(tgt_xy=p["tgt_xy"][idx], tgt_jet=p["tgt_jet"][idx])
    _check(out, ref, 1e-9)
    ev.close()
    q = configs.circle_layer_problem(n_panels=128, delta=1e-4, mode=4, n_targets=300, tol=1e-10)
    ref = oracle_lib.evaluate(q, want=("S", "D"))
    ev = lp.Evaluator(q, precision="fp64", levels=1).bind()
    out = ev.evaluate(want=("S", "D"))
    for k in ("S", "D"):
        got = out[k].cpu().numpy()
        assert np.linalg.norm(got - ref[k]) / np.linalg.norm(ref[k]) < 1e-10, k
    ev.close()


def test_batch_wave_with_single_level_plans(lp, oracle_lib):
    """A wave mixing single- and two-level plans returns what each plan
    returns alone."""
    from workloads import configs
    probs = [configs.star_batch_member(4100 + i, n) for i, n in enumerate((300, 1500, 700))]
    stream = torch.cuda.Stream()
    evs = [lp.Evaluator(p, precision="fp64", levels=lv, stream=stream.cuda_stream).bind()
           for p, lv in zip(probs, (1, 2, 1))]
    alone = [{k: v.cpu().numpy() for k, v in ev.evaluate().items()} for ev in evs]
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    outs = {k: [torch.full((len(p["tgt_xy"]),), float("nan"), dtype=torch.float64, device="cuda")
                for p in probs] for k in "VSD"}
    b = lp.lp_batch_create(stream.cuda_stream)
    lp.lp_batch_execute(b, [ev.plan for ev in evs], [len(p["tgt_xy"]) for p in probs],
                        [dev(p["tgt_xy"]) for p in probs], [dev(p["tgt_jet"]) for p in probs],
                        outs["V"], outs["S"], outs["D"])
    lp.lp_batch_sync(b)
    for i in range(len(probs)):
        for k in "VSD":
            got = outs[k][i].cpu().numpy()
            assert np.max(np.abs(got - alone[i][k])) <= 1e-12 * np.max(np.abs(alone[i][k])), (i, k)
    lp.lp_batch_destroy(b)
    for ev in evs:
        ev.close()


def test_automatic_levels(lp, disk):
    from workloads import configs
    ev = lp.Evaluator(disk, precision="fp64", levels="auto")
    assert ev.info()["levels"] == 1 and ev.info()["g_fh"] <= 1536
    ev.close()
    q = configs.circle_layer_problem(n_panels=256, delta=8e-6, n_targets=10)
    ev = lp.Evaluator(q, precision="fp64", levels="auto")
    assert ev.info()["levels"] == 2
    ev.close()
