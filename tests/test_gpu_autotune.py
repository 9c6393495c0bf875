"""The bin-side autotuner: a plan created with autotune times the binned
volume spread for its three candidate bin sides on the bound sources, keeps
the fastest, and still matches the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CANDIDATES = {"fp64": (16, 24, 32), "fp32": (16, 32, 48)}


@pytest.fixture(scope="module")
def lp():
    from paper_2409_11998_gb300 import build
    build.build()
    import paper_2409_11998_gb300 as lp
    return lp


@pytest.mark.parametrize("precision,tol,levels", [("fp64", 1e-9, 2), ("fp32", 1e-5, 2), ("fp64", 1e-9, 1)])
def test_autotuned_plan(lp, oracle_lib, precision, tol, levels):
    from workloads import configs
    p = configs.starfish(seed=2003, n_interior=2600, n_boundary_vertices=200, n_panels=256)
    idx = np.random.default_rng(5).choice(len(p["tgt_xy"]), 1000, replace=False)
    ref = oracle_lib.evaluate(p, targets=idx)
    ev = lp.Evaluator(p, precision=precision, tol=tol, levels=levels, autotune=True).bind()
    info = ev.info()
    times = [info["tune_ms_0"], info["tune_ms_1"], info["tune_ms_2"]]
    assert info["binned"] == 1 and info["bin_cells"] in CANDIDATES[precision]
    ok = [t for t in times if t > 0]
    assert ok and info["bin_cells"] == CANDIDATES[precision][times.index(min(ok))]
    out = ev.evaluate(tgt_xy=p["tgt_xy"][idx], tgt_jet=p["tgt_jet"][idx])
    for k in "VSD":
        got = out[k].cpu().numpy()
        assert np.linalg.norm(got - ref[k]) / np.linalg.norm(ref[k]) < tol, k
    # rebinding new sources keeps the tuned side
    ev.bind(src_f=2 * p["src_f"])
    assert ev.info()["bin_cells"] == info["bin_cells"]
    ev.close()


GRID_KEYS = ("grid_ms_s125_l1", "grid_ms_s125_l2", "grid_ms_s15_l1", "grid_ms_s15_l2", "grid_ms_s2_l1",
             "grid_ms_s2_l2")


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp64", 1e-9)])
def test_grid_autotuner_on_the_starfish(lp, oracle_lib, precision, tol):
    """LP_AUTOTUNE_FULL on the 1.2M-node starfish: the plan keeps the fastest
    of the six upsampling x level configurations, matches the oracle within
    the tolerance, and evaluates V, S, D no slower than the default plan."""
    import time
    from workloads import configs
    p = configs.starfish()
    stream = torch.cuda.Stream()

    def timed(ev):
        t_xy = torch.as_tensor(p["tgt_xy"], device="cuda")
        jet = torch.as_tensor(p["tgt_jet"], device="cuda")
        ev.evaluate(tgt_xy=t_xy, tgt_jet=jet)
        best = 1e30
        for _ in range(5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = ev.evaluate(tgt_xy=t_xy, tgt_jet=jet)
            best = min(best, time.perf_counter() - t0)
        return best, out

    ev = lp.Evaluator(p, precision=precision, tol=tol, stream=stream.cuda_stream, autotune="full").bind()
    info = ev.info()
    ms = [info[k] for k in GRID_KEYS]
    built = [m for m in ms if m > 0]
    assert len(built) >= 4, ms
    chosen = GRID_KEYS[ms.index(min(built))]
    sigma = {"s125": 1.25, "s15": 1.5, "s2": 2.0}[chosen.split("_")[2]]
    assert abs(info["sigma"] - sigma) < 1e-12 and info["levels"] == int(chosen[-1]), (chosen, info)
    t_tuned, out = timed(ev)
    idx = np.random.default_rng(9).choice(len(p["tgt_xy"]), 2000, replace=False)
    ref = oracle_lib.evaluate(p, targets=idx)
    for k in "VSD":
        got = out[k].cpu().numpy()[idx]
        assert np.linalg.norm(got - ref[k]) / np.linalg.norm(ref[k]) < tol, k
    ev.close()
    base = lp.Evaluator(p, precision=precision, tol=tol, stream=stream.cuda_stream).bind()
    t_default, _ = timed(base)
    base.close()
    assert t_tuned <= 1.05 * t_default, (t_tuned, t_default, chosen, ms)
