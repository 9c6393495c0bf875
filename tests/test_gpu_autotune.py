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
