"""lp_volume_jets: f-jets at targets estimated from the bound node values
(for callers without analytic derivatives) against the oracle's statement of
the same estimator, and V evaluated from them against the oracle's V from its
own estimated jets."""
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


def _sample(p, n, seed):
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    d, _ = cKDTree(p["bnd"]["xy"]).query(p["tgt_xy"])
    near = np.argsort(d, kind="stable")[: n // 5]
    return np.unique(np.concatenate([near, rng.choice(len(p["tgt_xy"]), n - len(near), replace=False)]))


@pytest.mark.parametrize("name", ["starfish", "disk"])
def test_jets_and_volume_potential_from_node_values(lp, oracle_lib, name):
    from oracle import jets as ojets
    from workloads import configs
    p = getattr(configs, name)()
    side = max(p["box_hi"][0] - p["box_lo"][0], p["box_hi"][1] - p["box_lo"][1])
    ev = lp.Evaluator(p, precision="fp64", tol=1e-9).bind()
    nt = len(p["tgt_xy"])
    txy = torch.as_tensor(p["tgt_xy"], device="cuda")
    jet = torch.empty((nt, 6), dtype=torch.float64, device="cuda")
    lp.lp_volume_jets(ev.plan, nt, txy, jet)
    got = jet.cpu().numpy()
    idx = _sample(p, 2000 if name == "starfish" else nt, 31)
    ref = ojets.estimate_jets(p["src_xy"], p["src_f"], p["tgt_xy"][idx], p["delta"], side)
    # same estimator: the GPU holds node offsets in single precision (~1e-7 of
    # rho), so components agree to ~1e-6 of their scale
    scale = np.max(np.abs(ref), axis=0) + 1e-300
    err = np.max(np.abs(got[idx] - ref), axis=0) / scale
    assert err[0] < 1e-9 and np.all(err[1:] < 1e-5), err
    # against the analytic jets the fit is a method error of a quadratic over
    # three node spacings (starfish: RMS ~5% in the first derivatives, ~20%
    # in the second, which enter V at delta^{3/2} and delta^2)
    inside = np.any(np.abs(p["tgt_jet"][idx]) > 0, axis=1)
    ana = p["tgt_jet"][idx][inside]
    rel = np.sqrt(np.mean((ref[inside] - ana) ** 2, axis=0)) / (np.sqrt(np.mean(ana ** 2, axis=0)) + 1e-300)
    assert rel[0] < 0.02 and np.all(rel[1:3] < 0.1) and np.all(rel[3:] < 0.5), rel
    # V from the estimated jets, against the oracle fed its own estimated jets
    out = ev.evaluate(tgt_xy=txy, tgt_jet=jet, want=("V",))
    q = dict(p)
    q["tgt_jet"] = p["tgt_jet"].copy()
    q["tgt_jet"][idx] = ref
    want = oracle_lib.evaluate(q, targets=idx, want=("V",))["V"]
    v = out["V"].cpu().numpy()[idx]
    assert np.linalg.norm(v - want) / np.linalg.norm(want) < 1e-9
    assert np.max(np.abs(v - want)) / np.max(np.abs(want)) < 5e-9
    ev.close()


def test_jets_need_bound_sources(lp):
    from workloads import configs
    p = configs.disk()
    ev = lp.Evaluator(p, precision="fp64")
    L = lp.library()
    t = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    j = torch.empty((4, 6), dtype=torch.float64, device="cuda")
    assert L.lp_volume_jets(ev.plan, 4, t.data_ptr(), j.data_ptr()) == 6   # LP_ERR_STATE
    ev.close()
