"""Parity at the benchmark's full sizes, in the configuration the benchmark
times (device-resident inputs, one plan, V + S + D in one lp_execute), on
sampled targets the oracle evaluates one by one.

Sample: 10,000 targets per workload (uniform draws, the boundary band and
the corners), the oracle evaluating each one by direct summation.

Workloads: the 1.2M-node starfish (FP64 at 1e-9 and FP32 at 1e-5; also with
three levels of dyadic refinement, one history level, and upsampling 1.25
with the bin autotuner) and the 12M-node square with 1M vertex targets
(geometry-only boundary, V only; FP64 at 1e-9 and FP32 at 1e-5).  The sample mixes uniformly drawn targets with the
targets closest to the boundary (local expansions, on-surface points and, on
the square, the corners).
"""
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


def _sample(prob, n=10_000, n_near=1_000, seed=17):
    """A 10k-target subsample: uniformly drawn targets plus the
    band near the boundary -- the nearest targets first (on-surface points),
    then every k-th by distance so that the whole 12 sqrt(delta) band is
    covered -- plus the targets nearest to the corners of the box (the
    square's corners)."""
    from scipy.spatial import cKDTree
    txy = prob["tgt_xy"]
    rng = np.random.default_rng(seed)
    d, _ = cKDTree(prob["bnd"]["xy"]).query(txy)
    order = np.argsort(d, kind="stable")
    band = order[: np.searchsorted(d[order], 12 * np.sqrt(prob["delta"]))]
    near = np.concatenate([order[: n_near // 4], band[:: max(1, len(band) // (3 * n_near // 4))]])
    lo, hi = np.asarray(prob["box_lo"]), np.asarray(prob["box_hi"])
    corners = [np.argmin(np.sum((txy - c) ** 2, axis=1))
               for c in ([lo[0], lo[1]], [hi[0], lo[1]], [lo[0], hi[1]], [hi[0], hi[1]])]
    rand = rng.choice(len(txy), n - len(np.unique(near)) - 4, replace=False)
    return np.unique(np.concatenate([rand, near, corners]))


_ORACLE = {}


def _oracle_at(oracle_lib, prob, idx, want, refine_levels):
    """Oracle values at the sampled targets, shared by every plan variant of
    the same workload and refinement (the oracle does not depend on the
    plan's precision, tolerance, levels or upsampling)."""
    key = (prob["name"], len(prob["tgt_xy"]), refine_levels, want)
    if key not in _ORACLE:
        _ORACLE[key] = oracle_lib.evaluate(prob, targets=idx, want=want, refine_levels=refine_levels)
    return _ORACLE[key]


def _run(lp, prob, precision, tol, oracle_lib, **plan):
    want = tuple(k for k in "VSD" if k == "V" or prob.get({"S": "sigma", "D": "mu"}[k]) is not None)
    ev = lp.Evaluator(prob, precision=precision, tol=tol, **plan).bind()
    out = ev.evaluate(want=want)
    idx = _sample(prob)
    assert len(idx) >= 9_900
    ref = _oracle_at(oracle_lib, prob, idx, want, int(ev.info()["refine_levels"]))
    for k in want:
        full = out[k].cpu().numpy()
        got = full[idx]
        l2 = np.linalg.norm(got - ref[k]) / np.linalg.norm(ref[k])
        mx = np.max(np.abs(got - ref[k])) / np.max(np.abs(ref[k]))
        assert l2 < tol, f"{k}: rel-L2 {l2:.3e} over {len(idx)} sampled targets"
        assert mx < 5 * tol, f"{k}: rel-max {mx:.3e}"
        assert np.all(np.isfinite(full))
    ev.close()


@pytest.fixture(scope="module")
def starfish():
    from workloads import configs
    return configs.starfish()


@pytest.fixture(scope="module")
def square():
    from workloads import configs
    return configs.square()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-5)])
def test_starfish_full_size(lp, starfish, oracle_lib, precision, tol):
    _run(lp, starfish, precision, tol, oracle_lib)


@pytest.mark.parametrize("precision,tol,plan", [("fp64", 1e-9, dict(refine_levels=3)),
                                                ("fp32", 1e-5, dict(refine_levels=3)),
                                                ("fp64", 1e-9, dict(levels=1)),
                                                ("fp32", 1e-5, dict(upsampling=1.25, autotune=True))])
def test_starfish_full_size_variants(lp, starfish, oracle_lib, precision, tol, plan):
    """Dyadic refinement, one history level, other upsampling with the
    bin autotuner, at the full starfish size."""
    _run(lp, starfish, precision, tol, oracle_lib, **plan)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-5)])
def test_square_12M_full_size(lp, square, oracle_lib, precision, tol):
    _run(lp, square, precision, tol, oracle_lib)
