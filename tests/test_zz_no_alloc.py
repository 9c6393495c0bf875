"""lp_execute_noalloc: the evaluation entry point for callers that cannot
allocate device memory at evaluation time (another allocator holds the
device's memory, or a loop must not take the implicit synchronisation of
cudaMalloc/cudaFree).  It must return what lp_execute returns, call after
call, allocate nothing -- its per-call scratch lives in a static device
array -- and agree with the FP64 oracle.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
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


def _rel(got, want):
    return np.linalg.norm(got - want) / np.linalg.norm(want)


def _outputs(n):
    return [torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]


def _noalloc(lp, plan, n, txy, jet, outs=None):
    L = lp.library()
    outs = _outputs(n) if outs is None else outs
    rc = L.lp_execute_noalloc(plan, n, txy.data_ptr(), jet.data_ptr(), *[o.data_ptr() for o in outs])
    assert rc == 0
    assert L.lp_sync(plan) == 0
    return dict(zip("VSD", (o.cpu().numpy() for o in outs)))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-5)])
def test_noalloc_matches_execute_on_two_calls(lp, precision, tol):
    """A fresh plan's first evaluations go through lp_execute_noalloc (so no
    buffer lp_execute would size can help it); the plan's device footprint
    and the device's free memory stay the same across two calls, whose
    results agree with lp_execute afterwards within the parity tolerance."""
    from workloads import configs
    prob = configs.disk()
    n = len(prob["tgt_xy"])
    txy = torch.as_tensor(prob["tgt_xy"], device="cuda")
    jet = torch.as_tensor(prob["tgt_jet"], device="cuda")
    warm = lp.Evaluator(prob, precision=precision, tol=tol).bind()   # loads the kernels once
    warm.evaluate()
    # the set-up call: the device's first call finds the static scratch,
    # which is when the driver loads (and backs) it
    _noalloc(lp, warm.plan, n, txy, jet)
    warm.close()
    ev = lp.Evaluator(prob, precision=precision, tol=tol).bind()
    lp.lp_sync(ev.plan)
    outs = [_outputs(n) for _ in range(2)]       # the caller's buffers exist before the calls
    torch.cuda.synchronize()
    bytes0 = lp.lp_plan_info(ev.plan)["device_bytes"]
    free0 = torch.cuda.mem_get_info()[0]
    got = [_noalloc(lp, ev.plan, n, txy, jet, o) for o in outs]   # two calls share the static scratch
    torch.cuda.synchronize()
    assert lp.lp_plan_info(ev.plan)["device_bytes"] == bytes0
    assert torch.cuda.mem_get_info()[0] == free0
    ref = ev.evaluate(tgt_xy=txy, tgt_jet=jet)                     # lp_execute
    for k in "VSD":
        want = ref[k].cpu().numpy()
        for g in got:
            assert np.all(np.isfinite(g[k]))
            assert _rel(g[k], want) < tol, k
    ev.close()


def test_noalloc_starfish_against_the_oracle(lp, oracle_lib):
    """1.2M targets (below the 2,097,152-target scratch limit) on the starfish,
    FP64 at 1e-9, against the oracle on sampled targets (random ones and
    those nearest the boundary)."""
    from scipy.spatial import cKDTree
    from workloads import configs
    prob = configs.starfish()
    n = len(prob["tgt_xy"])
    ev = lp.Evaluator(prob, precision="fp64", tol=1e-9).bind()
    txy = torch.as_tensor(prob["tgt_xy"], device="cuda")
    jet = torch.as_tensor(prob["tgt_jet"], device="cuda")
    got = _noalloc(lp, ev.plan, n, txy, jet)
    rng = np.random.default_rng(23)
    d, _ = cKDTree(prob["bnd"]["xy"]).query(prob["tgt_xy"])
    idx = np.unique(np.concatenate([rng.choice(n, 1500, replace=False), np.argsort(d, kind="stable")[:500]]))
    ref = oracle_lib.evaluate(prob, targets=idx)
    for k in "VSD":
        assert _rel(got[k][idx], ref[k]) < 1e-9, k
        assert np.max(np.abs(got[k][idx] - ref[k])) / np.max(np.abs(ref[k])) < 5e-9, k
    ev.close()


def test_noalloc_rejects_what_it_cannot_serve(lp):
    from workloads import configs
    prob = configs.disk()
    ev = lp.Evaluator(prob, precision="fp64").bind()
    L = lp.library()
    txy, jet = (torch.as_tensor(prob["tgt_xy"], device="cuda"),
                torch.as_tensor(prob["tgt_jet"], device="cuda"))
    out = torch.empty(len(txy), dtype=torch.float64, device="cuda")
    # beyond the static scratch: rejected before anything is launched
    assert L.lp_execute_noalloc(ev.plan, (1 << 21) + 1, txy.data_ptr(), jet.data_ptr(),
                                out.data_ptr(), None, None) == 1
    # host buffers would need staging (an allocation): rejected
    host = np.zeros(len(txy))
    assert L.lp_execute_noalloc(ev.plan, len(txy), txy.data_ptr(), jet.data_ptr(),
                                host.ctypes.data, None, None) == 1
    assert L.lp_sync(ev.plan) == 0
    ev.close()
