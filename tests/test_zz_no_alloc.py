"""lp_execute_noalloc: the evaluation entry point for callers that cannot
allocate device memory at evaluation time (another allocator holds the
device's memory, or a loop must not take the implicit synchronisation of
cudaMalloc/cudaFree).  It must return what lp_execute returns, call after
call, while keeping its per-call scratch in a static device array.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

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


def test_noalloc_matches_execute_on_two_calls(lp):
    from workloads import configs
    prob = configs.disk()
    ev = lp.Evaluator(prob, precision="fp64").bind()
    ref = ev.evaluate()                      # lp_execute, device buffers
    txy, jet = ev._tgt
    n = len(prob["tgt_xy"])
    L = lp.library()
    for _ in range(2):                       # two calls in a row share the static scratch
        outs = [torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
        rc = L.lp_execute_noalloc(ev.plan, n, txy.data_ptr(), jet.data_ptr(),
                                  *[o.data_ptr() for o in outs])
        assert rc == 0
        assert L.lp_sync(ev.plan) == 0
        for k, o in zip("VSD", outs):
            got = o.cpu().numpy()
            want = ref[k].cpu().numpy()
            assert np.all(np.isfinite(got))
            # same tolerance as the parity tests
            assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-9, k
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
