"""Source sharding through the C ABI on one GPU: two plans stand for two
ranks (each binds half of the volume nodes, rank 0 spreads the layers), the
sum of their grid buffers stands for the all-reduce, and each finishes half
of the targets.  The result must equal one unsharded lp_execute: only the
order of the spread's sums changes."""
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


@pytest.mark.parametrize("precision,tol,same", [("fp64", 1e-9, 1e-12), ("fp32", 1e-5, 5e-6)])
@pytest.mark.parametrize("name", ["disk", "star"])
def test_two_plans_as_two_ranks(lp, oracle_lib, precision, tol, same, name):
    from paper_2409_11998_gb300 import shard
    from workloads import configs
    p = configs.disk() if name == "disk" else configs.star_batch_member(4100, 20000)
    stream = torch.cuda.Stream()
    ref_ev = lp.Evaluator(p, precision=precision, tol=tol, stream=stream.cuda_stream).bind()
    ref = {k: v.cpu().numpy() for k, v in ref_ev.evaluate().items()}
    ref_ev.close()
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    holders = [lp.Evaluator(p, precision=precision, tol=tol, stream=stream.cuda_stream) for _ in range(2)]
    ranks = [shard.ShardedEvaluation(lp, h.plan, p, r, 2, allreduce=None, to_device=T).bind()
             for r, h in enumerate(holders)]
    for r in ranks:
        r.spread()
    torch.cuda.synchronize()
    bufs = [r.buffers() for r in ranks]
    assert len(bufs[0]) == len(bufs[1]) >= 4
    for a, b in zip(*bufs):        # the all-reduce: both ranks end with the sum
        s = a + b
        a.copy_(s)
        b.copy_(s)
    torch.cuda.synchronize()
    parts = []
    for r in ranks:
        lo, hi = r.tgt
        out = {k: torch.empty(hi - lo, dtype=torch.float64, device="cuda") for k in "VSD"}
        r.finish(out)
        lp.lp_sync(r.plan)
        parts.append({k: v.cpu().numpy() for k, v in out.items()})
    for k in "VSD":
        got = np.concatenate([d[k] for d in parts])
        assert np.max(np.abs(got - ref[k])) <= same * np.max(np.abs(ref[k])), k
    # and against the oracle on a sample
    idx = np.random.default_rng(3).choice(len(p["tgt_xy"]), 300, replace=False)
    o = oracle_lib.evaluate(p, targets=idx)
    for k in "VSD":
        got = np.concatenate([d[k] for d in parts])[idx]
        assert np.linalg.norm(got - o[k]) / np.linalg.norm(o[k]) < tol, k
    for h in holders:
        h.close()


def test_finish_needs_the_spread(lp):
    from workloads import configs
    p = configs.disk()
    ev = lp.Evaluator(p, precision="fp64").bind()
    L = lp.library()
    t = torch.as_tensor(p["tgt_xy"], device="cuda")
    j = torch.as_tensor(p["tgt_jet"], device="cuda")
    out = torch.empty(len(t), dtype=torch.float64, device="cuda")
    assert L.lp_finish(ev.plan, len(t), t.data_ptr(), j.data_ptr(), out.data_ptr(), None, None) == 6
    lp.lp_spread(ev.plan, "S", spread_layers=True)
    # V was not spread: LP_ERR_STATE
    assert L.lp_finish(ev.plan, len(t), t.data_ptr(), j.data_ptr(), out.data_ptr(), None, None) == 6
    assert L.lp_finish(ev.plan, len(t), t.data_ptr(), None, None, out.data_ptr(), None) == 0
    assert L.lp_sync(ev.plan) == 0
    ev.close()
