"""Batched waves (one launch per kernel for many uneven problems) return what
each problem returns alone, and match the oracle."""
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


def _problems():
    from workloads import configs
    sizes = [300, 1200, 4000, 700, 2500]
    return [configs.star_batch_member(4000 + i, n) for i, n in enumerate(sizes)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-5)])
def test_batch_equals_alone_and_oracle(lp, oracle_lib, precision, tol):
    probs = _problems()
    stream = torch.cuda.Stream()
    evs = [lp.Evaluator(p, precision=precision, tol=tol, stream=stream.cuda_stream).bind() for p in probs]
    alone = [ev.evaluate() for ev in evs]
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    txy = [dev(p["tgt_xy"]) for p in probs]
    jet = [dev(p["tgt_jet"]) for p in probs]
    outs = {k: [torch.full((len(p["tgt_xy"]),), float("nan"), dtype=torch.float64, device="cuda")
                for p in probs] for k in "VSD"}
    b = lp.lp_batch_create(stream.cuda_stream)
    for _ in range(2):
        lp.lp_batch_execute(b, [ev.plan for ev in evs], [len(p["tgt_xy"]) for p in probs], txy, jet,
                            outs["V"], outs["S"], outs["D"])
        lp.lp_batch_sync(b)
        for ev in evs:
            lp.lp_sync(ev.plan)
        for i, p in enumerate(probs):
            for k in "VSD":
                got = outs[k][i].cpu().numpy()
                ref = alone[i][k].cpu().numpy()
                # same arithmetic as alone; atomics may reorder sums (float: ~1e-7)
                same = 1e-12 if precision == "fp64" else 5e-6
                assert np.max(np.abs(got - ref)) <= same * np.max(np.abs(ref)) + 1e-300, (i, k)
    st = lp.lp_batch_stage_times(b)
    assert st["total"] > 0
    # against the oracle on a sample of each problem
    for i, p in enumerate(probs):
        idx = np.random.default_rng(i).choice(len(p["tgt_xy"]), min(120, len(p["tgt_xy"])), replace=False)
        ref = oracle_lib.evaluate(p, targets=idx)
        for k in "VSD":
            got = outs[k][i].cpu().numpy()[idx]
            assert np.linalg.norm(got - ref[k]) / np.linalg.norm(ref[k]) < tol, (i, k)
    lp.lp_batch_destroy(b)
    for ev in evs:
        ev.close()


def test_batch_rejects_mixed_or_duplicate(lp):
    probs = _problems()[:2]
    e64 = lp.Evaluator(probs[0], precision="fp64").bind()
    e32 = lp.Evaluator(probs[1], precision="fp32", tol=1e-5).bind()
    b = lp.lp_batch_create()
    t = [torch.as_tensor(p["tgt_xy"], device="cuda") for p in probs]
    o = [torch.empty(len(p["tgt_xy"]), dtype=torch.float64, device="cuda") for p in probs]
    with pytest.raises(lp.LpError) as e:
        lp.lp_batch_execute(b, [e64.plan, e32.plan], [len(x) for x in t], t, None, None, o, None)
    assert e.value.code == 1
    with pytest.raises(lp.LpError) as e:
        lp.lp_batch_execute(b, [e64.plan, e64.plan], [len(t[0])] * 2, [t[0], t[0]], None, None, [o[0], o[0]], None)
    assert e.value.code == 1
    lp.lp_batch_destroy(b)
    e64.close()
    e32.close()
