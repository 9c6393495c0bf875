"""Continuous batching: every request's V, S, D are the same as the request
evaluated alone, whether it ran in a wave with others or not."""
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


def test_results_same_alone_and_in_the_mix(lp, oracle_lib):
    from paper_2409_11998_gb300 import serve
    from workloads import configs
    pool = configs.serving_pool(n_meshes=4, t_min=1500, t_max=12000, seed=5100)
    # bursts of overlapping arrivals on every mesh, so waves mix meshes and
    # later requests for a mesh wait for its plan
    arrivals = [(0.001 * (i // 5), i % 4, 0.6 + 0.05 * i) for i in range(20)]
    srv = serve.Server(pool, precision="fp32", tol=1e-5, n_slots=2, max_wave=8, keep_outputs=True)
    srv.prewarm()
    reqs = srv.run(arrivals)
    stats = serve.latency_stats(reqs)
    assert stats["requests"] == 20 and stats["p99_ms"] >= stats["p50_ms"] > 0
    assert srv.created == 2 * len(pool) and srv.created_in_loop == 0   # every plan made before serving
    for r in reqs:
        p = pool[r.mesh]
        ev = lp.Evaluator(p, precision="fp32", tol=1e-5, levels=srv.levels).bind(src_f=p["src_f"] * r.scale,
                                                             sigma=p["sigma"] * r.scale,
                                                             mu=p["mu"] * r.scale)
        alone = ev.evaluate(tgt_jet=p["tgt_jet"] * r.scale)
        for k in "VSD":
            a = alone[k].cpu().numpy()
            b = r.outputs[k].cpu().numpy()
            assert np.max(np.abs(a - b)) <= 5e-6 * np.max(np.abs(a)), (r.rid, k)
        ev.close()
    # served results against the oracle (densities scaled as the request's)
    for r in reqs[:4]:
        p = dict(pool[r.mesh])
        for k in ("src_f", "sigma", "mu", "tgt_jet"):
            p[k] = pool[r.mesh][k] * r.scale
        idx = np.random.default_rng(r.rid).choice(len(p["tgt_xy"]), 200, replace=False)
        ref = oracle_lib.evaluate(p, targets=idx)
        for k in "VSD":
            got = r.outputs[k].cpu().numpy()[idx]
            assert np.linalg.norm(got - ref[k]) / np.linalg.norm(ref[k]) < 1e-5, (r.rid, k)
    srv.close()


def test_one_at_a_time_path(lp):
    from paper_2409_11998_gb300 import serve
    from workloads import configs
    pool = configs.serving_pool(n_meshes=2, t_min=1500, t_max=4000, seed=5200, precision="fp64", tol=1e-9)
    srv = serve.Server(pool, precision="fp64", tol=1e-9, one_at_a_time=True, keep_outputs=True)
    srv.prewarm()
    reqs = srv.run([(0.0, 0, 1.0), (0.0, 1, 1.0), (0.001, 0, 2.0)])
    a = reqs[0].outputs["V"].cpu().numpy()
    c = reqs[2].outputs["V"].cpu().numpy()
    assert np.allclose(2.0 * a, c, rtol=1e-12, atol=1e-14 * np.max(np.abs(a)))  # linear in the densities
    srv.close()


def test_abandoned_requests_leave_the_server_consistent(lp):
    """Clients that stop waiting: requests abandoned in the queue never
    launch, requests abandoned in flight finish with their wave and lose
    their outputs, and the others are served exactly as without them (the
    same results as the request alone); no plan stays busy."""
    from paper_2409_11998_gb300 import serve
    from workloads import configs
    pool = configs.serving_pool(n_meshes=3, t_min=1500, t_max=6000, seed=5300)
    # five requests per mesh at once: the first wave takes one per mesh, the
    # rest wait; every second request's client leaves after 0.2 ms
    arrivals = []
    for i in range(15):
        a = (0.0, i % 3, 0.7 + 0.05 * i)
        arrivals.append(a + (2e-4,) if i % 2 else a)
    srv = serve.Server(pool, precision="fp32", tol=1e-5, n_slots=1, max_wave=8, keep_outputs=True)
    srv.prewarm()
    reqs = srv.run(arrivals)
    left = [r for r in reqs if r.abandoned]
    kept = [r for r in reqs if not r.abandoned]
    assert len(left) >= 1 and len(kept) >= 8
    assert all(r.outputs is None for r in left)
    assert any(r.t_launch < 0 for r in left)          # dropped while waiting
    assert all(r.t_done >= r.t_launch >= 0 for r in kept)
    assert all(not inst.busy for lst in srv.pools.values() for inst in lst)
    st = serve.latency_stats(reqs)
    assert st["requests"] == len(kept) and st["abandoned"] == len(left)
    for r in kept[:4]:
        p = pool[r.mesh]
        ev = lp.Evaluator(p, precision="fp32", tol=1e-5, levels=srv.levels).bind(src_f=p["src_f"] * r.scale,
                                                             sigma=p["sigma"] * r.scale,
                                                             mu=p["mu"] * r.scale)
        alone = ev.evaluate(tgt_jet=p["tgt_jet"] * r.scale)
        for k in "VSD":
            a = alone[k].cpu().numpy()
            b = r.outputs[k].cpu().numpy()
            assert np.max(np.abs(a - b)) <= 5e-6 * np.max(np.abs(a)), (r.rid, k)
        ev.close()
    srv.close()
