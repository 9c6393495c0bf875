"""Host-side logic of the server (no GPU): arrivals and latency statistics."""
import numpy as np

from paper_2409_11998_gb300 import serve


def test_poisson_arrivals_rate_and_order():
    arr = serve.poisson_arrivals(200.0, 50.0, 5, seed=1)
    t = np.array([a[0] for a in arr])
    assert np.all(np.diff(t) > 0) and t[-1] < 50.0
    assert abs(len(arr) / 50.0 - 200.0) < 200.0 * 0.05
    meshes = np.array([a[1] for a in arr])
    assert set(meshes.tolist()) == set(range(5))
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 200) < 0.05 / 200 * 10


def test_latency_stats():
    reqs = [serve.Request(i, 0, arrival=0.01 * i, scale=1.0, t_done=0.01 * i + 0.002 * (i + 1), points=10)
            for i in range(100)]
    st = serve.latency_stats(reqs)
    lat = np.array([0.002 * (i + 1) for i in range(100)])
    assert abs(st["p50_ms"] - np.percentile(lat, 50) * 1e3) < 1e-9
    assert abs(st["p99_ms"] - np.percentile(lat, 99) * 1e3) < 1e-9
    assert st["requests"] == 100


class _FakeStream:
    """A slot stream whose work takes `delay` seconds of simulated GPU time."""
    delay = 0.05

    def __init__(self, device=None):
        self.cuda_stream = 0


class _FakeEvent:
    def __init__(self):
        self.t = None

    def record(self, stream):
        import time
        self.t = time.perf_counter() + stream.delay

    def query(self):
        import time
        return self.t is not None and time.perf_counter() >= self.t


class _FakeCuda:
    Stream = _FakeStream
    Event = _FakeEvent

    @staticmethod
    def stream(s):
        import contextlib
        return contextlib.nullcontext()

    @staticmethod
    def synchronize():
        pass


class _FakeTorch:
    cuda = _FakeCuda
    float64 = np.float64

    @staticmethod
    def as_tensor(a, device=None):
        return np.asarray(a)

    @staticmethod
    def empty(n, dtype=None, device=None):
        return np.full(n, np.nan)


def _tiny_problem(seed):
    rng = np.random.default_rng(seed)
    n, nb, nt = 20, 16, 5
    return {"src_xy": rng.uniform(-1, 1, (n, 2)), "src_w": np.full(n, 0.1), "src_f": rng.normal(size=n),
            "bnd": {"xy": rng.uniform(-1, 1, (nb, 2)), "w": np.full(nb, 0.1), "normal": np.zeros((nb, 2)),
                    "n_panels": 1, "order": nb},
            "sigma": rng.normal(size=nb), "mu": rng.normal(size=nb), "tgt_xy": rng.uniform(-1, 1, (nt, 2)),
            "tgt_jet": rng.normal(size=(nt, 6)), "box_lo": (-1.5, -1.5), "box_hi": (1.5, 1.5), "delta": 1e-3}


def test_abandoned_requests(monkeypatch):
    """A request whose client leaves while it waits is never launched; one
    whose client leaves while its wave runs completes with the wave and its
    outputs are dropped; every plan is idle again at the end, and the
    latency statistics count the abandoned requests apart."""
    launched = []

    class Plan:
        pass

    def batch_execute(b, plans, nts, txy, jets, V, S, D):
        launched.append(len(plans))
        for o in (V, S, D):
            for arr in o:
                arr[:] = 1.0

    fakes = {"lp_plan": lambda *a, **k: Plan(), "lp_plan_info": lambda h: {"device_bytes": 1000},
             "lp_volume": lambda *a: None, "lp_single_layer": lambda *a: None, "lp_double_layer": lambda *a: None,
             "lp_batch_create": lambda s: object(), "lp_batch_execute": batch_execute,
             "lp_batch_destroy": lambda b: None, "lp_sync": lambda h: None, "lp_destroy": lambda h: None,
             "lp_execute": lambda *a: None}
    for k, v in fakes.items():
        monkeypatch.setattr(serve, k, v)
    srv = serve.Server([_tiny_problem(1), _tiny_problem(2)], n_slots=1, keep_outputs=True,
                       torch_module=_FakeTorch)
    srv.prewarm()
    # (arrival, mesh, scale, abandon): A and C form the first wave (one request
    # per mesh); B waits for mesh 0's plan and is abandoned while waiting; C is
    # abandoned while its wave runs; D waits for mesh 1 and completes
    arrivals = [(0.0, 0, 1.0), (0.0, 0, 1.0, 0.01), (0.0, 1, 1.0, 0.02), (0.001, 1, 1.0)]
    reqs = srv.run(arrivals)
    a, b, c, d = reqs
    assert not a.abandoned and a.t_launch >= 0 and np.all(a.outputs["V"] == 1.0)
    assert b.abandoned and b.t_launch < 0 and b.outputs is None
    assert c.abandoned and c.t_launch >= 0 and c.outputs is None
    assert not d.abandoned and d.t_launch >= a.t_done and np.all(d.outputs["S"] == 1.0)
    assert launched == [2, 1]
    assert all(not inst.busy for lst in srv.pools.values() for inst in lst)
    st = serve.latency_stats(reqs)
    assert st["requests"] == 2 and st["abandoned"] == 2
    srv.close()
