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
