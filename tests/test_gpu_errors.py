"""Error contract of the C ABI on the GPU, with every failure made on the host
side from ordinary data: no kernel faults, traps or waits on anything.

* LP_ERR_NEWTON: a boundary panel whose parametrisation has zero speed at
  its middle (the same circular arc traversed as theta = theta_0 + c t^5), so
  that the closest point of a target on the arc's middle normal lies where
  the tangent frame of the local expansions (Sec. 4) is undefined.  The
  closest-point search of Sec. 2.2 must report it, and a regular panel of the
  same plan must not.
* LP_ERR_NOMEM: a plan whose device-memory budget is below what lp_plan or
  lp_volume needs; the allocation is refused before cudaMalloc is called.
* LP_ERR_TIMEOUT: lp_sync_timeout while the plan's stream is still busy
  behind a bounded spin kernel of about a quarter of a second.
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


def _circle_with_degenerate_panel(n_panels=64, p=16, bad=10, power=5):
    """Unit circle, n_panels Gauss-Legendre panels; panel `bad` covers its
    arc as theta = theta_mid + (dtheta/2) t^power (speed 0 at t = 0)."""
    tau, wq = np.polynomial.legendre.leggauss(p)
    dth = 2 * np.pi / n_panels
    th, w = [], []
    for i in range(n_panels):
        mid, c = (i + 0.5) * dth, 0.5 * dth
        if i == bad:
            th.append(mid + c * tau ** power)
            w.append(c * power * tau ** (power - 1) * wq)
        else:
            th.append(mid + c * tau)
            w.append(c * wq)
    th, w = np.concatenate(th), np.concatenate(w)
    xy = np.stack([np.cos(th), np.sin(th)], axis=1)
    return xy, w, xy.copy(), (bad + 0.5) * dth


def test_newton_status_on_degenerate_panel(lp):
    xy, w, nrm, th_bad = _circle_with_degenerate_panel()
    L = lp.library()
    delta = 1e-4                               # band 12 sqrt(delta) = 0.12
    plan = lp.lp_plan((-1.5, -1.5), (1.5, 1.5), delta, 1e-9, n_panels=64, panel_order=16,
                      bnd_xy=xy, bnd_w=w, bnd_normal=nrm)
    try:
        sigma = torch.ones(len(w), dtype=torch.float64, device="cuda")
        lp.lp_single_layer(plan, sigma)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        # control: a target on the middle normal of a regular panel
        th_ok = th_bad + np.pi
        t_ok = torch.tensor([[0.98 * np.cos(th_ok), 0.98 * np.sin(th_ok)]], dtype=torch.float64, device="cuda")
        assert L.lp_execute(plan, 1, t_ok.data_ptr(), None, None, out.data_ptr(), None) == 0
        assert L.lp_sync(plan) == 0
        assert np.isfinite(out.item())
        # the degenerate panel: same distance, middle normal of the zero-speed point
        t_bad = torch.tensor([[0.98 * np.cos(th_bad), 0.98 * np.sin(th_bad)]], dtype=torch.float64,
                             device="cuda")
        assert L.lp_execute(plan, 1, t_bad.data_ptr(), None, None, out.data_ptr(), None) == 0
        assert L.lp_sync(plan) == 7            # LP_ERR_NEWTON
        assert L.lp_sync(plan) == 0            # the status word was read and cleared
        assert b"closest-point" in L.lp_status_string(7)
    finally:
        lp.lp_destroy(plan)


def _disk_plan(lp, prob, **kw):
    b = prob["bnd"]
    return lp.lp_plan(prob["box_lo"], prob["box_hi"], prob["delta"], 1e-9, n_panels=b["n_panels"],
                      panel_order=b["order"], bnd_xy=b["xy"], bnd_w=b["w"], bnd_normal=b["normal"], **kw)


def test_nomem_from_the_plan_budget(lp):
    from workloads import configs
    prob = configs.disk()
    # a budget far below the grids: lp_plan refuses before any cudaMalloc
    with pytest.raises(lp.LpError) as e:
        _disk_plan(lp, prob, max_device_bytes=1 << 20)
    assert e.value.code == 3                   # LP_ERR_NOMEM
    # a budget that holds the plan but not the bound sources: lp_volume fails
    free_plan = _disk_plan(lp, prob)
    need = int(lp.lp_plan_info(free_plan)["device_bytes"])
    lp.lp_destroy(free_plan)
    plan = _disk_plan(lp, prob, max_device_bytes=need + 4096)
    try:
        assert int(lp.lp_plan_info(plan)["device_bytes"]) == need
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
        n = len(prob["src_w"])
        with pytest.raises(lp.LpError) as e:
            lp.lp_volume(plan, n, T(prob["src_xy"]), T(prob["src_w"]), T(prob["src_f"]))
        assert e.value.code == 3
        assert int(lp.lp_plan_info(plan)["device_bytes"]) <= need + 4096
        # the plan stays usable for what it holds: the layer potentials
        lp.lp_single_layer(plan, T(prob["sigma"]))
        lp.lp_sync(plan)
    finally:
        lp.lp_destroy(plan)


def test_sync_timeout_while_the_stream_is_busy(lp):
    from workloads import configs
    prob = configs.disk()
    stream = torch.cuda.Stream()
    ev = lp.Evaluator(prob, precision="fp64", stream=stream.cuda_stream).bind()
    ref = ev.evaluate()
    n = len(prob["tgt_xy"])
    txy, jet = ev._tgt
    outs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3)]
    with torch.cuda.stream(stream):
        torch.cuda._sleep(int(5e8))            # a bounded spin of ~0.25 s ahead of the evaluation
    lp.lp_execute(ev.plan, n, txy, jet, *outs)
    assert lp.lp_sync_timeout(ev.plan, 1.0) is False     # LP_ERR_TIMEOUT: still running
    assert lp.lp_sync_timeout(ev.plan, 60000.0) is True  # completes well within a minute
    for k, o in zip("VSD", outs):
        got, want = o.cpu().numpy(), ref[k].cpu().numpy()
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12, k
    L = lp.library()
    assert L.lp_sync_timeout(ev.plan, float("nan")) == 1
    ev.close()
