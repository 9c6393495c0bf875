"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: the FP64 path must match the oracle within the plan tolerance
(1e-9 relative L2 for V, S, D; the smooth part differs from the oracle's
direct sum only by the NUFFT error, the local part only by rounding).  The
FP32 path must match within 1e-5.  Element-wise maxima are checked against
the same bound scaled by the largest value.
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


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b))


def _compare(out, ref, keys, tol_l2, tol_max):
    for k in keys:
        got = out[k].cpu().numpy() if hasattr(out[k], "cpu") else out[k]
        l2, mx = _rel(got, ref[k])
        assert l2 < tol_l2, f"{k}: rel-L2 {l2:.3e}"
        assert mx < tol_max, f"{k}: rel-max {mx:.3e}"


@pytest.fixture(scope="module")
def disk():
    from workloads import configs
    return configs.disk()


@pytest.fixture(scope="module")
def disk_ref(disk, oracle_lib):
    return oracle_lib.evaluate(disk)


def test_disk_fp64_parity(lp, disk, disk_ref):
    ev = lp.Evaluator(disk, precision="fp64").bind()
    out = ev.evaluate()
    _compare(out, disk_ref, ("V", "S", "D"), 1e-9, 5e-9)
    ev.close()


def test_disk_fp64_parity_host_pointers(lp, disk, disk_ref):
    ev = lp.Evaluator(disk, precision="fp64", host=True).bind()
    out = ev.evaluate()
    _compare(out, disk_ref, ("V", "S", "D"), 1e-9, 5e-9)
    ev.close()


def test_disk_fp32_parity(lp, disk, disk_ref):
    ev = lp.Evaluator(disk, precision="fp32", tol=1e-5).bind()
    out = ev.evaluate()
    _compare(out, disk_ref, ("V", "S", "D"), 1e-5, 5e-5)
    ev.close()


@pytest.mark.parametrize("order", [3, 4])
def test_disk_lower_orders(lp, disk, oracle_lib, order):
    ref = oracle_lib.evaluate(disk, order=order)
    ev = lp.Evaluator(disk, precision="fp64", order=order).bind()
    out = ev.evaluate()
    _compare(out, ref, ("V", "S", "D"), 1e-9, 5e-9)
    ev.close()


def test_single_outputs_and_repeat(lp, disk, disk_ref):
    ev = lp.Evaluator(disk, precision="fp64").bind()
    for want in (("V",), ("S",), ("D",), ("S", "D")):
        out = ev.evaluate(want=want)
        _compare(out, disk_ref, want, 1e-9, 5e-9)
    a = ev.evaluate()
    b = ev.evaluate()
    for k in ("V", "S", "D"):
        # repeated calls agree to rounding (atomic accumulation order may vary)
        d = (a[k] - b[k]).abs().max().item()
        assert d <= 1e-13 * a[k].abs().max().item()
    ev.close()


def test_circle_layers_with_on_surface_targets(lp, oracle_lib):
    from workloads import configs
    p = configs.circle_layer_problem(n_panels=256, delta=1e-4, mode=3, n_targets=777, tol=1e-10)
    # add boundary nodes themselves as targets (on-surface)
    p["tgt_xy"] = np.concatenate([p["tgt_xy"], p["bnd"]["xy"][::5]])
    p["tgt_jet"] = np.zeros((len(p["tgt_xy"]), 6))
    ref = oracle_lib.evaluate(p, want=("S", "D"))
    ev = lp.Evaluator(p, precision="fp64")
    lp.lp_single_layer(ev.plan, torch.as_tensor(p["sigma"], device="cuda"))
    lp.lp_double_layer(ev.plan, torch.as_tensor(p["mu"], device="cuda"))
    out = ev.evaluate(want=("S", "D"))
    _compare(out, ref, ("S", "D"), 1e-10, 5e-10)
    ev.close()


def test_small_starfish_degraded_mesh(lp, oracle_lib):
    from workloads import configs
    p = configs.starfish(seed=2001, n_interior=2600, n_boundary_vertices=200, n_panels=256)
    idx = np.random.default_rng(0).choice(len(p["tgt_xy"]), 1500, replace=False)
    ref = oracle_lib.evaluate(p, targets=idx)
    ev = lp.Evaluator(p, precision="fp64").bind()
    out = ev.evaluate(tgt_xy=p["tgt_xy"][idx], tgt_jet=p["tgt_jet"][idx])
    _compare(out, ref, ("V", "S", "D"), 1e-9, 5e-9)
    ev.close()


def test_edge_cases(lp, disk, disk_ref):
    ev = lp.Evaluator(disk, precision="fp64").bind()
    # empty target set
    lp.lp_execute(ev.plan, 0, None, None, None, None, None)
    lp.lp_sync(ev.plan)
    # a single target, and a ragged count: errors measured against the whole
    # target set's RMS value (the metric's scale), not a 1-3 point subset's
    for n in (1, 3, 129):
        out = ev.evaluate(tgt_xy=disk["tgt_xy"][:n], tgt_jet=disk["tgt_jet"][:n])
        for k in "VSD":
            got = out[k].cpu().numpy()
            rms = np.linalg.norm(disk_ref[k]) / np.sqrt(len(disk_ref[k]))
            assert np.max(np.abs(got - disk_ref[k][:n])) < 5e-9 * rms, k
    # a target outside the box is reported, not written out of bounds
    bad = np.array([[10.0, 0.0]])
    with pytest.raises(lp.LpError) as e:
        ev.evaluate(tgt_xy=bad, tgt_jet=np.zeros((1, 6)))
    assert e.value.code == 2
    # NaN coordinates are rejected the same way
    with pytest.raises(lp.LpError):
        ev.evaluate(tgt_xy=np.array([[np.nan, 0.0]]), tgt_jet=np.zeros((1, 6)))
    # V at an exterior target inside the band has no expansion
    ext = np.array([[1.005, 0.0]])
    with pytest.raises(lp.LpError) as e:
        ev.evaluate(tgt_xy=ext, tgt_jet=np.zeros((1, 6)), want=("V",))
    assert e.value.code == 5
    out = ev.evaluate(tgt_xy=ext, tgt_jet=np.zeros((1, 6)), want=("S", "D"))
    assert np.isfinite(out["S"].cpu().numpy()).all()
    ev.close()


def test_no_volume_sources(lp, disk, oracle_lib):
    p = dict(disk)
    p["src_xy"] = np.zeros((0, 2))
    p["src_w"] = np.zeros(0)
    p["src_f"] = np.zeros(0)
    ref = oracle_lib.evaluate(p)
    ev = lp.Evaluator(p, precision="fp64").bind()
    out = ev.evaluate()
    got = out["V"].cpu().numpy()
    assert np.max(np.abs(got - ref["V"])) < 1e-15 + 1e-12 * np.max(np.abs(ref["V"]))
    ev.close()


def test_call_order_errors(lp, disk):
    ev = lp.Evaluator(disk, precision="fp64")
    with pytest.raises(lp.LpError) as e:
        ev.evaluate(want=("V",))
    assert e.value.code == 6
    ev.close()
