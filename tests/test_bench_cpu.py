"""bench.py's host-side arithmetic: the roofline picks the longest candidate
stage and reports it against the right peak with the algorithmic work of
that kernel."""
import bench


def _info(precision):
    return {"w": 12 if precision == 0 else 7, "es_nc": 13 if precision == 0 else 9, "g_nh": 2592 if precision == 0
            else 2916, "K_nh": 864 if precision == 0 else 729, "g_fh": 1024 if precision == 0 else 1152,
            "K_fh": 342 if precision == 0 else 288, "own_fft": 1, "precision": precision, "binned": 1}


def test_fp64_roofline_spread_or_interp():
    st = {"spread": 1.2, "spread_volume": 1.0, "multiplier": 0.5, "interp": 0.8}
    r = bench.roofline(_info(0), st, 1_000_000, 16384, 1_000_000, "fp64", workload="none")
    assert r["kernel"] == "spread_fx_kernel" and r["bound"] == "alu"
    # no ncu count for workload "none": the algorithmic estimate, 15 FP32
    # instructions per df64 multiply-add of the weight polynomials and 14
    # per fixed-point cell update, 32 lanes per warp instruction
    inst = 1_000_000 * 2 * (2 * 12 * 12 * 15 + 12 * 12 * 14) / 32
    assert r["instructions_per_step"] == int(inst) and r["instructions_source"].startswith("estimate")
    assert abs(r["achieved"] - inst / 1.0e-3 / 1e12) < 1e-3
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    assert abs(r["peak"] - 152 * 4 * bench.sm_max_mhz() * 1e6 / 1e12) < 1e-3
    # HBM fraction beside it: positions and strengths (24 B per node) and
    # both grids written once (8 B per cell)
    byts = 1_000_000 * 24 + (2592 ** 2 + 1024 ** 2) * 8
    assert r["hbm"]["algorithmic_bytes_per_step"] == byts
    assert abs(r["hbm_frac"] - byts / 1e-3 / 1e9 / r["hbm"]["peak"]) < 1e-4
    st["interp"] = 1.5
    r = bench.roofline(_info(0), st, 1_000_000, 16384, 1_000_000, "fp64", workload="none")
    assert r["kernel"] == "interp_dd_kernel"
    assert r["hbm"]["algorithmic_bytes_per_step"] == (2592 ** 2 + 1024 ** 2) * 8 * 3 + 1_000_000 * (16 + 24)


def test_fp32_roofline_dominant_stage():
    st = {"spread": 0.3, "spread_volume": 0.25, "multiplier": 0.28, "interp": 0.2}
    r = bench.roofline(_info(1), st, 1_000_000, 16384, 1_000_000, "fp32", workload="none")
    # a 2916-point near grid: three columns fit in 110 KB, two columns per CTA
    assert r["kernel"] == "fft_cols2_f32_kernel" and r["bound"] == "hbm"
    r6 = bench.roofline(dict(_info(1), g_nh=6144, K_nh=1536), st, 1_000_000, 16384, 1_000_000, "fp32",
                        workload="none")
    assert r6["kernel"] == "fft_cols_kernel"
    kp = lambda K: (K + 2) & ~1
    byts = 7 * 2916 * kp(729) * 8 + 7 * 1152 * kp(288) * 8
    assert r["hbm"]["algorithmic_bytes_per_step"] == byts and r["frac"] == r["hbm_frac"]
    st["multiplier"] = 0.1
    r = bench.roofline(_info(1), st, 1_000_000, 16384, 1_000_000, "fp32", workload="none")
    assert r["kernel"] == "spread_sub_kernel" and r["bound"] == "alu"
    assert r["instructions_per_step"] == int(1_000_000 * 2 * (49 + 2 * 7 * 8) / 32)


def test_single_level_plans_count_one_level():
    info = dict(_info(0), g_nh=0, K_nh=0)
    st = {"spread": 1.0, "spread_volume": 1.0, "multiplier": 0.5, "interp": 0.2}
    r = bench.roofline(info, st, 1000, 0, 1000, "fp64", workload="none")
    assert r["instructions_per_step"] == int(1000 * 1 * (2 * 12 * 12 * 15 + 12 * 12 * 14) / 32)
    assert r["hbm"]["algorithmic_bytes_per_step"] == 1000 * 24 + 1024 ** 2 * 8


def test_parity_block():
    import numpy as np
    gpu = {"V": np.array([1.0, 2.0, 3.0, 4.0]), "S": np.array([1.0, 1.0, 1.0, 1.0])}
    ref = {"V": np.array([2.0, 3.0]), "S": np.array([1.0, 2.0]), "D": np.array([0.5, 0.5])}
    p = bench.parity(gpu, ref, np.array([1, 2]))
    assert set(p) == {"V", "S"} and p["V"]["rel_l2"] == 0.0 and p["V"]["n_targets"] == 2
    assert abs(p["S"]["rel_max"] - 0.5) < 1e-15


def test_reference_arm_line_contract():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the keys of the GPU arm plus impl, cpu_baseline and an
    e2e object with zero copy bytes."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "disk", "--steps", "1",
                          "--warmup", "1"], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]
