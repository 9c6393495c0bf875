#!/usr/bin/env python
"""Benchmark of the V + S + D evaluation (heat-kernel splitting, arXiv 2409.11998).

Metric: source + target points per second, where one step evaluates V[f],
S[sigma] and D[mu] at every target of the workload through the C ABI:
lp_volume + lp_single_layer + lp_double_layer (bind the step's sources and
densities) + lp_execute (spread, FFTs, multiplier, interpolation, local part).
Points per step = N_V + N_B + N_t.

Default workload: the starfish r = 1 + 0.3 cos 5t with a degraded ~190k
triangle mesh (6 nodes per triangle), 1,024 x 16 boundary nodes, targets =
all quadrature nodes, FP64 at tolerance 1e-9.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lp|reference]

--impl reference times the FP64 CPU oracle (direct sums of the smoothed
kernel plus the same local expansions) on the host cores, on a bounded
sample of targets per step, and reports the same metric extrapolated to the
whole workload.  With N > 1 (torchrun), every rank runs an independent
replica of the workload on its own GPU (weak scaling, no collective on the
data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "source+target points/sec at 1e-9 (FP64) / 1e-5 (FP32) rel-L2; served p50/p99 latency"
UNIT = "points/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lp", choices=["lp", "reference"])
    ap.add_argument("--workload", default="starfish",
                    choices=["starfish", "disk", "square", "batch", "serve", "solve"])
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, cpu baseline, fp32 and serving lines")
    ap.add_argument("--batch-size", type=int, default=256, help="problems per wave (--workload batch)")
    ap.add_argument("--serve-seconds", type=float, default=8.0, help="seconds per arrival rate (--workload serve)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="plan precision of the timed line (fp64: tol 1e-9; fp32: tol 1e-5)")
    ap.add_argument("--levels", default="auto", choices=["auto", "1", "2"],
                    help="history levels of every plan (auto: one level when its grid side is <= 1536)")
    ap.add_argument("--bc", default="dirichlet", choices=["dirichlet", "neumann"],
                    help="boundary condition of --workload solve")
    ap.add_argument("--autotune", action="store_true",
                    help="plans time three bin sides on their sources at the first lp_volume")
    ap.add_argument("--refine-levels", type=int, default=0,
                    help="dyadic refinement levels of the local layer potentials (starfish/disk/square)")
    args = ap.parse_args()
    if args.refine_levels and args.workload in ("batch", "serve"):
        ap.error("--refine-levels applies to the single-problem workloads (batched waves take unrefined plans)")
    if not 0 <= args.refine_levels <= 6:
        ap.error("--refine-levels takes 0..6")
    return args


def make_problem(name):
    from workloads import configs
    if name == "starfish":
        return configs.starfish()
    if name == "disk":
        return configs.disk()
    if name == "square":
        return configs.square(precision="fp64", tol=1e-9)
    raise ValueError(name)


def describe(prob):
    m = prob["meta"]
    nb = len(prob["bnd"]["w"]) if prob["bnd"] is not None else 0
    desc = {
        "starfish": "starfish r=1+0.3cos5t, degraded Delaunay mesh (slivers with aspect ratio "
                    "log-uniform in [1,1e4], 2% non-conforming edges, 1% triangles removed), "
                    "6-node rule, 1024x16 boundary nodes, targets = all quadrature nodes",
        "disk": "unit disk, 2000 random-Delaunay triangles, 6-node rule, 64x16 boundary nodes, "
                "targets = vertices + 512 exterior points",
        "square": "[-1,1]^2, 2M jittered triangles, 6-node rule, targets = vertices",
    }[prob["name"]]
    return {"workload": desc, "n_triangles": m.get("n_triangles"), "n_sources": len(prob["src_w"]),
            "n_boundary_nodes": nb, "n_targets": len(prob["tgt_xy"]), "delta1": prob["delta"],
            "tol": prob["tol"]}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(parts)
            except Exception:
                pass
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------- GPU arm
def run_lp(args, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_2409_11998_gb300 as lp

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prob = make_problem(args.workload)
    nv, nb, nt = len(prob["src_w"]), len(prob["bnd"]["w"]), len(prob["tgt_xy"])
    points = nv + nb + nt
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    sxy, sw, sf = T(prob["src_xy"]), T(prob["src_w"]), T(prob["src_f"])
    sig, mu = layer_densities(prob, T)
    txy, jet = T(prob["tgt_xy"]), T(prob["tgt_jet"])
    outs = output_buffers(prob, nt, lambda: torch.empty(nt, dtype=torch.float64, device=dev))
    stream = torch.cuda.Stream(device=dev)
    fp64 = args.precision == "fp64"
    ev = lp.Evaluator(prob, precision=args.precision, tol=1e-9 if fp64 else 1e-5, stream=stream.cuda_stream,
                      refine_levels=args.refine_levels, levels=levels_arg(args), autotune=args.autotune)
    plan = ev.plan

    def step():
        lp.lp_volume(plan, nv, sxy, sw, sf)
        if sig is not None:
            lp.lp_single_layer(plan, sig)
        if mu is not None:
            lp.lp_double_layer(plan, mu)
        lp.lp_execute(plan, nt, txy, jet, outs[0], outs[1], outs[2])

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 3)):
        step()
        lp.lp_sync(plan)
    launches0 = lp.lp_plan_info(plan)["launches"]
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stages = []
    barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(local_rank)
    clk.start()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))          # evict L2 between steps (outside the step's events)
            e0[k].record(stream)
            step()
            e1[k].record(stream)
        lp.lp_sync(plan)
        stages.append(lp.lp_stage_times(plan))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = clk.stop()
    barrier(world)
    launches = lp.lp_plan_info(plan)["launches"] - launches0
    step_ms = [a.elapsed_time(b) for a, b in zip(e0, e1)]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, world)
    value = points * args.steps * world / (total_ms / 1e3)
    info = lp.lp_plan_info(plan)
    st = {k: statistics.mean(s[k] for s in stages) for k in stages[0]}

    roof = roofline(info, st, nv, nb, nt, precision=args.precision, n_out=sum(o is not None for o in outs),
                    workload=args.workload)

    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": dtype_of(info),
           "dtype_detail": dtype_detail(info),
           "data": "synthetic (seeded generators; no dataset)",
           "config": {**describe(prob), **refine_desc(args), "tol": ev.tol, "levels": int(info["levels"]),
                      "parallelism": "replicas" if world > 1 else "single",
                      "l2": "flushed by a 512 MiB write between timed steps, outside the step events",
                      "timing": "CUDA events on the plan stream around each step",
                      "grids": {"g_nh": int(info["g_nh"]), "g_fh": int(info["g_fh"]), "w": int(info["w"])}},
           "stages_ms": {k: round(v, 4) for k, v in st.items()},
           "roofline": roof, "gpu_launches": int(launches), "wall_s_timed_region": round(wall, 3),
           "clocks": clocks}

    gpu_out = {args.precision: {k: o.cpu().numpy() for k, o in zip("VSD", outs) if o is not None}}
    if rank == 0 and not args.no_extras:
        res["e2e"] = run_e2e(args, prob, dev, ev, points)
        if fp64:
            res["fp32_same_workload"] = run_fp32(args, prob, dev, stream, points)
            gpu_out["fp32"] = res["fp32_same_workload"].pop("_outputs")
            # the same FP32 path with the kernel width and grids chosen for
            # 1e-6: at 1e-5 its error is the truncation the width allows
            res["fp32_tol_1e-6"] = run_fp32(args, prob, dev, stream, points, tol=1e-6)
            gpu_out["fp32_tol_1e-6"] = res["fp32_tol_1e-6"].pop("_outputs")
        if args.workload == "starfish":
            res["square"] = run_square(args, dev, stream)
            wave = run_batch(args, rank, world, local_rank)
            res["batch"] = {"workload": wave["config"]["workload"], "points_per_wave": wave["config"]["points_per_wave"],
                            **wave["batch"]}
            res["served"] = run_serve(args, rank, world, local_rank, rates=(50, 200, 1000), seconds=1.5,
                                      max_requests=1200)
        if world == 1:
            checks = {}
            if "square" in res:
                checks["square"] = res["square"].pop("_check")
            res["cpu_baseline"] = cpu_baseline(prob, budget_s=15.0, refine_levels=args.refine_levels,
                                               gpu_out=gpu_out, checks=checks)
            res["parity"] = res["cpu_baseline"].pop("_parity")
            for name, par in res["cpu_baseline"].pop("_checks").items():
                for prec, p in par.items():
                    res[name][prec]["parity"] = p
        elif "square" in res:
            res["square"].pop("_check")
    ev.close()
    return res


def sm_max_mhz():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    mhz = 2070.0
    if os.path.exists(p):
        mhz = float(json.load(open(p)).get("sm_max_mhz", mhz))
    return mhz


def issue_peak_t():
    """Warp instructions per second the GPU can issue: 152 SMs x 4 schedulers
    x one instruction per clock x max SM clock (T/s)."""
    return 152 * 4 * sm_max_mhz() * 1e6 / 1e12


def fp32_fma_peak_t():
    """FP32 multiply-adds per second: 152 SMs x 128 lanes x max SM clock (T/s)."""
    return 152 * 128 * sm_max_mhz() * 1e6 / 1e12


def kernel_profile(name, workload):
    """ncu counters of a kernel per bench step (summed over its launches in a
    step) from profiles/traffic.json, valid only while the kernel's source
    file is unchanged (its sha256 prefix is stored with the entry)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    ent = json.load(open(p)).get(f"{name}@{workload}")
    if not ent:
        return None
    src = os.path.join(ROOT, "paper_2409_11998_gb300", "csrc", ent["file"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != ent["file_sha"]:
        return None
    return ent


def hbm_part(byts, ms):
    """Achieved HBM bandwidth of algorithmic bytes in ms, against the measured copy peak."""
    hbm, kind = peaks()
    gbs = byts / (ms / 1e3) / 1e9
    return {"achieved": round(gbs, 2), "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 5),
            "algorithmic_bytes_per_step": int(byts), "peak_source": f"{kind} (MEASURED_PEAKS.json hbm_gbs)"}


def roofline(info, st, nv, nb, nt, precision, n_out=3, workload="starfish"):
    """Roofline of this library's dominant kernel: among the candidates
    below, the one whose stage takes longest in the live step.

    Every candidate carries its HBM fraction ("hbm": algorithmic bytes per
    step -- positions, strengths and the grids written once for the spread;
    the grids read once, the targets read and the outputs written for the
    interpolation; b = 8 bytes per value for FP64 plans, 4 for FP32 -- over
    the live stage time, against the measured copy bandwidth).  The spreads
    and interpolations are instruction-issue bound (2w weight polynomials and
    w^2 cell updates per point, no reuse that HBM could feed), so their
    reported bound is "alu": warp instructions per second -- the kernel's
    instructions per step counted by ncu on this build (profiles/traffic.json,
    matched by source hash) over the live stage time -- against the issue
    peak of one instruction per scheduler per clock.  When no count matches
    the current source, the instructions are estimated from the algorithm
    and marked so.  The FP32 column pass is memory-bound and reported as
    "hbm"."""
    b = 8 if precision == "fp64" else 4
    W, nc = int(info["w"]), int(info["es_nc"])
    levels = [(info["g_nh"], info["K_nh"]), (info["g_fh"], info["K_fh"])]
    levels = [(g, K) for g, K in levels if g > 0]
    nl = len(levels)
    grid_cells = sum(g * g for g, _ in levels)
    vol_ms = st.get("spread_volume", st["spread"])
    df64 = precision == "fp64" and info.get("own_fft") and info.get("precision") == 0
    binned = bool(info.get("binned"))
    spread_bytes = nv * (2 * b + b) + grid_cells * b
    interp_bytes = grid_cells * b * n_out + nt * (2 * 8 + 8 * n_out)
    if df64:
        spread_name = "spread_fx_kernel" if binned else "spread_atomic_kernel"
        # df64 multiply-adds per point and level: 2w (nc - 1) for the weight
        # polynomials, about 15 FP32 instructions each (two-product 4,
        # two-sum 6, two adds, renormalising sum 3); the fixed-point spread
        # then takes about 14 per stencil cell (the strength-scaled product,
        # its two-level quantisation and two shared integer atomics);
        # the interpolation w (w + 1) df64 multiply-adds per channel
        cand = {"spread_volume": (vol_ms, spread_name, spread_bytes,
                                  nv * nl * (2 * W * (nc - 1) * 15 + W * W * 14) / 32),
                "interp": (st["interp"], "interp_dd_kernel", interp_bytes,
                           nt * nl * (2 * W * (nc - 1) + n_out * W * (W + 1)) * 15 / 32)}
    else:
        kp = lambda K: (int(K) + 2) & ~1
        cols_bytes = sum(7 * g * kp(K) * 2 * b for g, K in levels)
        # the single-precision column pass runs two columns per CTA when three
        # columns of the near grid fit in 110 KB of shared memory
        cols_name = "fft_cols2_f32_kernel" if 3 * int(levels[0][0]) * 8 <= 110 * 1024 else "fft_cols_kernel"
        cand = {"spread_volume": (vol_ms, "spread_sub_kernel" if binned else "spread_atomic_kernel", spread_bytes,
                                  nv * nl * (W * W + 2 * W * (nc - 1)) / 32),
                "multiplier": (st["multiplier"], cols_name, cols_bytes, None),
                "interp": (st["interp"], "interp_dd_kernel" if precision == "fp64" else "interp_kernel",
                           interp_bytes, nt * nl * (2 * W * nc + n_out * W * W) / 32)}
    dom = max(cand, key=lambda k: cand[k][0])
    ms, kname, byts, inst_est = cand[dom]
    prof = kernel_profile(kname, workload)
    hbm = hbm_part(byts, ms)
    out = {"kernel": kname, "stage": dom, "launch_ms": round(ms, 4),
           "traffic": prof.get("bytes_per_step") if prof else None,
           "traffic_unit": "DRAM bytes per step (ncu, all launches of the kernel in one step)",
           "hbm_frac": hbm["frac"], "hbm": hbm}
    if inst_est is None:   # memory-bound column pass
        out.update({"bound": "hbm", "achieved": hbm["achieved"], "peak": hbm["peak"], "unit": "GB/s",
                    "frac": hbm["frac"], "peak_source": hbm["peak_source"]})
        return out
    inst = prof.get("inst_per_step") if prof else None
    src = "ncu smsp__inst_executed.sum of this build (profiles/traffic.json)"
    if not inst:
        inst, src = inst_est, "estimate from the algorithm (no ncu count for this source)"
    ach = inst / (ms / 1e3) / 1e12
    peak = issue_peak_t()
    out.update({"bound": "alu", "achieved": round(ach, 4), "peak": round(peak, 4), "unit": "T warp-instructions/s",
                "frac": round(ach / peak, 4), "instructions_per_step": int(inst), "instructions_source": src,
                "peak_source": "152 SMs x 4 schedulers x 1 warp instruction per clock x sm_max_mhz "
                               "(MEASURED_PEAKS.json)"})
    return out


def layer_densities(prob, conv):
    """sigma and mu on the device (None where the workload carries none)."""
    return tuple(None if prob.get(k) is None else conv(prob[k]) for k in ("sigma", "mu"))


def output_buffers(prob, nt, make):
    """V, S, D output buffers; S and D only where the workload has sigma, mu."""
    return [make(), make() if prob.get("sigma") is not None else None,
            make() if prob.get("mu") is not None else None]


def dtype_of(info):
    if info.get("precision") == 1:
        return "f32 (FP64 zero mode)"
    return "df64+f64" if info.get("own_fft") else "f64"


def dtype_detail(info):
    if info.get("precision") == 1:
        return "FP32 arithmetic with FP64 foot search and outputs; tolerance 1e-5"
    if info.get("own_fft"):
        return ("volume spread, transforms, multiplier and interpolation in double-float (FP32 pairs, "
                "~48-bit); boundary spread, local expansions and outputs in FP64")
    return "FP64 throughout"


def levels_arg(args):
    return "auto" if args.levels == "auto" else int(args.levels)


def refine_desc(args):
    return {"refine_levels": args.refine_levels} if args.refine_levels else {}


def run_e2e(args, prob, dev, ev, points):
    """Same metric through the C ABI with HOST (pinned) buffers: every step
    copies the step's sources, densities, targets and jets to the device and
    reads V, S, D back."""
    import numpy as np
    import torch
    import paper_2409_11998_gb300 as lp
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
    h = {k: pin(prob[k]) for k in ("src_xy", "src_w", "src_f", "sigma", "mu", "tgt_xy", "tgt_jet")
         if prob.get(k) is not None}
    nt = len(prob["tgt_xy"])
    houts = output_buffers(prob, nt, lambda: torch.empty(nt, dtype=torch.float64).pin_memory())
    plan = ev.plan
    nv = len(prob["src_w"])

    def step():
        lp.lp_volume(plan, nv, h["src_xy"], h["src_w"], h["src_f"])
        if "sigma" in h:
            lp.lp_single_layer(plan, h["sigma"])
        if "mu" in h:
            lp.lp_double_layer(plan, h["mu"])
        lp.lp_execute(plan, nt, h["tgt_xy"], h["tgt_jet"], houts[0], houts[1], houts[2])
        lp.lp_sync(plan)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    n = max(5, args.steps)
    times = []
    for _ in range(n):
        t0 = time.perf_counter()
        step()                              # ends in lp_sync: the outputs are in host memory
        times.append(time.perf_counter() - t0)
    dt = statistics.median(times)
    h2d = sum(h[k].numel() * 8 for k in h)
    d2h = sum(o is not None for o in houts) * nt * 8
    return {"value": points / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": dt * 1e3, "steps": n,
            "statistic": "median host wall time per step (each step ends in lp_sync)",
            "mean_ms_per_step": statistics.mean(times) * 1e3,
            "api": "lp_volume/lp_single_layer/lp_double_layer/lp_execute/lp_sync on pinned host buffers"}


def run_fp32(args, prob, dev, stream, points, tol=1e-5):
    import numpy as np
    import torch
    import paper_2409_11998_gb300 as lp
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    ev = lp.Evaluator(prob, precision="fp32", tol=tol, stream=stream.cuda_stream, refine_levels=args.refine_levels,
                      levels=levels_arg(args))
    nv, nt = len(prob["src_w"]), len(prob["tgt_xy"])
    sxy, sw, sf, txy, jet = (T(prob[k]) for k in ("src_xy", "src_w", "src_f", "tgt_xy", "tgt_jet"))
    sig, mu = layer_densities(prob, T)
    outs = output_buffers(prob, nt, lambda: torch.empty(nt, dtype=torch.float64, device=dev))
    plan = ev.plan

    def step():
        lp.lp_volume(plan, nv, sxy, sw, sf)
        if sig is not None:
            lp.lp_single_layer(plan, sig)
        if mu is not None:
            lp.lp_double_layer(plan, mu)
        lp.lp_execute(plan, nt, txy, jet, *outs)

    for _ in range(3):
        step()
        lp.lp_sync(plan)
    ms = []
    for _ in range(max(3, args.steps // 2)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        lp.lp_sync(plan)
        ms.append(a.elapsed_time(b))
    st = lp.lp_stage_times(plan)
    info = lp.lp_plan_info(plan)
    roof = roofline(info, st, nv, len(prob["bnd"]["w"]), nt, precision="fp32",
                    n_out=sum(o is not None for o in outs), workload=args.workload)
    ev.close()
    return {"value": points / (statistics.mean(ms) / 1e3), "unit": UNIT, "dtype": "f32 (FP64 zero mode)",
            "tol": tol, "ms_per_step": statistics.mean(ms),
            "grids": {"g_nh": int(info["g_nh"]), "g_fh": int(info["g_fh"]), "w": int(info["w"])},
            "stages_ms": {k: round(v, 4) for k, v in st.items()}, "roofline": roof,
            "_outputs": {k: o.cpu().numpy() for k, o in zip("VSD", outs) if o is not None}}


def run_square(args, dev, stream, steps=10):
    """The 12M-node square (2M jittered triangles, 1M vertex targets, V
    only) at FP64 1e-9 and FP32 1e-5 and 1e-6: device-resident inputs, CUDA events
    around bind + execute, L2 flushed between steps.  The outputs go back
    with the result for the CPU-baseline leg to compare with the oracle."""
    import numpy as np
    import torch
    import paper_2409_11998_gb300 as lp
    from workloads import configs
    prob = configs.square(precision="fp64", tol=1e-9)
    nv, nt = len(prob["src_w"]), len(prob["tgt_xy"])
    nb = len(prob["bnd"]["w"])
    points = nv + nb + nt
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    sxy, sw, sf, txy, jet = (T(prob[k]) for k in ("src_xy", "src_w", "src_f", "tgt_xy", "tgt_jet"))
    out = torch.empty(nt, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {"workload": "[-1,1]^2, 2M jittered triangles (12M nodes), f = 1 + 32 Gaussians, targets = 1,002,001 "
                       "vertices (corners and edges included), V only",
           "points_per_step": points}
    outs = {}
    for key, prec, tol in (("fp64", "fp64", 1e-9), ("fp32", "fp32", 1e-5), ("fp32_tol_1e-6", "fp32", 1e-6)):
        ev = lp.Evaluator(prob, precision=prec, tol=tol, stream=stream.cuda_stream)
        plan = ev.plan

        def step():
            lp.lp_volume(plan, nv, sxy, sw, sf)
            lp.lp_execute(plan, nt, txy, jet, out, None, None)

        for _ in range(3):
            step()
            lp.lp_sync(plan)
        ms = []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                step()
                b.record(stream)
            lp.lp_sync(plan)
            ms.append(a.elapsed_time(b))
        outs[key] = {"V": out.cpu().numpy()}
        res[key] = {"ms_per_step": statistics.mean(ms), "points_per_s": points / (statistics.mean(ms) / 1e3),
                     "tol": tol, "stages_ms": {k: round(v, 4) for k, v in lp.lp_stage_times(plan).items()},
                     "grids": {"g_nh": int(ev.info()["g_nh"]), "g_fh": int(ev.info()["g_fh"]),
                               "w": int(ev.info()["w"])}}
        ev.close()
    del flush
    res["_check"] = (prob, outs)   # compared with the oracle in the CPU-baseline leg
    return res


def oracle_sample(prob, n, rng):
    """n targets: nine tenths drawn uniformly, one tenth from the band near
    the boundary (every k-th target by distance to the nearest boundary
    node, the nearest first), so that the local expansions are sampled too."""
    import numpy as np
    nt = len(prob["tgt_xy"])
    if n >= nt:
        return np.arange(nt)
    n_near = n // 10
    near = np.empty(0, dtype=np.int64)
    if prob.get("bnd") is not None and n_near > 0:
        from scipy.spatial import cKDTree
        d, _ = cKDTree(prob["bnd"]["xy"]).query(prob["tgt_xy"])
        order = np.argsort(d, kind="stable")
        band = order[: max(n_near, int(np.searchsorted(d[order], 12 * np.sqrt(prob["delta"]))))]
        near = band[:: max(1, len(band) // n_near)][:n_near]
    rest = np.setdiff1d(np.arange(nt), near)
    return np.concatenate([near, rng.choice(rest, n - len(near), replace=False)])


def parity(gpu, ref, idx):
    """Relative L2 and max error of GPU results against the oracle on the
    sampled targets, per output."""
    import numpy as np
    out = {}
    for k, want in ref.items():
        if k not in gpu:
            continue
        got = gpu[k][idx]
        out[k] = {"rel_l2": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
                  "rel_max": float(np.max(np.abs(got - want)) / np.max(np.abs(want))),
                  "n_targets": int(len(idx))}
    return out


def cpu_baseline(prob, budget_s=15.0, refine_levels=0, gpu_out=None, checks=None):
    """The oracle as it stands, on the host cores, on a bounded sample of
    targets; extrapolated to the workload's points/s.  The last (largest)
    sample also gives the error of every GPU result of the run against the
    oracle, and `checks` ({name: (problem, {precision: outputs})}) the error
    of other workloads' results on a 2000-target sample each (outside every
    timed region)."""
    import numpy as np
    ncores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(ncores))
    import oracle
    nt = len(prob["tgt_xy"])
    rng = np.random.default_rng(5)
    n = 32
    while True:
        idx = oracle_sample(prob, n, rng)
        t0 = time.perf_counter()
        ref = oracle.evaluate(prob, targets=idx, refine_levels=refine_levels)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or n >= nt:
            break
        n = min(nt, int(n * max(2.0, budget_s / 2 / max(dt, 1e-3))))
    per_target = dt / n
    t_full = per_target * nt
    points = len(prob["src_w"]) + len(prob["bnd"]["w"]) + nt
    par = {prec: parity(out, ref, idx) for prec, out in (gpu_out or {}).items()}
    extra = {}
    for name, (q, outs) in (checks or {}).items():
        qidx = oracle_sample(q, 2000, np.random.default_rng(11))
        qref = oracle.evaluate(q, targets=qidx, want=tuple(next(iter(outs.values())).keys()))
        extra[name] = {prec: parity(o, qref, qidx) for prec, o in outs.items()}
    par["sample"] = (f"{len(idx)} targets: {len(idx) - len(idx) // 10} uniform, {len(idx) // 10} from the "
                     f"boundary band; oracle = direct FP64 sums + the same local expansions")
    return {"value": points / t_full, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", ncores)),
            "kind": "oracle", "sample": f"{n} of {nt} targets (all sources), {dt:.2f} s; "
            f"extrapolated linearly in targets to the full workload ({t_full:.0f} s)", "_parity": par,
            "_checks": extra}


# ---------------------------------------------------------------- batched waves of uneven problems
def run_batch(args, rank, world, local_rank):
    """256 star domains r = 1 + a cos kt (a ~ U[0.1, 0.4], k in 3..9) of
    log-uniform 1k..200k triangles in one wave: one launch per kernel for
    the whole wave, against the same problems one lp_execute at a time."""
    import numpy as np
    import torch
    import paper_2409_11998_gb300 as lp
    from workloads import configs
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    rng = np.random.default_rng(4000)
    sizes = np.exp(rng.uniform(np.log(1000), np.log(200000), args.batch_size)).astype(int)
    probs = [configs.star_batch_member(4000 + i, int(n)) for i, n in enumerate(sizes)]
    points = sum(len(p["src_w"]) + len(p["bnd"]["w"]) + len(p["tgt_xy"]) for p in probs)
    out = {}
    stream = torch.cuda.Stream(device=dev)
    for prec, tol in (("fp64", 1e-9), ("fp32", 1e-5)):
        evs = [lp.Evaluator(p, precision=prec, tol=tol, stream=stream.cuda_stream, levels=levels_arg(args),
                            autotune=args.autotune).bind() for p in probs]
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
        txy = [T(p["tgt_xy"]) for p in probs]
        jet = [T(p["tgt_jet"]) for p in probs]
        o = {k: [torch.empty(len(p["tgt_xy"]), dtype=torch.float64, device=dev) for p in probs] for k in "VSD"}
        b = lp.lp_batch_create(stream.cuda_stream)
        plans = [e.plan for e in evs]
        nts = [len(p["tgt_xy"]) for p in probs]

        def wave():
            lp.lp_batch_execute(b, plans, nts, txy, jet, o["V"], o["S"], o["D"])

        def seq():
            for i, e in enumerate(evs):
                lp.lp_execute(e.plan, nts[i], txy[i], jet[i], o["V"][i], o["S"][i], o["D"][i])

        res = {}
        for name, fn in (("batched", wave), ("one_at_a_time", seq)):
            for _ in range(max(args.warmup, 2)):
                fn()
            torch.cuda.synchronize()
            ms = []
            for _ in range(max(3, args.steps // 5)):
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a_.record(stream)
                fn()
                b_.record(stream)
                torch.cuda.synchronize()
                ms.append(a_.elapsed_time(b_))
            res[name] = {"ms_per_wave": statistics.mean(ms), "points_per_s": points / (statistics.mean(ms) / 1e3)}
        wave()
        torch.cuda.synchronize()
        res["stages_ms"] = {k: round(v, 4) for k, v in lp.lp_batch_stage_times(b).items()}
        res["tol"] = tol
        res["single_level_plans"] = int(sum(e.info()["levels"] == 1 for e in evs))
        res["bin_sides"] = {str(c): int(sum(e.info()["bin_cells"] == c for e in evs))
                            for c in sorted(set(int(e.info()["bin_cells"]) for e in evs))}
        res["dtype"] = dtype_of(evs[0].info())
        out[prec] = res
        lp.lp_batch_destroy(b)
        for e in evs:
            e.close()
    r64 = out["fp64"]
    return {"metric": METRIC, "value": r64["batched"]["points_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": max(3, args.steps // 5), "warmup": max(args.warmup, 2),
            "ms_per_step": r64["batched"]["ms_per_wave"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": r64["dtype"], "data": "synthetic (seeded generators; no dataset)",
            "config": {"workload": f"{len(probs)} star domains r=1+a cos kt, a~U[0.1,0.4], k in 3..9, "
                                   "log-uniform 1k..200k triangles, one wave",
                       "n_problems": len(probs), "points_per_wave": points, "levels": args.levels,
                       "autotune": bool(args.autotune),
                       "triangles_total": int(sum(p["meta"]["n_triangles"] for p in probs))},
            "batch": out}


# ---------------------------------------------------------------- Dirichlet solve
def run_solve(args, rank, world, local_rank):
    """Interior Dirichlet (-mu/2 + D[mu] = g - V[f]) or Neumann (u/2 + D[u] =
    V[f] + S[g]) problem on the starfish (Sec. 5): GMRES at the 16k boundary
    nodes, D applied by the evaluator; one step = one solve to 1e-10 (FP64)
    from 0."""
    import numpy as np
    import torch
    import paper_2409_11998_gb300 as lp
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prob = make_problem("starfish")
    nv, nb = len(prob["src_w"]), len(prob["bnd"]["w"])
    fp64 = args.precision == "fp64"
    tol = 1e-10 if fp64 else 2e-4   # FP32 D stalls GMRES near 1e-4
    stream = torch.cuda.Stream(device=dev)
    ev = lp.Evaluator(prob, precision=args.precision, tol=1e-9 if fp64 else 1e-5, stream=stream.cuda_stream,
                      refine_levels=args.refine_levels, levels=levels_arg(args)).bind()
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    neumann = args.bc == "neumann"
    g, jb = T(prob["neumann_g" if neumann else "dirichlet_g"]), T(prob["bnd_jet"])
    solve = lp.lp_solve_neumann if neumann else lp.lp_solve_dirichlet
    mu = torch.empty(nb, dtype=torch.float64, device=dev)
    launches0 = None
    for k in range(max(args.warmup, 3) + args.steps):
        if k == max(args.warmup, 3):
            torch.cuda.synchronize()
            launches0 = lp.lp_plan_info(ev.plan)["launches"]
            times, its, res = [], [], []
        t0 = time.perf_counter()
        it, r = solve(ev.plan, g, mu, f_jet_b=jb, tol=tol, max_iter=300, restart=40)
        dt = time.perf_counter() - t0      # the call synchronises the plan stream
        if launches0 is not None:
            times.append(dt)
            its.append(it)
            res.append(r)
    launches = lp.lp_plan_info(ev.plan)["launches"] - launches0
    ms = statistics.mean(times) * 1e3
    info = ev.info()
    ev.close()
    return {"metric": METRIC, "value": (nv + nb) / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype_of(info),
            "data": "synthetic (seeded generators; no dataset)",
            "config": {"workload": f"interior {args.bc} solve on the starfish (1.2M volume nodes, 1024x16 "
                                   "boundary nodes): GMRES(40) from 0 to a relative residual "
                                   f"{tol:g}, " + ("g = cos x + sin 2y with its boundary mean removed and "
                                                   "shifted to int f + int g = 0" if neumann else
                                                   "g = cos x + sin 2y"), **refine_desc(args),
                       "levels": int(info["levels"]), "timing": "host wall time per solve (synchronising)"},
            "solve": {"iterations": its[-1], "residual": res[-1], "ms_per_iteration": ms / max(its[-1], 1),
                      "boundary_nodes": nb},
            "gpu_launches": int(launches)}


# ---------------------------------------------------------------- serving a request stream
def run_serve(args, rank, world, local_rank, pool=None, rates=(50, 100, 200, 500, 1000, 2000), seconds=None,
              max_requests=1500):
    """Poisson arrivals of V+S+D requests over a resident mesh pool (12
    meshes, 10k..5M triangles log-uniform on the disk, starfish and square
    domains), FP32 at 1e-5 with continuous batching, against one request at a
    time in FP64 at 1e-9.  Each rate sends arrivals for `seconds` or until
    `max_requests` have arrived, whichever is first, and every request is
    served to completion (latency includes queueing once the server
    saturates)."""
    import torch
    from paper_2409_11998_gb300 import serve
    from workloads import configs
    torch.cuda.set_device(local_rank)
    seconds = args.serve_seconds if seconds is None else seconds
    if pool is None:
        pool = configs.serving_pool()
    pool64 = [dict(p, precision="fp64", tol=1e-9) for p in pool]
    out = {"pool": [{"name": p["name"], "triangles": p["meta"]["n_triangles"],
                     "points": len(p["src_w"]) + len(p["bnd"]["w"]) + len(p["tgt_xy"])} for p in pool],
           "rates": {}}
    srv = serve.Server(pool, precision="fp32", tol=1e-5, n_slots=2, max_wave=32, levels=levels_arg(args))
    one = serve.Server(pool64, precision="fp64", tol=1e-9, one_at_a_time=True, levels=levels_arg(args))
    srv.prewarm()
    one.prewarm()
    srv.run(serve.poisson_arrivals(20, 1.0, len(pool), seed=1))   # warm-up
    one.run(serve.poisson_arrivals(5, 1.0, len(pool), seed=2))
    for lam in rates:
        arr = serve.poisson_arrivals(lam, min(seconds, max_requests / lam), len(pool), seed=int(lam))
        a = serve.latency_stats(srv.run(arr))
        b = serve.latency_stats(one.run(arr))
        out["rates"][str(lam)] = {"batched_fp32": a, "one_at_a_time_fp64": b}
    out["resident_bytes"] = srv.resident
    out["plans_created"] = srv.created
    out["plans_created_while_serving"] = srv.created_in_loop
    out["plans_evicted"] = srv.evicted
    out["arrival_window_s"] = {str(lam): round(min(seconds, max_requests / lam), 3) for lam in rates}
    srv.close()
    one.close()
    return out


# ---------------------------------------------------------------- reference arm
REFERENCE_UNAVAILABLE = {
    "batch": "the oracle evaluates one problem at a time; time it with --workload starfish|disk|square",
    "serve": "a latency workload of the GPU serving layer; the oracle has no request loop",
    "solve": "the oracle's Dirichlet solve is a dense direct solve, infeasible at 16k boundary nodes",
}


def run_reference(args, rank, world):
    import numpy as np
    if rank != 0:
        return None
    if args.workload in REFERENCE_UNAVAILABLE:
        return {"impl": "reference", "unavailable": REFERENCE_UNAVAILABLE[args.workload]}
    ncores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(ncores))
    import oracle
    prob = make_problem(args.workload)
    nt = len(prob["tgt_xy"])
    points = len(prob["src_w"]) + len(prob["bnd"]["w"]) + nt
    rng = np.random.default_rng(7)
    # size each step so that warmup + steps take about two minutes
    per_step = max(0.3, 120.0 / (args.steps + args.warmup))
    n = 16
    t0 = time.perf_counter()
    oracle.evaluate(prob, targets=rng.choice(nt, n, replace=False), refine_levels=args.refine_levels)
    per_target = (time.perf_counter() - t0) / n
    n = int(min(nt, max(8, per_step / max(per_target, 1e-9))))
    for _ in range(args.warmup):
        oracle.evaluate(prob, targets=rng.choice(nt, n, replace=False), refine_levels=args.refine_levels)
    times = []
    for _ in range(args.steps):
        idx = rng.choice(nt, n, replace=False)
        t0 = time.perf_counter()
        oracle.evaluate(prob, targets=idx, refine_levels=args.refine_levels)
        times.append(time.perf_counter() - t0)
    dt = statistics.mean(times)
    t_full = dt / n * nt
    value = points / t_full
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generators; no dataset)",
            "config": {**describe(prob), **refine_desc(args), "parallelism": "host cores (OpenMP over targets)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
                             "kind": "oracle",
                             "sample": f"{n} random targets per step (all {len(prob['src_w'])} sources "
                                       f"and {len(prob['bnd']['w'])} boundary nodes); points/s "
                                       f"extrapolated linearly in targets"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------- distributed helpers
def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "gloo"
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def main():
    args = parse()
    rank, world, local = dist_init()
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    elif args.workload == "batch":
        res = run_batch(args, rank, world, local)
    elif args.workload == "solve":
        res = run_solve(args, rank, world, local)
    elif args.workload == "serve":
        sv = run_serve(args, rank, world, local)
        top = sv["rates"][max(sv["rates"], key=float)]
        res = {"metric": METRIC, "value": top["batched_fp32"]["points_per_s"], "unit": UNIT, "n_gpus": world,
               "steps": None, "warmup": None, "ms_per_step": None, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 zero mode)",
               "data": "synthetic (seeded generators; no dataset)",
               "config": {"workload": "Poisson V+S+D request stream over 12 resident meshes (10k..5M "
                                      "triangles, disk/starfish/square), FP32 tol 1e-5, continuous batching",
                          "seconds_per_rate": args.serve_seconds},
               "served": sv}
    else:
        res = run_lp(args, rank, world, local)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
