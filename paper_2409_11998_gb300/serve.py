"""Continuous-batching evaluation server on one GPU.

Requests ask for V, S and D on one mesh of a resident pool with their own
densities (the mesh's f, sigma, mu scaled per request).  The server keeps
one plan (grids, tables, boundary structures) resident per mesh and stream
slot, created before serving starts (prewarm) while the device footprint of
resident plans stays under a budget.  Whenever a slot is free it forms a wave
from the waiting requests in arrival order, at most one request per mesh (a
plan holds one set of densities; a second request for the same mesh waits for
the next wave or the other slot), runs the wave as one lp_batch_execute on
the slot's stream -- waves on different slots overlap on the device -- and
records per-request latency from arrival to observed completion.  A plan is
created inside the request loop only when its mesh had no resident plan (it
was never admitted, or was evicted, least recently used first, to make room);
``created_in_loop`` counts those.

``one_at_a_time=True`` gives the reference serving path: one stream, one
request per call, lp_execute, in arrival order.

A client may stop waiting (it timed out, or its process died): an arrival
can carry the time at which its client abandons the request.  A request
abandoned while it waits is dropped without being launched; one abandoned
while its wave is on the GPU completes with the wave (kernels in flight are
never interrupted) and its outputs are dropped; either way its plan is
released as usual, and latency statistics count it apart.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import (lp_batch_create, lp_batch_destroy, lp_batch_execute, lp_destroy, lp_double_layer,
               lp_execute, lp_plan, lp_plan_info, lp_single_layer, lp_sync, lp_volume, LP_FP32, LP_FP64)


@dataclasses.dataclass
class Request:
    rid: int
    mesh: int
    arrival: float          # seconds from the start of the run
    scale: float            # density scaling of this request
    t_launch: float = -1.0
    t_done: float = -1.0
    points: int = 0
    outputs: dict | None = None
    abandon: float = float("inf")  # seconds from the start at which the client stops waiting
    abandoned: bool = False


def poisson_arrivals(rate, duration, n_meshes, seed=0, mesh_weights=None):
    """Arrival times of a Poisson process of the given rate over [0, duration),
    each request on a mesh drawn with the given weights (uniform by default)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    p = None if mesh_weights is None else np.asarray(mesh_weights) / np.sum(mesh_weights)
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        out.append((t, int(rng.choice(n_meshes, p=p)), float(rng.uniform(0.5, 1.5))))
    return out


def latency_stats(reqs):
    """p50/p99/mean latency and served points/s of the completed requests;
    abandoned requests are counted apart."""
    n_abandoned = sum(1 for r in reqs if r.abandoned)
    reqs = [r for r in reqs if not r.abandoned]
    lat = np.array([r.t_done - r.arrival for r in reqs])
    if lat.size == 0:
        return {"requests": 0, "abandoned": n_abandoned} if n_abandoned else {}
    span = max(r.t_done for r in reqs) - min(r.arrival for r in reqs)
    pts = sum(r.points for r in reqs)
    return {"requests": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "points_per_s": float(pts / span) if span > 0 else None, "span_s": float(span),
            **({"abandoned": n_abandoned} if n_abandoned else {})}


class _Mesh:
    def __init__(self, prob, torch, device):
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=device)
        b = prob["bnd"]
        self.prob = prob
        self.xy, self.w, self.f = T(prob["src_xy"]), T(prob["src_w"]), T(prob["src_f"])
        self.bxy, self.bw, self.bn = T(b["xy"]), T(b["w"]), T(b["normal"])
        self.sigma, self.mu = T(prob["sigma"]), T(prob["mu"])
        self.txy, self.jet = T(prob["tgt_xy"]), T(prob["tgt_jet"])
        self.points = len(prob["src_w"]) + len(b["w"]) + len(prob["tgt_xy"])


class _PlanInst:
    def __init__(self, handle, nbytes):
        self.h = handle
        self.bytes = nbytes
        self.busy = False
        self.last = 0.0


class Server:
    def __init__(self, pool, precision="fp32", tol=1e-5, n_slots=2, max_wave=32,
                 mem_budget=64 << 30, one_at_a_time=False, keep_outputs=False, device="cuda", levels="auto",
                 torch_module=None):
        # torch_module: a stand-in for the few torch stream, event and tensor
        # calls the loop makes, for exercising the scheduling without a GPU
        if torch_module is None:
            import torch as torch_module
        torch = torch_module
        self.torch = torch
        self.device = device
        self.prec = LP_FP32 if precision == "fp32" else LP_FP64
        self.tol = tol
        self.levels = levels              # history levels of every plan (lp_domain.levels)
        self.one = one_at_a_time
        self.max_wave = 1 if one_at_a_time else max_wave
        self.keep = keep_outputs
        self.budget = mem_budget
        self.meshes = [_Mesh(p, torch, device) for p in pool]
        n_slots = 1 if one_at_a_time else n_slots
        self.slots = []
        for _ in range(n_slots):
            st = torch.cuda.Stream(device=device)
            self.slots.append({"stream": st, "batch": None if one_at_a_time else lp_batch_create(st.cuda_stream),
                               "event": torch.cuda.Event(), "busy": False, "reqs": [], "insts": []})
        self.pools = collections.defaultdict(list)  # (slot, mesh) -> [_PlanInst]
        self.resident = 0
        self.created = 0
        self.created_in_loop = 0
        self.evicted = 0
        self.scan = 4 * self.max_wave    # waiting requests examined per wave

    # ---- plans ----
    def _new_plan(self, slot, mid):
        m = self.meshes[mid]
        p = m.prob
        b = p["bnd"]
        h = lp_plan(p["box_lo"], p["box_hi"], p["delta"], self.tol, precision=self.prec,
                    n_panels=b["n_panels"], panel_order=b["order"], bnd_xy=m.bxy, bnd_w=m.bw,
                    bnd_normal=m.bn, stream=self.slots[slot]["stream"].cuda_stream, levels=self.levels)
        inst = _PlanInst(h, int(lp_plan_info(h)["device_bytes"]))
        self.pools[(slot, mid)].append(inst)
        self.resident += inst.bytes
        self.created += 1
        return inst

    def _evict_for(self, need):
        idle = [(inst.last, key, inst) for key, lst in self.pools.items() for inst in lst if not inst.busy]
        idle.sort(key=lambda x: x[0])
        for _, key, inst in idle:
            if self.resident + need <= self.budget:
                break
            lp_sync(inst.h)
            lp_destroy(inst.h)
            self.pools[key].remove(inst)
            self.resident -= inst.bytes
            self.evicted += 1
        return self.resident + need <= self.budget

    def _acquire(self, slot, mid):
        """The idle resident plan of this mesh on this slot; if the mesh has
        none on this slot, a new one when the footprint budget allows
        (evicting idle plans first); None if its plan is busy or there is no
        room."""
        lst = self.pools[(slot, mid)]
        for inst in lst:
            if not inst.busy:
                inst.busy = True
                return inst
        if lst:
            return None                     # busy: the request waits for the next wave
        est = max([i.bytes for (s, m), l in self.pools.items() if m == mid for i in l] or [0])
        if not self._evict_for(est):
            return None
        inst = self._new_plan(slot, mid)
        self.created_in_loop += 1
        if self.resident > self.budget:
            self._evict_for(0)
        inst.busy = True
        return inst

    def prewarm(self):
        """Create one resident plan per (slot, mesh) while the budget allows."""
        for s in range(len(self.slots)):
            for mid in range(len(self.meshes)):
                if not self.pools[(s, mid)]:
                    self._new_plan(s, mid)
                    if self.resident > self.budget:
                        self._evict_for(0)
        self.torch.cuda.synchronize()

    # ---- waves ----
    def _launch(self, si, wave, now):
        torch = self.torch
        slot = self.slots[si]
        with torch.cuda.stream(slot["stream"]):
            plans, nts, txy, jets = [], [], [], []
            outs = {"V": [], "S": [], "D": []}
            for r, inst in wave:
                m = self.meshes[r.mesh]
                f = m.f * r.scale
                sig = m.sigma * r.scale
                mu = m.mu * r.scale
                jet = m.jet * r.scale
                lp_volume(inst.h, len(m.w), m.xy, m.w, f)
                lp_single_layer(inst.h, sig)
                lp_double_layer(inst.h, mu)
                o = {k: torch.empty(len(m.txy), dtype=torch.float64, device=self.device) for k in "VSD"}
                r.outputs = o
                r.points = m.points
                r.t_launch = now
                r._keep = (f, sig, mu, jet)
                plans.append(inst.h)
                nts.append(len(m.txy))
                txy.append(m.txy)
                jets.append(jet)
                for k in "VSD":
                    outs[k].append(o[k])
                if self.one:
                    lp_execute(inst.h, len(m.txy), m.txy, jet, o["V"], o["S"], o["D"])
            if not self.one:
                lp_batch_execute(slot["batch"], plans, nts, txy, jets, outs["V"], outs["S"], outs["D"])
            slot["event"].record(slot["stream"])
        slot["busy"] = True
        slot["reqs"] = [r for r, _ in wave]
        slot["insts"] = [i for _, i in wave]

    def _finish(self, si, now):
        slot = self.slots[si]
        for r in slot["reqs"]:
            r.t_done = now
            r._keep = None
            if r.abandon <= now:            # the client left while the wave ran
                r.abandoned = True
            if not self.keep or r.abandoned:
                r.outputs = None
        for inst in slot["insts"]:
            inst.busy = False
            inst.last = now
        slot["busy"] = False
        slot["reqs"], slot["insts"] = [], []

    def run(self, arrivals, poll_s=5e-5):
        """Serve the (time, mesh, scale[, abandon]) arrivals in real time;
        returns the requests with their launch and completion times (abandon:
        the time at which the client stops waiting; none by default)."""
        reqs = [Request(i, a[1], a[0], a[2], abandon=a[3] if len(a) > 3 else float("inf"))
                for i, a in enumerate(sorted(arrivals, key=lambda a: a[0]))]
        queue = collections.deque()
        nxt = 0
        done = 0
        t0 = time.perf_counter()
        while done < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                queue.append(reqs[nxt])
                nxt += 1
            if any(r.abandon <= now for r in queue):
                # clients that stopped waiting: their requests are never launched
                left = [r for r in queue if r.abandon <= now]
                for r in left:
                    r.abandoned = True
                    r.t_done = now
                queue = collections.deque(r for r in queue if r.abandon > now)
                done += len(left)
            progressed = False
            for si, slot in enumerate(self.slots):
                if slot["busy"] and slot["event"].query():
                    done += len(slot["reqs"])
                    self._finish(si, time.perf_counter() - t0)
                    progressed = True
            for si, slot in enumerate(self.slots):
                if slot["busy"] or not queue:
                    continue
                # the oldest waiting requests, at most one per mesh; the rest
                # keep their places in the queue
                wave, kept, meshes = [], [], set()
                while queue and len(wave) < self.max_wave and len(wave) + len(kept) < self.scan:
                    r = queue.popleft()
                    inst = None if r.mesh in meshes else self._acquire(si, r.mesh)
                    if inst is None:
                        kept.append(r)
                        continue
                    meshes.add(r.mesh)
                    wave.append((r, inst))
                for r in reversed(kept):
                    queue.appendleft(r)
                if wave:
                    self._launch(si, wave, time.perf_counter() - t0)
                    progressed = True
            if not progressed:
                if nxt < len(reqs) and not queue and not any(s["busy"] for s in self.slots):
                    wait = reqs[nxt].arrival - (time.perf_counter() - t0)
                    if wait > 2e-3:
                        time.sleep(wait - 1e-3)
                        continue
                time.sleep(poll_s)
        return reqs

    def close(self):
        self.torch.cuda.synchronize()
        for slot in self.slots:
            if slot["batch"] is not None:
                lp_batch_destroy(slot["batch"])
        for lst in self.pools.values():
            for inst in lst:
                lp_destroy(inst.h)
        self.pools.clear()
        self.resident = 0
