"""Source sharding on the CPU: the partition and reduction logic of
paper_2409_11998_gb300/shard.py run by two gloo ranks against a stand-in of
the library whose spread is linear in the sources (every node adds its
strength to a cell of a small grid) and whose finish reads the summed grids
at the targets.  Two ranks must reproduce one rank's result; the layers must
be counted once; every target belongs to exactly one rank."""
import json
import os
import socket
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, json
sys.path.insert(0, {root!r})
sys.path.insert(0, os.path.join({root!r}, "tests"))
import numpy as np
import torch
import torch.distributed as dist
from paper_2409_11998_gb300 import shard
from test_shard_cpu import FakeLib, problem
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
p = problem()
lib = FakeLib()
plan = lib.new_plan()
ev = shard.ShardedEvaluation(lib, plan, p, rank, world, view=lambda t, n, d: t).bind()
lo, hi = ev.tgt
out = {{k: np.zeros(hi - lo) for k in "VSD"}}
ev.evaluate(out)
print(json.dumps({{"rank": rank, "lo": lo, "hi": hi, "spread_layers": lib.layer_spreads,
                  "bound": lib.bound, **{{k: out[k].tolist() for k in "VSD"}}}}))
dist.destroy_process_group()
"""


def problem():
    rng = np.random.default_rng(77)
    n, nb, nt = 503, 64, 97
    return {"src_xy": rng.uniform(-1, 1, (n, 2)), "src_w": rng.uniform(0.1, 1, n), "src_f": rng.normal(size=n),
            "sigma": rng.normal(size=nb), "mu": rng.normal(size=nb), "tgt_xy": rng.uniform(-1, 1, (nt, 2)),
            "tgt_jet": rng.normal(size=(nt, 6)), "bnd_xy": rng.uniform(-1, 1, (nb, 2))}


class FakeLib:
    """Linear spread onto an 8 x 8 grid per channel, with the zero-mode sums;
    finish = the summed grid at each target's cell, plus the sums, plus a
    local term from the jet.  Grids are torch CPU tensors, reduced in place."""
    G = 8

    def __init__(self):
        self.layer_spreads = 0
        self.bound = 0

    def new_plan(self):
        import torch
        return {"grid": {k: torch.zeros(self.G * self.G, dtype=torch.float64) for k in "VSD"},
                "qred": torch.zeros(2, dtype=torch.float64)}

    def _cell(self, xy):
        c = np.clip(((np.asarray(xy) + 1) / 2 * self.G).astype(int), 0, self.G - 1)
        return c[:, 1] * self.G + c[:, 0]

    def lp_volume(self, plan, n, xy, w, f):
        plan["vol"] = (np.asarray(xy), np.asarray(w) * np.asarray(f))
        self.bound = int(n)

    def lp_single_layer(self, plan, s):
        plan["sigma"] = np.asarray(s)

    def lp_double_layer(self, plan, m):
        plan["mu"] = np.asarray(m)

    def lp_spread(self, plan, outputs, spread_layers):
        import torch
        for g in plan["grid"].values():
            g.zero_()
        xy, q = plan["vol"]
        np.add.at(plan["grid"]["V"].numpy(), self._cell(xy), q)
        plan["qred"].zero_()
        plan["qred"][0] = float(np.sum(q))
        if spread_layers:
            self.layer_spreads += 1
            b = problem()["bnd_xy"]
            np.add.at(plan["grid"]["S"].numpy(), self._cell(b), plan["sigma"])
            np.add.at(plan["grid"]["D"].numpy(), self._cell(b), plan["mu"])
            plan["qred"][1] = float(np.sum(plan["sigma"]))
        plan["outputs"] = outputs

    def lp_grid_buffers(self, plan):
        return [(plan["grid"][k], None, "float64") for k in plan["outputs"]] + [(plan["qred"], None, "float64")]

    def lp_finish(self, plan, n, txy, jet, V, S, D):
        c = self._cell(txy)
        for k, out in zip("VSD", (V, S, D)):
            if out is not None:
                out[:] = plan["grid"][k].numpy()[c] + 0.5 * plan["qred"][0].item() + 1e-3 * np.asarray(jet)[:, 0]
        if S is not None:
            S += 0.25 * plan["qred"][1].item()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_share_partitions_exactly():
    from paper_2409_11998_gb300 import shard
    for n in (0, 1, 7, 503, 1000):
        for world in (1, 2, 3, 8):
            parts = [shard.share(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1


def test_two_gloo_ranks_match_one_rank():
    from paper_2409_11998_gb300 import shard
    p = problem()
    lib = FakeLib()
    plan = lib.new_plan()
    ev = shard.ShardedEvaluation(lib, plan, p, 0, 1, allreduce=lambda t: None, view=lambda t, n, d: t).bind()
    ref = {k: np.zeros(len(p["tgt_xy"])) for k in "VSD"}
    ev.evaluate(ref)
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [q.communicate(timeout=180) for q in procs]
    for q, (o, e) in zip(procs, outs):
        assert q.returncode == 0, e[-3000:]
    res = sorted((json.loads(o.strip().splitlines()[-1]) for o, _ in outs), key=lambda d: d["rank"])
    assert [d["spread_layers"] for d in res] == [1, 0]          # the layers are spread once
    assert sum(d["bound"] for d in res) == len(p["src_w"])       # every node on exactly one rank
    assert res[0]["lo"] == 0 and res[0]["hi"] == res[1]["lo"] and res[1]["hi"] == len(p["tgt_xy"])
    for k in "VSD":
        got = np.concatenate([d[k] for d in res])
        assert np.allclose(got, ref[k], rtol=1e-13, atol=1e-13), k
