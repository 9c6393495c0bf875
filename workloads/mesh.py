"""Triangulations and their quadrature nodes.

* ``delaunay_mesh``: Delaunay triangulation (scipy/Qhull) of equispaced
  boundary vertices plus uniformly random interior points; triangles whose
  centroid falls outside the curve are dropped.  A triangle whose edge joins
  two consecutive boundary vertices is curved: its edge follows the curve.
* ``degrade``: the paper's robustness recipe (Sec. 6.4) adapted to a target
  mix: interior edges are split at a point whose position along the edge is
  log-uniform, producing slivers with aspect ratios log-uniform in [1, 1e4];
  a chosen fraction of the splits is made non-conforming (the two triangles
  sharing the edge are split at different points, leaving hanging nodes), and
  a fraction of triangles is removed to leave gaps.
* ``square_mesh``: a jittered structured mesh of [-1,1]^2.
* ``quadrature``: maps the 6-node rule onto every triangle; curved triangles
  use the map x(u, v) = v C + (1-v) gamma(tA + (tB - tA) u / (1-v)), which
  follows the curve along the boundary edge AB and is straight elsewhere.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import Delaunay

from .quadrature import triangle_rule6


def _tri_area2(P, T):
    a, b, c = P[T[:, 0]], P[T[:, 1]], P[T[:, 2]]
    return (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])


def delaunay_mesh(curve, n_interior, n_boundary, rng, min_wall_frac=0.5):
    """Random Delaunay mesh of the region inside ``curve``.

    Returns dict(P[nv,2], T[nt,3], curved[nt] bool, tA[nt], tB[nt], nbv)
    where for curved triangles vertices 0,1 are the boundary edge (in
    counter-clockwise order, parameters tA < tB) and vertex 2 is the third.
    The first ``nbv`` rows of P are the boundary vertices."""
    tb = 2 * np.pi * np.arange(n_boundary) / n_boundary
    B = curve.point(tb)
    lo, hi = curve.bbox()
    area_est = np.prod(hi - lo)
    h = np.sqrt(area_est / max(n_interior, 1))
    pts = []
    need = n_interior
    while need > 0:
        cand = lo + (hi - lo) * rng.random((int(need * 2.2) + 16, 2))
        cand = cand[curve.inside(cand)]
        if cand.size:
            # keep interior points away from the wall to avoid needle triangles there
            if hasattr(curve, "wall_distance"):
                d = curve.wall_distance(cand)
            else:
                d = _dist_to_polyline(cand, B)
            cand = cand[d > min_wall_frac * h * 0.5]
        pts.append(cand[:need])
        need -= len(pts[-1])
    I = np.concatenate(pts)[:n_interior]
    P = np.concatenate([B, I])
    T = Delaunay(P).simplices.astype(np.int64)
    cen = P[T].mean(axis=1)
    T = T[curve.inside(cen)]
    ar = _tri_area2(P, T)
    T[ar < 0] = T[ar < 0][:, [0, 2, 1]]
    return _mark_curved(P, T, n_boundary, tb)


def _dist_to_polyline(p, B):
    """Distance from points to the closed polyline through B (coarse check)."""
    A = B
    C = np.roll(B, -1, axis=0)
    d = np.full(len(p), np.inf)
    step = 4096
    for s in range(0, len(A), step):
        a, c = A[s:s + step], C[s:s + step]
        ac = c - a
        L2 = np.maximum((ac ** 2).sum(1), 1e-300)
        ap = p[:, None, :] - a[None, :, :]
        u = np.clip((ap * ac[None]).sum(-1) / L2[None], 0, 1)
        q = a[None] + u[..., None] * ac[None]
        d = np.minimum(d, np.sqrt(((p[:, None, :] - q) ** 2).sum(-1)).min(1))
    return d


def _mark_curved(P, T, nbv, tb):
    nt = len(T)
    curved = np.zeros(nt, dtype=bool)
    tA = np.zeros(nt)
    tB = np.zeros(nt)
    T = T.copy()
    for rot in range(3):
        a, b = T[:, rot].copy(), T[:, (rot + 1) % 3].copy()
        isb = (a < nbv) & (b < nbv) & (((a + 1) % nbv) == b) & ~curved
        if isb.any():
            idx = np.nonzero(isb)[0]
            c = T[idx, (rot + 2) % 3].copy()
            T[idx] = np.stack([a[idx], b[idx], c], axis=1)
            curved[idx] = True
            tA[idx] = tb[a[idx]]
            tB[idx] = np.where(b[idx] == 0, 2 * np.pi, tb[b[idx]])
    return {"P": P, "T": T, "curved": curved, "tA": tA, "tB": tB, "nbv": nbv}


def degrade(mesh, rng, nonconforming_frac=0.02, remove_frac=0.01,
            ar_max=1e4, split_frac=1.0):
    """Split interior edges into slivers (log-uniform aspect ratio in
    [1, ar_max]); make ``nonconforming_frac`` of the mesh's edges carry a
    hanging node; drop ``remove_frac`` of the triangles."""
    P, T, curved = mesh["P"], mesh["T"], mesh["curved"]
    nt = len(T)
    # edges -> up to two triangles
    E = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
    owner = np.tile(np.arange(nt), 3)
    Es = np.sort(E, axis=1)
    key = Es[:, 0] * (len(P) + 1) + Es[:, 1]
    order = np.argsort(key, kind="stable")
    ks = key[order]
    first = np.nonzero(np.r_[True, ks[1:] != ks[:-1]])[0]
    counts = np.diff(np.r_[first, len(ks)])
    n_edges = len(first)
    inner = first[counts == 2]
    pairs = np.stack([owner[order[inner]], owner[order[inner + 1]]], axis=1)
    pairs = pairs[rng.permutation(len(pairs))]
    used = curved.copy()  # curved triangles are never split
    sel = []
    for t1, t2 in pairs:
        if not used[t1] and not used[t2]:
            used[t1] = used[t2] = True
            sel.append((t1, t2))
    sel = np.array(sel, dtype=np.int64).reshape(-1, 2)
    if split_frac < 1.0:
        sel = sel[: int(len(sel) * split_frac)]
    n_nc = min(len(sel), int(round(nonconforming_frac * n_edges)))
    newP = [P]
    nP = len(P)
    keep = np.ones(nt, dtype=bool)
    out_T = []
    # split position s along the shared edge: aspect ratio ~ 1/s, log-uniform
    logs = rng.uniform(0.0, np.log10(ar_max), size=(len(sel), 2))
    for i, (t1, t2) in enumerate(sel):
        tri1 = T[t1]
        tri2 = T[t2]
        shared = np.intersect1d(tri1, tri2)
        u, v = shared[0], shared[1]
        s1 = 0.5 * 10.0 ** (-logs[i, 0]) if rng.random() < 0.5 else 1 - 0.5 * 10.0 ** (-logs[i, 0])
        pts = [P[u] + s1 * (P[v] - P[u])]
        if i < n_nc:
            s2 = 0.5 * 10.0 ** (-logs[i, 1]) if rng.random() < 0.5 else 1 - 0.5 * 10.0 ** (-logs[i, 1])
            pts.append(P[u] + s2 * (P[v] - P[u]))
        ids = list(range(nP, nP + len(pts)))
        newP.append(np.array(pts))
        nP += len(pts)
        for tri, pid in ((tri1, ids[0]), (tri2, ids[-1])):
            opp = [x for x in tri if x != u and x != v][0]
            out_T.append((u, pid, opp))
            out_T.append((pid, v, opp))
        keep[t1] = keep[t2] = False
    P2 = np.concatenate(newP)
    T_new = np.array(out_T, dtype=np.int64).reshape(-1, 3)
    T2 = np.concatenate([T[keep], T_new])
    cur2 = np.concatenate([curved[keep], np.zeros(len(T_new), dtype=bool)])
    tA2 = np.concatenate([mesh["tA"][keep], np.zeros(len(T_new))])
    tB2 = np.concatenate([mesh["tB"][keep], np.zeros(len(T_new))])
    ar = _tri_area2(P2, T2)
    flip = (ar < 0) & ~cur2
    T2[flip] = T2[flip][:, [0, 2, 1]]
    drop = rng.random(len(T2)) < remove_frac
    stats = {"n_split_pairs": int(len(sel)), "n_nonconforming_edges": int(n_nc),
             "n_edges_before": int(n_edges), "n_removed": int(drop.sum())}
    return {"P": P2, "T": T2[~drop], "curved": cur2[~drop], "tA": tA2[~drop],
            "tB": tB2[~drop], "nbv": mesh["nbv"], "stats": stats}


def square_mesh(n, rng, jitter=0.3, half=1.0):
    """(n x n) squares on [-half, half]^2, each split into two triangles,
    interior vertices jittered by U(-jitter*h, jitter*h) per coordinate."""
    h = 2 * half / n
    g = np.linspace(-half, half, n + 1)
    X, Y = np.meshgrid(g, g, indexing="xy")
    P = np.stack([X.ravel(), Y.ravel()], axis=1)
    ix = np.tile(np.arange(n + 1), n + 1)
    iy = np.repeat(np.arange(n + 1), n + 1)
    interior = (ix > 0) & (ix < n) & (iy > 0) & (iy < n)
    P[interior] += rng.uniform(-jitter * h, jitter * h, size=(interior.sum(), 2))
    i = np.arange(n)
    I, J = np.meshgrid(i, i, indexing="xy")
    v00 = (J * (n + 1) + I).ravel()
    v10, v01, v11 = v00 + 1, v00 + n + 1, v00 + n + 2
    alt = ((I + J) % 2 == 0).ravel()
    T1 = np.where(alt[:, None], np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
    T2 = np.where(alt[:, None], np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
    T = np.concatenate([T1, T2])
    nt = len(T)
    return {"P": P, "T": T, "curved": np.zeros(nt, dtype=bool), "tA": np.zeros(nt),
            "tB": np.zeros(nt), "nbv": 0}


def quadrature(mesh, curve=None):
    """6 nodes per triangle; returns (xy[N,2], w[N])."""
    bary, wr = triangle_rule6()
    P, T = mesh["P"], mesh["T"]
    A, B, C = P[T[:, 0]], P[T[:, 1]], P[T[:, 2]]
    # straight map
    xy = np.einsum("qk,tkd->tqd", bary, np.stack([A, B, C], axis=1))
    det = np.abs((B[:, 0] - A[:, 0]) * (C[:, 1] - A[:, 1]) - (B[:, 1] - A[:, 1]) * (C[:, 0] - A[:, 0]))
    w = 0.5 * det[:, None] * wr[None, :]
    cur = mesh["curved"]
    if curve is not None and cur.any():
        idx = np.nonzero(cur)[0]
        tA, tB = mesh["tA"][idx], mesh["tB"][idx]
        Cc = C[idx]
        u = bary[:, 1][None, :]
        v = bary[:, 2][None, :]
        s = u / (1.0 - v)
        dt = (tB - tA)[:, None]
        tau = tA[:, None] + dt * s
        g0 = curve.deriv(tau.ravel(), 0).reshape(len(idx), 6, 2)
        g1 = curve.deriv(tau.ravel(), 1).reshape(len(idx), 6, 2)
        x = v[..., None] * Cc[:, None, :] + (1.0 - v)[..., None] * g0
        du = dt[..., None] * g1
        dv = Cc[:, None, :] - g0 + (dt * s)[..., None] * g1
        J = np.abs(du[..., 0] * dv[..., 1] - du[..., 1] * dv[..., 0])
        xy[idx] = x
        w[idx] = 0.5 * J * wr[None, :]
    return np.ascontiguousarray(xy.reshape(-1, 2)), np.ascontiguousarray(w.reshape(-1))
