"""Concrete seeded workloads.

Each builder returns a *problem* dict:

    name, precision ('fp64'|'fp32'), tol, delta,
    box_lo, box_hi              box containing every source and target
    src_xy[N,2], src_w[N], src_f[N]     volume quadrature nodes, weights, f
    bnd: dict(n_panels, order, xy[NB,2], w[NB], normal[NB,2])
    sigma[NB], mu[NB]           single/double layer densities (may be None)
    tgt_xy[NT,2], tgt_jet[NT,6] targets and the Taylor jet of f there
                                (zero outside the domain)
    meta: dict of generator statistics

Seeds follow  seed = 1000 * config_index + problem_index.  delta defaults to
3 * mean(w) (the paper's delta = 3 dx^2 with dx^2 the mean quadrature weight,
Sec. 6).
"""
from __future__ import annotations

import numpy as np

from . import curves as C
from . import mesh as M
from .fields import GaussianSum, random_smooth_density
from .panels import make_panels, make_square_panels


def _box(*arrays, pad=1e-9):
    pts = np.concatenate([a for a in arrays if a is not None and len(a)])
    lo, hi = pts.min(axis=0), pts.max(axis=0)
    span = float(np.max(hi - lo))
    return (lo - pad * span).tolist(), (hi + pad * span).tolist()


def _finish(name, precision, tol, src_xy, src_w, f, bnd, sigma, mu, tgt_xy, tgt_jet, meta,
            delta=None, box=None):
    if delta is None:
        delta = 3.0 * float(np.mean(src_w))
    if box is None:
        box = _box(src_xy, bnd["xy"] if bnd is not None else None, tgt_xy)
    return {
        "name": name, "precision": precision, "tol": float(tol), "delta": float(delta),
        "box_lo": box[0], "box_hi": box[1],
        "src_xy": np.ascontiguousarray(src_xy, dtype=np.float64),
        "src_w": np.ascontiguousarray(src_w, dtype=np.float64),
        "src_f": np.ascontiguousarray(f, dtype=np.float64),
        "bnd": bnd, "sigma": sigma, "mu": mu,
        "tgt_xy": np.ascontiguousarray(tgt_xy, dtype=np.float64),
        "tgt_jet": np.ascontiguousarray(tgt_jet, dtype=np.float64),
        "meta": meta,
    }


def disk(seed=1000, n_interior=969, n_boundary_vertices=64, n_panels=64, order=16,
         n_exterior=512, precision="fp64", tol=1e-9):
    """Unit disk, ~2,000 random-Delaunay triangles, 6-node rule (~12k nodes),
    f = 3 Gaussians (centres |c| < 0.5, widths U[0.1, 0.3]), 64 x 16 boundary
    nodes, sigma = cos 3t, mu = 1, targets = mesh vertices + 512 points on
    r = 1.5."""
    rng = np.random.default_rng(seed)
    curve = C.Circle(1.0)
    mesh = M.delaunay_mesh(curve, n_interior, n_boundary_vertices, rng)
    xy, w = M.quadrature(mesh, curve)
    r = 0.5 * np.sqrt(rng.random(3))
    th = 2 * np.pi * rng.random(3)
    field = GaussianSum(np.stack([r * np.cos(th), r * np.sin(th)], 1), rng.uniform(0.1, 0.3, 3))
    f = field.value(xy)
    bnd = make_panels(curve, n_panels, order)
    sigma = np.cos(3 * bnd["t"])
    mu = np.ones_like(sigma)
    te = 2 * np.pi * np.arange(n_exterior) / n_exterior
    ext = 1.5 * np.stack([np.cos(te), np.sin(te)], 1)
    tgt = np.concatenate([mesh["P"], ext])
    jet = np.concatenate([field.jet(mesh["P"]), np.zeros((n_exterior, 6))])
    meta = {"n_triangles": int(len(mesh["T"])), "n_vertices": int(len(mesh["P"])),
            "curve": "circle r=1"}
    return _finish("disk", precision, tol, xy, w, f, bnd, sigma, mu, tgt, jet, meta)


def starfish(seed=2000, n_interior=53700, n_boundary_vertices=930, n_panels=1024, order=16,
             precision="fp64", tol=1e-9, nonconforming_frac=0.02, remove_frac=0.01):
    """Starfish r = 1 + 0.3 cos 5t, degraded mesh (~200k triangles, slivers
    with aspect ratio log-uniform in [1, 1e4], 2% non-conforming edges, 1%
    of triangles removed), f = 8 Gaussians (widths 0.02-0.2) +
    sin(6 pi x) cos(4 pi y), 1,024 x 16 boundary nodes with random smooth
    sigma, mu; targets = all quadrature nodes."""
    rng = np.random.default_rng(seed)
    curve = C.Star(0.3, 5)
    base = M.delaunay_mesh(curve, n_interior, n_boundary_vertices, rng)
    mesh = M.degrade(base, rng, nonconforming_frac=nonconforming_frac, remove_frac=remove_frac)
    xy, w = M.quadrature(mesh, curve)
    cen = []
    while len(cen) < 8:
        p = rng.uniform(-1.3, 1.3, size=(1, 2))
        if curve.inside(p)[0]:
            cen.append(p[0])
    field = GaussianSum(np.array(cen), rng.uniform(0.02, 0.2, 8),
                        sincos=(1.0, 6 * np.pi, 4 * np.pi))
    f = field.value(xy)
    bnd = make_panels(curve, n_panels, order)
    sigma = random_smooth_density(bnd["t"], rng)
    mu = random_smooth_density(bnd["t"], rng)
    jet = field.jet(xy)
    meta = {"n_triangles": int(len(mesh["T"])), "n_vertices": int(len(mesh["P"])),
            "curve": "starfish r=1+0.3cos5t", **mesh["stats"]}
    out = _finish("starfish", precision, tol, xy, w, f, bnd, sigma, mu, xy, jet, meta)
    # interior Dirichlet data: g = cos x + sin 2y on the boundary, and the
    # f-jet at the boundary nodes (for V[f] there)
    out["dirichlet_g"] = np.cos(bnd["xy"][:, 0]) + np.sin(2 * bnd["xy"][:, 1])
    out["bnd_jet"] = np.ascontiguousarray(field.jet(bnd["xy"]), dtype=np.float64)
    # interior Neumann data: the same function with its boundary mean removed,
    # shifted so that int f + int g = 0 (compatibility)
    h = out["dirichlet_g"]
    length = float(np.sum(bnd["w"]))
    out["neumann_g"] = h - float(np.sum(bnd["w"] * h)) / length - float(np.sum(w * f)) / length
    return out


def square(seed=3000, n=1000, jitter=0.3, panels_per_side=64, order=16, precision="fp32",
           tol=1e-5, n_gauss=32):
    """[-1,1]^2 with n x n squares split into 2 n^2 triangles (vertex jitter
    0.3 h), f = 1 + 32 Gaussians (widths 0.005-0.1); targets = vertices.
    The boundary carries geometry only (sigma = mu = None)."""
    rng = np.random.default_rng(seed)
    mesh = M.square_mesh(n, rng, jitter=jitter)
    xy, w = M.quadrature(mesh)
    field = GaussianSum(rng.uniform(-0.9, 0.9, size=(n_gauss, 2)), rng.uniform(0.005, 0.1, n_gauss),
                        background=1.0)
    f = field.value(xy)
    bnd = make_square_panels(1.0, panels_per_side, order)
    tgt = mesh["P"]
    jet = field.jet(tgt)
    meta = {"n_triangles": int(len(mesh["T"])), "n_vertices": int(len(mesh["P"])),
            "curve": "square [-1,1]^2 (corners)"}
    return _finish("square", precision, tol, xy, w, f, bnd, None, None, tgt, jet, meta)


def star_batch_member(seed, n_triangles, precision="fp64", tol=1e-9):
    """One problem of the batched workload: star domain r = 1 + a cos kt
    (a ~ U[0.1, 0.4], k in 3..9) at ``n_triangles`` triangles, 8-Gaussian f,
    128-2,048 boundary panels of 16 nodes; targets = all quadrature nodes."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.1, 0.4)
    k = int(rng.integers(3, 10))
    curve = C.Star(a, k)
    n_b = max(24, 8 * k, int(np.sqrt(n_triangles) * 2.5))
    n_int = max(8, (n_triangles - n_b) // 2)
    mesh = M.delaunay_mesh(curve, n_int, n_b, rng)
    xy, w = M.quadrature(mesh, curve)
    # coarse meshes of many-lobed stars can put straight edges across the
    # troughs: drop the nodes that fall outside the curve (a gap in the mesh)
    keep = curve.inside(xy)
    xy, w = xy[keep], w[keep]
    cen = []
    while len(cen) < 8:
        p = rng.uniform(-1 - a, 1 + a, size=(1, 2))
        if curve.inside(p)[0]:
            cen.append(p[0])
    field = GaussianSum(np.array(cen), rng.uniform(0.02, 0.2, 8))
    n_panels = int(np.clip(2 ** np.round(np.log2(max(128, n_b / 4))), 128, 2048))
    bnd = make_panels(curve, n_panels, 16)
    sigma = random_smooth_density(bnd["t"], rng)
    mu = random_smooth_density(bnd["t"], rng)
    meta = {"n_triangles": int(len(mesh["T"])), "a": a, "k": k}
    return _finish(f"star{seed}", precision, tol, xy, w, field.value(xy), bnd, sigma, mu,
                   xy, field.jet(xy), meta)


def circle_layer_problem(n_panels=256, order=16, n_targets=64, delta=1e-4, mode=3,
                         radii=(0.5, 0.9, 0.99, 1.0, 1.01, 1.1, 1.5), seed=0, tol=1e-12):
    """Unit circle with sigma = mu = cos(mode t) and targets on several
    circles (including r = 1 exactly); no volume sources."""
    rng = np.random.default_rng(seed)
    curve = C.Circle(1.0)
    bnd = make_panels(curve, n_panels, order)
    dens = np.cos(mode * bnd["t"])
    th = 2 * np.pi * rng.random(n_targets)
    rr = np.asarray(radii)[rng.integers(0, len(radii), n_targets)]
    tgt = np.stack([rr * np.cos(th), rr * np.sin(th)], 1)
    z = np.zeros((0, 2))
    return _finish("circle-layer", "fp64", tol, z, np.zeros(0), np.zeros(0), bnd, dens, dens.copy(),
                   tgt, np.zeros((n_targets, 6)), {"radii": list(radii)}, delta=delta,
                   box=([-1.6, -1.6], [1.6, 1.6]))


def serving_pool(n_meshes=12, t_min=10_000, t_max=5_000_000, seed=5000, precision="fp32", tol=1e-5,
                 max_delaunay=300_000):
    """Meshes for the serving workload: sizes log-uniform in [t_min, t_max]
    triangles on the disk, starfish and square domains (in turn); sizes above
    max_delaunay use the jittered structured square (fast to generate).
    Every problem carries sigma and mu; targets are the mesh vertices."""
    out = []
    sizes = np.exp(np.linspace(np.log(t_min), np.log(t_max), n_meshes))
    for i, T in enumerate(sizes):
        T = int(T)
        rng = np.random.default_rng(seed + i)
        dom = ("disk", "starfish", "square")[i % 3] if T <= max_delaunay else "square"
        if dom == "square":
            n = max(8, int(np.sqrt(T / 2)))
            mesh = M.square_mesh(n, rng, jitter=0.3)
            xy, w = M.quadrature(mesh)
            bnd = make_square_panels(1.0, max(8, n // 16), 16)
            s = bnd["xy"]
            sigma = 1.0 + 0.5 * np.sin(np.pi * s[:, 0]) * np.cos(np.pi * s[:, 1])
            mu = np.cos(0.5 * np.pi * s[:, 0]) + 0.3 * s[:, 1]
            field = GaussianSum(rng.uniform(-0.9, 0.9, size=(8, 2)), rng.uniform(0.02, 0.2, 8), background=1.0)
        else:
            curve = C.Circle(1.0) if dom == "disk" else C.Star(0.3, 5)
            n_b = max(64, int(np.sqrt(T) * 2.5))
            mesh = M.delaunay_mesh(curve, max(8, (T - n_b) // 2), n_b, rng)
            xy, w = M.quadrature(mesh, curve)
            keep = curve.inside(xy)
            xy, w = xy[keep], w[keep]
            n_pan = int(np.clip(2 ** np.round(np.log2(max(64, n_b / 2))), 64, 4096))
            bnd = make_panels(curve, n_pan, 16)
            sigma = random_smooth_density(bnd["t"], rng)
            mu = random_smooth_density(bnd["t"], rng)
            cen = []
            while len(cen) < 8:
                p = rng.uniform(-1.3, 1.3, size=(1, 2))
                if curve.inside(p)[0]:
                    cen.append(p[0])
            field = GaussianSum(np.array(cen), rng.uniform(0.02, 0.2, 8))
        tgt = mesh["P"]
        if dom != "square":
            tgt = tgt[(curve.inside(tgt)) | (np.arange(len(tgt)) < mesh["nbv"])]
        meta = {"n_triangles": int(len(mesh["T"])), "domain": dom}
        out.append(_finish(f"serve{i}-{dom}", precision, tol, xy, w, field.value(xy), bnd, sigma, mu,
                           tgt, field.jet(tgt), meta))
    return out
