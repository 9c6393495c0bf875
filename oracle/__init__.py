"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
the arithmetic lives in ``oracle.cpp`` (plain double-precision loops with
OpenMP over targets), compiled here with g++.

``evaluate(problem)`` returns V, S, D at the problem's targets as the sum of
  * the smooth part: direct O(N * N_t) sums of the smoothed kernel
    G_H[delta](r) = -ln r/(2 pi) - E1(r^2/(4 delta))/(4 pi)   (Sec. 2,
    eq. splitting2) and of its source-point normal derivative, and
  * the local part: the asymptotic expansions of Sec. 4 after a closest-point
    search on the boundary panels.
This is the quantity the NUFFT pipeline approximates to its tolerance.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force=False):
    """Compile oracle.cpp -> _build/liboracle.so (g++, OpenMP, -O2)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    tmp = _OUT + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i64, vp, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
        _lib.oracle_e1.restype = d
        _lib.oracle_e1.argtypes = [d]
        _lib.oracle_ein.restype = d
        _lib.oracle_ein.argtypes = [d]
        _lib.oracle_green_smooth.restype = d
        _lib.oracle_green_smooth.argtypes = [d, d]
        _lib.oracle_smooth_charge.argtypes = [i64, vp, vp, i64, vp, d, vp]
        _lib.oracle_smooth_dipole.argtypes = [i64, vp, vp, vp, i64, vp, d, vp]
        _lib.oracle_gl_nodes.argtypes = [i32, vp]
        _lib.oracle_gl_weights.argtypes = [i32, vp, vp]
        _lib.oracle_local_dyadic.restype = i32
        _lib.oracle_local_dyadic.argtypes = [i32, i32, vp, vp, vp, i64, vp, d, i32, d, i32, i32, vp, vp]
        _lib.oracle_local.restype = i32
        _lib.oracle_local.argtypes = [i32, i32, vp, vp, vp, i64, vp, vp, d, i32, d, vp, vp, vp, vp]
        _lib.oracle_frame.argtypes = [i32, i32, vp, vp, vp, i32, d, vp]
        _lib.oracle_local_formulas.argtypes = [vp, vp, d, i32, vp]
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def e1(z):
    return lib().oracle_e1(float(z))


def ein(z):
    return lib().oracle_ein(float(z))


def green_smooth(r, delta):
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    return np.array([lib().oracle_green_smooth(float(x * x), float(delta)) for x in r])


def gl_nodes(p):
    x = np.zeros(p)
    lib().oracle_gl_nodes(int(p), _p(x))
    return x


def smooth_charge(src_xy, q, tgt_xy, delta):
    src_xy, q, tgt_xy = _c(src_xy), _c(q), _c(tgt_xy)
    out = np.zeros(len(tgt_xy))
    lib().oracle_smooth_charge(len(src_xy), _p(src_xy), _p(q), len(tgt_xy), _p(tgt_xy),
                               float(delta), _p(out))
    return out


def smooth_dipole(src_xy, normal, m, tgt_xy, delta):
    src_xy, normal, m, tgt_xy = _c(src_xy), _c(normal), _c(m), _c(tgt_xy)
    out = np.zeros(len(tgt_xy))
    lib().oracle_smooth_dipole(len(src_xy), _p(src_xy), _p(normal), _p(m), len(tgt_xy),
                               _p(tgt_xy), float(delta), _p(out))
    return out


def local(bnd, sigma, mu, tgt_xy, jet, delta, order=5, on_tol=1e-12):
    """Local part per target: returns (VL, SL, DL, info[nt,4], status)."""
    bxy = _c(bnd["xy"]) if bnd is not None else np.zeros((0, 2))
    npan = bnd["n_panels"] if bnd is not None else 0
    p = bnd["order"] if bnd is not None else 0
    tgt_xy = _c(tgt_xy)
    nt = len(tgt_xy)
    sigma, mu, jet = _c(sigma), _c(mu), _c(jet)
    VL = np.zeros(nt) if jet is not None else None
    SL = np.zeros(nt) if sigma is not None else None
    DL = np.zeros(nt) if mu is not None else None
    info = np.zeros((nt, 4))
    st = lib().oracle_local(int(npan), int(p), _p(bxy), _p(sigma), _p(mu), nt, _p(tgt_xy),
                            _p(jet), float(delta), int(order), float(on_tol), _p(VL), _p(SL),
                            _p(DL), _p(info))
    return VL, SL, DL, info, st


def local_dyadic(bnd, sigma, mu, tgt_xy, delta, levels, order=5, on_tol=1e-12, m0=2):
    """Local layer potentials with `levels` steps of dyadic refinement
    (Sec. 4.4): the expansions at delta / 4^levels plus direct sums of the
    difference kernels on panels split into m0 2^(j-1) intervals at level j.
    Returns (SL, DL); either is None when its density is None."""
    bxy = _c(bnd["xy"])
    tgt_xy = _c(tgt_xy)
    nt = len(tgt_xy)
    sigma, mu = _c(sigma), _c(mu)
    SL = np.zeros(nt) if sigma is not None else None
    DL = np.zeros(nt) if mu is not None else None
    lib().oracle_local_dyadic(int(bnd["n_panels"]), int(bnd["order"]), _p(bxy), _p(sigma), _p(mu), nt,
                              _p(tgt_xy), float(delta), int(order), float(on_tol), int(levels), int(m0),
                              _p(SL), _p(DL))
    return SL, DL


def gl_weights(p):
    x = gl_nodes(p)
    w = np.zeros(p)
    lib().oracle_gl_weights(int(p), _p(x), _p(w))
    return w


def frame(bnd, sigma, mu, panel, t):
    out = np.zeros(14)
    lib().oracle_frame(bnd["n_panels"], bnd["order"], _p(_c(bnd["xy"])), _p(_c(sigma)),
                       _p(_c(mu)), int(panel), float(t), _p(out))
    keys = ["kappa", "g3", "g4", "s0", "s1", "s2", "m0", "m1", "m2", "m4", "Tx", "Ty", "bx", "by"]
    return dict(zip(keys, out))


def local_formulas(geom, jet6, delta, order=5):
    """geom = dict(r, sgn, kappa, g3, g4, s0, s1, s2, m0, m1, m2, m4, Tx, Ty)."""
    keys = ["r", "sgn", "kappa", "g3", "g4", "s0", "s1", "s2", "m0", "m1", "m2", "m4", "Tx", "Ty"]
    g = np.array([float(geom.get(k, 0.0)) for k in keys])
    j = _c(jet6 if jet6 is not None else np.zeros(6))
    out = np.zeros(3)
    lib().oracle_local_formulas(_p(g), _p(j), float(delta), int(order), _p(out))
    return {"V": out[0], "S": out[1], "D": out[2]}


def on_tolerance(problem):
    side = max(problem["box_hi"][0] - problem["box_lo"][0], problem["box_hi"][1] - problem["box_lo"][1])
    return 1e-12 * side


def evaluate(problem, targets=None, order=5, want=("V", "S", "D"), refine_levels=0):
    """V, S, D at the problem's targets (or at the given subset of target
    indices).  Returns a dict with totals and their smooth/local parts.
    With refine_levels > 0 the local parts of S and D are the dyadically
    refined ones (Sec. 4.4); V keeps its plain local part."""
    delta = problem["delta"]
    idx = np.arange(len(problem["tgt_xy"])) if targets is None else np.asarray(targets)
    txy = problem["tgt_xy"][idx]
    jet = problem["tgt_jet"][idx] if "V" in want else None
    bnd = problem["bnd"]
    sigma = problem["sigma"] if "S" in want else None
    mu = problem["mu"] if "D" in want else None
    out = {}
    if "V" in want:
        q = problem["src_f"] * problem["src_w"]
        out["VH"] = smooth_charge(problem["src_xy"], q, txy, delta) if len(q) else np.zeros(len(txy))
    if sigma is not None:
        out["SH"] = smooth_charge(bnd["xy"], sigma * bnd["w"], txy, delta)
    if mu is not None:
        out["DH"] = smooth_dipole(bnd["xy"], bnd["normal"], mu * bnd["w"], txy, delta)
    VL, SL, DL, info, st = local(bnd, sigma, mu, txy, jet, delta, order, on_tolerance(problem))
    if refine_levels > 0 and (sigma is not None or mu is not None):
        SL, DL = local_dyadic(bnd, sigma, mu, txy, delta, refine_levels, order=order,
                              on_tol=on_tolerance(problem))
    if "V" in want:
        out["VL"] = VL
        out["V"] = out["VH"] + VL
    if sigma is not None:
        out["SL"] = SL
        out["S"] = out["SH"] + SL
    if mu is not None:
        out["DL"] = DL
        out["D"] = out["DH"] + DL
    out["info"] = info
    out["status"] = st
    return out


def dirichlet_matrix(bnd, delta, order=5, on_tol=1e-12, refine_levels=0):
    """The discrete operator of the interior Dirichlet equation (Sec. 5,
    eq. dir_inteq) at the boundary nodes: A = -I/2 + D, with column j the
    double layer of the unit nodal density e_j evaluated at every boundary
    node (on-surface targets): smooth part by direct sums, local part by the
    on-surface expansions (with dyadic refinement when refine_levels > 0).
    Dense, built column by column -- for small boundaries only."""
    xy, nrm, w = bnd["xy"], bnd["normal"], bnd["w"]
    nb = len(xy)
    A = np.empty((nb, nb))
    for j in range(nb):
        e = np.zeros(nb)
        e[j] = 1.0
        DH = smooth_dipole(xy, nrm, e * w, xy, delta)
        if refine_levels > 0:
            _, DL = local_dyadic(bnd, None, e, xy, delta, refine_levels, order=order, on_tol=on_tol)
        else:
            _, _, DL, _, _ = local(bnd, None, e, xy, None, delta, order, on_tol)
        A[:, j] = DH + DL
    A[np.diag_indices(nb)] -= 0.5
    return A


def solve_dirichlet(bnd, g, delta, order=5, on_tol=1e-12, v_boundary=None, refine_levels=0):
    """mu solving -mu/2 + D[mu] = g - V[f] at the boundary nodes (Sec. 5,
    eq. dir_inteq) by a dense direct solve of dirichlet_matrix; v_boundary is
    V[f] at the boundary nodes (None: f = 0)."""
    A = dirichlet_matrix(bnd, delta, order, on_tol, refine_levels)
    rhs = np.asarray(g, dtype=np.float64) - (0.0 if v_boundary is None else np.asarray(v_boundary))
    return np.linalg.solve(A, rhs)


def solve_neumann(bnd, g, delta, order=5, on_tol=1e-12, v_boundary=None, refine_levels=0):
    """u on the boundary nodes for the interior Neumann problem
    (-lap u = f in the domain, du/dnu = g on the boundary), from the
    boundary equation of Sec. 5: u/2 + D[u] = V[f] + S[g] (D the on-surface
    principal value).  Constants are in the null space (D[1] = -1/2 on the
    boundary); the rank-one term (sum_i w_i u_i / |Gamma|) 1 selects the
    solution with zero boundary mean.  Dense direct solve, for small
    boundaries only; v_boundary is V[f] at the nodes (None: f = 0)."""
    xy, w = bnd["xy"], bnd["w"]
    nb = len(xy)
    A = dirichlet_matrix(bnd, delta, order, on_tol, refine_levels)  # -I/2 + D
    A[np.diag_indices(nb)] += 1.0                                    # I/2 + D
    A += np.outer(np.ones(nb), w) / np.sum(w)
    SH = smooth_charge(xy, np.asarray(g) * w, xy, delta)
    if refine_levels > 0:
        SL, _ = local_dyadic(bnd, np.asarray(g, dtype=np.float64), None, xy, delta, refine_levels, order=order,
                             on_tol=on_tol)
    else:
        _, SL, _, _, _ = local(bnd, np.asarray(g, dtype=np.float64), None, xy, None, delta, order, on_tol)
    rhs = SH + SL + (0.0 if v_boundary is None else np.asarray(v_boundary))
    return np.linalg.solve(A, rhs)
