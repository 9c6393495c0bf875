"""Python binding of the GB300 evaluator of 2D log-kernel volume and layer
potentials by heat-kernel splitting (arXiv 2409.11998).

Argument marshalling only: every step of the evaluation runs in the CUDA
library ``_build/liblp.so`` behind the C ABI of ``include/lp.h``.  The
functions below keep the C names (``lp_plan``, ``lp_volume``,
``lp_single_layer``, ``lp_double_layer``, ``lp_execute``, ``lp_sync``,
``lp_destroy``) and accept torch CUDA tensors (used in place) or host
arrays (numpy / CPU tensors; the library copies them).  Importing this
package fails loudly when the library has not been built: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblp.so")

LP_FP64, LP_FP32 = 0, 1
LP_REFINE_AUTO = -1  # refine_levels: levels from tol and order (Sec. 4.4)
LP_LEVELS_AUTO = -1  # levels: one history level when its grid is small
STATUS = {0: "LP_OK", 1: "LP_ERR_ARG", 2: "LP_ERR_OUT_OF_BOX", 3: "LP_ERR_NOMEM",
          4: "LP_ERR_CUDA", 5: "LP_ERR_UNSUPPORTED", 6: "LP_ERR_STATE", 7: "LP_ERR_NEWTON",
          8: "LP_ERR_TIMEOUT"}
EXPORTS = ("lp_plan", "lp_volume", "lp_single_layer", "lp_double_layer", "lp_execute", "lp_sync",
           "lp_destroy", "lp_status_string", "lp_plan_info", "lp_stage_times", "lp_execute_noalloc",
           "lp_batch_create", "lp_batch_execute", "lp_batch_sync", "lp_batch_stage_times",
           "lp_batch_destroy", "lp_solve_dirichlet", "lp_execute_graph", "lp_solve_neumann",
           "lp_sync_timeout", "lp_volume_jets", "lp_spread", "lp_grid_buffers", "lp_finish")


class LpError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({_lib().lp_status_string(code).decode()})")


class lp_domain(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("order", ctypes.c_int),
                ("box_lo", ctypes.c_double * 2), ("box_hi", ctypes.c_double * 2),
                ("n_panels", ctypes.c_int64), ("panel_order", ctypes.c_int),
                ("bnd_xy", ctypes.c_void_p), ("bnd_w", ctypes.c_void_p),
                ("bnd_normal", ctypes.c_void_p), ("stream", ctypes.c_void_p),
                ("refine_levels", ctypes.c_int),
                ("levels", ctypes.c_int),
                ("upsampling", ctypes.c_double),
                ("autotune", ctypes.c_int),
                ("max_device_bytes", ctypes.c_int64)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, d, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        L.lp_plan.argtypes = [ctypes.POINTER(lp_domain), d, d, ctypes.POINTER(vp)]
        L.lp_volume.argtypes = [vp, i64, vp, vp, vp]
        L.lp_single_layer.argtypes = [vp, vp]
        L.lp_double_layer.argtypes = [vp, vp]
        L.lp_execute.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        L.lp_execute_noalloc.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        L.lp_execute_graph.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        L.lp_batch_create.argtypes = [vp, ctypes.POINTER(vp)]
        L.lp_batch_execute.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp]
        L.lp_batch_sync.argtypes = [vp]
        L.lp_batch_stage_times.argtypes = [vp, vp]
        L.lp_batch_destroy.argtypes = [vp]
        L.lp_sync.argtypes = [vp]
        L.lp_sync_timeout.argtypes = [vp, d]
        L.lp_volume_jets.argtypes = [vp, i64, vp, vp]
        L.lp_spread.argtypes = [vp, i32, i32]
        L.lp_grid_buffers.argtypes = [vp, vp, vp, vp, ctypes.POINTER(i32)]
        L.lp_finish.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        L.lp_destroy.argtypes = [vp]
        L.lp_status_string.argtypes = [i32]
        L.lp_status_string.restype = ctypes.c_char_p
        L.lp_plan_info.argtypes = [vp, vp]
        L.lp_stage_times.argtypes = [vp, vp]
        L.lp_solve_dirichlet.argtypes = [vp, vp, vp, vp, d, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(d)]
        L.lp_solve_neumann.argtypes = [vp, vp, vp, vp, d, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(d)]
        for name in EXPORTS:
            if name != "lp_status_string":
                getattr(L, name).restype = i32
        _LIB = L
    return _LIB


def library():
    """The loaded ctypes library (raises ImportError if it is not built)."""
    return _lib()


def _check(code, where):
    if code != 0:
        raise LpError(code, where)


def _ptr(a):
    """Address of a contiguous float64 torch tensor or numpy array (or None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if str(a.dtype) != "torch.float64":
            raise ValueError("tensor must be float64")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous float64")
        return a.ctypes.data
    raise TypeError(f"unsupported buffer type {type(a)}")


def lp_plan(box_lo, box_hi, delta, tol, *, precision=LP_FP64, order=5, n_panels=0, panel_order=16,
            bnd_xy=None, bnd_w=None, bnd_normal=None, stream=0, refine_levels=0, levels=0, upsampling=0.0,
            autotune=False, max_device_bytes=0):
    dom = lp_domain()
    dom.precision = int(precision)
    dom.order = int(order)
    dom.box_lo[0], dom.box_lo[1] = float(box_lo[0]), float(box_lo[1])
    dom.box_hi[0], dom.box_hi[1] = float(box_hi[0]), float(box_hi[1])
    dom.n_panels = int(n_panels)
    dom.panel_order = int(panel_order)
    dom.bnd_xy = _ptr(bnd_xy)
    dom.bnd_w = _ptr(bnd_w)
    dom.bnd_normal = _ptr(bnd_normal)
    dom.stream = int(stream) if stream else None
    dom.refine_levels = LP_REFINE_AUTO if refine_levels == "auto" else int(refine_levels)
    dom.levels = LP_LEVELS_AUTO if levels == "auto" else int(levels)
    dom.upsampling = float(upsampling)
    dom.autotune = {False: 0, True: 1, "bins": 1, "full": 2}[autotune] if not isinstance(autotune, int) or \
        isinstance(autotune, bool) else int(autotune)
    dom.max_device_bytes = int(max_device_bytes)
    h = ctypes.c_void_p()
    _check(_lib().lp_plan(ctypes.byref(dom), float(delta), float(tol), ctypes.byref(h)), "lp_plan")
    return h


def lp_volume(plan, n, xy, w, f):
    _check(_lib().lp_volume(plan, int(n), _ptr(xy), _ptr(w), _ptr(f)), "lp_volume")


def lp_single_layer(plan, sigma):
    _check(_lib().lp_single_layer(plan, _ptr(sigma)), "lp_single_layer")


def lp_double_layer(plan, mu):
    _check(_lib().lp_double_layer(plan, _ptr(mu)), "lp_double_layer")


def lp_execute(plan, n_t, t_xy, f_jet, V=None, S=None, D=None):
    _check(_lib().lp_execute(plan, int(n_t), _ptr(t_xy), _ptr(f_jet), _ptr(V), _ptr(S), _ptr(D)),
           "lp_execute")


def lp_execute_noalloc(plan, n_t, t_xy, f_jet, V=None, S=None, D=None):
    """lp_execute without allocation: device buffers only, n_t <= 2**21
    (see include/lp.h)."""
    _check(_lib().lp_execute_noalloc(plan, int(n_t), _ptr(t_xy), _ptr(f_jet), _ptr(V), _ptr(S),
                                     _ptr(D)), "lp_execute_noalloc")


def lp_solve_neumann(plan, g, u, f_jet_b=None, tol=1e-10, max_iter=200, restart=30):
    """u/2 + D[u] = V[f] + S[g] at the plan's boundary nodes (Sec. 5) by GMRES;
    writes u (zero boundary mean), returns (iterations, true relative residual)."""
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    _check(_lib().lp_solve_neumann(plan, _ptr(g), _ptr(f_jet_b), _ptr(u), ctypes.c_double(tol),
                                   int(max_iter), int(restart), ctypes.byref(it), ctypes.byref(res)),
           "lp_solve_neumann")
    return it.value, res.value


def lp_execute_graph(plan, n_t, t_xy, f_jet, V, S, D):
    """lp_execute replayed from a CUDA graph after the first call with these
    arguments (device buffers only)."""
    _check(_lib().lp_execute_graph(plan, int(n_t), _ptr(t_xy), _ptr(f_jet), _ptr(V), _ptr(S), _ptr(D)),
           "lp_execute_graph")


def lp_solve_dirichlet(plan, g, mu, f_jet_b=None, tol=1e-10, max_iter=200, restart=30):
    """-mu/2 + D[mu] = g - V[f] at the plan's boundary nodes (Sec. 5) by GMRES;
    writes mu, returns (iterations, true relative residual)."""
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    _check(_lib().lp_solve_dirichlet(plan, _ptr(g), _ptr(f_jet_b), _ptr(mu), ctypes.c_double(tol),
                                     int(max_iter), int(restart), ctypes.byref(it), ctypes.byref(res)),
           "lp_solve_dirichlet")
    return it.value, res.value


def lp_batch_create(stream=0):
    h = ctypes.c_void_p()
    _check(_lib().lp_batch_create(int(stream) if stream else None, ctypes.byref(h)), "lp_batch_create")
    return h


def lp_batch_execute(batch, plans, n_t, t_xy, f_jet=None, V=None, S=None, D=None):
    """One wave: plans[i] evaluated at n_t[i] targets t_xy[i] (device
    tensors); V, S, D are lists of output tensors (entries may be None)."""
    n = len(plans)
    P = (ctypes.c_void_p * n)(*[p.value for p in plans])
    NT = (ctypes.c_int64 * n)(*[int(x) for x in n_t])

    def arr(lst):
        if lst is None:
            return None
        return (ctypes.c_void_p * n)(*[_ptr(x) for x in lst])
    args = [arr(t_xy), arr(f_jet), arr(V), arr(S), arr(D)]
    _check(_lib().lp_batch_execute(batch, n, P, NT, *[ctypes.cast(a, ctypes.c_void_p) if a is not None else None
                                                      for a in args]), "lp_batch_execute")


def lp_batch_sync(batch):
    _check(_lib().lp_batch_sync(batch), "lp_batch_sync")


def lp_batch_stage_times(batch):
    out = np.zeros(9, dtype=np.float32)
    _check(_lib().lp_batch_stage_times(batch, out.ctypes.data), "lp_batch_stage_times")
    keys = ["zero_copy", "spread", "fft_fwd", "multiplier", "fft_inv", "interp", "local", "total", "launches"]
    return dict(zip(keys, out.tolist()))


def lp_batch_destroy(batch):
    _check(_lib().lp_batch_destroy(batch), "lp_batch_destroy")


def lp_sync(plan):
    _check(_lib().lp_sync(plan), "lp_sync")


def lp_spread(plan, outputs="VSD", spread_layers=True):
    """Zero and spread the grids of the outputs (any of "V", "S", "D"): the
    bound volume nodes, and the boundary nodes when spread_layers."""
    mask = ("V" in outputs) * 1 + ("S" in outputs) * 2 + ("D" in outputs) * 4
    _check(_lib().lp_spread(plan, int(mask), 1 if spread_layers else 0), "lp_spread")


def lp_grid_buffers(plan):
    """[(device pointer, bytes, dtype)] of the buffers to sum across ranks
    (dtype "float64" or "float32")."""
    n = ctypes.c_int(9)
    ptrs = (ctypes.c_void_p * 9)()
    nbytes = (ctypes.c_int64 * 9)()
    dtypes = (ctypes.c_int * 9)()
    _check(_lib().lp_grid_buffers(plan, ptrs, nbytes, dtypes, ctypes.byref(n)), "lp_grid_buffers")
    return [(ptrs[i], nbytes[i], "float64" if dtypes[i] == 0 else "float32") for i in range(n.value)]


def lp_finish(plan, n_t, t_xy, f_jet, V=None, S=None, D=None):
    _check(_lib().lp_finish(plan, int(n_t), _ptr(t_xy), _ptr(f_jet), _ptr(V), _ptr(S), _ptr(D)), "lp_finish")


def lp_volume_jets(plan, n_t, t_xy, f_jet):
    """f-jets [n_t][6] at the targets estimated from the bound node values
    (weighted quadratic least squares within sqrt(3 delta_1)); writes f_jet."""
    _check(_lib().lp_volume_jets(plan, int(n_t), _ptr(t_xy), _ptr(f_jet)), "lp_volume_jets")


def lp_sync_timeout(plan, timeout_ms):
    """lp_sync with a bounded host wait; returns False (LP_ERR_TIMEOUT) if the
    plan's work is still running after timeout_ms, True once it completed."""
    code = _lib().lp_sync_timeout(plan, float(timeout_ms))
    if code == 8:
        return False
    _check(code, "lp_sync_timeout")
    return True


def lp_destroy(plan):
    _check(_lib().lp_destroy(plan), "lp_destroy")


def lp_plan_info(plan):
    out = np.zeros(37)
    _check(_lib().lp_plan_info(plan, out.ctypes.data), "lp_plan_info")
    keys = ["delta1", "delta2", "w", "beta", "g_nh", "K_nh", "P_nh", "g_fh", "K_fh", "P_fh", "L_fh",
            "band", "margin", "device_bytes", "precision", "order", "launches", "es_fit_err", "es_nc",
            "sigma_eff", "own_fft", "binned", "bin_cells", "refine_levels", "refine_table_err",
            "refine_subnodes", "levels", "sigma", "tune_ms_0", "tune_ms_1", "tune_ms_2",
            "grid_ms_s125_l1", "grid_ms_s125_l2", "grid_ms_s15_l1", "grid_ms_s15_l2", "grid_ms_s2_l1",
            "grid_ms_s2_l2"]
    return dict(zip(keys, out.tolist()))


def lp_stage_times(plan):
    out = np.zeros(11, dtype=np.float32)
    _check(_lib().lp_stage_times(plan, out.ctypes.data), "lp_stage_times")
    keys = ["spread", "fft_fwd", "multiplier", "fft_inv", "interp", "local", "total", "copies", "zero",
            "spread_volume", "refine"]
    return dict(zip(keys, out.tolist()))


class Evaluator:
    """Owns one plan.  ``problem`` is a dict as produced by ``workloads.configs``
    (numpy arrays); arrays are moved to the device once (torch) unless
    ``host=True``, in which case the C ABI receives host pointers."""

    def __init__(self, problem, precision=None, order=5, tol=None, device="cuda", host=False,
                 stream=None, refine_levels=0, levels=0, upsampling=0.0, autotune=False, max_device_bytes=0):
        import torch
        self.torch = torch
        self.host = host
        prec = problem.get("precision", "fp64") if precision is None else precision
        self.precision = LP_FP32 if prec in ("fp32", LP_FP32) else LP_FP64
        self.tol = problem["tol"] if tol is None else tol
        self.device = device
        b = problem.get("bnd")
        self._keep = []

        def dev(a):
            if a is None:
                return None
            if host:
                return np.ascontiguousarray(a, dtype=np.float64)
            t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=device)
            self._keep.append(t)
            return t

        self.stream = stream if stream is not None else (0 if host else torch.cuda.current_stream().cuda_stream)
        kw = {}
        if b is not None:
            kw = dict(n_panels=b["n_panels"], panel_order=b["order"], bnd_xy=dev(b["xy"]),
                      bnd_w=dev(b["w"]), bnd_normal=dev(b["normal"]))
        self.plan = lp_plan(problem["box_lo"], problem["box_hi"], problem["delta"], self.tol,
                            precision=self.precision, order=order, stream=self.stream,
                            refine_levels=refine_levels, levels=levels, upsampling=upsampling,
                            autotune=autotune, max_device_bytes=max_device_bytes, **kw)
        self.problem = problem

    def bind(self, src_xy=None, src_w=None, src_f=None, sigma=None, mu=None):
        p = self.problem
        dev = (lambda a: np.ascontiguousarray(a, dtype=np.float64)) if self.host else \
            (lambda a: self.torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=self.device))
        xy = p["src_xy"] if src_xy is None else src_xy
        w = p["src_w"] if src_w is None else src_w
        f = p["src_f"] if src_f is None else src_f
        self._src = [dev(xy), dev(w), dev(f)]
        lp_volume(self.plan, len(w), *self._src)
        s = p.get("sigma") if sigma is None else sigma
        m = p.get("mu") if mu is None else mu
        if s is not None:
            self._sig = dev(s)
            lp_single_layer(self.plan, self._sig)
        if m is not None:
            self._mu = dev(m)
            lp_double_layer(self.plan, self._mu)
        return self

    def evaluate(self, tgt_xy=None, tgt_jet=None, want=("V", "S", "D"), sync=True, graph=False):
        """V, S, D at the targets (default: the problem's).  graph=True goes
        through lp_execute_graph with device buffers kept by the evaluator
        (the problem's targets, or the given device tensors), so repeated
        calls replay one CUDA graph; the returned outputs are those buffers."""
        p = self.problem
        if graph:
            if self.host:
                raise ValueError("graph replay needs device buffers")
            torch = self.torch
            if tgt_xy is None:
                if getattr(self, "_graph_tgt", None) is None:
                    self._graph_tgt = (torch.as_tensor(np.ascontiguousarray(p["tgt_xy"]), device=self.device),
                                       torch.as_tensor(np.ascontiguousarray(p["tgt_jet"]), device=self.device))
                t, j = self._graph_tgt
            else:
                t, j = tgt_xy, tgt_jet
            n = len(t)
            key = (n, tuple(want))
            if getattr(self, "_graph_outs", None) is None or self._graph_outs[0] != key:
                self._graph_outs = (key, {k: torch.empty(n, dtype=torch.float64, device=self.device) for k in want})
            outs = self._graph_outs[1]
            lp_execute_graph(self.plan, n, t, j if "V" in want else None, outs.get("V"), outs.get("S"), outs.get("D"))
            if sync:
                lp_sync(self.plan)
            return outs
        txy = p["tgt_xy"] if tgt_xy is None else tgt_xy
        jet = p["tgt_jet"] if tgt_jet is None else tgt_jet
        n = len(txy)
        if self.host:
            t, j = np.ascontiguousarray(txy), np.ascontiguousarray(jet)
            outs = {k: np.zeros(n) for k in want}
        else:
            torch = self.torch
            t = torch.as_tensor(np.ascontiguousarray(txy), device=self.device) if not hasattr(txy, "data_ptr") else txy
            j = torch.as_tensor(np.ascontiguousarray(jet), device=self.device) if not hasattr(jet, "data_ptr") else jet
            outs = {k: torch.empty(n, dtype=torch.float64, device=self.device) for k in want}
        self._tgt = (t, j)
        lp_execute(self.plan, n, t, j if "V" in want else None, outs.get("V"), outs.get("S"), outs.get("D"))
        if sync:
            lp_sync(self.plan)
        return outs

    def solve_dirichlet(self, g, f_jet_b=None, tol=1e-10, max_iter=200, restart=30):
        """mu with -mu/2 + D[mu] = g - V[f] at the boundary nodes (Sec. 5);
        returns (mu, iterations, residual); mu is left bound as the plan's
        double-layer density."""
        n = len(self.problem["bnd"]["w"])
        conv = (lambda a: np.ascontiguousarray(a, dtype=np.float64)) if self.host else \
            (lambda a: self.torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=self.device))
        gd = conv(g)
        fj = None if f_jet_b is None else conv(f_jet_b)
        mu = np.zeros(n) if self.host else self.torch.empty(n, dtype=self.torch.float64, device=self.device)
        it, res = lp_solve_dirichlet(self.plan, gd, mu, f_jet_b=fj, tol=tol, max_iter=max_iter, restart=restart)
        self._mu = mu
        return mu, it, res

    def solve_neumann(self, g, f_jet_b=None, tol=1e-10, max_iter=200, restart=30):
        """u (zero boundary mean) with u/2 + D[u] = V[f] + S[g] at the boundary
        nodes (Sec. 5); returns (u, iterations, residual); g and u are left
        bound as the plan's single- and double-layer densities."""
        n = len(self.problem["bnd"]["w"])
        conv = (lambda a: np.ascontiguousarray(a, dtype=np.float64)) if self.host else \
            (lambda a: self.torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=self.device))
        gd = conv(g)
        fj = None if f_jet_b is None else conv(f_jet_b)
        u = np.zeros(n) if self.host else self.torch.empty(n, dtype=self.torch.float64, device=self.device)
        it, res = lp_solve_neumann(self.plan, gd, u, f_jet_b=fj, tol=tol, max_iter=max_iter, restart=restart)
        self._sig, self._mu = gd, u
        return u, it, res

    def info(self):
        return lp_plan_info(self.plan)

    def stage_times(self):
        return lp_stage_times(self.plan)

    def close(self):
        if self.plan is not None:
            lp_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
