"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every function declared in include/lp.h, and rejects invalid
arguments before touching the device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2409_11998_gb300 import build
    build.build()
    import paper_2409_11998_gb300 as lp
    return lp


def _declared():
    src = open(os.path.join(ROOT, "include", "lp.h")).read()
    return sorted(set(re.findall(r"^\s*(?:lp_status|const char\*)\s+(lp_\w+)\s*\(", src, re.M)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("lp_plan", "lp_volume", "lp_single_layer", "lp_double_layer", "lp_execute",
              "lp_sync", "lp_destroy", "lp_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    for name in _declared():
        assert name in exported, name
        assert hasattr(lib.library(), name)


def test_status_strings(lib):
    L = lib.library()
    for code in range(9):
        assert len(L.lp_status_string(code)) > 0
        assert L.lp_status_string(code) != b"unknown status"
    assert L.lp_status_string(99) == b"unknown status"


def test_invalid_arguments_rejected_without_device(lib):
    L = lib.library()
    dom = lib.lp_domain()
    dom.precision = 0
    dom.order = 5
    dom.box_lo[0] = dom.box_lo[1] = -1.0
    dom.box_hi[0] = dom.box_hi[1] = 1.0
    h = ctypes.c_void_p()
    assert L.lp_plan(None, 1e-3, 1e-9, ctypes.byref(h)) == 1
    assert L.lp_plan(ctypes.byref(dom), -1.0, 1e-9, ctypes.byref(h)) == 1
    assert L.lp_plan(ctypes.byref(dom), float("nan"), 1e-9, ctypes.byref(h)) == 1
    assert L.lp_plan(ctypes.byref(dom), 1e-3, 0.5, ctypes.byref(h)) == 1
    dom.order = 7
    assert L.lp_plan(ctypes.byref(dom), 1e-3, 1e-9, ctypes.byref(h)) == 1
    dom.order = 5
    dom.precision = 1
    assert L.lp_plan(ctypes.byref(dom), 1e-3, 1e-9, ctypes.byref(h)) == 1  # FP32 needs tol >= 1e-6
    dom.precision = 0
    dom.box_hi[0] = -2.0
    assert L.lp_plan(ctypes.byref(dom), 1e-3, 1e-9, ctypes.byref(h)) == 1
    dom.box_hi[0] = 1.0
    dom.n_panels = 4
    dom.panel_order = 1
    assert L.lp_plan(ctypes.byref(dom), 1e-3, 1e-9, ctypes.byref(h)) == 1
    dom.n_panels = 0
    for levels in (-2, 7):  # dyadic refinement takes 0..6 levels or LP_REFINE_AUTO (-1)
        dom.refine_levels = levels
        assert L.lp_plan(ctypes.byref(dom), 1e-3, 1e-9, ctypes.byref(h)) == 1
    dom.refine_levels = 0
    for levels, ups in ((3, 0.0), (-2, 0.0), (0, 1.1), (0, 4.0)):  # -1..2 levels; sigma 0 or 1.25..3
        dom.levels, dom.upsampling = levels, ups
        assert L.lp_plan(ctypes.byref(dom), 1e-3, 1e-9, ctypes.byref(h)) == 1
    dom.levels, dom.upsampling = 0, 1.25   # sigma 1.25 needs w = 21 at 1e-12 (> 16)
    assert L.lp_plan(ctypes.byref(dom), 1e-3, 1e-12, ctypes.byref(h)) == 1
    dom.upsampling = 0.0
    for fn in (L.lp_sync, L.lp_destroy):
        assert fn(None) == 1
    assert L.lp_sync_timeout(None, 1.0) == 1
    assert L.lp_volume_jets(None, 0, None, None) == 1
    assert L.lp_spread(None, 7, 1) == 1
    assert L.lp_finish(None, 0, None, None, None, None, None) == 1
    n = ctypes.c_int(9)
    assert L.lp_grid_buffers(None, None, None, None, ctypes.byref(n)) == 1
    dom.max_device_bytes = -1
    assert L.lp_plan(ctypes.byref(dom), 1e-3, 1e-9, ctypes.byref(h)) == 1
    dom.max_device_bytes = 0
    assert L.lp_volume(None, 0, None, None, None) == 1
    assert L.lp_execute(None, 0, None, None, None, None, None) == 1
    assert L.lp_execute_graph(None, 0, None, None, None, None, None) == 1
    it, res = ctypes.c_int(), ctypes.c_double()
    for solve in (L.lp_solve_dirichlet, L.lp_solve_neumann):
        assert solve(None, None, None, None, 1e-10, 10, 0, ctypes.byref(it), ctypes.byref(res)) == 1


def test_binding_rejects_wrong_dtypes(lib):
    with pytest.raises(ValueError):
        lib._ptr(np.zeros(3, dtype=np.float32))
    with pytest.raises(ValueError):
        lib._ptr(np.zeros((3, 2))[:, 0])


def test_missing_library_fails_loudly():
    """Without the built CUDA library the binding raises ImportError on first
    use, from every entry point: there is no CPU path to fall back to."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    child = (
        "import sys\n"
        f"sys.path.insert(0, {root!r})\n"
        "import paper_2409_11998_gb300 as lp\n"
        "lp.LIB_PATH = '/nonexistent/liblp.so'\n"
        "lp._LIB = None\n"
        "from workloads import configs\n"
        "p = configs.disk()\n"
        "b = p['bnd']\n"
        "plan = lambda: lp.lp_plan(p['box_lo'], p['box_hi'], p['delta'], 1e-9, precision=lp.LP_FP64,\n"
        "                          n_panels=b['n_panels'], panel_order=b['order'], bnd_xy=b['xy'],\n"
        "                          bnd_w=b['w'], bnd_normal=b['normal'])\n"
        "for call in (lambda: lp.library(), plan):\n"
        "    try:\n"
        "        call()\n"
        "    except ImportError:\n"
        "        continue\n"
        "    raise SystemExit('no ImportError')\n"
        "print('ok')\n")
    out = subprocess.run([sys.executable, "-c", child], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr[-2000:]
