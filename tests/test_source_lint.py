"""Static checks of the CUDA sources (no GPU needed).

A warp-synchronous intrinsic with a full mask must be executed by every lane
of the warp.  Written as the right operand of && or ||, or as a branch of ?:,
it is skipped by the lanes whose left operand decides the result, and the
remaining lanes wait for them forever.  This check rejects those forms."""
import os
import re

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2409_11998_gb300", "csrc")
SYNC = r"(__shfl\w*_sync|__ballot_sync|__any_sync|__all_sync|__match\w*_sync|__reduce\w*_sync|__syncwarp)"
BAD = re.compile(r"(&&|\|\||\?)\s*!?\s*\(?\s*" + SYNC)


def test_no_warp_collective_behind_short_circuit():
    hits = []
    for name in sorted(os.listdir(CSRC)):
        if not name.endswith((".cu", ".cuh")):
            continue
        with open(os.path.join(CSRC, name)) as fh:
            for no, line in enumerate(fh, 1):
                code = line.split("//")[0]
                if BAD.search(code):
                    hits.append(f"{name}:{no}: {line.strip()}")
    assert not hits, "\n".join(hits)


def test_lint_pattern_catches_the_forms():
    for bad in ["ok && __shfl_down_sync(0xffffffffu, x, 16)", "a || __ballot_sync(m, p)",
                "c ? __shfl_sync(m, v, 0) : 0", "ok && !__any_sync(m, p)"]:
        assert BAD.search(bad), bad
    for good in ["const int y = __shfl_down_sync(0xffffffffu, x, 16);", "ok = ok && y;"]:
        assert not BAD.search(good), good


def test_no_trap_assert_or_unbounded_loop():
    """Kernels report failures through status words, never by trapping, and
    hold no loop without a bound (no spin-waits on flags)."""
    bad = re.compile(r"__trap\s*\(|\bassert\s*\(|asm\s*(volatile\s*)?\(\s*\"trap|while\s*\(\s*(true|1)\s*\)|for\s*\(\s*;\s*;\s*\)")
    hits = []
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(CSRC, name)) as fh:
                for no, line in enumerate(fh, 1):
                    if bad.search(line.split("//")[0]):
                        hits.append(f"{name}:{no}: {line.strip()}")
    assert not hits, "\n".join(hits)


def test_oracle_separation():
    """The oracle is test infrastructure: the package never imports it, the
    oracle never reaches into the package, and bench.py runs it only in its
    CPU-baseline leg and its reference arm."""
    import ast
    root = os.path.join(os.path.dirname(__file__), "..")
    pkg = os.path.join(root, "paper_2409_11998_gb300")
    for dirpath, _, files in os.walk(pkg):
        for name in files:
            if name.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, name)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), name
                assert "oracle/" not in text and "liboracle" not in text, name
    for name in os.listdir(os.path.join(root, "oracle")):
        if name.endswith((".py", ".cpp", ".h")):
            text = open(os.path.join(root, "oracle", name)).read()
            assert "paper_2409_11998_gb300" not in text and "csrc" not in text, name
    tree = ast.parse(open(os.path.join(root, "bench.py")).read())
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, ast.Import) and any(a.name == "oracle" for a in node.names):
                    users.add(fn.name)
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))
           and any(a.name == "oracle" for a in n.names)]
    assert not top and users <= {"cpu_baseline", "run_reference"}, users
