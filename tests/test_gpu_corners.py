"""V at the corners of the square (quadrant reading): targets within 12 sqrt(delta)
of both edges of a corner take the exact quadrant integral of the local
volume potential, on the GPU as in the oracle, in both precisions."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lp():
    from paper_2409_11998_gb300 import build
    build.build()
    import paper_2409_11998_gb300 as lp
    return lp


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-5)])
def test_square_corner_regions(lp, oracle_lib, precision, tol):
    from workloads import configs
    p = configs.square(n=120, panels_per_side=16, precision=precision, tol=tol)
    band = 12 * np.sqrt(p["delta"])
    # targets packed into the four corner regions, on the edges and at the corners
    rng = np.random.default_rng(41)
    ab = np.concatenate([rng.uniform(0, band, (200, 2)), [[0, 0], [0, 0.3 * band], [0.5 * band, 0]]])
    pts = []
    for sx, sy in [(1, 1), (-1, 1), (-1, -1), (1, -1)]:
        pts.append(np.column_stack([sx * (1 - ab[:, 0]), sy * (1 - ab[:, 1])]))
    txy = np.concatenate(pts)
    from oracle import jets
    q = dict(p)
    q["tgt_xy"] = txy
    # jets of the problem's f at these targets, from its node values (both
    # sides take the same jets; the quadrant reading is what is compared)
    q["tgt_jet"] = jets.estimate_jets(p["src_xy"], p["src_f"], txy, p["delta"], 2.0)
    ev = lp.Evaluator(q, precision=precision, tol=tol).bind()
    out = ev.evaluate(want=("V",))["V"].cpu().numpy()
    ref = oracle_lib.evaluate(q, want=("V",))["V"]
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < tol
    assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) < 5 * tol
    ev.close()
