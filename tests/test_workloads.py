"""Checks of the seeded input generators against the recipe they state
(no method arithmetic lives in them; these tests pin the inputs)."""
import math

import numpy as np

from workloads import configs
from workloads import curves as C
from workloads import mesh as M
from workloads.panels import make_panels
from workloads.quadrature import triangle_rule6


def test_triangle_rule_exact_through_degree_four():
    """int over the reference triangle of x^i y^j = i! j! / (i + j + 2)!."""
    bary, w = triangle_rule6()
    assert np.all(w > 0) and np.all(bary > 0) and abs(w.sum() - 1.0) < 1e-15
    x, y = bary[:, 1], bary[:, 2]   # reference triangle (0,0), (1,0), (0,1)
    for i in range(5):
        for j in range(5 - i):
            got = 0.5 * np.sum(w * x ** i * y ** j)
            exact = math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)
            assert abs(got - exact) < 1e-15, (i, j)
    # degree 5 is not integrated exactly (the rule has 6 nodes)
    assert abs(0.5 * np.sum(w * x ** 5) - math.factorial(5) / math.factorial(7)) > 1e-8


def test_panels_integrate_arc_length():
    for curve, length in ((C.Circle(1.0), 2 * math.pi), (C.Ellipse(1.0, 0.6), None)):
        bnd = make_panels(curve, 32, 16)
        if length is None:  # ellipse perimeter from a fine trapezoid rule (periodic, spectral)
            t = np.linspace(0, 2 * np.pi, 20000, endpoint=False)
            length = float(np.mean(curve.speed(t)) * 2 * np.pi)
        assert abs(bnd["w"].sum() - length) < 1e-12 * length
        # outward normals, counter-clockwise order
        nrm, xy = bnd["normal"], bnd["xy"]
        assert np.allclose(np.hypot(nrm[:, 0], nrm[:, 1]), 1.0)
        assert np.all(np.sum(nrm * xy, axis=1) > 0)


def test_curved_mesh_quadrature_area():
    """Curved boundary triangles follow the curve: the weights of the disk
    mesh sum to pi with an error far below that of the inscribed 64-gon
    (5e-3); what remains is the 6-node rule on the curved maps."""
    d = configs.disk()
    assert len(d["src_w"]) == 6 * d["meta"]["n_triangles"]
    polygon = math.pi - 32 * math.sin(2 * math.pi / 64)
    assert abs(d["src_w"].sum() - math.pi) < 0.05 * polygon


def test_degraded_mesh_recipe():
    """Slivers with log-uniform aspect ratios up to ~1e4, 2% of the edges
    with a hanging node, 1% of the triangles removed (Sec. 6.4 recipe)."""
    rng = np.random.default_rng(7)
    curve = C.Star(0.3, 5)
    base = M.delaunay_mesh(curve, 4000, 240, rng)
    mesh = M.degrade(base, rng)
    st = mesh["stats"]
    assert st["n_nonconforming_edges"] == round(0.02 * st["n_edges_before"])
    n_before_drop = len(mesh["T"]) + st["n_removed"]
    p = st["n_removed"] / n_before_drop
    assert abs(p - 0.01) < 5 * math.sqrt(0.01 * 0.99 / n_before_drop)
    P, T = mesh["P"], mesh["T"]
    a, b, c = (np.linalg.norm(P[T[:, i]] - P[T[:, (i + 1) % 3]], axis=1) for i in range(3))
    area = 0.5 * np.abs((P[T[:, 1], 0] - P[T[:, 0], 0]) * (P[T[:, 2], 1] - P[T[:, 0], 1])
                        - (P[T[:, 1], 1] - P[T[:, 0], 1]) * (P[T[:, 2], 0] - P[T[:, 0], 0]))
    longest = np.maximum(np.maximum(a, b), c)
    aspect = longest ** 2 / (2 * area)     # ~1 for a well-shaped triangle
    assert aspect.max() > 1e3 and np.median(aspect) < 10
    assert np.mean(aspect > 100) > 0.1     # many slivers
    xy, w = M.quadrature(mesh, curve)
    star_area = math.pi * (1 + 0.3 ** 2 / 2)
    assert 0.97 * star_area < w.sum() < star_area  # 1% of triangles removed
    assert np.all(curve.inside(xy) | (np.abs(np.hypot(xy[:, 0], xy[:, 1]) - 1) < 0.31))


def test_generators_are_seeded():
    a, b = configs.disk(), configs.disk()
    for k in ("src_xy", "src_w", "src_f", "tgt_xy", "tgt_jet"):
        assert np.array_equal(a[k], b[k]), k
    c = configs.disk(seed=1001)
    assert not np.array_equal(a["src_xy"], c["src_xy"])
