"""Pins of the oracle's f-jet estimator (oracle/jets.py): a weighted
quadratic least-squares fit reproduces any quadratic exactly, converges at
the rates of a quadratic fit on a smooth field, and follows its stated
fallbacks (linear fit, weighted mean, zero jet; exact value at a node)."""
import numpy as np
import pytest

from oracle import jets


def _cloud(h, seed=0, lo=-1.0, hi=1.0):
    rng = np.random.default_rng(seed)
    g = np.arange(lo, hi + 1e-12, h)
    X, Y = np.meshgrid(g, g, indexing="ij")
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    return xy + rng.uniform(-0.3 * h, 0.3 * h, xy.shape)


def test_quadratic_reproduced_exactly():
    h = 0.02
    xy = _cloud(h)
    q = lambda x, y: 0.7 - 1.3 * x + 0.4 * y + 2.5 * x * x - 1.1 * x * y + 0.9 * y * y
    tgt = np.random.default_rng(3).uniform(-0.8, 0.8, (50, 2))
    J = jets.estimate_jets(xy, q(xy[:, 0], xy[:, 1]), tgt, delta=3 * h * h, box_side=2.0)
    x, y = tgt[:, 0], tgt[:, 1]
    want = np.stack([q(x, y), -1.3 + 5.0 * x - 1.1 * y, 0.4 - 1.1 * x + 1.8 * y,
                     np.full_like(x, 5.0), np.full_like(x, -1.1), np.full_like(x, 1.8)], axis=1)
    assert np.max(np.abs(J - want)) < 1e-9


def test_convergence_on_a_smooth_field():
    f = lambda x, y: np.sin(3 * x) * np.cos(2 * y) + x
    fx = lambda x, y: 3 * np.cos(3 * x) * np.cos(2 * y) + 1
    fyy = lambda x, y: -4 * np.sin(3 * x) * np.cos(2 * y)
    tgt = np.random.default_rng(4).uniform(-0.5, 0.5, (200, 2))
    e1, e2 = [], []
    for h in (0.04, 0.02, 0.01):
        xy = _cloud(h, seed=1)
        J = jets.estimate_jets(xy, f(xy[:, 0], xy[:, 1]), tgt, delta=3 * h * h, box_side=2.0)
        e1.append(np.sqrt(np.mean((J[:, 1] - fx(tgt[:, 0], tgt[:, 1])) ** 2)))
        e2.append(np.sqrt(np.mean((J[:, 5] - fyy(tgt[:, 0], tgt[:, 1])) ** 2)))
    r1 = np.log2(np.array(e1[:-1]) / np.array(e1[1:]))
    r2 = np.log2(np.array(e2[:-1]) / np.array(e2[1:]))
    # RMS errors over the targets; the nodes are jittered at every scale, so
    # the rates carry some noise: first derivatives O(rho^2), second O(rho)
    assert np.all(r1 > 1.6), (e1, r1)
    assert np.all(r2 > 0.6), (e2, r2)
    assert e2[-1] < 0.05 * np.sqrt(np.mean(fyy(tgt[:, 0], tgt[:, 1]) ** 2))


def test_fallbacks_and_node_value():
    delta = 3e-4                           # rho = 0.03
    far = jets.estimate_jets(np.array([[0.0, 0.0]]), np.array([2.0]), [[1.0, 1.0]], delta, 2.0)
    assert np.all(far == 0.0)              # no node within rho: zero jet
    one = jets.estimate_jets(np.array([[0.0, 0.0]]), np.array([2.0]), [[0.01, 0.0]], delta, 2.0)
    assert one[0, 0] == pytest.approx(2.0) and np.all(one[0, 1:] == 0.0)   # weighted mean
    ring = np.array([[0.01 * np.cos(t), 0.01 * np.sin(t)] for t in np.linspace(0, 2 * np.pi, 6)[:-1]])
    lin = jets.estimate_jets(ring, 1.0 + 2.0 * ring[:, 0] - ring[:, 1], [[0.0, 0.0]], delta, 2.0)
    assert np.allclose(lin[0], [1.0, 2.0, -1.0, 0, 0, 0], atol=1e-12)      # 5 neighbours: linear fit
    xy = _cloud(0.01)
    fv = np.cos(xy[:, 0]) * 7.0
    J = jets.estimate_jets(xy, fv, xy[100:103], delta=3e-4, box_side=2.0)
    assert np.all(J[:, 0] == fv[100:103])  # a target on a node takes the node's value
