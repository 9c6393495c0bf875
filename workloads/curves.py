"""Closed, counter-clockwise boundary curves with exact derivatives.

Every curve is parametrised by t in [0, 2*pi) and exposes ``deriv(t, n)`` for
n = 0..4, returning an array of shape (len(t), 2).  The interior of the domain
lies to the left of the direction of travel, so the outward normal at
gamma(t) is (y', -x') / |gamma'|.

The Fourier-coefficient family is the boundary parametrisation used for all
tests of the paper's numerical section (Sec. 6, eq. bdryparam):
    gamma(t) = r (sum_k alpha_k cos kt + sum_k beta_k sin kt) (cos st, sin st)
               + (x0, y0).
"""
from __future__ import annotations

import math
import numpy as np


class Curve:
    """Base class: subclasses implement ``deriv(t, n)``."""

    corners = False

    def deriv(self, t, n=0):  # pragma: no cover - interface
        raise NotImplementedError

    def point(self, t):
        return self.deriv(np.atleast_1d(np.asarray(t, dtype=np.float64)), 0)

    def speed(self, t):
        d = self.deriv(np.atleast_1d(np.asarray(t, dtype=np.float64)), 1)
        return np.hypot(d[:, 0], d[:, 1])

    def outward_normal(self, t):
        d = self.deriv(np.atleast_1d(np.asarray(t, dtype=np.float64)), 1)
        s = np.hypot(d[:, 0], d[:, 1])
        return np.stack([d[:, 1] / s, -d[:, 0] / s], axis=1)

    def inside(self, p):  # pragma: no cover - interface
        raise NotImplementedError

    def bbox(self, n=4096):
        t = np.linspace(0.0, 2 * np.pi, n, endpoint=False)
        p = self.point(t)
        return p.min(axis=0), p.max(axis=0)


def _unit_vec_deriv(t, n):
    """n-th derivative of e(t) = (cos t, sin t)."""
    c, s = np.cos(t), np.sin(t)
    table = [(c, s), (-s, c), (-c, -s), (s, -c)]
    a, b = table[n % 4]
    return np.stack([a, b], axis=1)


class PolarCurve(Curve):
    """gamma(t) = rho(t) (cos t, sin t) + center, rho given with derivatives."""

    def __init__(self, center=(0.0, 0.0)):
        self.center = np.asarray(center, dtype=np.float64)

    def rho(self, t, n):  # pragma: no cover - interface
        raise NotImplementedError

    def deriv(self, t, n=0):
        t = np.atleast_1d(np.asarray(t, dtype=np.float64))
        out = np.zeros((t.size, 2))
        for k in range(n + 1):
            out += math.comb(n, k) * self.rho(t, k)[:, None] * _unit_vec_deriv(t, n - k)
        if n == 0:
            out += self.center
        return out

    def inside(self, p):
        p = np.asarray(p, dtype=np.float64) - self.center
        th = np.arctan2(p[:, 1], p[:, 0])
        return np.hypot(p[:, 0], p[:, 1]) < self.rho(th, 0)

    def wall_distance(self, p):
        """Approximate distance to the curve along its normal: the radial gap
        times the cosine between the radial direction and the normal."""
        p = np.asarray(p, dtype=np.float64) - self.center
        th = np.arctan2(p[:, 1], p[:, 0])
        r0, r1 = self.rho(th, 0), self.rho(th, 1)
        return np.abs(r0 - np.hypot(p[:, 0], p[:, 1])) * r0 / np.sqrt(r0 * r0 + r1 * r1)


class Circle(PolarCurve):
    def __init__(self, radius=1.0, center=(0.0, 0.0)):
        super().__init__(center)
        self.radius = float(radius)

    def rho(self, t, n):
        return np.full_like(t, self.radius) if n == 0 else np.zeros_like(t)


class Star(PolarCurve):
    """rho(t) = r0 (1 + a cos(k t)): the starfish domain is Star(0.3, 5)."""

    def __init__(self, a=0.3, k=5, r0=1.0, center=(0.0, 0.0)):
        super().__init__(center)
        self.a, self.k, self.r0 = float(a), int(k), float(r0)

    def rho(self, t, n):
        if n == 0:
            return self.r0 * (1.0 + self.a * np.cos(self.k * t))
        ph = [np.cos, lambda x: -np.sin(x), lambda x: -np.cos(x), np.sin][n % 4]
        return self.r0 * self.a * (self.k ** n) * ph(self.k * t)


class FourierCurve(PolarCurve):
    """The paper's test-boundary family (eq. bdryparam) with s = 1."""

    def __init__(self, r=1.0, alpha=None, beta=None, center=(0.0, 0.0)):
        super().__init__(center)
        self.r = float(r)
        self.alpha = dict(alpha or {0: 1.0})
        self.beta = dict(beta or {})

    def rho(self, t, n):
        out = np.zeros_like(t)
        for k, a in self.alpha.items():
            if n == 0:
                out += a * np.cos(k * t)
            else:
                ph = [np.cos, lambda x: -np.sin(x), lambda x: -np.cos(x), np.sin][n % 4]
                out += a * (k ** n) * ph(k * t)
        for k, b in self.beta.items():
            ph = [np.sin, np.cos, lambda x: -np.sin(x), lambda x: -np.cos(x)][n % 4]
            out += b * (k ** n) * ph(k * t)
        return self.r * out


def paper_validation_curve():
    """Boundary of the asymptotics-validation test (Sec. 6.1): r = 1,
    alpha0 = 5/6, beta3 = 1/30, alpha5 = 1/15, alpha6 = alpha8 = alpha10 = 1/30."""
    return FourierCurve(1.0, {0: 5 / 6, 5: 1 / 15, 6: 1 / 30, 8: 1 / 30, 10: 1 / 30}, {3: 1 / 30})


class Ellipse(Curve):
    def __init__(self, a=1.0, b=0.6, center=(0.0, 0.0)):
        self.a, self.b = float(a), float(b)
        self.center = np.asarray(center, dtype=np.float64)

    def deriv(self, t, n=0):
        t = np.atleast_1d(np.asarray(t, dtype=np.float64))
        e = _unit_vec_deriv(t, n)
        out = np.stack([self.a * e[:, 0], self.b * e[:, 1]], axis=1)
        if n == 0:
            out += self.center
        return out

    def inside(self, p):
        p = np.asarray(p, dtype=np.float64) - self.center
        return (p[:, 0] / self.a) ** 2 + (p[:, 1] / self.b) ** 2 < 1.0


class Square(Curve):
    """Boundary of [-h, h]^2 travelled counter-clockwise; t in [0, 2 pi) is
    split into four equal parameter ranges, one per side (straight, with
    corners)."""

    corners = True

    def __init__(self, half=1.0):
        self.h = float(half)

    def deriv(self, t, n=0):
        t = np.atleast_1d(np.asarray(t, dtype=np.float64))
        q = np.mod(t, 2 * np.pi) / (np.pi / 2)
        side = np.minimum(q.astype(np.int64), 3)
        u = q - side  # in [0, 1)
        h = self.h
        starts = np.array([[-h, -h], [h, -h], [h, h], [-h, h]])
        dirs = np.array([[2 * h, 0.0], [0.0, 2 * h], [-2 * h, 0.0], [0.0, -2 * h]])
        if n == 0:
            return starts[side] + u[:, None] * dirs[side]
        if n == 1:
            return dirs[side] / (np.pi / 2)
        return np.zeros((t.size, 2))

    def inside(self, p):
        p = np.asarray(p, dtype=np.float64)
        return (np.abs(p[:, 0]) < self.h) & (np.abs(p[:, 1]) < self.h)
