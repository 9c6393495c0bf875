"""Source densities with analytic derivative jets, and boundary densities.

A jet is an array of shape (n, 6): (f, f_x, f_y, f_xx, f_xy, f_yy).
"""
from __future__ import annotations

import numpy as np


class GaussianSum:
    """f(x) = background + sum_i a_i exp(-|x - c_i|^2 / s_i^2)
             + amp_sc * sin(kx x) cos(ky y)."""

    def __init__(self, centers, widths, amps=None, background=0.0, sincos=None):
        self.c = np.asarray(centers, dtype=np.float64).reshape(-1, 2)
        self.s = np.asarray(widths, dtype=np.float64).reshape(-1)
        self.a = np.ones(len(self.s)) if amps is None else np.asarray(amps, dtype=np.float64)
        self.bg = float(background)
        self.sincos = sincos  # (amp, kx, ky) or None

    def jet(self, xy, chunk=1 << 20):
        xy = np.asarray(xy, dtype=np.float64)
        out = np.zeros((len(xy), 6))
        for s0 in range(0, len(xy), chunk):
            p = xy[s0:s0 + chunk]
            o = out[s0:s0 + chunk]
            o[:, 0] = self.bg
            for (cx, cy), s, a in zip(self.c, self.s, self.a):
                dx, dy = p[:, 0] - cx, p[:, 1] - cy
                e = a * np.exp(-(dx * dx + dy * dy) / (s * s))
                is2 = 1.0 / (s * s)
                o[:, 0] += e
                o[:, 1] += e * (-2 * dx * is2)
                o[:, 2] += e * (-2 * dy * is2)
                o[:, 3] += e * (4 * dx * dx * is2 * is2 - 2 * is2)
                o[:, 4] += e * (4 * dx * dy * is2 * is2)
                o[:, 5] += e * (4 * dy * dy * is2 * is2 - 2 * is2)
            if self.sincos is not None:
                A, kx, ky = self.sincos
                sx, cx_ = np.sin(kx * p[:, 0]), np.cos(kx * p[:, 0])
                sy, cy_ = np.sin(ky * p[:, 1]), np.cos(ky * p[:, 1])
                o[:, 0] += A * sx * cy_
                o[:, 1] += A * kx * cx_ * cy_
                o[:, 2] += -A * ky * sx * sy
                o[:, 3] += -A * kx * kx * sx * cy_
                o[:, 4] += -A * kx * ky * cx_ * sy
                o[:, 5] += -A * ky * ky * sx * cy_
        return out

    def value(self, xy, chunk=1 << 21):
        xy = np.asarray(xy, dtype=np.float64)
        out = np.full(len(xy), self.bg)
        for s0 in range(0, len(xy), chunk):
            p = xy[s0:s0 + chunk]
            o = out[s0:s0 + chunk]
            for (cx, cy), s, a in zip(self.c, self.s, self.a):
                o += a * np.exp(-((p[:, 0] - cx) ** 2 + (p[:, 1] - cy) ** 2) / (s * s))
            if self.sincos is not None:
                A, kx, ky = self.sincos
                o += A * np.sin(kx * p[:, 0]) * np.cos(ky * p[:, 1])
        return out


class PolyField:
    """f = c0 + cx x + cy y + cxx x^2 + cxy x y + cyy y^2 (exact jet)."""

    def __init__(self, c0=0.0, cx=0.0, cy=0.0, cxx=0.0, cxy=0.0, cyy=0.0):
        self.k = (c0, cx, cy, cxx, cxy, cyy)

    def jet(self, xy):
        c0, cx, cy, cxx, cxy, cyy = self.k
        x, y = xy[:, 0], xy[:, 1]
        out = np.empty((len(xy), 6))
        out[:, 0] = c0 + cx * x + cy * y + cxx * x * x + cxy * x * y + cyy * y * y
        out[:, 1] = cx + 2 * cxx * x + cxy * y
        out[:, 2] = cy + cxy * x + 2 * cyy * y
        out[:, 3] = 2 * cxx
        out[:, 4] = cxy
        out[:, 5] = 2 * cyy
        return out

    def value(self, xy):
        return self.jet(xy)[:, 0]


def fourier_density(t, coef_cos, coef_sin):
    """sigma(t) = sum_n a_n cos(n t) + b_n sin(n t)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    for n, a in enumerate(coef_cos):
        out += a * np.cos(n * t)
    for n, b in enumerate(coef_sin):
        out += b * np.sin(n * t)
    return out


def random_smooth_density(t, rng, n_modes=16):
    """Fourier modes 0..n_modes-1 with N(0,1)/(1+n^2) coefficients."""
    n = np.arange(n_modes)
    a = rng.standard_normal(n_modes) / (1.0 + n * n)
    b = rng.standard_normal(n_modes) / (1.0 + n * n)
    b[0] = 0.0
    return fourier_density(t, a, b)
