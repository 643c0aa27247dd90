"""Seeded 3D gradient noise for the synthetic scanned-surface stand-ins.

The paper's models are 3D scans (Fig. 5); their fine surface relief is stood in
for by gradient noise in the style of Perlin's "improved noise" (quintic fade,
gradients drawn from the 12 edge directions of a cube, a permutation table
hashing lattice corners).  Unlike the classic fixed table, the permutation here
is drawn from a seeded generator, so every workload is reproducible from its
seed and distinct seeds give distinct surfaces.

This module is workload generation only: nothing of the layer-editing method is
computed here.
"""
from __future__ import annotations

import numpy as np

# 16 gradient directions: the 12 cube-edge midpoint directions, with four of
# them repeated so that a 4-bit hash indexes the table uniformly.
_GRADS = np.array(
    [
        [1, 1, 0], [-1, 1, 0], [1, -1, 0], [-1, -1, 0],
        [1, 0, 1], [-1, 0, 1], [1, 0, -1], [-1, 0, -1],
        [0, 1, 1], [0, -1, 1], [0, 1, -1], [0, -1, -1],
        [1, 1, 0], [0, -1, 1], [-1, 1, 0], [0, -1, -1],
    ],
    dtype=np.float64,
)


class GradientNoise3:
    """3D gradient noise with a permutation drawn from ``seed``."""

    def __init__(self, seed: int):
        rng = np.random.default_rng(np.random.SeedSequence([0x6E6F6973, int(seed)]))
        perm = rng.permutation(256).astype(np.int64)
        self._p = np.concatenate([perm, perm])

    @staticmethod
    def _fade(t):
        # 6t^5 - 15t^4 + 10t^3: first and second derivatives vanish at 0 and 1.
        return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)

    def _corner(self, xi, yi, zi, fx, fy, fz):
        p = self._p
        h = p[p[p[xi & 255] + (yi & 255)] + (zi & 255)] & 15
        g = _GRADS[h]
        return g[..., 0] * fx + g[..., 1] * fy + g[..., 2] * fz

    def __call__(self, x, y, z):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        x0 = np.floor(x)
        y0 = np.floor(y)
        z0 = np.floor(z)
        fx, fy, fz = x - x0, y - y0, z - z0
        xi, yi, zi = x0.astype(np.int64), y0.astype(np.int64), z0.astype(np.int64)
        u, v, w = self._fade(fx), self._fade(fy), self._fade(fz)

        def lerp(a, b, t):
            return a + t * (b - a)

        c000 = self._corner(xi, yi, zi, fx, fy, fz)
        c100 = self._corner(xi + 1, yi, zi, fx - 1, fy, fz)
        c010 = self._corner(xi, yi + 1, zi, fx, fy - 1, fz)
        c110 = self._corner(xi + 1, yi + 1, zi, fx - 1, fy - 1, fz)
        c001 = self._corner(xi, yi, zi + 1, fx, fy, fz - 1)
        c101 = self._corner(xi + 1, yi, zi + 1, fx - 1, fy, fz - 1)
        c011 = self._corner(xi, yi + 1, zi + 1, fx, fy - 1, fz - 1)
        c111 = self._corner(xi + 1, yi + 1, zi + 1, fx - 1, fy - 1, fz - 1)
        x00 = lerp(c000, c100, u)
        x10 = lerp(c010, c110, u)
        x01 = lerp(c001, c101, u)
        x11 = lerp(c011, c111, u)
        return lerp(lerp(x00, x10, v), lerp(x01, x11, v), w)
