"""Exact-rational brute force for tiny cases, written independently of the oracle.

The oracle decides coverage with integer edge functions and an edge-owner rule on
counter-clockwise triangles.  Here the same question is asked another way: exact
barycentric coordinates (``fractions.Fraction``, any orientation) at the texel
centre, and for points exactly on an edge the rule "covered iff the point nudged by
an infinitesimal (+1, -eta) step, eta infinitesimally smaller still, lies strictly
inside".  That nudge is the geometric meaning of owning the left and top edges, so a
dropped term, a wrong sign or a swapped corner in either formulation shows up as a
disagreement.
"""
from __future__ import annotations

import math
from fractions import Fraction as F

import numpy as np

GRID_MAX = (1 << 21) - 1


def snap(u, extent):
    """Round-half-even of u * 256 * extent, exactly."""
    return round(F(float(u)) * 256 * extent)


def bary(P, V):
    """Exact barycentrics of point P in triangle V (3 integer points); None if degenerate."""
    (x0, y0), (x1, y1), (x2, y2) = V
    det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)
    if det == 0:
        return None, None
    px, py = P
    l1 = F((px - x0) * (y2 - y0) - (x2 - x0) * (py - y0), det)
    l2 = F((x1 - x0) * (py - y0) - (px - x0) * (y1 - y0), det)
    l0 = 1 - l1 - l2
    # gradients of (l0, l1, l2) with respect to (x, y)
    g1 = (F(y2 - y0, det), F(-(x2 - x0), det))
    g2 = (F(-(y1 - y0), det), F(x1 - x0, det))
    g0 = (-g1[0] - g2[0], -g1[1] - g2[1])
    return (l0, l1, l2), (g0, g1, g2)


def covered_nudged(lam, grad):
    for l, (gx, gy) in zip(lam, grad):
        if l > 0:
            continue
        if l < 0:
            return False
        # on this edge: the nudge (+1, -eta) must move inside
        if gx > 0 or (gx == 0 and -gy > 0):
            continue
        return False
    return True


def quantize_exactish(p, mn, S):
    """The quantiser as the oracle states it (double arithmetic, Python floats are IEEE double)."""
    f = math.floor((float(p) - float(mn)) * S + 0.5)
    return min(max(f, 0), GRID_MAX)


def atlas(mesh, W, H, mn, S):
    """(tri id plane, position planes) of a tiny atlas by testing every texel against every triangle."""
    tri = np.full((H, W), 0xFFFFFFFF, np.uint32)
    pos = np.zeros((3, H, W), np.int64)
    pos[0] = np.iinfo(np.int32).min
    q = [[quantize_exactish(mesh.pos[i, a], mn[a], S) for a in range(3)] for i in range(mesh.pos.shape[0])]
    for j in range(H):
        for i in range(W):
            P = (256 * i + 128, 256 * j + 128)
            for t in range(mesh.n_tri):
                V = [(snap(mesh.uv[mesh.tri_uv[t, k], 0], W), snap(mesh.uv[mesh.tri_uv[t, k], 1], H)) for k in range(3)]
                lam, grad = bary(P, V)
                if lam is None or not covered_nudged(lam, grad):
                    continue
                tri[j, i] = t
                for a in range(3):
                    val = sum(lam[k] * q[mesh.tri_pos[t, k]][a] for k in range(3))
                    pos[a, j, i] = math.floor(val + F(1, 2))
                break
    return tri, pos


def area_weight(mesh, t, W, H, mn, S, frac=8, cap=(1 << 35) - 1):
    q = [[quantize_exactish(mesh.pos[mesh.tri_pos[t, k], a], mn[a], S) for a in range(3)] for k in range(3)]
    d1 = [q[1][a] - q[0][a] for a in range(3)]
    d2 = [q[2][a] - q[0][a] for a in range(3)]
    n = [d1[1] * d2[2] - d1[2] * d2[1], d1[2] * d2[0] - d1[0] * d2[2], d1[0] * d2[1] - d1[1] * d2[0]]
    a3 = math.isqrt(n[0] ** 2 + n[1] ** 2 + n[2] ** 2)
    V = [(snap(mesh.uv[mesh.tri_uv[t, k], 0], W), snap(mesh.uv[mesh.tri_uv[t, k], 1], H)) for k in range(3)]
    # shoelace: twice the signed area
    a2 = abs(sum(V[k][0] * V[(k + 1) % 3][1] - V[(k + 1) % 3][0] * V[k][1] for k in range(3)))
    if a2 == 0:
        return 0
    return min((a3 << (16 + frac)) // a2, cap)


def pip_exact(x, y, poly):
    """Even-odd point in polygon with exact rationals (x, y and vertices are taken as exact)."""
    x, y = F(float(x)), F(float(y))
    inside = False
    n = len(poly)
    for e in range(n):
        ax, ay = F(float(poly[e][0])), F(float(poly[e][1]))
        bx, by = F(float(poly[(e + 1) % n][0])), F(float(poly[(e + 1) % n][1]))
        if (ay > y) != (by > y):
            xi = (bx - ax) * (y - ay) / (by - ay) + ax
            if x < xi:
                inside = not inside
    return inside
