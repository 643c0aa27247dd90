"""Seeded synthetic meshes with texture coordinates.

The paper edits layers of scanned cultural-heritage models (Fig. 5: a vessel of
312k triangles up to a statue of 10M).  Those scans are not available, so the
workloads use surfaces of revolution shaped like a vessel, with seeded gradient
noise standing in for scan relief, and two kinds of texture parametrisation:

* a cylindrical unwrap (u = angle / 2pi, v = height), one island with a seam;
* a chart atlas: the surface cut into rectangular charts, each chart laid out in
  UV space at a size proportional to its 3D extent, and the charts shelf-packed
  into the texture with a gutter between them (many islands, as in scanned-model
  atlases, Section 4.3.2).

Seam and chart-border vertices are duplicated in UV only, so a mesh has separate
position and UV index triples per triangle.  Everything here produces plain
float32 / uint32 arrays; nothing of the layer-editing method is computed here.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .noise import GradientNoise3


@dataclass
class Mesh:
    pos: np.ndarray      # float32 [n_pos, 3]
    uv: np.ndarray       # float32 [n_uv, 2]
    tri_pos: np.ndarray  # uint32 [n_tri, 3] indices into pos
    tri_uv: np.ndarray   # uint32 [n_tri, 3] indices into uv

    @property
    def n_tri(self) -> int:
        return int(self.tri_pos.shape[0])

    def check(self) -> "Mesh":
        assert self.pos.dtype == np.float32 and self.pos.ndim == 2 and self.pos.shape[1] == 3
        assert self.uv.dtype == np.float32 and self.uv.ndim == 2 and self.uv.shape[1] == 2
        assert self.tri_pos.dtype == np.uint32 and self.tri_pos.shape == self.tri_uv.shape
        assert self.tri_uv.dtype == np.uint32
        for a in (self.pos, self.uv, self.tri_pos, self.tri_uv):
            assert a.flags["C_CONTIGUOUS"]
        if self.n_tri:
            assert int(self.tri_pos.max()) < self.pos.shape[0]
            assert int(self.tri_uv.max()) < self.uv.shape[0]
        return self


def _vessel_surface(n_theta, n_h, noise_amp, noise_freq, seed, height=2.0):
    """Vertex grid of the vessel: radius 1 + 0.3 sin(3 pi h) + noise, h in [0,1]."""
    theta = 2.0 * np.pi * np.arange(n_theta, dtype=np.float64) / n_theta
    h = np.arange(n_h + 1, dtype=np.float64) / n_h
    th, hh = np.meshgrid(theta, h)                      # [n_h+1, n_theta]
    r = 1.0 + 0.3 * np.sin(3.0 * np.pi * hh)
    if noise_amp != 0.0:
        noise = GradientNoise3(seed)
        r = r + noise_amp * noise(noise_freq * np.cos(th), noise_freq * np.sin(th), noise_freq * hh)
    pos = np.stack([r * np.cos(th), r * np.sin(th), height * hh], axis=-1)
    return pos.reshape(-1, 3).astype(np.float32)


def vessel_cylindrical(n_theta: int, n_h: int, noise_amp: float = 0.02, noise_freq: float = 4.0,
                       seed: int = 1) -> Mesh:
    """Open vessel, 2*n_theta*n_h triangles, cylindrical UV unwrap (one island)."""
    pos = _vessel_surface(n_theta, n_h, noise_amp, noise_freq, seed)
    iu = np.arange(n_theta + 1, dtype=np.float64) / n_theta
    jv = np.arange(n_h + 1, dtype=np.float64) / n_h
    uu, vv = np.meshgrid(iu, jv)
    uv = np.stack([uu, vv], axis=-1).reshape(-1, 2).astype(np.float32)

    i = np.arange(n_theta, dtype=np.int64)
    j = np.arange(n_h, dtype=np.int64)
    ii, jj = np.meshgrid(i, j)
    ii, jj = ii.ravel(), jj.ravel()
    ip = (ii + 1) % n_theta
    pa, pb = jj * n_theta + ii, jj * n_theta + ip
    pc, pd = (jj + 1) * n_theta + ip, (jj + 1) * n_theta + ii
    su = n_theta + 1
    ua, ub = jj * su + ii, jj * su + ii + 1
    uc, ud = (jj + 1) * su + ii + 1, (jj + 1) * su + ii
    tri_pos = np.stack([np.stack([pa, pb, pc], 1), np.stack([pa, pc, pd], 1)], 1).reshape(-1, 3)
    tri_uv = np.stack([np.stack([ua, ub, uc], 1), np.stack([ua, uc, ud], 1)], 1).reshape(-1, 3)
    return Mesh(pos, uv, tri_pos.astype(np.uint32), tri_uv.astype(np.uint32)).check()


def _shelf_pack(widths, heights, side, gutter):
    """Place rectangles (texel units) on shelves, tallest first; None if they do not fit."""
    order = np.argsort(-heights, kind="stable")
    x = np.zeros_like(widths)
    y = np.zeros_like(heights)
    cx = cy = float(gutter)
    shelf_h = 0.0
    for k in order:
        w, hgt = widths[k], heights[k]
        if cx + w + gutter > side:
            cx = float(gutter)
            cy += shelf_h + gutter
            shelf_h = 0.0
        if cy + hgt + gutter > side or w + 2 * gutter > side:
            return None
        x[k], y[k] = cx, cy
        cx += w + gutter
        shelf_h = max(shelf_h, hgt)
    return x, y


def vessel_charts(n_theta: int, n_h: int, chart_q_theta: int, chart_q_h: int, side: int,
                  noise_amp: float = 0.005, noise_freq: float = 16.0, seed: int = 2,
                  gutter: int = 2) -> Mesh:
    """Vessel cut into rectangular charts of chart_q_theta x chart_q_h quads, shelf-packed
    into a side x side texture with a gutter (texels) between charts."""
    assert n_theta % chart_q_theta == 0 and n_h % chart_q_h == 0
    pos = _vessel_surface(n_theta, n_h, noise_amp, noise_freq, seed)
    P = pos.astype(np.float64).reshape(n_h + 1, n_theta, 3)
    nct, nch = n_theta // chart_q_theta, n_h // chart_q_h
    n_charts = nct * nch
    # 3D extent of each chart: mean length of its rows (theta direction) and columns (h).
    seg_t = np.linalg.norm(np.roll(P, -1, axis=1) - P, axis=-1)        # [n_h+1, n_theta]
    seg_h = np.linalg.norm(P[1:] - P[:-1], axis=-1)                    # [n_h, n_theta]
    w3 = np.empty(n_charts)
    h3 = np.empty(n_charts)
    for cj in range(nch):
        for ci in range(nct):
            k = cj * nct + ci
            t0, t1 = ci * chart_q_theta, (ci + 1) * chart_q_theta
            h0, h1 = cj * chart_q_h, (cj + 1) * chart_q_h
            w3[k] = seg_t[h0:h1 + 1, t0:t1].sum(axis=1).mean()
            cols = np.arange(t0, t1 + 1) % n_theta
            h3[k] = seg_h[h0:h1][:, cols].sum(axis=0).mean()
    # Largest texel-per-unit scale at which the shelf packer still fits everything.
    lo, hi = 0.0, float(side) / max(w3.max(), h3.max())
    best = None
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        placed = _shelf_pack(np.ceil(w3 * mid), np.ceil(h3 * mid), side, gutter)
        if placed is None:
            hi = mid
        else:
            lo, best = mid, placed
    assert best is not None, "charts do not fit"
    s = lo
    ox, oy = best

    uvs = []
    tri_pos = []
    tri_uv = []
    nuv_c = (chart_q_theta + 1) * (chart_q_h + 1)
    li = np.arange(chart_q_theta + 1)
    lj = np.arange(chart_q_h + 1)
    lii, ljj = np.meshgrid(li, lj)
    qi, qj = np.meshgrid(np.arange(chart_q_theta), np.arange(chart_q_h))
    qi, qj = qi.ravel(), qj.ravel()
    for cj in range(nch):
        for ci in range(nct):
            k = cj * nct + ci
            u = (ox[k] + lii / chart_q_theta * w3[k] * s) / side
            v = (oy[k] + ljj / chart_q_h * h3[k] * s) / side
            uvs.append(np.stack([u, v], -1).reshape(-1, 2))
            base = k * nuv_c
            gi = ci * chart_q_theta + qi
            gj = cj * chart_q_h + qj
            gip = (gi + 1) % n_theta
            pa, pb = gj * n_theta + gi, gj * n_theta + gip
            pc, pd = (gj + 1) * n_theta + gip, (gj + 1) * n_theta + gi
            su = chart_q_theta + 1
            ua, ub = base + qj * su + qi, base + qj * su + qi + 1
            uc, ud = base + (qj + 1) * su + qi + 1, base + (qj + 1) * su + qi
            tri_pos.append(np.stack([np.stack([pa, pb, pc], 1), np.stack([pa, pc, pd], 1)], 1).reshape(-1, 3))
            tri_uv.append(np.stack([np.stack([ua, ub, uc], 1), np.stack([ua, uc, ud], 1)], 1).reshape(-1, 3))
    uv = np.concatenate(uvs).astype(np.float32)
    return Mesh(pos, uv, np.concatenate(tri_pos).astype(np.uint32),
                np.concatenate(tri_uv).astype(np.uint32)).check()


def uv_square_patch(W: int, H: int, k: int = 1, pos_extent: float | None = None) -> Mesh:
    """Two triangles: UV square [0,1]^2 mapped to a planar 3D rectangle of k*W x k*H units
    in z = 0, plus one far-away anchor vertex so the bbox extent is exactly ``pos_extent``
    (default 2^21 - 1).  With that extent the position quantiser maps position units to grid
    units one to one, which makes exact closed forms available (area per texel = k^2)."""
    ext = float((1 << 21) - 1) if pos_extent is None else float(pos_extent)
    pos = np.array([[0, 0, 0], [k * W, 0, 0], [k * W, k * H, 0], [0, k * H, 0], [0, 0, ext]],
                   dtype=np.float32)
    uv = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float32)
    tri = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.uint32)
    return Mesh(pos, uv, tri.copy(), tri.copy()).check()


def random_soup(n_tri: int, seed: int, uv_lo: float = -0.2, uv_hi: float = 1.2,
                uv_size: float = 0.3) -> Mesh:
    """Unstructured triangles with random positions and random, overlapping UV triangles
    (some degenerate, some partly outside [0,1]^2).  For brute-force checks on tiny atlases."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-1.0, 1.0, size=(3 * n_tri, 3)).astype(np.float32)
    c = rng.uniform(uv_lo, uv_hi, size=(n_tri, 1, 2))
    d = rng.uniform(-uv_size, uv_size, size=(n_tri, 3, 2))
    uv = (c + d).reshape(-1, 2)
    # A few exactly degenerate and a few texel-centre-aligned UVs to exercise ties.
    if n_tri >= 4:
        uv[3:6] = uv[3]
    uv = uv.astype(np.float32)
    idx = np.arange(3 * n_tri, dtype=np.uint32).reshape(n_tri, 3)
    return Mesh(pos, uv, idx.copy(), idx.copy()).check()


def grid_patch(nx: int, ny: int, W: int, H: int, seed: int, jitter: float = 0.0) -> Mesh:
    """A regular nx x ny quad grid covering UV [0,1]^2 (shared UV vertices, so every interior
    texel centre is covered exactly once), with a random height field for positions."""
    rng = np.random.default_rng(seed)
    xs = np.linspace(0.0, 1.0, nx + 1)
    ys = np.linspace(0.0, 1.0, ny + 1)
    gx, gy = np.meshgrid(xs, ys)
    uvg = np.stack([gx, gy], -1)
    if jitter:
        inner = (slice(1, -1), slice(1, -1))
        uvg[inner] += rng.uniform(-jitter, jitter, size=uvg[inner].shape) / np.array([nx, ny])
    uv = uvg.reshape(-1, 2).astype(np.float32)
    z = rng.uniform(0.0, 0.2, size=gx.shape)
    pos = np.stack([gx * 3.0, gy * 2.0, z], -1).reshape(-1, 3).astype(np.float32)
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    i, j = i.ravel(), j.ravel()
    s = nx + 1
    a, b, c, d = j * s + i, j * s + i + 1, (j + 1) * s + i + 1, (j + 1) * s + i
    tri = np.stack([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], 1).reshape(-1, 3).astype(np.uint32)
    return Mesh(pos, uv, tri.copy(), tri.copy()).check()


def _grid_mesh(pos_grid: np.ndarray, wrap_u: bool, wrap_v: bool) -> tuple:
    """Triangles of an (nv+1) x (nu+1) parameter grid; positions wrap where the surface closes
    (duplicated in UV only), texture coordinates (u, v) = (i/nu, j/nv) never wrap."""
    nvp, nup = pos_grid.shape[:2]
    nu, nv = nup - 1, nvp - 1
    pu = nu if wrap_u else nup          # distinct position columns
    pv = nv if wrap_v else nvp          # distinct position rows
    pos = pos_grid[:pv, :pu].reshape(-1, 3).astype(np.float32)
    iu = np.arange(nup) / nu
    jv = np.arange(nvp) / nv
    uu, vv = np.meshgrid(iu, jv)
    uv = np.stack([uu, vv], -1).reshape(-1, 2).astype(np.float32)
    i, j = np.meshgrid(np.arange(nu), np.arange(nv))
    i, j = i.ravel(), j.ravel()
    ip, jp = (i + 1) % pu if wrap_u else i + 1, (j + 1) % pv if wrap_v else j + 1
    pa, pb, pc, pd = j * pu + i, j * pu + ip, jp * pu + ip, jp * pu + i
    ua, ub, uc, ud = j * nup + i, j * nup + i + 1, (j + 1) * nup + i + 1, (j + 1) * nup + i
    tri_pos = np.stack([np.stack([pa, pb, pc], 1), np.stack([pa, pc, pd], 1)], 1).reshape(-1, 3)
    tri_uv = np.stack([np.stack([ua, ub, uc], 1), np.stack([ua, uc, ud], 1)], 1).reshape(-1, 3)
    return Mesh(pos, uv, tri_pos.astype(np.uint32), tri_uv.astype(np.uint32)).check()


def displaced_sphere(n_lon: int, n_lat: int, noise_amp: float = 0.03, noise_freq: float = 3.0,
                     seed: int = 7) -> Mesh:
    """Unit sphere with seeded radial noise, equirectangular UV (u = longitude, v = latitude);
    2 * n_lon * n_lat triangles (those touching the poles have zero 3D area on one side)."""
    lon = 2.0 * np.pi * np.arange(n_lon + 1) / n_lon
    lat = np.pi * np.arange(n_lat + 1) / n_lat - np.pi / 2
    LO, LA = np.meshgrid(lon, lat)
    d = np.stack([np.cos(LA) * np.cos(LO), np.cos(LA) * np.sin(LO), np.sin(LA)], -1)
    r = 1.0 + noise_amp * GradientNoise3(seed)(noise_freq * d[..., 0], noise_freq * d[..., 1], noise_freq * d[..., 2])
    return _grid_mesh(d * r[..., None], wrap_u=True, wrap_v=False)


def torus(n_u: int, n_v: int, major: float = 1.0, minor: float = 0.35, noise_amp: float = 0.01,
          noise_freq: float = 4.0, seed: int = 9) -> Mesh:
    """Torus with seeded noise on the tube radius, UV = (angle around the axis, angle around the
    tube) / 2 pi; 2 * n_u * n_v triangles."""
    a = 2.0 * np.pi * np.arange(n_u + 1) / n_u
    b = 2.0 * np.pi * np.arange(n_v + 1) / n_v
    A, B = np.meshgrid(a, b)
    base = np.stack([np.cos(A), np.sin(A), np.zeros_like(A)], -1) * major
    rr = minor * (1.0 + noise_amp / minor * GradientNoise3(seed)(noise_freq * np.cos(A), noise_freq * np.sin(A),
                                                                 noise_freq * np.cos(B)))
    p = base + rr[..., None] * np.stack([np.cos(B) * np.cos(A), np.cos(B) * np.sin(A), np.sin(B)], -1)
    return _grid_mesh(p, wrap_u=True, wrap_v=True)
