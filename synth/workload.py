"""Seeded edit workloads: sphere strokes, orbit cameras, star-shaped lassos and the
three single-model configurations (small, large, roofline size).

Strokes are given in world units (a centre on the surface and a radius); turning
them into grid units is the library's job (and, independently, the oracle's).
Cameras are plain double-precision view-projection matrices.  Lasso polygons are
in screen pixels.  Nothing of the layer-editing method is computed here.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .mesh import Mesh, displaced_sphere, torus, vessel_charts, vessel_cylindrical


def _rng(*seed):
    return np.random.default_rng(np.random.SeedSequence([int(s) for s in seed]))


def bbox_diag(mesh: Mesh) -> float:
    p = mesh.pos.astype(np.float64)
    return float(np.linalg.norm(p.max(0) - p.min(0)))


def _area_cdf(mesh: Mesh) -> np.ndarray:
    cached = getattr(mesh, "_area_cdf", None)
    if cached is not None:
        return cached
    p = mesh.pos.astype(np.float64)
    a, b, c = p[mesh.tri_pos[:, 0]], p[mesh.tri_pos[:, 1]], p[mesh.tri_pos[:, 2]]
    cdf = np.cumsum(0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1))
    object.__setattr__(mesh, "_area_cdf", cdf)
    return cdf


def surface_points(mesh: Mesh, n: int, rng) -> np.ndarray:
    """n points uniform on the surface: triangle by 3D area, then uniform barycentrics."""
    p = mesh.pos
    cdf = _area_cdf(mesh)
    t = np.searchsorted(cdf, rng.uniform(0.0, cdf[-1], size=n), side="right")
    t = np.minimum(t, mesh.n_tri - 1)
    r1 = np.sqrt(rng.uniform(size=n))
    r2 = rng.uniform(size=n)
    w0, w1, w2 = 1.0 - r1, r1 * (1.0 - r2), r1 * r2
    a = p[mesh.tri_pos[t, 0]].astype(np.float64)
    b = p[mesh.tri_pos[t, 1]].astype(np.float64)
    c = p[mesh.tri_pos[t, 2]].astype(np.float64)
    return w0[:, None] * a + w1[:, None] * b + w2[:, None] * c


@dataclass
class Strokes:
    centre: np.ndarray   # float64 [n, 3] world units
    radius: np.ndarray   # float64 [n]    world units
    label: np.ndarray    # uint32 [n]
    layer: np.ndarray    # int32 [n] index of the target layer


def sphere_strokes(mesh: Mesh, n: int, seed: int, r_lo: float, r_hi: float, label_lo: int,
                   label_hi: int, n_layers: int = 1, log_uniform: bool = True) -> Strokes:
    """Radii as fractions of the bbox diagonal, log-uniform in [r_lo, r_hi] (or constant if equal);
    labels uniform in [label_lo, label_hi]; layers uniform in [0, n_layers)."""
    rng = _rng(0x5354524B, seed)
    diag = bbox_diag(mesh)
    c = surface_points(mesh, n, rng)
    if r_lo == r_hi:
        r = np.full(n, r_lo)
    elif log_uniform:
        r = np.exp(rng.uniform(np.log(r_lo), np.log(r_hi), size=n))
    else:
        r = rng.uniform(r_lo, r_hi, size=n)
    lab = rng.integers(label_lo, label_hi + 1, size=n).astype(np.uint32)
    lay = rng.integers(0, n_layers, size=n).astype(np.int32)
    return Strokes(c, r * diag, lab, lay)


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    eye, target, up = (np.asarray(v, dtype=np.float64) for v in (eye, target, up))
    f = target - eye
    f /= np.linalg.norm(f)
    s = np.cross(f, up)
    if np.linalg.norm(s) < 1e-9:
        s = np.cross(f, np.array([0.0, 1.0, 0.0]))
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = s, u, -f
    m[:3, 3] = -m[:3, :3] @ eye
    return m


def perspective01(fovy_deg: float, aspect: float, near: float, far: float) -> np.ndarray:
    """Right-handed perspective whose NDC depth runs from 0 at ``near`` to 1 at ``far``."""
    f = 1.0 / np.tan(np.radians(fovy_deg) / 2.0)
    m = np.zeros((4, 4))
    m[0, 0] = f / aspect
    m[1, 1] = f
    m[2, 2] = far / (near - far)
    m[2, 3] = near * far / (near - far)
    m[3, 2] = -1.0
    return m


def orthographic01(half_w: float, half_h: float, near: float, far: float) -> np.ndarray:
    m = np.eye(4)
    m[0, 0] = 1.0 / half_w
    m[1, 1] = 1.0 / half_h
    m[2, 2] = -1.0 / (far - near)
    m[2, 3] = -near / (far - near)
    return m


@dataclass
class Camera:
    vp: np.ndarray       # float64 [4, 4] row-major view-projection, clip = vp @ (x, y, z, 1)
    width: int
    height: int


def orbit_camera(mesh: Mesh, width: int, height: int, rng, fovy: float = 40.0) -> Camera:
    p = mesh.pos.astype(np.float64)
    lo, hi = p.min(0), p.max(0)
    centre = 0.5 * (lo + hi)
    radius = 0.5 * float(np.linalg.norm(hi - lo))
    az = rng.uniform(0.0, 2.0 * np.pi)
    el = np.radians(rng.uniform(-30.0, 60.0))
    dist = 2.5 * radius
    eye = centre + dist * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
    view = look_at(eye, centre)
    proj = perspective01(fovy, width / height, dist - 1.1 * radius, dist + 1.1 * radius)
    return Camera(proj @ view, width, height)


def project_px(cam: Camera, pts: np.ndarray) -> np.ndarray:
    """Screen pixel coordinates (row 0 at the bottom) of world points, in double; used
    only to place lassos where the model is."""
    h = np.concatenate([pts, np.ones((pts.shape[0], 1))], axis=1) @ cam.vp.T
    ndc = h[:, :2] / h[:, 3:4]
    return np.stack([(ndc[:, 0] * 0.5 + 0.5) * cam.width, (ndc[:, 1] * 0.5 + 0.5) * cam.height], 1)


def star_lasso(centre_px, n_vert: int, big_r: float, rng) -> np.ndarray:
    """Star polygon: vertex k at angle 2 pi k / n + jitter (|jitter| < pi/n), radius in
    [0.3, 1] * big_r around ``centre_px``.  float32 [n, 2] screen pixels."""
    k = np.arange(n_vert)
    ang = 2.0 * np.pi * k / n_vert + rng.uniform(-0.95, 0.95, size=n_vert) * np.pi / n_vert
    rad = rng.uniform(0.3, 1.0, size=n_vert) * big_r
    xy = np.stack([centre_px[0] + rad * np.cos(ang), centre_px[1] + rad * np.sin(ang)], 1)
    return xy.astype(np.float32)


@dataclass
class Lasso:
    cam: int             # index into the camera list
    poly: np.ndarray     # float32 [n, 2]
    label: int
    layer: int


def lassos(mesh: Mesh, cams: list, n: int, seed: int, label_lo: int, label_hi: int,
           n_layers: int, v_lo: int = 8, v_hi: int = 64) -> list:
    rng = _rng(0x4C53534F, seed)
    out = []
    for _ in range(n):
        ci = int(rng.integers(0, len(cams)))
        cam = cams[ci]
        for _try in range(100):
            c = project_px(cam, surface_points(mesh, 1, rng))[0]
            if 0 <= c[0] < cam.width and 0 <= c[1] < cam.height:
                break
        big_r = rng.uniform(0.05, 0.40) * min(cam.width, cam.height)
        nv = int(rng.integers(v_lo, v_hi + 1))
        out.append(Lasso(ci, star_lasso(c, nv, big_r, rng), int(rng.integers(label_lo, label_hi + 1)),
                         int(rng.integers(0, n_layers))))
    return out


@dataclass
class Workload:
    name: str
    mesh: Mesh
    width: int
    height: int
    tile: int
    dtype_bytes: int
    n_layers: int
    strokes: Strokes
    cams: list = field(default_factory=list)
    lassos: list = field(default_factory=list)
    n_labels: int = 256
    overlays: list = field(default_factory=list)   # (op, layer_a, layer_b)


def config_small(seed_mesh: int = 1) -> Workload:
    """Vessel 200 x 50 quads (20k triangles), 0.02 noise, cylindrical UV, 1024^2 uint8,
    two layers of 100 strokes each (radius 2% of the diagonal, labels 1..8), AND of the two,
    per-label area over 256 labels."""
    m = vessel_cylindrical(200, 50, noise_amp=0.02, noise_freq=4.0, seed=seed_mesh)
    s1 = sphere_strokes(m, 100, 11, 0.02, 0.02, 1, 8)
    s2 = sphere_strokes(m, 100, 12, 0.02, 0.02, 1, 8)
    s = Strokes(np.concatenate([s1.centre, s2.centre]), np.concatenate([s1.radius, s2.radius]),
                np.concatenate([s1.label, s2.label]),
                np.concatenate([np.zeros(100, np.int32), np.ones(100, np.int32)]))
    return Workload("vessel-20k-1024sq-u8", m, 1024, 1024, 32, 1, 2, s, overlays=[("and", 0, 1)])


def config_large(n_strokes: int = 10000, n_lassos: int = 200, n_cams: int = 8,
                 depth_side: int = 2048) -> Workload:
    """Vessel 1000 x 500 quads (1M triangles), 0.5% displacement noise, ~2k rectangular charts
    shelf-packed into 4096^2, 16 uint16 layers; sphere strokes with radii log-uniform in
    0.1-5% of the diagonal, labels 1..1000; star lassos of 8-64 vertices on orbit cameras with a
    depth_side^2 depth map."""
    m = vessel_charts(1000, 500, 25, 10, 4096, noise_amp=0.005, noise_freq=16.0, seed=2)
    s = sphere_strokes(m, n_strokes, 21, 0.001, 0.05, 1, 1000, n_layers=16)
    rng = _rng(0x43414D, 22)
    cams = [orbit_camera(m, depth_side, depth_side, rng) for _ in range(n_cams)]
    las = lassos(m, cams, n_lassos, 22, 1, 1000, 16)
    return Workload("vessel-1M-charts-4096sq-u16", m, 4096, 4096, 32, 2, 16, s, cams, las,
                    n_labels=1024)


def config_roofline(n_strokes: int = 1000, n_lassos: int = 20, n_cams: int = 4,
                    depth_side: int = 2048, n_theta: int = 2828, n_h: int = 1414,
                    side: int = 16384) -> Workload:
    """Vessel 2828 x 1414 quads (~8M triangles), 0.5% displacement, cylindrical UV, 16384^2,
    4 uint8 layers; sphere strokes with radii log-uniform in 1-30% of the diagonal, labels
    1..255; XOR and OR overlays; per-label area over 256 labels.  A few lassos on orbit cameras
    are added so that one pass exercises every step of the path."""
    m = vessel_cylindrical(n_theta, n_h, noise_amp=0.005, noise_freq=16.0, seed=3)
    s = sphere_strokes(m, n_strokes, 31, 0.01, 0.30, 1, 255, n_layers=4)
    rng = _rng(0x43414D, 32)
    cams = [orbit_camera(m, depth_side, depth_side, rng) for _ in range(n_cams)]
    las = lassos(m, cams, n_lassos, 32, 1, 255, 4)
    mt = m.n_tri / 1e6
    tri = f"{mt:.0f}M" if mt >= 1 else f"{m.n_tri / 1e3:.0f}k"
    return Workload(f"vessel-{tri}-{side}sq-u8", m, side, side, 32, 1, 4, s, cams, las,
                    overlays=[("xor", 0, 1), ("or", 2, 3)])


@dataclass
class BatchModel:
    mesh: Mesh
    side: int            # square atlas side
    strokes: Strokes     # sphere strokes, queue order interleaved with lassos by `order`
    cams: list
    lassos: list         # Lasso records (layer unused: one layer per model)
    order: np.ndarray    # queue: entries >= 0 are sphere stroke indices, entries < 0 are lasso -1-index


def batch_model(kind: str, n_tri: int, seed: int, n_sphere: int = 48, n_lasso: int = 16, depth_side: int = 1024,
                r_lo: float = 0.005, r_hi: float = 0.10) -> BatchModel:
    """One model of the batching workload: kind in {vessel, sphere, torus}, about n_tri triangles, an
    atlas side of the power of two nearest sqrt(8 n_tri) clamped to [512, 4096], 48 sphere strokes
    (radii log-uniform 0.5-10% of the diagonal) and 16 lassos on 2 orbit cameras, shuffled into one
    queue."""
    rng = _rng(0x4241, seed)
    n = max(int(np.sqrt(n_tri / 4.0)), 4)
    if kind == "vessel":
        m = vessel_cylindrical(2 * n, n, noise_amp=0.01, noise_freq=8.0, seed=seed)
    elif kind == "sphere":
        m = displaced_sphere(2 * n, n, seed=seed)
    else:
        m = torus(2 * n, n, seed=seed)
    side = int(2 ** np.clip(np.round(np.log2(np.sqrt(8.0 * m.n_tri))), 9, 12))
    st = sphere_strokes(m, n_sphere, seed * 7 + 1, r_lo, r_hi, 1, 255)
    cams = [orbit_camera(m, depth_side, depth_side, rng) for _ in range(2)]
    las = lassos(m, cams, n_lasso, seed * 7 + 2, 1, 255, 1)
    order = np.concatenate([np.arange(n_sphere), -1 - np.arange(n_lasso)])
    rng.shuffle(order)
    return BatchModel(m, side, st, cams, las, order)


def config_batch(n_models: int = 256, seed: int = 4, tri_lo: float = 5e3, tri_hi: float = 5e5, **kw) -> list:
    """The batching workload: n_models models of uneven size (triangles log-uniform in
    [tri_lo, tri_hi]), kinds drawn uniformly from vessel / displaced sphere / torus."""
    rng = _rng(0x42415443, seed)
    kinds = rng.choice(["vessel", "sphere", "torus"], size=n_models)
    tris = np.exp(rng.uniform(np.log(tri_lo), np.log(tri_hi), size=n_models))
    return [batch_model(str(k), int(t), 1000 * seed + i, **kw) for i, (k, t) in enumerate(zip(kinds, tris))]
