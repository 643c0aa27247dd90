"""Helpers for the GPU parity tests: run one workload through the CUDA library (via the
Python binding of the C ABI) and through the oracle, with the same seeded inputs."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2501_14807_gb300 import lcl

DEV = "cuda"


def to_np(t: torch.Tensor, dtype) -> np.ndarray:
    return t.detach().cpu().numpy().view(dtype)


def to_dev(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    view = {np.dtype(np.uint16): np.int16, np.dtype(np.uint32): np.int32,
            np.dtype(np.uint64): np.int64}.get(a.dtype, a.dtype)
    return torch.from_numpy(a.view(view)).to(DEV)


def gpu_atlas(mesh, W, H, T):
    m = lcl.Mesh.from_host(mesh, DEV)
    a = lcl.Atlas(W, H, T, mesh.n_tri, DEV)
    lcl.lcl_atlas_build(m, a)
    return m, a


def atlas_planes(a: lcl.Atlas):
    return {k: to_np(a.plane(k), np.int32) for k in ("pos_x", "pos_y", "pos_z")} | {
        "tri": to_np(a.plane("tri"), np.uint32)}


def assert_atlas_equal(a: lcl.Atlas, o: oracle.Atlas, rows=None):
    y0, y1 = (0, a.height) if rows is None else rows
    p = atlas_planes(a)
    assert np.array_equal(p["tri"][y0:y1], o.tri), "triangle plane differs"
    assert np.array_equal(p["pos_x"][y0:y1], o.px), "pos_x differs"
    assert np.array_equal(p["pos_y"][y0:y1], o.py), "pos_y differs"
    assert np.array_equal(p["pos_z"][y0:y1], o.pz), "pos_z differs"


def sphere_recs(o: oracle.Atlas, strokes):
    return oracle.sphere_records(o.mn, o.S, strokes.centre, strokes.radius, strokes.label)
