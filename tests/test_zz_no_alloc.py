"""lcl_select_sphere_static -- the sphere brush for callers that cannot allocate device memory
while they edit (a plugin inside a host application that owns the device memory, or an
interactive stroke loop that must not wait on an allocator or fail mid-stroke) -- called through
the C ABI and compared, bit for bit, with lcl_select_sphere given an ordinary workspace.

Two calls in a row with different strokes check that the shared scratch array, which keeps the
previous call's contents, is cleared where it must be.  The file sorts last so that a run that
stops at the first failure has already run every other test; it passes alone in a fresh process
(where its first call sets up the scratch address) and after the other tests."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from paper_2501_14807_gb300 import lcl

pytestmark = pytest.mark.gpu


def _records(atlas, strokes):
    return np.stack([lcl.lcl_quantize_sphere(atlas, strokes.centre[k], strokes.radius[k], strokes.label[k])
                     for k in range(len(strokes.radius))])


@pytest.mark.parametrize("dt", [torch.uint8, torch.int16])
def test_static_scratch_matches_workspace_entry_point_on_two_calls(dt):
    lib = lcl.library()
    mesh = synth.vessel_cylindrical(80, 30, noise_amp=0.02, seed=12)
    W, H, T = 512, 384, 32
    m = lcl.Mesh.from_host(mesh, "cuda")
    a = lcl.Atlas(W, H, T, mesh.n_tri, "cuda")
    lcl.lcl_atlas_build(m, a)
    code = lcl.LCL_U8 if dt == torch.uint8 else lcl.LCL_U16
    top = 255 if dt == torch.uint8 else 30000
    init = torch.randint(0, 9, (H, W), dtype=torch.int32).to(dt).cuda()
    ref_layer, new_layer = init.clone(), init.clone()
    stream = torch.cuda.current_stream().cuda_stream
    for call, (seed, n, rlo, rhi) in enumerate([(21, 40, 0.01, 0.3), (22, 25, 0.05, 0.6)]):
        recs = np.ascontiguousarray(_records(a, synth.sphere_strokes(mesh, n, seed, rlo, rhi, 1, top)),
                                    dtype=lcl.SPHERE_DTYPE)
        ref_hits = torch.zeros(n, dtype=torch.int64, device="cuda")
        new_hits = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        lcl.lcl_select_sphere(a, ref_layer, recs, hits_out=ref_hits)
        status = lib.lcl_select_sphere_static(C.byref(a.c), C.c_void_p(new_layer.data_ptr()), code,
                                              recs.ctypes.data_as(C.c_void_p), n,
                                              C.c_void_p(new_hits.data_ptr()), C.c_void_p(stream))
        assert status == 0, lcl.lcl_last_error()
        torch.cuda.synchronize()
        assert torch.equal(new_layer, ref_layer), f"call {call}: layers differ"
        assert torch.equal(new_hits, ref_hits), f"call {call}: hit counts differ"
        assert int(ref_hits.sum()) > 0


def test_static_scratch_rejects_sizes_beyond_its_maximum():
    lib = lcl.library()
    # An atlas of 16384 x 16384 at tile 16 has 1,048,576 tiles, above the 262,144 the array holds.
    # The check runs on the host before anything touches the (placeholder) buffer.
    big = lcl.lcl_atlas()
    nb = lib.lcl_atlas_bytes(16384, 16384, 16, 10)
    assert lib.lcl_atlas_bind(C.c_void_p(1 << 44), nb, 16384, 16384, 16, 10, C.byref(big)) == 0
    recs = np.zeros(1, lcl.SPHERE_DTYPE)
    st = lib.lcl_select_sphere_static(C.byref(big), C.c_void_p(1 << 45), lcl.LCL_U8,
                                      recs.ctypes.data_as(C.c_void_p), 1, None, None)
    assert st == 4 and "262144" in lcl.lcl_last_error()
    recs = np.zeros(4097, lcl.SPHERE_DTYPE)
    small = lcl.lcl_atlas()
    nb = lib.lcl_atlas_bytes(64, 64, 16, 10)
    assert lib.lcl_atlas_bind(C.c_void_p(1 << 44), nb, 64, 64, 16, 10, C.byref(small)) == 0
    st = lib.lcl_select_sphere_static(C.byref(small), C.c_void_p(1 << 45), lcl.LCL_U8,
                                      recs.ctypes.data_as(C.c_void_p), 4097, None, None)
    assert st == 4 and "4096" in lcl.lcl_last_error()
