"""The sparse layer pool (Section 4.2: the texture manager's arrays keyed by (width, height, type),
sparse textures that reserve room for many layers and commit memory only for layers in use) on the
GPU: reservation without commitment, zeroed layers, stable addresses, slot reuse, full arrays, and
edits on pool layers identical to the same edits on ordinary device tensors."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import DEV, gpu_atlas

pytestmark = pytest.mark.gpu

from paper_2501_14807_gb300 import lcl  # noqa: E402


def test_pool_reserves_much_and_commits_only_live_layers():
    pool = lcl.Pool(max_layers_per_array=4096)
    try:
        a = pool.acquire(4096, 4096, "u8")
        st = pool.stats()
        g = st["granularity"]
        slot = -(-4096 * 4096 // g) * g
        assert st["arrays"] == 1 and st["layers"] == 1
        assert st["committed_bytes"] == slot and st["reserved_bytes"] == 4096 * slot   # 64 GiB of addresses
        b = pool.acquire(384, 384, "f32")
        c = pool.acquire(300, 170, "u16")
        st = pool.stats()
        assert st["arrays"] == 3 and st["layers"] == 3
        assert st["committed_bytes"] % g == 0 and st["committed_bytes"] < 3 * slot
        torch.cuda.synchronize()
        for L in (a, b, c):
            assert int(L.data.view(torch.uint8).count_nonzero()) == 0
        assert b.mask is not None and int(b.mask.count_nonzero()) == 0 and a.mask is None
        for L in (a, b, c):
            pool.release(L)
        assert pool.stats()["committed_bytes"] == 0 and pool.stats()["layers"] == 0
    finally:
        pool.destroy()


def test_pool_slots_are_reused_zeroed_and_addresses_stay():
    pool = lcl.Pool(max_layers_per_array=3)
    try:
        L = [pool.acquire(256, 128, "u8") for _ in range(3)]
        ptrs = [x.data.data_ptr() for x in L]
        assert len(set(ptrs)) == 3
        with pytest.raises(lcl.LclError) as e:
            pool.acquire(256, 128, "u8")                    # every slot of the array in use
        assert e.value.status == 2
        for x in L:
            x.data.fill_(7)
        pool.release(L[1])
        again = pool.acquire(256, 128, "u8")
        torch.cuda.synchronize()
        assert again.data.data_ptr() == ptrs[1]             # the freed slot, at the same address
        assert int(again.data.count_nonzero()) == 0        # cleared on acquire
        assert L[0].data.data_ptr() == ptrs[0] and int((L[0].data == 7).sum()) == 256 * 128
        stale = L[1].handle
        with pytest.raises(lcl.LclError):
            lcl._check("lcl_pool_release", lcl.library().lcl_pool_release(pool.ptr, stale + 5, None))
    finally:
        pool.destroy()


def test_edits_on_pool_layers_equal_edits_on_tensors():
    mesh = synth.vessel_charts(120, 60, 20, 10, 512, seed=8)
    W = H = 512
    m, a = gpu_atlas(mesh, W, H, 32)
    o = oracle.Atlas(mesh, W, H, tile=32)
    st = synth.sphere_strokes(mesh, 30, 5, 0.02, 0.3, 1, 200)
    recs = oracle.sphere_records(o.mn, o.S, st.centre, st.radius, st.label)
    recs["flags"][::4] = lcl.pad_flags(2, 2)
    pool = lcl.Pool(max_layers_per_array=8)
    try:
        lab = pool.acquire(W, H, "u8")
        ref = torch.zeros((H, W), dtype=torch.uint8, device=DEV)
        lcl.lcl_select_sphere(a, lab.data, recs)
        lcl.lcl_select_sphere(a, ref, recs)
        num = pool.acquire(W, H, "f32")
        ref_num = lcl.NumericLayer(W, H, "f32", DEV)
        vals = recs.copy()
        vals["label"] = np.random.default_rng(3).uniform(-5, 5, len(vals)).astype(np.float32).view(np.uint32)
        lcl.lcl_numeric_sphere(a, num.numeric, vals)
        lcl.lcl_numeric_sphere(a, ref_num, vals)
        torch.cuda.synchronize()
        assert torch.equal(lab.data, ref) and int(ref.count_nonzero()) > 0
        assert torch.equal(num.data, ref_num.data)
        n_words = (W * H + 31) // 32
        assert torch.equal(num.mask[:n_words], ref_num.mask[:n_words])
        c1, a1 = lcl.lcl_label_area(a, lab.data, 256)
        c2, a2 = lcl.lcl_label_area(a, ref, 256)
        assert torch.equal(c1, c2) and torch.equal(a1, a2)
    finally:
        pool.destroy()
