"""Host logic of bench.py, on the CPU: where the roofline's peak and DRAM-traffic figures come from,
and the per-row algorithmic bytes and fractions."""
import hashlib
import json
import os
from types import SimpleNamespace

import numpy as np
import pytest

import bench


def _root_with(tmp_path, select_src=b"// kernel source\n", traffic=None, peaks=None):
    csrc = tmp_path / "paper_2501_14807_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "select.cu").write_bytes(select_src)
    (tmp_path / "profiles").mkdir()
    if traffic is not None:
        (tmp_path / "profiles" / "sphere_group_traffic.json").write_text(json.dumps(traffic))
    if peaks is not None:
        (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps(peaks))
    return str(tmp_path)


def test_traffic_is_reported_only_for_the_captured_source_and_workload(tmp_path, monkeypatch):
    src = b"__global__ void k() {}\n"
    sha = hashlib.sha256(src).hexdigest()[:16]
    rec = {"workload": "vessel-8M-16384sq-u8", "select_cu_sha256_16": sha, "dram_bytes_per_launch": 123}
    monkeypatch.setattr(bench, "ROOT", _root_with(tmp_path, src, traffic=rec))
    assert bench.profile_traffic(SimpleNamespace(name="vessel-8M-16384sq-u8")) == 123
    assert bench.profile_traffic(SimpleNamespace(name="vessel-2M-8192sq-u8")) is None
    (tmp_path / "paper_2501_14807_gb300" / "csrc" / "select.cu").write_bytes(src + b"// changed\n")
    assert bench.profile_traffic(SimpleNamespace(name="vessel-8M-16384sq-u8")) is None


def test_traffic_absent_is_null(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", _root_with(tmp_path))
    assert bench.profile_traffic(SimpleNamespace(name="vessel-8M-16384sq-u8")) is None


def test_peak_is_the_measured_copy_bandwidth_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", _root_with(tmp_path, peaks={"hbm_gbs": 6792.4, "bf16_tflops": 1900}))
    assert bench.peaks() == (6792.4, "measured")
    other = tmp_path / "other"
    other.mkdir()
    monkeypatch.setattr(bench, "ROOT", _root_with(other))
    assert bench.peaks() == (bench.FALLBACK_HBM_GBS, "fallback")


def _stub_workload(s=1):
    mesh = SimpleNamespace(pos=np.zeros((10, 3), np.float32), uv=np.zeros((12, 2), np.float32),
                           tri_pos=np.zeros((7, 3), np.uint32), tri_uv=np.zeros((7, 3), np.uint32), n_tri=7)
    cams = [SimpleNamespace(width=64, height=32), SimpleNamespace(width=16, height=16)]
    return SimpleNamespace(dtype_bytes=s, width=128, height=64, mesh=mesh, cams=cams,
                           lassos=[SimpleNamespace(cam=0), SimpleNamespace(cam=1), SimpleNamespace(cam=0)],
                           strokes=SimpleNamespace(radius=np.zeros(5)), overlays=[("xor", 0, 1)], n_layers=3)


@pytest.mark.parametrize("s", [1, 2])
def test_row_rooflines_units(s):
    w = _stub_workload(s)
    n = 128 * 64
    row_ms = [2.0, 4.0, 1.0, 3.0, 0.5, 1.5]          # per row, summed over 2 steps
    out = bench.row_rooflines(w, row_ms, 2, 1000 * (12 + s), 1000, 300, 5000.0)
    assert list(out) == list(bench.ROWS)
    expect = {
        "sphere": 1000 * (12 + s),
        "lasso": 300 * (12 + s) + (64 * 32 + 16 * 16 + 64 * 32) * 4,
        "overlay": n * (3 * s + 1 / 8),
        "area": 3 * (n * (s + 4) + 8 * 7),
    }
    for name, ms in zip(bench.ROWS, row_ms):
        r = out[name]
        assert r["ms_per_step"] == ms / 2
        assert r["gb_s"] == pytest.approx(r["algorithmic_bytes"] / (ms / 2 / 1e3) / 1e9)
        if name in expect:
            assert r["algorithmic_bytes"] == int(expect[name])
            assert r["bound"] == "hbm" and r["frac"] == pytest.approx(r["gb_s"] / 5000.0)
        else:
            assert r["bound"] == "raster" and "frac" not in r


def test_all_cores_oracle_sample_equals_its_bands_run_one_by_one():
    """The all-cores CPU baseline runs the same oracle on row bands in threads: its texel count must
    equal the single-threaded sample of each band added up (a 512^2 version of the roofline model,
    with lassos on its depth maps)."""
    import synth
    w = synth.config_roofline(n_strokes=12, n_lassos=3, depth_side=256, n_theta=88, n_h=44, side=512)
    texels, secs, bands = bench.oracle_sample_cores(w, 24, 3)
    assert bands == 3 and secs > 0
    assert texels == sum(bench.oracle_sample(w, 24, y0=24 * k)[0] for k in range(3))
    assert texels > 3 * 24 * 512 * (len(w.overlays) + w.n_layers)    # full-row passes plus some hits


def test_sphere_inside_texels_counts_covered_texels_of_contained_tiles():
    """bench.sphere_inside_texels: per stroke, the covered texels of the tiles whose box the sphere
    contains (farthest corner within r), checked against a plain loop; padded strokes count 0."""
    import numpy as np
    import torch

    import bench
    rng = np.random.default_rng(5)
    n_tiles = 300
    lo = rng.integers(0, 1000, size=(n_tiles, 3))
    hi = lo + rng.integers(0, 60, size=(n_tiles, 3))
    cnt = rng.integers(0, 1025, size=n_tiles)
    cnt[::7] = 0
    tb = np.zeros((n_tiles, 8), np.int32)
    tb[:, 0:3], tb[:, 3], tb[:, 4:7] = lo, cnt, hi

    class FakeAtlas:
        def tile_box(self):
            return torch.from_numpy(tb)

    from paper_2501_14807_gb300 import lcl
    recs = np.zeros(40, lcl.SPHERE_DTYPE)
    recs["cx"], recs["cy"], recs["cz"] = rng.integers(0, 1100, size=(3, 40))
    recs["r2"] = rng.integers(0, 400 ** 2, size=40)
    recs["flags"][5] = 0x21
    got = bench.sphere_inside_texels(FakeAtlas(), recs, "cpu", chunk=7)
    for k, r in enumerate(recs):
        c = np.array([r["cx"], r["cy"], r["cz"]])
        far = np.maximum(c - lo, hi - c)
        exp = int(cnt[((far ** 2).sum(1) <= r["r2"]) & (cnt > 0)].sum()) if not (r["flags"] & 15) else 0
        assert got[k] == exp
    assert got.sum() > 0
    assert bench.sphere_bytes(10, 4, 1) == 6 * 13 + 4 * 1.125


def test_sphere_group_bytes_against_a_plain_loop():
    """bench.sphere_group_bytes: per group of strokes, tiles reached by some stroke cost label bytes per
    covered texel, tiles some stroke's surface crosses 12 B more, tiles only contained 1/8 B more;
    checked against a plain per-tile loop."""
    import numpy as np
    import torch

    import bench
    rng = np.random.default_rng(8)
    n_tiles = 200
    lo = rng.integers(0, 1000, size=(n_tiles, 3))
    hi = lo + rng.integers(0, 80, size=(n_tiles, 3))
    cnt = rng.integers(0, 1025, size=n_tiles)
    cnt[::9] = 0
    tb = np.zeros((n_tiles, 8), np.int32)
    tb[:, 0:3], tb[:, 3], tb[:, 4:7] = lo, cnt, hi

    class FakeAtlas:
        def tile_box(self):
            return torch.from_numpy(tb)

    from paper_2501_14807_gb300 import lcl
    recs = np.zeros(23, lcl.SPHERE_DTYPE)
    recs["cx"], recs["cy"], recs["cz"] = rng.integers(0, 1100, size=(3, 23))
    recs["r2"] = rng.integers(0, 500 ** 2, size=23)
    got, groups = bench.sphere_group_bytes(FakeAtlas(), recs, "cpu", 2, group=8)
    assert groups == 3
    exp = 0.0
    for g0 in range(0, 23, 8):
        for t in range(n_tiles):
            if cnt[t] == 0:
                continue
            reach = cross = False
            for r in recs[g0:g0 + 8]:
                c = np.array([r["cx"], r["cy"], r["cz"]])
                near = np.maximum(np.maximum(lo[t] - c, c - hi[t]), 0)
                far = np.maximum(c - lo[t], hi[t] - c)
                if (near ** 2).sum() <= r["r2"]:
                    reach = True
                    if (far ** 2).sum() > r["r2"]:
                        cross = True  # the sphere's surface crosses the tile
            if reach:
                exp += cnt[t] * 2 + (cnt[t] * 12 if cross else cnt[t] / 8)
    assert abs(got - exp) < 1e-6 * exp and exp > 0


def test_large_model_summary_from_the_child_run():
    child = {"config": {"workload": "vessel-1M-charts-4096sq-u16: ..."}, "value": 123.0, "unit": "Gtexels/s",
             "ms_per_step": 40.0, "steps": 5, "warmup": 3, "dtype": "int64",
             "rows": {"sphere": {"ms_per_step": 20.0, "frac": 0.5, "what": "x"}, "atlas": {"ms_per_step": 3.0}},
             "roofline": {"frac_of_group_bytes": 0.3}, "e2e": {"value": 100.0}, "gpu_launches": 77,
             "clocks": {"sm_mhz": 2070.0}}
    out = "warning line\n" + json.dumps({"value": 1}) + "\n" + json.dumps(child) + "\n"
    s = bench.parse_large(0, out, "")
    assert s["value"] == 123.0 and s["ms_per_step"] == 40.0 and s["dtype"] == "int64"
    assert s["rows"] == {"sphere": {"ms_per_step": 20.0, "frac": 0.5}, "atlas": {"ms_per_step": 3.0}}
    assert s["sphere_frac_of_group_bytes"] == 0.3 and s["e2e"] == 100.0 and s["gpu_launches"] == 77
    # a failed child run is reported, not raised
    bad = bench.parse_large(1, "", "Traceback ...\nRuntimeError: out of memory\n")
    assert "error" in bad and "out of memory" in bad["error"]
    assert "error" in bench.parse_large(0, "no json here\n", "")


def test_latency_split_of_served_requests():
    R = lambda a, l, d, g: SimpleNamespace(t_arrive=a, t_launch=l, t_done=d, t_gpu=g)  # noqa: E731
    reqs = [R(0.0, 0.001, 0.003, 0.0005) for _ in range(99)] + [R(0.0, 0.050, 0.052, 0.002)]
    s = bench.latency_split(reqs)
    assert s["arrival_to_launch_p50_p99"][0] == 1.0 and 1.0 < s["arrival_to_launch_p50_p99"][1] <= 50.0
    assert s["launch_to_done_p50_p99"] == [2.0, 2.0]
    assert s["epoch_gpu_p50_p99_max"][0] == 0.5 and s["epoch_gpu_p50_p99_max"][2] == 2.0
    # no GPU times (a server that could not time its epochs): that part is null
    assert bench.latency_split([R(0.0, 0.001, 0.002, -1.0)])["epoch_gpu_p50_p99_max"] is None
