"""Benchmark: one step = one pass of the whole layer-editing path over one model.

Workload (default): the roofline-size model -- a displaced vessel of 2828 x 1414 quads
(~8M triangles) with a cylindrical unwrap into a 16384 x 16384 atlas (int32 x3 positions
+ uint32 triangle ids, 4.3 GB, far larger than L2) and 4 uint8 layers.  One step runs,
through the C ABI:
  atlas build (quantise, UV rasterise, interpolate, boxes, area weights)
  1000 sphere strokes (radii log-uniform 1-30% of the bbox diagonal), one call per layer,
      one launch per stroke (it applies its stroke and culls the next)
  4 depth maps (2048^2) and 20 star lassos on them
  XOR(L0, L1) and OR(L2, L3) overlays, per-label area (256 labels) of the 4 layers

Metric: layer texels processed per second -- every texel an edit selected, plus every
texel of each overlay and each area query -- over the whole step.  The roofline object is
for the sphere edits (the dominant kernels): algorithmic bytes = hit texels x (12 B of
position + 1 B of label), over their CUDA-event time, against the measured HBM copy peak.

With N GPUs (torchrun, one rank each) the texture is split into N row bands (tile rows dealt
out evenly): each rank builds its band atlas, applies every stroke and lasso to its rows, runs the
overlays and area queries on them and sums the area tables with one all-reduce per step; texels
add up over ranks and the slowest rank sets the time (strong scaling: the total work is fixed).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "layer-edit Gtexels/s and % of HBM roofline; p50/p99 edit latency (serving)"
UNIT = "Gtexels/s"
FALLBACK_HBM_GBS = 6800.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def make_workload(args):
    import synth
    if args.config == "roofline":
        return synth.config_roofline(n_strokes=args.strokes, n_lassos=args.lassos)
    if args.config == "large":
        return synth.config_large(n_strokes=args.strokes, n_lassos=args.lassos)
    if args.config == "mid":   # a smaller version of the roofline model (default 4096^2), for quick runs and profiles
        side = args.atlas_side or 4096
        return synth.config_roofline(n_strokes=args.strokes, n_lassos=args.lassos, n_theta=round(2828 * side / 16384),
                                     n_h=round(1414 * side / 16384), side=side)
    return synth.config_small()


def workload_desc(w, args):
    return {
        "workload": f"{w.name}: {w.mesh.n_tri} triangles, {w.width}x{w.height} atlas (tile {w.tile}), "
                    f"{w.n_layers} x u{8 * w.dtype_bytes} layers, {len(w.strokes.radius)} sphere strokes, "
                    f"{len(w.lassos)} lassos on {len(w.cams)} depth maps, overlays "
                    f"{'/'.join(o[0] for o in w.overlays)}, per-label area x{w.n_layers}",
        "atlas": f"{w.width}x{w.height}",
        "n_tri": w.mesh.n_tri,
        "layers": w.n_layers,
        "strokes": int(len(w.strokes.radius)),
        "lassos": len(w.lassos),
        "n_labels": w.n_labels,
        "l2": "inputs larger than L2" if w.width * w.height * 16 > 129e6 else "inputs smaller than L2",
    }


# ---------------------------------------------------------------------------------------
# CPU baseline / reference arm: the oracle, as it stands, on a bounded row band
# ---------------------------------------------------------------------------------------

def _oracle_band(w, y0, y1, mn, S, recs, ms, dms):
    """The oracle over texture rows [y0, y1) of the workload: the same strokes, the lassos of the
    cameras in ms / dms (with their full depth maps), overlays and area queries.  Returns texels."""
    import oracle
    rows = y1 - y0
    o = oracle.Atlas(w.mesh, w.width, w.height, tile=w.tile, y0=y0, y1=y1, quant=(mn, S))
    dt = np.uint8 if w.dtype_bytes == 1 else np.uint16
    layers = [np.zeros((rows, w.width), dt) for _ in range(w.n_layers)]
    texels = 0
    for li in range(w.n_layers):
        sel = np.nonzero(w.strokes.layer == li)[0]
        texels += int(oracle.select_sphere(o, layers[li], recs[sel]).sum())
    for L in w.lassos:
        if L.cam >= len(ms):
            continue
        h, _ = oracle.select_lasso(o, layers[L.layer], ms[L.cam], dms[L.cam], L.poly, L.label, want_ambiguous=False)
        texels += h
    for op, ia, ib in w.overlays:
        oracle.overlay(o, layers[ia], layers[ib], op)
        texels += rows * w.width
    for li in range(w.n_layers):
        oracle.label_area(o, layers[li], w.n_labels)
        texels += rows * w.width
    return texels


def oracle_sample(w, rows, n_cams_used=None, y0=0):
    """Runs the oracle over texture rows [y0, y0 + rows) of the workload: the same strokes, lassos
    (with their full depth maps), overlays and area queries.  Returns (texels, seconds)."""
    import oracle
    t0 = time.perf_counter()
    mn, S = oracle.quant_params(w.mesh.pos)
    recs = oracle.sphere_records(mn, S, w.strokes.centre, w.strokes.radius, w.strokes.label)
    cams = w.cams if n_cams_used is None else w.cams[:n_cams_used]
    ms = [oracle.camera_mq(c.vp, mn, S) for c in cams]
    dms = [oracle.depth(w.mesh, mn, S, m, c.width, c.height) for m, c in zip(ms, cams)]
    texels = _oracle_band(w, y0, y0 + rows, mn, S, recs, ms, dms)
    return texels, time.perf_counter() - t0


def oracle_sample_cores(w, rows, n_threads):
    """The same plain oracle on all host cores: the depth maps once, one thread per camera, then
    row bands [k rows, (k + 1) rows), one thread each (the C oracle runs without the GIL; each band
    has its own atlas rows and layers).  Returns (texels, seconds, bands)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    t0 = time.perf_counter()
    mn, S = oracle.quant_params(w.mesh.pos)
    recs = oracle.sphere_records(mn, S, w.strokes.centre, w.strokes.radius, w.strokes.label)
    ms = [oracle.camera_mq(c.vp, mn, S) for c in w.cams]
    bands = [(k * rows, min((k + 1) * rows, w.height)) for k in range(max(n_threads, 1)) if k * rows < w.height]
    with ThreadPoolExecutor(max(n_threads, 1)) as ex:
        dms = list(ex.map(lambda mc: oracle.depth(w.mesh, mn, S, mc[0], mc[1].width, mc[1].height), zip(ms, w.cams)))
        texels = sum(ex.map(lambda b: _oracle_band(w, b[0], b[1], mn, S, recs, ms, dms), bands))
    return texels, time.perf_counter() - t0, len(bands)


def cpu_baseline(w, rows):
    texels, secs = oracle_sample(w, rows)
    return {"value": texels / secs / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"texture rows [0, {rows}) of the same workload ({rows * w.width} texels): all strokes, "
                      f"lassos (full depth maps), overlays and area queries; {texels} texels in {secs:.2f} s, "
                      f"single-threaded C (-O2)"}


def cpu_baseline_all_cores(w, rows):
    """The oracle on every host core (row bands of `rows` rows, one thread each); a failure is
    reported in the line instead of ending the run."""
    try:
        n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        texels, secs, bands = oracle_sample_cores(w, rows, n)
    except Exception as e:  # the single-threaded baseline above stands either way
        return {"kind": "oracle", "error": f"{type(e).__name__}: {e}"[:200]}
    return {"value": texels / secs / 1e9, "unit": UNIT, "cores": bands, "kind": "oracle",
            "sample": f"texture rows [0, {bands * rows}) of the same workload in {bands} bands of {rows} rows, one "
                      f"thread each, after the depth maps (one thread per camera): {texels} texels in {secs:.2f} s, "
                      f"the same C as the single-threaded baseline"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(args)
    rows = args.cpu_rows
    for _ in range(args.warmup):
        oracle_sample(w, rows)
    tot_t, tot_x = 0.0, 0
    times = []
    for _ in range(args.steps):
        x, s = oracle_sample(w, rows)
        tot_t += s
        tot_x += x
        times.append(s)
    val = tot_x / tot_t / 1e9
    cb = {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
          "sample": f"texture rows [0, {rows}) of the workload per step ({rows * w.width} texels), all strokes, "
                    f"lassos, overlays and area queries; single-threaded C oracle"}
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": workload_desc(w, args), "cpu_baseline": cb,
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------

class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2501_14807_gb300 import lcl, shard

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = make_workload(args)
    W, H = w.width, w.height
    cpu = cpu_baseline(w, args.cpu_rows) if (rank == 0 and world == 1 and args.cpu_rows > 0) else None
    cpu_all = cpu_baseline_all_cores(w, args.cpu_rows) if cpu is not None else None

    # N ranks split the texture into row bands (one band atlas and the same rows of every layer per
    # rank; every stroke, lasso and depth map on every rank; the area tables summed over ranks)
    y0, y1 = shard.band_rows(H, w.tile, world, rank) if world > 1 else (0, H)
    rows = y1 - y0
    mesh = lcl.Mesh.from_host(w.mesh, dev)
    atlas = lcl.Atlas(W, H, w.tile, w.mesh.n_tri, dev, band=(y0, y1) if world > 1 else None)
    ws_atlas = torch.empty(lcl.lcl_atlas_workspace_bytes(mesh, W, rows), dtype=torch.uint8, device=dev)
    lcl.lcl_atlas_build(mesh, atlas, ws_atlas)
    lt = torch.uint8 if w.dtype_bytes == 1 else torch.int16
    layers = [torch.zeros((rows, W), dtype=lt, device=dev) for _ in range(w.n_layers)]
    outs = [torch.empty((rows, W), dtype=lt, device=dev) for _ in w.overlays]
    per_layer = []
    for li in range(w.n_layers):
        sel = np.nonzero(w.strokes.layer == li)[0]
        recs = np.stack([lcl.lcl_quantize_sphere(atlas, w.strokes.centre[k], w.strokes.radius[k],
                                                 w.strokes.label[k]) for k in sel]) if len(sel) else \
            np.zeros(0, lcl.SPHERE_DTYPE)
        per_layer.append(np.ascontiguousarray(recs, dtype=lcl.SPHERE_DTYPE))
    n_strokes = sum(len(r) for r in per_layer)
    ws_sel = torch.empty(lcl.lcl_select_workspace_bytes(atlas, max(len(r) for r in per_layer)), dtype=torch.uint8,
                         device=dev)
    sphere_hits = [torch.zeros(max(len(r), 1), dtype=torch.int64, device=dev) for r in per_layer]
    inside_per_layer = [sphere_inside_texels(atlas, r, dev) for r in per_layer]
    # every layer's strokes are one call of >= 2 unpadded strokes: the grouped path
    grouped = [sphere_group_bytes(atlas, r, dev, w.dtype_bytes) for r in per_layer]
    assert all(len(r) >= 2 and not (r["flags"] & 15).any() for r in per_layer)
    torch.cuda.empty_cache()
    cams = [lcl.lcl_camera_from_vp(atlas, c.vp, c.width, c.height) for c in w.cams]
    depths = [torch.empty((c.height, c.width), dtype=torch.float32, device=dev) for c in w.cams]
    ws_depth = torch.empty(max([lcl.lcl_depth_workspace_bytes(mesh, c.width, c.height) for c in w.cams] + [256]),
                           dtype=torch.uint8, device=dev)
    lasso_hits = torch.zeros(max(len(w.lassos), 1), dtype=torch.int64, device=dev)
    table_buf = torch.empty(2 * w.n_layers * w.n_labels, dtype=torch.int64, device=dev)   # counts | areas
    counts = [table_buf[li * w.n_labels:(li + 1) * w.n_labels] for li in range(w.n_layers)]
    areas = [table_buf[(w.n_layers + li) * w.n_labels:(w.n_layers + li + 1) * w.n_labels] for li in range(w.n_layers)]
    stream = torch.cuda.current_stream(dev)

    # one event at each boundary between the rows of a step (recorded on the launching stream)
    ev_rows = [torch.cuda.Event(enable_timing=True) for _ in range(len(ROWS) + 1)]

    def step(mesh_dev, timed=False):
        mark = (lambda i: ev_rows[i].record(stream)) if timed else (lambda i: None)
        mark(0)
        lcl.lcl_atlas_build(mesh_dev, atlas, ws_atlas, stream)
        mark(1)
        for li, layer in enumerate(layers):
            lcl.lcl_select_sphere(atlas, layer, per_layer[li], sphere_hits[li], ws_sel, stream)
        mark(2)
        for ci, cam in enumerate(cams):
            lcl.lcl_depth_render(mesh_dev, atlas, cam, depths[ci], ws_depth, stream)
        mark(3)
        for k, L in enumerate(w.lassos):
            lcl.lcl_select_lasso(atlas, layers[L.layer], cams[L.cam], depths[L.cam], L.poly, L.label,
                                 lcl.DEFAULT_BIAS, lasso_hits[k:k + 1], ws_sel, stream)
        mark(4)
        for oi, (op, ia, ib) in enumerate(w.overlays):
            lcl.lcl_overlay(atlas, layers[ia], layers[ib], outs[oi], op, 0, stream)
        mark(5)
        for li, layer in enumerate(layers):
            lcl.lcl_label_area(atlas, layer, w.n_labels, counts[li], areas[li], stream)
        if world > 1:   # the whole texture's tables: one all-reduce of the integer sums
            shard.reduce_tables([table_buf])
        mark(6)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step(mesh)
    barrier()

    # texels per step (identical every step: the same strokes on the same atlas)
    sph_hits = sum(int(h[:len(r)].sum().item()) for h, r in zip(sphere_hits, per_layer))
    las_hits = int(lasso_hits[:len(w.lassos)].sum().item())
    las_each = [int(x) for x in lasso_hits[:len(w.lassos)].tolist()]  # per lasso, in launch order
    texels = sph_hits + las_hits + (len(w.overlays) + w.n_layers) * W * rows

    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = lcl.lcl_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    row_ms = [0.0] * len(ROWS)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step(mesh, timed=True)
        e1.record(stream)
        e1.synchronize()
        for i in range(len(ROWS)):
            row_ms[i] += ev_rows[i].elapsed_time(ev_rows[i + 1])
    sph_ms = row_ms[ROWS.index("sphere")]
    barrier()
    e1.record(stream)
    barrier()
    total_ms = e0.elapsed_time(e1)
    launches = lcl.lcl_kernel_launches() - launches0
    clk = clocks.stop()

    # end-to-end through the public API from host buffers: mesh upload from pinned memory each
    # step, result tables (area + hit counts) read back each step
    pinned = [torch.from_numpy(np.ascontiguousarray(a).view(dt)).pin_memory()
              for a, dt in ((w.mesh.pos, np.float32), (w.mesh.uv, np.float32), (w.mesh.tri_pos, np.int32),
                            (w.mesh.tri_uv, np.int32))]
    h2d = sum(p.numel() * p.element_size() for p in pinned)
    dev_bufs = [torch.empty_like(p, device=dev) for p in pinned]
    mesh_e2e = lcl.Mesh(*dev_bufs)
    host_counts = [torch.empty(w.n_labels, dtype=torch.int64).pin_memory() for _ in range(2 * w.n_layers)]
    host_hits = [torch.empty(h.numel(), dtype=torch.int64).pin_memory() for h in sphere_hits + [lasso_hits]]
    d2h = sum(t.numel() * 8 for t in host_counts + host_hits)

    def e2e_step():
        for p, d in zip(pinned, dev_bufs):
            d.copy_(p, non_blocking=True)
        step(mesh_e2e)
        for i in range(w.n_layers):
            host_counts[2 * i].copy_(counts[i], non_blocking=True)
            host_counts[2 * i + 1].copy_(areas[i], non_blocking=True)
        for hh, dd in zip(host_hits, sphere_hits + [lasso_hits]):
            hh.copy_(dd, non_blocking=True)

    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    f1.record(stream)
    barrier()
    e2e_ms = f0.elapsed_time(f1)

    by_radius = sphere_radius_breakdown(w, atlas, layers, per_layer, inside_per_layer, ws_sel, stream, dev) \
        if rank == 0 else None

    (total_ms, e2e_ms, sph_ms), all_texels = combine_ranks([total_ms, e2e_ms, sph_ms], texels, world, dev)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    serving = serving_summary(args.serving_models, 20000.0, args.serving_seconds) \
        if (world == 1 and args.serving_models > 0) else None
    # the batching workload (256 models, 64 queued strokes each), outside the timed region
    batch = batch_summary(args.batch_models, 5, 2, torch_device=local) if (world == 1 and args.batch_models > 0) else None
    # the single large model on 16 u16 layers, as its own run in a child process
    large = large_summary(args.large_steps) if (world == 1 and args.config == "roofline" and args.large_steps > 0) \
        else None
    peak, peak_kind = peaks()
    sph_inside = int(sum(int(x.sum()) for x in inside_per_layer))
    sph_bytes = sph_hits * (12 + w.dtype_bytes)          # the per-unit bytes of the hot-path scope: 12 B + label
    n_groups = sum(g for _, g in grouped)
    grp_bytes = sum(b for b, _ in grouped)
    achieved = sph_bytes / (sph_ms / args.steps / 1e3) / 1e9
    value = all_texels * args.steps / (total_ms / 1e3) / 1e9
    traffic = profile_traffic(w)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "int64", "data": "synthetic (seeded vessels; scans unavailable)",
        "config": dict(workload_desc(w, args),
                       parallelism=(f"{world} row bands of the one texture, one per GPU (tile rows dealt out evenly; "
                                    "strokes, lassos and depth maps on every GPU; the area tables summed by one "
                                    "all-reduce per step)") if world > 1 else "1 GPU, the whole texture"),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": traffic,
                     "kernel": f"sphere edit, grouped: k_group_cull + k_group_apply per {SPHERE_GROUP} consecutive "
                               "strokes of a call (a launch = one group), timed over the whole sphere row",
                     "algorithmic_bytes_per_launch": sph_bytes / max(n_groups, 1),
                     "bytes_model": "12 B position + label per selected texel, summed over the strokes (the scope's "
                                    "per-unit bytes).  The grouped apply reads a tile's positions once per group "
                                    "(and none for tiles every stroke of the group contains: coverage bits only) "
                                    "and writes each texel once per group, so this sum exceeds the bytes moved "
                                    "and the fraction can exceed 1",
                     "hit_texels": sph_hits, "hit_texels_inside_tiles": sph_inside,
                     "strokes": n_strokes, "launches": n_groups,
                     "group_bytes_per_launch": grp_bytes / max(n_groups, 1),
                     "group_bytes_model": "per group: label bytes x covered texels of every tile a stroke reaches, "
                                          "+ 12 B x covered texels of tiles a sphere surface crosses, + 1/8 B x "
                                          "covered texels of tiles only contained (sphere_group_bytes)",
                     "frac_of_group_bytes": grp_bytes / (sph_ms / args.steps / 1e3) / 1e9 / peak,
                     "ms_per_launch": sph_ms / args.steps / max(n_groups, 1)},
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "e2e": {"value": all_texels * args.steps / (e2e_ms / 1e3) / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "serving": serving,
        "batch": batch,
        "large": large,
        "breakdown": {"sphere_ms_per_step": sph_ms / args.steps, "sphere_hit_texels": sph_hits,
                      "lasso_hit_texels": las_hits, "lasso_hit_texels_each": las_each, "texels_per_step": texels},
        "rows": row_rooflines(w, row_ms, args.steps, sph_bytes, sph_hits, las_hits, peak),
        "sphere_group_bytes": {"groups": n_groups, "bytes": grp_bytes,
                               "gb_s": grp_bytes / (sph_ms / args.steps / 1e3) / 1e9},
        "sphere_by_radius": by_radius,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


ROWS = ("atlas", "sphere", "depth", "lasso", "overlay", "area")


def sphere_inside_texels(atlas, records, dev, chunk=16):
    """Per stroke, the covered texels of the tiles whose box lies inside the stroke's sphere (the
    library selects them from the coverage bits without reading their positions): tile boxes against
    each stroke on the device, chunk strokes at a time.  Strokes with texture padding count 0 (the
    library reads positions for them).  Returns a numpy int64 array."""
    import torch
    tb = atlas.tile_box().to(torch.int64)
    lo, cnt, hi = tb[:, 0:3], tb[:, 3], tb[:, 4:7]
    out = np.zeros(len(records), np.int64)
    for k0 in range(0, len(records), chunk):
        r = records[k0:k0 + chunk]
        c = torch.tensor(np.stack([r["cx"], r["cy"], r["cz"]], 1).astype(np.int64), device=dev)[:, None, :]
        far = torch.maximum(c - lo[None], hi[None] - c)
        inside = ((far * far).sum(-1) <= torch.tensor(r["r2"].astype(np.int64), device=dev)[:, None]) & (cnt > 0)[None]
        n = (inside.to(torch.int64) * cnt[None]).sum(1).cpu().numpy()
        n[(r["flags"] & 15) != 0] = 0
        out[k0:k0 + len(r)] = n
    return out


SPHERE_GROUP = 32  # strokes per grouped launch pair of the library (k_group_cull + k_group_apply)


def sphere_group_bytes(atlas, records, dev, label_bytes, group=SPHERE_GROUP):
    """Bytes the grouped sphere apply moves at tile granularity for one call applying `records` (the
    library applies a call of two or more unpadded strokes on a label layer `group` strokes per
    launch): per group, every tile that some stroke of the group reaches costs its covered texels'
    labels; a tile that some stroke's surface crosses also costs their 12-byte positions, a tile that
    every stroke reaching it contains only their coverage bits.  Tile boxes against the strokes on
    the device, one group at a time.  Returns (bytes, groups)."""
    import torch
    tb = atlas.tile_box().to(torch.int64)
    lo, cnt, hi = tb[:, 0:3], tb[:, 3], tb[:, 4:7]
    cov = cnt > 0
    total, groups = 0.0, 0
    for g0 in range(0, len(records), group):
        r = records[g0:g0 + group]
        c = torch.tensor(np.stack([r["cx"], r["cy"], r["cz"]], 1).astype(np.int64), device=dev)[:, None, :]
        r2 = torch.tensor(np.minimum(r["r2"].astype(np.int64), 1 << 50), device=dev)[:, None]
        near = torch.clamp(torch.maximum(lo[None] - c, c - hi[None]), min=0)
        reach = ((near * near).sum(-1) <= r2) & cov[None]
        far = torch.maximum(c - lo[None], hi[None] - c)
        sure = ((far * far).sum(-1) <= r2) & reach
        any_r, cross = reach.any(0), (reach & ~sure).any(0)
        total += float((cnt * any_r).sum()) * label_bytes + float((cnt * cross).sum()) * 12 + \
            float((cnt * (any_r & ~cross)).sum()) / 8
        groups += 1
    return total, groups


def sphere_bytes(hits, inside, label_bytes):
    """Algorithmic bytes of sphere edits: a selected texel that must be tested costs its 12-byte position
    and its label; a texel of a tile inside the sphere costs its coverage bit and its label."""
    hits, inside = np.asarray(hits, np.float64), np.asarray(inside, np.float64)
    return (hits - inside) * (12 + label_bytes) + inside * (label_bytes + 1 / 8)


def row_rooflines(w, row_ms, steps, sph_bytes, sph_hits, las_hits, peak):
    """Per-row CUDA-event time of one step and, for the streaming rows, algorithmic bytes over
    that time against the HBM peak.  Bytes per unit (s = label bytes):
      sphere           hit texels x (12 + s) (sph_bytes, computed by the caller)
      lasso            hit texels x (12 + s), plus the depth map read once per lasso
      overlay          every texel x (3 s + 1/8)
      area             every texel x (s + 4), plus 8 B per triangle
      atlas            every texel x (16 + 1/8) written plus the mesh read (a rasteriser:
                       reported, not bound by HBM)
      depth            every screen pixel x 4 written plus the quantised vertices read"""
    s = w.dtype_bytes
    n = w.width * w.height
    m = w.mesh
    mesh_bytes = m.pos.nbytes + m.uv.nbytes + m.tri_pos.nbytes + m.tri_uv.nbytes
    cam_px = sum(c.width * c.height for c in w.cams)
    lasso_depth = sum(w.cams[L.cam].width * w.cams[L.cam].height * 4 for L in w.lassos)
    spec = {
        "atlas": (n * (16 + 1 / 8) + mesh_bytes, "raster", "atlas build (quantise, UV raster, resolve, boxes)"),
        "sphere": (sph_bytes, "hbm", f"{len(w.strokes.radius)} sphere strokes, {sph_hits} hit texels"),
        "depth": (cam_px * 4 + m.pos.nbytes + m.tri_pos.nbytes, "raster", f"{len(w.cams)} depth maps"),
        "lasso": (las_hits * (12 + s) + lasso_depth, "hbm", f"{len(w.lassos)} lassos, {las_hits} hit texels"),
        "overlay": (len(w.overlays) * n * (3 * s + 1 / 8), "hbm", f"{len(w.overlays)} full-layer overlays"),
        "area": (w.n_layers * (n * (s + 4) + 8 * m.n_tri), "hbm", f"{w.n_layers} per-label area queries"),
    }
    out = {}
    for name, ms in zip(ROWS, row_ms):
        b, bound, what = spec[name]
        t = ms / steps
        gbs = b / (t / 1e3) / 1e9 if t > 0 else 0.0
        r = {"ms_per_step": t, "what": what, "algorithmic_bytes": int(b), "gb_s": gbs, "bound": bound}
        if bound == "hbm":
            r["frac"] = gbs / peak
        out[name] = r
    return out


def sphere_radius_breakdown(w, atlas, layers, per_layer, inside_per_layer, ws_sel, stream, dev):
    """Per-radius breakdown of the sphere strokes, outside the timed region: every stroke again as
    its own call (zeroing, cull and apply launches), timed with CUDA events, binned by radius in
    half-decades of the bounding-box diagonal.  Bytes are 12 + label bytes per hit texel (and, beside
    them, the bytes the kernel needs, sphere_bytes), against the measured copy peak.  Small strokes are bound by launch and cull
    latency; the chained call of the timed region hides part of that.  The host queues all calls of a
    layer behind a short device-side sleep, so the intervals are GPU time, not Python launch time."""
    import torch
    from paper_2501_14807_gb300 import lcl

    peak, _ = peaks()
    pos = np.asarray(w.mesh.pos, np.float64)
    diag = float(np.linalg.norm(pos.max(0) - pos.min(0)))
    hits = torch.zeros(1, dtype=torch.int64, device=dev)
    rows = []  # (radius fraction, hit texels, ms)
    torch.cuda.synchronize(dev)
    for li, recs in enumerate(per_layer):
        sel = np.nonzero(w.strokes.layer == li)[0]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(recs) + 1)]
        hs = torch.zeros(len(recs), dtype=torch.int64, device=dev)
        # a bounded device-side sleep (about 60 us of SM cycles per call) lets the host queue every
        # call first, so that each interval is the GPU's time for its call, not the host's launch time
        with torch.cuda.stream(stream):
            torch.cuda._sleep(int(120_000 * len(recs)))
        ev[0].record(stream)
        for k in range(len(recs)):
            lcl.lcl_select_sphere(atlas, layers[li], recs[k:k + 1], hs[k:k + 1], ws_sel, stream)
            ev[k + 1].record(stream)
        torch.cuda.synchronize(dev)
        hh = hs.cpu().numpy()
        for k in range(len(recs)):
            rows.append((float(w.strokes.radius[sel[k]]) / diag, int(hh[k]), ev[k].elapsed_time(ev[k + 1]),
                         int(inside_per_layer[li][k])))
    edges = [0.0, 0.001, 0.00316, 0.01, 0.0316, 0.1, 0.316, 10.0]
    out = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        b = [r for r in rows if lo <= r[0] < hi]
        if not b:
            continue
        hit = sum(r[1] for r in b)
        ms = sum(r[2] for r in b)
        gbs = hit * (12 + w.dtype_bytes) / (ms / 1e3) / 1e9
        inside = sum(r[3] for r in b)
        out.append({"radius_of_diagonal": [lo, hi], "strokes": len(b), "hit_texels": hit, "ms": ms,
                    "us_per_stroke": 1e3 * ms / len(b), "gb_s": gbs, "frac": gbs / peak,
                    "hit_texels_inside_tiles": inside,
                    "frac_of_bytes_needed": float(sphere_bytes(hit, inside, w.dtype_bytes)) / (ms / 1e3) / 1e9 / peak})
    return {"timing": "one call per stroke (zeroing, cull, apply), CUDA events between calls queued ahead of the "
                      "GPU (GPU time per call, not host launch time); not the chained timed call",
            "bins": out}


def combine_ranks(times_ms, texels, world, device):
    """Whole-job figures over ranks: the maximum of each time and the sum of the texels (each rank
    edits its own rows of the texture, so the texels add up; the slowest rank sets the time)."""
    import torch
    import torch.distributed as dist
    tt = torch.tensor(list(times_ms), dtype=torch.float64, device=device)
    tx = torch.tensor([float(texels)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dist.all_reduce(tx, op=dist.ReduceOp.SUM)
    return tt.tolist(), tx.item()


def run_batch(args):
    """Batching workload as its own JSON line (see batch_summary)."""
    r = batch_summary(args.models or 256, args.steps, args.warmup, torch_device=0)
    line = {"metric": METRIC, "value": r["batched"]["gtexels_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["batched"]["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic", "config": r.pop("config"), "gpu_launches": 4}
    line.update(r)
    print(json.dumps(line), flush=True)


def batch_summary(n_models, steps, warmup, torch_device=0):
    """Batching workload: many models of uneven size, 64 queued sphere/lasso strokes each, edited by
    one batched launch (descriptor upload + cull + persistent apply), against the same strokes as
    per-model, per-stroke calls.  Both arms do identical work (bit-identical results, checked).
    Bytes: hit texels x (12 B position + 1 B label), the per-stroke algorithmic bytes summed over
    strokes, over the batched time, against the measured copy peak."""
    import torch

    import synth
    from paper_2501_14807_gb300 import lcl

    dev = torch.device("cuda", torch_device)
    torch.cuda.set_device(dev)
    bms = synth.config_batch(n_models, depth_side=1024)
    models, queues, layers, inits = [], [], [], []
    for bm in bms:
        mesh = lcl.Mesh.from_host(bm.mesh, dev)
        a = lcl.Atlas(bm.side, bm.side, 32, bm.mesh.n_tri, dev)
        lcl.lcl_atlas_build(mesh, a)
        cams = [lcl.lcl_camera_from_vp(a, c.vp, c.width, c.height) for c in bm.cams]
        depths = []
        for c in cams:
            d = torch.empty((c.height, c.width), dtype=torch.float32, device=dev)
            lcl.lcl_depth_render(mesh, a, c, d)
            depths.append(d)
        q = []
        for e in bm.order:
            if e >= 0:
                q.append(("sphere", lcl.lcl_quantize_sphere(a, bm.strokes.centre[e], bm.strokes.radius[e],
                                                            bm.strokes.label[e])))
            else:
                L = bm.lassos[-1 - e]
                q.append(("lasso", (cams[L.cam], depths[L.cam], L.poly, L.label, lcl.DEFAULT_BIAS)))
        layer = torch.zeros((bm.side, bm.side), dtype=torch.uint8, device=dev)
        models.append(a)
        queues.append(q)
        layers.append(layer)
    hit_bufs = [torch.zeros(len(q), dtype=torch.int64, device=dev) for q in queues]
    ws_sel = torch.empty(max(lcl.lcl_select_workspace_bytes(a, 1) for a in models), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def sequential():
        for a, q, layer, hb in zip(models, queues, layers, hit_bufs):
            for k, (kind, payload) in enumerate(q):
                if kind == "sphere":
                    lcl.lcl_select_sphere(a, layer, np.array([payload], lcl.SPHERE_DTYPE), hb[k:k + 1], ws_sel, stream)
                else:
                    cam, depth, poly, label, bias = payload
                    lcl.lcl_select_lasso(a, layer, cam, depth, poly, label, bias, hb[k:k + 1], ws_sel, stream)

    batch = lcl.Batch(list(zip(models, layers)), queues)

    def batched_default():
        batch.config = None
        lcl.lcl_batch_edit(batch, stream)

    def timed(fn, steps):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
            torch.cuda.synchronize(dev)   # the staging of a batch is reused by the next one
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    for _ in range(warmup):
        sequential()
    torch.cuda.synchronize(dev)
    ref = [l.clone() for l in layers]
    hits = int(sum(int(h.sum().item()) for h in hit_bufs))
    l0 = lcl.lcl_kernel_launches()
    seq_ms = timed(sequential, steps)
    seq_launches = (lcl.lcl_kernel_launches() - l0) // steps
    for l in layers:
        l.zero_()
    # default launch shape, then the autotuner on the uploaded batch, then one CUDA graph of the
    # tuned launch; every timed step uploads the descriptors and replays the graph
    for _ in range(warmup):
        batched_default()
        torch.cuda.synchronize(dev)
    def_ms = timed(batched_default, steps)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    lcl.lcl_batch_upload(batch, stream)
    upload_host_ms = 1e3 * (time.perf_counter() - t0)
    tuned, tune_ms = lcl.lcl_batch_tune(batch, stream, reps=2)
    graph = lcl.BatchGraph(batch.limits, tuned, batch.workspace)

    def batched():
        lcl.lcl_batch_upload(batch, stream)
        graph.replay()

    for _ in range(warmup):
        batched()
        torch.cuda.synchronize(dev)
    clocks = Clocks(torch_device)
    clocks.start()
    time.sleep(0.3)
    bat_ms = timed(batched, steps)
    clk = clocks.stop()
    same = all(torch.equal(r, l) for r, l in zip(ref, layers))
    n_strokes = sum(len(q) for q in queues)
    peak, peak_kind = peaks()
    gbs = hits * 13 / (bat_ms / 1e3) / 1e9
    return {"config": {"workload": f"batching: {len(models)} models ({sum(b.mesh.n_tri for b in bms)} triangles, "
                                   f"atlases 512^2-4096^2 u8), {n_strokes} queued strokes (48 sphere + 16 lasso "
                                   f"per model)", "mode": "batched launch (descriptor upload + CUDA graph replay "
                                                          "of the tuned shape) vs per-model per-stroke calls"},
            "batched": {"ms": bat_ms, "gtexels_s": hits / (bat_ms / 1e3) / 1e9, "config": tuned.as_dict(),
                        "graph": True, "launches": 4},
            "batched_default_shape": {"ms": def_ms, "config": lcl.batch_config().as_dict(), "graph": False},
            "upload_host_ms": upload_host_ms,
            "autotune": {"best_ms": tune_ms, "candidates": "threads 64/128/256 x split 1/2/4/8 x CTAs/SM all/half"},
            "per_stroke_calls": {"ms": seq_ms, "gtexels_s": hits / (seq_ms / 1e3) / 1e9, "launches": int(seq_launches)},
            "speedup": seq_ms / bat_ms, "identical_results": bool(same), "hit_texels": hits,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": gbs / peak, "bytes": "hit texels x 13 B, summed over strokes (per-stroke "
                                                      "algorithmic bytes; positions are read once per tile)"},
            "steps": steps, "warmup": warmup, "clocks": clk}


def serving_setup(n_models, seed=5):
    """Models of the serving workload (drawn like the batching workload) and payload samplers."""
    import synth
    from paper_2501_14807_gb300 import serve
    bms = synth.config_batch(n_models, seed=seed, depth_side=1024)
    models = [serve.ServedModel(b.mesh, b.side, b.cams, n_layers=2) for b in bms]
    # the HBM budget holds the first half of the models (the resident set: model i is the i-th most
    # popular under the Zipf law of the trace); the other half are spillover models admitted on demand
    budget = int(sum(serve.model_image_layout(m)[3] for m in models[: len(models) // 2]))

    def sphere_of(m, rng):
        st = bms[m].strokes
        k = int(rng.integers(0, len(st.radius)))
        return (st.centre[k], float(st.radius[k]), int(rng.integers(1, 256)))

    def lasso_of(m, rng):
        L = bms[m].lassos[int(rng.integers(0, len(bms[m].lassos)))]
        return (L.cam, L.poly, int(rng.integers(1, 256)))

    return models, budget, sphere_of, lasso_of


def latency_split(reqs):
    """Where the served requests' time goes, in ms (p50 and p99): arrival -> their epoch's launch
    (queued on the host: admissions, epochs in flight), launch -> the host seeing the epoch complete,
    and the GPU time of the epoch itself (events around its work; -1 where unavailable)."""
    t = np.array([r.t_arrive for r in reqs])
    t_l = np.array([r.t_launch for r in reqs])
    t_g = np.array([r.t_gpu for r in reqs])
    wait, after = t_l - t, np.array([r.t_done for r in reqs]) - t_l
    ok = t_g >= 0
    return {
        "arrival_to_launch_p50_p99": [round(1e3 * float(np.percentile(wait, q)), 3) for q in (50, 99)],
        "launch_to_done_p50_p99": [round(1e3 * float(np.percentile(after, q)), 3) for q in (50, 99)],
        "epoch_gpu_p50_p99_max": ([round(1e3 * float(np.percentile(t_g[ok], q)), 3) for q in (50, 99)] +
                                  [round(1e3 * float(t_g[ok].max()), 3)]) if ok.any() else None}


def native_serving_run(models, budget, sphere_of, lasso_of, rate, duration, seed=5):
    """One open-loop run of the native server (lcl_serve_*) after a 0.2 s warm-up trace: latency
    statistics (overall, per second of arrival, hot half vs spillover models) and the server's
    counters over the timed trace."""
    from paper_2501_14807_gb300 import serve
    srv = serve.NativeServer(models, hbm_budget_bytes=budget)
    try:
        srv.run(serve.poisson_requests(len(models), rate, 0.2, seed + 1, sphere_of=sphere_of, lasso_of=lasso_of))
        reqs = serve.poisson_requests(len(models), rate, duration, seed, sphere_of=sphere_of, lasso_of=lasso_of)
        s0 = srv.stats()
        srv.run(reqs)
        s1 = srv.stats()
    finally:
        srv.close()
    st = serve.latency_stats(reqs)
    lat = np.array([r.t_done - r.t_arrive for r in reqs])
    t = np.array([r.t_arrive for r in reqs])
    cold = np.array([r.model >= len(models) // 2 for r in reqs])
    st.update({k: int(s1[k] - s0[k]) for k in ("epochs", "admissions", "spills", "deferred")})
    st["admitted_gb"] = (s1["admitted_bytes"] - s0["admitted_bytes"]) / 1e9
    st["host_busy_s"] = round(s1["host_busy_s"] - s0["host_busy_s"], 3)
    st["p99_ms_by_second"] = [round(1e3 * float(np.percentile(lat[(t >= i) & (t < i + 1)], 99)), 2)
                              for i in range(int(duration)) if ((t >= i) & (t < i + 1)).any()]
    st["latency_split_ms"] = latency_split(reqs)
    if cold.any() and (~cold).any():
        st["p99_ms_resident_half"] = 1e3 * float(np.percentile(lat[~cold], 99))
        st["p99_ms_spillover_half"] = 1e3 * float(np.percentile(lat[cold], 99))
        st["spillover_request_frac"] = float(cold.mean())
    return st


def large_summary(steps):
    """The single large model (a 1M-triangle vessel in ~2k charts shelf-packed into a 4096^2 atlas,
    16 u16 layers, 10k sphere strokes, 200 lassos on 2048^2 depth maps), run by this script in a
    child process (`--config large`), outside the headline's timed region: its step throughput,
    per-row times, end-to-end figure and clocks.  A failure is reported in the line instead of
    ending the run."""
    cmd = [sys.executable, os.path.abspath(__file__), "--config", "large", "--steps", str(steps), "--warmup", "3",
           "--cpu-rows", "0", "--serving-models", "0", "--batch-models", "0", "--large-steps", "0"]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    except subprocess.TimeoutExpired:
        return {"error": "the large-model run timed out"}
    return parse_large(r.returncode, r.stdout, r.stderr)


def parse_large(rc, stdout, stderr):
    """The large-model summary from the child run's output (its last JSON line)."""
    lines = [ln for ln in stdout.splitlines() if ln.startswith("{")]
    if rc != 0 or not lines:
        tail = stderr.strip().splitlines()[-1:] if stderr else []
        return {"error": f"the large-model run exited {rc}: {' '.join(tail)}"}
    d = json.loads(lines[-1])
    return {"command": "bench.py --config large (child process)", "workload": d["config"]["workload"],
            "value": d["value"], "unit": d["unit"], "ms_per_step": d["ms_per_step"], "steps": d["steps"],
            "warmup": d["warmup"], "dtype": d["dtype"],
            "rows": {k: {kk: v[kk] for kk in ("ms_per_step", "frac") if kk in v} for k, v in d["rows"].items()},
            "sphere_frac_of_group_bytes": d["roofline"].get("frac_of_group_bytes"),
            "e2e": d["e2e"]["value"], "gpu_launches": d["gpu_launches"], "clocks": d["clocks"]}


def serving_summary(n_models, rate, duration):
    """The serving workload for the headline line: n_models models, an HBM budget that holds the
    first half (the resident set) and spillover models admitted on demand, Poisson arrivals, served by
    the native loop (continuous batching, admission by footprint and request rate)."""
    import torch

    models, budget, sphere_of, lasso_of = serving_setup(n_models)
    out = native_serving_run(models, budget, sphere_of, lasso_of, rate, duration)
    out.update({"models": len(models), "offered_rps": rate, "seconds": duration, "budget_gib": budget / 2**30,
                "scheduler": "native loop in liblcl.so (lcl_serve_*)",
                "mix": "70% sphere / 20% lasso / 10% overlay+area, Zipf(1.1) models, the first half resident "
                       "under the budget, the rest spillover"})
    torch.cuda.empty_cache()
    return out


# The paper's per-edit times for its Vessel (312k triangles, GTX 970, OpenGL, texture editing +
# padding), Fig. 6, by layer side and tool radius in pixels -- context only.
PAPER_FIG6_VESSEL_MS = {2048: [0.86, 0.86, 0.86, 0.86, 0.86], 4096: [1.89, 1.9, 1.91, 1.91, 2.01],
                        8192: [5.61, 5.64, 5.68, 5.74, 5.89]}
TOOL_RADII_PX = [10, 40, 70, 100, 200]


def run_tool(args):
    """The paper's editing experiment (Fig. 6): one layer of a vessel of ~312k triangles at 2048^2,
    4096^2 and 8192^2, edited with the circular tool of radius 10-200 px at points along the model
    on a 1920 x 1080 view; per edit the tool selection with texture padding (radius 2, outline
    thickness 2; the paper states neither), and without padding.  The depth map is rendered once per
    view, as in the paper (it changes with the camera, not with the edit)."""
    import torch

    import synth
    from paper_2501_14807_gb300 import lcl

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    mesh = synth.vessel_cylindrical(560, 280, noise_amp=0.005, noise_freq=16.0, seed=7)
    Ws, Hs = 1920, 1080
    p = mesh.pos.astype(np.float64)
    lo, hi = p.min(0), p.max(0)
    centre, radius = 0.5 * (lo + hi), 0.5 * float(np.linalg.norm(hi - lo))
    el, az, dist = np.radians(15.0), 0.4, 2.2 * radius
    eye = centre + dist * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
    cam_host = synth.Camera(synth.perspective01(40.0, Ws / Hs, dist - 1.1 * radius, dist + 1.1 * radius) @
                            synth.look_at(eye, centre), Ws, Hs)
    rng = np.random.default_rng(61)
    pts = synth.surface_points(mesh, 400, rng)
    scr = synth.project_px(cam_host, pts)
    facing = (pts - centre)[:, :2] @ (eye - centre)[:2] > 0
    ok = facing & (scr[:, 0] > 250) & (scr[:, 0] < Ws - 250) & (scr[:, 1] > 250) & (scr[:, 1] < Hs - 250)
    spots = scr[ok][:24]
    n_edits = len(spots)
    m = lcl.Mesh.from_host(mesh, dev)
    stream = torch.cuda.current_stream(dev)
    rows, tot_tex, tot_ms = [], 0, 0.0
    for side in (2048, 4096, 8192):
        a = lcl.Atlas(side, side, 32, mesh.n_tri, dev)
        lcl.lcl_atlas_build(m, a)
        cam = lcl.lcl_camera_from_vp(a, cam_host.vp, Ws, Hs)
        depth = torch.empty((Hs, Ws), dtype=torch.float32, device=dev)
        lcl.lcl_depth_render(m, a, cam, depth)
        layer = torch.zeros((side, side), dtype=torch.uint8, device=dev)
        ws = torch.empty(lcl.lcl_select_workspace_bytes(a, 1), dtype=torch.uint8, device=dev)
        hits = torch.zeros(n_edits, dtype=torch.int64, device=dev)
        for ri, r in enumerate(TOOL_RADII_PX):
            res = {}
            for mode, flags in (("tea", 0), ("tea_tpa", lcl.pad_flags(2, 2))):
                tools = [lcl.make_tool((float(x), float(y)), (2.0 * r, 2.0 * r), None, flags) for x, y in spots]

                def edits():
                    for k, t in enumerate(tools):
                        lcl.lcl_select_tool(a, layer, cam, depth, t, 1 + k % 250, lcl.DEFAULT_BIAS, hits[k:k + 1], ws,
                                            stream)

                for _ in range(max(args.warmup, 1)):
                    edits()
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    edits()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms = e0.elapsed_time(e1) / (args.steps * n_edits)
                res[mode] = ms
                if mode == "tea_tpa":
                    h = int(hits.sum().item())
                    tot_tex += h * args.steps
                    tot_ms += ms * n_edits * args.steps
                    res["hit_texels_per_edit"] = h / n_edits
            rows.append({"layer_side": side, "radius_px": r, "ms_per_edit_tea": res["tea"],
                         "ms_per_edit_tea_tpa": res["tea_tpa"], "hit_texels_per_edit": res["hit_texels_per_edit"],
                         "paper_fig6_ms": PAPER_FIG6_VESSEL_MS[side][ri]})
        del a, layer, depth
        torch.cuda.empty_cache()
    line = {"metric": METRIC, "value": tot_tex / (tot_ms / 1e3) / 1e9 if tot_ms else 0.0, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded vessel standing in for the paper's scanned Vessel)",
            "config": {"workload": f"editing tool: vessel {mesh.n_tri} triangles, one u8 layer at 2048^2/4096^2/"
                                   f"8192^2, circle radius 10-200 px on a {Ws}x{Hs} view, {n_edits} edits per "
                                   f"radius, padding radius 2 / thickness 2", "view": f"{Ws}x{Hs}"},
            "per_edit": rows,
            "note": "paper_fig6_ms: the paper's GTX 970 OpenGL times for its scanned Vessel, context only"}
    print(json.dumps(line), flush=True)


def run_numeric(args):
    """Numeric layers (Section 4.2) on the roofline-size model: 16384^2 atlas of the ~8M-triangle
    vessel, float32 data textures with their mask bits.  One step: the 1000 sphere strokes of the
    roofline workload written as values (a seeded "age" in [0, 2000)) into two numeric layers
    (500 each), their sum (arithmetic overlay), a selection by value (sum > 1000) into a u8 label
    layer, and the zonal statistics of the sum over the selection's labels.  Reports every row's
    CUDA-event time and algorithmic bytes against the HBM peak."""
    import torch

    from paper_2501_14807_gb300 import lcl

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = synth_roofline(args)
    W, H = w.width, w.height
    mesh = lcl.Mesh.from_host(w.mesh, dev)
    atlas = lcl.Atlas(W, H, w.tile, w.mesh.n_tri, dev)
    lcl.lcl_atlas_build(mesh, atlas)
    A, B, S = (lcl.NumericLayer(W, H, "f32", dev) for _ in range(3))
    zones = torch.zeros((H, W), dtype=torch.uint8, device=dev)
    rng = np.random.default_rng(91)
    ages = rng.uniform(0, 2000, size=len(w.strokes.radius)).astype(np.float32)
    recs = np.stack([lcl.lcl_quantize_sphere(atlas, w.strokes.centre[k], w.strokes.radius[k], 0)
                     for k in range(len(ages))])
    recs["label"] = ages.view(np.uint32)
    half = len(recs) // 2
    per = [np.ascontiguousarray(recs[:half]), np.ascontiguousarray(recs[half:])]
    ws = torch.empty(lcl.lcl_select_workspace_bytes(atlas, max(len(r) for r in per)), dtype=torch.uint8, device=dev)
    hits = [torch.zeros(max(len(r), 1), dtype=torch.int64, device=dev) for r in per]
    sel_hits = torch.zeros(1, dtype=torch.int64, device=dev)
    stats = torch.empty(256 * 48, dtype=torch.uint8, device=dev)
    thr = int(np.float32(1000.0).view(np.uint32))
    stream = torch.cuda.current_stream(dev)
    names = ("edit", "arith", "select", "stats")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]

    def step(timed):
        mark = (lambda i: ev[i].record(stream)) if timed else (lambda i: None)
        mark(0)
        lcl.lcl_numeric_sphere(atlas, A, per[0], hits[0], ws, stream)
        lcl.lcl_numeric_sphere(atlas, B, per[1], hits[1], ws, stream)
        mark(1)
        lcl.lcl_numeric_arith(atlas, A, B, S, "add", stream=stream)
        mark(2)
        lcl.lcl_numeric_select(atlas, S, "gt", thr, zones, 1, sel_hits, stream)
        mark(3)
        lcl.lcl_numeric_stats(atlas, S, zones, 256, stats, stream)
        mark(4)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize(dev)
    n_hit = int(hits[0].sum().item() + hits[1].sum().item())
    n_sel = int(sel_hits.item())
    row_ms = [0.0] * len(names)
    clocks = Clocks(0)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(True)
        ev[-1].synchronize()
        for i in range(len(names)):
            row_ms[i] += ev[i].elapsed_time(ev[i + 1])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    total_ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    peak, peak_kind = peaks()
    n = W * H
    spec = {  # algorithmic bytes per step (f32 values, 1 mask bit per texel, coverage bits)
        "edit": (n_hit * (12 + 4 + 1 / 8), f"{len(recs)} value strokes, {n_hit} hit texels (12 B position + 4 B "
                                            f"value + 1 mask bit each)"),
        "arith": (n * (3 * 4 + 4 / 8), "float32 a + b over every texel (3 x 4 B + 3 mask bits + 1 cover bit)"),
        "select": (n * (4 + 2 / 8) + n_sel, f"sum > 1000 into u8 labels, {n_sel} selected (4 B + 2 bits per texel, "
                                             "1 B per label written)"),
        "stats": (n * (4 + 1 + 4 + 2 / 8) + 8 * w.mesh.n_tri, "zonal statistics, 256 zones (4 B value + 1 B zone + "
                                                              "4 B triangle + 2 bits per texel, 8 B per triangle)"),
    }
    rows = {}
    for name, ms in zip(names, row_ms):
        b, what = spec[name]
        t = ms / args.steps
        gbs = b / (t / 1e3) / 1e9
        rows[name] = {"ms_per_step": t, "what": what, "algorithmic_bytes": int(b), "gb_s": gbs, "frac": gbs / peak}
    texels = n_hit + 3 * n
    line = {"metric": METRIC, "value": texels * args.steps / (total_ms / 1e3) / 1e9, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded vessel)",
            "config": {"workload": f"numeric layers: {w.name}, {w.mesh.n_tri} triangles, {W}x{H} atlas, float32 "
                                   f"layers with mask bits: {len(recs)} value strokes into two layers, their sum, "
                                   f"a selection by value, zonal statistics over 256 zones",
                       "l2": "inputs larger than L2"},
            "roofline": {"bound": "hbm", "peak": peak, "peak_kind": peak_kind, "unit": "GB/s"},
            "rows": rows, "clocks": clk,
            "note": "texels per step: every hit texel of the value strokes plus every texel of the sum, the "
                    "selection and the statistics"}
    print(json.dumps(line), flush=True)


def synth_roofline(args):
    """The roofline model (16384^2), or the same model scaled to --atlas-side for profiles."""
    import synth
    side = args.atlas_side or 16384
    return synth.config_roofline(n_strokes=args.strokes, n_lassos=0, n_theta=round(2828 * side / 16384),
                                 n_h=round(1414 * side / 16384), side=side)


def run_pool(args):
    """The sparse layer pool (lcl_pool_*): time to commit (acquire, clear included) and return (release)
    one layer of several sizes, median of 20 each with the device idle; then the serving workload
    served with layers taken from the pool against the same trace served with ordinary device
    tensors (continuous batching both times)."""
    import torch

    from paper_2501_14807_gb300 import lcl, serve

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    pool = lcl.Pool(max_layers_per_array=64, device=dev)
    sizes = []
    for side, kind in ((1024, "u8"), (4096, "u8"), (4096, "f32"), (16384, "u8")):
        acq, rel = [], []
        for _ in range(22):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            L = pool.acquire(side, side, kind)
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            pool.release(L)
            t2 = time.perf_counter()
            acq.append(t1 - t0)
            rel.append(t2 - t1)
        sizes.append({"side": side, "type": kind, "acquire_us": 1e6 * statistics.median(acq[2:]),
                      "release_us": 1e6 * statistics.median(rel[2:])})
    st = pool.stats()
    pool.destroy()
    models, budget, sphere_of, lasso_of = serving_setup(args.models or 64)
    out = {}
    for mode, use_pool in (("tensors", False), ("layer_pool", True)):
        srv = serve.Server(models, hbm_budget_bytes=budget, layer_pool=use_pool)
        warm = serve.poisson_requests(len(models), args.rate, 0.2, 6, sphere_of=sphere_of, lasso_of=lasso_of)
        srv.run(warm)
        reqs = serve.poisson_requests(len(models), args.rate, args.duration, 5, sphere_of=sphere_of,
                                      lasso_of=lasso_of)
        clocks = Clocks(0)
        clocks.start()
        srv.run(reqs)
        clk = clocks.stop()
        r = serve.latency_stats(reqs)
        r.update({"spills": srv.spills, "admissions": srv.admissions, "clocks": clk})
        if use_pool:
            r["pool"] = srv.pool.stats()
        out[mode] = r
        srv.close()
        del srv
        torch.cuda.empty_cache()
    p = out["layer_pool"]
    line = {"metric": METRIC, "value": p["throughput_rps"], "unit": "requests/s", "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": 1e3 * args.duration, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"sparse layer pool: commit / return times per layer; serving {len(models)} "
                                   f"models under a {budget / 2**30:.2f} GiB budget, Poisson {args.rate:.0f} req/s for "
                                   f"{args.duration:.1f} s, layers from the pool vs ordinary tensors"},
            "p50_ms": p["p50_ms"], "p99_ms": p["p99_ms"], "pool_layer_times": sizes,
            "pool_granularity": st["granularity"], "served": out}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Serving workload: resident + spillover models (as in the batching workload), 2 layers each,
    an HBM budget that holds about half of them, open-loop Poisson arrivals (70% sphere strokes, 20%
    lassos, 10% overlay + area queries, models by a Zipf(1.1) law).  Served by the native loop
    (lcl_serve_*), by the Python scheduler (serve.Server, the same policy with its bookkeeping in
    Python) and one request per call (the baseline); the same trace for all three."""
    import torch

    from paper_2501_14807_gb300 import serve

    torch.cuda.set_device(0)
    models, budget, sphere_of, lasso_of = serving_setup(args.models or 128)
    clocks = Clocks(0)
    clocks.start()
    out = {"native": native_serving_run(models, budget, sphere_of, lasso_of, args.rate, args.duration)}
    out["native"]["clocks"] = clocks.stop()
    torch.cuda.empty_cache()
    for mode in ("python_batched", "per_request"):
        srv = serve.Server(models, hbm_budget_bytes=budget)
        reqs = serve.poisson_requests(len(models), args.rate, args.duration, 5, sphere_of=sphere_of,
                                      lasso_of=lasso_of)
        warm = serve.poisson_requests(len(models), args.rate, 0.2, 6, sphere_of=sphere_of, lasso_of=lasso_of)
        (srv.run if mode == "python_batched" else srv.run_per_request)(warm)
        (srv.run if mode == "python_batched" else srv.run_per_request)(reqs)
        st = serve.latency_stats(reqs)
        st.update({"epochs": srv.epochs, "spills": srv.spills, "admissions": srv.admissions,
                   "host_s": {k: round(v, 3) for k, v in srv.host_s.items()}})
        out[mode] = st
        srv.close()
        del srv
        torch.cuda.empty_cache()
    b = out["native"]
    line = {"metric": METRIC, "value": b["throughput_rps"], "unit": "requests/s", "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": 1e3 * args.duration, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"serving: {len(models)} models (half resident under a {budget / 2**30:.2f} GiB "
                                   f"budget), Poisson {args.rate:.0f} req/s for {args.duration:.1f} s, mix 70% sphere / "
                                   f"20% lasso / 10% overlay+area, Zipf(1.1) model choice"},
            "p50_ms": b["p50_ms"], "p99_ms": b["p99_ms"], "served": out, "gpu_launches": None}
    print(json.dumps(line), flush=True)


def profile_traffic(w):
    """DRAM bytes per grouped sphere-edit launch (one group's cull and apply) from the committed ncu
    summary, if it was taken on the current kernel source (null otherwise)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "sphere_group_traffic.json")
    src = os.path.join(ROOT, "paper_2501_14807_gb300", "csrc", "select.cu")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    if d.get("select_cu_sha256_16") != h or d.get("workload") != w.name:
        return None
    return d.get("dram_bytes_per_launch")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="roofline",
                    choices=["roofline", "large", "mid", "small", "batch", "serve", "tool", "numeric", "pool"])
    ap.add_argument("--rate", type=float, default=20000.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--duration", type=float, default=5.0, help="serving: trace length (s)")
    ap.add_argument("--models", type=int, default=None,
                    help="models in the batching (default 256) / serving (default 128: 64 resident + 64 spilled) workload")
    ap.add_argument("--batch-models", type=int, default=256,
                    help="models of the batching workload reported in the headline line (0: skip)")
    ap.add_argument("--serving-models", type=int, default=128,
                    help="models of the serving run reported in the headline line (0: skip)")
    ap.add_argument("--serving-seconds", type=float, default=10.0,
                    help="length of the headline serving trace (Poisson 20k requests/s)")
    ap.add_argument("--large-steps", type=int, default=5,
                    help="timed steps of the large-model (16 u16 layers) run reported in the headline line (0: skip)")
    ap.add_argument("--atlas-side", type=int, default=None,
                    help="mid config: atlas side (default 4096; the mesh is scaled with it)")
    ap.add_argument("--strokes", type=int, default=None)
    ap.add_argument("--lassos", type=int, default=None)
    ap.add_argument("--cpu-rows", type=int, default=64, help="rows of the texture the CPU oracle baseline covers")
    args = ap.parse_args()
    defaults = {"roofline": (1000, 20), "mid": (1000, 20), "large": (10000, 200), "small": (200, 0), "batch": (0, 0),
                "serve": (0, 0), "tool": (0, 0), "numeric": (1000, 0), "pool": (0, 0)}
    if args.strokes is None:
        args.strokes = defaults[args.config][0]
    if args.lassos is None:
        args.lassos = defaults[args.config][1]
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.config == "batch":
        run_batch(args)
    elif args.config == "serve":
        run_serve(args)
    elif args.config == "tool":
        run_tool(args)
    elif args.config == "numeric":
        run_numeric(args)
    elif args.config == "pool":
        run_pool(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
