"""Reference replays of a served trace, for the serving tests.

replay_oracle: the plain definition (the CPU oracle), each model's requests applied alone, in
    arrival order: spheres, lassos on the oracle's own depth maps, and overlay + per-label area
    queries evaluated on the layers as they stand when the query arrives (Section 4.3.1 / Fig. 3
    for the edit each request performs).  Lasso texels the oracle flags as ambiguous are
    recorded per layer, since only they may differ from the GPU (the lasso tolerance).
replay_alone: the library's own single-call path on fresh layers (one call per request).

Both are test scaffolding; the serving module itself only schedules."""
from __future__ import annotations

import collections
import concurrent.futures as cf
import os

import numpy as np

SPHERE, LASSO, QUERY = 0, 1, 2


def _by_model(requests):
    by_model = collections.defaultdict(list)
    for i, r in enumerate(requests):
        by_model[r.model].append((i, r))
    return by_model


def _oracle_model(spec, reqs, bias):
    import oracle

    side = spec.side
    o = oracle.Atlas(spec.mesh, side, side, tile=spec.tile)
    ms = [oracle.camera_mq(c.vp, o.mn, o.S) for c in spec.cams]
    dms = [oracle.depth(spec.mesh, o.mn, o.S, m, c.width, c.height) for m, c in zip(ms, spec.cams)]
    layers = [np.zeros((side, side), np.uint8) for _ in range(spec.n_layers)]
    amb = [np.zeros((side, side), bool) for _ in range(spec.n_layers)]
    touched = [0] * spec.n_layers
    results = {}
    for i, r in reqs:
        if r.kind == SPHERE:
            c, rad, label = r.sphere
            rec = oracle.sphere_records(o.mn, o.S, [c], [rad], [label])
            touched[r.layer] += int(oracle.select_sphere(o, layers[r.layer], rec)[0])
        elif r.kind == LASSO:
            ci, poly, label = r.lasso
            h, a = oracle.select_lasso(o, layers[r.layer], ms[ci], dms[ci], poly, label, bias=bias)
            touched[r.layer] += h
            amb[r.layer] |= a != 0
        else:
            op, la, lb, n_labels = r.query
            out = oracle.overlay(o, layers[la], layers[lb], op)
            cnt, area = oracle.label_area(o, out, n_labels)
            results[i] = (cnt, area, int((amb[la] | amb[lb]).sum()))
    return layers, amb, touched, results


def replay_oracle(server_models, requests, bias=2.0 ** -10, threads=None):
    """Returns ({model: (layers, ambiguous masks, texels touched per layer)},
    {request index: (counts, areas, ambiguous texels in the queried layers)}), numpy arrays.
    Models run in threads (the oracle's C code releases the GIL)."""
    by_model = _by_model(requests)
    threads = threads or min(len(by_model), os.cpu_count() or 1) or 1
    layers, results = {}, {}
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        futs = {mi: ex.submit(_oracle_model, server_models[mi], reqs, bias) for mi, reqs in by_model.items()}
        for mi, f in futs.items():
            ls, amb, touched, res = f.result()
            layers[mi] = (ls, amb, touched)
            results.update(res)
    return layers, results


def replay_alone(server_models, requests, device="cuda"):
    """Applies each model's requests alone, in arrival order, with single-stroke library calls on
    fresh layers; returns ({model: layers}, {request index: (counts, areas)}) for comparison."""
    import torch

    from paper_2501_14807_gb300 import lcl

    dev = torch.device(device)
    layers, results = {}, {}
    for mi, reqs in _by_model(requests).items():
        spec = server_models[mi]
        mesh = lcl.Mesh.from_host(spec.mesh, dev)
        a = lcl.Atlas(spec.side, spec.side, spec.tile, spec.mesh.n_tri, dev)
        lcl.lcl_atlas_build(mesh, a)
        ls = [torch.zeros((spec.side, spec.side), dtype=torch.uint8, device=dev) for _ in range(spec.n_layers)]
        cams = [lcl.lcl_camera_from_vp(a, c.vp, c.width, c.height) for c in spec.cams]
        depths = []
        for c in cams:
            d = torch.empty((c.height, c.width), dtype=torch.float32, device=dev)
            lcl.lcl_depth_render(mesh, a, c, d)
            depths.append(d)
        for i, r in reqs:
            if r.kind == SPHERE:
                c, rad, label = r.sphere
                lcl.lcl_select_sphere(a, ls[r.layer], np.array([lcl.lcl_quantize_sphere(a, c, rad, label)],
                                                               lcl.SPHERE_DTYPE))
            elif r.kind == LASSO:
                ci, poly, label = r.lasso
                lcl.lcl_select_lasso(a, ls[r.layer], cams[ci], depths[ci], poly, label)
            else:
                op, la, lb, n_labels = r.query
                out = torch.empty_like(ls[la])
                lcl.lcl_overlay(a, ls[la], ls[lb], out, op)
                cnt, area = lcl.lcl_label_area(a, out, n_labels)
                results[i] = (cnt.cpu().numpy().view(np.uint64), area.cpu().numpy().view(np.uint64))
        layers[mi] = ls
    torch.cuda.synchronize(dev)
    return layers, results
