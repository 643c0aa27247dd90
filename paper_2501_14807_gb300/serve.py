"""Serving loop: many models resident on the device, edit and query requests arriving
continuously, batched into launches, with per-request latency.

The paper's architecture keeps every layer on the GPU and lets the CPU only manage (Section 4),
and its texture manager reserves texture memory and commits it on demand (Section 4.2, sparse
textures).  This module is the server-side counterpart for many models at once:

* a resident pool: each model's atlas, layers and depth maps live in device memory while the pool's
  HBM budget allows; a model that is needed when the budget is full evicts the idle model with the
  lowest recent request rate (requests decayed with a 1 s time constant; least recently used among
  equals), whose layers are copied to pinned host memory on a copy stream (its atlas and depth maps
  only on the first spill: they never change) and copied back when it is admitted again;
* per-model FIFO queues: a model's requests are applied in arrival order;
* asynchronous admission: a spilled model with queued work is copied back on the copy stream and
  its requests join the first epoch built after that copy has completed, so epochs of resident
  models never wait for an admission; an admitted model cannot be evicted before an epoch has used
  it (otherwise two models could keep evicting each other); an admission that would exceed the
  budget while the resident models are busy waits for a later epoch;
* continuous batching: every epoch takes, for each ready model with queued work, the leading run of
  edit requests (up to 64 per layer) and at most one query, uploads all edits as one batch
  (``lcl_batch_upload``) and replays a CUDA graph of the batched launch, followed by the queries
  (``lcl_overlay`` + ``lcl_label_area``) on one compute stream, and records an event; requests that
  arrive meanwhile join the next epoch, which is prepared on the host while the previous one runs
  (several epochs in flight, each with its own workspace, staging and graph);
* one launch shape for every epoch: the workspaces are sized for the largest possible epoch (every
  layer of every model with a full queue), so the graph captured once per in-flight slot serves
  every epoch;
* latency: host arrival time to the host observing the epoch's completion event;
* optionally (``layer_pool=True``) layers come from the sparse layer pool (``lcl_pool_*``): a model's
  layers are committed when it is built or admitted and returned to the pool once its spill copy has
  completed, so spilled models hold no device memory for their layers.

Everything that computes runs in liblcl.so; this module only schedules.
"""
from __future__ import annotations

import collections
import heapq
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import lcl

SPHERE, LASSO, QUERY = 0, 1, 2
TAU_S = 1.0   # time constant of the request-rate score that picks eviction victims


@dataclass
class Request:
    t_arrive: float          # seconds, on the server's clock (relative to run start)
    model: int
    kind: int                # SPHERE, LASSO or QUERY
    layer: int = 0
    sphere: object = None    # (centre[3], radius, label) in world units
    lasso: object = None     # (camera index, polygon float32 [n, 2], label)
    query: object = None     # (op name, layer a, layer b, n_labels)
    t_done: float = -1.0
    result: object = None    # QUERY: (counts, areas) as numpy uint64 arrays
    t_launch: float = -1.0   # native server: when the request's epoch was launched
    t_gpu: float = -1.0      # native server: seconds the GPU spent on the request's epoch


@dataclass
class ServedModel:
    """Host description of one servable model (mesh, atlas side, cameras)."""
    mesh: object
    side: int
    cams: list               # synth.Camera list (view-projection matrices)
    n_layers: int = 2
    tile: int = 32


@dataclass
class _Slot:
    spec: ServedModel
    atlas: object = None
    mesh_dev: object = None
    layers: list = field(default_factory=list)
    cams: list = field(default_factory=list)     # lcl_camera
    depths: list = field(default_factory=list)   # device float32 maps
    host: dict = None                            # pinned copies while spilled
    resident: bool = False
    last_used: float = 0.0
    busy_until: object = None                    # event of the last epoch that used it
    spilled: object = None                       # event after the last spill's device-to-host copy
    bytes: int = 0
    pool_layers: list = field(default_factory=list)  # lcl.PoolLayer of each layer (layer pool only)
    ready: object = None                         # event after the last admission's host-to-device copy
    buf: object = None                           # the model's device buffer (atlas | layers | depth maps)
    lay: tuple = None                            # its layout (_layout)
    score: float = 0.0                           # requests received, decayed with time constant TAU_S
    t_score: float = 0.0
    key: float = -math.inf                       # victim-heap key (see Server._touch)
    idx: int = 0


class Server:
    """Resident pool + FIFO queues + continuous batching over one compute stream."""

    def __init__(self, models, hbm_budget_bytes, device="cuda", max_edits_per_layer=lcl.BATCH_MAX_STROKES,
                 max_in_flight=2, result_ring=4096, max_labels=256, config=None, graphs=True, layer_pool=False):
        self.dev = torch.device(device)
        # layer pool (the sparse layer pool of lcl_pool_*): layers are committed when a model is built
        # or admitted and returned when its spill copy has completed (polled, not waited for)
        self.pool = lcl.Pool(max_layers_per_array=max(sum(m.n_layers for m in models), 1),
                             device=self.dev) if layer_pool else None
        self._idle = torch.cuda.Stream(self.dev) if layer_pool else None   # no work: releases need no wait
        self._to_release = []
        self.max_admitting = 16
        self.host_s = collections.Counter()   # host seconds spent building epochs, admitting, spilling
        self.max_in_flight = max_in_flight
        self.config = config                    # batched launch shape (None: the library default)
        self.use_graphs = graphs                # replay a captured launch (else launch directly)
        self._ring = torch.empty((result_ring, 2, max_labels), dtype=torch.int64).pin_memory()
        self._ring_next = 0
        self.max_labels = max_labels
        self.budget = int(hbm_budget_bytes)
        self.max_edits = int(max_edits_per_layer)
        self.compute = torch.cuda.Stream(self.dev)
        self.copy = torch.cuda.Stream(self.dev)
        self.slots = [_Slot(spec=m, idx=i) for i, m in enumerate(models)]
        self._heap = [(-math.inf, i) for i in range(len(models))]   # every model starts with rate 0
        self.resident_bytes = 0
        self.spills = 0
        self.admissions = 0
        self.epochs = 0
        for i, s in enumerate(self.slots):
            self._build(s)
            if self.resident_bytes > self.budget:
                self._spill(s)
        torch.cuda.synchronize(self.dev)
        self.ws_sel = None
        # the largest epoch: every layer of every model, each with a full queue of edits
        def tiles_of(m):   # tiles per side, super-tiles per side
            t = -(-m.side // m.tile)
            return t, -(-t // lcl.SUPER)

        pairs = sum(m.n_layers for m in models)
        supers = sum(m.n_layers * tiles_of(m)[1] ** 2 for m in models)
        tiles = sum(m.n_layers * tiles_of(m)[0] ** 2 for m in models)
        self.limits = lcl.batch_limits(pairs, pairs * self.max_edits, pairs * self.max_edits, supers, tiles)
        n_stg = int(lcl.library().lcl_batch_staging_bytes(lcl.C.byref(self.limits)))
        self._ws = [lcl.batch_workspace(self.limits, self.dev) for _ in range(max_in_flight)]
        self._stg = [torch.empty(n_stg, dtype=torch.uint8).pin_memory() for _ in range(max_in_flight)]
        with torch.cuda.stream(self.compute):
            self._graphs = [lcl.BatchGraph(self.limits, self.config, ws) if graphs else None for ws in self._ws]
        torch.cuda.synchronize(self.dev)

    # ---- pool ---------------------------------------------------------------------------

    def _layout(self, s: _Slot):
        """Offsets of a model's one device buffer: atlas | layers (unless pooled) | depth maps, each
        section 256-byte aligned.  Returns (atlas bytes, layer offset, layer stride, depth offsets, total)."""
        spec = s.spec
        a256 = lambda x: (x + 255) // 256 * 256  # noqa: E731
        ab = int(lcl.library().lcl_atlas_bytes(spec.side, spec.side, spec.tile, spec.mesh.n_tri))
        lb = a256(spec.side * spec.side)
        off_l = a256(ab)
        off = off_l + (0 if self.pool is not None else spec.n_layers * lb)
        offs_d = []
        for c in spec.cams:
            offs_d.append(off)
            off += a256(4 * c.width * c.height)
        return ab, off_l, lb, offs_d, off

    def _views(self, s: _Slot, buf):
        """Layer and depth-map views of a model buffer laid out by _layout."""
        spec = s.spec
        _, off_l, lb, offs_d, _ = s.lay
        n = spec.side * spec.side
        if self.pool is None:
            s.layers = [buf[off_l + i * lb: off_l + i * lb + n].view(spec.side, spec.side)
                        for i in range(spec.n_layers)]
        s.depths = [buf[o: o + 4 * c.width * c.height].view(torch.float32).view(c.height, c.width)
                    for o, c in zip(offs_d, spec.cams)]

    def _build(self, s: _Slot):
        spec = s.spec
        s.lay = self._layout(s)
        buf = torch.empty(s.lay[4], dtype=torch.uint8, device=self.dev)
        s.mesh_dev = lcl.Mesh.from_host(spec.mesh, self.dev)
        s.atlas = lcl.Atlas(spec.side, spec.side, spec.tile, spec.mesh.n_tri, self.dev, buffer=buf)
        lcl.lcl_atlas_build(s.mesh_dev, s.atlas)
        self._views(s, buf)
        if self.pool is not None:
            s.pool_layers = [self.pool.acquire(spec.side, spec.side, "u8") for _ in range(spec.n_layers)]
            s.layers = [pl.data for pl in s.pool_layers]
        else:
            for l in s.layers:
                l.zero_()
        s.cams = [lcl.lcl_camera_from_vp(s.atlas, c.vp, c.width, c.height) for c in spec.cams]
        for c, d in zip(s.cams, s.depths):
            lcl.lcl_depth_render(s.mesh_dev, s.atlas, c, d)
        # the renders (and the layers' clearing) run on the current stream: a spill, whose copy runs
        # on the copy stream, waits for them like for an epoch
        s.busy_until = torch.cuda.Event()
        s.busy_until.record(torch.cuda.current_stream(self.dev))
        s.buf = buf
        layer_bytes = 0
        if self.pool is not None:   # committed in whole allocation-granularity units
            g = self.pool.stats()["granularity"]
            layer_bytes = sum(-(-l.numel() // g) * g for l in s.layers)
        s.bytes = s.lay[4] + layer_bytes
        s.resident = True
        self.resident_bytes += s.bytes

    def _spill(self, s: _Slot):
        """Copies a resident model to its pinned host image (allocated on the first spill and reused)
        on the copy stream and releases its device buffer without waiting: the copy stream's order
        puts any later re-admission after this copy, and record_stream keeps the device memory from
        being reused before the copy has read it.  The atlas and depth maps never change, so after
        the first spill only the layers' section is copied (one copy)."""
        if s.busy_until is not None:
            self.copy.wait_event(s.busy_until)
        _, off_l, lb, offs_d, total = s.lay
        if s.host is None:
            s.host = {"image": torch.empty(total, dtype=torch.uint8).pin_memory(), "full": False,
                      "layers": [torch.empty(l.shape, dtype=l.dtype).pin_memory() for l in s.layers]
                      if self.pool is not None else None}
        host = s.host
        with torch.cuda.stream(self.copy):
            if not host["full"]:
                host["image"].copy_(s.buf, non_blocking=True)
                host["full"] = True
            elif self.pool is None:
                end = off_l + s.spec.n_layers * lb
                host["image"][off_l:end].copy_(s.buf[off_l:end], non_blocking=True)
            if self.pool is not None:
                for h, l in zip(host["layers"], s.layers):
                    h.copy_(l, non_blocking=True)
        s.buf.record_stream(self.copy)
        s.spilled = torch.cuda.Event()
        s.spilled.record(self.copy)
        if self.pool is not None:
            self._to_release.append((s.spilled, s.pool_layers))
            s.pool_layers = []
        s.atlas = _Rebind(s.atlas)
        s.layers, s.depths = [], []
        s.buf = None
        s.mesh_dev = None
        s.resident = False
        self.resident_bytes -= s.bytes
        self.spills += 1

    @staticmethod
    def _score(s: _Slot, now: float):
        """The model's recent request rate: requests decayed with time constant TAU_S."""
        return s.score * math.exp(-(now - s.t_score) / TAU_S)

    def _touch(self, s: _Slot, now: float):
        s.score = self._score(s, now) + 1.0
        s.t_score = now
        # rank key of the victim heap: log(score at time 0) = log(score) + t / TAU_S orders models by
        # their current rate at any time, so keys never need refreshing (stale entries are skipped)
        s.key = math.log(s.score) + now / TAU_S
        heapq.heappush(self._heap, (s.key, s.idx))
        if len(self._heap) > 8 * len(self.slots) + 1024:   # drop the stale entries
            self._heap = [(sl.key, sl.idx) for sl in self.slots]
            heapq.heapify(self._heap)

    def _reap(self):
        """Returns to the layer pool the layers of spilled models whose copy to the host is done."""
        keep = []
        for ev, layers in self._to_release:
            if ev.query():
                for pl in layers:
                    self.pool.release(pl, stream=self._idle)
            else:
                keep.append((ev, layers))
        self._to_release = keep

    def _admit(self, s: _Slot, now: float, keep=(), force=False):
        """Makes a spilled model resident again, evicting idle models with the lowest recent request
        rate (never one in `keep`, the models already taken into the epoch being built).  If the
        budget cannot be met now (the other resident models are busy), the admission is deferred
        and False returned, unless `force` or nothing else is resident."""
        th = time.perf_counter()
        if self.resident_bytes + s.bytes > self.budget:
            # candidates by rising request rate from the heap (entries whose key changed since are
            # stale and dropped); models that cannot go now are pushed back afterwards
            held = []
            while self._heap and self.resident_bytes + s.bytes > self.budget:
                key, i = heapq.heappop(self._heap)
                v = self.slots[i]
                if key != v.key:
                    continue
                held.append((key, i))
                if not v.resident or v is s or v.ready is not None or id(v) in keep:
                    continue
                if v.busy_until is None or v.busy_until.query():
                    self._spill(v)
            for e in held:
                heapq.heappush(self._heap, e)
            if self.resident_bytes + s.bytes > self.budget and not (force or self.resident_bytes == 0):
                self.host_s["admit"] += time.perf_counter() - th
                return False
        h = s.host
        buf = torch.empty(s.lay[4], dtype=torch.uint8, device=self.dev)
        buf.record_stream(self.copy)
        if self.pool is not None:
            self._reap()
            s.pool_layers = [self.pool.acquire(l.shape[1], l.shape[0], "u8", stream=self.copy) for l in h["layers"]]
        with torch.cuda.stream(self.copy):
            buf.copy_(h["image"], non_blocking=True)
            if self.pool is not None:
                for pl, l in zip(s.pool_layers, h["layers"]):
                    pl.data.copy_(l, non_blocking=True)
        s.atlas = s.atlas.restore(buf)
        self._views(s, buf)
        if self.pool is not None:
            s.layers = [pl.data for pl in s.pool_layers]
        s.buf = buf
        s.ready = torch.cuda.Event()
        s.ready.record(self.copy)
        buf.record_stream(self.compute)
        s.resident = True
        self.resident_bytes += s.bytes
        self.admissions += 1
        self.host_s["admit"] += time.perf_counter() - th
        return True

    # ---- requests -----------------------------------------------------------------------

    def _epoch(self, queues, now):
        """Takes the next epoch's work from the FIFO queues and launches it; returns
        (event, requests, query results, batch)."""
        models, work, queries, taken = [], [], [], []
        in_epoch = set()
        waits = []
        admitting = sum(1 for sl in self.slots if sl.ready is not None)
        for mi, q in queues.items():
            if not q:
                continue
            s = self.slots[mi]
            if not s.resident:
                # admission runs on the copy stream; the model's requests join a later epoch, once
                # its copy is done, so this epoch's resident models do not wait for it (at most
                # max_admitting admissions in flight)
                if admitting < self.max_admitting and self._admit(s, now, keep=in_epoch):
                    admitting += 1
                continue
            if s.ready is not None:
                if not s.ready.query():
                    continue
                waits.append(s.ready)
                s.ready = None
            in_epoch.add(id(s))
            s.last_used = now
            reqs, per_layer_n = [], collections.Counter()
            while q and q[0].kind != QUERY and per_layer_n[q[0].layer] < self.max_edits:
                per_layer_n[q[0].layer] += 1
                reqs.append(q.popleft())
            if reqs:
                sph = [r for r in reqs if r.kind == SPHERE]
                recs = iter(lcl.lcl_quantize_spheres(s.atlas, [r.sphere[0] for r in sph], [r.sphere[1] for r in sph],
                                                     [r.sphere[2] for r in sph])) if sph else iter(())
                per_layer = collections.defaultdict(list)
                for r in reqs:
                    if r.kind == SPHERE:
                        per_layer[r.layer].append(("sphere", next(recs)))
                    else:
                        ci, poly, label = r.lasso
                        per_layer[r.layer].append(("lasso", (s.cams[ci], s.depths[ci], poly, label, lcl.DEFAULT_BIAS)))
                for li, ops in per_layer.items():
                    models.append((s.atlas, s.layers[li]))
                    work.append(ops)
                taken.extend(reqs)
            elif q and q[0].kind == QUERY:
                req = q.popleft()
                queries.append((s, req))
                taken.append(req)
        if not taken:
            return None
        slot = self.epochs % self.max_in_flight
        batch = None
        for w in waits:   # already complete: orders the compute stream after the admission copies
            self.compute.wait_event(w)
        with torch.cuda.stream(self.compute):
            if models:
                batch = lcl.Batch(models, work, self._ws[slot], self._stg[slot], limits=self.limits,
                                  config=self.config)
                if self.use_graphs:
                    lcl.lcl_batch_upload(batch, self.compute)
                    self._graphs[slot].replay()
                else:
                    lcl.lcl_batch_edit(batch, self.compute)
            results = []
            for s, req in queries:
                op, la, lb, n_labels = req.query
                out = torch.empty_like(s.layers[la])
                lcl.lcl_overlay(s.atlas, s.layers[la], s.layers[lb], out, op, 0, self.compute)
                cnt, area = lcl.lcl_label_area(s.atlas, out, n_labels, stream=self.compute)
                ri = self._ring_next
                self._ring_next = (ri + 1) % self._ring.shape[0]
                self._ring[ri, 0, :n_labels].copy_(cnt, non_blocking=True)
                self._ring[ri, 1, :n_labels].copy_(area, non_blocking=True)
                results.append((req, ri, n_labels, out, cnt, area))
        ev = torch.cuda.Event()
        ev.record(self.compute)
        for r in taken:
            self.slots[r.model].busy_until = ev
        self.epochs += 1
        return ev, taken, results, batch

    def run(self, requests, poll_s=20e-6, stall_limit_s=60.0):
        """Serves `requests` (sorted by t_arrive, seconds from now) open-loop; fills t_done/result.
        Raises RuntimeError if no request completes for stall_limit_s seconds while work is queued."""
        pending = collections.deque(requests)
        queues = collections.defaultdict(collections.deque)
        in_flight = collections.deque()
        t0 = time.perf_counter()
        outstanding = len(requests)
        last_progress, last_outstanding = t0, outstanding
        while outstanding:
            now = time.perf_counter() - t0
            if outstanding != last_outstanding:
                last_progress, last_outstanding = time.perf_counter(), outstanding
            elif not pending and time.perf_counter() - last_progress > stall_limit_s:
                raise RuntimeError(f"serving loop made no progress for {stall_limit_s} s "
                                   f"({outstanding} requests outstanding)")
            while pending and pending[0].t_arrive <= now:
                r = pending.popleft()
                queues[r.model].append(r)
                self._touch(self.slots[r.model], now)
            while in_flight and in_flight[0][0].query():
                ev, taken, results, _batch = in_flight.popleft()
                done = time.perf_counter() - t0
                for r in taken:
                    r.t_done = done
                for req, ri, nl, *_ in results:
                    req.result = (self._ring[ri, 0, :nl].numpy().view(np.uint64).copy(),
                                  self._ring[ri, 1, :nl].numpy().view(np.uint64).copy())
                outstanding -= len(taken)
            if len(in_flight) < self.max_in_flight and any(queues[m] for m in queues):
                th = time.perf_counter()
                ep = self._epoch(queues, now)
                self.host_s["epoch"] += time.perf_counter() - th
                if ep is not None:
                    in_flight.append(ep)
                    continue
            if not in_flight and not any(queues[m] for m in queues) and pending:
                wait = pending[0].t_arrive - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 1e-3))
            else:
                time.sleep(poll_s)
        torch.cuda.synchronize(self.dev)
        if self.pool is not None:
            self._reap()
        return requests

    def close(self):
        """Synchronises the device and returns every pooled layer (layer pool only)."""
        if self.pool is not None:
            torch.cuda.synchronize(self.dev)
            self.pool.destroy()
            self.pool = None

    def run_per_request(self, requests, poll_s=20e-6):
        """The same trace served without batching: each request, in arrival order, is one
        single-stroke (or overlay + area) call on the compute stream; its completion event is
        polled.  The baseline the batched loop is compared with."""
        pending = collections.deque(requests)
        in_flight = collections.deque()
        ws = None
        t0 = time.perf_counter()
        done_n = 0
        while done_n < len(requests):
            now = time.perf_counter() - t0
            while in_flight and in_flight[0][0].query():
                ev, req, res = in_flight.popleft()
                req.t_done = time.perf_counter() - t0
                if res is not None:
                    req.result = (res[0].numpy().view(np.uint64).copy(), res[1].numpy().view(np.uint64).copy())
                done_n += 1
            if pending and pending[0].t_arrive <= now and len(in_flight) < 4096:
                req = pending.popleft()
                s = self.slots[req.model]
                self._touch(s, now)
                if not s.resident:
                    self._admit(s, now, force=True)
                if s.ready is not None:
                    self.compute.wait_event(s.ready)
                    s.ready = None
                s.last_used = now
                res = None
                with torch.cuda.stream(self.compute):
                    if ws is None:
                        ws = torch.empty(max(lcl.lcl_select_workspace_bytes(sl.atlas, 1) for sl in self.slots
                                             if sl.resident), dtype=torch.uint8, device=self.dev)
                    if req.kind == SPHERE:
                        c, r, label = req.sphere
                        lcl.lcl_select_sphere(s.atlas, s.layers[req.layer], lcl.lcl_quantize_spheres(s.atlas, [c], [r], [label]),
                                              None, ws, self.compute)
                    elif req.kind == LASSO:
                        ci, poly, label = req.lasso
                        lcl.lcl_select_lasso(s.atlas, s.layers[req.layer], s.cams[ci], s.depths[ci], poly, label,
                                             lcl.DEFAULT_BIAS, None, ws, self.compute)
                    else:
                        op, la, lb, n_labels = req.query
                        out = torch.empty_like(s.layers[la])
                        lcl.lcl_overlay(s.atlas, s.layers[la], s.layers[lb], out, op, 0, self.compute)
                        cnt, area = lcl.lcl_label_area(s.atlas, out, n_labels, stream=self.compute)
                        ri = self._ring_next
                        self._ring_next = (ri + 1) % self._ring.shape[0]
                        self._ring[ri, 0, :n_labels].copy_(cnt, non_blocking=True)
                        self._ring[ri, 1, :n_labels].copy_(area, non_blocking=True)
                        res = (self._ring[ri, 0, :n_labels], self._ring[ri, 1, :n_labels], out, cnt, area)
                ev = torch.cuda.Event()
                ev.record(self.compute)
                s.busy_until = ev
                in_flight.append((ev, req, res))
                continue
            time.sleep(poll_s if in_flight else min(1e-3, max(0.0, (pending[0].t_arrive - now) if pending else 0.0)))
        torch.cuda.synchronize(self.dev)
        return requests

    def layers_of(self, mi):
        s = self.slots[mi]
        if s.resident:
            if s.ready is not None:
                s.ready.synchronize()
            return [l.clone() for l in s.layers]
        s.spilled.synchronize()
        if self.pool is not None:
            return [h.to(self.dev) for h in s.host["layers"]]
        _, off_l, lb, _, _ = s.lay
        n, side = s.spec.side * s.spec.side, s.spec.side
        return [s.host["image"][off_l + i * lb: off_l + i * lb + n].view(side, side).to(self.dev)
                for i in range(s.spec.n_layers)]


class _Rebind:
    """The lcl_atlas of a spilled model: its struct, ready to be re-bound to a new device buffer."""

    def __init__(self, atlas):
        self.width, self.height, self.tile, self.n_tri = atlas.width, atlas.height, atlas.tile, int(atlas.c.n_tri)
        self.bbox_min, self.scale = list(atlas.c.bbox_min), atlas.c.scale

    def restore(self, buf):
        a = lcl.Atlas(self.width, self.height, self.tile, self.n_tri, buf.device, buffer=buf)
        a.c.bbox_min[:] = self.bbox_min
        a.c.scale = self.scale
        return a


def model_image_layout(spec):
    """Device image of a served model: atlas buffer | layers | depth maps, sections 256-byte aligned.
    Returns (layer offset, layer stride, depth-map offsets, total bytes)."""
    a256 = lambda x: (x + 255) // 256 * 256  # noqa: E731
    ab = int(lcl.library().lcl_atlas_bytes(spec.side, spec.side, spec.tile, spec.mesh.n_tri))
    lb = a256(spec.side * spec.side)
    off_l = a256(ab)
    off = off_l + spec.n_layers * lb
    offs_d = []
    for c in spec.cams:
        offs_d.append(off)
        off += a256(4 * c.width * c.height)
    return off_l, lb, offs_d, off


class NativeServer:
    """The same serving policy run by the library's native loop (lcl_serve_*): admission and eviction
    by recent request rate, per-model FIFO queues, continuous batching with epochs in flight, queries,
    latency per request -- all in a host thread of liblcl.so; Python only prepares the models and
    submits the whole trace (arrival times on the server clock) before collecting completions.

    models: ServedModel list; hbm_budget_bytes: the device arena for model images."""

    def __init__(self, models, hbm_budget_bytes, device="cuda", max_edits_per_layer=lcl.BATCH_MAX_STROKES,
                 max_in_flight=4, max_labels=256, max_queries=16):
        self.dev = torch.device(device)
        self.lib = lcl.library()
        self.specs = list(models)
        self.max_labels = max_labels
        cfg = lcl.lcl_serve_config()
        cfg.arena_bytes = int(hbm_budget_bytes) // 256 * 256
        cfg.max_in_flight, cfg.max_edits, cfg.max_queries, cfg.max_labels = (max_in_flight, max_edits_per_layer,
                                                                              max_queries, max_labels)
        self.ptr = lcl.C.c_void_p()
        lcl._check("lcl_serve_create", self.lib.lcl_serve_create(lcl.C.byref(cfg), lcl.C.byref(self.ptr)))
        self.images, self._keep = [], []
        self.bytes = []
        for spec in self.specs:
            self._register(spec)
        self.arena = torch.empty(cfg.arena_bytes, dtype=torch.uint8, device=self.dev)
        wb = int(self.lib.lcl_serve_work_bytes(self.ptr))
        hb = int(self.lib.lcl_serve_host_work_bytes(self.ptr))
        self.work = torch.empty(max(wb, 256), dtype=torch.uint8, device=self.dev)
        self.host_work = torch.empty(max(hb, 256), dtype=torch.uint8).pin_memory()
        torch.cuda.synchronize(self.dev)
        lcl._check("lcl_serve_start", self.lib.lcl_serve_start(self.ptr, lcl._ptr(self.arena), lcl._ptr(self.work),
                                                               self.work.numel(), lcl._ptr(self.host_work),
                                                               self.host_work.numel()))

    def _register(self, spec):
        """Builds the model's device image (atlas | layers | depth maps) once, keeps it in pinned host
        memory and registers it; the device copy is dropped (the server admits it when needed)."""
        off_l, lb, offs_d, off = model_image_layout(spec)
        buf = torch.zeros(off, dtype=torch.uint8, device=self.dev)
        mesh = lcl.Mesh.from_host(spec.mesh, self.dev)
        atlas = lcl.Atlas(spec.side, spec.side, spec.tile, spec.mesh.n_tri, self.dev, buffer=buf)
        lcl.lcl_atlas_build(mesh, atlas)
        cams = [lcl.lcl_camera_from_vp(atlas, c.vp, c.width, c.height) for c in spec.cams]
        for c, o in zip(cams, offs_d):
            d = buf[o: o + 4 * c.width * c.height].view(torch.float32).view(c.height, c.width)
            lcl.lcl_depth_render(mesh, atlas, c, d)
        image = torch.empty(off, dtype=torch.uint8).pin_memory()
        image.copy_(buf)
        cam_arr = (lcl.lcl_camera * max(len(cams), 1))(*cams)
        offs_arr = (lcl.C.c_size_t * max(len(offs_d), 1))(*offs_d)
        d = lcl.lcl_serve_model()
        d.side, d.tile, d.n_tri, d.n_layers = spec.side, spec.tile, spec.mesh.n_tri, spec.n_layers
        d.bbox_min[:] = list(atlas.c.bbox_min)
        d.scale = atlas.c.scale
        d.cams = lcl.C.cast(cam_arr, lcl.C.c_void_p)
        d.depth_offsets = lcl.C.cast(offs_arr, lcl.C.c_void_p)
        d.n_cams = len(cams)
        d.host_image = image.data_ptr()
        d.image_bytes, d.layer_offset, d.layer_stride = off, off_l, lb
        mid = lcl.C.c_int32()
        lcl._check("lcl_serve_add_model", self.lib.lcl_serve_add_model(self.ptr, lcl.C.byref(d), lcl.C.byref(mid)))
        self.images.append(image)
        self._keep.append((cam_arr, offs_arr))
        self.bytes.append(off)
        del buf, mesh, atlas

    def stats(self):
        st = lcl.lcl_serve_stats()
        lcl._check("lcl_serve_stats_get", self.lib.lcl_serve_stats_get(self.ptr, lcl.C.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    spills = property(lambda self: int(self.stats()["spills"]))
    admissions = property(lambda self: int(self.stats()["admissions"]))
    epochs = property(lambda self: int(self.stats()["epochs"]))

    def run(self, requests, start_delay_s=0.05, stall_limit_s=60.0):
        """Serves `requests` (sorted by t_arrive, seconds from the start) open-loop: the whole trace is
        submitted at once with arrival times on the server clock, then completions are collected;
        fills t_done (seconds from the start) and, for queries, result = (counts, areas)."""
        n = len(requests)
        rec = np.zeros(n, lcl.SERVE_REQUEST_DTYPE)
        n_q = sum(1 for r in requests if r.kind == QUERY)
        results = np.zeros((max(n_q, 1), 2, self.max_labels), np.uint64)
        qi = 0
        base = results.ctypes.data
        for i, r in enumerate(requests):
            x = rec[i]
            x["t_arrive"] = r.t_arrive
            x["tag"] = i
            x["model"] = r.model
            x["kind"] = r.kind
            x["layer"] = r.layer
            if r.kind == SPHERE:
                c, rad, label = r.sphere
                x["centre"] = c
                x["radius"] = rad
                x["label"] = label
            elif r.kind == LASSO:
                ci, poly, label = r.lasso
                poly = np.asarray(poly, np.float32)
                x["cam"] = ci
                x["n_vertices"] = poly.shape[0]
                x["poly"][:2 * poly.shape[0]] = poly.reshape(-1)
                x["label"] = label
            else:
                op, la, lb, n_labels = r.query
                x["op"] = lcl.OPS[op]
                x["layer"], x["layer_b"], x["n_labels"] = la, lb, n_labels
                x["result"] = base + qi * results.strides[0]
                r._qi = qi
                qi += 1
        # the arrival times go on the server clock only now, once the records are ready, so that no
        # request is late before the loop sees it
        t0 = float(self.lib.lcl_serve_clock()) + start_delay_s
        rec["t_arrive"] += t0
        lcl._check("lcl_serve_submit", self.lib.lcl_serve_submit(self.ptr, rec.ctypes.data, n))
        out = (lcl.lcl_serve_done * 4096)()
        got = lcl.C.c_int32()
        left = n
        last = time.perf_counter()
        while left:
            lcl._check("lcl_serve_poll", self.lib.lcl_serve_poll(self.ptr, out, 4096, lcl.C.byref(got)))
            for k in range(got.value):
                r = requests[out[k].tag]
                r.t_done = out[k].t_done - t0
                r.t_launch = out[k].t_launch - t0
                r.t_gpu = out[k].t_gpu
            left -= got.value
            if got.value:
                last = time.perf_counter()
            elif time.perf_counter() - last > stall_limit_s:
                raise RuntimeError(f"serving loop made no progress for {stall_limit_s} s ({left} requests outstanding)")
            else:
                time.sleep(200e-6)
        for r in requests:
            if r.kind == QUERY:
                nl = r.query[3]
                r.result = (results[r._qi, 0, :nl].copy(), results[r._qi, 1, :nl].copy())
        return requests

    def layers_of(self, mi):
        spec = self.specs[mi]
        out = []
        for li in range(spec.n_layers):
            h = np.empty((spec.side, spec.side), np.uint8)
            lcl._check("lcl_serve_read_layer", self.lib.lcl_serve_read_layer(self.ptr, mi, li, h.ctypes.data))
            out.append(torch.from_numpy(h).to(self.dev))
        return out

    def close(self):
        if self.ptr:
            self.lib.lcl_serve_destroy(self.ptr)
            self.ptr = lcl.C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poisson_requests(n_models, rate_hz, duration_s, seed, mix=(0.7, 0.2, 0.1), zipf_s=1.1, n_layers=2,
                     sphere_of=None, lasso_of=None, n_labels=256):
    """Open-loop arrivals: exponential gaps at `rate_hz`, kinds by `mix` (sphere, lasso, query),
    model by a Zipf(zipf_s) law over the models, layers uniform.  sphere_of(model, rng) and
    lasso_of(model, rng) draw the payloads."""
    rng = np.random.default_rng(seed)
    n = int(rate_hz * duration_s)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    w = 1.0 / np.arange(1, n_models + 1) ** zipf_s
    models = rng.choice(n_models, size=n, p=w / w.sum())
    kinds = rng.choice(3, size=n, p=np.array(mix) / sum(mix))
    out = []
    for i in range(n):
        m, k = int(models[i]), int(kinds[i])
        r = Request(float(t[i]), m, k, layer=int(rng.integers(0, n_layers)))
        if k == SPHERE:
            r.sphere = sphere_of(m, rng)
        elif k == LASSO:
            r.lasso = lasso_of(m, rng)
        else:
            r.query = (["and", "or", "xor"][int(rng.integers(0, 3))], 0, 1, n_labels)
        out.append(r)
    return out


def latency_stats(requests):
    lat = np.array([r.t_done - r.t_arrive for r in requests])
    span = max(r.t_done for r in requests) - min(r.t_arrive for r in requests)
    return {"requests": len(requests), "throughput_rps": len(requests) / span, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)), "max_ms": 1e3 * float(lat.max())}
