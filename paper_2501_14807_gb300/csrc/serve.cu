// serve.cu -- the request server: a native loop (one host thread) that keeps many models resident in
// a device arena under a budget, admits and evicts them by recent request rate, and batches queued
// edits and queries of many models into epochs (one batched upload + one graph replay + the queries
// per epoch), several epochs in flight.  The paper's CPU-side manager (Section 4, Fig. 2; the texture
// manager of Section 4.2) for many models at once; every request performs the edit of Section 4.3.1
// through the library's batched edit, so results are those of the single-request calls in per-model
// arrival order.
//
// Ordering and memory rules (the loop thread is the only one that touches model state):
//  - one compute stream runs every epoch in order, so a model's requests run in FIFO order;
//  - one copy stream runs admissions (host image -> arena) and spills (arena layers -> host image) in
//    order, so an arena range freed by a spill can be handed to an admission at once: the admission's
//    copy is queued behind the spill's;
//  - a model is spilled only when its last epoch has completed (the compute stream no longer uses it),
//    and it joins an epoch only once its admission copy has completed;
//  - a slot (workspace, staging, graph, query scratch) is reused only after its epoch has completed;
//  - the compute stream uses no copy engine: an epoch's descriptors are read from the slot's pinned
//    staging, and its query tables written to the slot's pinned tables, by copy kernels through the
//    memory's mapped device address, so epochs never wait behind admission or spill copies (a run with
//    a host-to-device copy loop beside the server made an epoch's GPU time 0.2 ms -> 5.5 ms when the
//    descriptors went through the copy engines).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lcl_impl.cuh"

static_assert(sizeof(lcl_serve_request) == 608, "lcl_serve_request layout");
static_assert(sizeof(lcl_serve_model) == 96, "lcl_serve_model layout");
static_assert(sizeof(lcl_serve_config) == 32 && sizeof(lcl_serve_done) == 32 && sizeof(lcl_serve_stats) == 80,
              "serve struct layouts");

namespace {

constexpr double kTau = 1.0;  // time constant of the request-rate score that picks eviction victims

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct Model {
    lcl_serve_model desc;
    std::vector<lcl_camera> cams;
    std::vector<size_t> depth_off;
    size_t atlas_bytes = 0;
    int32_t tiles = 0, supers = 0;  // per layer
    lcl_atlas atlas;                // bound into the arena while resident
    bool resident = false, admitting = false;
    bool fresh = false;             // admitted for queued work that no epoch has taken yet: not evicted
    size_t off = 0;                 // arena offset while resident
    cudaEvent_t ready = nullptr;    // admission copy done (while admitting)
    int64_t last_seq = -1;          // last epoch that used the model
    double score = 0.0, t_score = 0.0;
    std::deque<const lcl_serve_request *> queue;
    bool in_epoch = false;
};

struct Query {
    const lcl_serve_request *req;
    size_t host_off;  // its tables in the slot's host area
};

struct Slot {
    void *ws = nullptr;
    size_t ws_bytes = 0;
    void *staging = nullptr;
    size_t staging_bytes = 0;
    uint8_t *scratch = nullptr;       // max_queries overlay outputs
    uint64_t *tables = nullptr;       // max_queries x 2 max_labels (device)
    uint64_t *host_tables = nullptr;  // the same (pinned host)
    // device addresses of the pinned staging and host tables (NULL if the memory is not mapped): through
    // them the epoch's descriptors and query tables move by copy kernels on the compute stream, so an
    // epoch never queues behind admission or spill copies on the copy engines
    const void *staging_dev = nullptr;
    uint64_t *host_tables_dev = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool busy = false;
    std::vector<lcl_batch_model> bm;
    std::vector<lcl_batch_stroke> bs;
    std::vector<lcl_batch_lasso> bl;
};

struct Epoch {
    int64_t seq;
    int slot;
    double t_launch;
    cudaEvent_t start = nullptr;  // recorded on the compute stream before the epoch's work (GPU time: start..done)
    cudaEvent_t done = nullptr;
    std::vector<const lcl_serve_request *> reqs;
    std::vector<Query> queries;
};

}  // namespace

struct lcl_server {
    lcl_serve_config cfg;
    int device = 0;
    std::vector<Model> models;
    size_t max_layer_bytes = 0;
    lcl_batch_limits limits;
    // caller memory
    uint8_t *arena = nullptr;
    uint8_t *work = nullptr;
    uint8_t *host_work = nullptr;
    std::map<size_t, size_t> free_ranges;  // arena offset -> bytes
    std::vector<Slot> slots;
    cudaStream_t compute = nullptr, copy = nullptr;
    std::vector<cudaEvent_t> event_pool;
    // requests (submission thread appends under mu; the loop takes them under mu)
    std::mutex mu;
    std::deque<lcl_serve_request> reqs;
    size_t next_release = 0;
    std::vector<lcl_serve_done> done;
    uint64_t n_submitted = 0, n_done = 0;
    lcl_status err = LCL_OK;
    std::string err_msg;
    // loop state
    std::mutex state_mu;  // held by the loop while it changes model state; lcl_serve_read_layer takes it
    std::thread loop;
    std::atomic<bool> stop{false};
    bool started = false;
    std::deque<Epoch> in_flight;
    int64_t next_seq = 0, completed_seq = -1;
    int admitting = 0;
    std::vector<int32_t> active;  // models with queued requests
    // stats
    uint64_t epochs = 0, admissions = 0, spills = 0, resident_bytes = 0, resident_models = 0;
    uint64_t admitted_bytes = 0, deferred = 0;
    double host_busy = 0.0;
};

namespace lcl {
namespace {

size_t image_need(const Model &m) { return a256(m.desc.image_bytes); }

lcl_status loop_fail(lcl_server *s, cudaError_t e, const char *where) {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->err == LCL_OK) {
        s->err = LCL_ERR_CUDA;
        s->err_msg = std::string("serving loop: ") + where + ": " + cudaGetErrorString(e);
    }
    return LCL_ERR_CUDA;
}

lcl_status loop_fail_status(lcl_server *s, lcl_status st, const char *where) {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->err == LCL_OK) {
        s->err = st;
        s->err_msg = std::string("serving loop: ") + where + ": " + lcl_last_error();
    }
    return st;
}

cudaEvent_t take_event(lcl_server *s) {
    if (!s->event_pool.empty()) {
        cudaEvent_t e = s->event_pool.back();
        s->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;  // with timing: an epoch's GPU time is measured between two of them
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

bool arena_alloc(lcl_server *s, size_t bytes, size_t *off) {
    for (auto it = s->free_ranges.begin(); it != s->free_ranges.end(); ++it) {
        if (it->second >= bytes) {
            *off = it->first;
            const size_t rest = it->second - bytes, at = it->first + bytes;
            s->free_ranges.erase(it);
            if (rest) s->free_ranges[at] = rest;
            return true;
        }
    }
    return false;
}

void arena_free(lcl_server *s, size_t off, size_t bytes) {
    auto it = s->free_ranges.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != s->free_ranges.end() && it->first + it->second == next->first) {
        it->second += next->second;
        s->free_ranges.erase(next);
    }
    if (it != s->free_ranges.begin()) {
        auto prev = std::prev(it);
        if (prev->first + prev->second == it->first) {
            prev->second += it->second;
            s->free_ranges.erase(it);
        }
    }
}

double rate(const Model &m, double now) { return m.score * std::exp(-(now - m.t_score) / kTau); }

void touch(Model &m, double now) {
    m.score = rate(m, now) + 1.0;
    m.t_score = now;
}

// Points the model's atlas struct at its arena image.
void bind_resident(lcl_server *s, Model &m) {
    lcl_atlas_bind(s->arena + m.off, m.atlas_bytes, m.desc.side, m.desc.side, m.desc.tile, m.desc.n_tri, &m.atlas);
    for (int a = 0; a < 3; ++a) m.atlas.bbox_min[a] = m.desc.bbox_min[a];
    m.atlas.scale = m.desc.scale;
}

// Copies a resident, idle model's layers back to its host image and frees its arena range (the copy
// stream orders any later admission into that range behind this copy).
lcl_status spill(lcl_server *s, Model &m) {
    const size_t n = (size_t)m.desc.n_layers * m.desc.layer_stride;
    cudaError_t e = cudaMemcpyAsync(static_cast<uint8_t *>(m.desc.host_image) + m.desc.layer_offset,
                                    s->arena + m.off + m.desc.layer_offset, n, cudaMemcpyDeviceToHost, s->copy);
    if (e != cudaSuccess) return loop_fail(s, e, "spill copy");
    arena_free(s, m.off, image_need(m));
    m.resident = false;
    s->resident_bytes -= image_need(m);
    s->resident_models -= 1;
    s->spills += 1;
    return LCL_OK;
}

// Copies a model's image into the arena at `off` on the copy stream and marks it resident (its
// requests may join an epoch once the copy's event has completed).
bool place(lcl_server *s, Model &m, size_t off, bool fresh, lcl_status *st) {
    const size_t need = image_need(m);
    m.off = off;
    cudaError_t e = cudaMemcpyAsync(s->arena + off, m.desc.host_image, m.desc.image_bytes, cudaMemcpyHostToDevice,
                                    s->copy);
    if (e == cudaSuccess) {
        m.ready = take_event(s);
        e = m.ready ? cudaEventRecord(m.ready, s->copy) : cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        *st = loop_fail(s, e, "admission copy");
        return false;
    }
    bind_resident(s, m);
    m.resident = true;
    m.admitting = true;
    m.fresh = fresh;
    s->admitting += 1;
    s->resident_bytes += need;
    s->resident_models += 1;
    s->admissions += 1;
    s->admitted_bytes += m.desc.image_bytes;
    return true;
}

// Admits a model with queued work: frees room by spilling idle resident models with the lowest recent
// request rate (never one in the epoch being built, one being admitted, or one admitted for work no
// epoch has taken yet -- without that rule two models could keep evicting each other), then places it.
// Returns false (nothing placed) if room cannot be made now.
bool admit(lcl_server *s, Model &m, double now, lcl_status *st) {
    const size_t need = image_need(m);
    size_t off = 0;
    while (!arena_alloc(s, need, &off)) {
        Model *victim = nullptr;
        double best = INFINITY;
        for (Model &v : s->models) {
            if (!v.resident || v.admitting || v.fresh || v.in_epoch || &v == &m || v.last_seq > s->completed_seq)
                continue;
            const double r = rate(v, now);
            if (r < best) {
                best = r;
                victim = &v;
            }
        }
        if (!victim) {
            s->deferred += 1;
            return false;
        }
        if ((*st = spill(s, *victim)) != LCL_OK) return false;
    }
    return place(s, m, off, true, st);
}

// Builds and launches one epoch on a free slot; returns false if there was nothing to run.
bool run_epoch(lcl_server *s, double now, lcl_status *st) {
    int si = -1;
    for (int i = 0; i < (int)s->slots.size(); ++i)
        if (!s->slots[i].busy) {
            si = i;
            break;
        }
    if (si < 0) return false;
    Slot &sl = s->slots[si];
    sl.bm.clear();
    sl.bs.clear();
    sl.bl.clear();
    Epoch ep;
    ep.seq = s->next_seq;
    ep.slot = si;
    std::vector<int32_t> used;
    std::vector<cudaEvent_t> waits;
    const int32_t max_edits = s->cfg.max_edits;
    for (size_t ai = 0; ai < s->active.size(); ++ai) {
        const int32_t mi = s->active[ai];
        Model &m = s->models[mi];
        if (m.queue.empty()) continue;
        if (!m.resident) {
            if (s->admitting < s->cfg.max_admitting) admit(s, m, now, st);
            if (*st != LCL_OK) return false;
            continue;  // its requests join an epoch after the copy
        }
        if (m.admitting) continue;
        // leading edits (at most max_edits per layer)
        int32_t per_layer[256] = {0};
        std::vector<const lcl_serve_request *> edits;
        while (!m.queue.empty()) {
            const lcl_serve_request *r = m.queue.front();
            if (r->kind == LCL_REQ_QUERY || per_layer[r->layer] >= max_edits) break;
            per_layer[r->layer] += 1;
            edits.push_back(r);
            m.queue.pop_front();
        }
        // then the query that follows them (it runs after the epoch's edits on the same stream, so it
        // sees them; later edits wait for the next epoch)
        if (!m.queue.empty() && m.queue.front()->kind == LCL_REQ_QUERY &&
            (int32_t)ep.queries.size() < s->cfg.max_queries) {
            const lcl_serve_request *r = m.queue.front();
            m.queue.pop_front();
            ep.queries.push_back({r, 0});
            ep.reqs.push_back(r);
        } else if (edits.empty()) {
            continue;
        }
        m.in_epoch = true;
        m.fresh = false;
        used.push_back(mi);
        for (int32_t li = 0; li < m.desc.n_layers && !edits.empty(); ++li) {
            if (!per_layer[li]) continue;
            lcl_batch_model b;
            std::memset(&b, 0, sizeof(b));
            b.atlas = &m.atlas;
            b.layer = s->arena + m.off + m.desc.layer_offset + (size_t)li * m.desc.layer_stride;
            b.dtype = LCL_U8;
            b.first_stroke = (int32_t)sl.bs.size();
            for (const lcl_serve_request *r : edits) {
                if (r->layer != li) continue;
                lcl_batch_stroke k;
                std::memset(&k, 0, sizeof(k));
                if (r->kind == LCL_REQ_SPHERE) {
                    k.kind = LCL_STROKE_SPHERE;
                    if (lcl_quantize_sphere(&m.atlas, r->centre, r->radius, (uint32_t)r->label, &k.sphere) != LCL_OK) {
                        *st = loop_fail_status(s, LCL_ERR_INVALID_ARG, "sphere request");
                        return false;
                    }
                } else {
                    k.kind = LCL_STROKE_LASSO;
                    k.lasso = (int32_t)sl.bl.size();
                    lcl_batch_lasso L;
                    std::memset(&L, 0, sizeof(L));
                    L.camera = m.cams[r->cam];
                    L.depth = reinterpret_cast<const float *>(s->arena + m.off + m.depth_off[r->cam]);
                    L.poly_xy = r->poly;
                    L.n_vertices = r->n_vertices;
                    L.label = (uint32_t)r->label;
                    L.bias = 1.0f / 1024.0f;
                    sl.bl.push_back(L);
                }
                sl.bs.push_back(k);
            }
            b.n_strokes = (int32_t)sl.bs.size() - b.first_stroke;
            sl.bm.push_back(b);
        }
        ep.reqs.insert(ep.reqs.end(), edits.begin(), edits.end());
    }
    for (int32_t mi : used) s->models[mi].in_epoch = false;
    if (ep.reqs.empty()) return false;
    ep.start = take_event(s);
    // a failure from here on ends the loop; the epoch's events go back to the pool (freed by destroy)
    auto abandon = [&](lcl_status fs) {
        if (ep.start) s->event_pool.push_back(ep.start);
        if (ep.done) s->event_pool.push_back(ep.done);
        *st = fs;
        return false;
    };
    cudaError_t e = ep.start ? cudaEventRecord(ep.start, s->compute) : cudaErrorMemoryAllocation;
    if (e != cudaSuccess) return abandon(loop_fail(s, e, "epoch start event"));
    if (!sl.bm.empty()) {
        const lcl_status us = batch_upload_impl(&s->limits, sl.bm.data(), (int32_t)sl.bm.size(), sl.bs.data(),
                                                (int32_t)sl.bs.size(), sl.bl.data(), (int32_t)sl.bl.size(), sl.ws,
                                                sl.ws_bytes, sl.staging, sl.staging_bytes, s->compute, sl.staging_dev);
        if (us != LCL_OK) return abandon(loop_fail_status(s, us, "batch upload"));
        e = cudaGraphLaunch(sl.graph, s->compute);
        if (e != cudaSuccess) return abandon(loop_fail(s, e, "batch graph launch"));
    }
    const size_t n_tab = 2 * (size_t)s->cfg.max_labels;
    for (size_t qi = 0; qi < ep.queries.size(); ++qi) {
        Query &q = ep.queries[qi];
        const lcl_serve_request *r = q.req;
        Model &m = s->models[r->model];
        const uint8_t *la = s->arena + m.off + m.desc.layer_offset + (size_t)r->layer * m.desc.layer_stride;
        const uint8_t *lb = s->arena + m.off + m.desc.layer_offset + (size_t)r->layer_b * m.desc.layer_stride;
        uint8_t *out = sl.scratch + qi * s->max_layer_bytes;
        uint64_t *tab = sl.tables + qi * n_tab;
        lcl_status qs = overlay_impl(&m.atlas, la, lb, out, 1, r->op, 0u, s->compute);
        if (qs == LCL_OK) qs = label_area_impl(&m.atlas, out, 1, (uint32_t)r->n_labels, tab, tab + r->n_labels, s->compute);
        if (qs != LCL_OK) return abandon(loop_fail_status(s, qs, "query launch"));
        q.host_off = qi * n_tab;
        e = sl.host_tables_dev ? copy_by_kernel(sl.host_tables_dev + q.host_off, tab, 16 * (size_t)r->n_labels, s->compute)
                               : cudaMemcpyAsync(sl.host_tables + q.host_off, tab, 16 * (size_t)r->n_labels,
                                                 cudaMemcpyDeviceToHost, s->compute);
        if (e != cudaSuccess) return abandon(loop_fail(s, e, "query result copy"));
    }
    ep.done = take_event(s);
    e = ep.done ? cudaEventRecord(ep.done, s->compute) : cudaErrorMemoryAllocation;
    if (e != cudaSuccess) return abandon(loop_fail(s, e, "epoch event"));
    for (int32_t mi : used) s->models[mi].last_seq = ep.seq;
    ep.t_launch = now_s();
    sl.busy = true;
    s->next_seq += 1;
    s->epochs += 1;
    s->in_flight.push_back(std::move(ep));
    return true;
}

void serve_loop(lcl_server *s) {
    cudaSetDevice(s->device);
    lcl_status st = LCL_OK;
    while (!s->stop.load(std::memory_order_relaxed) && st == LCL_OK) {
        bool worked = false;
        {
            std::lock_guard<std::mutex> state(s->state_mu);
            const double now = now_s();
            // arrivals whose time has come
            {
                std::lock_guard<std::mutex> lock(s->mu);
                while (s->next_release < s->reqs.size() && s->reqs[s->next_release].t_arrive <= now) {
                    const lcl_serve_request *r = &s->reqs[s->next_release++];
                    Model &m = s->models[r->model];
                    if (m.queue.empty()) s->active.push_back(r->model);
                    m.queue.push_back(r);
                    touch(m, now);
                }
            }
            // completed epochs (in order on the compute stream)
            while (!s->in_flight.empty()) {
                Epoch &ep = s->in_flight.front();
                const cudaError_t q = cudaEventQuery(ep.done);
                if (q == cudaErrorNotReady) break;
                if (q != cudaSuccess) {
                    st = loop_fail(s, q, "epoch");
                    break;
                }
                const double t = now_s();
                float gpu_ms = 0.0f;
                if (cudaEventElapsedTime(&gpu_ms, ep.start, ep.done) != cudaSuccess) gpu_ms = -1.0f;
                Slot &sl = s->slots[ep.slot];
                for (const Query &qq : ep.queries)
                    std::memcpy(qq.req->result, sl.host_tables + qq.host_off, 16 * (size_t)qq.req->n_labels);
                {
                    std::lock_guard<std::mutex> lock(s->mu);
                    for (const lcl_serve_request *r : ep.reqs)
                        s->done.push_back({r->tag, t, ep.t_launch, gpu_ms < 0.0f ? -1.0 : 1e-3 * gpu_ms});
                    s->n_done += ep.reqs.size();
                }
                s->completed_seq = ep.seq;
                sl.busy = false;
                s->event_pool.push_back(ep.done);
                s->event_pool.push_back(ep.start);
                s->in_flight.pop_front();
                worked = true;
            }
            if (st != LCL_OK) break;
            // admissions whose copy is done
            for (Model &m : s->models) {
                if (!m.admitting) continue;
                const cudaError_t q = cudaEventQuery(m.ready);
                if (q == cudaErrorNotReady) continue;
                if (q != cudaSuccess) {
                    st = loop_fail(s, q, "admission");
                    break;
                }
                cudaStreamWaitEvent(s->compute, m.ready, 0);  // orders the compute stream after the copy
                s->event_pool.push_back(m.ready);
                m.ready = nullptr;
                m.admitting = false;
                s->admitting -= 1;
                worked = true;
            }
            if (st != LCL_OK) break;
            // drop models whose queues ran empty from the active list
            size_t k = 0;
            for (size_t i = 0; i < s->active.size(); ++i)
                if (!s->models[s->active[i]].queue.empty()) s->active[k++] = s->active[i];
            s->active.resize(k);
            if (!s->active.empty() && (int32_t)s->in_flight.size() < s->cfg.max_in_flight) {
                const double t0 = now_s();
                if (run_epoch(s, now, &st)) worked = true;
                s->host_busy += now_s() - t0;
            }
        }
        if (!worked) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace
}  // namespace lcl

using namespace lcl;

extern "C" {

double lcl_serve_clock(void) { return now_s(); }

lcl_status lcl_serve_create(const lcl_serve_config *config, lcl_server **out) {
    if (!config || !out) return fail(LCL_ERR_INVALID_ARG, "NULL argument");
    lcl_serve_config c = *config;
    if (c.max_in_flight == 0) c.max_in_flight = 4;
    if (c.max_edits == 0) c.max_edits = LCL_BATCH_MAX_STROKES;
    if (c.max_queries == 0) c.max_queries = 16;
    if (c.max_labels == 0) c.max_labels = 256;
    if (c.max_admitting == 0) c.max_admitting = 16;
    if (c.arena_bytes < 256 || c.max_in_flight < 1 || c.max_in_flight > 8 || c.max_edits < 1 ||
        c.max_edits > LCL_BATCH_MAX_STROKES || c.max_queries < 1 || c.max_queries > 1024 || c.max_labels < 1 ||
        c.max_labels > 65536 || c.max_admitting < 1 || c.max_admitting > 1024)
        return fail(LCL_ERR_INVALID_ARG, "serve config out of range");
    lcl_server *s = new lcl_server();
    s->cfg = c;
    cudaGetDevice(&s->device);
    *out = s;
    return LCL_OK;
}

lcl_status lcl_serve_add_model(lcl_server *s, const lcl_serve_model *d, int32_t *id) {
    if (!s || !d || !id) return fail(LCL_ERR_INVALID_ARG, "NULL argument");
    if (s->started) return fail(LCL_ERR_UNSUPPORTED, "models are registered before lcl_serve_start");
    const size_t ab = lcl_atlas_bytes(d->side, d->side, d->tile, d->n_tri);
    if (!ab || d->n_layers < 1 || d->n_layers > 256 || d->n_cams < 0 || d->n_cams > 1024 || !d->host_image ||
        !(d->scale > 0.0) || (d->n_cams && (!d->cams || !d->depth_offsets)))
        return fail(LCL_ERR_INVALID_ARG, "serve model: sizes, counts or pointers");
    const size_t plane = (size_t)d->side * d->side;
    if (d->layer_offset < ab || d->layer_offset % 256 || d->layer_stride < plane || d->layer_stride % 256 ||
        d->layer_offset + (size_t)d->n_layers * d->layer_stride > d->image_bytes)
        return fail(LCL_ERR_INVALID_ARG, "serve model: layer layout outside the image");
    for (int32_t c = 0; c < d->n_cams; ++c) {
        const lcl_camera &cam = d->cams[c];
        if (cam.width < 1 || cam.height < 1 || cam.width > 16384 || cam.height > 16384 || d->depth_offsets[c] % 256 ||
            d->depth_offsets[c] + 4 * (size_t)cam.width * cam.height > d->image_bytes)
            return fail(LCL_ERR_INVALID_ARG, "serve model: camera or depth map outside the image");
    }
    if (a256(d->image_bytes) > s->cfg.arena_bytes) return fail(LCL_ERR_INVALID_ARG, "serve model larger than the arena");
    Model m;
    m.desc = *d;
    m.cams.assign(d->cams, d->cams + d->n_cams);
    m.depth_off.assign(d->depth_offsets, d->depth_offsets + d->n_cams);
    m.desc.cams = nullptr;
    m.desc.depth_offsets = nullptr;
    m.atlas_bytes = ab;
    const int32_t t = (d->side + d->tile - 1) / d->tile, sp = (t + LCL_SUPER - 1) / LCL_SUPER;
    m.tiles = t * t;
    m.supers = sp * sp;
    std::memset(&m.atlas, 0, sizeof(m.atlas));
    s->max_layer_bytes = std::max(s->max_layer_bytes, a256(plane));
    *id = (int32_t)s->models.size();
    s->models.push_back(std::move(m));
    return LCL_OK;
}

static void serve_limits(const lcl_server *s, lcl_batch_limits *lim) {
    std::memset(lim, 0, sizeof(*lim));
    int64_t pairs = 0, supers = 0, tiles = 0;
    for (const Model &m : s->models) {
        pairs += m.desc.n_layers;
        supers += (int64_t)m.desc.n_layers * m.supers;
        tiles += (int64_t)m.desc.n_layers * m.tiles;
    }
    lim->models = (int32_t)std::max<int64_t>(pairs, 1);
    lim->strokes = (int32_t)std::max<int64_t>(pairs * s->cfg.max_edits, 1);
    lim->lassos = lim->strokes;
    lim->supers = std::max<int64_t>(supers, 1);
    lim->tiles = std::max<int64_t>(tiles, 1);
}

static size_t slot_device_bytes(const lcl_server *s, const lcl_batch_limits &lim) {
    return a256(lcl_batch_workspace_bytes(&lim)) + a256(s->cfg.max_queries * s->max_layer_bytes) +
           a256((size_t)s->cfg.max_queries * 16 * s->cfg.max_labels);
}

static size_t slot_host_bytes(const lcl_server *s, const lcl_batch_limits &lim) {
    return a256(lcl_batch_staging_bytes(&lim)) + a256((size_t)s->cfg.max_queries * 16 * s->cfg.max_labels);
}

size_t lcl_serve_work_bytes(const lcl_server *s) {
    if (!s) return 0;
    lcl_batch_limits lim;
    serve_limits(s, &lim);
    return (size_t)s->cfg.max_in_flight * slot_device_bytes(s, lim);
}

size_t lcl_serve_host_work_bytes(const lcl_server *s) {
    if (!s) return 0;
    lcl_batch_limits lim;
    serve_limits(s, &lim);
    return (size_t)s->cfg.max_in_flight * slot_host_bytes(s, lim);
}

lcl_status lcl_serve_start(lcl_server *s, void *arena, void *work, size_t work_bytes, void *host_work,
                           size_t host_work_bytes) {
    if (!s || !arena || !work || !host_work) return fail(LCL_ERR_INVALID_ARG, "NULL argument");
    if (s->started) return fail(LCL_ERR_UNSUPPORTED, "server already started");
    if (s->models.empty()) return fail(LCL_ERR_INVALID_ARG, "no models registered");
    if ((reinterpret_cast<uintptr_t>(arena) | reinterpret_cast<uintptr_t>(work)) & 255)
        return fail(LCL_ERR_INVALID_ARG, "arena and work must be 256-byte aligned");
    if (reinterpret_cast<uintptr_t>(host_work) & 15) return fail(LCL_ERR_INVALID_ARG, "host work must be 16-byte aligned");
    if (work_bytes < lcl_serve_work_bytes(s) || host_work_bytes < lcl_serve_host_work_bytes(s))
        return fail(LCL_ERR_OUT_OF_MEMORY, "work buffers smaller than lcl_serve_work_bytes / lcl_serve_host_work_bytes");
    s->arena = static_cast<uint8_t *>(arena);
    s->work = static_cast<uint8_t *>(work);
    s->host_work = static_cast<uint8_t *>(host_work);
    s->free_ranges.clear();
    s->free_ranges[0] = s->cfg.arena_bytes & ~size_t(255);
    serve_limits(s, &s->limits);
    cudaError_t e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "lcl_serve_start: streams");
    const size_t dev_slot = slot_device_bytes(s, s->limits), host_slot = slot_host_bytes(s, s->limits);
    s->slots.resize(s->cfg.max_in_flight);
    for (int i = 0; i < s->cfg.max_in_flight; ++i) {
        Slot &sl = s->slots[i];
        uint8_t *d = s->work + i * dev_slot;
        uint8_t *h = s->host_work + i * host_slot;
        sl.ws_bytes = lcl_batch_workspace_bytes(&s->limits);
        sl.ws = d;
        sl.scratch = d + a256(sl.ws_bytes);
        sl.tables = reinterpret_cast<uint64_t *>(sl.scratch + a256(s->cfg.max_queries * s->max_layer_bytes));
        sl.staging_bytes = lcl_batch_staging_bytes(&s->limits);
        sl.staging = h;
        sl.host_tables = reinterpret_cast<uint64_t *>(h + a256(sl.staging_bytes));
        void *dp = nullptr;
        if (cudaHostGetDevicePointer(&dp, sl.staging, 0) == cudaSuccess && dp) {
            sl.staging_dev = dp;
            dp = nullptr;
            if (cudaHostGetDevicePointer(&dp, sl.host_tables, 0) == cudaSuccess && dp)
                sl.host_tables_dev = static_cast<uint64_t *>(dp);
        }
        cudaGetLastError();  // a host buffer that is not mapped leaves the copy-engine path
        // one captured graph of the batched launch per slot: its shape depends only on the limits
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(s->compute, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "lcl_serve_start: capture");
        const lcl_status ls = batch_launch_impl(&s->limits, nullptr, sl.ws, sl.ws_bytes, s->compute);
        e = cudaStreamEndCapture(s->compute, &g);
        if (ls != LCL_OK) return ls;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&sl.graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "lcl_serve_start: graph");
    }
    // the first models, in registration order, while they fit
    for (Model &m : s->models) {
        lcl_status st = LCL_OK;
        size_t off = 0;
        if (!arena_alloc(s, image_need(m), &off)) continue;
        if (!place(s, m, off, false, &st)) return fail(st == LCL_OK ? LCL_ERR_CUDA : st, s->err_msg);
    }
    s->started = true;
    s->loop = std::thread(serve_loop, s);
    return LCL_OK;
}

lcl_status lcl_serve_submit(lcl_server *s, const lcl_serve_request *r, int32_t n) {
    if (!s || (n > 0 && !r) || n < 0) return fail(LCL_ERR_INVALID_ARG, "NULL argument or negative count");
    for (int32_t i = 0; i < n; ++i) {
        const lcl_serve_request &q = r[i];
        if (q.model < 0 || q.model >= (int32_t)s->models.size()) return fail(LCL_ERR_INVALID_ARG, "request model");
        const Model &m = s->models[q.model];
        if (q.layer < 0 || q.layer >= m.desc.n_layers) return fail(LCL_ERR_INVALID_ARG, "request layer");
        if (!std::isfinite(q.t_arrive)) return fail(LCL_ERR_INVALID_ARG, "request arrival time");
        if (q.kind == LCL_REQ_SPHERE) {
            if (q.label < 0 || q.label > 255 || !(q.radius >= 0.0) || !std::isfinite(q.radius) ||
                !std::isfinite(q.centre[0]) || !std::isfinite(q.centre[1]) || !std::isfinite(q.centre[2]))
                return fail(LCL_ERR_INVALID_ARG, "sphere request");
            lcl_sphere tmp;
            lcl_atlas probe;
            std::memset(&probe, 0, sizeof(probe));
            for (int a = 0; a < 3; ++a) probe.bbox_min[a] = m.desc.bbox_min[a];
            probe.scale = m.desc.scale;
            if (lcl_quantize_sphere(&probe, q.centre, q.radius, 1u, &tmp) != LCL_OK) return LCL_ERR_INVALID_ARG;
        } else if (q.kind == LCL_REQ_LASSO) {
            if (q.label < 0 || q.label > 255 || q.cam < 0 || q.cam >= m.desc.n_cams || q.n_vertices < 3 ||
                q.n_vertices > LCL_MAX_LASSO_VERTICES)
                return fail(LCL_ERR_INVALID_ARG, "lasso request");
            for (int k = 0; k < 2 * q.n_vertices; ++k)
                if (!std::isfinite(q.poly[k])) return fail(LCL_ERR_INVALID_ARG, "lasso request polygon");
        } else if (q.kind == LCL_REQ_QUERY) {
            if (q.layer_b < 0 || q.layer_b >= m.desc.n_layers || q.op < LCL_AND || q.op > LCL_MASK || !q.result ||
                q.n_labels < 1 || q.n_labels > s->cfg.max_labels)
                return fail(LCL_ERR_INVALID_ARG, "query request");
        } else {
            return fail(LCL_ERR_INVALID_ARG, "request kind");
        }
    }
    std::lock_guard<std::mutex> lock(s->mu);
    double last = s->reqs.empty() ? -INFINITY : s->reqs.back().t_arrive;
    for (int32_t i = 0; i < n; ++i) {
        if (r[i].t_arrive < last) return fail(LCL_ERR_INVALID_ARG, "requests must come in order of arrival time");
        last = r[i].t_arrive;
    }
    for (int32_t i = 0; i < n; ++i) s->reqs.push_back(r[i]);
    s->n_submitted += (uint64_t)n;
    return LCL_OK;
}

lcl_status lcl_serve_poll(lcl_server *s, lcl_serve_done *out, int32_t max, int32_t *n_out) {
    if (!s || !n_out || max < 0 || (max > 0 && !out)) return fail(LCL_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    const int32_t n = (int32_t)std::min<size_t>((size_t)max, s->done.size());
    std::copy(s->done.begin(), s->done.begin() + n, out);
    s->done.erase(s->done.begin(), s->done.begin() + n);
    *n_out = n;
    if (s->err != LCL_OK) return fail(s->err, s->err_msg);
    return LCL_OK;
}

lcl_status lcl_serve_stats_get(lcl_server *s, lcl_serve_stats *out) {
    if (!s || !out) return fail(LCL_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> state(s->state_mu);
    std::lock_guard<std::mutex> lock(s->mu);
    out->submitted = s->n_submitted;
    out->done = s->n_done;
    out->epochs = s->epochs;
    out->admissions = s->admissions;
    out->spills = s->spills;
    out->resident_bytes = s->resident_bytes;
    out->resident_models = s->resident_models;
    out->host_busy_s = s->host_busy;
    out->admitted_bytes = s->admitted_bytes;
    out->deferred = s->deferred;
    return LCL_OK;
}

lcl_status lcl_serve_read_layer(lcl_server *s, int32_t model, int32_t layer, void *dst) {
    if (!s || !dst || model < 0 || model >= (int32_t)s->models.size()) return fail(LCL_ERR_INVALID_ARG, "bad argument");
    Model &m = s->models[model];
    if (layer < 0 || layer >= m.desc.n_layers) return fail(LCL_ERR_INVALID_ARG, "bad layer");
    for (;;) {  // every submitted request done
        {
            std::lock_guard<std::mutex> lock(s->mu);
            if (s->err != LCL_OK) return fail(s->err, s->err_msg);
            if (s->n_done == s->n_submitted) break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    std::lock_guard<std::mutex> state(s->state_mu);
    cudaError_t e = cudaStreamSynchronize(s->copy);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->compute);
    if (e != cudaSuccess) return cuda_fail(e, "lcl_serve_read_layer");
    const size_t plane = (size_t)m.desc.side * m.desc.side, off = m.desc.layer_offset + (size_t)layer * m.desc.layer_stride;
    if (m.resident) {
        e = cudaMemcpy(dst, s->arena + m.off + off, plane, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "lcl_serve_read_layer copy");
    } else {
        std::memcpy(dst, static_cast<const uint8_t *>(m.desc.host_image) + off, plane);
    }
    return LCL_OK;
}

lcl_status lcl_serve_destroy(lcl_server *s) {
    if (!s) return LCL_OK;
    s->stop.store(true);
    if (s->loop.joinable()) s->loop.join();
    if (s->compute) cudaStreamSynchronize(s->compute);
    if (s->copy) cudaStreamSynchronize(s->copy);
    for (Slot &sl : s->slots)
        if (sl.graph) cudaGraphExecDestroy(sl.graph);
    for (Epoch &ep : s->in_flight) {
        if (ep.done) cudaEventDestroy(ep.done);
        if (ep.start) cudaEventDestroy(ep.start);
    }
    for (Model &m : s->models)
        if (m.ready) cudaEventDestroy(m.ready);
    for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
    if (s->compute) cudaStreamDestroy(s->compute);
    if (s->copy) cudaStreamDestroy(s->copy);
    delete s;
    return LCL_OK;
}

}  // extern "C"
