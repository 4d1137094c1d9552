// Batched multi-scene decode: every pipeline stage of all scenes of a batch runs as one
// persistent, work-stealing launch (the scenes are independent, Sec. 3.4.2 decodes each
// scene's groups in parallel; a batch widens the same parallelism across scenes).
//
// Plan (host, once): every scene gets its scratch carve-out, and every stage gets a work list:
// the parameter block of each scene that has work in the stage and the prefix sums of the
// scenes' item counts (an item is one CTA of the single-scene kernel).  The lists go to
// device memory once.  Run: a fixed number of launches -- static tables; attributes per
// coding mode; raw geometry copy, geometry tokens, duplicate prefix; popcount scan with the
// parent scatter; leaf walk -- enqueued without allocation or host synchronisation, so a
// run can be captured in a CUDA graph.  Each launch
// is a grid of resident CTAs that claim items from an atomic counter in increasing order.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "sgs_ctx.h"
#include "sgs_device.cuh"
#include "sgs_internal.h"

namespace sgs {

int resident_ctas(const void *kernel, int threads, size_t smem) {
    struct Entry {
        const void *kernel;
        int device, threads;
        size_t smem;
        int ctas;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry &e : cache)
        if (e.kernel == kernel && e.device == dev && e.threads == threads && e.smem == smem) return e.ctas;
    int per = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    cache.push_back({kernel, dev, threads, smem, per * sms});
    return per * sms;
}

namespace {

constexpr int kMaxLaunches = 16 + SGS_MAX_DEPTH;

enum Kind { K_TABLES, K_FIXED, K_ATTR, K_LEARNED, K_COPY, K_GEO, K_DUP, K_SCAN, K_WALK, K_LEARNED_PE };
enum Role { R_MAIN, R_ATTR, R_GEO };

struct LaunchRec {
    Kind kind;
    int variant;   // vector / out_index variant
    Role role;
    uint64_t prefix_off, param_off, scene_off;  // byte offsets in the plan's list area
    uint32_t stride;
    int n;
    uint32_t total;
};

inline uint64_t a256(uint64_t x) { return (x + 255) & ~255ull; }
inline uint64_t a16(uint64_t x) { return (x + 15) & ~15ull; }

size_t stage_bytes(Kind k) {
    switch (k) {
        case K_TABLES: return stage_tables_bytes();
        case K_FIXED: return stage_fixed_bytes();
        case K_ATTR: return stage_rans_attr_bytes();
        case K_LEARNED: return stage_learned_bytes();
        case K_COPY: return stage_geo_copy_bytes();
        case K_GEO: return stage_rans_geo_bytes();
        case K_DUP: return stage_dup_bytes();
        case K_SCAN: return stage_scan_bytes();
        case K_LEARNED_PE: return stage_learned_pe_bytes();
        default: return stage_walk_bytes();
    }
}

uint32_t stage_items(Kind k, int variant, const SceneRef &r, void *par) {
    switch (k) {
        case K_TABLES: return stage_tables(r, par);
        case K_FIXED: return r.info->mode == SGS_MODE_FIXED ? stage_fixed(r, variant != 0, par) : 0;
        case K_ATTR: return stage_rans_attr(r, variant != 0, par);
        case K_LEARNED: return stage_learned(r, par);
        case K_COPY: return stage_geo_copy(r, par);
        case K_GEO: return stage_rans_geo(r, par);
        case K_DUP: return stage_dup(r, par);
        case K_SCAN: return stage_scan(r, variant, par);
        case K_LEARNED_PE: return stage_learned_pe(r, par);
        default: return stage_walk(r, par);
    }
}

cudaError_t launch_kind(Kind k, int variant, const MultiArgs &m, cudaStream_t st) {
    switch (k) {
        case K_TABLES: return launch_tables_multi(m, st);
        case K_FIXED: return launch_fixed_multi(variant != 0, m, st);
        case K_ATTR: return launch_rans_attr_multi(variant != 0, m, st);
        case K_LEARNED: return launch_learned_multi(m, st);
        case K_COPY: return launch_geo_copy_multi(m, st);
        case K_GEO: return launch_rans_geo_multi(m, st);
        case K_DUP: return launch_dup_multi(m, st);
        case K_SCAN: return launch_scan_multi(variant, m, st);
        case K_LEARNED_PE: return launch_learned_pe_multi(m, st);
        default: return launch_walk_multi(m, st);
    }
}

// First kernel of a run: zeroes the counters, status words, completion counts and times
// (n16 16-byte units) and stamps the run's start on the device global timer.
__global__ void k_run_begin(uint4 *zero, uint32_t n16, unsigned long long *t_start) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += gridDim.x * blockDim.x)
        zero[i] = make_uint4(0, 0, 0, 0);
    if (blockIdx.x == 0 && threadIdx.x == 0) *t_start = globaltimer_ns();
}

__global__ void k_status_fold(const int *status, int n, int *out) {
    int worst = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) worst = min(worst, status[i]);
    for (int o = 16; o > 0; o >>= 1) worst = min(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if ((threadIdx.x & 31) == 0 && worst < 0) atomicMin(out, worst);
}

}  // namespace

// Device layout of a plan, from `base`:
//   scene scratch (each a256) | counters[kMaxLaunches] | status[n] | done[n] | t_done[n] |
//   t_start | lists (per launch: prefix, scene ids, parameters; then need[n])
// Every run zeroes the span from the counters to t_done.
struct BatchLayout {
    std::vector<Scratch> scratch;
    std::vector<GeoPlan> plans;
    std::vector<LaunchRec> launches;
    std::vector<uint8_t> lists;  // uploaded to lists_off
    std::vector<uint32_t> need;  // work items of each scene over all launches
    std::vector<sgs_scene_out> outs;  // each scene's outputs as the stages see them
    uint64_t zero_off, zero_bytes, status_off, done_off, times_off, start_off, need_off, lists_off, total;
};

static int build_layout(const sgs_batch_item *items, int n, uint8_t *base, BatchLayout *L) {
    L->scratch.assign(n, Scratch());
    L->plans.assign(n, GeoPlan());
    L->outs.assign(n, sgs_scene_out());
    L->launches.clear();
    L->lists.clear();
    uint64_t off = 0;
    for (int i = 0; i < n; ++i) {
        const sgs_batch_item &it = items[i];
        if (!it.bits_dev || ((uintptr_t)it.bits_dev & 15)) return SGS_E_INVALID;
        if (it.info.n_rows && (!it.out.attr || !it.out.pos)) return SGS_E_INVALID;
        // learned geometry decodes level by level (a launch sequence per scene): scene_decode only
        if (it.info.geo_mode == SGS_GEO_LEARNED && it.info.n_geo_coded) return SGS_E_UNSUPPORTED;
        const size_t need = scratch_need(it.info, nullptr, nullptr);
        if (need != it.info.scratch_bytes) return SGS_E_INVALID;  // info not from scene_query
        scratch_need(it.info, &L->scratch[i], base ? base + off : nullptr);
        L->outs[i] = effective_out(it.info, it.out, L->scratch[i]);
        make_geo_plan(it.info, &L->plans[i]);
        off += a256(need);
    }
    L->zero_off = off;
    off += a256(4ull * kMaxLaunches);
    L->status_off = off;
    off += a256(4ull * (n > 0 ? n : 1));
    L->done_off = off;
    off += a256(4ull * (n > 0 ? n : 1));
    L->times_off = off;
    off += a256(8ull * (n > 0 ? n : 1));
    L->zero_bytes = off - L->zero_off;
    L->start_off = off;
    off += 256;
    L->lists_off = off;
    L->need.assign(n, 0);
    std::vector<SceneRef> refs(n);
    for (int i = 0; i < n; ++i) {
        refs[i].bits = items[i].bits_dev;
        refs[i].info = &items[i].info;
        refs[i].out = &L->outs[i];
        refs[i].s = &L->scratch[i];
        refs[i].plan = &L->plans[i];
        refs[i].status = reinterpret_cast<int *>(base ? base + L->status_off + 4ull * i : nullptr);
    }
    alignas(16) uint8_t par[1024];
    auto add = [&](Kind k, int variant, Role role) -> int {
        const size_t bytes = stage_bytes(k);
        if (bytes > sizeof(par)) return SGS_E_UNSUPPORTED;
        LaunchRec rec;
        rec.kind = k;
        rec.variant = variant;
        rec.role = role;
        rec.stride = (uint32_t)a16(bytes);
        std::vector<uint32_t> prefix(1, 0), scene;
        std::vector<uint8_t> params;
        for (int i = 0; i < n; ++i) {
            memset(par, 0, sizeof(par));
            const uint32_t c = stage_items(k, variant, refs[i], par);
            if (!c) continue;
            if ((uint64_t)prefix.back() + c >= (1ull << 31)) return SGS_E_UNSUPPORTED;
            if ((uint64_t)L->need[i] + c >= (1ull << 31)) return SGS_E_UNSUPPORTED;
            params.insert(params.end(), par, par + rec.stride);
            prefix.push_back(prefix.back() + c);
            scene.push_back((uint32_t)i);
        }
        rec.n = (int)prefix.size() - 1;
        rec.total = prefix.back();
        if (rec.total == 0) return SGS_OK;
        if ((int)L->launches.size() >= kMaxLaunches) return SGS_E_UNSUPPORTED;
        L->lists.resize(a16(L->lists.size()));
        rec.prefix_off = L->lists.size();
        L->lists.insert(L->lists.end(), reinterpret_cast<uint8_t *>(prefix.data()),
                        reinterpret_cast<uint8_t *>(prefix.data() + prefix.size()));
        L->lists.resize(a16(L->lists.size()));
        rec.scene_off = L->lists.size();
        L->lists.insert(L->lists.end(), reinterpret_cast<uint8_t *>(scene.data()),
                        reinterpret_cast<uint8_t *>(scene.data() + scene.size()));
        L->lists.resize(a16(L->lists.size()));
        rec.param_off = L->lists.size();
        L->lists.insert(L->lists.end(), params.begin(), params.end());
        for (size_t j = 0; j < scene.size(); ++j) L->need[scene[j]] += prefix[j + 1] - prefix[j];
        L->launches.push_back(rec);
        return SGS_OK;
    };
    int rc = add(K_TABLES, 0, R_MAIN);
    for (int v = 0; v < 2 && rc == SGS_OK; ++v) rc = add(K_FIXED, 1 - v, R_ATTR);
    for (int v = 0; v < 2 && rc == SGS_OK; ++v) rc = add(K_ATTR, v, R_ATTR);
    if (rc == SGS_OK) rc = add(K_LEARNED, 0, R_ATTR);
    if (rc == SGS_OK) rc = add(K_COPY, 0, R_GEO);
    if (rc == SGS_OK) rc = add(K_GEO, 0, R_GEO);
    if (rc == SGS_OK) rc = add(K_DUP, 0, R_GEO);
    if (rc == SGS_OK) rc = add(K_SCAN, 1, R_GEO);  // tile sums
    if (rc == SGS_OK) rc = add(K_SCAN, 0, R_GEO);  // prefixes
    if (rc == SGS_OK) rc = add(K_SCAN, 2, R_GEO);  // parent entries
    if (rc == SGS_OK) rc = add(K_WALK, 0, R_GEO);
    // the position-aware model reads the voxels the walk wrote: after it, on its stream
    if (rc == SGS_OK) rc = add(K_LEARNED_PE, 0, R_GEO);
    if (rc != SGS_OK) return rc;
    L->lists.resize(a16(L->lists.size()));
    L->need_off = L->lists.size();
    L->lists.insert(L->lists.end(), reinterpret_cast<uint8_t *>(L->need.data()),
                    reinterpret_cast<uint8_t *>(L->need.data() + L->need.size()));
    L->total = a256(L->lists_off + L->lists.size());
    return SGS_OK;
}

}  // namespace sgs

using namespace sgs;

struct sgs_batch {
    int device;
    int n;
    uint8_t *base;
    bool owns;
    BatchLayout L;
};

namespace {

// Binds the launch records to the device addresses of the lists.
MultiArgs multi_args(const sgs_batch &b, const LaunchRec &r, int idx) {
    MultiArgs m;
    uint8_t *lists = b.base + b.L.lists_off;
    m.params = lists + r.param_off;
    m.stride = r.stride;
    m.prefix = reinterpret_cast<const uint32_t *>(lists + r.prefix_off);
    m.n = r.n;
    m.total = r.total;
    m.counter = reinterpret_cast<uint32_t *>(b.base + b.L.zero_off) + idx;
    m.scene_id = reinterpret_cast<const uint32_t *>(lists + r.scene_off);
    m.done = reinterpret_cast<uint32_t *>(b.base + b.L.done_off);
    m.need = reinterpret_cast<const uint32_t *>(lists + b.L.need_off);
    m.t_done = reinterpret_cast<unsigned long long *>(b.base + b.L.times_off);
    return m;
}

// Sets each launch's shared-memory limit and caches its resident grid, so a run makes no
// attribute or occupancy query (it may be inside a stream capture).
int warm(const sgs_batch &b) {
    for (size_t i = 0; i < b.L.launches.size(); ++i) {
        MultiArgs m = multi_args(b, b.L.launches[i], (int)i);
        m.total = 0;
        if (launch_kind(b.L.launches[i].kind, b.L.launches[i].variant, m, 0) != cudaSuccess) return SGS_E_CUDA;
    }
    return SGS_OK;
}

int batch_init(sgs_ctx *c, const sgs_batch_item *items, int n, uint8_t *base, sgs_batch *b) {
    b->device = c->device;
    b->n = n;
    b->base = base;
    int rc = build_layout(items, n, base, &b->L);
    if (rc != SGS_OK) return rc;
    return warm(*b);
}

int batch_run(sgs_ctx *c, sgs_batch *b, cudaStream_t st) {
    const BatchLayout &L = b->L;
    {
        const uint32_t n16 = (uint32_t)(L.zero_bytes / 16);
        k_run_begin<<<(n16 + 255) / 256 < 64 ? (n16 + 255) / 256 : 64, 256, 0, st>>>(
            reinterpret_cast<uint4 *>(b->base + L.zero_off), n16,
            reinterpret_cast<unsigned long long *>(b->base + L.start_off));
        if (cudaGetLastError() != cudaSuccess) return SGS_E_CUDA;
        c->launches += 1;
    }
    cudaStream_t role_stream[3] = {st, c->aux, c->geo};
    // The tables feed both halves: they run first on the caller's stream, then the attribute
    // and geometry streams fork.  The learned-model launch goes last on the attribute
    // stream, after the whole geometry chain: its persistent CTAs fill every SM (one per SM)
    // for most of the run, so a geometry stage queued behind them would wait for the whole
    // learned decode, and with it every scene's completion.  Fixed-length and static
    // scenes thus complete while the learned decode has not started.
    bool forked = false;
    int learned = -1;
    auto launch = [&](size_t i) -> int {
        const LaunchRec &r = L.launches[i];
        if (r.kind != K_TABLES && !forked) {
            if (cudaEventRecord(c->fork, st) != cudaSuccess || cudaStreamWaitEvent(c->aux, c->fork, 0) != cudaSuccess ||
                cudaStreamWaitEvent(c->geo, c->fork, 0) != cudaSuccess)
                return SGS_E_CUDA;
            forked = true;
        }
        if (launch_kind(r.kind, r.variant, multi_args(*b, r, (int)i), role_stream[r.role]) != cudaSuccess)
            return SGS_E_CUDA;
        c->launches += 1;
        return SGS_OK;
    };
    for (size_t i = 0; i < L.launches.size(); ++i) {
        if (L.launches[i].kind == K_LEARNED) {
            learned = (int)i;
            continue;
        }
        if (launch(i) != SGS_OK) return SGS_E_CUDA;
    }
    if (learned >= 0) {
        if (forked && (cudaEventRecord(c->gjoin, c->geo) != cudaSuccess ||
                       cudaStreamWaitEvent(c->aux, c->gjoin, 0) != cudaSuccess))
            return SGS_E_CUDA;
        if (launch((size_t)learned) != SGS_OK) return SGS_E_CUDA;
    }
    if (forked && (cudaEventRecord(c->join, c->aux) != cudaSuccess || cudaEventRecord(c->gjoin, c->geo) != cudaSuccess ||
                   cudaStreamWaitEvent(st, c->join, 0) != cudaSuccess ||
                   cudaStreamWaitEvent(st, c->gjoin, 0) != cudaSuccess))
        return SGS_E_CUDA;
    if (b->n) {
        k_status_fold<<<1, 256, 0, st>>>(reinterpret_cast<const int *>(b->base + L.status_off), b->n, c->status_dev);
        if (cudaGetLastError() != cudaSuccess) return SGS_E_CUDA;
        c->launches += 1;
    }
    return SGS_OK;
}

}  // namespace

extern "C" int scene_batch_bytes(const sgs_batch_item *items, int n, size_t *bytes) {
    if ((!items && n) || n < 0 || !bytes) return SGS_E_INVALID;
    BatchLayout L;
    // sizes do not depend on the base address: lay out at a stand-in address, never used
    int rc = build_layout(items, n, reinterpret_cast<uint8_t *>(uintptr_t(1) << 20), &L);
    if (rc != SGS_OK) return rc;
    *bytes = L.total;
    return SGS_OK;
}

extern "C" int scene_batch_plan(sgs_ctx *c, const sgs_batch_item *items, int n, sgs_batch **out) {
    if (!c || (!items && n) || n < 0 || !out) return SGS_E_INVALID;
    *out = nullptr;
    if (cudaSetDevice(c->device) != cudaSuccess) return SGS_E_CUDA;
    size_t bytes = 0;
    int rc = scene_batch_bytes(items, n, &bytes);
    if (rc != SGS_OK) return rc;
    sgs_batch *b = new (std::nothrow) sgs_batch();
    if (!b) return SGS_E_NOMEM;
    void *mem = nullptr;
    if (cudaMalloc(&mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return SGS_E_NOMEM;
    }
    b->owns = true;
    rc = batch_init(c, items, n, static_cast<uint8_t *>(mem), b);
    if (rc == SGS_OK && !b->L.lists.empty() &&
        cudaMemcpy(b->base + b->L.lists_off, b->L.lists.data(), b->L.lists.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess)
        rc = SGS_E_CUDA;
    if (rc != SGS_OK) {
        cudaFree(mem);
        delete b;
        return rc;
    }
    *out = b;
    return SGS_OK;
}

extern "C" int scene_batch_run(sgs_ctx *c, sgs_batch *b, sgs_stream stream) {
    if (!c || !b || b->device != c->device) return SGS_E_INVALID;
    if (cudaSetDevice(c->device) != cudaSuccess) return SGS_E_CUDA;
    return batch_run(c, b, (cudaStream_t)stream);
}

extern "C" int scene_batch_status(const sgs_batch *b, int *status, int n) {
    if (!b || (!status && n) || n != b->n) return SGS_E_INVALID;
    if (n == 0) return SGS_OK;
    if (cudaSetDevice(b->device) != cudaSuccess) return SGS_E_CUDA;
    if (cudaMemcpy(status, b->base + b->L.status_off, 4ull * n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SGS_E_CUDA;
    return SGS_OK;
}

extern "C" int scene_batch_times(const sgs_batch *b, double *ms, int n) {
    if (!b || (!ms && n) || n != b->n) return SGS_E_INVALID;
    if (n == 0) return SGS_OK;
    if (cudaSetDevice(b->device) != cudaSuccess) return SGS_E_CUDA;
    std::vector<unsigned long long> t(n);
    unsigned long long t0 = 0;
    if (cudaMemcpy(t.data(), b->base + b->L.times_off, 8ull * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&t0, b->base + b->L.start_off, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SGS_E_CUDA;
    for (int i = 0; i < n; ++i)
        ms[i] = (b->L.need[i] && t[i] >= t0) ? (double)(t[i] - t0) * 1e-6 : -1.0;
    return SGS_OK;
}

extern "C" void scene_batch_free(sgs_batch *b) {
    if (!b) return;
    if (b->owns && b->base) {
        cudaSetDevice(b->device);
        cudaFree(b->base);
    }
    delete b;
}

extern "C" int scene_decode_batch(sgs_ctx *c, const sgs_batch_item *items, int n, sgs_stream stream) {
    if (!c || (!items && n) || n < 0) return SGS_E_INVALID;
    if (cudaSetDevice(c->device) != cudaSuccess) return SGS_E_CUDA;
    size_t bytes = 0;
    int rc = scene_batch_bytes(items, n, &bytes);
    if (rc != SGS_OK) return rc;
    if (bytes > c->scratch_bytes) return SGS_E_NOMEM;
    sgs_batch b;
    b.owns = false;
    rc = batch_init(c, items, n, c->scratch, &b);
    if (rc != SGS_OK) return rc;
    const cudaStream_t st = (cudaStream_t)stream;
    // the lists go in stream order: a previous call's kernels on this stream are done with
    // the context scratch before they are overwritten
    if (!b.L.lists.empty() && cudaMemcpyAsync(b.base + b.L.lists_off, b.L.lists.data(), b.L.lists.size(),
                                              cudaMemcpyHostToDevice, st) != cudaSuccess)
        return SGS_E_CUDA;
    return batch_run(c, &b, st);
}
