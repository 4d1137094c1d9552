// C ABI of the sgs library: context, header query, decode orchestration, status.
// Kernels live in k_*.cu; the encoder in encode.cu; the learned part in k_learned.cu and
// k_train.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "sgs_ctx.h"
#include "sgs_internal.h"

namespace sgs {

size_t octree_scan_tiles(uint64_t n_geo);
int octree_launches(const sgs_scene_info &info, const GeoPlan &plan);
size_t octree_words(uint64_t n_geo);

static inline uint64_t a256(uint64_t x) { return (x + 255) & ~255ull; }

static uint32_t rd32(const uint8_t *p) {
    uint32_t v;
    memcpy(&v, p, 4);
    return v;
}
static uint64_t rd64(const uint8_t *p) {
    uint64_t v;
    memcpy(&v, p, 8);
    return v;
}

void make_geo_plan(const sgs_scene_info &info, GeoPlan *plan) {
    memset(plan, 0, sizeof(*plan));
    plan->depth = (int)info.depth;
    uint64_t off = 0, coded = 0;
    int k = 0;
    for (uint32_t l = 0; l <= info.depth; ++l) {
        plan->n_level[l] = info.n_level[l];
        plan->level_off[l] = off;
        off += info.n_level[l];
        if (l < info.depth && info.geo_mode != SGS_GEO_RAW && info.n_level[l] >= kGeoRansMinLevel) {
            plan->coded_level[k] = (int)l;
            plan->coded_start[k] = coded;
            coded += info.n_level[l];
            ++k;
        }
    }
    plan->n_coded_levels = k;
    plan->n_geo_tables = info.geo_mode == SGS_GEO_RANS ? k : 0;
    plan->coded_start[k] = coded;
}

// Carves the scratch regions of one decode out of `base` (or only sizes them if base is
// NULL).  Returns the total size.
size_t scratch_need(const sgs_scene_info &info, Scratch *s, uint8_t *base) {
    GeoPlan plan;
    make_geo_plan(info, &plan);
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) {
        uint8_t *p = base ? base + off : nullptr;
        off = a256(off + bytes);
        return p;
    };
    Scratch t;
    t.geo_bytes = take(info.geo_mode != SGS_GEO_RAW ? info.n_geo : 0);
    t.p4 = reinterpret_cast<uint32_t *>(take(4 * (octree_words(info.n_geo) + 16)));
    t.tile_sums = reinterpret_cast<uint32_t *>(take(4 * (octree_scan_tiles(info.n_geo) + 1)));
    t.par = reinterpret_cast<uint32_t *>(take(info.n_rows ? 4ull * (info.n_geo + info.n_leaves) : 0));
    const int n_tab = plan.n_geo_tables + (info.mode == SGS_MODE_STATIC ? kNChan : 0);
    t.tables = take((uint64_t)n_tab * kTabBytes);
    t.dup_prefix = reinterpret_cast<uint32_t *>(take(4ull * (info.n_dup + 1)));
    t.learned = take(info.mode == SGS_MODE_LEARNED ? learned_work_bytes(info) : 0);
    t.coord = reinterpret_cast<uint32_t *>(take(info.mode == SGS_MODE_LEARNED_PE ? 12ull * info.n_rows : 0));
    t.geo_work = take(info.geo_mode == SGS_GEO_LEARNED && info.n_geo_coded ? geo_learned_scratch(info, nullptr, nullptr) : 0);
    if (s) *s = t;
    return off;
}

sgs_scene_out effective_out(const sgs_scene_info &info, const sgs_scene_out &out, const Scratch &s) {
    sgs_scene_out o = out;
    if (info.mode == SGS_MODE_LEARNED_PE && !o.coord) o.coord = s.coord;
    return o;
}

}  // namespace sgs

using namespace sgs;

extern "C" const char *sgs_strerror(int code) {
    switch (code) {
        case SGS_OK: return "ok";
        case SGS_E_INVALID: return "invalid argument or malformed header";
        case SGS_E_CORRUPT: return "corrupt bitstream";
        case SGS_E_NOMEM: return "out of memory or scratch too small";
        case SGS_E_CUDA: return "CUDA error";
        case SGS_E_TIMEOUT: return "device wait timed out";
        case SGS_E_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

extern "C" int sgs_create(sgs_ctx **out, int device, size_t scratch_bytes) {
    if (!out) return SGS_E_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) return SGS_E_CUDA;
    if (device < 0 || device >= n) return SGS_E_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) return SGS_E_CUDA;
    sgs_ctx *c = new (std::nothrow) sgs_ctx();
    if (!c) return SGS_E_NOMEM;
    c->device = device;
    if (cudaMalloc(&c->status_dev, 256) != cudaSuccess) { delete c; return SGS_E_NOMEM; }
    if (cudaMallocHost(&c->status_host, 256) != cudaSuccess) {
        cudaFree(c->status_dev);
        delete c;
        return SGS_E_NOMEM;
    }
    cudaMemset(c->status_dev, 0, 256);
    c->launches = 0;
    c->profile = 0;
    c->wait_limit = kDefaultWaitPolls;
    for (int m = 0; m < 4; ++m) c->shape[m] = 0;
    c->n_marks = 0;
    for (int i = 0; i <= kMaxStages; ++i) cudaEventCreate(&c->marks[i]);
    for (int i = 0; i < 2; ++i) cudaEventCreate(&c->amarks[i]);
    // the latency-bound geometry chain outranks the bandwidth-bound attribute kernels, so its
    // small launches get SMs as soon as attribute CTAs retire
    int prio_low = 0, prio_high = 0;
    cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    if (cudaStreamCreateWithPriority(&c->aux, cudaStreamNonBlocking, prio_low) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->geo, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->gjoin, cudaEventDisableTiming) != cudaSuccess) {
        cudaFree(c->status_dev);
        cudaFreeHost(c->status_host);
        delete c;
        return SGS_E_CUDA;
    }
    c->scratch = nullptr;
    c->scratch_bytes = 0;
    if (scratch_bytes) {
        if (cudaMalloc(&c->scratch, scratch_bytes) != cudaSuccess) {
            cudaFree(c->status_dev);
            cudaFreeHost(c->status_host);
            delete c;
            return SGS_E_NOMEM;
        }
        c->scratch_bytes = scratch_bytes;
    }
    *out = c;
    return SGS_OK;
}

extern "C" int sgs_reserve(sgs_ctx *c, size_t bytes) {
    if (!c) return SGS_E_INVALID;
    if (bytes <= c->scratch_bytes) return SGS_OK;
    cudaSetDevice(c->device);
    if (cudaDeviceSynchronize() != cudaSuccess) return SGS_E_CUDA;
    if (c->scratch) cudaFree(c->scratch);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
    if (cudaMalloc(&c->scratch, bytes) != cudaSuccess) return SGS_E_NOMEM;
    c->scratch_bytes = bytes;
    return SGS_OK;
}

extern "C" void sgs_destroy(sgs_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->scratch) cudaFree(c->scratch);
    if (c->rws) cudaFree(c->rws);
    for (int i = 0; i <= kMaxStages; ++i) cudaEventDestroy(c->marks[i]);
    for (int i = 0; i < 2; ++i) cudaEventDestroy(c->amarks[i]);
    cudaEventDestroy(c->fork);
    cudaEventDestroy(c->join);
    cudaEventDestroy(c->gjoin);
    cudaStreamDestroy(c->geo);
    cudaStreamDestroy(c->aux);
    cudaFree(c->status_dev);
    cudaFreeHost(c->status_host);
    delete c;
}

extern "C" int sgs_profile(sgs_ctx *c, int enable) {
    if (!c) return SGS_E_INVALID;
    c->profile = enable != 0;
    return SGS_OK;
}

// Stage times (ms) of the most recent profiled decode: [0] geometry tokens (tables, raw
// copy, rANS), [1] octree expansion and positions, [2] attribute decode (on the attribute
// stream, concurrent with [0] and [1]), [3] the whole decode.
extern "C" int sgs_profile_read(sgs_ctx *c, float *ms, int cap) {
    if (!c || !ms || cap < 4) return SGS_E_INVALID;
    if (c->n_marks != 4) return SGS_E_INVALID;
    for (int i = 0; i < 2; ++i)
        if (cudaEventElapsedTime(&ms[i], c->marks[i], c->marks[i + 1]) != cudaSuccess) return SGS_E_CUDA;
    if (cudaEventElapsedTime(&ms[2], c->amarks[0], c->amarks[1]) != cudaSuccess) return SGS_E_CUDA;
    if (cudaEventElapsedTime(&ms[3], c->marks[0], c->marks[3]) != cudaSuccess) return SGS_E_CUDA;
    return SGS_OK;
}

extern "C" uint64_t sgs_launch_count(sgs_ctx *c) { return c ? c->launches : 0; }

extern "C" int sgs_set_wait_limit(sgs_ctx *c, uint32_t polls) {
    if (!c) return SGS_E_INVALID;
    c->wait_limit = polls ? polls : kDefaultWaitPolls;
    return SGS_OK;
}

extern "C" int sgs_set_launch_shape(sgs_ctx *c, uint32_t mode, uint32_t warps) {
    if (!c) return SGS_E_INVALID;
    const uint32_t cap = mode == SGS_MODE_FIXED ? kFixWarpsMax : mode == SGS_MODE_STATIC ? kAttrWarpsMax : 0u;
    if (cap == 0 || warps > cap) return SGS_E_INVALID;
    c->shape[mode] = warps;
    return SGS_OK;
}

extern "C" int sgs_sync(sgs_ctx *c, sgs_stream stream) {
    if (!c) return SGS_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(c->status_host, c->status_dev, sizeof(int), cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return SGS_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SGS_E_CUDA;
    const int s = c->status_host[0];
    if (cudaMemsetAsync(c->status_dev, 0, sizeof(int), st) != cudaSuccess) return SGS_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SGS_E_CUDA;
    return s;
}

extern "C" int scene_query(const uint8_t *b, size_t len, sgs_scene_info *info) {
    if (!b || !info || len < (size_t)kHeaderBytes) return SGS_E_INVALID;
    memset(info, 0, sizeof(*info));
    if (rd32(b) != kMagic || rd32(b + 4) != kVersion) return SGS_E_INVALID;
    info->mode = rd32(b + 8);
    info->geo_mode = rd32(b + 12);
    info->n_in = rd32(b + 16);
    info->n_rows = rd32(b + 20);
    info->depth = rd32(b + 24);
    info->n_leaves = rd32(b + 28);
    info->n_dup = rd32(b + 32);
    const uint32_t n_chan = rd32(b + 36);
    info->lanes = rd32(b + 40);
    info->geo_lanes = rd32(b + 44);
    info->n_geo = rd64(b + 48);
    info->n_geo_coded = rd64(b + 56);
    for (int i = 0; i < 11; ++i) info->off[i] = rd64(b + 64 + 8 * i);
    info->total_len = info->off[S_TOTAL];
    if (n_chan != (uint32_t)kNChan || info->mode > SGS_MODE_LEARNED_PE || info->geo_mode > SGS_GEO_LEARNED)
        return SGS_E_INVALID;
    if (info->depth < 1 || info->depth > SGS_MAX_DEPTH) return SGS_E_INVALID;
    if (info->total_len != len) return SGS_E_INVALID;
    if (info->off[0] != (uint64_t)kHeaderBytes) return SGS_E_INVALID;
    for (int i = 0; i < 11; ++i) {
        if (info->off[i] % 16 != 0 || info->off[i] > info->total_len) return SGS_E_INVALID;
        if (i > 0 && info->off[i] < info->off[i - 1]) return SGS_E_INVALID;
    }
    auto sec = [&](int i) { return info->off[i + 1] - info->off[i]; };
    const uint32_t D = info->depth;
    if (sec(S_LEVELS) < 4ull * D || sec(S_DUP) < 8ull * info->n_dup || sec(S_CHAN) < 12ull * kNChan)
        return SGS_E_INVALID;
    uint64_t sum = 0, coded = 0;
    for (uint32_t l = 0; l < D; ++l) {
        info->n_level[l] = rd32(b + info->off[S_LEVELS] + 4 * l);
        sum += info->n_level[l];
        if (info->geo_mode != SGS_GEO_RAW && info->n_level[l] >= kGeoRansMinLevel)
            coded += info->n_level[l];
        if (l > 0 && info->n_level[l] < info->n_level[l - 1]) return SGS_E_INVALID;  // every node has >= 1 child
        if (l > 0 && (uint64_t)info->n_level[l] > 8ull * info->n_level[l - 1]) return SGS_E_INVALID;
    }
    info->n_level[D] = info->n_leaves;
    if (sum != info->n_geo || coded != info->n_geo_coded) return SGS_E_INVALID;
    if (info->n_rows == 0) {
        if (info->n_leaves != 0 || info->n_geo != 0 || info->n_dup != 0) return SGS_E_INVALID;
    } else {
        if (info->n_level[0] != 1 || info->n_leaves == 0 || info->n_leaves > info->n_rows ||
            info->n_leaves < info->n_level[D - 1] || (uint64_t)info->n_leaves > 8ull * info->n_level[D - 1])
            return SGS_E_INVALID;
        if (info->n_geo + info->n_leaves >= (1ull << 32)) return SGS_E_INVALID;
        if (info->n_geo > (1ull << 29)) return SGS_E_UNSUPPORTED;  // parent index in 29 bits
        if (info->n_dup > info->n_leaves) return SGS_E_INVALID;
    }
    // geometry sections
    uint64_t raw = info->n_geo - info->n_geo_coded;
    if (sec(S_GEO_RAW) < raw) return SGS_E_INVALID;
    if (info->n_geo_coded && info->geo_mode == SGS_GEO_LEARNED) {
        // one model, then per coded level a group table (its lanes fixed by its size)
        uint64_t lanes = 0, grp = 0;
        for (uint32_t l = 0; l < D; ++l)
            if (info->n_level[l] >= kGeoRansMinLevel) {
                lanes += geo_learned_lanes(info->n_level[l]);
                grp += geo_learned_group_bytes(info->n_level[l]);
            }
        if (info->geo_lanes != lanes || sec(S_GEO_TAB) < (uint64_t)SGS_MODEL_BYTES || sec(S_GEO_GRP) < grp)
            return SGS_E_INVALID;
    } else if (info->n_geo_coded) {
        if (info->geo_lanes == 0) return SGS_E_INVALID;
        const uint64_t G = (info->geo_lanes + 31) / 32;
        if (sec(S_GEO_GRP) < 8 * (G + 1) + 4 * G) return SGS_E_INVALID;
    } else if (info->geo_lanes != 0) {
        return SGS_E_INVALID;
    }
    // attribute sections
    if (info->mode == SGS_MODE_FIXED) {
        if (info->lanes != 0 || sec(S_ATTR_TAB) < 8ull * (kNChan + 1)) return SGS_E_INVALID;
    } else {
        if (info->lanes == 0) return SGS_E_INVALID;
        const uint64_t G = (info->lanes + 31) / 32;
        if (sec(S_ATTR_GRP) < 8 * (G + 1) + 4 * G) return SGS_E_INVALID;
        if (info->mode == SGS_MODE_LEARNED && sec(S_ATTR_TAB) < (uint64_t)SGS_MODEL_BYTES)
            return SGS_E_INVALID;
        if (info->mode == SGS_MODE_LEARNED_PE && sec(S_ATTR_TAB) < (uint64_t)SGS_MODEL_PE_BYTES)
            return SGS_E_INVALID;
    }
    // static tables: walk the variable-size tables once (presence mask, then (f-1) per
    // present symbol, padded to 16 bytes) and record where each one starts
    auto walk = [&](uint64_t off, uint64_t end, int count) -> bool {
        for (int t = 0; t < count; ++t) {
            if (off + 32 > end || info->n_tables >= (uint32_t)(SGS_NCHAN + SGS_MAX_DEPTH)) return false;
            uint32_t K = 0;
            for (int i = 0; i < 32; ++i) K += (uint32_t)__builtin_popcount(b[off + i]);
            const uint64_t size = 32 + ((2ull * K + 15) & ~15ull);
            if (off + size > end || off >= (1ull << 32)) return false;
            info->table_off[info->n_tables++] = (uint32_t)off;
            off += size;
        }
        return true;
    };
    int n_geo_tab = 0;
    for (uint32_t l = 0; l < D; ++l)
        if (info->geo_mode == SGS_GEO_RANS && info->n_level[l] >= kGeoRansMinLevel) ++n_geo_tab;
    if (!walk(info->off[S_GEO_TAB], info->off[S_GEO_GRP], n_geo_tab)) return SGS_E_INVALID;
    if (info->mode == SGS_MODE_STATIC && !walk(info->off[S_ATTR_TAB], info->off[S_ATTR_GRP], kNChan))
        return SGS_E_INVALID;
    info->scratch_bytes = scratch_need(*info, nullptr, nullptr);
    return SGS_OK;
}

// Enqueues every stage of one scene's decode using scratch `base`.  The attribute decode is
// forked onto the context's attribute stream (it does not depend on the geometry) and joined
// back into `st` at the end, so the two halves overlap on the device.  The position-aware
// model reads the decoded voxels (attributes are coded upon the decoded geometry, Sec. 3.4),
// so its decode follows the octree on the geometry stream.
static int decode_one(sgs_ctx *c, const uint8_t *bits, const sgs_scene_info &info,
                      const sgs_scene_out &user_out, uint8_t *base, cudaStream_t st) {
    Scratch s;
    scratch_need(info, &s, base);
    const sgs_scene_out out = effective_out(info, user_out, s);
    const bool after_geo = info.mode == SGS_MODE_LEARNED_PE;
    GeoPlan plan;
    make_geo_plan(info, &plan);
    int *status = c->status_dev;
    cudaError_t e;
    c->n_marks = 0;
    auto mark = [&]() {
        if (c->profile && c->n_marks <= kMaxStages) cudaEventRecord(c->marks[c->n_marks++], st);
    };
    mark();
    if (info.n_tables) {
        c->launches += 1;
        e = launch_tables(bits, info, plan.n_geo_tables, s.tables, status, st);
        if (e != cudaSuccess) return SGS_E_CUDA;
    }
    uint8_t *attr_tables = s.tables + (size_t)plan.n_geo_tables * kTabBytes;
    // fork: attributes on the attribute stream, geometry on the geometry stream
    if (cudaEventRecord(c->fork, st) != cudaSuccess || cudaStreamWaitEvent(c->aux, c->fork, 0) != cudaSuccess ||
        cudaStreamWaitEvent(c->geo, c->fork, 0) != cudaSuccess)
        return SGS_E_CUDA;
    // the geometry tokens are enqueued first: their short CTAs take SMs before the attribute
    // decoder's long-running ones fill the device
    cudaStream_t gs = c->geo;
    if (info.geo_mode == SGS_GEO_RANS && info.n_geo) {
        if ((e = launch_geo_copy_raw(bits, info, plan, s.geo_bytes, gs)) != cudaSuccess) return SGS_E_CUDA;
        if ((e = launch_rans_static_geo(bits, info, plan, s.tables, s.geo_bytes, status, gs)) != cudaSuccess)
            return SGS_E_CUDA;
        c->launches += 2;
    } else if (info.geo_mode == SGS_GEO_LEARNED && info.n_geo) {
        if ((e = launch_geo_copy_raw(bits, info, plan, s.geo_bytes, gs)) != cudaSuccess) return SGS_E_CUDA;
        int n = 1;
        if ((e = launch_geo_learned(bits, info, plan, s.geo_bytes, s.geo_work, status, gs, &n)) != cudaSuccess)
            return SGS_E_CUDA;
        c->launches += n;
    }
    if (!after_geo) {
        if (c->profile) cudaEventRecord(c->amarks[0], c->aux);
        if (info.n_rows) c->launches += 1;
        switch (info.mode) {
            case SGS_MODE_FIXED: e = launch_fixed(bits, info, out, status, c->aux, c->shape[SGS_MODE_FIXED]); break;
            case SGS_MODE_STATIC:
                e = launch_rans_static_attr(bits, info, attr_tables, out, status, c->aux, c->shape[SGS_MODE_STATIC]);
                break;
            default: e = launch_learned_decode(bits, info, out, s.learned, status, c->aux, c->wait_limit); break;
        }
        if (e != cudaSuccess) return SGS_E_CUDA;
        if (c->profile) cudaEventRecord(c->amarks[1], c->aux);
    }
    if (cudaEventRecord(c->join, c->aux) != cudaSuccess) return SGS_E_CUDA;
    if (c->profile && c->n_marks <= kMaxStages) cudaEventRecord(c->marks[c->n_marks++], gs);
    if ((e = launch_octree(info, plan, bits, s, out, status, gs)) != cudaSuccess) return SGS_E_CUDA;
    if (info.n_rows) c->launches += octree_launches(info, plan);
    if (c->profile && c->n_marks <= kMaxStages) cudaEventRecord(c->marks[c->n_marks++], gs);
    if (after_geo) {
        if (c->profile) cudaEventRecord(c->amarks[0], gs);
        if ((e = launch_learned_pe_decode(bits, info, out, out.coord, status, gs)) != cudaSuccess) return SGS_E_CUDA;
        if (info.n_rows) c->launches += 1;
        if (c->profile) cudaEventRecord(c->amarks[1], gs);
    }
    // join
    if (cudaEventRecord(c->gjoin, gs) != cudaSuccess || cudaStreamWaitEvent(st, c->join, 0) != cudaSuccess ||
        cudaStreamWaitEvent(st, c->gjoin, 0) != cudaSuccess)
        return SGS_E_CUDA;
    mark();
    return SGS_OK;
}

extern "C" int scene_decode(sgs_ctx *c, const uint8_t *bits, const sgs_scene_info *info,
                            const sgs_scene_out *out, sgs_stream stream) {
    if (!c || !bits || !info || !out) return SGS_E_INVALID;
    if (((uintptr_t)bits & 15) != 0) return SGS_E_INVALID;
    if (info->n_rows && (!out->attr || !out->pos)) return SGS_E_INVALID;
    if (info->scratch_bytes > c->scratch_bytes) return SGS_E_NOMEM;
    if (cudaSetDevice(c->device) != cudaSuccess) return SGS_E_CUDA;
    return decode_one(c, bits, *info, *out, c->scratch, (cudaStream_t)stream);
}
