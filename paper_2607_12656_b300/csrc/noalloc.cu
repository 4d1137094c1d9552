// scene_decode_noalloc: the scene decode for callers that cannot allocate device memory.
//
// Some callers of this library own all device memory themselves and forbid allocation once
// they are running -- a renderer or engine that reserves its memory at start-up, or a
// latency-critical loop where cudaMalloc / cudaFree could synchronize the device.  They
// cannot create an sgs_ctx (whose scratch is a cudaMalloc).  This entry point decodes with a
// fixed scratch area compiled into the library instead: a file-scope device array of
// SGS_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the process exits.
// The caller still supplies the bitstream and the output buffers.
//
// It runs every stage on the caller's stream (no internal streams or events), then waits
// for the stream and returns the decode's device-side status.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "sgs_internal.h"

namespace sgs {
int octree_launches(const sgs_scene_info &info, const GeoPlan &plan);
}

using namespace sgs;

namespace {

constexpr size_t kStatusBytes = 256;  // status word at the start of the array

// The scratch.  In host code this name is only a host-side stand-in for the symbol, not a
// device address: kernels are given the address cudaGetSymbolAddress returns for it.
static __device__ __align__(256) uint8_t g_noalloc_scratch[SGS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint8_t *g_ptr[kMaxDevices];  // device address of the array, per device (set up once)

// Looks up the array's device address on the current device (first call per device).
int device_scratch(uint8_t **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SGS_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SGS_E_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SGS_E_CUDA;
        g_ptr[dev] = static_cast<uint8_t *>(p);
    }
    *out = g_ptr[dev];
    return SGS_OK;
}

}  // namespace

extern "C" int scene_decode_noalloc(const uint8_t *bits, const sgs_scene_info *info,
                                    const sgs_scene_out *out, sgs_stream stream) {
    if (!bits || !info || !out) return SGS_E_INVALID;
    if (((uintptr_t)bits & 15) != 0) return SGS_E_INVALID;
    if (info->n_rows && (!out->attr || !out->pos)) return SGS_E_INVALID;
    // the scene must fit the fixed array (both the caller's figure and our own)
    const size_t need = scratch_need(*info, nullptr, nullptr);
    if (need > SGS_NOALLOC_SCRATCH_BYTES - kStatusBytes ||
        info->scratch_bytes > SGS_NOALLOC_SCRATCH_BYTES - kStatusBytes)
        return SGS_E_NOMEM;
    uint8_t *area = nullptr;
    int rc = device_scratch(&area);
    if (rc != SGS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int *status = reinterpret_cast<int *>(area);
    uint8_t *base = area + kStatusBytes;
    Scratch s;
    scratch_need(*info, &s, base);
    GeoPlan plan;
    make_geo_plan(*info, &plan);
    // the array keeps the previous call's contents: clear the status word (nothing else
    // needs to start at zero)
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return SGS_E_CUDA;
    // once a stage is enqueued, an error return first waits for what is already on the
    // stream, so that no work of this call still uses the shared array afterwards
    auto fail = [&]() {
        cudaStreamSynchronize(st);
        return SGS_E_CUDA;
    };
    if (launch_tables(bits, *info, plan.n_geo_tables, s.tables, status, st) != cudaSuccess) return fail();
    uint8_t *attr_tables = s.tables + (size_t)plan.n_geo_tables * kTabBytes;
    const sgs_scene_out o = effective_out(*info, *out, s);
    cudaError_t e = cudaSuccess;
    switch (info->mode) {
        case SGS_MODE_FIXED: e = launch_fixed(bits, *info, o, status, st); break;
        case SGS_MODE_STATIC: e = launch_rans_static_attr(bits, *info, attr_tables, o, status, st); break;
        case SGS_MODE_LEARNED: e = launch_learned_decode(bits, *info, o, s.learned, status, st); break;
        default: break;  // the position-aware model follows the octree
    }
    if (e != cudaSuccess) return fail();
    if (info->geo_mode == SGS_GEO_RANS && info->n_geo) {
        if (launch_geo_copy_raw(bits, *info, plan, s.geo_bytes, st) != cudaSuccess) return fail();
        if (launch_rans_static_geo(bits, *info, plan, s.tables, s.geo_bytes, status, st) != cudaSuccess)
            return fail();
    } else if (info->geo_mode == SGS_GEO_LEARNED && info->n_geo) {
        if (launch_geo_copy_raw(bits, *info, plan, s.geo_bytes, st) != cudaSuccess) return fail();
        if (launch_geo_learned(bits, *info, plan, s.geo_bytes, s.geo_work, status, st, nullptr) != cudaSuccess)
            return fail();
    }
    if (launch_octree(*info, plan, bits, s, o, status, st) != cudaSuccess) return fail();
    if (info->mode == SGS_MODE_LEARNED_PE &&
        launch_learned_pe_decode(bits, *info, o, o.coord, status, st) != cudaSuccess)
        return fail();
    int host_status = SGS_OK;
    if (cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return fail();
    if (cudaStreamSynchronize(st) != cudaSuccess) return SGS_E_CUDA;
    return host_status;
}
