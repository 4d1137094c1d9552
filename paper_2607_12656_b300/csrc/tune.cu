// sgs_autotune: picks the lane count (group size W = rows per lane) of a scene by encoding it
// at each candidate W and timing the decode on the device.  W is the paper's complexity knob
// (Sec. 4, implementation details): larger groups code better, smaller ones decode with more
// parallelism.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sgs_ctx.h"
#include "sgs_internal.h"

namespace {

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    bool alloc(size_t n) { return cudaMalloc(&p, n ? n : 16) == cudaSuccess; }
};

}  // namespace

extern "C" int sgs_autotune(sgs_ctx *c, const sgs_tune_request *rq, sgs_tune_result *res) {
    if (!c || !rq || !res || !rq->pos || !rq->attr || rq->n == 0) return SGS_E_INVALID;
    if (rq->mode > SGS_MODE_LEARNED_PE) return SGS_E_INVALID;
    if (rq->mode == SGS_MODE_FIXED && rq->n_cand != 1) return SGS_E_INVALID;
    if (rq->n_shape > SGS_TUNE_MAX_CAND) return SGS_E_INVALID;
    const uint32_t cap = rq->mode == SGS_MODE_FIXED ? sgs::kFixWarpsMax : rq->mode == SGS_MODE_STATIC ? sgs::kAttrWarpsMax : 0u;
    for (uint32_t k = 0; k < rq->n_shape; ++k)
        if (rq->warps_per_cta[k] > cap) return SGS_E_INVALID;
    if ((rq->mode == SGS_MODE_LEARNED || rq->mode == SGS_MODE_LEARNED_PE) && !rq->model) return SGS_E_INVALID;
    if (rq->n_cand < 1 || rq->n_cand > SGS_TUNE_MAX_CAND || rq->reps < 1) return SGS_E_INVALID;
    for (uint32_t k = 0; k < rq->n_cand; ++k)
        if (rq->rows_per_lane[k] < 1 && rq->mode != SGS_MODE_FIXED) return SGS_E_INVALID;
    memset(res, 0, sizeof(*res));
    if (cudaSetDevice(c->device) != cudaSuccess) return SGS_E_CUDA;
    const uint32_t kept = rq->n - rq->n / 10;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SGS_E_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = SGS_OK;
    std::vector<uint8_t> buf;
    uint32_t saved_shape[4];
    for (int m = 0; m < 4; ++m) saved_shape[m] = c->shape[m];
    for (uint32_t k = 0; k < rq->n_cand && rc == SGS_OK; ++k) {
        sgs_encode_params prm;
        memset(&prm, 0, sizeof(prm));
        prm.mode = rq->mode;
        prm.geo_mode = rq->geo_mode;
        prm.depth = rq->depth;
        prm.lanes = rq->mode == SGS_MODE_FIXED
                        ? 0u
                        : std::max<uint32_t>(1, (kept + rq->rows_per_lane[k] - 1) / rq->rows_per_lane[k]);
        for (int i = 0; i < SGS_NCHAN; ++i) prm.bits[i] = 8;
        prm.model = rq->model;
        size_t len = 0;
        rc = scene_encode(c, rq->pos, rq->attr, rq->n, &prm, nullptr, 0, &len);
        if (rc != SGS_E_INVALID || len == 0) {
            if (rc == SGS_OK) rc = SGS_E_INVALID;
            break;
        }
        buf.resize(len);
        if ((rc = scene_encode(c, rq->pos, rq->attr, rq->n, &prm, buf.data(), buf.size(), &len)) != SGS_OK) break;
        sgs_scene_info info;
        if ((rc = scene_query(buf.data(), len, &info)) != SGS_OK) break;
        if ((rc = sgs_reserve(c, info.scratch_bytes)) != SGS_OK) break;
        DevBuf bits, attr, pos;
        if (!bits.alloc(len) || !attr.alloc(4ull * SGS_NCHAN * info.n_rows) || !pos.alloc(12ull * info.n_rows)) {
            rc = SGS_E_NOMEM;
            break;
        }
        if (cudaMemcpy(bits.p, buf.data(), len, cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = SGS_E_CUDA;
            break;
        }
        sgs_scene_out out;
        memset(&out, 0, sizeof(out));
        out.attr = static_cast<float *>(attr.p);
        out.pos = static_cast<float *>(pos.p);
        // every launch shape (or only the context's own), the fastest kept
        const uint32_t n_shape = rq->n_shape ? rq->n_shape : 1u;
        for (uint32_t h = 0; h < n_shape && rc == SGS_OK; ++h) {
            if (rq->n_shape) c->shape[rq->mode] = rq->warps_per_cta[h];
            std::vector<float> t;
            for (uint32_t r = 0; r <= rq->reps && rc == SGS_OK; ++r) {  // first run untimed
                cudaEventRecord(e0, st);
                rc = scene_decode(c, static_cast<const uint8_t *>(bits.p), &info, &out, (sgs_stream)st);
                cudaEventRecord(e1, st);
                if (rc == SGS_OK) rc = sgs_sync(c, (sgs_stream)st);
                float ms = 0.f;
                if (rc == SGS_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = SGS_E_CUDA;
                if (r) t.push_back(ms);
            }
            if (rc != SGS_OK) break;
            std::sort(t.begin(), t.end());
            const float med = t[t.size() / 2];
            if (h == 0 || med < res->ms[k]) {
                res->ms[k] = med;
                res->warps[k] = rq->n_shape ? rq->warps_per_cta[h] : c->shape[rq->mode];
            }
        }
        if (rc != SGS_OK) break;
        res->lanes[k] = prm.lanes;
        res->bytes[k] = len;
    }
    for (int m = 0; m < 4; ++m) c->shape[m] = saved_shape[m];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (rc != SGS_OK) return rc;
    // smallest bitstream within the target, else the fastest
    int best = -1;
    for (uint32_t k = 0; k < rq->n_cand; ++k)
        if (rq->max_ms > 0.f && res->ms[k] <= rq->max_ms && (best < 0 || res->bytes[k] < res->bytes[best]))
            best = (int)k;
    if (best < 0) {
        best = 0;
        for (uint32_t k = 1; k < rq->n_cand; ++k)
            if (res->ms[k] < res->ms[best]) best = (int)k;
    }
    res->best = (uint32_t)best;
    res->best_warps = res->warps[best];
    return SGS_OK;
}
