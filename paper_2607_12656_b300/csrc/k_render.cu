// Tile splatting of a decoded scene into an image (the consumer of the decoded SoA; 3DGS
// forward rasterisation, Kerbl et al. 2023): what the paper's decoded scenes are rendered with.
//
// 1. k_rs_pre: one thread per Gaussian: camera-space mean, projected 2D covariance (+0.3 I)
//    and its conic, radius ceil(3 sqrt(lambda_max)), the rectangle of 16 x 16 tiles it
//    touches, colour from the degree-3 spherical harmonics along the view ray, opacity.
// 2. exclusive scan of the tile counts; k_rs_emit writes one (tile << 32 | depth bits, index)
//    entry per touched tile, Gaussians in index order.
// 3. stable LSD radix sort of the entries on the depth's 32 bits, then the tile's bits,
//    8 bits per pass: per-block digit counts, a digit-major scan, and a scatter that ranks
//    equal digits in item order (warp match_any, then a prefix over the block's warps).
// 4. k_rs_ranges: each tile's [begin, end) in the sorted entries.
// 5. k_rs_render: one CTA per tile, one thread per pixel: the tile's Gaussians front to back
//    in batches staged in shared memory; alpha = min(0.99, opacity exp(power)), skipped below
//    1/255; compositing stops before the transmittance would fall below 1e-4.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "sgs_ctx.h"
#include "sgs_device.cuh"
#include "sgs_internal.h"

namespace sgs {

namespace {

constexpr int kTile = 16;

struct Cam {
    float r[9], o[3], fx, fy, cx, cy;
    int w, h, tx, ty;
};

__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y) {
    const float pi = 3.14159265358979323846f;
    const float c0 = 0.5f / sqrtf(pi), c1 = sqrtf(3.0f / (4.0f * pi));
    const float c20 = 0.5f * sqrtf(15.0f / pi), c22 = 0.25f * sqrtf(5.0f / pi), c24 = 0.25f * sqrtf(15.0f / pi);
    const float c30 = 0.25f * sqrtf(35.0f / (2.0f * pi)), c31 = 0.5f * sqrtf(105.0f / pi),
                c32 = 0.25f * sqrtf(21.0f / (2.0f * pi)), c33 = 0.25f * sqrtf(7.0f / pi), c35 = 0.25f * sqrtf(105.0f / pi);
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = c0;
    Y[1] = -c1 * y; Y[2] = c1 * z; Y[3] = -c1 * x;
    Y[4] = c20 * x * y; Y[5] = -c20 * y * z; Y[6] = c22 * (2 * zz - xx - yy); Y[7] = -c20 * x * z; Y[8] = c24 * (xx - yy);
    Y[9] = -c30 * y * (3 * xx - yy); Y[10] = c31 * x * y * z; Y[11] = -c32 * y * (4 * zz - xx - yy);
    Y[12] = c33 * z * (2 * zz - 3 * xx - 3 * yy); Y[13] = -c32 * x * (4 * zz - xx - yy); Y[14] = c35 * z * (xx - yy);
    Y[15] = -c30 * x * (xx - 3 * yy);
}

struct Pre {
    float2 *uv;
    float4 *conic_op;   // A, B, C, opacity
    float4 *colour;
    float *depth;
    uint2 *rect;        // x0 | y0 << 16, x1 | y1 << 16
    uint32_t *count;    // tiles touched (0: culled)
};

__global__ void k_rs_pre(const float *attr, const float *pos, uint32_t n, Cam c, Pre P) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float px = pos[i], py = pos[(size_t)n + i], pz = pos[2ull * n + i];
    const float qx = px - c.o[0], qy = py - c.o[1], qz = pz - c.o[2];
    const float tx = c.r[0] * qx + c.r[1] * qy + c.r[2] * qz;
    const float ty = c.r[3] * qx + c.r[4] * qy + c.r[5] * qz;
    const float tz = c.r[6] * qx + c.r[7] * qy + c.r[8] * qz;
    P.count[i] = 0;
    P.depth[i] = 0.0f;
    if (!(tz > 0.2f)) return;
    const float s0 = expf(attr[49ull * n + i]), s1 = expf(attr[50ull * n + i]), s2 = expf(attr[51ull * n + i]);
    float w = attr[52ull * n + i], x = attr[53ull * n + i], y = attr[54ull * n + i], z = attr[55ull * n + i];
    const float qn = sqrtf(w * w + x * x + y * y + z * z);
    w /= qn; x /= qn; y /= qn; z /= qn;
    const float R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    const float M[9] = {R[0] * s0, R[1] * s1, R[2] * s2, R[3] * s0, R[4] * s1, R[5] * s2, R[6] * s0, R[7] * s1, R[8] * s2};
    float S[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S[3 * a + b] = M[3 * a] * M[3 * b] + M[3 * a + 1] * M[3 * b + 1] + M[3 * a + 2] * M[3 * b + 2];
    const float j00 = c.fx / tz, j02 = -c.fx * tx / (tz * tz), j11 = c.fy / tz, j12 = -c.fy * ty / (tz * tz);
    float T[6];  // J Rw, 2 x 3
    for (int b = 0; b < 3; ++b) {
        T[b] = j00 * c.r[b] + j02 * c.r[6 + b];
        T[3 + b] = j11 * c.r[3 + b] + j12 * c.r[6 + b];
    }
    float TS[6];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) TS[3 * a + b] = T[3 * a] * S[b] + T[3 * a + 1] * S[3 + b] + T[3 * a + 2] * S[6 + b];
    const float ca = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + 0.3f;
    const float cb = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
    const float cc = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + 0.3f;
    const float det = ca * cc - cb * cb;
    if (!(det > 0.0f)) return;
    const float mid = 0.5f * (ca + cc);
    const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
    const float r = ceilf(3.0f * sqrtf(lam));
    const float u = c.fx * tx / tz + c.cx, v = c.fy * ty / tz + c.cy;
    const int x0 = (int)fminf(fmaxf(floorf((u - r) / kTile), 0.0f), (float)c.tx);
    const int x1 = (int)fminf(fmaxf(floorf((u + r) / kTile) + 1.0f, 0.0f), (float)c.tx);
    const int y0 = (int)fminf(fmaxf(floorf((v - r) / kTile), 0.0f), (float)c.ty);
    const int y1 = (int)fminf(fmaxf(floorf((v + r) / kTile) + 1.0f, 0.0f), (float)c.ty);
    if (x1 <= x0 || y1 <= y0) return;
    const float dn = sqrtf(qx * qx + qy * qy + qz * qz);
    float Y[16];
    sh_basis(qx / dn, qy / dn, qz / dn, Y);
    float col[3];
    for (int ch = 0; ch < 3; ++ch) {
        float acc = attr[(size_t)ch * n + i] * Y[0];
        for (int k = 1; k < 16; ++k) acc += attr[(size_t)(3 + 15 * ch + k - 1) * n + i] * Y[k];
        col[ch] = fmaxf(0.5f + acc, 0.0f);
    }
    const float op = 1.0f / (1.0f + expf(-attr[48ull * n + i]));
    P.uv[i] = make_float2(u, v);
    P.conic_op[i] = make_float4(cc / det, -cb / det, ca / det, op);
    P.colour[i] = make_float4(col[0], col[1], col[2], 0.0f);
    P.depth[i] = tz;
    P.rect[i] = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
    P.count[i] = (uint32_t)((x1 - x0) * (y1 - y0));
}

// ------------------------------------------------------------------ entries and sort

// Gaussians in depth order: sidx[k] is the k-th nearest (ties by index), cnt_s[k] its tile
// count; depth keys are the positive floats' bits, which order as the floats.
__global__ void k_rs_depth_keys(uint32_t n, Pre P, uint32_t *keys, uint32_t *vals) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = __float_as_uint(P.depth[i]);
    vals[i] = i;
}

__global__ void k_rs_gather_counts(uint32_t n, const uint32_t *sidx, const uint32_t *count, uint32_t *cnt_s) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) cnt_s[k] = count[sidx[k]];
}

// One warp per Gaussian, in depth order: its entries (tile id, Gaussian), tiles in row-major
// order of its rectangle, written by the warp's lanes together.  A stable sort on the tile
// then leaves each tile's Gaussians in depth order.
__global__ void k_rs_emit(uint32_t n, Pre P, const uint32_t *sidx, const uint32_t *off, int tiles_x, uint32_t *keys,
                          uint32_t *vals) {
    const uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31;
    if (k >= n) return;
    const uint32_t i = sidx[k];
    const uint32_t cnt = P.count[i];
    if (cnt == 0) return;
    const uint2 r = P.rect[i];
    const uint32_t x0 = r.x & 0xFFFFu, y0 = r.x >> 16, w = (r.y & 0xFFFFu) - x0;
    const uint32_t base = off[k];
    // entry j covers tile (x0 + j % w, y0 + j / w): one division per lane, then steps of 32
    uint32_t q = lane / w, rr = lane - q * w;
    const uint32_t dq = 32u / w, dr = 32u - dq * w;
    for (uint32_t j = lane; j < cnt; j += 32) {
        keys[base + j] = (y0 + q) * (uint32_t)tiles_x + x0 + rr;
        vals[base + j] = i;
        q += dq;
        rr += dr;
        if (rr >= w) {
            rr -= w;
            ++q;
        }
    }
}

// Each warp takes kRngIlp x 32 consecutive entries (all loaded first), their neighbours by
// shuffles, and only the entries just outside its run from memory.
constexpr int kRngIlp = 8;
constexpr uint32_t kRngEntries = 256 * kRngIlp;  // per CTA of 256 threads

__global__ void __launch_bounds__(256) k_rs_ranges(const uint32_t *keys, uint32_t n, uint2 *ranges) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t wbase = (uint64_t)blockIdx.x * kRngEntries + (uint64_t)(threadIdx.x >> 5) * 32 * kRngIlp;
    uint32_t t[kRngIlp];
#pragma unroll
    for (int r = 0; r < kRngIlp; ++r) {
        const uint64_t i = wbase + 32 * r + lane;
        t[r] = i < n ? keys[i] : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int r = 0; r < kRngIlp; ++r) {
        const uint32_t up = __shfl_up_sync(0xffffffffu, t[r], 1), dn = __shfl_down_sync(0xffffffffu, t[r], 1);
        const uint32_t before = __shfl_sync(0xffffffffu, r > 0 ? t[r > 0 ? r - 1 : 0] : 0u, 31);
        const uint32_t after = __shfl_sync(0xffffffffu, r + 1 < kRngIlp ? t[r + 1 < kRngIlp ? r + 1 : r] : 0u, 0);
        const uint64_t i = wbase + 32 * r + lane;
        if (i >= n) continue;
        const uint32_t prev = lane ? up : (r > 0 ? before : (i ? keys[i - 1] : 0u));
        const uint32_t next = lane < 31 ? dn : (r + 1 < kRngIlp ? after : (i + 1 < n ? keys[i + 1] : 0u));
        if (i == 0 || prev != t[r]) ranges[t[r]].x = (uint32_t)i;
        if (i + 1 == n || next != t[r]) ranges[t[r]].y = (uint32_t)i + 1;
    }
}

__global__ void __launch_bounds__(kTile * kTile) k_rs_render(const uint2 *ranges, const uint32_t *vals, Pre P, Cam c,
                                                              float *img) {
    __shared__ float2 s_uv[kTile * kTile];
    __shared__ float4 s_co[kTile * kTile];
    __shared__ float4 s_col[kTile * kTile];
    const int tile = blockIdx.x;
    const int tx = tile % c.tx, ty = tile / c.tx;
    const int x = tx * kTile + (threadIdx.x % kTile), y = ty * kTile + (threadIdx.x / kTile);
    const bool inside = x < c.w && y < c.h;
    const uint2 rg = ranges[tile];
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    bool done = !inside;
    const float fx = (float)x, fy = (float)y;
    for (uint32_t b = rg.x; b < rg.y; b += kTile * kTile) {
        if (__syncthreads_count(done) == kTile * kTile) break;
        const uint32_t e = b + threadIdx.x;
        if (e < rg.y) {
            const uint32_t g = vals[e];
            s_uv[threadIdx.x] = P.uv[g];
            s_co[threadIdx.x] = P.conic_op[g];
            s_col[threadIdx.x] = P.colour[g];
        }
        __syncthreads();
        const uint32_t m = min((uint32_t)(kTile * kTile), rg.y - b);
        for (uint32_t j = 0; j < m && !done; ++j) {
            const float dx = s_uv[j].x - fx, dy = s_uv[j].y - fy;
            const float4 co = s_co[j];
            const float power = -0.5f * (co.x * dx * dx + co.z * dy * dy) - co.y * dx * dy;
            if (power > 0.0f) continue;
            const float alpha = fminf(0.99f, co.w * expf(power));
            if (alpha < 1.0f / 255.0f) continue;
            const float test_t = T * (1.0f - alpha);
            if (test_t < 0.0001f) { done = true; continue; }
            const float wgt = alpha * T;
            C0 += s_col[j].x * wgt;
            C1 += s_col[j].y * wgt;
            C2 += s_col[j].z * wgt;
            T = test_t;
        }
    }
    if (inside) {
        const size_t hw = (size_t)c.w * c.h, p = (size_t)y * c.w + x;
        img[p] = C0;
        img[hw + p] = C1;
        img[2 * hw + p] = C2;
    }
}

inline uint64_t a256(uint64_t v) { return (v + 255) & ~255ull; }

}  // namespace

}  // namespace sgs

using namespace sgs;

namespace {

int ensure_ws(sgs_ctx *c, size_t bytes) {
    if (bytes <= c->rws_bytes) return SGS_OK;
    if (c->rws) cudaFree(c->rws);
    c->rws = nullptr;
    c->rws_bytes = 0;
    if (cudaMalloc(&c->rws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SGS_E_NOMEM;
    }
    c->rws_bytes = bytes;
    return SGS_OK;
}


}  // namespace

extern "C" int sgs_render(sgs_ctx *ctx, const float *attr, const float *pos, uint32_t n, const sgs_camera *cam,
                          float *image, sgs_stream stream) {
    if (!ctx || !cam || !image || (n && (!attr || !pos)) || cam->width == 0 || cam->height == 0 ||
        cam->width > 16384 || cam->height > 16384 || !(cam->fx > 0.0f) || !(cam->fy > 0.0f))
        return SGS_E_INVALID;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return SGS_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    Cam c;
    memcpy(c.r, cam->rot, sizeof(c.r));
    memcpy(c.o, cam->origin, sizeof(c.o));
    c.fx = cam->fx; c.fy = cam->fy; c.cx = cam->cx; c.cy = cam->cy;
    c.w = (int)cam->width; c.h = (int)cam->height;
    c.tx = (c.w + kTile - 1) / kTile; c.ty = (c.h + kTile - 1) / kTile;
    const uint32_t n_tiles = (uint32_t)(c.tx * c.ty);
    // per-Gaussian arrays and their depth sort, scan sums, tile ranges
    const uint64_t nn = n ? n : 1;
    const uint32_t nsb = (uint32_t)((nn + kScanBlock - 1) / kScanBlock);
    const uint32_t gnb = (uint32_t)((nn + kSortChunk - 1) / kSortChunk);
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) { const uint64_t o = off; off = a256(off + bytes); return o; };
    const uint64_t o_uv = take(8 * nn), o_co = take(16 * nn), o_col = take(16 * nn), o_dep = take(4 * nn),
                   o_rect = take(8 * nn), o_cnt = take(4 * nn), o_off = take(4 * nn), o_sums = take(4ull * (nsb + 1)),
                   o_rng = take(8ull * n_tiles), o_gk0 = take(4 * nn), o_gk1 = take(4 * nn), o_gv0 = take(4 * nn),
                   o_gv1 = take(4 * nn), o_gc = take(4ull * 256 * gnb), o_gco = take(4ull * 256 * gnb),
                   o_gcs = take(4ull * ((256ull * gnb + kScanBlock - 1) / kScanBlock + 1)), o_cs = take(4 * nn);
    int rc = ensure_ws(ctx, off);
    if (rc) return rc;
    uint8_t *b = ctx->rws;
    Pre P;
    P.uv = reinterpret_cast<float2 *>(b + o_uv);
    P.conic_op = reinterpret_cast<float4 *>(b + o_co);
    P.colour = reinterpret_cast<float4 *>(b + o_col);
    P.depth = reinterpret_cast<float *>(b + o_dep);
    P.rect = reinterpret_cast<uint2 *>(b + o_rect);
    P.count = reinterpret_cast<uint32_t *>(b + o_cnt);
    uint32_t *offs = reinterpret_cast<uint32_t *>(b + o_off);
    uint32_t *sums = reinterpret_cast<uint32_t *>(b + o_sums);
    uint32_t *gk[2] = {reinterpret_cast<uint32_t *>(b + o_gk0), reinterpret_cast<uint32_t *>(b + o_gk1)};
    uint32_t *gv[2] = {reinterpret_cast<uint32_t *>(b + o_gv0), reinterpret_cast<uint32_t *>(b + o_gv1)};
    uint32_t *cnt_s = reinterpret_cast<uint32_t *>(b + o_cs);
    auto radix = [&](uint32_t **k2, uint32_t **v2, uint32_t count, int bits, uint32_t *cnt, uint32_t *cnt_off,
                     uint32_t *csums) -> int {
        const uint32_t nb = (count + kSortChunk - 1) / kSortChunk;
        int cur = 0;
        (void)nb;
        for (int sh = 0; sh < bits; sh += 8) {
            if (radix_pass(k2[cur], v2[cur], count, sh, cnt, cnt_off, csums, k2[cur ^ 1], v2[cur ^ 1], st) !=
                cudaSuccess)
                return -1;
            cur ^= 1;
            ctx->launches += 5;
        }
        return cur;
    };
    uint32_t E = 0;
    int gcur = 0;
    if (n) {
        k_rs_pre<<<(n + 255) / 256, 256, 0, st>>>(attr, pos, n, c, P);
        k_rs_depth_keys<<<(n + 255) / 256, 256, 0, st>>>(n, P, gk[0], gv[0]);
        gcur = radix(gk, gv, n, 32, reinterpret_cast<uint32_t *>(b + o_gc), reinterpret_cast<uint32_t *>(b + o_gco),
                     reinterpret_cast<uint32_t *>(b + o_gcs));
        if (gcur < 0) return SGS_E_CUDA;
        k_rs_gather_counts<<<(n + 255) / 256, 256, 0, st>>>(n, gv[gcur], P.count, cnt_s);
        if (scan_u32(cnt_s, n, sums, offs, st) != cudaSuccess) return SGS_E_CUDA;
        ctx->launches += 6;
        if (cudaMemcpyAsync(&E, sums + nsb, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SGS_E_CUDA;
    }
    // entries (double-buffered tile keys and Gaussian indices) and the sort's digit counts;
    // the per-Gaussian results live below `fixed`, kept when the workspace grows
    const uint64_t fixed = off;
    const uint64_t ne = E ? E : 1;
    const uint32_t nb = (uint32_t)((ne + kSortChunk - 1) / kSortChunk);
    const uint32_t ncnt = 256u * nb, ncsb = (ncnt + kScanBlock - 1) / kScanBlock;
    const uint64_t o_k0 = take(4 * ne), o_k1 = take(4 * ne), o_v0 = take(4 * ne), o_v1 = take(4 * ne),
                   o_c = take(4ull * ncnt), o_co2 = take(4ull * ncnt), o_cs2 = take(4ull * (ncsb + 1));
    if (off > ctx->rws_bytes) {
        uint8_t *nbuf = nullptr;
        if (cudaMalloc(&nbuf, off) != cudaSuccess) {
            cudaGetLastError();
            return SGS_E_NOMEM;
        }
        if (cudaMemcpyAsync(nbuf, ctx->rws, fixed, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaFree(nbuf);
            return SGS_E_CUDA;
        }
        cudaFree(ctx->rws);
        ctx->rws = nbuf;
        ctx->rws_bytes = off;
        b = nbuf;
        P.uv = reinterpret_cast<float2 *>(b + o_uv);
        P.conic_op = reinterpret_cast<float4 *>(b + o_co);
        P.colour = reinterpret_cast<float4 *>(b + o_col);
        P.depth = reinterpret_cast<float *>(b + o_dep);
        P.rect = reinterpret_cast<uint2 *>(b + o_rect);
        P.count = reinterpret_cast<uint32_t *>(b + o_cnt);
        offs = reinterpret_cast<uint32_t *>(b + o_off);
        gv[0] = reinterpret_cast<uint32_t *>(b + o_gv0);
        gv[1] = reinterpret_cast<uint32_t *>(b + o_gv1);
    }
    uint32_t *keys[2] = {reinterpret_cast<uint32_t *>(b + o_k0), reinterpret_cast<uint32_t *>(b + o_k1)};
    uint32_t *vals[2] = {reinterpret_cast<uint32_t *>(b + o_v0), reinterpret_cast<uint32_t *>(b + o_v1)};
    uint2 *ranges = reinterpret_cast<uint2 *>(b + o_rng);
    if (cudaMemsetAsync(ranges, 0, 8ull * n_tiles, st) != cudaSuccess) return SGS_E_CUDA;
    int cur = 0;
    if (E) {
        k_rs_emit<<<(uint32_t)((32ull * n + 255) / 256), 256, 0, st>>>(n, P, gv[gcur], offs, c.tx, keys[0], vals[0]);
        int tile_bits = 0;
        while ((1u << tile_bits) < n_tiles) ++tile_bits;
        cur = radix(keys, vals, E, tile_bits, reinterpret_cast<uint32_t *>(b + o_c),
                    reinterpret_cast<uint32_t *>(b + o_co2), reinterpret_cast<uint32_t *>(b + o_cs2));
        if (cur < 0) return SGS_E_CUDA;
        k_rs_ranges<<<(uint32_t)((E + kRngEntries - 1) / kRngEntries), 256, 0, st>>>(keys[cur], E, ranges);
        ctx->launches += 2;
    }
    ctx->launches += 1;
    k_rs_render<<<n_tiles, kTile * kTile, 0, st>>>(ranges, vals[cur], P, c, image);
    if (cudaGetLastError() != cudaSuccess) return SGS_E_CUDA;
    return SGS_OK;
}
