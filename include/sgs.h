/*
 * sgs.h -- C ABI of the B300 decoder for SpeedyGS-compressed 3D Gaussian Splatting scenes.
 *
 * A scene's bitstream holds a geometry stream (sparse-octree occupancy tokens, Sec. 3.4
 * "Geometry Occupancy Coding") and an attribute stream (56 channels per Gaussian in Morton
 * order, Sec. 3.4 "Autoregressive Attribute Coding"), coded either with channel-wise
 * fixed-length codes (Sec. 3.4.1), channel-wise static-frequency rANS, or rANS driven by the
 * local autoregressive context model (Sec. 3.4.2; groups of W Gaussians = rANS lanes).
 * Decoding reproduces the quantized scene exactly; the coders change only the bytes.
 *
 * Conventions
 *   - Every entry point returns an int status: SGS_OK (0) or a negative SGS_E_* code.
 *     No C++ exception crosses this boundary.
 *   - "device" pointers are CUDA device pointers on the context's device; "host" pointers are
 *     ordinary host memory (pageable or pinned).
 *   - The caller owns every input and output buffer.  The context owns its device scratch,
 *     its status word and its internal streams.
 *   - A context is not thread safe: use one per host thread or guard it.
 *   - Decode entry points are asynchronous on the given stream; their device-side status
 *     (corrupt stream, timed-out wait) is read with sgs_sync().
 *
 * Output layout (structure of arrays, rows in (Morton code, original index) order unless an
 * out_index is given):
 *   attr  float [56][n_rows]   channel c at attr + c * n_rows
 *   pos   float [3][n_rows]    voxel centres coord * 2^-D + 2^-(D+1)
 *   coord uint32 [3][n_rows]   voxel coordinates (optional)
 * Channel order: 0..2 SH DC, 3..47 SH rest (3 + colour*15 + k-1), 48 opacity logit,
 * 49..51 log-scale, 52..55 rotation.
 */
#ifndef SGS_H
#define SGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SGS_OK 0
#define SGS_E_INVALID -1      /* bad argument or malformed header                        */
#define SGS_E_CORRUPT -2      /* bitstream failed validation or a rANS end check         */
#define SGS_E_NOMEM -3        /* scratch too small, or an allocation failed             */
#define SGS_E_CUDA -4         /* a CUDA call failed                                       */
#define SGS_E_TIMEOUT -5      /* a bounded device-side wait gave up                       */
#define SGS_E_UNSUPPORTED -6  /* feature not built                                        */

#define SGS_MODE_FIXED 0      /* channel-wise fixed-length codes (Sec. 3.4.1)            */
#define SGS_MODE_STATIC 1     /* channel-wise static-frequency rANS                       */
#define SGS_MODE_LEARNED 2    /* rANS with the learned context model (Sec. 3.4.2)        */
#define SGS_MODE_LEARNED_PE 3 /* rANS with the position-aware learned model: the Fourier
                                 positional embedding of Sec. 3.4.2 (L = 12 bands, d = 32)
                                 and a conditional Laplace head (Sec. 3.2)                  */
#define SGS_GEO_RAW 0         /* occupancy tokens stored as bytes                         */
#define SGS_GEO_RANS 1        /* levels of >= 4096 nodes coded with per-level rANS tables */
#define SGS_GEO_LEARNED 2     /* levels of >= 4096 nodes coded with a learned model of the
                                 level above (Eq. 8): context = (parent byte, child index),
                                 the SGS_MODEL_BYTES integer model with the level as its
                                 channel; each coded level in lanes of about 128 tokens.
                                 Decoded by scene_decode and scene_decode_noalloc (level by
                                 level); a batch plan refuses it (SGS_E_UNSUPPORTED)        */

#define SGS_NCHAN 56
#define SGS_MAX_DEPTH 21

typedef struct sgs_ctx sgs_ctx;
typedef void *sgs_stream; /* a cudaStream_t (0 = legacy default stream) */

/* Header facts of a bitstream, filled by scene_query (host only, no device work). */
typedef struct {
    uint32_t mode, geo_mode;
    uint32_t n_in;          /* Gaussians before pruning                                  */
    uint32_t n_rows;        /* decoded Gaussians N' (rows of every output array)         */
    uint32_t depth;         /* octree depth D                                            */
    uint32_t n_leaves;      /* unique voxels U                                           */
    uint32_t n_dup;         /* duplicate-count entries                                   */
    uint32_t lanes;         /* attribute rANS lanes L (0 for fixed-length)              */
    uint32_t geo_lanes;     /* geometry rANS lanes (0 if no level is coded)             */
    uint32_t n_level[SGS_MAX_DEPTH + 1]; /* nodes per level 0..D-1, then U at [D]       */
    uint64_t n_geo;         /* occupancy bytes (internal nodes)                          */
    uint64_t n_geo_coded;   /* of which rANS coded                                       */
    uint64_t off[11];       /* section offsets: levels, dup, chan, geo_raw, geo_tab,
                               geo_grp, geo_pay, attr_tab, attr_grp, attr_pay, total   */
    uint64_t total_len;     /* bitstream bytes                                           */
    uint64_t scratch_bytes; /* device scratch scene_decode needs for this scene          */
    uint32_t n_tables;      /* static tables: coded octree levels, then 56 attribute ones */
    uint32_t table_off[SGS_NCHAN + SGS_MAX_DEPTH]; /* byte offset of each table in the bitstream */
} sgs_scene_info;

/* Caller-allocated device outputs of one scene (sizes from sgs_scene_info.n_rows). */
typedef struct {
    float *attr;              /* device [56][n_rows], required                             */
    float *pos;               /* device [3][n_rows], required                              */
    uint32_t *coord;          /* device [3][n_rows] or NULL                                */
    const uint32_t *out_index;/* device [n_rows] or NULL: row r is written to column
                                 out_index[r] (a permutation of 0..n_rows-1, caller-checked) */
} sgs_scene_out;

/* Encoder parameters. */
typedef struct {
    uint32_t mode;            /* SGS_MODE_*                                               */
    uint32_t geo_mode;        /* SGS_GEO_*                                                */
    uint32_t depth;           /* 1..21                                                    */
    uint32_t lanes;           /* attribute rANS lanes (entropy-coded modes), >= 1          */
    uint32_t geo_lanes;       /* geometry rANS lanes, 0 = about 128 tokens per lane        */
    uint32_t bits[SGS_NCHAN]; /* fixed-length bit widths 1..16 (8 is forced for rANS modes)*/
    const void *model;        /* learned modes: the frozen model (SGS_MODEL_BYTES, or
                                 SGS_MODEL_PE_BYTES for SGS_MODE_LEARNED_PE), else NULL    */
    const void *geo_model;    /* SGS_GEO_LEARNED: the geometry model (SGS_MODEL_BYTES; its
                                 inputs u = (b - 128, 32 k - 112, 16 popcount(b) - 64,
                                 32 rank - 112) of parent byte b and child index k, rank =
                                 set bits of b below k; channel = level), else NULL        */
} sgs_encode_params;

#define SGS_MODEL_BYTES 36384

/* Frozen position-aware model (the model section of SGS_MODE_LEARNED_PE), little endian:
 *   f32 s1, s2 (requantisation scales, in (0, 127]), smu, slr (head multipliers, > 0);
 *   16 zero bytes; i32 B1[56][64] (channel embedding and projection bias folded in);
 *   i32 b2[64]; i32 b3[2] + 8 zero bytes; i8 W1[64][80] over [u (4); phi (75); 0]
 *   (the projection folded in); i8 W2[64][64]; i8 W3[2][64].  Biases below 2^23 in
 *   magnitude.  Inference: h = clamp(rint(fl32(acc * s)), 0, 127) per layer; mean
 *   mu8 = 32640 + clamp(rint(z0 * smu), +-32640) (1/256 symbol); n = 4096 +
 *   clamp(rint(z1 * slr), -2048, 1536) (log2 rate in 1/256, plus 16); token CDF
 *   cdf(s) = s + floor(65280 F(s - 1/2) / 2^23), F the Laplace CDF through EXP2Q.        */
#define SGS_MODEL_PE_BYTES 23984

/* Training parameters of the context model (the learned part, Sec. 3.4.2). */
typedef struct {
    uint32_t steps;           /* Adam steps (2000 in the 1M-Gaussian workload)            */
    uint32_t batch;           /* tokens per step (65536), <= 2^20                          */
    uint32_t seed;            /* batch sampler seed (splitmix64 counter stream)            */
    float lr;                 /* Adam learning rate (1e-3)                                 */
} sgs_train_params;

/* Float weights of the context model, all fp32, row-major:
 *   emb[56][16], w1[64][20], b1[64], w2[64][64], b2[64], w3[256][64], b3[256].             */
#define SGS_WEIGHTS_FLOATS (56 * 16 + 64 * 20 + 64 + 64 * 64 + 64 + 256 * 64 + 256)

/* Float weights of the position-aware model, all fp32, row-major:
 *   emb[56][16], wp[32][75], bp[32] (the projection PE = wp phi + bp of Sec. 3.4.2),
 *   w1[64][52] over [u / 128 (4), emb (16), PE (32)], b1[64], w2[64][64], b2[64],
 *   w3[2][64], b3[2] (mean 127.5 + 64 z0 clipped to [0, 255], log2 rate z1 clipped to
 *   [-8, 6]).                                                                            */
#define SGS_WEIGHTS_PE_FLOATS (56 * 16 + 32 * 75 + 32 + 64 * 52 + 64 + 64 * 64 + 64 + 2 * 64 + 2)

/* ------------------------------------------------------------------ context */

/* Text of a status code (static storage). */
const char *sgs_strerror(int code);

/* Creates a context on CUDA device `device` owning `scratch_bytes` of device scratch
 * (grown on demand by sgs_reserve, never inside a decode call).  *out is NULL on failure.
 * Errors: SGS_E_INVALID (bad device), SGS_E_NOMEM, SGS_E_CUDA.                            */
int sgs_create(sgs_ctx **out, int device, size_t scratch_bytes);

/* Grows the context's scratch to at least `scratch_bytes` (synchronizes the device). */
int sgs_reserve(sgs_ctx *ctx, size_t scratch_bytes);

void sgs_destroy(sgs_ctx *ctx);

/* Waits for `stream` and returns the worst device-side status recorded by decode calls on
 * this context since the last sgs_sync (then clears it).  Returns SGS_E_CORRUPT,
 * SGS_E_TIMEOUT, SGS_E_CUDA or SGS_OK.                                                      */
int sgs_sync(sgs_ctx *ctx, sgs_stream stream);

/* Enables (1) or disables (0) stage timing: decode calls then record CUDA events on their
 * stream between the geometry-token, octree and attribute stages. */
int sgs_profile(sgs_ctx *ctx, int enable);

/* Stage times in ms of the most recent profiled single-scene decode (after the stream has
 * completed it): ms[0] geometry tokens (table expansion, raw copy, rANS), ms[1] octree
 * expansion and positions, ms[2] attribute decode and dequantization (measured on the
 * context's attribute stream, where it runs concurrently with ms[0] and ms[1]), ms[3] the
 * whole decode.  cap >= 4.  Errors: SGS_E_INVALID (no profiled decode), SGS_E_CUDA.         */
int sgs_profile_read(sgs_ctx *ctx, float *ms, int cap);

/* Number of CUDA kernels enqueued by decode calls on this context since its creation. */
uint64_t sgs_launch_count(sgs_ctx *ctx);

/* Poll budget of the device-side waits of this context's learned-model decodes (the
 * hand-offs between the decoder's producer and consumer warps, Sec. 3.4.2's per-group
 * decode).  Each wait polls at most `polls` times (with a short sleep between polls) and
 * then gives up: the decode's status becomes SGS_E_TIMEOUT (read with sgs_sync), every warp
 * of the CTA leaves its loop and the context stays usable.  polls = 0 restores the default,
 * 2^24 polls (seconds, far beyond any legitimate wait).  Failure detection without a GPU
 * fault: a budget of 1 makes the first wait that is not already satisfied give up.
 * Applies to scene_decode calls made after it.  Errors: SGS_E_INVALID (NULL ctx).          */
int sgs_set_wait_limit(sgs_ctx *ctx, uint32_t polls);

/* ------------------------------------------------------------------ decode */

/* Parses and validates the header of a bitstream (host bytes `bits`, `len` bytes, at least
 * the header and the level table; the section offsets are checked against total_len).
 * Definition of the fields: Sec. 3.4 split into geometry and attribute streams.
 * Errors: SGS_E_INVALID (short buffer, bad magic/version/sizes/offsets, or, for
 * SGS_GEO_LEARNED, a model section shorter than SGS_MODEL_BYTES or lanes and group tables
 * that are not the coded levels' own), SGS_E_UNSUPPORTED (an octree beyond 2^29 nodes).    */
int scene_query(const uint8_t *bits, size_t len, sgs_scene_info *info);

/* Decodes one scene: occupancy tokens -> octree expansion (Sec. 3.4, Geometry Occupancy
 * Coding) -> positions; attribute tokens (fixed-length unpack, static rANS or learned
 * rANS, Sec. 3.4.1-3.4.2) -> dequantization v = fl(fl(q*step) + offset) into `out`.
 * bits_dev: device copy of the whole bitstream (16-byte aligned), info from scene_query on
 * the same bytes.  Asynchronous on `stream`; uses only the context's scratch.
 * Errors: SGS_E_INVALID (NULL output, misaligned input), SGS_E_NOMEM (scratch smaller than
 * info->scratch_bytes; nothing is launched), SGS_E_CUDA (launch failure).  Device-side
 * corruption is reported by sgs_sync.                                                       */
int scene_decode(sgs_ctx *ctx, const uint8_t *bits_dev, const sgs_scene_info *info,
                 const sgs_scene_out *out, sgs_stream stream);

/* Size of the fixed device scratch area scene_decode_noalloc uses (64 MiB; enough for the
 * 1,000,000-Gaussian depth-16 fixed-length scene). */
#define SGS_NOALLOC_SCRATCH_BYTES (64u << 20)

/* Decodes one scene without allocating anything: for callers that cannot allocate device
 * memory (an engine or renderer that owns all device memory and forbids allocation after
 * start-up, or a latency-critical loop where cudaMalloc / cudaFree could synchronize the
 * device), and so cannot create an sgs_ctx.  The paper has no counterpart; this is runtime
 * plumbing.  Instead of a context's scratch it uses a fixed device array of
 * SGS_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU that loads the
 * library holds until the process exits.  Arguments are those of scene_decode (bits_dev:
 * device copy of the whole bitstream, 16-byte aligned; info from scene_query; out:
 * caller-allocated device outputs), on the current CUDA device, on `stream`.
 *   - Synchronous: returns after the decode has completed on `stream`, with its status
 *     (SGS_OK, SGS_E_CORRUPT, SGS_E_TIMEOUT).  It reads the status back and synchronizes
 *     the stream, so it must never be called while a stream is being captured into a CUDA
 *     graph (scene_decode is the call to capture).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress).
 *   - Every call on a device shares the one array and finds the previous call's contents
 *     (the call clears what must start at zero).  Calls that overlap on the GPU -- from two
 *     host threads, or on two streams -- race on the array and must not be made.
 * Errors: SGS_E_INVALID (NULL or misaligned arguments), SGS_E_NOMEM (the scene needs more
 * scratch than SGS_NOALLOC_SCRATCH_BYTES minus 256 bytes; nothing is launched), SGS_E_CUDA. */
int scene_decode_noalloc(const uint8_t *bits_dev, const sgs_scene_info *info,
                         const sgs_scene_out *out, sgs_stream stream);

/* One scene of a batch: its bitstream (device, 16-byte aligned), its scene_query result and
 * its caller-allocated outputs (as for scene_decode). */
typedef struct {
    const uint8_t *bits_dev;
    sgs_scene_info info;
    sgs_scene_out out;
} sgs_batch_item;

/* Batched decode (no counterpart in the paper, which decodes one scene at a time; the scenes
 * are independent, and Sec. 3.4.2's parallelism over groups extends across them).  Every
 * pipeline stage of all n scenes runs as ONE persistent launch: its CTAs take work items
 * (the lanes' groups, table expansions, scan tiles, blocks of octree leaves of every scene)
 * from a shared counter, so a run is at most 14 stage launches whatever n is (plus one
 * kernel that starts the run and one that folds the scenes' status words).
 *
 * A plan binds the items' buffers (bitstreams, outputs) and holds, in one device block, every
 * scene's scratch, the per-stage work lists and per-scene status words. */
typedef struct sgs_batch sgs_batch;

/* Device bytes of a plan for these items (the scratch of every scene plus the work lists).
 * Errors: SGS_E_INVALID (NULL, misaligned bitstream, missing outputs, info not produced by
 * scene_query), SGS_E_UNSUPPORTED (more than 2^31 work items in a stage, or a scene whose
 * geometry is SGS_GEO_LEARNED-coded: decode those with scene_decode). */
int scene_batch_bytes(const sgs_batch_item *items, int n, size_t *bytes);

/* Builds a plan on ctx's device: allocates its device block (cudaMalloc) and uploads the
 * work lists (synchronously).  The items array may be freed afterwards; the buffers it
 * points to must stay valid while the plan is used.  Errors: as scene_batch_bytes, plus
 * SGS_E_NOMEM, SGS_E_CUDA. */
int scene_batch_plan(sgs_ctx *ctx, const sgs_batch_item *items, int n, sgs_batch **plan);

/* Enqueues one decode of every scene of the plan on `stream` (the context's internal
 * streams fork from it and join back).  Allocates nothing and does not wait for the device,
 * so the call can be captured in a CUDA graph and replayed; every run re-decodes the bound
 * bitstreams into the bound outputs.  A run's status goes to the context (sgs_sync) and per
 * scene to scene_batch_status.  Runs of one plan, or of plans sharing the context, must be
 * ordered on one stream.  Errors: SGS_E_INVALID (plan of another device), SGS_E_CUDA. */
int scene_batch_run(sgs_ctx *ctx, sgs_batch *plan, sgs_stream stream);

/* Copies the per-scene status words of the plan's last completed run (n = the plan's
 * scene count) to host memory; call after the run's stream has finished.  Blocking. */
int scene_batch_status(const sgs_batch *plan, int *status, int n);

/* Per-scene completion times of the plan's last completed run (n = the plan's scene count),
 * in milliseconds: from the run's first kernel to the end of the scene's last work item over
 * all of the run's launches, both read from the device's global nanosecond timer.  Each
 * scene keeps a completion count that every finished work item increments; the item that
 * completes it stamps the time.  A scene without work items gets -1.  Blocking; call after
 * the run's stream has finished. */
int scene_batch_times(const sgs_batch *plan, double *ms, int n);

/* Frees the plan's device block (after its runs have finished). */
void scene_batch_free(sgs_batch *plan);

/* One-shot batched decode with the context's scratch as the plan's device block: needs
 * scene_batch_bytes(items, n) <= the context's scratch (else SGS_E_NOMEM, nothing enqueued).
 * Asynchronous; the work lists are copied to the scratch in `stream` order, so calls that
 * share the context must use one stream.  Status via sgs_sync.  Same errors as scene_decode. */
int scene_decode_batch(sgs_ctx *ctx, const sgs_batch_item *items, int n, sgs_stream stream);

/* ------------------------------------------------------------------ encode */

/* Encodes a scene given as host arrays pos[3][n] (in [0,1)) and attr[56][n] (finite):
 * prune floor(n/10) of lowest opacity, voxelize, Morton sort, octree, per-channel quantize,
 * then code (Sec. 3.3-3.4).  Writes at most `cap` bytes to `out` (host) and sets *out_len.
 * If cap is too small returns SGS_E_INVALID with *out_len = the size needed.  With a ctx the
 * attribute streams' interleaved rANS coding (static and learned) runs on its device; ctx may
 * be NULL except in learned mode, and then static coding runs on the host.  Either way the
 * bytes are the same.
 * Errors: SGS_E_INVALID, SGS_E_NOMEM, SGS_E_CUDA.                                            */
int scene_encode(sgs_ctx *ctx, const float *pos, const float *attr, uint32_t n,
                 const sgs_encode_params *params, uint8_t *out, size_t cap, size_t *out_len);

/* Quantized tokens of a scene exactly as the encoder codes them: host uint8 [n_rows][56]
 * (rows in Morton order) for 8-bit channels, after pruning.  *n_rows set.  Used to train
 * the context model on the scene's own tokens.  cap in bytes.                               */
int scene_tokens(const float *pos, const float *attr, uint32_t n, uint32_t depth,
                 uint8_t *tokens, size_t cap, uint32_t *n_rows);

/* Training samples of the learned geometry coder (SGS_GEO_LEARNED): for every node of each
 * level of >= 4096 nodes (levels 1..depth-1, in order, nodes in order), its context inputs
 * u [4] (of its parent byte b and child index k, as sgs_encode_params.geo_model), its level
 * as the channel and its occupancy byte as the symbol: host int32 u [cap][4], uint32
 * chan [cap], uint8 sym [cap]; *n_samples set; SGS_E_INVALID if cap is too small.          */
int scene_geo_samples(const float *pos, const float *attr, uint32_t n, uint32_t depth, int32_t *u,
                      uint32_t *chan, uint8_t *sym, uint64_t cap, uint64_t *n_samples);

/* As scene_tokens, plus the rows' voxel coordinates (host uint32 [3][n_rows], the decoder's
 * coord output), the inputs of the position-aware model's training and freeze.  cap: rows
 * the caller's arrays hold.                                                                  */
int scene_rows(const float *pos, const float *attr, uint32_t n, uint32_t depth, uint8_t *tokens,
               uint32_t *coord, uint32_t cap, uint32_t *n_rows);

/* ------------------------------------------------------------------ rendering */

/* A pinhole camera: world point p maps to camera space t = rot (p - origin) (rot row-major,
 * camera axes x right, y down, z forward) and to pixel (fx t_x / t_z + cx, fy t_y / t_z + cy);
 * pixel (x, y) is sampled at its integer coordinates. */
typedef struct {
    float rot[9];
    float origin[3];
    float fx, fy, cx, cy;
    uint32_t width, height;   /* 1 .. 16384 */
} sgs_camera;

/* Renders n decoded Gaussians (device attr [56][n] and pos [3][n], as scene_decode writes
 * them) into image_dev (device float [3][height][width], background 0) with tile splatting,
 * the 3DGS forward pass the paper's decoded scenes are drawn with (no counterpart in the
 * paper's coder; its tables' rendering column): per Gaussian the projected 2D covariance
 * (+0.3 I), radius ceil(3 sqrt(lambda_max)) and the 16 x 16-pixel tiles it touches, colour
 * from the degree-3 spherical harmonics (channels 0-47) along the view ray, opacity
 * sigmoid(channel 48), scales exp(channels 49-51), rotation the quaternion (w, x, y, z) of
 * channels 52-55; per pixel the tile's Gaussians front to back (depth, then index), alpha =
 * min(0.99, opacity exp(-0.5 d^T Sigma'^-1 d)) skipped below 1/255, compositing stopped
 * before the transmittance falls below 1e-4; Gaussians with camera depth <= 0.2 are culled.
 * Synchronous: reads back the number of (tile, Gaussian) pairs to size the sort.  The
 * context keeps a workspace for it (grown with cudaMalloc when a frame needs more, freed
 * by sgs_destroy).  Errors: SGS_E_INVALID, SGS_E_NOMEM, SGS_E_CUDA. */
int sgs_render(sgs_ctx *ctx, const float *attr_dev, const float *pos_dev, uint32_t n, const sgs_camera *camera,
               float *image_dev, sgs_stream stream);

/* ------------------------------------------------------------------ autotuning */

/* Lane-count tuning: the paper's complexity knob is the group size W, Gaussians per
 * autoregressive group (Sec. 4, implementation details: W = 256 for the main model, 32 for
 * the fast one); here lanes = ceil(N' / W).  sgs_autotune encodes the given scene at every
 * candidate W, decodes each bitstream on the context's device `reps` times (CUDA events,
 * median), and picks the smallest bitstream whose decode time is at most max_ms (the fastest
 * one if max_ms <= 0 or none qualifies).  With shape candidates (n_shape > 0) each W is also
 * decoded at every candidate launch shape of the attribute decoder (sgs_set_launch_shape)
 * and keeps its fastest; the context's own shapes are restored before returning.  For
 * SGS_MODE_FIXED (no lanes) n_cand must be 1 and rows_per_lane is ignored: only shapes are
 * searched. */
#define SGS_TUNE_MAX_CAND 16
typedef struct {
    const float *pos, *attr;  /* host scene, as for scene_encode                           */
    uint32_t n;
    uint32_t mode;            /* SGS_MODE_STATIC, SGS_MODE_LEARNED or SGS_MODE_LEARNED_PE */
    uint32_t depth;
    uint32_t geo_mode;
    const void *model;        /* learned modes: the frozen model                          */
    uint32_t n_cand;          /* 1 .. SGS_TUNE_MAX_CAND                                   */
    uint32_t rows_per_lane[SGS_TUNE_MAX_CAND];  /* candidate W values, >= 1              */
    float max_ms;             /* decode-time target, <= 0: fastest                         */
    uint32_t reps;            /* timed decodes per candidate (>= 1)                       */
    uint32_t n_shape;         /* 0 .. SGS_TUNE_MAX_CAND launch shapes to try (0: built-in) */
    uint32_t warps_per_cta[SGS_TUNE_MAX_CAND];  /* candidate shapes, as sgs_set_launch_shape */
} sgs_tune_request;

typedef struct {
    uint32_t best;            /* index of the chosen candidate                            */
    uint32_t lanes[SGS_TUNE_MAX_CAND];
    uint64_t bytes[SGS_TUNE_MAX_CAND];   /* bitstream size                                */
    float ms[SGS_TUNE_MAX_CAND];         /* median decode time (at the candidate's best shape) */
    uint32_t warps[SGS_TUNE_MAX_CAND];   /* the candidate's fastest shape (0: built-in)   */
    uint32_t best_warps;                 /* warps[best]                                    */
} sgs_tune_result;

/* Launch shape of the attribute decoder in the context's single-scene decodes of `mode`
 * (the autotuner's second knob besides W): SGS_MODE_FIXED, warps per CTA of the
 * fixed-length unpack (1..8, each warp one channel x 1,024 rows); SGS_MODE_STATIC, the
 * most groups of 32 lanes (warps) per CTA sharing one copy of the 56 tables (1..32; fewer
 * when the scene has fewer groups than SMs x this).  0 restores the built-in shape (8; 32).
 * Results do not depend on the shape.  Errors: SGS_E_INVALID (other mode, out of range).    */
int sgs_set_launch_shape(sgs_ctx *ctx, uint32_t mode, uint32_t warps_per_cta);

/* Allocates device memory for the trial bitstreams and outputs (freed before returning)
 * and may grow the context's scratch.  Synchronous.  Errors: SGS_E_INVALID (bad request),
 * SGS_E_NOMEM, SGS_E_CUDA, or the status of a failed trial decode. */
int sgs_autotune(sgs_ctx *ctx, const sgs_tune_request *req, sgs_tune_result *res);

/* ------------------------------------------------------------------ learned part */

/* Trains the context model (Sec. 3.4.2; loss = code length in bits, Eq. 9) on the device:
 * tokens_dev device uint8 [n_rows][56]; lanes = rANS lanes of the scene (contexts stop at
 * lane starts); weights_dev device fp32 [SGS_WEIGHTS_FLOATS], initial values in, trained
 * values out; adam_dev device fp32 [2 * SGS_WEIGHTS_FLOATS] Adam moments, zero to start
 * (or a previous run's state to resume at step `step0`); loss_dev device fp32 [steps] or
 * NULL.  Synchronous.  Errors: SGS_E_INVALID, SGS_E_NOMEM, SGS_E_CUDA.                      */
int sgs_train(sgs_ctx *ctx, const uint8_t *tokens_dev, uint32_t n_rows, uint32_t lanes,
              const sgs_train_params *params, uint32_t step0, float *weights_dev,
              float *adam_dev, float *loss_dev);

/* One forward/backward pass on the device for a given batch of token positions
 * (pos_dev device int64 [batch], p = 56 * row + channel): loss (bits per token, fp32 host)
 * and gradients grad_dev device fp32 [SGS_WEIGHTS_FLOATS].  For gradient checks.            */
int sgs_train_grad(sgs_ctx *ctx, const uint8_t *tokens_dev, uint32_t n_rows, uint32_t lanes,
                   const int64_t *pos_dev, uint32_t batch, const float *weights_dev,
                   float *grad_dev, float *loss_host);

/* Freezes fp32 weights (host, SGS_WEIGHTS_FLOATS) to the integer model (host,
 * SGS_MODEL_BYTES): int8 weights, int32 biases with the channel embedding folded in,
 * requantization multipliers from an integer calibration pass over 65,536 tokens of
 * tokens (host uint8 [n_rows][56]) drawn with `seed`.  Errors: SGS_E_INVALID.              */
int sgs_freeze(const float *weights, const uint8_t *tokens, uint32_t n_rows, uint32_t lanes,
               uint32_t seed, uint8_t *model_out);

/* As sgs_freeze, for a model whose contexts are an explicit sample set rather than the
 * previous tokens of a row (the learned geometry coder's (parent byte, child index) inputs,
 * SGS_GEO_LEARNED): u host int32 [n][4] in [-128, 127], chan host uint32 [n] below
 * SGS_NCHAN; calibration sample k is entry sample_pos(seed, 2^20 - 1, k, n) of the set, with
 * the trainer's counter-based sampler.  Writes SGS_MODEL_BYTES.  Errors: SGS_E_INVALID
 * (missing arrays, n = 0, non-finite weights, inputs out of range).                        */
int sgs_freeze_samples(const float *weights, const int32_t *u, const uint32_t *chan, uint64_t n,
                       uint32_t seed, uint8_t *model_out);

/* The position-aware model (SGS_MODE_LEARNED_PE; float layout SGS_WEIGHTS_PE_FLOATS): as
 * sgs_train / sgs_train_grad / sgs_freeze with the rows' voxel coordinates (coord_dev device,
 * coord host: uint32 [3][n_rows], from scene_rows) at octree depth `depth`.  Loss = code
 * length in bits under the discretised Laplace (Sec. 3.2) with the coder's one-count floor,
 * p(s) = (1 + 65280 P(s)) / 65536.  The freeze folds the embedding projection into layer 1
 * and writes SGS_MODEL_PE_BYTES.  Errors: SGS_E_INVALID, SGS_E_NOMEM, SGS_E_CUDA.          */
int sgs_train_pe(sgs_ctx *ctx, const uint8_t *tokens_dev, const uint32_t *coord_dev, uint32_t depth,
                 uint32_t n_rows, uint32_t lanes, const sgs_train_params *params, uint32_t step0,
                 float *weights_dev, float *adam_dev, float *loss_dev);
int sgs_train_pe_grad(sgs_ctx *ctx, const uint8_t *tokens_dev, const uint32_t *coord_dev, uint32_t depth,
                      uint32_t n_rows, uint32_t lanes, const int64_t *pos_dev, uint32_t batch,
                      const float *weights_dev, float *grad_dev, float *loss_host);
int sgs_freeze_pe(const float *weights, const uint8_t *tokens, const uint32_t *coord, uint32_t depth,
                  uint32_t n_rows, uint32_t lanes, uint32_t seed, uint8_t *model_out);

#ifdef __cplusplus
}
#endif
#endif /* SGS_H */
