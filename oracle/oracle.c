/*
 * CPU oracle, native part.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * CPU-baseline leg of the benchmark call it; the library never does.  It shares no code,
 * header or table with the CUDA library.
 *
 * Plain, sequential, obviously-correct loops for the parts of the method that are too slow
 * in numpy:
 *   - interleaved rANS encode/decode (the entropy coder standing in for the paper's "AC",
 *     Sec. 3.4 and Tab. decoding_complexity; rANS after Duda, lane interleaving after
 *     Giesen arXiv:1402.3392), with the decoder taking one static table per symbol
 *     position (channel-wise coding of attributes, per-level coding of octree bytes);
 *   - the integer local autoregressive context model and its integer softmax -> 16-bit
 *     frequency table (the learned CDF of Sec. 3.4 "Autoregressive Prediction Coding",
 *     made integer so encoder and decoder agree bit for bit), and the learned decoder.
 *
 *   - the position-aware model (Fourier positional embedding, Laplace head) and its decoder:
 *     integer sums, fp32 requantisation with one multiply and round-half-to-even, and the
 *     integer Laplace CDF.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (the only floating point is the fp32
 * requantisation of the position-aware model: single multiplies, never fused).
 *
 * Stream format of one group of up to 32 lanes (words are uint16, little endian):
 *   32 initial states, lane j ascending, each as (hi word, lo word);
 *   then for step t = 0, 1, ...: for each lane j ascending that still has a symbol t:
 *   decode symbol t, and if the state fell below 2^16 read one word into its low half.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PROB_BITS 16u
#define OR_M (1u << OR_PROB_BITS)
#define OR_L (1u << 16)
#define OR_NSYM 256
#define OR_HID 64
#define OR_CTX 4
#define OR_NCHAN 56

/* ---------------------------------------------------------------- rANS encode */

/* Encodes lanes [lane_lo, lane_hi) (lane_lo a multiple of 32) group by group.
 * Lane j's symbols sit at positions [lane_start[j], lane_start[j+1]) of f[] and c[],
 * which hold the frequency and cumulative frequency of each coded symbol.
 * Writes the groups' streams back to back into out (each padded with zero bytes to a
 * multiple of 16), grp_off[g] (byte offset of group g from out, n_groups+1 entries) and
 * grp_words[g] (words in group g, padding excluded).
 * Returns the bytes written, -1 if cap is too small, -2 on bad input.               */
int64_t or_rans_encode(int64_t lane_lo, int64_t lane_hi, const int64_t *lane_start,
                       const uint32_t *f, const uint32_t *c, uint8_t *out, int64_t cap,
                       uint64_t *grp_off, uint32_t *grp_words)
{
    if (lane_lo % 32 != 0 || lane_hi < lane_lo) return -2;
    int64_t pos = 0;
    int64_t g = 0;
    grp_off[0] = 0;
    for (int64_t j0 = lane_lo; j0 < lane_hi; j0 += 32, ++g) {
        int64_t j1 = j0 + 32 < lane_hi ? j0 + 32 : lane_hi;
        int nl = (int)(j1 - j0);
        int64_t maxn = 0, tot = 0;
        for (int64_t j = j0; j < j1; ++j) {
            int64_t n = lane_start[j + 1] - lane_start[j];
            if (n > maxn) maxn = n;
            tot += n;
        }
        /* at most one word per symbol, plus two per lane for the final state */
        uint16_t *w = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)(tot + 2 * nl + 1));
        if (!w) return -2;
        int64_t nw = 0;
        uint32_t x[32];
        for (int j = 0; j < nl; ++j) x[j] = OR_L;
        for (int64_t t = maxn - 1; t >= 0; --t) {
            for (int j = nl - 1; j >= 0; --j) {
                int64_t n = lane_start[j0 + j + 1] - lane_start[j0 + j];
                if (t >= n) continue;
                int64_t p = lane_start[j0 + j] + t;
                uint32_t fs = f[p], cs = c[p];
                if (fs == 0 || fs > OR_M || (uint64_t)cs + fs > OR_M) { free(w); return -2; }
                if ((uint64_t)x[j] >= ((uint64_t)fs << 16)) {
                    w[nw++] = (uint16_t)(x[j] & 0xFFFFu);
                    x[j] >>= 16;
                }
                x[j] = ((x[j] / fs) << OR_PROB_BITS) + (x[j] % fs) + cs;
            }
        }
        for (int j = nl - 1; j >= 0; --j) {
            w[nw++] = (uint16_t)(x[j] & 0xFFFFu);
            w[nw++] = (uint16_t)(x[j] >> 16);
        }
        int64_t bytes = 2 * nw;
        int64_t padded = (bytes + 15) / 16 * 16;
        if (pos + padded > cap) { free(w); return -1; }
        /* reverse: the decoder reads the last word pushed first */
        for (int64_t k = 0; k < nw; ++k) {
            uint16_t v = w[nw - 1 - k];
            out[pos + 2 * k] = (uint8_t)(v & 0xFF);
            out[pos + 2 * k + 1] = (uint8_t)(v >> 8);
        }
        memset(out + pos + bytes, 0, (size_t)(padded - bytes));
        grp_words[g] = (uint32_t)nw;
        pos += padded;
        grp_off[g + 1] = (uint64_t)pos;
        free(w);
    }
    return pos;
}

/* ---------------------------------------------------------------- rANS decode */

typedef struct {
    const uint8_t *base; /* group stream */
    int64_t n_words;     /* words in the group */
    int64_t next;        /* next word to read */
    int bad;
} or_reader;

static uint32_t or_read(or_reader *r)
{
    if (r->next >= r->n_words) { r->bad = 1; return 0; }
    const uint8_t *p = r->base + 2 * r->next;
    r->next++;
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8);
}

/* Symbol s with cum(s) <= slot < cum(s) + f(s), by a plain linear walk. */
static int or_find(const uint32_t *freq, uint32_t slot, uint32_t *f_out, uint32_t *c_out)
{
    uint32_t cum = 0;
    for (int s = 0; s < OR_NSYM; ++s) {
        if (slot < cum + freq[s]) { *f_out = freq[s]; *c_out = cum; return s; }
        cum += freq[s];
    }
    return -1;
}

static int or_group_setup(or_reader *r, uint32_t *x, int nl, const uint8_t *payload,
                          int64_t pay_len, uint64_t off, uint32_t n_words)
{
    if (off > (uint64_t)pay_len || (uint64_t)n_words * 2 > (uint64_t)pay_len - off) return -1;
    r->base = payload + off;
    r->n_words = n_words;
    r->next = 0;
    r->bad = 0;
    for (int j = 0; j < nl; ++j) {
        uint32_t hi = or_read(r), lo = or_read(r);
        x[j] = (hi << 16) | lo;
        if (x[j] < OR_L) r->bad = 1;
    }
    return r->bad ? -1 : 0;
}

static int or_group_finish(const or_reader *r, const uint32_t *x, int nl)
{
    if (r->bad || r->next != r->n_words) return -1;
    for (int j = 0; j < nl; ++j)
        if (x[j] != OR_L) return -1;
    return 0;
}

/* Decodes lanes [0, n_lanes) coded with static tables.  Symbol position p (lane-major, as
 * in the encoder) uses table tab_id[p] of freq[n_tab][256].  Writes syms[p].
 * Returns 0, or -1 if the stream is corrupt (bad state, overrun, or a failed end check). */
int or_rans_decode_static(int64_t n_lanes, const int64_t *lane_start, const uint8_t *tab_id,
                          const uint32_t *freq, int n_tab, const uint8_t *payload,
                          int64_t pay_len, const uint64_t *grp_off, const uint32_t *grp_words,
                          uint8_t *syms)
{
    int64_t g = 0;
    for (int64_t j0 = 0; j0 < n_lanes; j0 += 32, ++g) {
        int64_t j1 = j0 + 32 < n_lanes ? j0 + 32 : n_lanes;
        int nl = (int)(j1 - j0);
        or_reader r;
        uint32_t x[32];
        if (or_group_setup(&r, x, nl, payload, pay_len, grp_off[g], grp_words[g])) return -1;
        int64_t maxn = 0;
        for (int j = 0; j < nl; ++j) {
            int64_t n = lane_start[j0 + j + 1] - lane_start[j0 + j];
            if (n > maxn) maxn = n;
        }
        for (int64_t t = 0; t < maxn; ++t) {
            for (int j = 0; j < nl; ++j) {
                int64_t n = lane_start[j0 + j + 1] - lane_start[j0 + j];
                if (t >= n) continue;
                int64_t p = lane_start[j0 + j] + t;
                if (tab_id[p] >= n_tab) return -1;
                const uint32_t *tab = freq + (size_t)tab_id[p] * OR_NSYM;
                uint32_t slot = x[j] & (OR_M - 1), fs, cs;
                int s = or_find(tab, slot, &fs, &cs);
                if (s < 0) return -1;
                syms[p] = (uint8_t)s;
                x[j] = fs * (x[j] >> OR_PROB_BITS) + slot - cs;
                if (x[j] < OR_L) x[j] = (x[j] << 16) | or_read(&r);
            }
            if (r.bad) return -1;
        }
        if (or_group_finish(&r, x, nl)) return -1;
    }
    return 0;
}

/* As or_rans_decode_static with 16-bit table ids (the context tables of a learned octree
 * level: one table per distinct (parent byte, child index)). */
int or_rans_decode_static16(int64_t n_lanes, const int64_t *lane_start, const uint16_t *tab_id,
                          const uint32_t *freq, int n_tab, const uint8_t *payload,
                          int64_t pay_len, const uint64_t *grp_off, const uint32_t *grp_words,
                          uint8_t *syms)
{
    int64_t g = 0;
    for (int64_t j0 = 0; j0 < n_lanes; j0 += 32, ++g) {
        int64_t j1 = j0 + 32 < n_lanes ? j0 + 32 : n_lanes;
        int nl = (int)(j1 - j0);
        or_reader r;
        uint32_t x[32];
        if (or_group_setup(&r, x, nl, payload, pay_len, grp_off[g], grp_words[g])) return -1;
        int64_t maxn = 0;
        for (int j = 0; j < nl; ++j) {
            int64_t n = lane_start[j0 + j + 1] - lane_start[j0 + j];
            if (n > maxn) maxn = n;
        }
        for (int64_t t = 0; t < maxn; ++t) {
            for (int j = 0; j < nl; ++j) {
                int64_t n = lane_start[j0 + j + 1] - lane_start[j0 + j];
                if (t >= n) continue;
                int64_t p = lane_start[j0 + j] + t;
                if (tab_id[p] >= n_tab) return -1;
                const uint32_t *tab = freq + (size_t)tab_id[p] * OR_NSYM;
                uint32_t slot = x[j] & (OR_M - 1), fs, cs;
                int s = or_find(tab, slot, &fs, &cs);
                if (s < 0) return -1;
                syms[p] = (uint8_t)s;
                x[j] = fs * (x[j] >> OR_PROB_BITS) + slot - cs;
                if (x[j] < OR_L) x[j] = (x[j] << 16) | or_read(&r);
            }
            if (r.bad) return -1;
        }
        if (or_group_finish(&r, x, nl)) return -1;
    }
    return 0;
}

/* ------------------------------------------------- integer context model (learned) */

typedef struct {
    int8_t w1[OR_HID * OR_CTX];       /* [64][4] */
    int32_t b1[OR_NCHAN * OR_HID];    /* [56][64], channel embedding folded in */
    int32_t m1, sh1;
    int8_t w2[OR_HID * OR_HID];       /* [64][64] */
    int32_t b2[OR_HID];
    int32_t m2, sh2;
    int8_t w3[OR_NSYM * OR_HID];      /* [256][64] */
    int32_t b3[OR_NSYM];
    uint32_t ms, ss;                  /* logit-gap multiplier and shift */
} or_model;

int or_model_size(void) { return (int)sizeof(or_model); }

/* h = clamp((acc * m + 2^(sh-1)) >> sh, 0, 127) in 64-bit arithmetic (ReLU = clamp at 0) */
static int32_t or_requant(int32_t acc, int32_t m, int32_t sh)
{
    int64_t v = ((int64_t)acc * (int64_t)m + ((int64_t)1 << (sh - 1))) >> sh;
    if (v < 0) v = 0;
    if (v > 127) v = 127;
    return (int32_t)v;
}

/* Logits z[256] of channel c given context u[4] (u_j = s_{i-j} - 128, or 0 past the lane start). */
void or_model_logits(const or_model *M, const int32_t *u, int c, int32_t *z)
{
    int32_t h1[OR_HID], h2[OR_HID];
    for (int o = 0; o < OR_HID; ++o) {
        int32_t acc = M->b1[c * OR_HID + o];
        for (int j = 0; j < OR_CTX; ++j) acc += (int32_t)M->w1[o * OR_CTX + j] * u[j];
        h1[o] = or_requant(acc, M->m1, M->sh1);
    }
    for (int o = 0; o < OR_HID; ++o) {
        int32_t acc = M->b2[o];
        for (int k = 0; k < OR_HID; ++k) acc += (int32_t)M->w2[o * OR_HID + k] * h1[k];
        h2[o] = or_requant(acc, M->m2, M->sh2);
    }
    for (int s = 0; s < OR_NSYM; ++s) {
        int32_t acc = M->b3[s];
        for (int k = 0; k < OR_HID; ++k) acc += (int32_t)M->w3[s * OR_HID + k] * h2[k];
        z[s] = acc;
    }
}

/* Integer softmax -> frequencies summing to exactly 2^16, each >= 1.
 * exp2q[f] = round(2^(23 - f/256)), f = 0..255.                                       */
void or_logits_to_freq(const int32_t *z, uint32_t ms, uint32_t ss, const uint32_t *exp2q,
                       uint32_t *freq)
{
    int32_t zmax = z[0];
    int amax = 0;
    for (int k = 1; k < OR_NSYM; ++k)
        if (z[k] > zmax) { zmax = z[k]; amax = k; }
    uint32_t e[OR_NSYM];
    uint64_t E = 0;
    for (int k = 0; k < OR_NSYM; ++k) {
        uint64_t d = (uint64_t)((int64_t)zmax - (int64_t)z[k]);
        uint64_t t = (d * (uint64_t)ms) >> ss;
        if (t > 6144) t = 6144;
        e[k] = exp2q[t & 255] >> (t >> 8);
        E += e[k];
    }
    uint64_t R = ((uint64_t)(OR_M - OR_NSYM) << 32) / E;
    uint64_t sum = 0;
    for (int k = 0; k < OR_NSYM; ++k) {
        freq[k] = 1u + (uint32_t)(((uint64_t)e[k] * R) >> 32);
        sum += freq[k];
    }
    freq[amax] += (uint32_t)(OR_M - sum);
}

static void or_context(const uint8_t *syms, int64_t row, int64_t row0, int c, int32_t *u)
{
    for (int j = 1; j <= OR_CTX; ++j) {
        int64_t r = row - j;
        u[j - 1] = (r >= row0) ? (int32_t)syms[r * OR_NCHAN + c] - 128 : 0;
    }
}

/* Frequency table of symbol (row, c) of a lane that starts at row0; syms row-major [rows][56]. */
void or_learned_freq(const or_model *M, const uint32_t *exp2q, const uint8_t *syms,
                     int64_t row, int64_t row0, int c, uint32_t *freq)
{
    int32_t u[OR_CTX], z[OR_NSYM];
    or_context(syms, row, row0, c, u);
    or_model_logits(M, u, c, z);
    or_logits_to_freq(z, M->ms, M->ss, exp2q, freq);
}

/* Encoder helper: f and cum of every symbol of lanes [lane_lo, lane_hi), written lane-major
 * from index 0 (lane lane_lo first).  lane_row[j] = first row of lane j (n_lanes+1 entries). */
void or_learned_fc(const or_model *M, const uint32_t *exp2q, const uint8_t *syms,
                   const int64_t *lane_row, int64_t lane_lo, int64_t lane_hi,
                   uint32_t *f, uint32_t *cum)
{
    uint32_t freq[OR_NSYM];
    int64_t p = 0;
    for (int64_t j = lane_lo; j < lane_hi; ++j) {
        for (int64_t i = lane_row[j]; i < lane_row[j + 1]; ++i) {
            for (int c = 0; c < OR_NCHAN; ++c) {
                or_learned_freq(M, exp2q, syms, i, lane_row[j], c, freq);
                uint8_t s = syms[i * OR_NCHAN + c];
                uint32_t cc = 0;
                for (int k = 0; k < s; ++k) cc += freq[k];
                f[p] = freq[s];
                cum[p] = cc;
                ++p;
            }
        }
    }
}

/* Learned decoder for lanes [lane_lo, lane_hi) (lane_lo a multiple of 32).  grp_off and
 * grp_words are indexed from group lane_lo/32.  Writes syms row-major [rows][56] (only the
 * rows of the decoded lanes).  Returns 0 or -1 (corrupt).                              */
int or_rans_decode_learned(const or_model *M, const uint32_t *exp2q, const int64_t *lane_row,
                           int64_t lane_lo, int64_t lane_hi, const uint8_t *payload,
                           int64_t pay_len, const uint64_t *grp_off, const uint32_t *grp_words,
                           uint8_t *syms)
{
    if (lane_lo % 32 != 0) return -1;
    uint32_t freq[OR_NSYM];
    int64_t g = lane_lo / 32;
    for (int64_t j0 = lane_lo; j0 < lane_hi; j0 += 32, ++g) {
        int64_t j1 = j0 + 32 < lane_hi ? j0 + 32 : lane_hi;
        int nl = (int)(j1 - j0);
        or_reader r;
        uint32_t x[32];
        if (or_group_setup(&r, x, nl, payload, pay_len, grp_off[g], grp_words[g])) return -1;
        int64_t maxn = 0;
        for (int j = 0; j < nl; ++j) {
            int64_t n = (lane_row[j0 + j + 1] - lane_row[j0 + j]) * OR_NCHAN;
            if (n > maxn) maxn = n;
        }
        for (int64_t t = 0; t < maxn; ++t) {
            for (int j = 0; j < nl; ++j) {
                int64_t row0 = lane_row[j0 + j];
                int64_t n = (lane_row[j0 + j + 1] - row0) * OR_NCHAN;
                if (t >= n) continue;
                int64_t row = row0 + t / OR_NCHAN;
                int c = (int)(t % OR_NCHAN);
                or_learned_freq(M, exp2q, syms, row, row0, c, freq);
                uint32_t slot = x[j] & (OR_M - 1), fs, cs;
                int s = or_find(freq, slot, &fs, &cs);
                if (s < 0) return -1;
                syms[row * OR_NCHAN + c] = (uint8_t)s;
                x[j] = fs * (x[j] >> OR_PROB_BITS) + slot - cs;
                if (x[j] < OR_L) x[j] = (x[j] << 16) | or_read(&r);
            }
            if (r.bad) return -1;
        }
        if (or_group_finish(&r, x, nl)) return -1;
    }
    return 0;
}

/* Integer forward of layers 1-2 for calibration: returns max acc1 and max acc2 over the
 * samples (rows[k], chans[k]) of syms (lane starts given per sample in row0s[k]).      */
void or_calib_max(const int8_t *w1, const int32_t *b1, int32_t m1, int32_t sh1,
                  const int8_t *w2, const int32_t *b2, const uint8_t *syms,
                  const int64_t *rows, const int64_t *row0s, const int32_t *chans, int64_t n,
                  int64_t *max1, int64_t *max2)
{
    int64_t a1max = INT64_MIN, a2max = INT64_MIN;
    for (int64_t k = 0; k < n; ++k) {
        int32_t u[OR_CTX], h1[OR_HID];
        int c = chans[k];
        or_context(syms, rows[k], row0s[k], c, u);
        for (int o = 0; o < OR_HID; ++o) {
            int32_t acc = b1[c * OR_HID + o];
            for (int j = 0; j < OR_CTX; ++j) acc += (int32_t)w1[o * OR_CTX + j] * u[j];
            if (acc > a1max) a1max = acc;
            h1[o] = (m1 > 0) ? or_requant(acc, m1, sh1) : 0;
        }
        if (m1 > 0) {
            for (int o = 0; o < OR_HID; ++o) {
                int32_t acc = b2[o];
                for (int q = 0; q < OR_HID; ++q) acc += (int32_t)w2[o * OR_HID + q] * h1[q];
                if (acc > a2max) a2max = acc;
            }
        }
    }
    *max1 = a1max;
    *max2 = a2max;
}

/* ---------------------------------------------------------------- position-aware model */

#define OR_NPHI 75
#define OR_KIN 80
#define OR_BANDS 12

typedef struct {
    float s1, s2, smu, slr;           /* requant scales and head multipliers */
    int32_t b1[OR_NCHAN * OR_HID];    /* [56][64], embedding and projection bias folded in */
    int32_t b2[OR_HID];
    int32_t b3[2];
    int8_t w1[OR_HID * OR_KIN];       /* [64][80]: u (4), phi (75), 0 */
    int8_t w2[OR_HID * OR_HID];
    int8_t w3[2 * OR_HID];
} or_pe_model;

int or_pe_model_size(void) { return (int)sizeof(or_pe_model); }

/* Embedding inputs of a voxel v (3 coordinates) at depth D: floor(128 mu) per axis, then
 * for band k the sines and then the cosines of 2 pi 2^k mu on a 256-step phase grid. */
void or_pe_phi(const uint32_t *v, int depth, const int8_t *sin8, int32_t *phi)
{
    for (int a = 0; a < 3; ++a) {
        uint64_t two = 2ull * v[a] + 1ull;
        phi[a] = (int32_t)((two << 6) >> depth);
        for (int k = 0; k < OR_BANDS; ++k) {
            uint32_t th = (uint32_t)(((two << (k + 8)) >> (depth + 1)) & 255u);
            phi[3 + 3 * k + a] = sin8[th];
            phi[3 + 3 * OR_BANDS + 3 * k + a] = sin8[(th + 64u) & 255u];
        }
    }
}

static int32_t or_rq_f32(int32_t acc, float s)
{
    float v = rintf((float)acc * s);
    if (v < 0.0f) v = 0.0f;
    if (v > 127.0f) v = 127.0f;
    return (int32_t)v;
}

/* Head parameters (mean in 1/256 symbol, n = 4096 + log2-rate in 1/256) of channel c. */
void or_pe_head(const or_pe_model *M, const int32_t *u, int c, const int32_t *phi,
                int32_t *mu8, int32_t *n)
{
    int32_t x[OR_KIN], h1[OR_HID], h2[OR_HID];
    for (int j = 0; j < OR_CTX; ++j) x[j] = u[j];
    for (int k = 0; k < OR_NPHI; ++k) x[OR_CTX + k] = phi[k];
    x[OR_KIN - 1] = 0;
    for (int o = 0; o < OR_HID; ++o) {
        int32_t acc = M->b1[c * OR_HID + o];
        for (int k = 0; k < OR_KIN; ++k) acc += (int32_t)M->w1[o * OR_KIN + k] * x[k];
        h1[o] = or_rq_f32(acc, M->s1);
    }
    for (int o = 0; o < OR_HID; ++o) {
        int32_t acc = M->b2[o];
        for (int k = 0; k < OR_HID; ++k) acc += (int32_t)M->w2[o * OR_HID + k] * h1[k];
        h2[o] = or_rq_f32(acc, M->s2);
    }
    int32_t z[2];
    for (int o = 0; o < 2; ++o) {
        int32_t acc = M->b3[o];
        for (int k = 0; k < OR_HID; ++k) acc += (int32_t)M->w3[o * OR_HID + k] * h2[k];
        z[o] = acc;
    }
    float vm = rintf((float)z[0] * M->smu);
    if (vm < -32640.0f) vm = -32640.0f;
    if (vm > 32640.0f) vm = 32640.0f;
    float vl = rintf((float)z[1] * M->slr);
    if (vl < -2048.0f) vl = -2048.0f;
    if (vl > 1536.0f) vl = 1536.0f;
    *mu8 = 32640 + (int32_t)vm;
    *n = 4096 + (int32_t)vl;
}

/* Cumulative count below symbol s (0..256) of the integer Laplace with (mu8, n). */
uint32_t or_pe_cdf(int32_t mu8, int32_t n, int s, const uint32_t *exp2q)
{
    if (s <= 0) return 0;
    if (s >= OR_NSYM) return OR_M;
    int q = (n + 255) >> 8;
    uint64_t R = exp2q[(uint32_t)(-n) & 255u] >> (23 - q);
    int64_t d = 256 * (int64_t)s - 128 - mu8;
    uint64_t ad = (uint64_t)(d < 0 ? -d : d);
    uint64_t t = (ad * R) >> 16;
    if (t > 6144) t = 6144;
    uint64_t e = exp2q[t & 255] >> (t >> 8);
    uint64_t F = d < 0 ? (e >> 1) : ((1ull << 23) - (e >> 1));
    return (uint32_t)s + (uint32_t)((F * 65280ull) >> 23);
}

/* Decodes lanes [lane_lo, lane_hi) (lane_lo a multiple of 32) coded with the position-aware
 * model: the stream order and the group format are those of the plain learned decoder; token (row, c) is found by walking
 * the CDF upwards from symbol 0.  coord: uint32 [3][n_rows] voxel coordinates of the rows. */
int or_rans_decode_pe(const or_pe_model *M, const uint32_t *exp2q, const int8_t *sin8,
                      const uint32_t *coord, int64_t n_rows, int depth, const int64_t *lane_row,
                      int64_t lane_lo, int64_t lane_hi, const uint8_t *payload, int64_t pay_len,
                      const uint64_t *grp_off, const uint32_t *grp_words, uint8_t *syms)
{
    if (lane_lo % 32 != 0) return -1;
    int64_t g = lane_lo / 32;
    for (int64_t j0 = lane_lo; j0 < lane_hi; j0 += 32, ++g) {
        int64_t j1 = j0 + 32 < lane_hi ? j0 + 32 : lane_hi;
        int nl = (int)(j1 - j0);
        or_reader r;
        uint32_t x[32];
        if (or_group_setup(&r, x, nl, payload, pay_len, grp_off[g], grp_words[g])) return -1;
        int64_t maxn = 0;
        for (int j = 0; j < nl; ++j) {
            int64_t n = (lane_row[j0 + j + 1] - lane_row[j0 + j]) * OR_NCHAN;
            if (n > maxn) maxn = n;
        }
        for (int64_t t = 0; t < maxn; ++t) {
            for (int j = 0; j < nl; ++j) {
                int64_t row0 = lane_row[j0 + j];
                int64_t n = (lane_row[j0 + j + 1] - row0) * OR_NCHAN;
                if (t >= n) continue;
                int64_t row = row0 + t / OR_NCHAN;
                int c = (int)(t % OR_NCHAN);
                int32_t u[OR_CTX], phi[OR_NPHI], mu8, nn;
                uint32_t v[3] = {coord[row], coord[n_rows + row], coord[2 * n_rows + row]};
                or_context(syms, row, row0, c, u);
                or_pe_phi(v, depth, sin8, phi);
                or_pe_head(M, u, c, phi, &mu8, &nn);
                uint32_t slot = x[j] & (OR_M - 1);
                int s = 0;
                while (s < OR_NSYM - 1 && or_pe_cdf(mu8, nn, s + 1, exp2q) <= slot) ++s;
                uint32_t cs = or_pe_cdf(mu8, nn, s, exp2q);
                uint32_t fs = or_pe_cdf(mu8, nn, s + 1, exp2q) - cs;
                syms[row * OR_NCHAN + c] = (uint8_t)s;
                x[j] = fs * (x[j] >> OR_PROB_BITS) + slot - cs;
                if (x[j] < OR_L) x[j] = (x[j] << 16) | or_read(&r);
            }
            if (r.bad) return -1;
        }
        if (or_group_finish(&r, x, nl)) return -1;
    }
    return 0;
}
