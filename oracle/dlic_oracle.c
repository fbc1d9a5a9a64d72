/*
 * DLIC coding oracle: test infrastructure, not part of the library.
 *
 * A plain, slow, sequential CPU restatement of the coding method of
 * "Accelerated Deep Lossless Image Coding with Unified Parallelized GPU Coding
 * Architecture" (Barzen et al.), written from the paper's description:
 *   - Eq. 1 / Sec. II-A: a network estimates P(x_i | causal neighbours);
 *   - Sec. II-A, Fig. 1 and 2: the neighbourhood window holds only already
 *     decoded pixels; pixels outside the image take a dummy value;
 *   - Sec. II-B "Preprocessor": wavefront processing, identical network inputs
 *     at encode and decode;
 *   - Sec. II-B "Neural Network Architecture": dense layers, 256-way softmax;
 *   - Sec. IV "Higher Bit Depth": 12-bit pixels, 4096 output neurons;
 *   - Sec. II-B "rANS": rANS coder, many coder instances and bitstreams, at
 *     most one per pixel row, 32-bit arithmetic.
 * Where the paper is silent (window radius, dummy value, table quantisation,
 * rANS constants, stream assignment, container layout) this file follows the
 * readings written down beside each function.
 *
 * Only the test-suite, the smoke check and the bench's CPU-baseline leg load
 * this file.  It shares no code with the CUDA library.  Floating point is
 * IEEE single precision with every operation written out (fmaf, one rounding
 * per operation; build with -ffp-contract=off), so that the order of every
 * rounding is the one stated here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_INVALID 1
#define OR_ERR_CAPACITY 2
#define OR_ERR_CORRUPT 3

#define NPRI 12           /* priors of the default radius-2 window */
#define MAXPRI 96         /* largest window the coder takes */
#define NSYM 256            /* symbols of an 8-bit image */
#define NSYM_MAX 4096       /* symbols of a 12-bit image (Sec. IV "Higher Bit Depth") */
#define TOTAL_M 65536u      /* frequency table total, 2^16 */
#define RANS_L 65536u       /* rANS lower bound, 2^16 */

/* ------------------------------------------------------------------ */
/* Model blob (little-endian; layout fixed in the model format)        */
/* ------------------------------------------------------------------ */

/* Causal window: rows r-u .. r-1 at columns c-l .. c+r, then row r at
 * columns c-l .. c-1 (n2 = u (l + r + 1) + l priors, in that order).  A 3D
 * window (Sec. IV "3D Dependencies": two layers, the lower one may reach
 * below the target's row) adds, from the previous slice, rows r-pu .. r+pd
 * at columns c-pl .. c+pr, row by row, left to right: n = n2 + n3 priors,
 * n3 = (pu + pd + 1)(pl + pr + 1). */
typedef struct { int u, l, r, n2, pu, pd, pl, pr, n3, n, vol; } window_t;

#define MAXLAYERS 9            /* up to 8 hidden layers and the output layer */

typedef struct {
    int precision;               /* 0 = FP32, 1 = INT8 */
    window_t win;
    int h1, h2;
    int nl;                      /* dense layers: hidden layers + the output layer */
    int nsym, bits;              /* output neurons = symbols: 256 (8-bit) or 4096 (12-bit) */
    float tscale;
    uint32_t lut[64];
    float *w[MAXLAYERS], *b[MAXLAYERS];   /* FP32 network: W[l] is out x in, row-major */
    int8_t *q[MAXLAYERS];                 /* INT8 network weights, out x in */
    float *s[MAXLAYERS], *o[MAXLAYERS];   /* INT8 per-output scale and offset */
    int n_in[MAXLAYERS], n_out[MAXLAYERS];
    uint64_t hash;
} model_t;

static uint32_t rd_u32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

static float rd_f32(const uint8_t *p) {
    uint32_t u = rd_u32(p);
    float f;
    memcpy(&f, &u, 4);
    return f;
}

/* FNV-1a, 64-bit (Fowler, Noll, Vo): the model identity kept in bitstreams. */
uint64_t or_fnv1a64(const uint8_t *p, size_t n) {
    uint64_t h = 0xCBF29CE484222325ull;
    for (size_t i = 0; i < n; i++) {
        h ^= p[i];
        h *= 0x100000001B3ull;
    }
    return h;
}

static void model_free(model_t *m) {
    for (int l = 0; l < MAXLAYERS; l++) {
        free(m->w[l]); free(m->b[l]); free(m->q[l]); free(m->s[l]); free(m->o[l]);
    }
}

/* Two layouts (little-endian):
 *   "DLM1": u32 precision, n_in, h1, h2, n_out (256, or 4096 for 12-bit
 *           pixels), window, f32 tscale,
 *           u32 lut[64], then 3 dense layers (288-byte header);
 *   "DLM2" (deeper networks, Sec. II-B: six dense layers): u32 precision,
 *           n_in, L (hidden layers, 1..8), widths[8] (hidden widths, unused
 *           entries 0), n_out (256), window, f32 tscale, u32 0, u32 lut[64],
 *           then L + 1 dense layers (320-byte header).
 * Each dense layer: FP32 W f32[out][in], b f32[out]; INT8 W i8[out][in],
 * s f32[out], o f32[out]. */
static int model_load(model_t *m, const uint8_t *blob, size_t n) {
    memset(m, 0, sizeof(*m));
    int deep = 0;
    uint32_t widths[MAXLAYERS] = {0};
    if (n >= 320 && memcmp(blob, "DLM2", 4) == 0) {
        deep = 1;
    } else if (n < 288 || memcmp(blob, "DLM1", 4) != 0) {
        return OR_ERR_INVALID;
    }
    m->precision = (int)rd_u32(blob + 4);
    uint32_t n_in = rd_u32(blob + 8), h1, h2, n_out, radius;
    const uint8_t *pre;   /* tscale, then (after any padding) the lut */
    if (deep) {
        uint32_t L = rd_u32(blob + 12);
        if (L < 1 || L > MAXLAYERS - 1) return OR_ERR_INVALID;
        for (uint32_t l = 0; l < 8; l++) {
            widths[l] = rd_u32(blob + 16 + 4 * l);
            if ((l < L) != (widths[l] != 0)) return OR_ERR_INVALID;
            if (l < L && widths[l] > 4096) return OR_ERR_INVALID;
        }
        m->nl = (int)L + 1;
        n_out = rd_u32(blob + 48);
        radius = rd_u32(blob + 52);
        h1 = widths[0];
        h2 = widths[L - 1];
        pre = blob + 56;
    } else {
        h1 = rd_u32(blob + 12);
        h2 = rd_u32(blob + 16);
        n_out = rd_u32(blob + 20);
        radius = rd_u32(blob + 24);
        widths[0] = h1;
        widths[1] = h2;
        m->nl = 3;
        pre = blob + 28;
    }
    if (m->precision != 0 && m->precision != 1) return OR_ERR_INVALID;
    /* window field: 2 = the default radius-2 window; otherwise
     * 1 << 24 | u | l << 8 | r << 16 with 1 <= u <= 8, l <= 8 and r <= 2
     * (a right reach of at most 2 keeps every prior on an earlier wave of
     * t = 3 row + column).
     * A 3D window: 2 << 28 | u | l << 4 | r << 8 | pu << 10 | pd << 14 |
     * pl << 18 | pr << 22 (4 bits each, r 2 bits), pu, pd, pl, pr <= 8. */
    if (radius == 2) {
        m->win.u = 2; m->win.l = 2; m->win.r = 2;
    } else if ((radius >> 24) == 1) {
        m->win.u = (int)(radius & 0xFF); m->win.l = (int)((radius >> 8) & 0xFF); m->win.r = (int)((radius >> 16) & 0xFF);
    } else if ((radius >> 28) == 2 && ((radius >> 26) & 3) == 0) {
        m->win.u = (int)(radius & 0xF); m->win.l = (int)((radius >> 4) & 0xF); m->win.r = (int)((radius >> 8) & 3);
        m->win.pu = (int)((radius >> 10) & 0xF); m->win.pd = (int)((radius >> 14) & 0xF);
        m->win.pl = (int)((radius >> 18) & 0xF); m->win.pr = (int)((radius >> 22) & 0xF);
        if (m->win.pu > 8 || m->win.pd > 8 || m->win.pl > 8 || m->win.pr > 8) return OR_ERR_INVALID;
        m->win.vol = 1;
        m->win.n3 = (m->win.pu + m->win.pd + 1) * (m->win.pl + m->win.pr + 1);
    } else {
        return OR_ERR_INVALID;
    }
    if (m->win.u < 1 || m->win.u > 8 || m->win.l > 8 || m->win.r > 2) return OR_ERR_INVALID;
    m->win.n2 = m->win.u * (m->win.l + m->win.r + 1) + m->win.l;
    m->win.n = m->win.n2 + m->win.n3;
    /* 256 outputs code 8-bit pixels; 4096 outputs 12-bit pixels (Sec. IV
     * "Higher Bit Depth"), with the FP32 network only (an INT8 input byte
     * cannot hold a 12-bit prior) */
    if (m->win.n > MAXPRI || (int)n_in != m->win.n || (n_out != NSYM && n_out != NSYM_MAX)) return OR_ERR_INVALID;
    if (n_out == NSYM_MAX && m->precision != 0) return OR_ERR_INVALID;
    m->nsym = (int)n_out;
    m->bits = n_out == NSYM_MAX ? 12 : 8;
    if (h1 < 1 || h1 > 4096 || h2 < 1 || h2 > 4096) return OR_ERR_INVALID;
    m->h1 = (int)h1; m->h2 = (int)h2;
    m->tscale = rd_f32(pre);
    if (!(m->tscale > 0.0f)) return OR_ERR_INVALID;
    const uint8_t *lutp = deep ? blob + 64 : blob + 32;
    for (int k = 0; k < 64; k++) {
        m->lut[k] = rd_u32(lutp + 4 * k);
        if (m->lut[k] > (1u << 23)) return OR_ERR_INVALID;
    }
    if (m->lut[0] != (1u << 23)) return OR_ERR_INVALID;
    int dims_in[MAXLAYERS], dims_out[MAXLAYERS];
    for (int l = 0; l < m->nl; l++) {
        dims_in[l] = l == 0 ? m->win.n : (int)widths[l - 1];
        dims_out[l] = l == m->nl - 1 ? m->nsym : (int)widths[l];
    }
    size_t need = deep ? 320 : 288;
    for (int l = 0; l < m->nl; l++) {
        size_t wn = (size_t)dims_in[l] * dims_out[l];
        need += m->precision == 0 ? 4 * wn + 4 * (size_t)dims_out[l] : wn + 8 * (size_t)dims_out[l];
    }
    if (need != n) return OR_ERR_INVALID;
    const uint8_t *p = blob + (deep ? 320 : 288);
    for (int l = 0; l < m->nl; l++) {
        int ni = dims_in[l], no = dims_out[l];
        m->n_in[l] = ni; m->n_out[l] = no;
        size_t wn = (size_t)ni * no;
        if (m->precision == 0) {
            m->w[l] = malloc(4 * wn); m->b[l] = malloc(4 * (size_t)no);
            for (size_t i = 0; i < wn; i++) m->w[l][i] = rd_f32(p + 4 * i);
            p += 4 * wn;
            for (int i = 0; i < no; i++) m->b[l][i] = rd_f32(p + 4 * i);
            p += 4 * (size_t)no;
        } else {
            m->q[l] = malloc(wn); m->s[l] = malloc(4 * (size_t)no); m->o[l] = malloc(4 * (size_t)no);
            memcpy(m->q[l], p, wn);
            p += wn;
            for (int i = 0; i < no; i++) m->s[l][i] = rd_f32(p + 4 * i);
            p += 4 * (size_t)no;
            for (int i = 0; i < no; i++) m->o[l][i] = rd_f32(p + 4 * i);
            p += 4 * (size_t)no;
        }
    }
    m->hash = or_fnv1a64(blob, n);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Causal prior gather (Sec. II-A, Fig. 1 left; dummy value per Fig. 1 */
/* right; "any window shape", Sec. II-A, e.g. the 9x9 window of Fig. 6 */
/* with the target in the last row, third column from the right).       */
/* Reading: rows r-u..r-1 at columns c-l..c+r, then row r at columns    */
/* c-l..c-1, row by row, left to right; pixels outside the image read   */
/* as 0.  The default window (u, l, r) = (2, 2, 2) gives the 12 priors  */
/*   row r-2: c-2..c+2, row r-1: c-2..c+2, row r: c-2, c-1.            */
/* ------------------------------------------------------------------ */

/* Pixel i of an image of 8-bit (u8) or 12-bit (u16) samples. */
static uint32_t px_at(const void *img, int bits, size_t i) {
    return bits == 12 ? ((const uint16_t *)img)[i] : ((const uint8_t *)img)[i];
}

static void gather_win(const window_t *w, const void *img, int bits, int H, int W, int r, int c, uint16_t *pri) {
    const int wid = w->l + w->r + 1;
    for (int k = 0; k < w->n2; k++) {
        int dr, dc;
        if (k < w->u * wid) {
            dr = -w->u + k / wid;
            dc = -w->l + k % wid;
        } else {
            dr = 0;
            dc = -w->l + (k - w->u * wid);
        }
        int rr = r + dr, cc = c + dc;
        pri[k] = (uint16_t)((rr >= 0 && rr < H && cc >= 0 && cc < W) ? px_at(img, bits, (size_t)rr * W + cc) : 0);
    }
}

/* A 3D window at (r, c) of a slice: the slice's own window, then the lower
 * layer from `below` (the previous slice, H x W), or zeros for the first
 * slice (below == NULL). */
static void gather_win3(const window_t *w, const void *below, const void *img, int bits, int H, int W, int r,
                        int c, uint16_t *pri) {
    gather_win(w, img, bits, H, W, r, c, pri);
    const int wid = w->pl + w->pr + 1;
    for (int k = 0; k < w->n3; k++) {
        int rr = r - w->pu + k / wid, cc = c - w->pl + k % wid;
        pri[w->n2 + k] =
            (uint16_t)((below && rr >= 0 && rr < H && cc >= 0 && cc < W) ? px_at(below, bits, (size_t)rr * W + cc) : 0);
    }
}

void or_gather(const uint8_t *img, int H, int W, int r, int c, uint8_t pri[NPRI]) {
    const window_t w = {2, 2, 2, NPRI, 0, 0, 0, 0, 0, NPRI, 0};
    uint16_t p16[NPRI];
    gather_win(&w, img, 8, H, W, r, c, p16);
    for (int k = 0; k < NPRI; k++) pri[k] = (uint8_t)p16[k];
}

/* The priors of window (u, l, r) at pixel (r0, c0); returns their count. */
int or_gather_window(int u, int l, int rr, const uint8_t *img, int H, int W, int r0, int c0, uint8_t *pri) {
    const int n2 = u * (l + rr + 1) + l;
    const window_t w = {u, l, rr, n2, 0, 0, 0, 0, 0, n2, 0};
    uint16_t p16[MAXPRI];
    if (n2 > MAXPRI) return -1;
    gather_win(&w, img, 8, H, W, r0, c0, p16);
    for (int k = 0; k < w.n; k++) pri[k] = (uint8_t)p16[k];
    return w.n;
}

/* The priors of a 3D window at (r0, c0) of a slice with the previous slice
 * `below` (NULL for the first slice); returns their count. */
int or_gather_window3(int u, int l, int rr, int pu, int pd, int pl, int pr, const uint8_t *below, const uint8_t *img,
                      int H, int W, int r0, int c0, uint8_t *pri) {
    const int n2 = u * (l + rr + 1) + l, n3 = (pu + pd + 1) * (pl + pr + 1);
    const window_t w = {u, l, rr, n2, pu, pd, pl, pr, n3, n2 + n3, 1};
    uint16_t p16[MAXPRI];
    if (n2 + n3 > MAXPRI) return -1;
    gather_win3(&w, below, img, 8, H, W, r0, c0, p16);
    for (int k = 0; k < w.n; k++) pri[k] = (uint8_t)p16[k];
    return w.n;
}

/* ------------------------------------------------------------------ */
/* Density-estimation network (Sec. II-B).                              */
/* FP32 reading: input v/128 - 1 (8-bit) or v/2048 - 1 (12-bit), exact; */
/* each unit starts from its bias and                                   */
/* accumulates fma(x_k, w_jk, acc) for k = 0, 1, ... in order; ReLU on  */
/* hidden units.                                                        */
/* INT8 reading: input v - 128, exact integer dot products, hidden      */
/* units clamp(rint(fma(acc, s_j, o_j)), 0, 255), logits               */
/* fma(acc, s_j, o_j).                                                  */
/* ------------------------------------------------------------------ */

static void mlp_fp32(const model_t *m, const uint16_t *pri, float *z) {
    float a[4096], b[4096];
    const float scale = m->bits == 12 ? 0.00048828125f : 0.0078125f;   /* 2^-11 or 2^-7 */
    for (int k = 0; k < m->win.n; k++) a[k] = fmaf((float)pri[k], scale, -1.0f);
    float *in = a, *out = b;
    for (int l = 0; l < m->nl; l++) {
        int ni = m->n_in[l], no = m->n_out[l];
        for (int j = 0; j < no; j++) {
            float acc = m->b[l][j];
            for (int k = 0; k < ni; k++) acc = fmaf(in[k], m->w[l][(size_t)j * ni + k], acc);
            if (l < m->nl - 1) acc = acc > 0.0f ? acc : 0.0f;
            out[j] = acc;
        }
        float *t = in; in = out; out = t;
    }
    for (int i = 0; i < m->nsym; i++) z[i] = in[i];
}

static float requant_u8(int32_t acc, float s, float o) {
    float t = rintf(fmaf((float)acc, s, o));
    if (t < 0.0f) t = 0.0f;
    if (t > 255.0f) t = 255.0f;
    return t;
}

static void mlp_int8(const model_t *m, const uint16_t *pri, float *z) {
    int32_t a[4096], b[4096];
    for (int k = 0; k < m->win.n; k++) a[k] = (int32_t)pri[k] - 128;
    int32_t *in = a, *out = b;
    for (int l = 0; l < m->nl; l++) {
        int ni = m->n_in[l], no = m->n_out[l];
        for (int j = 0; j < no; j++) {
            int32_t acc = 0;
            for (int k = 0; k < ni; k++) acc += (int32_t)m->q[l][(size_t)j * ni + k] * in[k];
            if (l < m->nl - 1)
                out[j] = (int32_t)requant_u8(acc, m->s[l][j], m->o[l][j]);
            else
                z[j] = fmaf((float)acc, m->s[l][j], m->o[l][j]);
        }
        int32_t *t = in; in = out; out = t;
    }
}

static void mlp(const model_t *m, const uint16_t *pri, float *z) {
    if (m->precision == 0) mlp_fp32(m, pri, z);
    else mlp_int8(m, pri, z);
}

/* ------------------------------------------------------------------ */
/* PDF -> integer frequency table.  The paper codes each pixel with the */
/* network's softmax PDF (Sec. II-B) and leaves the quantisation open.  */
/* Reading (fixed-point, bit-exact on any IEEE machine):                */
/*   m   = max_i z_i                                                    */
/*   y_i = min((m - z_i) * tscale, 1535)       (two roundings)          */
/*   u_i = rint(y_i)                          (half to even)            */
/*   w_i = lut[u_i mod 64] >> (u_i div 64)     ~ 2^23 * exp(z_i - m)    */
/*   W   = sum_i w_i,   Q = floor((2^16 - K) * 2^32 / W)                */
/*   c_i = i + floor(P_i * Q / 2^32),  P_i = sum_{j<i} w_j,  c_K = 2^16 */
/*   f_i = c_{i+1} - c_i    (every f_i >= 1, sum f_i = 2^16)            */
/* for K symbols: 256 (2^16 - K = 65280) or 4096 for 12-bit pixels     */
/* (Sec. IV "Higher Bit Depth"; 2^16 - K = 61440, and W, P_i up to     */
/* 2^35 in 64-bit integers).                                            */
/* ------------------------------------------------------------------ */

int or_table_k(const float *z, int K, float tscale, const uint32_t lut[64], uint32_t *cum) {
    if (K < 2 || K > NSYM_MAX) return OR_ERR_INVALID;
    float m = z[0];
    for (int i = 1; i < K; i++)
        if (z[i] > m) m = z[i];
    uint32_t w[NSYM_MAX];
    uint64_t Wsum = 0;
    for (int i = 0; i < K; i++) {
        float d = m - z[i];
        float y = d * tscale;
        if (!(y <= 1535.0f)) y = 1535.0f;
        int u = (int)rintf(y);
        w[i] = lut[u & 63] >> (u >> 6);
        Wsum += w[i];
    }
    if (Wsum == 0 || Wsum > (uint64_t)K << 23) return OR_ERR_INVALID;
    uint64_t Q = ((uint64_t)(TOTAL_M - (uint32_t)K) << 32) / Wsum;
    uint64_t P = 0;
    for (int i = 0; i < K; i++) {
        cum[i] = (uint32_t)i + (uint32_t)((P * Q) >> 32);
        P += w[i];
    }
    cum[K] = TOTAL_M;
    return OR_OK;
}

int or_table_from_logits(const float z[NSYM], float tscale, const uint32_t lut[64],
                         uint32_t cum[NSYM + 1]) {
    return or_table_k(z, NSYM, tscale, lut, cum);
}

/* ------------------------------------------------------------------ */
/* rANS (Sec. II-B "rANS"; Duda's range variant).  Generic in the state */
/* lower bound 2^Lb, the word size 2^bb and the table total 2^Mb so     */
/* that small instances can be checked exhaustively; the coder itself   */
/* uses Lb = bb = Mb = 16 (32-bit state, 16-bit words, tables of 2^16). */
/*   encode: while x >= ((L >> Mb) << bb) * f: emit x mod b, x /= b     */
/*           x = (x div f) * M + (x mod f) + c                          */
/*   decode: slot = x mod M, s such that c_s <= slot < c_s + f_s,       */
/*           x = f_s * (x div M) + slot - c_s,                          */
/*           while x < L: x = x * b + next word                         */
/* ------------------------------------------------------------------ */

int or_rans_enc_step(uint64_t *x, uint32_t f, uint32_t c, int Lb, int bb, int Mb,
                     uint32_t *emitted, int max_emit) {
    uint64_t L = 1ull << Lb, b = 1ull << bb;
    uint64_t x_max = ((L >> Mb) << bb) * f;
    int n = 0;
    while (*x >= x_max) {
        if (n >= max_emit) return -1;
        emitted[n++] = (uint32_t)(*x % b);
        *x /= b;
    }
    *x = (*x / f) * (1ull << Mb) + (*x % f) + c;
    return n;
}

int or_rans_dec_step(uint64_t *x, const uint32_t *cum, int nsym, int Lb, int bb, int Mb,
                     const uint32_t *words, int nwords, int *pos) {
    uint64_t L = 1ull << Lb, M = 1ull << Mb;
    uint32_t slot = (uint32_t)(*x % M);
    int s = 0;
    while (s + 1 < nsym && cum[s + 1] <= slot) s++;
    uint32_t f = cum[s + 1] - cum[s];
    *x = (uint64_t)f * (*x >> Mb) + slot - cum[s];
    while (*x < L) {
        if (*pos >= nwords) return -1;
        *x = (*x << bb) | words[(*pos)++];
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* Wavefront order (Sec. II-B "Preprocessor", Fig. 1 right).  Reading:  */
/* pixel (r, c) belongs to wave t = 3r + c, the smallest slope for      */
/* which every prior of a window with a right reach of at most 2 lies   */
/* on an earlier wave (prior (r - d, c + e), d >= 1, e <= 2, is on wave */
/* t - 3d + e < t).                                                     */
/* Streams (Sec. II-B "rANS": at most one per row): row r is coded by   */
/* stream r mod S, S <= H, and each stream holds its pixels ordered by  */
/* (t, r) ascending, which is the order in which a wavefront decoder    */
/* meets them.                                                          */
/* ------------------------------------------------------------------ */

typedef struct { int r, c; } px_t;

/* Fills order[] with the pixels of stream s in (t, r) ascending order. */
static size_t stream_order(int H, int W, int S, int s, px_t *order) {
    size_t n = 0;
    int T = 3 * (H - 1) + W;
    for (int t = 0; t < T; t++)
        for (int r = s; r < H; r += S) {
            int c = t - 3 * r;
            if (c >= 0 && c < W) { order[n].r = r; order[n].c = c; n++; }
        }
    return n;
}

/* ------------------------------------------------------------------ */
/* Container.  Reading (the paper stores one bitstream per coder         */
/* instance and says nothing of the framing):                           */
/*   "DLC1", u32 H, u32 W, u8 window rows u (2 for the default         */
/*   window), u8 precision (bit 4 set for 12-bit pixels), u16 S, u64    */
/*   model hash, u32 words[S], then                                     */
/*   S payloads of u16 words.  Each payload                             */
/*   opens with the final encoder state (high half first) followed by   */
/*   the renormalisation words in the order the decoder reads them.     */
/* All fields little-endian.                                            */
/* ------------------------------------------------------------------ */

static void wr_u16(uint8_t *p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void wr_u32(uint8_t *p, uint32_t v) { wr_u16(p, v & 0xFFFF); wr_u16(p + 2, v >> 16); }

size_t or_max_encoded_bytes(int H, int W, int S) {
    if (S > H) S = H;
    return 24 + 4 * (size_t)S + 2 * ((size_t)H * W + 2 * (size_t)S);
}

/* Per-pixel table of the model at pixel (r, c) of an image whose pixels
 * before (r, c) in wave order are those of img (later pixels are not read). */
/* img holds u8 samples for a model of 256 outputs, u16 for 4096; z_out
 * and cum_out take the model's symbol count (+ 1). */
int or_pixel_table(const uint8_t *blob, size_t blob_n, const void *img, int H, int W,
                   int r, int c, float *z_out, uint32_t *cum_out) {
    model_t m;
    int st = model_load(&m, blob, blob_n);
    if (st) return st;
    if (m.win.vol) {
        model_free(&m);
        return OR_ERR_INVALID;   /* a 3D window needs the previous slice */
    }
    uint16_t pri[MAXPRI];
    float z[NSYM_MAX];
    uint32_t cum[NSYM_MAX + 1];
    gather_win(&m.win, img, m.bits, H, W, r, c, pri);
    mlp(&m, pri, z);
    st = or_table_k(z, m.nsym, m.tscale, m.lut, cum);
    if (z_out) memcpy(z_out, z, sizeof(float) * m.nsym);
    if (cum_out) memcpy(cum_out, cum, sizeof(uint32_t) * (m.nsym + 1));
    model_free(&m);
    return st;
}

/* Logits of the model for a batch of prior vectors (n x window size, u16),
 * n x the model's symbol count. */
int or_logits(const uint8_t *blob, size_t blob_n, const uint16_t *pri, int n, float *z_out) {
    model_t m;
    int st = model_load(&m, blob, blob_n);
    if (st) return st;
    for (int i = 0; i < n; i++) mlp(&m, pri + (size_t)i * m.win.n, z_out + (size_t)i * m.nsym);
    model_free(&m);
    return OR_OK;
}

/* The model's priors at (r, c): the 2D window, or a 3D window over the
 * slice img and the previous slice `below` (NULL for the first slice). */
static void gather_model(const model_t *m, const void *below, const void *img, int H, int W, int r, int c,
                         uint16_t *pri) {
    if (m->win.vol)
        gather_win3(&m->win, below, img, m->bits, H, W, r, c, pri);
    else
        gather_win(&m->win, img, m->bits, H, W, r, c, pri);
}

static int symbol_tables(const model_t *m, const void *below, const void *img, int H, int W, uint32_t *fc_out,
                         double *bits_out) {
    double bits = 0.0;
    float z[NSYM_MAX];
    uint32_t cum[NSYM_MAX + 1];
    for (int r = 0; r < H; r++)
        for (int c = 0; c < W; c++) {
            uint16_t pri[MAXPRI];
            gather_model(m, below, img, H, W, r, c, pri);
            mlp(m, pri, z);
            int st = or_table_k(z, m->nsym, m->tscale, m->lut, cum);
            if (st) return st;
            uint32_t v = px_at(img, m->bits, (size_t)r * W + c);
            if (v >= (uint32_t)m->nsym) return OR_ERR_INVALID;   /* a 12-bit sample above 4095 */
            uint32_t f = cum[v + 1] - cum[v];
            fc_out[(size_t)r * W + c] = f | (cum[v] << 16);
            bits -= log2((double)f / 65536.0);
        }
    if (bits_out) *bits_out = bits;
    return OR_OK;
}

/* Per-pixel (f, c) of every pixel in raster order, as f | c << 16 and,
 * optionally, the ideal code length sum of -log2(f / 2^16) in float64. */
int or_symbol_tables(const uint8_t *blob, size_t blob_n, const void *img, int H, int W,
                     uint32_t *fc_out, double *bits_out) {
    model_t m;
    int st = model_load(&m, blob, blob_n);
    if (st) return st;
    st = m.win.vol ? OR_ERR_INVALID : symbol_tables(&m, NULL, img, H, W, fc_out, bits_out);
    model_free(&m);
    return st;
}

/* Codes one slice (or 2D image) into a container at out; below is the
 * previous slice for a 3D window (NULL otherwise).  Returns the bytes
 * written or minus an error code. */
static int64_t encode_slice(const model_t *m, const void *below, const void *img, int H, int W, int S,
                            uint8_t *out, size_t cap) {
    if (H < 1 || W < 1 || S < 1 || H > 65535 * 64 || W > 65535 * 64) return -OR_ERR_INVALID;
    if (S > H) S = H;
    if (S > 65535) return -OR_ERR_INVALID;
    if (cap < or_max_encoded_bytes(H, W, S)) return -OR_ERR_CAPACITY;
    size_t N = (size_t)H * W;
    uint32_t *fc = malloc(4 * N);
    int st = symbol_tables(m, below, img, H, W, fc, NULL);
    if (st) { free(fc); return -st; }

    memcpy(out, "DLC1", 4);
    wr_u32(out + 4, (uint32_t)H);
    wr_u32(out + 8, (uint32_t)W);
    /* rows of the window above the pixel (2 for the default window), with
     * bit 7 set in the slices of a volume coded with a 3D window */
    out[12] = (uint8_t)(m->win.u | (m->win.vol ? 0x80 : 0));
    /* precision, with bit 4 set for 12-bit pixels */
    out[13] = (uint8_t)(m->precision | (m->bits == 12 ? 0x10 : 0));
    wr_u16(out + 14, (uint32_t)S);
    for (int k = 0; k < 8; k++) out[16 + k] = (uint8_t)(m->hash >> (8 * k));
    size_t pos = 24 + 4 * (size_t)S;

    px_t *order = malloc(sizeof(px_t) * ((size_t)(H / S + 1) * W));
    uint32_t *emit = malloc(4 * ((size_t)(H / S + 1) * W + 4));
    for (int s = 0; s < S; s++) {
        size_t n = stream_order(H, W, S, s, order);
        uint64_t x = RANS_L;
        size_t ne = 0;
        for (size_t k = n; k-- > 0;) {
            uint32_t v = fc[(size_t)order[k].r * W + order[k].c];
            uint32_t e[4];
            int got = or_rans_enc_step(&x, v & 0xFFFF, v >> 16, 16, 16, 16, e, 4);
            for (int j = 0; j < got; j++) emit[ne++] = e[j];
        }
        uint32_t words = (uint32_t)(ne + 2);
        wr_u32(out + 24 + 4 * (size_t)s, words);
        wr_u16(out + pos, (uint32_t)(x >> 16));
        wr_u16(out + pos + 2, (uint32_t)(x & 0xFFFF));
        pos += 4;
        for (size_t k = ne; k-- > 0;) { wr_u16(out + pos, emit[k]); pos += 2; }
    }
    free(order); free(emit); free(fc);
    return (int64_t)pos;
}

/* Encodes one H x W image with S streams (S is clipped to H).  Returns the
 * number of bytes written to out, or minus an error code. */
int64_t or_encode(const uint8_t *blob, size_t blob_n, const void *img, int H, int W, int S,
                  uint8_t *out, size_t cap) {
    model_t m;
    int st = model_load(&m, blob, blob_n);
    if (st) return -st;
    int64_t n = m.win.vol ? -OR_ERR_INVALID : encode_slice(&m, NULL, img, H, W, S, out, cap);
    model_free(&m);
    return n;
}

/* Encodes a volume of D slices of H x W (slice z at vol + z H W) with a 3D
 * window, each slice as its own container with S streams, back to back;
 * offsets[z] .. offsets[z + 1] bound slice z's container.  Returns the total
 * bytes or minus an error code. */
int64_t or_encode_volume(const uint8_t *blob, size_t blob_n, const void *vol, int D, int H, int W, int S,
                         uint8_t *out, size_t cap, uint64_t *offsets) {
    if (D < 1) return -OR_ERR_INVALID;
    model_t m;
    int st = model_load(&m, blob, blob_n);
    if (st) return -st;
    if (!m.win.vol) { model_free(&m); return -OR_ERR_INVALID; }
    size_t pos = 0, N = (size_t)H * W;
    offsets[0] = 0;
    for (int z = 0; z < D; z++) {
        const size_t bps = m.bits == 12 ? 2 : 1;   /* bytes per sample */
        const uint8_t *v8 = (const uint8_t *)vol;
        int64_t n = encode_slice(&m, z ? v8 + (size_t)(z - 1) * N * bps : NULL, v8 + (size_t)z * N * bps, H, W, S,
                                 out + pos, cap - pos);
        if (n < 0) { model_free(&m); return n; }
        pos += (size_t)n;
        offsets[z + 1] = pos;
    }
    model_free(&m);
    return (int64_t)pos;
}

/* Decodes one bitstream into img_out (H x W, dims read from the header and
 * checked against the caller's).  Pixels are decoded one at a time in wave
 * order (t ascending, then r ascending): a topological order of the causal
 * dependencies that visits every stream in its own order.  below: the
 * decoded previous slice for a 3D window (NULL otherwise). */
static int decode_slice(const model_t *m, const void *below, const uint8_t *in, size_t n, void *img_out,
                        int H, int W) {
    if (H < 1 || W < 1) return OR_ERR_INVALID;
    if (n < 24 || memcmp(in, "DLC1", 4) != 0) return OR_ERR_CORRUPT;
    int h = (int)rd_u32(in + 4), w = (int)rd_u32(in + 8);
    int S = in[14] | (in[15] << 8);
    uint64_t hash = 0;
    for (int k = 0; k < 8; k++) hash |= (uint64_t)in[16 + k] << (8 * k);
    if (h != H || w != W || in[12] != (m->win.u | (m->win.vol ? 0x80 : 0)) ||
        in[13] != (m->precision | (m->bits == 12 ? 0x10 : 0)) ||
        hash != m->hash || S < 1 || S > H || n < 24 + 4 * (size_t)S)
        return OR_ERR_CORRUPT;
    uint32_t *words = malloc(4 * (size_t)S), *start = malloc(4 * (size_t)S);
    size_t total = 0;
    for (int s = 0; s < S; s++) {
        words[s] = rd_u32(in + 24 + 4 * (size_t)s);
        start[s] = (uint32_t)total;
        total += words[s];
    }
    if (24 + 4 * (size_t)S + 2 * total != n) {
        free(words); free(start);
        return OR_ERR_CORRUPT;
    }
    const uint8_t *pay = in + 24 + 4 * (size_t)S;
    uint32_t *all = malloc(4 * (total + 1));
    for (size_t k = 0; k < total; k++) all[k] = pay[2 * k] | (pay[2 * k + 1] << 8);
    uint64_t *x = malloc(8 * (size_t)S);
    int *pos = malloc(sizeof(int) * (size_t)S);
    int st = OR_OK;
    for (int s = 0; s < S && st == OR_OK; s++) {
        const uint32_t *ws = all + start[s];
        if (words[s] < 2) { st = OR_ERR_CORRUPT; break; }
        x[s] = ((uint64_t)ws[0] << 16) | ws[1];
        pos[s] = 2;
        if (x[s] < RANS_L) st = OR_ERR_CORRUPT;
    }
    memset(img_out, 0, (size_t)H * W * (m->bits == 12 ? 2 : 1));
    float z[NSYM_MAX];
    uint32_t cum[NSYM_MAX + 1];
    int T = 3 * (H - 1) + W;
    for (int t = 0; t < T && st == OR_OK; t++) {
        for (int r = 0; r < H && st == OR_OK; r++) {
            int c = t - 3 * r;
            if (c < 0 || c >= W) continue;
            int s = r % S;
            uint16_t pri[MAXPRI];
            gather_model(m, below, img_out, H, W, r, c, pri);
            mlp(m, pri, z);
            if (or_table_k(z, m->nsym, m->tscale, m->lut, cum)) { st = OR_ERR_INVALID; break; }
            int sym = or_rans_dec_step(&x[s], cum, m->nsym, 16, 16, 16, all + start[s], (int)words[s],
                                       &pos[s]);
            if (sym < 0) { st = OR_ERR_CORRUPT; break; }
            if (m->bits == 12)
                ((uint16_t *)img_out)[(size_t)r * W + c] = (uint16_t)sym;
            else
                ((uint8_t *)img_out)[(size_t)r * W + c] = (uint8_t)sym;
        }
    }
    for (int s = 0; s < S && st == OR_OK; s++)
        if (x[s] != RANS_L || (uint32_t)pos[s] != words[s]) st = OR_ERR_CORRUPT;
    free(all); free(x); free(pos); free(words); free(start);
    return st;
}

int or_decode(const uint8_t *blob, size_t blob_n, const uint8_t *in, size_t n, void *img_out,
              int H, int W) {
    model_t m;
    int st = model_load(&m, blob, blob_n);
    if (st) return st;
    st = m.win.vol ? OR_ERR_INVALID : decode_slice(&m, NULL, in, n, img_out, H, W);
    model_free(&m);
    return st;
}

/* Decodes a volume coded by or_encode_volume: slice z from bytes
 * offsets[z] .. offsets[z + 1] of in, slices in order (every prior of the
 * lower layer lies in the slice before, already decoded).  Returns the first
 * slice's error, if any. */
int or_decode_volume(const uint8_t *blob, size_t blob_n, const uint8_t *in, const uint64_t *offsets, int D,
                     void *vol_out, int H, int W) {
    if (D < 1) return OR_ERR_INVALID;
    model_t m;
    int st = model_load(&m, blob, blob_n);
    if (st) return st;
    if (!m.win.vol) { model_free(&m); return OR_ERR_INVALID; }
    const size_t N = (size_t)H * W * (m.bits == 12 ? 2 : 1);   /* bytes per slice */
    uint8_t *v8 = (uint8_t *)vol_out;
    for (int z = 0; z < D && st == OR_OK; z++)
        st = decode_slice(&m, z ? v8 + (size_t)(z - 1) * N : NULL, in + offsets[z], offsets[z + 1] - offsets[z],
                          v8 + (size_t)z * N, H, W);
    model_free(&m);
    return st;
}
