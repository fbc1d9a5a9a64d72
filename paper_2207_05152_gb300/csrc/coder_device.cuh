// Device building blocks of the coder: causal gather, the density network
// evaluated one pixel per thread on the CUDA cores, and the PDF -> frequency
// table quantisation.  Every floating-point operation is an explicit
// round-to-nearest intrinsic so that the results do not depend on compiler
// contraction and match any other IEEE implementation of the same sequence.
#pragma once

#include "internal.cuh"

namespace dlic {

// Prior order of the radius-2 causal window (Sec. II-A, Fig. 1 left):
// row r-2: c-2..c+2, row r-1: c-2..c+2, row r: c-2, c-1.  Pixels outside the
// image are the dummy value 0 (Fig. 1 right).
__device__ __forceinline__ void gather_priors(const uint8_t *img, int64_t pitch, int H, int W,
                                              int r, int c, uint8_t pri[kPriors]) {
#pragma unroll
    for (int k = 0; k < kPriors; k++) {
        const int dr = k < 5 ? -2 : (k < 10 ? -1 : 0);
        const int dc = k < 5 ? k - 2 : (k < 10 ? k - 7 : k - 12);
        const int rr = r + dr, cc = c + dc;
        pri[k] = (rr >= 0 && rr < H && cc >= 0 && cc < W) ? img[rr * pitch + cc] : (uint8_t)0;
    }
}

// ---------------------------------------------------------------------------
// FP32 network, one pixel per thread.  Each unit starts from its bias and
// accumulates fma(x_k, w_jk, acc) for k ascending (Sec. II-B; the fixed order
// makes encode and decode predictions identical, Sec. II-B "Preprocessor").
// Hidden activations live in shared memory as [unit][CH] columns.
// ---------------------------------------------------------------------------
template <int CH>
__device__ __forceinline__ void fp32_hidden(const DevModel &m, const uint8_t pri[kPriors],
                                            float *h1s, float *h2s, int tid) {
    float x[kPriors];
#pragma unroll
    for (int k = 0; k < kPriors; k++) x[k] = __fmaf_rn((float)pri[k], 0.0078125f, -1.0f);
    for (int j0 = 0; j0 < m.h1; j0 += 4) {
        float a0 = __ldg(m.b1 + j0), a1 = __ldg(m.b1 + j0 + 1), a2 = __ldg(m.b1 + j0 + 2),
              a3 = __ldg(m.b1 + j0 + 3);
#pragma unroll
        for (int k = 0; k < kPriors; k++) {
            const float4 w = __ldg(reinterpret_cast<const float4 *>(m.w1t + k * m.h1 + j0));
            a0 = __fmaf_rn(x[k], w.x, a0);
            a1 = __fmaf_rn(x[k], w.y, a1);
            a2 = __fmaf_rn(x[k], w.z, a2);
            a3 = __fmaf_rn(x[k], w.w, a3);
        }
        h1s[(j0 + 0) * CH + tid] = a0 > 0.0f ? a0 : 0.0f;
        h1s[(j0 + 1) * CH + tid] = a1 > 0.0f ? a1 : 0.0f;
        h1s[(j0 + 2) * CH + tid] = a2 > 0.0f ? a2 : 0.0f;
        h1s[(j0 + 3) * CH + tid] = a3 > 0.0f ? a3 : 0.0f;
    }
    for (int j0 = 0; j0 < m.h2; j0 += 4) {
        float a0 = __ldg(m.b2 + j0), a1 = __ldg(m.b2 + j0 + 1), a2 = __ldg(m.b2 + j0 + 2),
              a3 = __ldg(m.b2 + j0 + 3);
        for (int k = 0; k < m.h1; k++) {
            const float xk = h1s[k * CH + tid];
            const float4 w = __ldg(reinterpret_cast<const float4 *>(m.w2t + k * m.h2 + j0));
            a0 = __fmaf_rn(xk, w.x, a0);
            a1 = __fmaf_rn(xk, w.y, a1);
            a2 = __fmaf_rn(xk, w.z, a2);
            a3 = __fmaf_rn(xk, w.w, a3);
        }
        h2s[(j0 + 0) * CH + tid] = a0 > 0.0f ? a0 : 0.0f;
        h2s[(j0 + 1) * CH + tid] = a1 > 0.0f ? a1 : 0.0f;
        h2s[(j0 + 2) * CH + tid] = a2 > 0.0f ? a2 : 0.0f;
        h2s[(j0 + 3) * CH + tid] = a3 > 0.0f ? a3 : 0.0f;
    }
}

template <int CH>
__device__ __forceinline__ void fp32_logits4(const DevModel &m, const float *h2s, int tid, int j0,
                                             float z[4]) {
    float a0 = __ldg(m.b3 + j0), a1 = __ldg(m.b3 + j0 + 1), a2 = __ldg(m.b3 + j0 + 2),
          a3 = __ldg(m.b3 + j0 + 3);
    for (int k = 0; k < m.h2; k++) {
        const float xk = h2s[k * CH + tid];
        const float4 w = __ldg(reinterpret_cast<const float4 *>(m.w3t + k * kSymbols + j0));
        a0 = __fmaf_rn(xk, w.x, a0);
        a1 = __fmaf_rn(xk, w.y, a1);
        a2 = __fmaf_rn(xk, w.z, a2);
        a3 = __fmaf_rn(xk, w.w, a3);
    }
    z[0] = a0; z[1] = a1; z[2] = a2; z[3] = a3;
}

// ---------------------------------------------------------------------------
// INT8 network, one pixel per thread, dp4a on the CUDA cores.  Inputs v - 128,
// exact integer dot products, hidden units clamp(rint(fma(acc, s, o)), 0, 255),
// logits fma(acc, s, o).  Hidden activations are packed 4 per u32 in shared
// memory as [unit / 4][CH] columns.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int dp4a_ss(uint32_t a, uint32_t b, int c) {
    int d;
    asm("dp4a.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ int dp4a_us(uint32_t a, uint32_t b, int c) {
    int d;
    asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t requant_u8(int acc, float s, float o) {
    int v = __float2int_rn(__fmaf_rn(__int2float_rn(acc), s, o));
    return (uint32_t)min(max(v, 0), 255);
}

template <int CH>
__device__ __forceinline__ void int8_hidden(const DevModel &m, const uint8_t pri[kPriors],
                                            uint32_t *h1s, uint32_t *h2s, int tid) {
    uint32_t x[3];
#pragma unroll
    for (int k4 = 0; k4 < 3; k4++)
        x[k4] = (uint32_t)(uint8_t)(pri[4 * k4] ^ 0x80) | ((uint32_t)(uint8_t)(pri[4 * k4 + 1] ^ 0x80) << 8) |
                ((uint32_t)(uint8_t)(pri[4 * k4 + 2] ^ 0x80) << 16) |
                ((uint32_t)(uint8_t)(pri[4 * k4 + 3] ^ 0x80) << 24);
    for (int j0 = 0; j0 < m.h1; j0 += 4) {
        int a[4] = {0, 0, 0, 0};
#pragma unroll
        for (int k4 = 0; k4 < 3; k4++) {
            const uint4 w = __ldg(reinterpret_cast<const uint4 *>(m.q1t + k4 * m.h1 + j0));
            a[0] = dp4a_ss(x[k4], w.x, a[0]);
            a[1] = dp4a_ss(x[k4], w.y, a[1]);
            a[2] = dp4a_ss(x[k4], w.z, a[2]);
            a[3] = dp4a_ss(x[k4], w.w, a[3]);
        }
        uint32_t packed = 0;
#pragma unroll
        for (int q = 0; q < 4; q++)
            packed |= requant_u8(a[q], __ldg(m.s1 + j0 + q), __ldg(m.o1 + j0 + q)) << (8 * q);
        h1s[(j0 >> 2) * CH + tid] = packed;
    }
    for (int j0 = 0; j0 < m.h2; j0 += 4) {
        int a[4] = {0, 0, 0, 0};
        for (int k4 = 0; k4 < (m.h1 >> 2); k4++) {
            const uint32_t xk = h1s[k4 * CH + tid];
            const uint4 w = __ldg(reinterpret_cast<const uint4 *>(m.q2t + k4 * m.h2 + j0));
            a[0] = dp4a_us(xk, w.x, a[0]);
            a[1] = dp4a_us(xk, w.y, a[1]);
            a[2] = dp4a_us(xk, w.z, a[2]);
            a[3] = dp4a_us(xk, w.w, a[3]);
        }
        uint32_t packed = 0;
#pragma unroll
        for (int q = 0; q < 4; q++)
            packed |= requant_u8(a[q], __ldg(m.s2 + j0 + q), __ldg(m.o2 + j0 + q)) << (8 * q);
        h2s[(j0 >> 2) * CH + tid] = packed;
    }
}

template <int CH>
__device__ __forceinline__ void int8_logits4(const DevModel &m, const uint32_t *h2s, int tid, int j0,
                                             float z[4]) {
    int a[4] = {0, 0, 0, 0};
    for (int k4 = 0; k4 < (m.h2 >> 2); k4++) {
        const uint32_t xk = h2s[k4 * CH + tid];
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(m.q3t + k4 * kSymbols + j0));
        a[0] = dp4a_us(xk, w.x, a[0]);
        a[1] = dp4a_us(xk, w.y, a[1]);
        a[2] = dp4a_us(xk, w.z, a[2]);
        a[3] = dp4a_us(xk, w.w, a[3]);
    }
#pragma unroll
    for (int q = 0; q < 4; q++)
        z[q] = __fmaf_rn(__int2float_rn(a[q]), __ldg(m.s3 + j0 + q), __ldg(m.o3 + j0 + q));
}

// ---------------------------------------------------------------------------
// PDF -> frequency table (fixed point).  With m = max z:
//   u_i = rint(min((m - z_i) * tscale, 1535)),  w_i = lut[u_i & 63] >> (u_i >> 6)
//   W = sum w_i,  Q = floor(65280 * 2^32 / W)
//   c_i = i + floor(P_i * Q / 2^32) with P_i = sum_{j<i} w_j,  c_256 = 2^16.
// Every f_i = c_{i+1} - c_i is >= 1 and the table sums to 2^16, the total the
// rANS coder needs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t table_weight(float m, float z, float tscale, const uint32_t *lut_s) {
    float y = __fmul_rn(__fsub_rn(m, z), tscale);
    y = y <= 1535.0f ? y : 1535.0f;
    const int u = __float2int_rn(y);
    return lut_s[u & 63] >> (u >> 6);
}

// The same weight from the expanded table lut2[u] = lut[u mod 64] >> (u div 64)
// (kTableSteps entries, built once per CTA by expand_lut).
constexpr int kTableSteps = 1536;
__device__ __forceinline__ uint32_t table_weight2(float m, float z, float tscale, const uint32_t *lut2_s) {
    float y = __fmul_rn(__fsub_rn(m, z), tscale);
    y = y <= 1535.0f ? y : 1535.0f;
    return lut2_s[__float2int_rn(y)];
}
__device__ __forceinline__ void expand_lut(const uint32_t *lut_g, uint32_t *lut2_s, int tid, int nthreads) {
    for (int u = tid; u < kTableSteps; u += nthreads) lut2_s[u] = __ldg(lut_g + (u & 63)) >> (u >> 6);
}

// Order-preserving map of a float to an unsigned integer (and back), so
// that a warp-wide unsigned maximum finds the float maximum.
__device__ __forceinline__ uint32_t float_key(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__device__ __forceinline__ uint32_t table_q(uint32_t W) {
    return (uint32_t)((65280ull << 32) / (unsigned long long)W);
}

}  // namespace dlic
