// Coding kernels on the CUDA cores: the all-pixels-at-once prediction of the
// encoder and the wavefront decoder (Sec. II-A, Fig. 2; Sec. II-B).  One
// thread evaluates the network for one pixel.  These kernels serve the FP32
// network everywhere and the INT8 network where the tensor-core kernels do
// not apply.
#include "coder_device.cuh"
#include "decode_setup.cuh"

namespace dlic {

constexpr int kCH = kPredictTile;   // pixels per CTA (one per thread)

template <int PREC>
struct HiddenBuf;
template <>
struct HiddenBuf<DLIC_FP32> {
    using T = float;
    static constexpr int per_unit = 1;
};
template <>
struct HiddenBuf<DLIC_INT8> {
    using T = uint32_t;
    static constexpr int per_unit = 4;
};

template <int PREC>
__device__ __forceinline__ void hidden(const DevModel &m, const uint8_t *pri, void *h1, void *h2, int tid) {
    if constexpr (PREC == DLIC_FP32)
        fp32_hidden<kCH>(m, pri, (float *)h1, (float *)h2, tid);
    else
        int8_hidden<kCH>(m, pri, (uint32_t *)h1, (uint32_t *)h2, tid);
}

template <int PREC>
__device__ __forceinline__ void logits4(const DevModel &m, const void *h2, int tid, int j0, float z[4]) {
    if constexpr (PREC == DLIC_FP32)
        fp32_logits4<kCH>(m, (const float *)h2, tid, j0, z);
    else
        int8_logits4<kCH>(m, (const uint32_t *)h2, tid, j0, z);
}

template <int PREC>
__host__ __device__ inline size_t hidden_bytes(int h) {
    return (size_t)h / HiddenBuf<PREC>::per_unit * kCH * 4;
}

// ---------------------------------------------------------------------------
// Networks of other than two hidden layers (Sec. II-B "Neural Network
// Architecture": six dense layers), one pixel per thread, from the model's
// layer table.  The same arithmetic as the fixed-depth helpers: FP32 units
// start from the bias and accumulate fma(x_k, w_jk, acc) for k ascending,
// then ReLU; INT8 units are exact dp4a dot products, requantised to u8.
// Hidden layer l of L writes shared buffer B when L - 1 - l is even, else A,
// so that the last hidden layer is always in B.  With G > 1 threads per
// pixel, thread group g computes the unit quads g, g + G, ... of every layer
// and the CTA meets at a barrier after each layer (every group reaches it;
// inactive threads compute nothing).  Shared-memory column tid is the pixel's.
// ---------------------------------------------------------------------------
template <int PREC, int G>
__device__ void deep_hidden(const DevModel &m, const uint8_t pri[kPriors], uint8_t *A, uint8_t *B, int tid, int g,
                            bool active) {
    const int L = m.nl - 1;
    for (int l = 0; l < L; l++) {
        if (G > 1 && l > 0) __syncthreads();
        if (!active) continue;
        const DevLayer ly = m.layers[l];
        uint8_t *out = ((L - 1 - l) & 1) ? A : B;
        const uint8_t *in = ((L - l) & 1) ? A : B;   // written by layer l - 1
        if constexpr (PREC == DLIC_FP32) {
            const float *wt = static_cast<const float *>(ly.w);
            const float *xs = reinterpret_cast<const float *>(in);
            float *os = reinterpret_cast<float *>(out);
            float x0[kPriors];
#pragma unroll
            for (int k = 0; k < kPriors; k++) x0[k] = __fmaf_rn((float)pri[k], 0.0078125f, -1.0f);
            for (int j0 = 4 * g; j0 < ly.n_out; j0 += 4 * G) {
                float a0 = __ldg(ly.a + j0), a1 = __ldg(ly.a + j0 + 1), a2 = __ldg(ly.a + j0 + 2),
                      a3 = __ldg(ly.a + j0 + 3);
                if (l == 0) {   // n_in = kPriors (the default window)
#pragma unroll
                    for (int k = 0; k < kPriors; k++) {
                        const float4 w = __ldg(reinterpret_cast<const float4 *>(wt + (size_t)k * ly.n_out + j0));
                        a0 = __fmaf_rn(x0[k], w.x, a0);
                        a1 = __fmaf_rn(x0[k], w.y, a1);
                        a2 = __fmaf_rn(x0[k], w.z, a2);
                        a3 = __fmaf_rn(x0[k], w.w, a3);
                    }
                } else {
                    for (int k = 0; k < ly.n_in; k++) {
                        const float xk = xs[k * kCH + tid];
                        const float4 w = __ldg(reinterpret_cast<const float4 *>(wt + (size_t)k * ly.n_out + j0));
                        a0 = __fmaf_rn(xk, w.x, a0);
                        a1 = __fmaf_rn(xk, w.y, a1);
                        a2 = __fmaf_rn(xk, w.z, a2);
                        a3 = __fmaf_rn(xk, w.w, a3);
                    }
                }
                os[(j0 + 0) * kCH + tid] = a0 > 0.0f ? a0 : 0.0f;
                os[(j0 + 1) * kCH + tid] = a1 > 0.0f ? a1 : 0.0f;
                os[(j0 + 2) * kCH + tid] = a2 > 0.0f ? a2 : 0.0f;
                os[(j0 + 3) * kCH + tid] = a3 > 0.0f ? a3 : 0.0f;
            }
        } else {
            const uint32_t *wq = static_cast<const uint32_t *>(ly.w);
            const uint32_t *xs = reinterpret_cast<const uint32_t *>(in);
            uint32_t *os = reinterpret_cast<uint32_t *>(out);
            uint32_t x0[kPriors / 4];   // priors v - 128 as signed bytes
#pragma unroll
            for (int k4 = 0; k4 < kPriors / 4; k4++)
                x0[k4] = (uint32_t)(uint8_t)(pri[4 * k4] ^ 0x80) | ((uint32_t)(uint8_t)(pri[4 * k4 + 1] ^ 0x80) << 8) |
                         ((uint32_t)(uint8_t)(pri[4 * k4 + 2] ^ 0x80) << 16) |
                         ((uint32_t)(uint8_t)(pri[4 * k4 + 3] ^ 0x80) << 24);
            const int k4n = ly.n_in >> 2;
            for (int j0 = 4 * g; j0 < ly.n_out; j0 += 4 * G) {
                int a[4] = {0, 0, 0, 0};
                if (l == 0) {   // n_in = kPriors: signed inputs
#pragma unroll
                    for (int k4 = 0; k4 < kPriors / 4; k4++) {
                        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(wq + (size_t)k4 * ly.n_out + j0));
                        a[0] = dp4a_ss(x0[k4], w.x, a[0]);
                        a[1] = dp4a_ss(x0[k4], w.y, a[1]);
                        a[2] = dp4a_ss(x0[k4], w.z, a[2]);
                        a[3] = dp4a_ss(x0[k4], w.w, a[3]);
                    }
                } else {        // u8 hidden units
                    for (int k4 = 0; k4 < k4n; k4++) {
                        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(wq + (size_t)k4 * ly.n_out + j0));
                        const uint32_t xk = xs[k4 * kCH + tid];
                        a[0] = dp4a_us(xk, w.x, a[0]);
                        a[1] = dp4a_us(xk, w.y, a[1]);
                        a[2] = dp4a_us(xk, w.z, a[2]);
                        a[3] = dp4a_us(xk, w.w, a[3]);
                    }
                }
                uint32_t packed = 0;
#pragma unroll
                for (int q = 0; q < 4; q++)
                    packed |= requant_u8(a[q], __ldg(ly.a + j0 + q), __ldg(ly.o + j0 + q)) << (8 * q);
                os[(j0 >> 2) * kCH + tid] = packed;
            }
        }
    }
    if (G > 1) __syncthreads();
}

// Logits j0 .. j0 + 3 of the output layer from the last hidden layer (in B).
template <int PREC>
__device__ __forceinline__ void deep_logits4(const DevModel &m, const uint8_t *B, int tid, int j0, float z[4]) {
    const DevLayer ly = m.layers[m.nl - 1];
    if constexpr (PREC == DLIC_FP32) {
        const float *wt = static_cast<const float *>(ly.w);
        const float *xs = reinterpret_cast<const float *>(B);
        float a0 = __ldg(ly.a + j0), a1 = __ldg(ly.a + j0 + 1), a2 = __ldg(ly.a + j0 + 2), a3 = __ldg(ly.a + j0 + 3);
        for (int k = 0; k < ly.n_in; k++) {
            const float xk = xs[k * kCH + tid];
            const float4 w = __ldg(reinterpret_cast<const float4 *>(wt + (size_t)k * kSymbols + j0));
            a0 = __fmaf_rn(xk, w.x, a0);
            a1 = __fmaf_rn(xk, w.y, a1);
            a2 = __fmaf_rn(xk, w.z, a2);
            a3 = __fmaf_rn(xk, w.w, a3);
        }
        z[0] = a0; z[1] = a1; z[2] = a2; z[3] = a3;
    } else {
        const uint32_t *wq = static_cast<const uint32_t *>(ly.w);
        const uint32_t *xs = reinterpret_cast<const uint32_t *>(B);
        int a[4] = {0, 0, 0, 0};
        for (int k4 = 0; k4 < (ly.n_in >> 2); k4++) {
            const uint32_t xk = xs[k4 * kCH + tid];
            const uint4 w = __ldg(reinterpret_cast<const uint4 *>(wq + (size_t)k4 * kSymbols + j0));
            a[0] = dp4a_us(xk, w.x, a[0]);
            a[1] = dp4a_us(xk, w.y, a[1]);
            a[2] = dp4a_us(xk, w.z, a[2]);
            a[3] = dp4a_us(xk, w.w, a[3]);
        }
#pragma unroll
        for (int q = 0; q < 4; q++) z[q] = __fmaf_rn(__int2float_rn(a[q]), __ldg(ly.a + j0 + q), __ldg(ly.o + j0 + q));
    }
}

// Hidden layers and logits of either network depth: the fixed-depth helpers
// for two hidden layers, the layer table otherwise.
template <int PREC, bool DEEP>
__device__ __forceinline__ void net_hidden(const DevModel &m, const uint8_t *pri, uint8_t *A, uint8_t *B, int tid) {
    if constexpr (DEEP)
        deep_hidden<PREC, 1>(m, pri, A, B, tid, 0, true);
    else
        hidden<PREC>(m, pri, A, B, tid);
}
template <int PREC, bool DEEP>
__device__ __forceinline__ void net_logits4(const DevModel &m, const uint8_t *B, int tid, int j0, float z[4]) {
    if constexpr (DEEP)
        deep_logits4<PREC>(m, B, tid, j0, z);
    else
        logits4<PREC>(m, B, tid, j0, z);
}

// ---------------------------------------------------------------------------
// Encoder prediction: every pixel of every image at once (the encoder knows
// all priors).  Writes (f, c) of the pixel's own value as f | c << 16.
// ---------------------------------------------------------------------------
template <int PREC, bool DEEP>
__global__ void __launch_bounds__(kCH) k_predict_cc(DevModel m, EncBatch b) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t lut_s[64];
    const int tid = threadIdx.x;
    if (tid < 64) lut_s[tid] = m.lut[tid];
    __syncthreads();

    const int tile = blockIdx.x;
    int ii = 0;
    while (ii + 1 < b.n && b.img[ii + 1].tile_begin <= tile) ii++;
    const EncImage &im = b.img[ii];
    const int64_t p = (int64_t)(tile - im.tile_begin) * kCH + tid;   // tile_px == kCH
    if (p >= (int64_t)im.H * im.W) return;
    const int r = (int)(p / im.W), c = (int)(p % im.W);

    uint8_t pri[kPriors];
    gather_priors(im.pixels, im.pitch, im.H, im.W, r, c, pri);
    uint8_t *h1 = smem;
    uint8_t *h2 = smem + hidden_bytes<PREC>(DEEP ? m.hmax : m.h1);
    net_hidden<PREC, DEEP>(m, pri, h1, h2, tid);

    float zmax = -INFINITY;
    for (int j0 = 0; j0 < kSymbols; j0 += 4) {
        float z[4];
        net_logits4<PREC, DEEP>(m, h2, tid, j0, z);
#pragma unroll
        for (int q = 0; q < 4; q++) zmax = z[q] > zmax ? z[q] : zmax;
    }
    const int sym = im.pixels[r * im.pitch + c];
    uint32_t W = 0, Ps = 0, ws = 0;
    for (int j0 = 0; j0 < kSymbols; j0 += 4) {
        float z[4];
        net_logits4<PREC, DEEP>(m, h2, tid, j0, z);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int i = j0 + q;
            const uint32_t w = table_weight(zmax, z[q], m.tscale, lut_s);
            W += w;
            Ps += i < sym ? w : 0u;
            ws = i == sym ? w : ws;
        }
    }
    const uint32_t Q = table_q(W);
    const uint32_t c_lo = (uint32_t)sym + __umulhi(Ps, Q);
    const uint32_t c_hi = sym == kSymbols - 1 ? kTotal : (uint32_t)sym + 1u + __umulhi(Ps + ws, Q);
    uint32_t *fc = reinterpret_cast<uint32_t *>(b.ws + im.fc_off);
    fc[b.raster ? (int64_t)r * im.W + c : stream_index(im.H, im.W, im.S, r, c)] = (c_hi - c_lo) | (c_lo << 16);
}

// ---------------------------------------------------------------------------
// Encoder prediction with the FP32 network, 64 pixels per CTA: the layers
// as register tiles on the CUDA cores (each unit of each pixel still starts
// from its bias and accumulates fma(x_k, w_jk, acc) for k ascending, so the
// result is the same as one pixel per thread), weights read as 16-byte rows
// through L1/L2, activations in shared memory [unit][pitch kF32Pitch]; then
// one warp per pixel for the frequency table of the pixel's own value.
// ---------------------------------------------------------------------------
constexpr int kF32Tile = 64, kF32Pitch = kF32Tile + 4, kF32Threads = 256;

// xs holds the tile's inputs [64][k1] (the window's priors padded to 16).
__host__ __device__ inline size_t f32_predict_smem(int h1, int h2, int k1) {
    const size_t xs = (size_t)kF32Tile * k1 * 4, h1t = (size_t)h1 * kF32Pitch * 4, z = (size_t)kF32Tile * kSymbols * 4;
    const size_t region = xs + h1t > z ? xs + h1t : z;   // z overlays xs and h1t
    return region + (size_t)h2 * kF32Pitch * 4;
}

// acc[i][j] (units 4 uq + i, pixels p0 + j) over k rows of w (row stride ldw)
// and the activation rows act[k][p0 ..] (pitch kF32Pitch).
template <int J>
__device__ __forceinline__ void f32_tile(float (&acc)[4][J], const float *w, int ldw, const float *act, int K, int uq,
                                         int p0) {
#pragma unroll 2
    for (int k = 0; k < K; k++) {
        const float4 wv = __ldg(reinterpret_cast<const float4 *>(w + (size_t)k * ldw) + uq);
        const float wk[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
        for (int j4 = 0; j4 < J / 4; j4++) {
            const float4 xv = *reinterpret_cast<const float4 *>(act + k * kF32Pitch + p0 + 4 * j4);
            const float xk[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int jj = 0; jj < 4; jj++) acc[i][4 * j4 + jj] = __fmaf_rn(xk[jj], wk[i], acc[i][4 * j4 + jj]);
        }
    }
}

__device__ __forceinline__ uint32_t f32_key(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void __launch_bounds__(kF32Threads, 2) k_predict_f32(DevModel m, EncBatch b) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t lut_s[kTableSteps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int h1 = m.h1, h2 = m.h2, npri = m.n_in, K1 = (npri + 15) / 16 * 16;
    expand_lut(m.lut, lut_s, tid, kF32Threads);
    float *xs = reinterpret_cast<float *>(smem);                         // [64][K1]
    float *h1t = xs + kF32Tile * K1;                                      // [h1][pitch]
    float *zs = reinterpret_cast<float *>(smem);                         // [64][256], after layer 2
    const size_t region = f32_predict_smem(h1, h2, K1) - (size_t)h2 * kF32Pitch * 4;
    float *h2t = reinterpret_cast<float *>(smem + region);                // [h2][pitch]

    const int tile = blockIdx.x;
    int ii = 0;
    while (ii + 1 < b.n && b.img[ii + 1].tile_begin <= tile) ii++;
    const EncImage &im = b.img[ii];
    const int64_t p_base = (int64_t)(tile - im.tile_begin) * kF32Tile;
    const int64_t npx = (int64_t)im.H * im.W;
    // inputs x/128 - 1 of the 64 pixels (pixels past the image get zeros)
    for (int i = tid; i < kF32Tile * npri; i += kF32Threads) {
        const int p = i / npri, q = i % npri;
        const int64_t pp = p_base + p;
        float v = 0.0f;
        if (pp < npx) {
            const int r = (int)(pp / im.W), c = (int)(pp % im.W);
            int dz, dr, dc;
            window_offset(m, q, dz, dr, dc);
            const int rr = r + dr, cc = c + dc;
            const uint8_t *src = dz ? im.below : im.pixels;   // the previous slice for a 3D window
            const uint32_t pv =
                (src && rr >= 0 && rr < im.H && cc >= 0 && cc < im.W) ? src[(int64_t)rr * im.pitch + cc] : 0u;
            v = __fmaf_rn((float)pv, 0.0078125f, -1.0f);
        }
        xs[p * K1 + q] = v;
    }
    __syncthreads();
    // layer 1: thread = (unit, 4 pixels)
    for (int it = tid; it < h1 * (kF32Tile / 4); it += kF32Threads) {
        const int u = it % h1, p0 = 4 * (it / h1);
        float a[4];
        const float bias = __ldg(m.b1 + u);
#pragma unroll
        for (int j = 0; j < 4; j++) a[j] = bias;
#pragma unroll 4
        for (int k = 0; k < npri; k++) {
            const float w = __ldg(m.w1t + k * h1 + u);
#pragma unroll
            for (int j = 0; j < 4; j++) a[j] = __fmaf_rn(xs[(p0 + j) * K1 + k], w, a[j]);
        }
        *reinterpret_cast<float4 *>(h1t + u * kF32Pitch + p0) =
            make_float4(a[0] > 0.0f ? a[0] : 0.0f, a[1] > 0.0f ? a[1] : 0.0f, a[2] > 0.0f ? a[2] : 0.0f,
                        a[3] > 0.0f ? a[3] : 0.0f);
    }
    __syncthreads();
    // layer 2: thread = (4 units, 8 pixels)
    for (int it = tid; it < (h2 / 4) * (kF32Tile / 8); it += kF32Threads) {
        const int uq = it % (h2 / 4), p0 = 8 * (it / (h2 / 4));
        float acc[4][8];
        const float4 bb = __ldg(reinterpret_cast<const float4 *>(m.b2) + uq);
#pragma unroll
        for (int j = 0; j < 8; j++) {
            acc[0][j] = bb.x; acc[1][j] = bb.y; acc[2][j] = bb.z; acc[3][j] = bb.w;
        }
        f32_tile<8>(acc, m.w2t, h2, h1t, h1, uq, p0);
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j4 = 0; j4 < 2; j4++)
                *reinterpret_cast<float4 *>(h2t + (4 * uq + i) * kF32Pitch + p0 + 4 * j4) = make_float4(
                    acc[i][4 * j4] > 0.0f ? acc[i][4 * j4] : 0.0f, acc[i][4 * j4 + 1] > 0.0f ? acc[i][4 * j4 + 1] : 0.0f,
                    acc[i][4 * j4 + 2] > 0.0f ? acc[i][4 * j4 + 2] : 0.0f,
                    acc[i][4 * j4 + 3] > 0.0f ? acc[i][4 * j4 + 3] : 0.0f);
    }
    __syncthreads();
    // logits: thread = (4 units, 8 pixels); z [pixel][256] overlays xs and h1t
    for (int it = tid; it < (kSymbols / 4) * (kF32Tile / 8); it += kF32Threads) {
        const int uq = it % (kSymbols / 4), p0 = 8 * (it / (kSymbols / 4));
        float acc[4][8];
        const float4 bb = __ldg(reinterpret_cast<const float4 *>(m.b3) + uq);
#pragma unroll
        for (int j = 0; j < 8; j++) {
            acc[0][j] = bb.x; acc[1][j] = bb.y; acc[2][j] = bb.z; acc[3][j] = bb.w;
        }
        f32_tile<8>(acc, m.w3t, kSymbols, h2t, h2, uq, p0);
#pragma unroll
        for (int j = 0; j < 8; j++)
            *reinterpret_cast<float4 *>(zs + (p0 + j) * kSymbols + 4 * uq) =
                make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
    }
    __syncthreads();
    // frequency table of each pixel's own value, one warp per pixel
    uint32_t *fc = reinterpret_cast<uint32_t *>(b.ws + im.fc_off);
    for (int p = warp; p < kF32Tile; p += kF32Threads / 32) {
        const int64_t pp = p_base + p;
        if (pp >= npx) break;
        const int r = (int)(pp / im.W), c = (int)(pp % im.W);
        const int sym = im.pixels[r * im.pitch + c];
        float z[8];
        const float4 za = *reinterpret_cast<const float4 *>(zs + p * kSymbols + 8 * lane);
        const float4 zc = *reinterpret_cast<const float4 *>(zs + p * kSymbols + 8 * lane + 4);
        z[0] = za.x; z[1] = za.y; z[2] = za.z; z[3] = za.w; z[4] = zc.x; z[5] = zc.y; z[6] = zc.z; z[7] = zc.w;
        uint32_t key = f32_key(z[0]);
#pragma unroll
        for (int q = 1; q < 8; q++) key = max(key, f32_key(z[q]));
        const uint32_t km = __reduce_max_sync(0xffffffffu, key);
        const float mx = __uint_as_float((km & 0x80000000u) ? (km & 0x7FFFFFFFu) : ~km);
        uint32_t lw = 0, lp = 0, lsym = 0;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int i = 8 * lane + q;
            const uint32_t w = table_weight2(mx, z[q], m.tscale, lut_s);
            lw += w;
            lp += i < sym ? w : 0u;
            lsym = i == sym ? w : lsym;
        }
        const uint32_t W = __reduce_add_sync(0xffffffffu, lw);
        const uint32_t Ps = __reduce_add_sync(0xffffffffu, lp);
        const uint32_t ws = __reduce_add_sync(0xffffffffu, lsym);
        if (lane == 0) {
            const uint32_t Q = table_q(W);
            const uint32_t c_lo = (uint32_t)sym + __umulhi(Ps, Q);
            const uint32_t c_hi = sym == kSymbols - 1 ? kTotal : (uint32_t)sym + 1u + __umulhi(Ps + ws, Q);
            fc[b.raster ? (int64_t)r * im.W + c : stream_index(im.H, im.W, im.S, r, c)] = (c_hi - c_lo) | (c_lo << 16);
        }
    }
}

bool f32_predict_supported(const DevModel &m) {
    return m.precision == DLIC_FP32 && m.nl == 3 && m.h1 % 4 == 0 && m.h2 % 4 == 0 && m.h1 <= kMaxHidden && m.h2 <= kMaxHidden &&
           f32_predict_smem(m.h1, m.h2, (m.n_in + 15) / 16 * 16) <= 200 * 1024;
}

// ---------------------------------------------------------------------------
// Wavefront decoder (Sec. II-B "Preprocessor"): one CTA per image.  Wave t
// holds the pixels (r, t - 3r); all their priors were decoded on earlier
// waves.  Pixels of a wave are predicted in parallel; the rANS step of
// pixels that share a stream (rows S apart) runs in row order.
// ---------------------------------------------------------------------------
// Threads per pixel and per CTA of the decoder for deeper networks.
constexpr int kDeepGroups = 8, kDeepThreads = kCH * kDeepGroups;
static_assert(kDeepThreads <= kSetupThreads, "decode_setup serves CTAs of up to kSetupThreads threads");

template <int PREC>
__global__ void __launch_bounds__(kCH) k_decode_cc(DevModel m, DecBatch b) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t lut_s[64];
    __shared__ int s_err;
    const int tid = threadIdx.x;
    const DecImage &im = b.img[blockIdx.x];
    if (tid < 64) lut_s[tid] = m.lut[tid];
    if (tid == 0) s_err = 0;
    StreamState *st = reinterpret_cast<StreamState *>(b.ws + im.st_off);
    const uint8_t *in = b.in + im.in_off;
    int S;
    const uint16_t *pay;
    if (!decode_setup(m, im, in, st, &S, &pay)) {
        if (tid == 0) b.status[im.sidx] = DLIC_ERR_CORRUPT;
        return;
    }
    float *zs = reinterpret_cast<float *>(smem);                        // [256][CH]
    uint8_t *h1 = smem;                                                  // aliases zs (dead by then)
    uint8_t *h2 = smem + (size_t)kSymbols * kCH * 4;
    const int H = im.H, W = im.W;
    const int T = 3 * (H - 1) + W;
    for (int t = 0; t < T; t++) {
        if (s_err) break;
        const int r_lo = t - W + 1 > 0 ? (t - W + 3) / 3 : 0;
        const int r_hi = min(H - 1, t / 3);
        const int n_t = r_hi - r_lo + 1;
        for (int base = 0; base < n_t; base += kCH) {
            const int pix = base + tid;
            const bool active = pix < n_t;
            const int r = r_lo + pix, c = t - 3 * r;
            uint32_t Q = 0;
            if (active) {
                uint8_t pri[kPriors];
                gather_priors(im.pixels, im.pitch, H, W, r, c, pri);
                hidden<PREC>(m, pri, h1, h2, tid);
                float zmax = -INFINITY;
                for (int j0 = 0; j0 < kSymbols; j0 += 4) {
                    float z[4];
                    logits4<PREC>(m, h2, tid, j0, z);
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        zs[(j0 + q) * kCH + tid] = z[q];
                        zmax = z[q] > zmax ? z[q] : zmax;
                    }
                }
                uint32_t Wsum = 0;
                for (int i = 0; i < kSymbols; i++) {
                    const float zi = zs[i * kCH + tid];
                    Wsum += table_weight(zmax, zi, m.tscale, lut_s);
                    zs[i * kCH + tid] = __fsub_rn(zmax, zi);   // keep m - z for the search
                }
                Q = table_q(Wsum);
            }
            const int rounds = (min(kCH, n_t - base) + S - 1) / S;
            for (int rnd = 0; rnd < rounds; rnd++) {
                if (active && tid / S == rnd) {
                    StreamState q = st[r % S];
                    const uint32_t slot = q.x & 0xFFFFu;
                    uint32_t P = 0, c_lo = 0, f = 1;
                    int sym = kSymbols - 1;
                    for (int i = 0; i < kSymbols; i++) {
                        float y = __fmul_rn(zs[i * kCH + tid], m.tscale);
                        y = y <= 1535.0f ? y : 1535.0f;
                        const int u = __float2int_rn(y);
                        const uint32_t w = lut_s[u & 63] >> (u >> 6);
                        const uint32_t lo = (uint32_t)i + __umulhi(P, Q);
                        const uint32_t hi = i == kSymbols - 1 ? kTotal : (uint32_t)i + 1u + __umulhi(P + w, Q);
                        if (hi > slot) {
                            sym = i;
                            c_lo = lo;
                            f = hi - lo;
                            break;
                        }
                        P += w;
                    }
                    q.x = f * (q.x >> 16) + slot - c_lo;
                    if (q.x < kRansL) {
                        if (q.pos < q.end) {
                            q.x = (q.x << 16) | pay[q.pos];
                            q.pos++;
                        } else {
                            s_err = 1;
                        }
                    }
                    st[r % S] = q;
                    im.pixels[(int64_t)r * im.pitch + c] = (uint8_t)sym;
                }
                __syncthreads();
            }
        }
    }
    __syncthreads();
    // final states must be back at the initial value L with every word read
    for (int s = tid; s < S && !s_err; s += kCH) {
        const StreamState q = st[s];
        if (q.x != kRansL || q.pos != q.end) s_err = 1;
    }
    __syncthreads();
    if (tid == 0) b.status[im.sidx] = s_err ? DLIC_ERR_CORRUPT : DLIC_OK;
}

// ---------------------------------------------------------------------------
// Wavefront decoder for networks of other than two hidden layers: the
// decoder above with kDeepGroups threads per pixel.  Thread (g, p) owns
// pixel slot p of the wave's chunk and unit group g: it computes the unit
// quads g, g + G, ... of every layer (a CTA barrier after each layer), the
// logits quads of the same pattern, and the table weights of those symbols.
// The partial maxima and weight sums meet in shared memory (a maximum and an
// integer sum: the same values in any order); the rANS step of the pixel
// runs in group 0 in the row order of the one-thread-per-pixel decoder.
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(kDeepThreads) k_decode_deep(DevModel m, DecBatch b) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t lut_s[64];
    __shared__ float s_zmax[kDeepGroups][kCH];
    __shared__ uint32_t s_wsum[kDeepGroups][kCH];
    __shared__ int s_err;
    const int tid = threadIdx.x, p = tid % kCH, g = tid / kCH;
    const DecImage &im = b.img[blockIdx.x];
    if (tid < 64) lut_s[tid] = m.lut[tid];
    if (tid == 0) s_err = 0;
    StreamState *st = reinterpret_cast<StreamState *>(b.ws + im.st_off);
    const uint8_t *in = b.in + im.in_off;
    int S;
    const uint16_t *pay;
    if (!decode_setup(m, im, in, st, &S, &pay)) {
        if (tid == 0) b.status[im.sidx] = DLIC_ERR_CORRUPT;
        return;
    }
    float *zs = reinterpret_cast<float *>(smem);                        // [256][CH]
    uint8_t *A = smem;                                                   // aliases zs (dead by then)
    uint8_t *B = smem + (size_t)kSymbols * kCH * 4;
    const int H = im.H, W = im.W;
    const int T = 3 * (H - 1) + W;
    for (int t = 0; t < T; t++) {
        if (s_err) break;
        const int r_lo = t - W + 1 > 0 ? (t - W + 3) / 3 : 0;
        const int r_hi = min(H - 1, t / 3);
        const int n_t = r_hi - r_lo + 1;
        for (int base = 0; base < n_t; base += kCH) {
            const int pix = base + p;
            const bool active = pix < n_t;
            const int r = r_lo + pix, c = t - 3 * r;
            uint8_t pri[kPriors];
            if (active) gather_priors(im.pixels, im.pitch, H, W, r, c, pri);
            deep_hidden<PREC, kDeepGroups>(m, pri, A, B, p, g, active);   // ends at a barrier
            float zmax = -INFINITY;
            if (active) {
                for (int j0 = 4 * g; j0 < kSymbols; j0 += 4 * kDeepGroups) {
                    float z[4];
                    deep_logits4<PREC>(m, B, p, j0, z);
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        zs[(j0 + q) * kCH + p] = z[q];
                        zmax = z[q] > zmax ? z[q] : zmax;
                    }
                }
            }
            s_zmax[g][p] = zmax;
            __syncthreads();
            float mx = s_zmax[0][p];
#pragma unroll
            for (int k = 1; k < kDeepGroups; k++) mx = s_zmax[k][p] > mx ? s_zmax[k][p] : mx;
            uint32_t wpart = 0;
            if (active) {
                for (int j0 = 4 * g; j0 < kSymbols; j0 += 4 * kDeepGroups)
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const float zi = zs[(j0 + q) * kCH + p];
                        wpart += table_weight(mx, zi, m.tscale, lut_s);
                        zs[(j0 + q) * kCH + p] = __fsub_rn(mx, zi);   // keep m - z for the search
                    }
            }
            s_wsum[g][p] = wpart;
            __syncthreads();
            uint32_t Wsum = 0;
#pragma unroll
            for (int k = 0; k < kDeepGroups; k++) Wsum += s_wsum[k][p];
            const uint32_t Q = active ? table_q(Wsum) : 0u;
            const int rounds = (min(kCH, n_t - base) + S - 1) / S;
            for (int rnd = 0; rnd < rounds; rnd++) {
                if (g == 0 && active && p / S == rnd) {
                    StreamState q = st[r % S];
                    const uint32_t slot = q.x & 0xFFFFu;
                    uint32_t P = 0, c_lo = 0, f = 1;
                    int sym = kSymbols - 1;
                    for (int i = 0; i < kSymbols; i++) {
                        float y = __fmul_rn(zs[i * kCH + p], m.tscale);
                        y = y <= 1535.0f ? y : 1535.0f;
                        const int u = __float2int_rn(y);
                        const uint32_t w = lut_s[u & 63] >> (u >> 6);
                        const uint32_t lo = (uint32_t)i + __umulhi(P, Q);
                        const uint32_t hi = i == kSymbols - 1 ? kTotal : (uint32_t)i + 1u + __umulhi(P + w, Q);
                        if (hi > slot) {
                            sym = i;
                            c_lo = lo;
                            f = hi - lo;
                            break;
                        }
                        P += w;
                    }
                    q.x = f * (q.x >> 16) + slot - c_lo;
                    if (q.x < kRansL) {
                        if (q.pos < q.end) {
                            q.x = (q.x << 16) | pay[q.pos];
                            q.pos++;
                        } else {
                            s_err = 1;
                        }
                    }
                    st[r % S] = q;
                    im.pixels[(int64_t)r * im.pitch + c] = (uint8_t)sym;
                }
                __syncthreads();
            }
        }
    }
    __syncthreads();
    // final states must be back at the initial value L with every word read
    for (int s2 = tid; s2 < S && !s_err; s2 += kDeepThreads) {
        const StreamState q = st[s2];
        if (q.x != kRansL || q.pos != q.end) s_err = 1;
    }
    __syncthreads();
    if (tid == 0) b.status[im.sidx] = s_err ? DLIC_ERR_CORRUPT : DLIC_OK;
}

static bool deep_net(const DevModel &m) { return m.nl != 3; }

// A (the first hidden layer, or every other one of a deeper network) and B
template <int PREC>
static size_t predict_smem(const DevModel &m) {
    return deep_net(m) ? 2 * hidden_bytes<PREC>(m.hmax) : hidden_bytes<PREC>(m.h1) + hidden_bytes<PREC>(m.h2);
}

// the table [256][CH] (A aliases it; every hidden width is <= 256) and B
template <int PREC>
static size_t decode_smem(const DevModel &m) {
    return (size_t)kSymbols * kCH * 4 + hidden_bytes<PREC>(deep_net(m) ? m.hmax : m.h2);
}

template <int PREC, bool DEEP>
static cudaError_t predict_cc(const DevModel &m, const EncBatch &b, cudaStream_t st) {
    const size_t sm = predict_smem<PREC>(m);
    cudaError_t e = cudaFuncSetAttribute(k_predict_cc<PREC, DEEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_predict_cc<PREC, DEEP><<<b.total_tiles, kCH, sm, st>>>(m, b);
    return cudaGetLastError();
}

template <int PREC, bool DEEP>
static cudaError_t decode_cc(const DevModel &m, const DecBatch &b, cudaStream_t st) {
    const size_t sm = decode_smem<PREC>(m);
    void (*kern)(DevModel, DecBatch) = DEEP ? k_decode_deep<PREC> : k_decode_cc<PREC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<b.n, DEEP ? kDeepThreads : kCH, sm, st>>>(m, b);
    return cudaGetLastError();
}

cudaError_t launch_predict_cc(const DevModel &m, const EncBatch &b, cudaStream_t st) {
    if (b.total_tiles == 0) return cudaSuccess;
    if (!default_window(m) && !(m.precision == DLIC_FP32 && f32_predict_supported(m))) return cudaErrorNotSupported;
    const bool deep = deep_net(m);
    if (m.precision == DLIC_FP32 && f32_predict_supported(m)) {
        // 64-pixel tiles, as the encoder plans them for the CUDA-core path
        const size_t sm = f32_predict_smem(m.h1, m.h2, (m.n_in + 15) / 16 * 16);
        cudaFuncSetAttribute(k_predict_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_predict_f32<<<b.total_tiles, kF32Threads, sm, st>>>(m, b);
        return cudaGetLastError();
    }
    if (m.precision == DLIC_FP32) return deep ? predict_cc<DLIC_FP32, true>(m, b, st) : predict_cc<DLIC_FP32, false>(m, b, st);
    return deep ? predict_cc<DLIC_INT8, true>(m, b, st) : predict_cc<DLIC_INT8, false>(m, b, st);
}

cudaError_t launch_decode_cc(const DevModel &m, const DecBatch &b, cudaStream_t st) {
    if (b.n == 0) return cudaSuccess;
    if (!default_window(m)) return cudaErrorNotSupported;   // one thread per pixel: the 12-prior window only
    const bool deep = deep_net(m);
    if (m.precision == DLIC_FP32) return deep ? decode_cc<DLIC_FP32, true>(m, b, st) : decode_cc<DLIC_FP32, false>(m, b, st);
    return deep ? decode_cc<DLIC_INT8, true>(m, b, st) : decode_cc<DLIC_INT8, false>(m, b, st);
}

}  // namespace dlic
