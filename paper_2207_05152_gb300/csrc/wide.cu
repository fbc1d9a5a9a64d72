// Networks with hidden layers wider than the layer-table kernels hold
// (Sec. II-B "Neural Network Architecture": 128 to 4096 neurons per hidden
// layer; the one-pixel-per-thread encoder and the unit-split decoder keep a
// pixel's activations on chip and stop at 256).  Here the network runs one
// layer at a time over a set of pixels, with the activations in the
// workspace:
//   - encode: every pixel is known, so the sets are chunks of up to
//     kWideChunk pixels in raster order; per chunk the inputs, one GEMM-like
//     kernel per dense layer, then one warp per pixel for the frequency table
//     of the pixel's own value;
//   - decode: the sets are the waves t = 3r + c (Sec. II-B "Preprocessor"),
//     enqueued one after another on the stream (the stream order is the
//     wavefront's dependency order): inputs gathered from the pixels already
//     decoded into the output image, the layers, then one warp per stream of
//     the wave for the table, the slot search and the rANS step, which writes
//     the pixel.  Stream states are the grid decoder's (set up and checked by
//     its set-up and finish kernels).
// The arithmetic is that of the other kernels, so bitstreams are identical:
// FP32 units start at their bias and accumulate fma(x_k, w_jk, acc) for k
// ascending (one thread per output, K walked in order through shared-memory
// chunks); INT8 units are exact integer dot products (dp4a) requantised as
// clamp(rint(fma(acc, s, o)), 0, 255), logits fma(acc, s, o).
#include <algorithm>

#include "coder_device.cuh"

namespace dlic {

constexpr int kWideChunk = 4096;     // pixels per pass through the layers
// (the INT8 encoder's tensor-core passes: 1024 tiles of its 4096 x 4096
// layers, enough to spread evenly over the SMs)
constexpr int kWideChunkTc = 8192;
constexpr int kWideTileP = 128, kWideTileU = 64, kWideKC = 32, kWideThreads = 256;

// The pixels of one pass: np pixels in raster order from p0 (encode), or the
// np pixels of wave t in rows r0, r0 + 1, ... (decode).
struct WideSet {
    const uint8_t *img;   // where the priors are read (the image being coded, or the output being decoded)
    int64_t pitch;
    int H, W;
    int wave;
    int64_t p0;
    int t, r0, np;
};

__device__ __forceinline__ void wide_pixel(const WideSet &q, int i, int &r, int &c) {
    if (q.wave) {
        r = q.r0 + i;
        c = q.t - 3 * r;
    } else {
        const int64_t p = q.p0 + i;
        r = (int)(p / q.W);
        c = (int)(p % q.W);
    }
}

// Network inputs of the set's pixels, [np][kPriors]: the default window's
// priors (two rows above at columns c-2..c+2, then (r, c-2), (r, c-1); 0
// outside the image) as v/128 - 1 (FP32) or v - 128 as signed bytes (INT8);
__global__ void k_wide_inputs(WideSet q, int prec, void *X) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= q.np * kPriors) return;
    const int i = idx / kPriors, k = idx % kPriors;
    int r, c;
    wide_pixel(q, i, r, c);
    const int dr = k < 5 ? -2 : (k < 10 ? -1 : 0);
    const int dc = k < 5 ? k - 2 : (k < 10 ? k - 7 : k - 12);
    const int rr = r + dr, cc = c + dc;
    const uint32_t v = rr >= 0 && cc >= 0 && cc < q.W ? q.img[(int64_t)rr * q.pitch + cc] : 0u;
    if (prec == DLIC_FP32)
        static_cast<float *>(X)[idx] = __fmaf_rn((float)v, 0.0078125f, -1.0f);
    else
        static_cast<uint8_t *>(X)[idx] = (uint8_t)(v ^ 0x80u);
}

// One FP32 dense layer over np pixels: Y[p][j] = act(b_j + sum_k X[p][k]
// W[j][k]) with the weights transposed Wt[k][j].  A CTA computes 128 pixels x
// 64 units, a thread 8 pixels x 4 units, K in chunks of 32 through shared
// memory; each accumulator is one thread's, bias first and k ascending.
__global__ void __launch_bounds__(kWideThreads) k_wide_f32(const float *X, int ldx, int K, const float *Wt,
                                                           const float *bias, int N, float *Y, int ldy, int np,
                                                           int relu) {
    __shared__ __align__(16) float xs[kWideKC][kWideTileP + 4];
    __shared__ __align__(16) float ws[kWideKC][kWideTileU];
    const int tid = threadIdx.x, tc = tid % 16, tr = tid / 16;
    const int p0 = blockIdx.x * kWideTileP, u0 = blockIdx.y * kWideTileU;
    float acc[8][4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int j = u0 + 4 * tc + u;
        const float bj = j < N ? bias[j] : 0.0f;
#pragma unroll
        for (int p = 0; p < 8; p++) acc[p][u] = bj;
    }
    for (int k0 = 0; k0 < K; k0 += kWideKC) {
        const int kn = min(kWideKC, K - k0);
        for (int e = tid; e < kWideTileP * kWideKC; e += kWideThreads) {
            const int p = e / kWideKC, kk = e % kWideKC;
            xs[kk][p] = p0 + p < np && kk < kn ? X[(size_t)(p0 + p) * ldx + k0 + kk] : 0.0f;
        }
        for (int e = tid; e < kWideKC * kWideTileU; e += kWideThreads) {
            const int kk = e / kWideTileU, u = e % kWideTileU;
            ws[kk][u] = kk < kn && u0 + u < N ? Wt[(size_t)(k0 + kk) * N + u0 + u] : 0.0f;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kn; kk++) {
            const float4 xa = *reinterpret_cast<const float4 *>(&xs[kk][8 * tr]);
            const float4 xb = *reinterpret_cast<const float4 *>(&xs[kk][8 * tr + 4]);
            const float4 w = *reinterpret_cast<const float4 *>(&ws[kk][4 * tc]);
            const float x[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
            const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int p = 0; p < 8; p++)
#pragma unroll
                for (int u = 0; u < 4; u++) acc[p][u] = __fmaf_rn(x[p], wv[u], acc[p][u]);
        }
        __syncthreads();
    }
    const int j = u0 + 4 * tc;
    if (j >= N) return;   // N is a multiple of 4
#pragma unroll
    for (int p = 0; p < 8; p++) {
        const int pp = p0 + 8 * tr + p;
        if (pp >= np) break;
        float o[4];
#pragma unroll
        for (int u = 0; u < 4; u++) o[u] = relu ? (acc[p][u] > 0.0f ? acc[p][u] : 0.0f) : acc[p][u];
        *reinterpret_cast<float4 *>(Y + (size_t)pp * ldy + j) = make_float4(o[0], o[1], o[2], o[3]);
    }
}

// One INT8 dense layer: acc_j = sum_k x_k q_jk exactly (dp4a over the packed
// weights Q[k4][j]; signed inputs for the first layer, u8 units after), then
// the requantised u8 unit (hidden) or the logit fma(acc, s, o) (output, FP32
// into Y).  X and hidden Y are bytes [np][ld], ld a multiple of 4; with
// bf16out a hidden unit u goes out as the tensor-core layers' input, the
// exact bf16(u) (Y as uint16 [np][ldy]).
__global__ void __launch_bounds__(kWideThreads) k_wide_i8(const uint8_t *X, int ldx, int K4, const uint32_t *Q,
                                                          const float *s, const float *o, int N, void *Y, int ldy,
                                                          int np, int first, int logits, int bf16out) {
    __shared__ uint32_t xs[kWideKC][kWideTileP + 4];
    __shared__ __align__(16) uint32_t ws[kWideKC][kWideTileU];
    const int tid = threadIdx.x, tc = tid % 16, tr = tid / 16;
    const int p0 = blockIdx.x * kWideTileP, u0 = blockIdx.y * kWideTileU;
    int acc[8][4] = {};
    for (int k0 = 0; k0 < K4; k0 += kWideKC) {
        const int kn = min(kWideKC, K4 - k0);
        for (int e = tid; e < kWideTileP * kWideKC; e += kWideThreads) {
            const int p = e / kWideKC, kk = e % kWideKC;
            xs[kk][p] = p0 + p < np && kk < kn ? reinterpret_cast<const uint32_t *>(X + (size_t)(p0 + p) * ldx)[k0 + kk]
                                               : 0u;
        }
        for (int e = tid; e < kWideKC * kWideTileU; e += kWideThreads) {
            const int kk = e / kWideTileU, u = e % kWideTileU;
            ws[kk][u] = kk < kn && u0 + u < N ? Q[(size_t)(k0 + kk) * N + u0 + u] : 0u;
        }
        __syncthreads();
        for (int kk = 0; kk < kn; kk++) {
            const uint4 w = *reinterpret_cast<const uint4 *>(&ws[kk][4 * tc]);
            const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int p = 0; p < 8; p++) {
                const uint32_t x = xs[kk][8 * tr + p];
#pragma unroll
                for (int u = 0; u < 4; u++) acc[p][u] = first ? dp4a_ss(x, wv[u], acc[p][u]) : dp4a_us(x, wv[u], acc[p][u]);
            }
        }
        __syncthreads();
    }
    const int j = u0 + 4 * tc;
    if (j >= N) return;
    float sj[4], oj[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
        sj[u] = s[j + u];
        oj[u] = o[j + u];
    }
#pragma unroll
    for (int p = 0; p < 8; p++) {
        const int pp = p0 + 8 * tr + p;
        if (pp >= np) break;
        if (logits) {
            float z[4];
#pragma unroll
            for (int u = 0; u < 4; u++) z[u] = __fmaf_rn(__int2float_rn(acc[p][u]), sj[u], oj[u]);
            *reinterpret_cast<float4 *>(static_cast<float *>(Y) + (size_t)pp * ldy + j) = make_float4(z[0], z[1], z[2], z[3]);
        } else if (bf16out) {
            uint32_t pk[2] = {0u, 0u};
#pragma unroll
            for (int u = 0; u < 4; u++)
                pk[u >> 1] |= (__float_as_uint((float)requant_u8(acc[p][u], sj[u], oj[u])) >> 16) << (16 * (u & 1));
            *reinterpret_cast<uint2 *>(static_cast<uint16_t *>(Y) + (size_t)pp * ldy + j) = make_uint2(pk[0], pk[1]);
        } else {
            uint32_t packed = 0;
#pragma unroll
            for (int u = 0; u < 4; u++) packed |= requant_u8(acc[p][u], sj[u], oj[u]) << (8 * u);
            *reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(Y) + (size_t)pp * ldy + j) = packed;
        }
    }
}

// A pixel's 256 logits, eight per lane (values 8 lane .. 8 lane + 7), and
// their table weights w_i (see coder_device.cuh) with the row maximum.
__device__ __forceinline__ void wide_weights(const DevModel &m, const float *z, const uint32_t *lut2, uint32_t (&w)[8]) {
    const int lane = threadIdx.x & 31;
    const float4 za = *reinterpret_cast<const float4 *>(z + 8 * lane);
    const float4 zc = *reinterpret_cast<const float4 *>(z + 8 * lane + 4);
    const float v[8] = {za.x, za.y, za.z, za.w, zc.x, zc.y, zc.z, zc.w};
    float lmax = v[0];
#pragma unroll
    for (int q = 1; q < 8; q++) lmax = fmaxf(lmax, v[q]);
    const float mx = key_float(__reduce_max_sync(0xffffffffu, float_key(lmax)));
#pragma unroll
    for (int q = 0; q < 8; q++) w[q] = table_weight2(mx, v[q], m.tscale, lut2);
}

// Encode: the table entry (f | c << 16) of each set pixel's own value, one
// warp per pixel, into fc (stream order, or raster order for dlic_predict).
__global__ void __launch_bounds__(kWideThreads) k_wide_table_enc(DevModel m, WideSet q, const float *Z, uint32_t *fc,
                                                                 int S, int raster) {
    __shared__ uint32_t lut2[kTableSteps];
    expand_lut(m.lut, lut2, threadIdx.x, kWideThreads);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (kWideThreads / 32) + (threadIdx.x >> 5);
    if (i >= q.np) return;
    int r, c;
    wide_pixel(q, i, r, c);
    const int sym = q.img[(int64_t)r * q.pitch + c];
    uint32_t w[8];
    wide_weights(m, Z + (size_t)i * kSymbols, lut2, w);
    uint32_t lsum = 0, lp = 0, lw = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int v = 8 * lane + k;
        lsum += w[k];
        lp += v < sym ? w[k] : 0u;
        lw = v == sym ? w[k] : lw;
    }
    const uint32_t W = __reduce_add_sync(0xffffffffu, lsum);
    const uint32_t Ps = __reduce_add_sync(0xffffffffu, lp);
    const uint32_t ws = __reduce_add_sync(0xffffffffu, lw);
    if (lane == 0) {
        const uint32_t Q = table_q(W);
        const uint32_t c_lo = (uint32_t)sym + __umulhi(Ps, Q);
        const uint32_t c_hi = sym == kSymbols - 1 ? kTotal : (uint32_t)sym + 1u + __umulhi(Ps + ws, Q);
        fc[raster ? (int64_t)r * q.W + c : stream_index(q.H, q.W, S, r, c)] = (c_hi - c_lo) | (c_lo << 16);
    }
}

// Decode: the wave's pixels of one image, one warp per stream (pixels i, i
// + S, ... of the wave share stream (r0 + i) mod S and go in row order): the
// table, the symbol whose range holds the slot x mod 2^16 (the last value
// whose lower boundary c_i does not exceed it), the rANS step, the pixel to
// the output image.  Stream states as the grid decoder keeps them; a
// container that its set-up refused (ok flag 0) is skipped.
struct WideDecState {
    uint32_t *hdr, *x, *pos, *end;
    const uint16_t *words;   // the input, as 16-bit words
    int32_t *status;
    uint8_t *out;
    int64_t pitch;
};
__global__ void __launch_bounds__(kWideThreads) k_wide_table_dec(DevModel m, WideSet q, const float *Z,
                                                                 WideDecState d) {
    __shared__ uint32_t lut2[kTableSteps];
    if (!d.hdr[1]) return;
    expand_lut(m.lut, lut2, threadIdx.x, kWideThreads);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int S = (int)d.hdr[0];
    const int g = blockIdx.x * (kWideThreads / 32) + (threadIdx.x >> 5);
    if (g >= min(q.np, S)) return;
    for (int i = g; i < q.np; i += S) {
        int r, c;
        wide_pixel(q, i, r, c);
        const int s = r % S;
        uint32_t w[8];
        wide_weights(m, Z + (size_t)i * kSymbols, lut2, w);
        uint32_t lsum = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) lsum += w[k];
        const uint32_t Wsum = __reduce_add_sync(0xffffffffu, lsum);
        const uint32_t Q = table_q(Wsum);
        uint32_t incl = lsum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        const uint32_t excl = incl - lsum;
        const uint32_t x = d.x[s];
        const uint32_t slot = x & 0xFFFFu;
        // c at the lane's first value; the slot's lane is the last one whose
        // first boundary does not exceed it
        const uint32_t ball = __ballot_sync(0xffffffffu, 8u * lane + __umulhi(excl, Q) <= slot);
        const int Lh = 31 - __clz(ball);
        uint32_t cb[9], Pp = excl;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            cb[k] = 8u * lane + k + __umulhi(Pp, Q);
            Pp += w[k];
        }
        cb[8] = lane == 31 ? kTotal : 8u * lane + 8u + __umulhi(Pp, Q);
        uint32_t sym = 8u * lane, f = cb[1] - cb[0], clo = cb[0];
#pragma unroll
        for (int k = 1; k < 8; k++)
            if (cb[k] <= slot) {
                sym = 8u * lane + k;
                f = cb[k + 1] - cb[k];
                clo = cb[k];
            }
        sym = __shfl_sync(0xffffffffu, sym, Lh);
        f = __shfl_sync(0xffffffffu, f, Lh);
        clo = __shfl_sync(0xffffffffu, clo, Lh);
        if (lane == 0) {
            uint32_t xn = f * (x >> 16) + slot - clo;
            if (xn < kRansL) {
                const uint32_t pos = d.pos[s];
                if (pos < d.end[s]) {
                    xn = (xn << 16) | d.words[pos];
                    d.pos[s] = pos + 1;
                } else {
                    atomicMax(d.status, (int)DLIC_ERR_CORRUPT);
                }
            }
            d.x[s] = xn;
            d.out[(int64_t)r * d.pitch + c] = (uint8_t)sym;
        }
        __syncwarp();
    }
}

bool wide_supported(const DevModel &m) { return m.bits == 8 && m.hmax > kMaxHidden; }

namespace {

// The scratch of one pass (kWideChunk pixels): two activation buffers of
// hmax units, the logits Z [pixel][256] (FP32) and the inputs X.  With
// bf16 (the INT8 encoder) an activation buffer holds the tensor-core
// layers' bf16 inputs [kWideChunk][hpad].
struct WideScratch {
    uint8_t *A, *B, *X;
    float *Z;
    size_t bytes;
    int hpad;
};
WideScratch wide_scratch(const DevModel &m, uint8_t *base, bool bf16) {
    auto a256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const int hpad = (m.hmax + 63) / 64 * 64;
    const size_t chunk = bf16 ? kWideChunkTc : kWideChunk;
    const size_t act = bf16 ? a256(chunk * hpad * 2) : a256(chunk * m.hmax * (m.precision == DLIC_FP32 ? 4 : 1));
    WideScratch w;
    w.hpad = hpad;
    w.A = base;
    w.B = base + act;
    w.Z = reinterpret_cast<float *>(base + 2 * act);
    w.X = base + 2 * act + a256(chunk * kSymbols * 4);
    w.bytes = 2 * act + a256(chunk * kSymbols * 4) + a256(chunk * kPriors * 4);
    return w;
}

// Inputs and every layer of the network over one set (np <= kWideChunk, or
// kWideChunkTc with tc);
// the logits land in Z.  tc (INT8, encode): the layers after the first on
// the tensor cores (wide_tc.cu), their inputs as bf16.
cudaError_t wide_network(const DevModel &m, const DevLayer *hl, const WideSet &q, uint8_t *scratch, bool tc,
                         int *err, cudaStream_t st) {
    const WideScratch w = wide_scratch(m, scratch, tc);
    uint8_t *A = w.A, *B = w.B, *X = w.X;
    float *Z = w.Z;
    k_wide_inputs<<<(q.np * kPriors + 255) / 256, 256, 0, st>>>(q, m.precision, X);
    if (tc) {
        // the first layer (K = the 12 signed priors: too short a contraction
        // for the tensor cores to gain) by dp4a into A as bf16, then every
        // later layer on the tensor cores, B and A in turn, the logits into Z
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const DevLayer &l0 = hl[0];
        const dim3 grid((q.np + kWideTileP - 1) / kWideTileP, (l0.n_out + kWideTileU - 1) / kWideTileU);
        k_wide_i8<<<grid, kWideThreads, 0, st>>>(X, kPriors, (l0.n_in + 3) / 4, static_cast<const uint32_t *>(l0.w),
                                                 l0.a, l0.o, l0.n_out, A, w.hpad, q.np, 1, 0, 1);
        cudaError_t e = cudaGetLastError();
        for (int l = 1; l < m.nl && e == cudaSuccess; l++) {
            const bool last = l == m.nl - 1;
            const uint16_t *in = reinterpret_cast<const uint16_t *>(l & 1 ? A : B);
            void *out = last ? static_cast<void *>(Z) : static_cast<void *>(l & 1 ? B : A);
            e = launch_wide_tc(hl[l], in, w.hpad, q.np, out, last ? kSymbols : w.hpad, last, sms, err, st);
        }
        return e;
    }
    const uint8_t *in = X;
    int ldin = kPriors;
    for (int l = 0; l < m.nl; l++) {
        const DevLayer &ly = hl[l];
        const bool last = l == m.nl - 1;
        uint8_t *out = last ? reinterpret_cast<uint8_t *>(Z) : (l & 1 ? B : A);
        const dim3 grid((q.np + kWideTileP - 1) / kWideTileP, (ly.n_out + kWideTileU - 1) / kWideTileU);
        if (m.precision == DLIC_FP32)
            k_wide_f32<<<grid, kWideThreads, 0, st>>>(reinterpret_cast<const float *>(in), ldin, ly.n_in,
                                                      static_cast<const float *>(ly.w), ly.a, ly.n_out,
                                                      reinterpret_cast<float *>(out), ly.n_out, q.np, !last);
        else
            k_wide_i8<<<grid, kWideThreads, 0, st>>>(in, ldin, (ly.n_in + 3) / 4, static_cast<const uint32_t *>(ly.w),
                                                     ly.a, ly.o, ly.n_out, out, ly.n_out, q.np, l == 0, last, 0);
        in = out;
        ldin = ly.n_out;
    }
    return cudaGetLastError();
}

}  // namespace

// whether the layers after the first run on the tensor cores (INT8)
static bool wide_tc_layers(const DevModel &m, const DevLayer *hl) {
    if (m.precision != DLIC_INT8) return false;
    for (int l = 1; l < m.nl; l++)
        if (!hl || !hl[l].wtc) return false;
    return true;
}

size_t wide_scratch_bytes(const DevModel &m, bool encode) {
    (void)encode;   // INT8 networks run their wide layers on the tensor cores in both directions
    return wide_supported(m) ? wide_scratch(m, nullptr, m.precision == DLIC_INT8).bytes : 0;
}

cudaError_t launch_predict_wide(const DevModel &m, const DevLayer *hl, const EncBatch &b, uint8_t *scratch, int *err,
                                cudaStream_t st) {
    // (the workspace holds bf16 activations whenever the network is INT8)
    const bool tc = wide_tc_layers(m, hl);
    for (int k = 0; k < b.n; k++) {
        const EncImage &im = b.img[k];
        const int64_t N = (int64_t)im.H * im.W;
        uint32_t *fc = reinterpret_cast<uint32_t *>(b.ws + im.fc_off);
        const int64_t chunk = tc ? kWideChunkTc : kWideChunk;
        for (int64_t p0 = 0; p0 < N; p0 += chunk) {
            const WideSet q{im.pixels, im.pitch, im.H, im.W, 0, p0, 0, 0, (int)std::min<int64_t>(chunk, N - p0)};
            cudaError_t e = wide_network(m, hl, q, scratch, tc, err, st);
            if (e != cudaSuccess) return e;
            k_wide_table_enc<<<(q.np + 7) / 8, kWideThreads, 0, st>>>(m, q, wide_scratch(m, scratch, tc).Z, fc, im.S,
                                                                       b.raster);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_decode_wide(const DevModel &m, const DevLayer *hl, const DecBatch &b, uint8_t *scratch,
                               cudaStream_t st) {
    cudaError_t e = launch_batch_setup(m, b, st);
    if (e != cudaSuccess) return e;
    // INT8: the layers after the first on the tensor cores, as in the encoder
    // (the same exact integer sums, so the same tables)
    const bool tc = wide_tc_layers(m, hl);
    const float *Z = wide_scratch(m, scratch, tc).Z;
    for (int k = 0; k < b.n && e == cudaSuccess; k++) {
        const DecImage &im = b.img[k];
        WideDecState d;
        d.hdr = reinterpret_cast<uint32_t *>(b.ws + im.st_off);
        d.x = d.hdr + 64;
        d.pos = d.x + (size_t)im.D * im.S;
        d.end = d.pos + (size_t)im.D * im.S;
        d.words = reinterpret_cast<const uint16_t *>(b.in);
        d.status = b.status + im.sidx;
        d.out = im.pixels;
        d.pitch = im.pitch;
        const int H = im.H, W = im.W, T = 3 * (H - 1) + W;
        for (int t = 0; t < T && e == cudaSuccess; t++) {
            // rows r with 0 <= t - 3r < W
            const int r_lo = t - W + 1 > 0 ? (t - W + 3) / 3 : 0, r_hi = std::min(H - 1, t / 3);
            for (int r0 = r_lo; r0 <= r_hi && e == cudaSuccess; r0 += kWideChunk) {
                const int np = std::min(kWideChunk, r_hi - r0 + 1);
                const WideSet q{im.pixels, im.pitch, H, W, 1, 0, t, r0, np};
                e = wide_network(m, hl, q, scratch, tc, b.status + im.sidx, st);
                if (e != cudaSuccess) break;
                // one warp per stream of the pass (at most H streams)
                const int warps = std::min(np, H);
                k_wide_table_dec<<<(warps + 7) / 8, kWideThreads, 0, st>>>(m, q, Z, d);
                e = cudaGetLastError();
            }
        }
    }
    if (e == cudaSuccess) e = launch_batch_finish(b, st);
    return e;
}

}  // namespace dlic
