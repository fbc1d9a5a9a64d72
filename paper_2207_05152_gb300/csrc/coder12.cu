// Coding kernels for 12-bit pixels (Sec. IV "Higher Bit Depth": one 12-bit
// channel, a network of 4096 output neurons, one per value).  FP32 networks
// of any depth, read from the model's layer table, on the CUDA cores.
//
// Samples are u16 (0..4095); row r of an image starts at pixels + r * pitch
// bytes.  Network inputs are v / 2048 - 1 (exact in FP32).  The frequency
// table is the 8-bit one over K = 4096 values: m = max z,
// u_i = rint(min((m - z_i) tscale, 1535)), w_i = lut[u_i mod 64] >> (u_i div 64),
// W = sum w_i, Q = floor((2^16 - 4096) 2^32 / W), c_i = i + floor(P_i Q / 2^32)
// with P_i = sum_{j<i} w_j, c_4096 = 2^16.  W and P_i reach 2^35, so they
// and the products P_i Q (< 2^60) are 64-bit.  Every FP32 unit starts from
// its bias and accumulates fma(x_k, w_jk, acc) for k ascending, so the
// encoder and the decoder compute the same logits bit for bit.
#include "coder_device.cuh"
#include "decode_setup.cuh"

namespace dlic {

constexpr int k12Warps = 8, k12Threads = 32 * k12Warps;
constexpr int k12PixPerWarp = 8;                       // encoder: pixels per warp (register tile)
constexpr int k12Tile = k12Warps * k12PixPerWarp;      // encoder: pixels per CTA
static_assert(k12Tile == kPredictTile, "the encoder plans CUDA-core tiles of kPredictTile pixels");
constexpr uint64_t k12Slack = kTotal - kSymbols12;     // 2^16 - 4096: the table's free mass
constexpr int k12InPitch = 16;                         // encoder: floats per pixel of the input rows
constexpr int k12PerLane = kSymbols12 / 32;            // decoder: consecutive values each lane searches
constexpr int k12Chains = 8;                           // decoder: logits each lane computes side by side
static_assert(kSymbols12 % (32 * k12Chains) == 0, "the logit loop covers the values in whole steps");

__device__ __forceinline__ uint32_t px12(const uint8_t *img, int64_t pitch, int r, int c) {
    return *reinterpret_cast<const uint16_t *>(img + (int64_t)r * pitch + 2 * (int64_t)c);
}

// Network inputs of the default window (the prior order of gather_priors),
// 0 outside the image (Fig. 1 right).
__device__ __forceinline__ float input12(const uint8_t *img, int64_t pitch, int H, int W, int r, int c, int k) {
    const int dr = k < 5 ? -2 : (k < 10 ? -1 : 0);
    const int dc = k < 5 ? k - 2 : (k < 10 ? k - 7 : k - 12);
    const int rr = r + dr, cc = c + dc;
    const uint32_t v = (rr >= 0 && rr < H && cc >= 0 && cc < W) ? px12(img, pitch, rr, cc) : 0u;
    return __fmaf_rn((float)v, 0.00048828125f, -1.0f);   // v / 2048 - 1
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float o = __shfl_xor_sync(0xffffffffu, v, off);
        v = o > v ? o : v;
    }
    return v;
}

__device__ __forceinline__ uint64_t warp_sum64(uint64_t v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ uint64_t table_q12(uint64_t W) { return W ? (k12Slack << 32) / W : 0ull; }

// ---------------------------------------------------------------------------
// Encoder prediction: 64 pixels per CTA, 8 per warp.  Each lane computes
// units lane, lane + 32, ... of every layer for the warp's 8 pixels (one
// weight load, 8 FMAs).  The 4096 logits are computed twice: the first pass
// finds each pixel's maximum, the second turns the logits into weights and
// sums W, P of the pixel's own value and its weight.
// Shared memory per warp: inputs [8][16], two activation buffers [8][hmax].
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t predict12_warp_floats(int hmax) {
    return (size_t)k12PixPerWarp * k12InPitch + 2 * (size_t)k12PixPerWarp * hmax;
}

__global__ void __launch_bounds__(k12Threads) k_predict12(DevModel m, EncBatch b, int *err) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t lut2[kTableSteps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    expand_lut(m.lut, lut2, tid, k12Threads);
    __syncthreads();

    const int tile = blockIdx.x;
    int ii = 0;
    while (ii + 1 < b.n && b.img[ii + 1].tile_begin <= tile) ii++;
    const EncImage &im = b.img[ii];
    const int64_t npx = (int64_t)im.H * im.W;
    const int64_t p0 = (int64_t)(tile - im.tile_begin) * k12Tile + (int64_t)warp * k12PixPerWarp;
    if (p0 >= npx) return;   // the whole warp past the image (no CTA barrier follows)
    const int hmax = m.hmax;
    float *xin = reinterpret_cast<float *>(smem) + (size_t)warp * predict12_warp_floats(hmax);
    float *bufA = xin + k12PixPerWarp * k12InPitch;
    float *bufB = bufA + (size_t)k12PixPerWarp * hmax;

    int rr[k12PixPerWarp], cc[k12PixPerWarp];
#pragma unroll
    for (int p = 0; p < k12PixPerWarp; p++) {
        const int64_t pp = p0 + p < npx ? p0 + p : p0;   // pixels past the image repeat the first
        rr[p] = (int)(pp / im.W);
        cc[p] = (int)(pp % im.W);
    }
    for (int i = lane; i < k12PixPerWarp * kPriors; i += 32) {
        const int p = i / kPriors, k = i % kPriors;
        int r = 0, c = 0;
#pragma unroll
        for (int q = 0; q < k12PixPerWarp; q++)
            if (q == p) {
                r = rr[q];
                c = cc[q];
            }
        xin[p * k12InPitch + k] = input12(im.pixels, im.pitch, im.H, im.W, r, c, k);
    }
    __syncwarp();

    // hidden layers
    const int L = m.nl - 1;
    const float *in = xin;
    int ld_in = k12InPitch;
    float *out = bufA;
    for (int l = 0; l < L; l++) {
        const DevLayer ly = m.layers[l];
        const float *wt = static_cast<const float *>(ly.w);
        for (int u = lane; u < ly.n_out; u += 32) {
            float acc[k12PixPerWarp];
            const float bias = __ldg(ly.a + u);
#pragma unroll
            for (int p = 0; p < k12PixPerWarp; p++) acc[p] = bias;
            for (int k = 0; k < ly.n_in; k++) {
                const float w = __ldg(wt + (size_t)k * ly.n_out + u);
#pragma unroll
                for (int p = 0; p < k12PixPerWarp; p++) acc[p] = __fmaf_rn(in[p * ld_in + k], w, acc[p]);
            }
#pragma unroll
            for (int p = 0; p < k12PixPerWarp; p++) out[p * hmax + u] = acc[p] > 0.0f ? acc[p] : 0.0f;
        }
        __syncwarp();
        in = out;
        ld_in = hmax;
        out = out == bufA ? bufB : bufA;
    }

    // output layer, pass 1: the maximum logit of each pixel
    const DevLayer lo = m.layers[L];
    const float *wo = static_cast<const float *>(lo.w);
    const int hl = lo.n_in;
    float mx[k12PixPerWarp];
#pragma unroll
    for (int p = 0; p < k12PixPerWarp; p++) mx[p] = -INFINITY;
    for (int i = lane; i < kSymbols12; i += 32) {
        float acc[k12PixPerWarp];
        const float bias = __ldg(lo.a + i);
#pragma unroll
        for (int p = 0; p < k12PixPerWarp; p++) acc[p] = bias;
        for (int k = 0; k < hl; k++) {
            const float w = __ldg(wo + (size_t)k * kSymbols12 + i);
#pragma unroll
            for (int p = 0; p < k12PixPerWarp; p++) acc[p] = __fmaf_rn(in[p * ld_in + k], w, acc[p]);
        }
#pragma unroll
        for (int p = 0; p < k12PixPerWarp; p++) mx[p] = acc[p] > mx[p] ? acc[p] : mx[p];
    }
#pragma unroll
    for (int p = 0; p < k12PixPerWarp; p++) mx[p] = warp_max(mx[p]);

    // pass 2: the same logits, their weights, W, P below the pixel's value and its weight
    uint32_t sym[k12PixPerWarp], wl[k12PixPerWarp], pl[k12PixPerWarp], ws[k12PixPerWarp];
#pragma unroll
    for (int p = 0; p < k12PixPerWarp; p++) {
        sym[p] = px12(im.pixels, im.pitch, rr[p], cc[p]);
        wl[p] = pl[p] = ws[p] = 0u;   // lane sums of at most 128 weights of <= 2^23
    }
    for (int i = lane; i < kSymbols12; i += 32) {
        float acc[k12PixPerWarp];
        const float bias = __ldg(lo.a + i);
#pragma unroll
        for (int p = 0; p < k12PixPerWarp; p++) acc[p] = bias;
        for (int k = 0; k < hl; k++) {
            const float w = __ldg(wo + (size_t)k * kSymbols12 + i);
#pragma unroll
            for (int p = 0; p < k12PixPerWarp; p++) acc[p] = __fmaf_rn(in[p * ld_in + k], w, acc[p]);
        }
#pragma unroll
        for (int p = 0; p < k12PixPerWarp; p++) {
            const uint32_t w = table_weight2(mx[p], acc[p], m.tscale, lut2);
            wl[p] += w;
            pl[p] += (uint32_t)i < sym[p] ? w : 0u;
            ws[p] = (uint32_t)i == sym[p] ? w : ws[p];
        }
    }
    uint32_t *fc = reinterpret_cast<uint32_t *>(b.ws + im.fc_off);
#pragma unroll
    for (int p = 0; p < k12PixPerWarp; p++) {
        const uint64_t Wt = warp_sum64(wl[p]), Ps = warp_sum64(pl[p]), Wsym = warp_sum64(ws[p]);
        if (lane == p && p0 + p < npx) {
            // a sample above 4095 has no table entry: the image is refused
            if (sym[p] >= (uint32_t)kSymbols12) atomicCAS(err, DLIC_OK, DLIC_ERR_INVALID);
            const uint64_t Q = table_q12(Wt);
            const uint32_t c_lo = sym[p] + (uint32_t)((Ps * Q) >> 32);
            const uint32_t c_hi =
                sym[p] == kSymbols12 - 1 ? kTotal : sym[p] + 1u + (uint32_t)(((Ps + Wsym) * Q) >> 32);
            fc[b.raster ? (int64_t)rr[p] * im.W + cc[p] : stream_index(im.H, im.W, im.S, rr[p], cc[p])] =
                (c_hi - c_lo) | (c_lo << 16);
        }
    }
}

// ---------------------------------------------------------------------------
// Wavefront decoder (Sec. II-B "Preprocessor"): one CTA of 8 warps per
// image.  The pixels of wave t = 3r + c go to the warps in chunks of 8, one
// pixel per warp: the warp computes its network (lanes over units and
// values), keeps the 4096 logits in shared memory, turns them into weights
// in place, and each lane sums the weights of 128 consecutive values; a
// 64-bit warp scan gives the cumulative mass at every lane's first value.
// The rANS step then needs one lane: the one whose value range holds the
// slot walks its 128 values.  Pixels that share a stream (rows S apart) take
// their rANS steps in row order (rounds of the chunk, a CTA barrier each).
// Shared memory per warp: the table [4096] (logits, then weights) and two
// activation buffers [hmax].
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t decode12_warp_bytes(int hmax) { return 4ull * kSymbols12 + 8ull * hmax; }

__global__ void __launch_bounds__(k12Threads) k_decode12(DevModel m, DecBatch b) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t lut2[kTableSteps];
    __shared__ int s_err;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DecImage &im = b.img[blockIdx.x];
    expand_lut(m.lut, lut2, tid, k12Threads);
    if (tid == 0) s_err = 0;
    StreamState *st = reinterpret_cast<StreamState *>(b.ws + im.st_off);
    const uint8_t *in = b.in + im.in_off;
    int S;
    const uint16_t *pay;
    if (!decode_setup(m, im, in, st, &S, &pay)) {   // its barriers also publish lut2 and s_err
        if (tid == 0) b.status[im.sidx] = DLIC_ERR_CORRUPT;
        return;
    }
    const int hmax = m.hmax;
    uint8_t *wbase = smem + (size_t)warp * decode12_warp_bytes(hmax);
    float *zs = reinterpret_cast<float *>(wbase);         // logits, then (as u32) the weights
    uint32_t *wts = reinterpret_cast<uint32_t *>(wbase);
    float *hA = reinterpret_cast<float *>(wbase + 4ull * kSymbols12);
    float *hB = hA + hmax;
    const int L = m.nl - 1;
    const DevLayer lo = m.layers[L];
    const float *wo = static_cast<const float *>(lo.w);
    const int H = im.H, W = im.W;
    const int T = 3 * (H - 1) + W;
    for (int t = 0; t < T; t++) {
        if (s_err) break;
        const int r_lo = t - W + 1 > 0 ? (t - W + 3) / 3 : 0;
        const int r_hi = min(H - 1, t / 3);
        const int n_t = r_hi - r_lo + 1;
        for (int base = 0; base < n_t; base += k12Warps) {
            const int pix = base + warp;
            const bool active = pix < n_t;   // uniform over the warp
            const int r = r_lo + pix, c = t - 3 * r;
            uint64_t Q = 0, P0 = 0;
            uint32_t lsum = 0;
            if (active) {
                // hidden layers: layer 0 from the window in registers
                float x[kPriors];
#pragma unroll
                for (int k = 0; k < kPriors; k++) x[k] = input12(im.pixels, im.pitch, H, W, r, c, k);
                const float *hin = nullptr;
                float *hout = hA;
                for (int l = 0; l < L; l++) {
                    const DevLayer ly = m.layers[l];
                    const float *wt = static_cast<const float *>(ly.w);
                    for (int u = lane; u < ly.n_out; u += 32) {
                        float acc = __ldg(ly.a + u);
                        if (l == 0) {
#pragma unroll
                            for (int k = 0; k < kPriors; k++) acc = __fmaf_rn(x[k], __ldg(wt + (size_t)k * ly.n_out + u), acc);
                        } else {
                            for (int k = 0; k < ly.n_in; k++)
                                acc = __fmaf_rn(hin[k], __ldg(wt + (size_t)k * ly.n_out + u), acc);
                        }
                        hout[u] = acc > 0.0f ? acc : 0.0f;
                    }
                    __syncwarp();
                    hin = hout;
                    hout = hout == hA ? hB : hA;
                }
                // logits and their maximum: each lane runs eight values'
                // chains side by side (values i, i + 32, ..., i + 224)
                float mx = -INFINITY;
                for (int i = lane; i < kSymbols12; i += 32 * k12Chains) {
                    float acc[k12Chains];
#pragma unroll
                    for (int j = 0; j < k12Chains; j++) acc[j] = __ldg(lo.a + i + 32 * j);
                    for (int k = 0; k < lo.n_in; k++) {
                        const float hk = hin[k];
                        const float *wk = wo + (size_t)k * kSymbols12 + i;
#pragma unroll
                        for (int j = 0; j < k12Chains; j++) acc[j] = __fmaf_rn(hk, __ldg(wk + 32 * j), acc[j]);
                    }
#pragma unroll
                    for (int j = 0; j < k12Chains; j++) {
                        zs[i + 32 * j] = acc[j];
                        mx = acc[j] > mx ? acc[j] : mx;
                    }
                }
                mx = warp_max(mx);
                __syncwarp();
                // weights in place over the lane's consecutive values, and their sum
                const int i0 = k12PerLane * lane;
                for (int i = i0; i < i0 + k12PerLane; i++) {
                    const uint32_t w = table_weight2(mx, zs[i], m.tscale, lut2);
                    wts[i] = w;
                    lsum += w;
                }
                // inclusive scan of the lane sums: the mass below each lane's first value
                uint64_t incl = lsum;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint64_t o = __shfl_up_sync(0xffffffffu, incl, off);
                    if (lane >= off) incl += o;
                }
                P0 = incl - lsum;
                Q = table_q12(__shfl_sync(0xffffffffu, incl, 31));
            }
            const int rounds = (min(k12Warps, n_t - base) + S - 1) / S;
            for (int rnd = 0; rnd < rounds; rnd++) {
                if (active && warp / S == rnd) {
                    StreamState q = st[r % S];
                    const uint32_t slot = q.x & 0xFFFFu;
                    const int i0 = k12PerLane * lane;
                    const uint32_t c0 = (uint32_t)i0 + (uint32_t)((P0 * Q) >> 32);
                    const uint32_t c1 = lane == 31 ? kTotal
                                                   : (uint32_t)(i0 + k12PerLane) + (uint32_t)(((P0 + lsum) * Q) >> 32);
                    if (c0 <= slot && slot < c1) {   // exactly one lane: the ranges tile [0, 2^16)
                        uint64_t P = P0;
                        uint32_t c_lo = c0, f = 1;
                        int sym = i0 + k12PerLane - 1;
                        for (int i = i0; i < i0 + k12PerLane; i++) {
                            const uint32_t w = wts[i];
                            const uint32_t lo_i = (uint32_t)i + (uint32_t)((P * Q) >> 32);
                            const uint32_t hi_i =
                                i == kSymbols12 - 1 ? kTotal : (uint32_t)i + 1u + (uint32_t)(((P + w) * Q) >> 32);
                            if (hi_i > slot) {
                                sym = i;
                                c_lo = lo_i;
                                f = hi_i - lo_i;
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
                        *reinterpret_cast<uint16_t *>(im.pixels + (int64_t)r * im.pitch + 2 * (int64_t)c) =
                            (uint16_t)sym;
                    }
                }
                __syncthreads();
            }
        }
    }
    __syncthreads();
    // final states must be back at the initial value L with every word read
    for (int s = tid; s < S && !s_err; s += k12Threads) {
        const StreamState q = st[s];
        if (q.x != kRansL || q.pos != q.end) s_err = 1;
    }
    __syncthreads();
    if (tid == 0) b.status[im.sidx] = s_err ? DLIC_ERR_CORRUPT : DLIC_OK;
}

cudaError_t launch_predict12(const DevModel &m, const EncBatch &b, int *err, cudaStream_t st) {
    if (b.total_tiles == 0) return cudaSuccess;
    if (m.bits != 12 || m.precision != DLIC_FP32 || !default_window(m) || !m.layers) return cudaErrorNotSupported;
    const size_t sm = 4ull * k12Warps * predict12_warp_floats(m.hmax);
    cudaError_t e = cudaFuncSetAttribute(k_predict12, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_predict12<<<b.total_tiles, k12Threads, sm, st>>>(m, b, err);
    return cudaGetLastError();
}

cudaError_t launch_decode12(const DevModel &m, const DecBatch &b, cudaStream_t st) {
    if (b.n == 0) return cudaSuccess;
    if (m.bits != 12 || m.precision != DLIC_FP32 || !default_window(m) || !m.layers) return cudaErrorNotSupported;
    const size_t sm = (size_t)k12Warps * decode12_warp_bytes(m.hmax);
    cudaError_t e = cudaFuncSetAttribute(k_decode12, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_decode12<<<b.n, k12Threads, sm, st>>>(m, b);
    return cudaGetLastError();
}

}  // namespace dlic
