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
#include "tc.cuh"

namespace dlic {

constexpr int k12Warps = 8, k12Threads = 32 * k12Warps;
constexpr int k12PixPerWarp = 8;                       // encoder: pixels per warp (register tile)
constexpr int k12Tile = k12Warps * k12PixPerWarp;      // encoder: pixels per CTA
static_assert(k12Tile == kPredictTile, "the encoder plans CUDA-core tiles of kPredictTile pixels");
constexpr uint64_t k12Slack = kTotal - kSymbols12;     // 2^16 - 4096: the table's free mass
constexpr int k12InPitch = 16;                         // encoder: floats per pixel of the input rows
constexpr int k12PerLane = kSymbols12 / 32;            // decoder: consecutive values each lane searches

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
// Wavefront decoder (Sec. II-B "Preprocessor"): one cluster of P CTAs per
// image.  CTA k owns the rows whose stream (r mod S) is k mod P, so every
// stream's state stays in one CTA.  Per wave t = 3r + c each CTA takes its
// pixels in chunks of 8 in row order: the priors come back from the output
// image through L2 (other CTAs decoded them in earlier waves; one cluster
// barrier per wave orders those stores before these loads), the hidden
// layers run with thread = unit and the chunk's 8 pixels in registers, and
// the 4096 logits with thread = value, so that every weight load of the
// 4096 x h output layer (the bulk of the work) feeds 8 FMAs; each unit and
// value accumulates from its bias in the fixed k order of the encoder.  One
// warp per pixel then turns its 4096 logits into weights in place, each lane
// summing 128 consecutive values, a 64-bit warp scan gives every lane's
// cumulative mass, and the lane whose value range holds the slot walks it.
// Pixels of one stream in one wave (S below the wave's length) take their
// rANS steps in row order.
// Shared memory: the chunk's logits, then weights [8][4096], and two
// activation buffers [hmax][8] (unit-major, a unit's 8 pixels as two
// 16-byte vectors).
// ---------------------------------------------------------------------------
constexpr int k12DecThreads = 512, k12DecWarps = k12DecThreads / 32, k12DecPix = 8;
static_assert(k12DecWarps >= k12DecPix, "one table warp per pixel of a chunk");
// The output layer streams through two stages of two 16 x 256 weight tiles
// (the model's tiled copy: tile (block q, k tile kt) holds rows 16 kt ..
// 16 kt + 15 of W^T at values 256 q .. 256 q + 255, 16 KB).
constexpr int k12TileRows = 16, k12TileFloats = k12TileRows * 256, k12StageFloats = 2 * k12TileFloats;
constexpr long long k12CopyWaitLimit = 4000000000LL;   // clock cycles (about 2 s); a copy from L2 always lands
__host__ __device__ inline size_t decode12_smem_bytes(int hmax) {
    return 4ull * k12DecPix * kSymbols12 + 2ull * 4 * k12StageFloats + 2ull * 4 * k12DecPix * (size_t)hmax +
           4ull * k12DecPix * 16;
}

__device__ __forceinline__ uint32_t px12_cg(const uint8_t *img, int64_t pitch, int r, int c) {
    return __ldcg(reinterpret_cast<const unsigned short *>(img + (int64_t)r * pitch + 2 * (int64_t)c));
}

__global__ void __launch_bounds__(k12DecThreads, 1) k_decode12(DevModel m, DecBatch b, int P) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t lut2[kTableSteps];
    __shared__ int s_err, s_n;
    __shared__ int s_rows[k12DecPix * 32];   // this CTA's rows of the wave (a slice of them)
    __shared__ uint64_t wbar[2];             // output-layer stages filled
    __shared__ int s_cfail;                  // a stage's copy did not land: no further copies
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t k = 0;
    if (P > 1) asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(k));
    const DecImage &im = b.img[blockIdx.x / P];
    expand_lut(m.lut, lut2, tid, k12DecThreads);
    if (tid == 0) {
        s_err = 0;
        s_cfail = 0;
        tc::mbar_init(&wbar[0], 1);
        tc::mbar_init(&wbar[1], 1);
        tc::fence_mbar_init();
    }
    StreamState *st = reinterpret_cast<StreamState *>(b.ws + im.st_off);
    const uint8_t *in = b.in + im.in_off;
    int S;
    const uint16_t *pay;
    // every CTA parses the same header; the cluster barrier after it keeps
    // the set-up writes of the stream states ahead of every update
    const bool ok = decode_setup(m, im, in, st, &S, &pay);   // its barriers also publish lut2 and s_err
    if (P > 1) asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    if (!ok) {
        if (tid == 0 && k == 0) atomicMax(b.status + im.sidx, (int)DLIC_ERR_CORRUPT);
        return;   // uniform: every CTA read the same header
    }
    const int hmax = m.hmax;
    float *zs = reinterpret_cast<float *>(smem);                                   // [8][4096]
    float *wstage = zs + (size_t)k12DecPix * kSymbols12;                           // [2][2 tiles]
    float *hA = wstage + 2 * k12StageFloats, *hB = hA + (size_t)k12DecPix * hmax;  // [hmax][8]
    float *xin = hB + (size_t)k12DecPix * hmax;                                    // [8][16]
    const int L = m.nl - 1;
    const DevLayer lo = m.layers[L];
    const float *wo = static_cast<const float *>(lo.w);
    const int hl = lo.n_in;
    const int H = im.H, W = im.W;
    const int T = 3 * (H - 1) + W;
    const int KT = (hl + k12TileRows - 1) / k12TileRows;   // k tiles of the output layer
    const int nstage = (kSymbols12 / 512) * KT;            // stages per chunk: 8 value-block pairs x KT
    long long g0 = 0;                                      // stages issued and consumed so far
    // stage g: blocks 2 qp, 2 qp + 1 at k tile kt (g - g0 = qp KT + kt)
    auto issue = [&](long long g) {
        const int loc = (int)(g - g0), qp = loc / KT, kt = loc % KT, stg = (int)(g & 1);
        const uint32_t bar_a = tc::smem_addr(&wbar[stg]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(4u * k12StageFloats)
                     : "memory");
        for (int h = 0; h < 2; h++)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             tc::smem_addr(wstage + stg * k12StageFloats + h * k12TileFloats)),
                         "l"(m.w3t + ((size_t)(2 * qp + h) * KT + kt) * k12TileFloats), "r"(4u * k12TileFloats),
                         "r"(bar_a)
                         : "memory");
    };
    for (int t = 0; t < T; t++) {
        const int r_lo = t - W + 1 > 0 ? (t - W + 3) / 3 : 0;
        const int r_hi = min(H - 1, t / 3);
        const bool repeats = r_hi - r_lo + 1 > S;   // two rows of one stream on this wave
        // this CTA's rows of the wave, k8 * 32 of them at a time, in row order
        for (int seg = r_lo; seg <= r_hi; seg += k12DecPix * 32) {
            if (tid == 0) s_n = 0;
            __syncthreads();
            if (warp == 0) {
                int n = 0;
                for (int g = 0; g < k12DecPix; g++) {
                    const int r = seg + 32 * g + lane;
                    const bool own = r <= r_hi && (P == 1 || ((r % S) & (P - 1)) == (int)k);
                    const uint32_t bal = __ballot_sync(0xffffffffu, own);
                    if (own) s_rows[n + __popc(bal & ((1u << lane) - 1u))] = r;
                    n += __popc(bal);
                }
                if (lane == 0) s_n = n;
            }
            __syncthreads();
            const int nk = s_n;
            for (int base = 0; base < nk; base += k12DecPix) {
                const int np = min(k12DecPix, nk - base);
                // priors of the chunk's pixels (pixels past np repeat the first)
                for (int i = tid; i < k12DecPix * kPriors; i += k12DecThreads) {
                    const int p = i / kPriors, q = i % kPriors;
                    const int r = s_rows[base + (p < np ? p : 0)], c = t - 3 * r;
                    const int dr = q < 5 ? -2 : (q < 10 ? -1 : 0);
                    const int dc = q < 5 ? q - 2 : (q < 10 ? q - 7 : q - 12);
                    const int rr = r + dr, cc = c + dc;
                    const uint32_t v = (rr >= 0 && rr < H && cc >= 0 && cc < W) ? px12_cg(im.pixels, im.pitch, rr, cc) : 0u;
                    xin[p * 16 + q] = __fmaf_rn((float)v, 0.00048828125f, -1.0f);   // v / 2048 - 1
                }
                __syncthreads();
                // hidden layers: thread = unit, the chunk's 8 pixels side by side
                float *hin = nullptr, *hout = hA;
                for (int l = 0; l < L; l++) {
                    const DevLayer ly = m.layers[l];
                    const float *wt = static_cast<const float *>(ly.w);
                    const int ph = tid >> 8;   // pixels 4 ph .. 4 ph + 3
                    for (int u = tid & 255; u < ly.n_out; u += 256) {
                        float acc[4];
                        const float bias = __ldg(ly.a + u);
#pragma unroll
                        for (int p = 0; p < 4; p++) acc[p] = bias;
                        for (int kk = 0; kk < ly.n_in; kk++) {
                            const float w = __ldg(wt + (size_t)kk * ly.n_out + u);
                            if (l == 0) {
#pragma unroll
                                for (int p = 0; p < 4; p++) acc[p] = __fmaf_rn(xin[(4 * ph + p) * 16 + kk], w, acc[p]);
                            } else {
                                const float4 a = *reinterpret_cast<const float4 *>(hin + kk * k12DecPix + 4 * ph);
                                const float x[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                                for (int p = 0; p < 4; p++) acc[p] = __fmaf_rn(x[p], w, acc[p]);
                            }
                        }
                        float4 o0;
                        o0.x = acc[0] > 0.0f ? acc[0] : 0.0f; o0.y = acc[1] > 0.0f ? acc[1] : 0.0f;
                        o0.z = acc[2] > 0.0f ? acc[2] : 0.0f; o0.w = acc[3] > 0.0f ? acc[3] : 0.0f;
                        *reinterpret_cast<float4 *>(hout + u * k12DecPix + 4 * ph) = o0;
                    }
                    __syncthreads();
                    hin = hout;
                    hout = hout == hA ? hB : hA;
                }
                // logits: thread = value, one weight load for the 8 pixels
                // logits: two value blocks of 256 at a time, their weights
                // through the stages; thread = (block hh, value pair jp, pixel
                // quad pq): per k row one 8-byte weight load and one 16-byte
                // activation load feed 8 FMAs
                {
                    const int hh = tid >> 8, jp = tid & 127, pq = (tid >> 7) & 1;
                    if (tid == 0 && !s_cfail)
                        for (int q = 0; q < 2 && q < nstage; q++) issue(g0 + q);
                    for (int qp = 0; qp < kSymbols12 / 512; qp++) {
                        const int j0 = 256 * (2 * qp + hh) + 2 * jp;
                        float acc[2][4];
                        const float b0v = __ldg(lo.a + j0), b1v = __ldg(lo.a + j0 + 1);
#pragma unroll
                        for (int p = 0; p < 4; p++) {
                            acc[0][p] = b0v;
                            acc[1][p] = b1v;
                        }
                        for (int kt = 0; kt < KT; kt++) {
                            const long long g = g0 + (long long)qp * KT + kt;
                            const int stg = (int)(g & 1);
                            if (!*reinterpret_cast<volatile int *>(&s_cfail) &&
                                !tc::mbar_wait(&wbar[stg], (uint32_t)((g >> 1) & 1), k12CopyWaitLimit)) {
                                s_cfail = 1;
                                s_err = 1;
                            }
                            const float *tile = wstage + stg * k12StageFloats + hh * k12TileFloats;
                            const int rows = min(k12TileRows, hl - k12TileRows * kt);
                            for (int rr = 0; rr < rows; rr++) {
                                const int kk = k12TileRows * kt + rr;
                                const float2 w = *reinterpret_cast<const float2 *>(tile + rr * 256 + 2 * jp);
                                const float4 a = *reinterpret_cast<const float4 *>(hin + kk * k12DecPix + 4 * pq);
                                const float x[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                                for (int p = 0; p < 4; p++) {
                                    acc[0][p] = __fmaf_rn(x[p], w.x, acc[0][p]);
                                    acc[1][p] = __fmaf_rn(x[p], w.y, acc[1][p]);
                                }
                            }
                            __syncthreads();   // every reader is done with this stage
                            if (tid == 0 && !s_cfail && g + 2 < g0 + nstage) issue(g + 2);
                        }
#pragma unroll
                        for (int p = 0; p < 4; p++) {
                            zs[(size_t)(4 * pq + p) * kSymbols12 + j0] = acc[0][p];
                            zs[(size_t)(4 * pq + p) * kSymbols12 + j0 + 1] = acc[1][p];
                        }
                    }
                    g0 += nstage;
                }
                __syncthreads();
                // tables, one warp per pixel: maximum, weights in place, lane sums
                uint64_t Q = 0, P0 = 0;
                uint32_t lsum = 0;
                const int i0 = k12PerLane * lane;
                float *zw = zs + (size_t)warp * kSymbols12;
                uint32_t *wts = reinterpret_cast<uint32_t *>(zw);
                if (warp < np) {
                    float mx = -INFINITY;
                    for (int i = lane; i < kSymbols12; i += 32) mx = zw[i] > mx ? zw[i] : mx;
                    mx = warp_max(mx);
                    __syncwarp();
                    for (int i = i0; i < i0 + k12PerLane; i++) {
                        const uint32_t w = table_weight2(mx, zw[i], m.tscale, lut2);
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
                // rANS steps: all at once, or in row order when a stream repeats
                for (int rnd = 0; rnd < (repeats ? np : 1); rnd++) {
                    if (warp < np && (!repeats || warp == rnd)) {
                        const int r = s_rows[base + warp], c = t - 3 * r;
                        const int s = r % S;
                        StreamState q = st[s];
                        const uint32_t slot = q.x & 0xFFFFu;
                        const uint32_t c0 = (uint32_t)i0 + (uint32_t)((P0 * Q) >> 32);
                        const uint32_t c1 =
                            lane == 31 ? kTotal : (uint32_t)(i0 + k12PerLane) + (uint32_t)(((P0 + lsum) * Q) >> 32);
                        if (c0 <= slot && slot < c1) {   // exactly one lane: the ranges tile [0, 2^16)
                            uint64_t Pc = P0;
                            uint32_t c_lo = c0, f = 1;
                            int sym = i0 + k12PerLane - 1;
                            for (int i = i0; i < i0 + k12PerLane; i++) {
                                const uint32_t w = wts[i];
                                const uint32_t lo_i = (uint32_t)i + (uint32_t)((Pc * Q) >> 32);
                                const uint32_t hi_i =
                                    i == kSymbols12 - 1 ? kTotal : (uint32_t)i + 1u + (uint32_t)(((Pc + w) * Q) >> 32);
                                if (hi_i > slot) {
                                    sym = i;
                                    c_lo = lo_i;
                                    f = hi_i - lo_i;
                                    break;
                                }
                                Pc += w;
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
                            st[s] = q;
                            *reinterpret_cast<uint16_t *>(im.pixels + (int64_t)r * im.pitch + 2 * (int64_t)c) =
                                (uint16_t)sym;
                        }
                    }
                    if (repeats) __syncthreads();
                }
                __syncthreads();   // the logits and activations are free again
            }
        }
        // this wave's pixels in the image before any CTA's next gather
        if (P > 1) asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        else __syncthreads();
    }
    // the final states of this CTA's streams must be back at L with every word read
    for (int s = tid; s < S; s += k12DecThreads)
        if (P == 1 || (s & (P - 1)) == (int)k) {
            const StreamState q = st[s];
            if (q.x != kRansL || q.pos != q.end) s_err = 1;
        }
    __syncthreads();
    if (tid == 0) atomicMax(b.status + im.sidx, s_err ? (int)DLIC_ERR_CORRUPT : (int)DLIC_OK);
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
    const size_t sm = decode12_smem_bytes(m.hmax);
    cudaError_t e = cudaFuncSetAttribute(k_decode12, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_decode12, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    // cluster size: about 8 pixels of the longest wave per CTA, at most 16
    int wave = 1;
    for (int i = 0; i < b.n; i++) wave = max(wave, min(b.img[i].H, (b.img[i].W + 2) / 3));
    int P = 1;
    while (P < 16 && P * k12DecPix < wave) P <<= 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(k12DecThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    for (;;) {
        attr[0].val.clusterDim.x = (unsigned)P;
        cfg.gridDim = dim3((unsigned)(b.n * P));
        int nclusters = 0;
        if (P == 1 || (cudaOccupancyMaxActiveClusters(&nclusters, k_decode12, &cfg) == cudaSuccess && nclusters > 0))
            break;
        cudaGetLastError();
        P >>= 1;
    }
    return cudaLaunchKernelEx(&cfg, k_decode12, m, b, P);
}

}  // namespace dlic
