// Coding kernels on the CUDA cores: the all-pixels-at-once prediction of the
// encoder and the wavefront decoder (Sec. II-A, Fig. 2; Sec. II-B).  One
// thread evaluates the network for one pixel.  These kernels serve the FP32
// network everywhere and the INT8 network where the tensor-core kernels do
// not apply.
#include "coder_device.cuh"

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
// Encoder prediction: every pixel of every image at once (the encoder knows
// all priors).  Writes (f, c) of the pixel's own value as f | c << 16.
// ---------------------------------------------------------------------------
template <int PREC>
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
    void *h1 = smem;
    void *h2 = smem + hidden_bytes<PREC>(m.h1);
    hidden<PREC>(m, pri, h1, h2, tid);

    float zmax = -INFINITY;
    for (int j0 = 0; j0 < kSymbols; j0 += 4) {
        float z[4];
        logits4<PREC>(m, h2, tid, j0, z);
#pragma unroll
        for (int q = 0; q < 4; q++) zmax = z[q] > zmax ? z[q] : zmax;
    }
    const int sym = im.pixels[r * im.pitch + c];
    uint32_t W = 0, Ps = 0, ws = 0;
    for (int j0 = 0; j0 < kSymbols; j0 += 4) {
        float z[4];
        logits4<PREC>(m, h2, tid, j0, z);
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
    fc[stream_index(im.H, im.W, im.S, r, c)] = (c_hi - c_lo) | (c_lo << 16);
}

// ---------------------------------------------------------------------------
// Wavefront decoder (Sec. II-B "Preprocessor"): one CTA per image.  Wave t
// holds the pixels (r, t - 3r); all their priors were decoded on earlier
// waves.  Pixels of a wave are predicted in parallel; the rANS step of
// pixels that share a stream (rows S apart) runs in row order.
// ---------------------------------------------------------------------------
struct StreamState {
    uint32_t x, pos, end, pad;
};

__device__ __forceinline__ uint32_t rd_le32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

// Parses and checks the header, then sets up every stream's state from the
// word counts.  Returns false (uniformly across the CTA) for a corrupt header.
__device__ bool decode_setup(const DevModel &m, const DecImage &im, const uint8_t *in,
                             StreamState *st, int *S_out, const uint16_t **pay_out) {
    __shared__ int s_ok, s_S;
    __shared__ uint32_t s_part[256];
    const int tid = threadIdx.x, nth = blockDim.x;
    if (tid == 0) {
        int ok = im.in_bytes >= (uint64_t)kHeaderBytes;
        int S = 0;
        if (ok) {
            const uint8_t *h = in;
            uint64_t hash = 0;
            for (int k = 0; k < 8; k++) hash |= (uint64_t)h[16 + k] << (8 * k);
            S = h[14] | (h[15] << 8);
            ok = h[0] == 'D' && h[1] == 'L' && h[2] == 'C' && h[3] == '1' &&
                 rd_le32(h + 4) == (uint32_t)im.H && rd_le32(h + 8) == (uint32_t)im.W && h[12] == 2 &&
                 h[13] == m.precision && hash == m.hash && S >= 1 && S <= im.H &&
                 im.in_bytes >= (uint64_t)kHeaderBytes + 4ull * S;
        }
        s_ok = ok;
        s_S = S;
    }
    __syncthreads();
    if (!s_ok) return false;
    const int S = s_S;
    const uint8_t *cnt = in + kHeaderBytes;
    // block-wide exclusive scan of the word counts (chunked per thread)
    const int per = (S + nth - 1) / nth;
    const int s0 = min(S, tid * per), s1 = min(S, s0 + per);
    uint32_t sum = 0;
    int bad = 0;
    for (int s = s0; s < s1; s++) {
        const uint32_t c = rd_le32(cnt + 4 * s);
        bad |= c < 2;
        sum += c;
    }
    s_part[tid] = sum;
    if (bad) s_ok = 0;
    __syncthreads();
    if (tid == 0) {
        uint64_t acc = 0;
        for (int k = 0; k < nth; k++) {
            const uint32_t v = s_part[k];
            s_part[k] = (uint32_t)acc;
            acc += v;
        }
        if ((uint64_t)kHeaderBytes + 4ull * S + 2ull * acc != im.in_bytes) s_ok = 0;
    }
    __syncthreads();
    if (!s_ok) return false;
    const uint16_t *pay = reinterpret_cast<const uint16_t *>(in + kHeaderBytes + 4 * S);
    uint32_t start = s_part[tid];
    for (int s = s0; s < s1; s++) {
        const uint32_t c = rd_le32(cnt + 4 * s);
        StreamState q;
        q.x = ((uint32_t)pay[start] << 16) | pay[start + 1];
        q.pos = start + 2;
        q.end = start + c;
        q.pad = 0;
        if (q.x < kRansL) s_ok = 0;
        st[s] = q;
        start += c;
    }
    __syncthreads();
    *S_out = S;
    *pay_out = pay;
    return s_ok != 0;
}

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
    void *h1 = smem;                                                     // aliases zs (dead by then)
    void *h2 = smem + (size_t)kSymbols * kCH * 4;
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

template <int PREC>
static size_t predict_smem(const DevModel &m) {
    return hidden_bytes<PREC>(m.h1) + hidden_bytes<PREC>(m.h2);
}

template <int PREC>
static size_t decode_smem(const DevModel &m) {
    return (size_t)kSymbols * kCH * 4 + hidden_bytes<PREC>(m.h2);
}

cudaError_t launch_predict_cc(const DevModel &m, const EncBatch &b, cudaStream_t st) {
    if (b.total_tiles == 0) return cudaSuccess;
    if (m.precision == DLIC_FP32) {
        const size_t sm = predict_smem<DLIC_FP32>(m);
        cudaFuncSetAttribute(k_predict_cc<DLIC_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_predict_cc<DLIC_FP32><<<b.total_tiles, kCH, sm, st>>>(m, b);
    } else {
        const size_t sm = predict_smem<DLIC_INT8>(m);
        cudaFuncSetAttribute(k_predict_cc<DLIC_INT8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_predict_cc<DLIC_INT8><<<b.total_tiles, kCH, sm, st>>>(m, b);
    }
    return cudaGetLastError();
}

cudaError_t launch_decode_cc(const DevModel &m, const DecBatch &b, cudaStream_t st) {
    if (b.n == 0) return cudaSuccess;
    if (m.precision == DLIC_FP32) {
        const size_t sm = decode_smem<DLIC_FP32>(m);
        cudaFuncSetAttribute(k_decode_cc<DLIC_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_decode_cc<DLIC_FP32><<<b.n, kCH, sm, st>>>(m, b);
    } else {
        const size_t sm = decode_smem<DLIC_INT8>(m);
        cudaFuncSetAttribute(k_decode_cc<DLIC_INT8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_decode_cc<DLIC_INT8><<<b.n, kCH, sm, st>>>(m, b);
    }
    return cudaGetLastError();
}

}  // namespace dlic
