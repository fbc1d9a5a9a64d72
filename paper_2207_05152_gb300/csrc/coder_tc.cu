// Encoder prediction on the tensor cores (INT8 network): every pixel of
// every image at once (Sec. II-A, Fig. 2 left; the network is the bulk of the
// work, Sec. III-B, Fig. 4), 128 pixels per tile.
//
// The INT8 network's operands are small integers (priors v - 128 in
// [-128, 127], hidden activations in [0, 255], weights in [-127, 127]); each
// is exact in bf16 and every partial sum of at most 128 products stays below
// 2^23, so tcgen05 BF16 MMAs with FP32 accumulation compute the integer dot
// products exactly.  Per tile and layer: threads write the A operand to
// shared memory (no-swizzle K-major core matrices), one thread issues the
// MMAs into tensor memory, and the epilogue (requantisation, or the
// frequency table after the last layer) reads the accumulators back with
// tcgen05.ld, one pixel per thread.
//
// CTA: four warpgroups, two per tile slot.  A slot owns 256 tensor-memory
// columns and its own A buffers, so one slot's epilogue overlaps the other's
// MMAs; within a slot the two warpgroups read the same accumulator rows
// (pixels) and split the columns: hidden units for the requantisation,
// symbols for the frequency table (partial maxima and sums meet in shared
// memory).  Weights stay in shared memory for the whole persistent CTA.
#include "coder_device.cuh"
#include "tc.cuh"

namespace dlic {

constexpr int kTcTile = 128;
constexpr int kTcSlots = 2;
constexpr long long kTcWaitLimit = 4000000000LL;   // clock cycles (about 2 s)

struct TcLayout {
    uint32_t w1, w2, w3, a1[kTcSlots], a23[kTcSlots], s1, o1, s2, o2, s3, o3, lut, total;
};

// k1: the first layer's K, the window's priors padded to 16.  A slot's A1
// tile (pixels x k1) and its hidden-activation tile share one buffer: the
// first layer's MMA has read A1 before the first requantisation writes.
__host__ __device__ inline TcLayout tc_layout(int h1, int h2, int k1) {
    TcLayout L;
    uint32_t off = 0;
    auto take = [&](uint32_t bytes) {
        const uint32_t o = off;
        off += (bytes + 127u) & ~127u;
        return o;
    };
    L.w1 = take(2u * k1 * h1);
    L.w2 = take(2u * h1 * h2);
    L.w3 = take(512u * h2);
    int hmax = h1 > h2 ? h1 : h2;
    hmax = hmax > k1 ? hmax : k1;
    for (int j = 0; j < kTcSlots; j++) {
        L.a23[j] = take(kTcTile * hmax * 2);
        L.a1[j] = L.a23[j];
    }
    L.s1 = take(4u * h1);
    L.o1 = take(4u * h1);
    L.s2 = take(4u * h2);
    L.o2 = take(4u * h2);
    L.s3 = take(4u * kSymbols);
    L.o3 = take(4u * kSymbols);
    L.lut = take(4u * kTableSteps);
    L.total = off;
    return L;
}

constexpr int kTcThreads = 512;
__device__ __forceinline__ void slot_sync(int slot) {
    asm volatile("bar.sync %0, 256;" ::"r"(slot + 1) : "memory");
}

// Requantises 16 accumulator columns to u8 activations and stores them as
// bf16 into row `row` of a K-major operand with K = kdim columns.
__device__ __forceinline__ void requant_store16(const uint32_t (&v)[16], const float *s, const float *o,
                                                uint8_t *a, int row, int c0, int kdim) {
    uint32_t packed[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
        float lo = rintf(__fmaf_rn(__uint_as_float(v[2 * q]), s[c0 + 2 * q], o[c0 + 2 * q]));
        float hi = rintf(__fmaf_rn(__uint_as_float(v[2 * q + 1]), s[c0 + 2 * q + 1], o[c0 + 2 * q + 1]));
        lo = fminf(fmaxf(lo, 0.0f), 255.0f);
        hi = fminf(fmaxf(hi, 0.0f), 255.0f);
        packed[q] = __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
    }
    *reinterpret_cast<uint4 *>(a + tc::kmajor_offset(row, c0, kdim)) =
        make_uint4(packed[0], packed[1], packed[2], packed[3]);
    *reinterpret_cast<uint4 *>(a + tc::kmajor_offset(row, c0 + 8, kdim)) =
        make_uint4(packed[4], packed[5], packed[6], packed[7]);
}

// DEF: the default window of 12 priors (K1 = 16, offsets as constants).
template <bool DEF>
__global__ void __launch_bounds__(kTcThreads, 1) k_encode_tc(DevModel m, EncBatch b, int *err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bars[kTcSlots];
    __shared__ uint32_t tmem_base;
    __shared__ int wg_fail[kTcSlots];
    __shared__ float s_max[kTcSlots][2][128];
    __shared__ char4 s_woff[kMaxPriors];   // (row, column, slice) offset of every prior of the window
    __shared__ uint32_t s_w[kTcSlots][3][128];   // the high half's W, P_sym and w_sym
    const int tid = threadIdx.x, wg = tid >> 7, t = tid & 127, warp = tid >> 5;
    const int slot = wg & 1, half = wg >> 1;
    const int h1 = m.h1, h2 = m.h2;
    const int NPRI = DEF ? kPriors : m.n_in, K1 = DEF ? 16 : (m.n_in + 15) / 16 * 16;
    const TcLayout L = tc_layout(h1, h2, K1);

    // weights (already in operand layout) and epilogue parameters
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(m.tc_w);
        uint4 *dst = reinterpret_cast<uint4 *>(smem + L.w1);
        const int n16 = (int)(m.tc_w_bytes / 16);
        for (int i = tid; i < n16; i += blockDim.x) dst[i] = __ldg(src + i);
        float *s1 = reinterpret_cast<float *>(smem + L.s1), *o1 = reinterpret_cast<float *>(smem + L.o1);
        float *s2 = reinterpret_cast<float *>(smem + L.s2), *o2 = reinterpret_cast<float *>(smem + L.o2);
        float *s3 = reinterpret_cast<float *>(smem + L.s3), *o3 = reinterpret_cast<float *>(smem + L.o3);
        for (int i = tid; i < h1; i += blockDim.x) { s1[i] = m.s1[i]; o1[i] = m.o1[i]; }
        for (int i = tid; i < h2; i += blockDim.x) { s2[i] = m.s2[i]; o2[i] = m.o2[i]; }
        for (int i = tid; i < kSymbols; i += blockDim.x) { s3[i] = m.s3[i]; o3[i] = m.o3[i]; }
        expand_lut(m.lut, reinterpret_cast<uint32_t *>(smem + L.lut), tid, blockDim.x);
        if (tid < m.n_in) {
            int dz, dr, dc;
            window_offset(m, tid, dz, dr, dc);
            s_woff[tid] = make_char4((signed char)dr, (signed char)dc, (signed char)dz, 0);
        }
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 256 * kTcSlots);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int j = 0; j < kTcSlots; j++) tc::mbar_init(&bars[j], 1);
        tc::fence_mbar_init();
    }
    if (tid < kTcSlots) wg_fail[tid] = 0;
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    const float *s1 = reinterpret_cast<const float *>(smem + L.s1), *o1 = reinterpret_cast<const float *>(smem + L.o1);
    const float *s2 = reinterpret_cast<const float *>(smem + L.s2), *o2 = reinterpret_cast<const float *>(smem + L.o2);
    const float *s3 = reinterpret_cast<const float *>(smem + L.s3), *o3 = reinterpret_cast<const float *>(smem + L.o3);
    const uint32_t *lut = reinterpret_cast<const uint32_t *>(smem + L.lut);
    uint8_t *a1 = smem + L.a1[slot];
    uint8_t *a23 = smem + L.a23[slot];
    const uint32_t tm = tmem_base + 256u * slot;                     // this slot's columns
    const uint32_t tm_row = tm + ((uint32_t)(32 * (warp & 3)) << 16); // this warp's lane quarter
    const uint32_t sa1 = tc::smem_addr(a1), sa23 = tc::smem_addr(a23);
    const uint32_t sw1 = tc::smem_addr(smem + L.w1), sw2 = tc::smem_addr(smem + L.w2),
                   sw3 = tc::smem_addr(smem + L.w3);
    uint32_t phase = 0;

    // One layer: D[tm] = A[sa] (128 x K) * W[sw]^T (N x K), then wait.
    auto layer = [&](uint32_t sa, uint32_t sw, int K, int N) -> bool {
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        slot_sync(slot);
        if (half == 0 && t == 0) {
            tc::fence_after_sync();
            const uint32_t idesc = tc::idesc_bf16_f32(kTcTile, N);
            for (int ks = 0; ks < K / 16; ks++)
                tc::mma_bf16(tm, tc::make_desc(sa + 256u * ks, 128u, 16u * K),
                             tc::make_desc(sw + 256u * ks, 128u, 16u * K), idesc, ks > 0);
            tc::mma_commit(&bars[slot]);
            if (!tc::mbar_wait(&bars[slot], phase, kTcWaitLimit)) wg_fail[slot] = 1;
        }
        phase ^= 1u;
        slot_sync(slot);
        tc::fence_after_sync();
        return wg_fail[slot] == 0;
    };

    for (int tile = blockIdx.x * kTcSlots + slot; tile < b.total_tiles; tile += gridDim.x * kTcSlots) {
        int ii = 0;
        while (ii + 1 < b.n && b.img[ii + 1].tile_begin <= tile) ii++;
        const EncImage &im = b.img[ii];
        const int64_t p = (int64_t)(tile - im.tile_begin) * kTcTile + t;
        const bool active = p < (int64_t)im.H * im.W;
        const int r = active ? (int)(p / im.W) : 0, c = active ? (int)(p % im.W) : 0;

        // A1: the window's priors as v - 128 (pixels outside the image are
        // 0), padded to K1 with zeros; the two warpgroups of the slot take
        // alternate 8-column chunks
        for (int j = half; j < K1 / 8; j += 2) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                uint32_t pair = 0;
#pragma unroll
                for (int hb = 0; hb < 2; hb++) {
                    const int q = 8 * j + 2 * e + hb;
                    uint32_t v = 0u;
                    if (active && q < NPRI) {
                        int dr, dc, pv;
                        if (DEF) {
                            dr = q < 5 ? -2 : (q < 10 ? -1 : 0);
                            dc = q < 5 ? q - 2 : (q < 10 ? q - 7 : q - 12);
                            const int rr = r + dr, cc = c + dc;
                            pv = (rr >= 0 && cc >= 0 && cc < im.W) ? im.pixels[(int64_t)rr * im.pitch + cc] : 0;
                        } else {
                            // a 3D window reads its lower layer from the previous slice
                            const char4 o = s_woff[q];
                            const int rr = r + o.x, cc = c + o.y;
                            const uint8_t *src = o.z ? im.below : im.pixels;
                            pv = (src && rr >= 0 && rr < im.H && cc >= 0 && cc < im.W) ? src[(int64_t)rr * im.pitch + cc]
                                                                                      : 0;
                        }
                        v = tc::bf16_of_int(pv - 128);
                    }
                    pair |= v << (16 * hb);
                }
                w[e] = pair;
            }
            *reinterpret_cast<uint4 *>(a1 + tc::kmajor_offset(t, 8 * j, K1)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        if (!layer(sa1, sw1, K1, h1)) break;
        // requantisation: each warpgroup of the slot takes half of the
        // 16-column chunks (the first half the odd one)
        const int n1 = h1 / 16, f1 = (n1 + 1) / 2;
        for (int c0 = half ? 16 * f1 : 0; c0 < (half ? h1 : 16 * f1); c0 += 16) {
            uint32_t v[16];
            tc::tmem_ld16(tm_row + c0, v);
            tc::tmem_wait_ld();
            requant_store16(v, s1, o1, a23, t, c0, h1);
        }
        if (!layer(sa23, sw2, h1, h2)) break;
        const int n2 = h2 / 16, f2 = (n2 + 1) / 2;
        for (int c0 = half ? 16 * f2 : 0; c0 < (half ? h2 : 16 * f2); c0 += 16) {
            uint32_t v[16];
            tc::tmem_ld16(tm_row + c0, v);
            tc::tmem_wait_ld();
            requant_store16(v, s2, o2, a23, t, c0, h2);
        }
        if (!layer(sa23, sw3, h2, kSymbols)) break;

        // frequency table of the pixel's own value (see coder_device.cuh);
        // this warpgroup's 128 symbols, then the halves combine
        const int sb = 128 * half;
        float zmax = -INFINITY;
        for (int c0 = sb; c0 < sb + 128; c0 += 16) {
            uint32_t v[16];
            tc::tmem_ld16(tm_row + c0, v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 16; q++) {
                const float z = __fmaf_rn(__uint_as_float(v[q]), s3[c0 + q], o3[c0 + q]);
                zmax = z > zmax ? z : zmax;
            }
        }
        s_max[slot][half][t] = zmax;
        slot_sync(slot);
        zmax = fmaxf(zmax, s_max[slot][half ^ 1][t]);
        const int sym = active ? im.pixels[r * im.pitch + c] : 0;
        uint32_t Wsum = 0, Ps = 0, ws = 0;
        for (int c0 = sb; c0 < sb + 128; c0 += 16) {
            uint32_t v[16];
            tc::tmem_ld16(tm_row + c0, v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 16; q++) {
                const int i = c0 + q;
                const float z = __fmaf_rn(__uint_as_float(v[q]), s3[i], o3[i]);
                const uint32_t w = table_weight2(zmax, z, m.tscale, lut);
                // at the pixel's own value: the running total so far and its weight
                const bool at = i == sym;
                Ps = at ? Wsum : Ps;
                ws = at ? w : ws;
                Wsum += w;
            }
        }
        // this half's part of sum_{i < sym} w_i: all of it when sym lies above the half
        if (sym >= sb + 128) Ps = Wsum;
        if (half == 1) {
            s_w[slot][0][t] = Wsum;
            s_w[slot][1][t] = Ps;
            s_w[slot][2][t] = ws;
        }
        slot_sync(slot);
        if (half == 0) {
            Wsum += s_w[slot][0][t];
            Ps += s_w[slot][1][t];   // the two halves' parts of sum_{i < sym} w_i
            ws += s_w[slot][2][t];   // w_sym from whichever half holds sym
        }
        if (active && half == 0) {
            const uint32_t Q = table_q(Wsum);
            const uint32_t c_lo = (uint32_t)sym + __umulhi(Ps, Q);
            const uint32_t c_hi = sym == kSymbols - 1 ? kTotal : (uint32_t)sym + 1u + __umulhi(Ps + ws, Q);
            uint32_t *fc = reinterpret_cast<uint32_t *>(b.ws + im.fc_off);
            fc[b.raster ? (int64_t)r * im.W + c : stream_index(im.H, im.W, im.S, r, c)] = (c_hi - c_lo) | (c_lo << 16);
        }
        tc::fence_before_sync();   // tensor-memory reads done before the next tile's MMAs
    }
    if (tid < kTcSlots && wg_fail[tid]) atomicExch(err, DLIC_ERR_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem_base, 256 * kTcSlots);
    }
}

bool tc_supported(const DevModel &m) {
    return m.precision == DLIC_INT8 && m.tc_w != nullptr && m.h1 <= 128 && m.h2 <= 128;
}

size_t tc_weight_bytes(int h1, int h2, int k1) {
    const TcLayout L = tc_layout(h1, h2, k1);
    return L.w3 + 512u * h2;
}

// Host image of the bf16 operand tiles W1 (h1 x 16), W2 (h2 x h1), W3
// (256 x h2) from the int8 weights (row-major [out][in]).
void tc_pack_weights(int h1, int h2, int n_in, int k1, const int8_t *q1, const int8_t *q2, const int8_t *q3,
                     uint16_t *out) {
    const TcLayout L = tc_layout(h1, h2, k1);
    uint8_t *base = reinterpret_cast<uint8_t *>(out);
    for (size_t i = 0; i < tc_weight_bytes(h1, h2, k1) / 2; i++) out[i] = 0;
    for (int j = 0; j < h1; j++)
        for (int k = 0; k < n_in; k++)
            *reinterpret_cast<uint16_t *>(base + L.w1 + tc::kmajor_offset(j, k, k1)) = tc::bf16_of_int(q1[j * n_in + k]);
    for (int j = 0; j < h2; j++)
        for (int k = 0; k < h1; k++)
            *reinterpret_cast<uint16_t *>(base + L.w2 + tc::kmajor_offset(j, k, h1)) = tc::bf16_of_int(q2[j * h1 + k]);
    for (int j = 0; j < kSymbols; j++)
        for (int k = 0; k < h2; k++)
            *reinterpret_cast<uint16_t *>(base + L.w3 + tc::kmajor_offset(j, k, h2)) = tc::bf16_of_int(q3[j * h2 + k]);
}

cudaError_t launch_predict_tc(const DevModel &m, const EncBatch &b, int *err, int num_sms, cudaStream_t st) {
    if (b.total_tiles == 0) return cudaSuccess;
    const TcLayout L = tc_layout(m.h1, m.h2, (m.n_in + 15) / 16 * 16);
    void (*kern)(DevModel, EncBatch, int *) = default_window(m) ? k_encode_tc<true> : k_encode_tc<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    const int per_cta = kTcSlots;
    int grid = (b.total_tiles + per_cta - 1) / per_cta;
    if (grid > num_sms) grid = num_sms;
    kern<<<grid, kTcThreads, L.total, st>>>(m, b, err);
    return cudaGetLastError();
}

}  // namespace dlic
