// Wavefront decoder on the tensor cores (INT8 network, hidden widths 128).
//
// Sec. II-B "Preprocessor": decoding proceeds in waves; wave t holds the
// pixels (r, t - 3r), whose causal priors were all decoded on earlier waves,
// and every pixel of a wave is predicted and decoded in parallel.
//
// One thread-block cluster of P CTAs decodes one image.  CTA k owns the
// rANS streams s with s mod P == k and so the rows r with (r mod S) mod P
// == k: every stream belongs to exactly one CTA, which keeps its state and
// its payload words in shared memory.  Per wave each CTA:
//   1. gathers the 12 priors of its pixels from a ring buffer of the last
//      columns of every live row (a replicated copy in every CTA),
//   2. runs the three dense layers as tcgen05 MMAs with the weights as the
//      A operand (M = 128 units) and the wave's pixels as the B operand
//      (N = pixels, padded to 16), so a handful of pixels still fills the
//      M dimension; FP32 accumulators in tensor memory are exact integers,
//   3. turns the 256 logits of each pixel into its frequency table with one
//      warp per pixel (warp max, prefix sum, ballot search) and performs the
//      rANS decoding step of the pixel's stream,
//   4. writes the decoded pixel to the image and, through distributed shared
//      memory, to every CTA's ring buffer,
// then the cluster synchronises once before the next wave.
#include "coder_device.cuh"
#include "tc.cuh"

namespace dlic {

constexpr int kDecThreads = 256;
constexpr int kDecWarps = kDecThreads / 32;
constexpr int kDecHidden = 128;
constexpr long long kDecWaitLimit = 4000000000LL;

struct DecTcLayout {
    uint32_t w1, w2, w3, b1, b23, z, ring, rows, lut, st_x, st_pos, st_end, pay, total;
};

// Shared-memory plan for chunks of up to nt pixels, `rows` ring rows (also
// the bound on the pixels of one wave), `g` owned streams and `pay_words`
// staged payload words.
__host__ __device__ inline DecTcLayout dec_layout(int nt, int rows, int g, int pay_words) {
    DecTcLayout L;
    uint32_t off = 0;
    auto take = [&](uint32_t bytes) {
        const uint32_t o = off;
        off += (bytes + 127u) & ~127u;
        return o;
    };
    L.w1 = take(32u * kDecHidden);
    L.w2 = take(2u * kDecHidden * kDecHidden);
    L.w3 = take(512u * kDecHidden);
    L.b1 = take(32u * nt);
    L.b23 = take(2u * nt * kDecHidden);
    L.z = take(4u * nt * kSymbols);
    L.ring = take(16u * rows);
    L.rows = take(4u * rows);
    L.lut = take(4u * 64);
    L.st_x = take(4u * g);
    L.st_pos = take(4u * g);
    L.st_end = take(4u * g);
    L.pay = take(2u * pay_words);
    L.total = off;
    return L;
}

struct DecTcParams {
    int P;            // CTAs per image (cluster size)
    int nt;           // pixels per chunk (multiple of 16, <= 128)
    int ring_rows;    // power of two
    int max_g;        // owned streams per CTA (upper bound)
    int pay_words;    // staged payload capacity per CTA (words); 0 = read from global
};

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t map_shared(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster_u8(uint32_t addr, uint32_t v) {
    asm volatile("st.shared::cluster.u8 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// floor(65280 * 2^32 / W) for 2^23 <= W <= 2^31, exactly: a single-precision
// quotient (within a few units of the result) corrected with the exact
// 64-bit remainder.
__device__ __forceinline__ uint32_t table_q_fast(uint32_t W) {
    const long long num = 65280LL << 32;
    long long q = (long long)__fdiv_rn(280375465082880.0f, __uint2float_rn(W));
    long long rem = num - q * (long long)W;
#pragma unroll 1
    for (int k = 0; k < 16 && rem < 0; k++) {
        q -= 1;
        rem += W;
    }
#pragma unroll 1
    for (int k = 0; k < 16 && rem >= (long long)W; k++) {
        q += 1;
        rem -= W;
    }
    return (uint32_t)q;
}

__global__ void __launch_bounds__(kDecThreads, 1) k_decode_tc(DevModel m, DecBatch b, DecTcParams prm) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok, s_S, s_err, s_fail;
    __shared__ uint32_t s_part[kDecThreads];
    __shared__ uint32_t s_gpart[kDecThreads];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = prm.P, NT = prm.nt;
    const uint32_t k = P > 1 ? cluster_rank() : 0u;
    const int img_idx = blockIdx.x / P;
    const DecImage &im = b.img[img_idx];
    const uint8_t *in = b.in + im.in_off;
    const int H = im.H, W = im.W;
    const DecTcLayout L = dec_layout(NT, prm.ring_rows, prm.max_g, prm.pay_words);

    // --- set-up: weights, parameters, tensor memory, header and streams ---
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(m.tc_w);
        uint4 *dst = reinterpret_cast<uint4 *>(smem + L.w1);
        const int n16 = (int)(m.tc_w_bytes / 16);
        for (int i = tid; i < n16; i += kDecThreads) dst[i] = __ldg(src + i);
        uint32_t *lut = reinterpret_cast<uint32_t *>(smem + L.lut);
        if (tid < 64) lut[tid] = m.lut[tid];
        uint32_t *ring = reinterpret_cast<uint32_t *>(smem + L.ring);
        for (int i = tid; i < prm.ring_rows * 4; i += kDecThreads) ring[i] = 0u;
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 256);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
        s_err = 0;
        s_fail = 0;
        int ok = im.in_bytes >= (uint64_t)kHeaderBytes;
        int S = 0;
        if (ok) {
            uint64_t hash = 0;
            for (int q = 0; q < 8; q++) hash |= (uint64_t)in[16 + q] << (8 * q);
            S = in[14] | (in[15] << 8);
            const uint32_t hh = in[4] | (in[5] << 8) | (in[6] << 16) | ((uint32_t)in[7] << 24);
            const uint32_t ww = in[8] | (in[9] << 8) | (in[10] << 16) | ((uint32_t)in[11] << 24);
            ok = in[0] == 'D' && in[1] == 'L' && in[2] == 'C' && in[3] == '1' && hh == (uint32_t)H &&
                 ww == (uint32_t)W && in[12] == 2 && in[13] == m.precision && hash == m.hash && S >= 1 &&
                 S <= H && (S + P - 1) / P <= prm.max_g && im.in_bytes >= (uint64_t)kHeaderBytes + 4ull * S;
        }
        s_ok = ok;
        s_S = S;
    }
    __syncthreads();
    const int S = s_S;
    const int G = (S - (int)k + P - 1) / P;    // streams owned by this CTA: s = k + P g
    uint32_t *st_x = reinterpret_cast<uint32_t *>(smem + L.st_x);
    uint32_t *st_pos = reinterpret_cast<uint32_t *>(smem + L.st_pos);
    uint32_t *st_end = reinterpret_cast<uint32_t *>(smem + L.st_end);
    const uint16_t *pay = reinterpret_cast<const uint16_t *>(in + kHeaderBytes + 4 * S);
    const uint16_t *wsrc = pay;
    if (s_ok) {
        // exclusive scan of the word counts of all streams (chunked per thread)
        const uint8_t *cnt = in + kHeaderBytes;
        const int per = (S + kDecThreads - 1) / kDecThreads;
        const int s0 = min(S, tid * per), s1 = min(S, s0 + per);
        uint32_t sum = 0, gsum = 0;
        int bad = 0;
        for (int s = s0; s < s1; s++) {
            const uint32_t c = cnt[4 * s] | (cnt[4 * s + 1] << 8) | (cnt[4 * s + 2] << 16) | ((uint32_t)cnt[4 * s + 3] << 24);
            bad |= c < 2;
            sum += c;
            if (s % P == (int)k) gsum += c;
        }
        s_part[tid] = sum;
        s_gpart[tid] = gsum;
        if (bad) s_ok = 0;
        __syncthreads();
        if (tid == 0) {
            uint64_t acc = 0, gacc = 0;
            for (int q = 0; q < kDecThreads; q++) {
                const uint32_t v = s_part[q], gv = s_gpart[q];
                s_part[q] = (uint32_t)acc;
                s_gpart[q] = (uint32_t)gacc;
                acc += v;
                gacc += gv;
            }
            if ((uint64_t)kHeaderBytes + 4ull * S + 2ull * acc != im.in_bytes) s_ok = 0;
            // payload of the owned streams staged in shared memory if it fits
            s_fail = gacc <= (uint64_t)prm.pay_words ? 1 : 0;
        }
        __syncthreads();
        const bool staged = s_fail != 0;
        if (s_ok) {
            uint16_t *spay = reinterpret_cast<uint16_t *>(smem + L.pay);
            uint32_t start = s_part[tid], lstart = s_gpart[tid];
            for (int s = s0; s < s1; s++) {
                const uint32_t c = cnt[4 * s] | (cnt[4 * s + 1] << 8) | (cnt[4 * s + 2] << 16) | ((uint32_t)cnt[4 * s + 3] << 24);
                if (s % P == (int)k) {
                    const int g = s / P;
                    const uint32_t base = staged ? lstart : start;
                    st_x[g] = ((uint32_t)pay[start] << 16) | pay[start + 1];
                    st_pos[g] = base + 2;
                    st_end[g] = base + c;
                    if (staged)
                        for (uint32_t q = 0; q < c; q++) spay[lstart + q] = pay[start + q];
                    lstart += c;
                }
                start += c;
            }
            if (staged) wsrc = spay;
        }
        __syncthreads();
        if (s_ok)
            for (int g = tid; g < G; g += kDecThreads)
                if (st_x[g] < kRansL) s_err = 1;
        if (tid == 0) s_fail = 0;
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // Every CTA of the cluster reads the same header, so this exit is uniform.
    if (!s_ok) {
        if (tid == 0 && k == 0) atomicMax(b.status + img_idx, (int)DLIC_ERR_CORRUPT);
        if (warp == 0) tc::tmem_dealloc(tmem_base, 256);
        return;
    }

    const uint32_t tm = tmem_base;
    const int q4 = warp & 3, cg = warp >> 2;                 // lane quarter, column group
    const int unit = 32 * q4 + lane;                          // hidden / output unit of this thread
    const uint32_t tm_q = tm + ((uint32_t)(32 * q4) << 16);
    const float s1r = m.s1[unit], o1r = m.o1[unit], s2r = m.s2[unit], o2r = m.o2[unit];
    const float s3a = m.s3[unit], o3a = m.o3[unit], s3b = m.s3[128 + unit], o3b = m.o3[128 + unit];
    uint8_t *ring = smem + L.ring;
    const uint32_t ring_addr = tc::smem_addr(ring);
    const uint32_t *lut = reinterpret_cast<const uint32_t *>(smem + L.lut);
    uint8_t *b1 = smem + L.b1;
    uint8_t *b23 = smem + L.b23;
    float *zb = reinterpret_cast<float *>(smem + L.z);
    const uint32_t sb1 = tc::smem_addr(b1), sb23 = tc::smem_addr(b23);
    const uint32_t sw1 = tc::smem_addr(smem + L.w1), sw2 = tc::smem_addr(smem + L.w2),
                   sw3 = tc::smem_addr(smem + L.w3);
    const int rmask = prm.ring_rows - 1;
    uint32_t phase = 0;

    // Issues one layer's MMAs (thread 0), waits for them, and synchronises the
    // CTA.  After a timeout no further MMAs are issued; the wave loop still
    // runs to the end so that every cluster barrier is met.
    auto run_layer = [&](int layer, int NP) {
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0 && !s_fail) {
            tc::fence_after_sync();
            if (layer == 1) {
                tc::mma_bf16(tm, tc::make_desc(sw1, 128u, 256u), tc::make_desc(sb1, 128u, 256u),
                             tc::idesc_bf16_f32(128, NP), 0u);
            } else if (layer == 2) {
                for (int ks = 0; ks < kDecHidden / 16; ks++)
                    tc::mma_bf16(tm, tc::make_desc(sw2 + 256u * ks, 128u, 16u * kDecHidden),
                                 tc::make_desc(sb23 + 256u * ks, 128u, 16u * kDecHidden),
                                 tc::idesc_bf16_f32(128, NP), ks > 0);
            } else {
                for (int half = 0; half < 2; half++)
                    for (int ks = 0; ks < kDecHidden / 16; ks++)
                        tc::mma_bf16(tm + (uint32_t)(half * NP),
                                     tc::make_desc(sw3 + 16u * 16u * kDecHidden * half + 256u * ks, 128u,
                                                   16u * kDecHidden),
                                     tc::make_desc(sb23 + 256u * ks, 128u, 16u * kDecHidden),
                                     tc::idesc_bf16_f32(128, NP), ks > 0);
            }
            tc::mma_commit(&bar);
            if (!tc::mbar_wait(&bar, phase, kDecWaitLimit)) s_fail = 1;
        }
        phase ^= 1u;
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    };

    // Epilogue of a hidden layer: unit `unit`, pixel columns of this warp's
    // column group -> u8 activations as bf16 into b23 (row = pixel, k = unit).
    auto hidden_epilogue = [&](int NP, float s, float o) {
        for (int c0 = 16 * cg; c0 < NP; c0 += 32) {
            uint32_t v[16];
            tc::tmem_ld16(tm_q + (uint32_t)c0, v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 16; e++) {
                float h = rintf(__fmaf_rn(__uint_as_float(v[e]), s, o));
                h = fminf(fmaxf(h, 0.0f), 255.0f);
                const uint32_t mine = __float_as_uint(h) >> 16;
                const uint32_t other = __shfl_xor_sync(0xffffffffu, mine, 1);
                if ((lane & 1) == 0)
                    *reinterpret_cast<uint32_t *>(b23 + tc::kmajor_offset(c0 + e, unit, kDecHidden)) = mine | (other << 16);
            }
        }
    };

    int *rowlist = reinterpret_cast<int *>(smem + L.rows);
    __shared__ int s_wcnt[kDecWarps];
    const int T = 3 * (H - 1) + W;
    for (int t = 0; t < T; t++) {
        const int r_lo = t - W + 1 > 0 ? (t - W + 3) / 3 : 0;
        const int r_hi = min(H - 1, t / 3);
        // rows of this wave owned by this CTA, in increasing order
        int nk = 0;
        for (int seg = r_lo; seg <= r_hi; seg += kDecThreads) {
            const int r = seg + tid;
            const bool own = r <= r_hi && ((r % S) % P) == (int)k;
            const uint32_t bal = __ballot_sync(0xffffffffu, own);
            if (lane == 0) s_wcnt[warp] = __popc(bal);
            __syncthreads();
            int before = nk, total = 0;
#pragma unroll
            for (int w2 = 0; w2 < kDecWarps; w2++) {
                const int cw = s_wcnt[w2];
                before += w2 < warp ? cw : 0;
                total += cw;
            }
            if (own) rowlist[before + __popc(bal & ((1u << lane) - 1u))] = r;
            nk += total;
            __syncthreads();
        }
        for (int base = 0; base < nk; base += NT) {
            const int nc = min(NT, nk - base);
            const int NP = (nc + 15) & ~15;
            // 1. priors of the chunk's pixels (zero rows pad the chunk to NP)
            if (tid < NP) {
                uint32_t w8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                if (tid < nc) {
                    const int r = rowlist[base + tid], c = t - 3 * r;
#pragma unroll
                    for (int q = 0; q < kPriors; q++) {
                        const int dr = q < 5 ? -2 : (q < 10 ? -1 : 0);
                        const int dc = q < 5 ? q - 2 : (q < 10 ? q - 7 : q - 12);
                        const int rr = r + dr, cc = c + dc;
                        const int v = (rr >= 0 && cc >= 0 && cc < W) ? ring[((rr & rmask) << 4) + (cc & 15)] : 0;
                        w8[q >> 1] |= (uint32_t)tc::bf16_of_int(v - 128) << (16 * (q & 1));
                    }
                }
                *reinterpret_cast<uint4 *>(b1 + tc::kmajor_offset(tid, 0, 16)) = make_uint4(w8[0], w8[1], w8[2], w8[3]);
                *reinterpret_cast<uint4 *>(b1 + tc::kmajor_offset(tid, 8, 16)) = make_uint4(w8[4], w8[5], w8[6], w8[7]);
            }
            // 2. the three layers
            run_layer(1, NP);
            hidden_epilogue(NP, s1r, o1r);
            run_layer(2, NP);
            hidden_epilogue(NP, s2r, o2r);
            run_layer(3, NP);
            for (int c0 = 16 * cg; c0 < NP; c0 += 32) {
                uint32_t va[16], vb[16];
                tc::tmem_ld16(tm_q + (uint32_t)c0, va);
                tc::tmem_ld16(tm_q + (uint32_t)(NP + c0), vb);
                tc::tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < 16; e++) {
                    zb[(c0 + e) * kSymbols + unit] = __fmaf_rn(__uint_as_float(va[e]), s3a, o3a);
                    zb[(c0 + e) * kSymbols + 128 + unit] = __fmaf_rn(__uint_as_float(vb[e]), s3b, o3b);
                }
            }
            tc::fence_before_sync();
            __syncthreads();
            // 3. tables and rANS steps, one warp per pixel; pixels that share a
            //    stream go to the same warp (by local stream index), in row
            //    order.
            for (int i = 0; i < nc; i++) {
                const int r = rowlist[base + i], c = t - 3 * r;
                const int g = (r % S) / P;
                if (g % kDecWarps != warp) continue;
                const float4 za = *reinterpret_cast<const float4 *>(zb + i * kSymbols + 8 * lane);
                const float4 zc = *reinterpret_cast<const float4 *>(zb + i * kSymbols + 8 * lane + 4);
                const float z[8] = {za.x, za.y, za.z, za.w, zc.x, zc.y, zc.z, zc.w};
                float mx = z[0];
#pragma unroll
                for (int q = 1; q < 8; q++) mx = z[q] > mx ? z[q] : mx;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
                uint32_t w[8], lsum = 0;
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    w[q] = table_weight(mx, z[q], m.tscale, lut);
                    lsum += w[q];
                }
                uint32_t incl = lsum;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
                    if (lane >= off) incl += o;
                }
                const uint32_t Wsum = __shfl_sync(0xffffffffu, incl, 31);
                const uint32_t Q = table_q_fast(Wsum);
                const uint32_t excl = incl - lsum;
                const uint32_t x = st_x[g];
                const uint32_t slot = x & 0xFFFFu;
                const uint32_t cs = 8u * lane + __umulhi(excl, Q);
                const uint32_t ball = __ballot_sync(0xffffffffu, cs <= slot);
                const int Lh = 31 - __clz(ball);
                uint32_t sym = 0, f = 1, clo = 0;
                if (lane == Lh) {
                    uint32_t Pp = excl;
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const uint32_t i8 = 8u * lane + q;
                        const uint32_t lo = i8 + __umulhi(Pp, Q);
                        const uint32_t hi = i8 == 255 ? kTotal : i8 + 1u + __umulhi(Pp + w[q], Q);
                        if (hi > slot) {
                            sym = i8;
                            f = hi - lo;
                            clo = lo;
                            break;
                        }
                        Pp += w[q];
                    }
                }
                sym = __shfl_sync(0xffffffffu, sym, Lh);
                f = __shfl_sync(0xffffffffu, f, Lh);
                clo = __shfl_sync(0xffffffffu, clo, Lh);
                if (lane == 0) {
                    uint32_t xn = f * (x >> 16) + slot - clo;
                    if (xn < kRansL) {
                        const uint32_t pos = st_pos[g];
                        if (pos < st_end[g]) {
                            xn = (xn << 16) | wsrc[pos];
                            st_pos[g] = pos + 1;
                        } else {
                            s_err = 1;
                        }
                    }
                    st_x[g] = xn;
                    im.pixels[(int64_t)r * im.pitch + c] = (uint8_t)sym;
                }
                if (lane < P) {
                    const uint32_t a = ring_addr + (uint32_t)(((r & rmask) << 4) + (c & 15));
                    if (P > 1)
                        st_cluster_u8(map_shared(a, (uint32_t)lane), sym);
                    else
                        ring[((r & rmask) << 4) + (c & 15)] = (uint8_t)sym;
                }
                __syncwarp();
            }
            __syncthreads();
        }
        if (P > 1)
            cluster_sync_all();
        else
            __syncthreads();
    }
    // final states must be back at the initial value with every word read
    for (int g = tid; g < G; g += kDecThreads)
        if (st_x[g] != kRansL || st_pos[g] != st_end[g]) s_err = 1;
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && (s_err || s_fail))
        atomicMax(b.status + img_idx, s_fail ? (int)DLIC_ERR_TIMEOUT : (int)DLIC_ERR_CORRUPT);
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tm, 256);
    }
    if (P > 1) cluster_sync_all();   // no CTA leaves while others may still write its ring
}

bool tc_decode_supported(const DevModel &m) {
    return m.precision == DLIC_INT8 && m.tc_w != nullptr && m.h1 == kDecHidden && m.h2 == kDecHidden;
}

// Chooses the cluster size and chunking for a batch and launches the kernel.
// P = 8 when the batch is small enough for every image to get its own
// 8-SM cluster, else one CTA per image.
cudaError_t launch_decode_tc(const DevModel &m, const DecBatch &b, int cluster, int num_sms, cudaStream_t st) {
    if (b.n == 0) return cudaSuccess;
    int maxH = 1, maxW = 1;
    for (int i = 0; i < b.n; i++) {
        maxH = max(maxH, b.img[i].H);
        maxW = max(maxW, b.img[i].W);
    }
    int P = cluster;
    if (P <= 0) P = (b.n * 8 <= num_sms) ? 8 : 1;
    const int wave_px = min(maxH, (maxW + 2) / 3);
    const int per_cta = (wave_px + P - 1) / P + 1;
    DecTcParams prm;
    prm.P = P;
    prm.nt = min(64, (per_cta + 15) & ~15);
    int rows = 1;
    while (rows < min(maxH, (maxW + 2) / 3) + 4) rows <<= 1;
    prm.ring_rows = rows;
    prm.max_g = (min(maxH, 65535) + P - 1) / P;
    const DecTcLayout L0 = dec_layout(prm.nt, rows, prm.max_g, 0);
    const int budget = 227 * 1024 - 4096;
    prm.pay_words = L0.total < (uint32_t)budget ? (int)((budget - L0.total) / 2) & ~63 : 0;
    if (prm.pay_words > 65536) prm.pay_words = 65536;
    const DecTcLayout L = dec_layout(prm.nt, rows, prm.max_g, prm.pay_words);
    if (L.total > (uint32_t)(227 * 1024)) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_decode_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    if (P > 8) {
        e = cudaFuncSetAttribute(k_decode_tc, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(b.n * P));
    cfg.blockDim = dim3(kDecThreads);
    cfg.dynamicSmemBytes = L.total;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_decode_tc, m, b, prm);
}

}  // namespace dlic
