// Training step of the density network (row a7): categorical cross-entropy
// in bits (Sec. III-A, Table I reports "vloss in bpp"), hand-written forward
// and backward (adjoint) kernels, Adam on FP32 master weights.
//
//   x  = v / 128 - 1 (12 priors, padded to 16)
//   a1 = x W1^T + b1,  h1 = relu(a1)
//   a2 = h1 W2^T + b2, h2 = relu(a2)
//   z  = h2 W3^T + b3, loss = mean_b (logsumexp(z_b) - z_b[y_b]) / ln 2
//   dz = (softmax(z) - onehot(y)) / (B ln 2)
//   dW3 = dz^T h2, db3 = sum dz, dh2 = dz W3, da2 = dh2 * [a2 > 0]
//   dW2 = da2^T h1, db2 = sum da2, dh1 = da2 W2, da1 = dh1 * [a1 > 0]
//   dW1 = da1^T x,  db1 = sum da1
//
// Two arithmetic modes: BF16 operands with FP32 accumulation on the tensor
// cores (tcgen05, TMA-fed, epilogues fused), and plain FP32 on the CUDA
// cores.  Every product is a GEMM C = A B^T.  In the BF16 modes the
// activations stay row-major [batch][features]: the weight gradients read
// them as MN-major operands, so no transposed copy of an activation is
// written; the Adam kernel keeps row-major and transposed bf16 copies of the
// weights.  The FP32 GEMMs take K-major operands only, so in that mode the
// producing epilogues also write transposed copies of the activations.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "internal.cuh"
#include "tc.cuh"

namespace dlic {

constexpr float kLn2 = 0.69314718055994530942f;
constexpr float kLog2e = 1.44269504088896340736f;
constexpr long long kGemmWaitLimit = 4000000000LL;

enum Epi { EPI_F32 = 0, EPI_BIAS_RELU = 1, EPI_SOFTMAX = 2, EPI_RELU_GRAD = 3 };

// Arguments of the row epilogues (per GEMM output row m, N columns).
struct EpiArgs {
    int M, N;
    int ldc;                    // EPI_F32: row stride of C
    int ldT;                    // row stride (pitch) of the transposed outputs [N][ldT]
    float *c;                   // EPI_F32: output (+ blockIdx.z * M * ldc)
    const float *bias;          // BIAS_RELU, SOFTMAX
    void *out, *outT;           // row-major [M][N] and transposed [N][M] outputs (bf16 or fp32)
    const void *act;            // RELU_GRAD (FP32 path): activation [M][N] whose sign masks the gradient
    const uint16_t *mask;       // RELU_GRAD (BF16 paths): that sign as bits, [M][N / 16] words
    uint16_t *mask_out;         // BIAS_RELU (BF16 paths): the output's sign bits, [M][N / 16] words
    const uint8_t *tgt;         // SOFTMAX: targets
    float inv_batch_ln2;        // SOFTMAX: 1 / (B ln 2)
    const float *vw;            // SOFTMAX: loss weight per target value (frequency-weighted loss), or null
    const float *wnorm;         // SOFTMAX with vw: device {1 / (W ln 2), 1 / W}, W = sum_b vw[y_b]
    float *colsum;              // per-CTA column sums [gridDim.x][N] (db), or null
    float *loss;                // SOFTMAX: per-CTA loss sums [gridDim.x]
    int bf16;                   // outputs (and act) are bf16, else fp32
    int split;                  // bf16 outputs also get a low plane: lo = bf16(v - hi)
    size_t out_plane, outT_plane; // element offsets of the low planes
};

__device__ __forceinline__ uint16_t f2bf(float f) {
    const __nv_bfloat16 b = __float2bfloat16_rn(f);
    return *reinterpret_cast<const uint16_t *>(&b);
}
__device__ __forceinline__ float bf2f(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }

__device__ __forceinline__ void store_val(const EpiArgs &e, void *base, size_t idx, float v, size_t plane) {
    if (e.bf16) {
        const uint16_t hi = f2bf(v);
        reinterpret_cast<uint16_t *>(base)[idx] = hi;
        if (e.split) reinterpret_cast<uint16_t *>(base)[idx + plane] = f2bf(v - bf2f(hi));
    } else {
        reinterpret_cast<float *>(base)[idx] = v;
    }
}
__device__ __forceinline__ float load_val(const EpiArgs &e, const void *base, size_t idx) {
    return e.bf16 ? bf2f(reinterpret_cast<const uint16_t *>(base)[idx]) : reinterpret_cast<const float *>(base)[idx];
}

// A source of one output row in chunks of 16 columns.
struct TmemRow {
    uint32_t taddr;
    __device__ __forceinline__ void load16(int n0, float (&v)[16]) const {
        uint32_t u[16];
        tc::tmem_ld16(taddr + (uint32_t)n0, u);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = __uint_as_float(u[j]);
    }
};
struct GlobalRow {
    const float *p;
    __device__ __forceinline__ void load16(int n0, float (&v)[16]) const {
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
            const float4 q = *reinterpret_cast<const float4 *>(p + n0 + j);
            v[j] = q.x; v[j + 1] = q.y; v[j + 2] = q.z; v[j + 3] = q.w;
        }
    }
};

// Adds 16 column values of this thread's row into the shared column
// partials: a reduce-scatter across the warp (each lane ends with one
// column's warp total for lanes 0..15 after four halving steps), then one
// plain store per column into the warp's slot, cs[slot * stride + column].
// Exactly one warp writes each (slot, column), and the four slots are added
// in a fixed order afterwards, so the bias gradients are the same bits on
// every run.
__device__ __forceinline__ void colsum_add(float *cs, int slot, int stride, float (&v)[16]) {
    const int lane = threadIdx.x & 31;
    float a[16];
#pragma unroll
    for (int j = 0; j < 16; j++) a[j] = v[j];
#pragma unroll
    for (int step = 8; step >= 1; step >>= 1) {
        const bool upper = (lane & step) != 0;
#pragma unroll
        for (int j = 0; j < step; j++) {
            const float send = upper ? a[j] : a[j + step];
            const float keep = upper ? a[j + step] : a[j];
            a[j] = keep + __shfl_xor_sync(0xffffffffu, send, step);
        }
    }
    // lane holds the sum over its 16-lane half for column (lane & 15)
    a[0] += __shfl_xor_sync(0xffffffffu, a[0], 16);
    if (lane < 16) cs[slot * stride + lane] = a[0];
}

// Column sums go through shared memory: `cs` holds four slots of N floats
// zeroed by the caller; warp w of the CTA's four stores its rows' column
// totals into slot w (colsum_add).
template <class Row>
__device__ void row_epilogue(int epi, const EpiArgs &e, const Row &row, int m, bool valid, float *cs,
                             float *loss_acc) {
    const int N = e.N;
    const int cslot = (threadIdx.x >> 5) & 3;
    if (epi == EPI_F32) {
        if (!valid) return;
        float *c = e.c + (size_t)blockIdx.z * e.M * e.ldc + (size_t)m * e.ldc;
        for (int n0 = 0; n0 < N; n0 += 16) {
            float v[16];
            row.load16(n0, v);
#pragma unroll
            for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4 *>(c + n0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
        return;
    }
    if (epi == EPI_BIAS_RELU) {
        for (int n0 = 0; n0 < N; n0 += 16) {
            float v[16];
            row.load16(n0, v);
            if (!valid) continue;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const float h = fmaxf(v[j] + e.bias[n0 + j], 0.0f);
                store_val(e, e.out, (size_t)m * N + n0 + j, h, e.out_plane);
                store_val(e, e.outT, (size_t)(n0 + j) * e.ldT + m, h, e.outT_plane);
            }
        }
        return;
    }
    if (epi == EPI_RELU_GRAD) {
        for (int n0 = 0; n0 < N; n0 += 16) {
            float v[16];
            row.load16(n0, v);
            if (!valid) {
                if (cs) {
#pragma unroll
                    for (int j = 0; j < 16; j++) v[j] = 0.0f;
                    colsum_add(cs + n0, cslot, N, v);
                }
                continue;
            }
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const float a = load_val(e, e.act, (size_t)m * N + n0 + j);
                const float g = a > 0.0f ? v[j] : 0.0f;
                if (e.out) store_val(e, e.out, (size_t)m * N + n0 + j, g, e.out_plane);
                store_val(e, e.outT, (size_t)(n0 + j) * e.ldT + m, g, e.outT_plane);
                v[j] = g;
            }
            if (cs) colsum_add(cs + n0, cslot, N, v);
        }
        return;
    }
    // EPI_SOFTMAX: loss in bits and dz = (softmax - onehot) / (B ln 2)
    float mx = -INFINITY;
    for (int n0 = 0; n0 < N; n0 += 16) {
        float v[16];
        row.load16(n0, v);
#pragma unroll
        for (int j = 0; j < 16; j++) mx = fmaxf(mx, v[j] + e.bias[n0 + j]);
    }
    float se = 0.0f;
    for (int n0 = 0; n0 < N; n0 += 16) {
        float v[16];
        row.load16(n0, v);
#pragma unroll
        for (int j = 0; j < 16; j++) se += expf(v[j] + e.bias[n0 + j] - mx);
    }
    const float lse = mx + logf(se);
    const int y = valid ? e.tgt[m] : 0;
    const float inv = 1.0f / se;
    // the row's gradient scale and loss weight: 1 / (B ln 2) and 1, or with
    // value weights w_y / (W ln 2) and w_y / W
    const float rw = e.vw ? e.vw[y] : 1.0f;
    const float gscale = e.vw ? rw * e.wnorm[0] : e.inv_batch_ln2, lw = e.vw ? rw * e.wnorm[1] : 1.0f;
    for (int n0 = 0; n0 < N; n0 += 16) {
        float v[16];
        row.load16(n0, v);
        if (!valid) {
            if (cs) {
#pragma unroll
                for (int j = 0; j < 16; j++) v[j] = 0.0f;
                colsum_add(cs + n0, cslot, N, v);
            }
            continue;
        }
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const float zz = v[j] + e.bias[n0 + j];
            float g = expf(zz - mx) * inv;
            if (n0 + j == y) {
                g -= 1.0f;
                *loss_acc += lw * ((lse - zz) / kLn2);
            }
            g *= gscale;
            store_val(e, e.out, (size_t)m * N + n0 + j, g, e.out_plane);
            store_val(e, e.outT, (size_t)(n0 + j) * e.ldT + m, g, e.outT_plane);
            v[j] = g;
        }
        if (cs) colsum_add(cs + n0, cslot, N, v);
    }
}

// ---------------------------------------------------------------------------
// tcgen05 GEMM: C[M x N] = A[M x K] * B[N x K]^T, bf16 operands fed by TMA
// with 128-byte swizzling, FP32 accumulators in tensor memory, a fused
// epilogue.  One 128 x N tile per CTA (N <= 256); split-K over gridDim.z for
// EPI_F32.
//
// Each operand is read either K-major (a row of 64 K values per M or N
// index, 128 bytes) or MN-major (a row of 64 M or N values per K index):
// the weight gradients dW = dY^T X take both factors straight from the
// row-major activations [batch][features], so no transposed copy of any
// activation is ever written.  An MN-major tile is a column of 64-wide
// boxes, 8 KB apart; columns past the operand's extent are zero-filled (or,
// for whole boxes, skipped: they only feed outputs that are discarded).
//
// Warp 0 loads, warp 1 issues MMAs, warps 2..9 run the epilogue: two warps
// per tensor-memory lane quarter, each on half of the columns of its 32
// rows, with row-major outputs leaving as 16-byte vectors.
// ---------------------------------------------------------------------------
constexpr int kGemmThreads = 320;
constexpr int kEpiThreads = 256;
constexpr int kGemmMaxStages = 4;

struct GemmCfg {
    int stages;      // pipeline depth (<= kGemmMaxStages)
    int a_mn, b_mn;  // operand major-ness (1 = MN-major)
    int n_mma;       // MMA N: N rounded up to 16 (K-major B) or 64 (MN-major B)
    int b_boxes;     // MN-major B: 64-wide boxes inside the operand
};

// K-major, 128-byte swizzle: 8-row groups 1024 bytes apart; a K step of 16
// advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t desc_k128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
// MN-major, 128-byte swizzle: 64-wide MN blocks 8192 bytes apart (leading
// byte offset), 8-row K groups 1024 bytes apart (stride byte offset); a K
// step of 16 advances the start address by 2048 bytes.
__device__ __forceinline__ uint64_t desc_mn128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(8192 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_addr(bar)), "r"(bytes) : "memory");
}
// 2^x with the MUFU approximation (relative error about 2^-22; flushes
// results below 2^-126 to zero).
__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 2, %0;" ::"r"(kEpiThreads) : "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// bf16 > 0 for the two halves of a packed pair, as bits 0 and 1.
__device__ __forceinline__ uint32_t bf16x2_positive(uint32_t p) {
    const uint32_t lo = p & 0xFFFFu, hi = p >> 16;
    return (uint32_t)(lo != 0u && (lo & 0x8000u) == 0u) | ((uint32_t)(hi != 0u && (hi & 0x8000u) == 0u) << 1);
}

// 16 consecutive values of row m as bf16 (and, in split mode, the low plane
// bf16(v - hi)) with two 16-byte stores per plane.  Returns which of the
// stored (high-plane) values are positive, bit j for value j.
__device__ __forceinline__ uint32_t store_row16(const EpiArgs &e, const float (&v)[16], int m, int n0) {
    uint32_t hi[8];
#pragma unroll
    for (int j = 0; j < 8; j++) hi[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
    uint32_t pos = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) pos |= bf16x2_positive(hi[j]) << (2 * j);
    uint4 *o = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(e.out) + (size_t)m * e.N + n0);
    o[0] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    o[1] = make_uint4(hi[4], hi[5], hi[6], hi[7]);
    if (e.split) {
        uint32_t lo[8];
#pragma unroll
        for (int j = 0; j < 8; j++)
            lo[j] = pack_bf16x2(v[2 * j] - __uint_as_float(hi[j] << 16), v[2 * j + 1] - __uint_as_float(hi[j] & 0xFFFF0000u));
        uint4 *ol = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(e.out) + e.out_plane + (size_t)m * e.N + n0);
        ol[0] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        ol[1] = make_uint4(lo[4], lo[5], lo[6], lo[7]);
    }
    return pos;
}

// Walks this thread's 16-column chunks [n_lo, n_hi) of its tensor-memory row,
// loading the next chunk while the current one is processed.
template <class F>
__device__ __forceinline__ void for_chunks(uint32_t taddr, int n_lo, int n_hi, F &&f) {
    if (n_lo >= n_hi) return;
    uint32_t cur[16], nxt[16];
    tc::tmem_ld16(taddr + (uint32_t)n_lo, cur);
    tc::tmem_wait_ld();
    for (int n0 = n_lo; n0 < n_hi; n0 += 16) {
        const bool more = n0 + 16 < n_hi;
        if (more) tc::tmem_ld16(taddr + (uint32_t)(n0 + 16), nxt);
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = __uint_as_float(cur[j]);
        f(n0, v);
        if (more) {
            tc::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; j++) cur[j] = nxt[j];
        }
    }
}

// SPLIT: operands come as high and low bf16 planes (x = hi + lo) and every K
// step issues hi*hi + lo*hi + hi*lo, which keeps about 16 significant bits of
// each operand.
template <bool SPLIT, bool PERSIST>
__global__ void __launch_bounds__(kGemmThreads, SPLIT || PERSIST ? 1 : 2)
    k_gemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const __grid_constant__ CUtensorMap mapAl, const __grid_constant__ CUtensorMap mapBl, int K,
              int kb_per_split, int epi, GemmCfg g, EpiArgs e, int *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[kGemmMaxStages], empty[kGemmMaxStages], tfull[2], tempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    __shared__ float cs[4 * 256];   // column partials, one slot per lane quarter
    __shared__ __align__(16) float s_bias[256];
    __shared__ float red[2][2][128];
    __shared__ float s_loss[kGemmThreads / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = e.N, NS = g.stages;
    const uint32_t a_bytes = 128 * 128, b_bytes = (uint32_t)g.n_mma * 128;
    const uint32_t b_al = (b_bytes + 1023) & ~1023u;
    const uint32_t stage_bytes = SPLIT ? 2 * (a_bytes + b_al) : a_bytes + b_al;
    // tiles of this CTA: m-tiles blockIdx.x, blockIdx.x + gridDim.x, ...;
    // with two accumulators the epilogue of one tile overlaps the loads and
    // MMAs of the next
    const int mt = (e.M + 127) / 128, nacc = PERSIST ? 2 : 1;
    const int ntiles = !PERSIST ? 1 : (int)blockIdx.x < mt ? (mt - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t b_load = g.b_mn ? 8192u * g.b_boxes : b_bytes;
    const int nkb_total = (K + 63) / 64;
    const int kb0 = blockIdx.z * kb_per_split;
    const int kb1 = min(nkb_total, kb0 + kb_per_split);
    const int nkb = max(0, kb1 - kb0);

    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 256 * nacc);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < NS; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; a++) {
            tc::mbar_init(&tfull[a], 1);
            tc::mbar_init(&tempty[a], kEpiThreads / 32);   // one arrival per epilogue warp
        }
        tc::fence_mbar_init();
        s_fail = 0;
    }
    for (int n = tid; n < 4 * 256; n += kGemmThreads) cs[n] = 0.0f;
    for (int n = tid; n < 256; n += kGemmThreads) {
        // the softmax works in base 2: its bias is stored pre-scaled by log2(e)
        const float bv = e.bias && n < N ? e.bias[n] : 0.0f;
        s_bias[n] = epi == EPI_SOFTMAX ? bv * kLog2e : bv;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = tmem_base;

    if (warp == 0 && lane == 0) {
        // producer: every K block of every tile through the NS stages
        int it = 0;
        for (int j = 0; j < ntiles && !*reinterpret_cast<volatile int *>(&s_fail); j++) {
            const int m0 = ((int)blockIdx.x + j * (int)gridDim.x) * 128;
            // bytes a stage's loads deliver (whole boxes past the extent are skipped)
            const int a_boxes = m0 + 64 < e.M ? 2 : 1;
            const uint32_t a_load = g.a_mn ? 8192u * a_boxes : a_bytes;
            // the sign bits that will mask this tile's gradient, pulled into L2
            if (epi == EPI_RELU_GRAD) {
                const uint32_t bytes = (uint32_t)(min(128, e.M - m0) * (N / 16) * 2);
                const void *src = e.mask + (size_t)m0 * (N / 16);
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"((bytes + 15u) & ~15u)
                             : "memory");
            }
            for (int i = 0; i < nkb; i++, it++) {
                const int s = it % NS;
                if (!tc::mbar_wait(&empty[s], ((it / NS) & 1) ^ 1, kGemmWaitLimit)) { s_fail = 1; break; }
                uint8_t *st = smem + s * stage_bytes;
                const int k = (kb0 + i) * 64;
                const uint32_t bar = tc::smem_addr(&full[s]);
                mbar_expect_tx(&full[s], SPLIT ? 2 * (a_load + b_load) : a_load + b_load);
#pragma unroll 1
                for (int pl = 0; pl < (SPLIT ? 2 : 1); pl++) {
                    const CUtensorMap *ma = pl ? &mapAl : &mapA, *mb = pl ? &mapBl : &mapB;
                    uint8_t *sa = st + pl * (a_bytes + b_al), *sb = sa + a_bytes;
                    if (g.a_mn)
                        for (int h = 0; h < a_boxes; h++) tma_load_2d(tc::smem_addr(sa + 8192 * h), ma, m0 + 64 * h, k, bar);
                    else
                        tma_load_2d(tc::smem_addr(sa), ma, k, m0, bar);
                    if (g.b_mn)
                        for (int h = 0; h < g.b_boxes; h++) tma_load_2d(tc::smem_addr(sb + 8192 * h), mb, 64 * h, k, bar);
                    else
                        tma_load_2d(tc::smem_addr(sb), mb, k, (int)blockIdx.y * N, bar);   // n-block of a wide B
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = tc::idesc_bf16_f32(128, g.n_mma) | ((uint32_t)g.a_mn << 15) | ((uint32_t)g.b_mn << 16);
        // start-address step per K = 16 (descriptor units of 16 bytes)
        const uint32_t astep = g.a_mn ? 128u : 2u, bstep = g.b_mn ? 128u : 2u;
        int it = 0;
        for (int j = 0; j < ntiles && !*reinterpret_cast<volatile int *>(&s_fail); j++) {
            const int acc = j % nacc;
            const uint32_t tma = tm + 256u * (uint32_t)acc;
            // the epilogue of the tile that last used this accumulator is done
            if (j >= nacc && !tc::mbar_wait(&tempty[acc], ((j / nacc) - 1) & 1, kGemmWaitLimit)) { s_fail = 1; break; }
            tc::fence_after_sync();
            for (int i = 0; i < nkb; i++, it++) {
                const int s = it % NS;
                if (!tc::mbar_wait(&full[s], (it / NS) & 1, kGemmWaitLimit)) { s_fail = 1; break; }
                tc::fence_after_sync();
                uint8_t *st = smem + s * stage_bytes;
                auto dA = [&](uint8_t *p) { return g.a_mn ? desc_mn128(tc::smem_addr(p)) : desc_k128(tc::smem_addr(p)); };
                auto dB = [&](uint8_t *p) { return g.b_mn ? desc_mn128(tc::smem_addr(p)) : desc_k128(tc::smem_addr(p)); };
                const uint64_t da = dA(st), db = dB(st + a_bytes);
#pragma unroll
                for (int ks = 0; ks < 4; ks++) tc::mma_bf16(tma, da + astep * ks, db + bstep * ks, idesc, (i | ks) != 0);
                if (SPLIT) {
                    const uint64_t dal = dA(st + a_bytes + b_al), dbl = dB(st + 2 * a_bytes + b_al);
#pragma unroll
                    for (int ks = 0; ks < 4; ks++) {
                        tc::mma_bf16(tma, dal + astep * ks, db + bstep * ks, idesc, 1u);
                        tc::mma_bf16(tma, da + astep * ks, dbl + bstep * ks, idesc, 1u);
                    }
                }
                tc::mma_commit(&empty[s]);
            }
            tc::mma_commit(&tfull[acc]);
        }
    } else if (warp >= 2) {
      const int etid = tid - 64;   // epilogue thread 0 .. kEpiThreads - 1
      for (int j = 0; j < ntiles; j++) {
        const int acc = j % nacc, tile = (int)blockIdx.x + j * (int)gridDim.x, m0 = tile * 128;
        if (lane == 0 && !*reinterpret_cast<volatile int *>(&s_fail) &&
            !tc::mbar_wait(&tfull[acc], (j / nacc) & 1, kGemmWaitLimit))
            s_fail = 1;
        __syncwarp();
        if (!*reinterpret_cast<volatile int *>(&s_fail)) tc::mbar_wait(&tfull[acc], (j / nacc) & 1, 1000);   // every lane observes the completed phase
        tc::fence_after_sync();
        float loss_acc = 0.0f;
        const int q = warp & 3, hf = (warp - 2) >> 2;
        const int row = 32 * q + lane, m = m0 + row;
        const bool valid = m < e.M;
        // the two halves split the 16-column chunks (the first takes the odd one)
        const int nch = N / 16, first = (nch + 1) / 2;
        int n_lo = hf ? 16 * first : 0, n_hi = hf ? N : 16 * first;
        if (s_fail) n_hi = n_lo;
        const uint32_t taddr = tm + 256u * (uint32_t)acc + ((uint32_t)(32 * q) << 16);
        if (epi == EPI_F32) {
            float *c = e.c + (size_t)blockIdx.z * e.M * e.ldc + (size_t)m * e.ldc + (size_t)blockIdx.y * N;
            if (nkb == 0) {
                if (valid)
                    for (int n0 = n_lo; n0 < n_hi; n0 += 4) *reinterpret_cast<float4 *>(c + n0) = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                for_chunks(taddr, n_lo, n_hi, [&](int n0, float (&v)[16]) {
                    if (valid)
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            *reinterpret_cast<float4 *>(c + n0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                });
            }
        } else if (epi == EPI_BIAS_RELU) {
            for_chunks(taddr, n_lo, n_hi, [&](int n0, float (&v)[16]) {
#pragma unroll
                for (int j = 0; j < 16; j++) v[j] = fmaxf(v[j] + s_bias[n0 + j], 0.0f);
                if (valid) {
                    const uint32_t pos = store_row16(e, v, m, n0);
                    if (e.mask_out) e.mask_out[(size_t)m * (N / 16) + n0 / 16] = (uint16_t)pos;
                }
            });
        } else if (epi == EPI_RELU_GRAD) {
            // the sign bits of the activation that masks the gradient (written
            // by its forward epilogue), one chunk ahead
            const uint16_t *mp = e.mask + (size_t)m * (N / 16);
            uint32_t mb = valid && n_lo < n_hi ? mp[n_lo / 16] : 0u;
            for_chunks(taddr, n_lo, n_hi, [&](int n0, float (&v)[16]) {
                const uint32_t bits = mb;
                if (valid && n0 + 16 < n_hi) mb = mp[n0 / 16 + 1];
#pragma unroll
                for (int j = 0; j < 16; j++) v[j] = (bits >> j) & 1u ? v[j] : 0.0f;
                if (valid) store_row16(e, v, m, n0);
                if (e.colsum) colsum_add(cs + n0, q, 256, v);
            });
        } else {
            // EPI_SOFTMAX: running maximum and rescaled sum over this half's
            // columns in base 2 (z2 = z log2 e), then the halves combine
            // through shared memory
            float m2 = -INFINITY, s2 = 0.0f;
            for_chunks(taddr, n_lo, n_hi, [&](int n0, float (&v)[16]) {
                float z[16], cm = m2;
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    z[j] = fmaf(v[j], kLog2e, s_bias[n0 + j]);
                    cm = fmaxf(cm, z[j]);
                }
                float add = 0.0f;
#pragma unroll
                for (int j = 0; j < 16; j++) add += fast_exp2(z[j] - cm);
                s2 = s2 * fast_exp2(m2 - cm) + add;
                m2 = cm;
            });
            red[0][hf][row] = m2;
            red[1][hf][row] = s2;
            epi_sync();
            const float ma = red[0][0][row], mb = red[0][1][row];
            const float mx = fmaxf(ma, mb);
            const float se = red[1][0][row] * fast_exp2(ma - mx) + red[1][1][row] * fast_exp2(mb - mx);
            const float lse2 = mx + log2f(se);
            const int y = valid ? e.tgt[m] : -1;
            // the row's gradient scale and loss weight: 1 / (B ln 2) and 1,
            // or with value weights w_y / (W ln 2) and w_y / W
            const float rw = e.vw && valid ? e.vw[y] : 1.0f;
            const float rs = e.vw ? rw * e.wnorm[0] : e.inv_batch_ln2, lw = e.vw ? rw * e.wnorm[1] : 1.0f;
            const float scale = valid ? rs / se : 0.0f;
            for_chunks(taddr, n_lo, n_hi, [&](int n0, float (&v)[16]) {
                const bool has_y = (y & ~15) == n0;
                if (has_y) {
                    // -log2 p_y = lse2 - z2_y
#pragma unroll
                    for (int j = 0; j < 16; j++)
                        if (n0 + j == y) loss_acc += lw * (lse2 - fmaf(v[j], kLog2e, s_bias[n0 + j]));
                }
#pragma unroll
                for (int j = 0; j < 16; j++) v[j] = fast_exp2(fmaf(v[j], kLog2e, s_bias[n0 + j]) - mx) * scale;
                if (has_y) {
#pragma unroll
                    for (int j = 0; j < 16; j++)
                        if (n0 + j == y) v[j] -= rs;
                }
                if (valid) store_row16(e, v, m, n0);
                if (e.colsum) colsum_add(cs + n0, q, 256, v);
            });
        }
        for (int off = 16; off > 0; off >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
        if (lane == 0) s_loss[warp] = loss_acc;
        tc::fence_before_sync();
        epi_sync();   // the tile's accumulator is read out, its column and loss partials are in place
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(&tempty[acc])) : "memory");
        if (e.colsum)
            for (int n = etid; n < N; n += kEpiThreads)
                e.colsum[(size_t)tile * N + n] = ((cs[n] + cs[256 + n]) + cs[512 + n]) + cs[768 + n];
        if (e.loss && etid == 0) {
            float t = 0.0f;
            for (int w = 2; w < kGemmThreads / 32; w++) t += s_loss[w];
            e.loss[tile] = t;
        }
        epi_sync();   // (the next tile overwrites the partials)
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && s_fail) atomicExch(err, DLIC_ERR_TIMEOUT);
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tm, 256 * nacc);
    }
}

// ---------------------------------------------------------------------------
// CUDA-core FP32 GEMM: C = A B^T (fp32, K-major), 128 x 128 tiles, 8 x 8
// outputs per thread, raw FP32 output (split-K over gridDim.z).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gemm_f32(const float *A, int lda, const float *B, int ldb, float *C, int M,
                                                  int N, int K, int k_per_split, int ldc) {
    __shared__ float As[8][128 + 4];
    __shared__ float Bs[8][128 + 4];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * 128;
    const int kbeg = blockIdx.z * k_per_split, kend = min(K, kbeg + k_per_split);
    const int tr = tid / 16, tc_ = tid % 16;
    float acc[8][8] = {};
    for (int k0 = kbeg; k0 < kend; k0 += 8) {
        // each thread loads 4 elements of A and 4 of B (transposed into smem)
        for (int i = 0; i < 4; i++) {
            const int idx = tid + 256 * i;         // 0..1023 = 128 rows x 8 k
            const int r = idx / 8, kk = idx % 8;
            const int gk = k0 + kk;
            As[kk][r] = (m0 + r < M && gk < kend) ? A[(size_t)(m0 + r) * lda + gk] : 0.0f;
            Bs[kk][r] = (n0 + r < N && gk < kend) ? B[(size_t)(n0 + r) * ldb + gk] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 8; kk++) {
            float a[8], b[8];
#pragma unroll
            for (int i = 0; i < 8; i++) a[i] = As[kk][tr * 8 + i];
#pragma unroll
            for (int j = 0; j < 8; j++) b[j] = Bs[kk][tc_ * 8 + j];
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 8; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    float *Cz = C + (size_t)blockIdx.z * M * ldc;
    for (int i = 0; i < 8; i++) {
        const int m = m0 + tr * 8 + i;
        if (m >= M) continue;
        for (int j = 0; j < 8; j++) {
            const int n = n0 + tc_ * 8 + j;
            if (n < N) Cz[(size_t)m * ldc + n] = acc[i][j];
        }
    }
}

// Row epilogue over an FP32 C in global memory (the FP32 path); 128 rows per
// CTA so the per-CTA column sums match the tensor-core kernel's layout.
__global__ void __launch_bounds__(128) k_row_epilogue(const float *C, int epi, EpiArgs e) {
    extern __shared__ float cs[];   // four slots of N column partials
    const int tid = threadIdx.x;
    for (int n = tid; n < 4 * e.N; n += 128) cs[n] = 0.0f;
    __syncthreads();
    const int m = blockIdx.x * 128 + tid;
    float loss_acc = 0.0f;
    GlobalRow src{C + (size_t)min(m, e.M - 1) * e.N};
    row_epilogue(epi, e, src, m, m < e.M, e.colsum ? cs : nullptr, &loss_acc);
    __shared__ float s_loss[4];
    for (int off = 16; off > 0; off >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
    if ((tid & 31) == 0) s_loss[tid >> 5] = loss_acc;
    __syncthreads();
    if (e.colsum)
        for (int n = tid; n < e.N; n += 128)
            e.colsum[(size_t)blockIdx.x * e.N + n] = ((cs[n] + cs[e.N + n]) + cs[2 * e.N + n]) + cs[3 * e.N + n];
    if (e.loss && tid == 0) e.loss[blockIdx.x] = s_loss[0] + s_loss[1] + s_loss[2] + s_loss[3];
}

// ---------------------------------------------------------------------------
// Small kernels: features, reductions, Adam, weight shadows.
// ---------------------------------------------------------------------------
// One network input: v / 128 - 1 for an 8-bit sample (u8 contexts), v /
// 2048 - 1 for a 12-bit one (u16 contexts, Sec. IV "Higher Bit Depth"); both
// exact in FP32.  A 12-bit sample above 4095 sets DLIC_ERR_INVALID.
__device__ __forceinline__ float ctx_input(const void *ctx, int wide, size_t i, int *err) {
    if (!wide) return (float)static_cast<const uint8_t *>(ctx)[i] * 0.0078125f - 1.0f;
    const uint32_t v = static_cast<const uint16_t *>(ctx)[i];
    if (v > 4095u) atomicExch(err, (int)DLIC_ERR_INVALID);
    return (float)v * 0.00048828125f - 1.0f;
}

// v / 128 - 1 has at most 8 significant bits: exact in bf16, low plane 0;
// v / 2048 - 1 has up to 12, and its low plane carries the rest.
// Network inputs of n_in priors per context, K padded to k1 (a multiple of
// 16); the transposed copy XT [k1][ldT] only for the FP32 path (XT
// non-null).  BF16: one context per thread; the 12-prior window of u8
// contexts reads three words and writes two 16-byte rows (plus a zero low
// plane in split mode).
__global__ void k_features(const void *ctx, int wide, int B, int n_in, int k1, int ldT, void *X, void *XT, int bf16,
                           size_t xplane, int *err) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (bf16 && (n_in != kPriors || wide)) {
        uint16_t *o = static_cast<uint16_t *>(X) + (size_t)b * k1;
        for (int k = 0; k < k1; k += 2) {
            const float x0 = k < n_in ? ctx_input(ctx, wide, (size_t)b * n_in + k, err) : 0.0f;
            const float x1 = k + 1 < n_in ? ctx_input(ctx, wide, (size_t)b * n_in + k + 1, err) : 0.0f;
            const uint32_t hi = pack_bf16x2(x0, x1);
            reinterpret_cast<uint32_t *>(o)[k / 2] = hi;
            if (xplane)
                reinterpret_cast<uint32_t *>(o + xplane)[k / 2] =
                    pack_bf16x2(x0 - bf2f((uint16_t)(hi & 0xFFFFu)), x1 - bf2f((uint16_t)(hi >> 16)));
        }
        return;
    }
    if (bf16) {
        const uint8_t *c = static_cast<const uint8_t *>(ctx) + (size_t)b * kPriors;
        const bool al4 = (reinterpret_cast<uintptr_t>(c) & 3u) == 0;
        uint32_t w[8];
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const uint32_t v = al4 ? reinterpret_cast<const uint32_t *>(c)[q]
                                   : c[4 * q] | (c[4 * q + 1] << 8) | (c[4 * q + 2] << 16) | ((uint32_t)c[4 * q + 3] << 24);
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const float x0 = (float)((v >> (16 * h)) & 0xFFu) * 0.0078125f - 1.0f;
                const float x1 = (float)((v >> (16 * h + 8)) & 0xFFu) * 0.0078125f - 1.0f;
                w[2 * q + h] = pack_bf16x2(x0, x1);
            }
        }
        w[6] = w[7] = 0u;
        uint4 *o = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(X) + (size_t)b * 16);
        o[0] = make_uint4(w[0], w[1], w[2], w[3]);
        o[1] = make_uint4(w[4], w[5], w[6], w[7]);
        if (xplane) {
            uint4 *ol = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(X) + xplane + (size_t)b * 16);
            ol[0] = ol[1] = make_uint4(0u, 0u, 0u, 0u);
        }
        return;
    }
    for (int k = 0; k < k1; k++) {
        const float x = k < n_in ? ctx_input(ctx, wide, (size_t)b * n_in + k, err) : 0.0f;
        reinterpret_cast<float *>(X)[(size_t)b * k1 + k] = x;
        reinterpret_cast<float *>(XT)[(size_t)k * ldT + b] = x;
    }
}

// First layer of the BF16 modes on the CUDA cores in FP32 (K = the
// window's priors, at most 96, is too thin for the tensor cores to pay):
// h1 = ReLU(b1 + sum_k W1[j][k] x_k), written as bf16 rows (and low planes
// when p1 != 0).  32 contexts per block, thread = hidden unit holding its
// NMAX weights (zero past n_in); the bf16 tile is staged in shared memory and
// leaves as 16-byte rows.
constexpr int kL1Ctx = 32;
template <int NMAX>
__global__ void __launch_bounds__(256) k_layer1(const void *ctx, int wide, int B, int n_in, const float *W1,
                                                const float *b1, int h1, uint16_t *H1, size_t p1, uint16_t *M1, int *err) {
    __shared__ __align__(16) uint16_t thi[kL1Ctx * kMaxHidden];
    __shared__ __align__(16) uint16_t tlo[kL1Ctx * kMaxHidden];
    __shared__ float xs[kL1Ctx][NMAX];
    __shared__ uint16_t smask[kL1Ctx][kMaxHidden / 16];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, b0 = blockIdx.x * kL1Ctx;
    for (int i = tid; i < kL1Ctx * NMAX; i += 256) {
        const int r = i / NMAX, k = i % NMAX;
        xs[r][k] = b0 + r < B && k < n_in ? ctx_input(ctx, wide, (size_t)(b0 + r) * n_in + k, err) : 0.0f;
    }
    __syncthreads();
    // every thread runs the loop (the sign ballots need whole warps); units
    // j >= h1 have zero weights and store nothing
    const int j = tid;
    const bool unit = j < h1;
    float w[NMAX];
#pragma unroll
    for (int k = 0; k < NMAX; k++) w[k] = unit && k < n_in ? W1[j * n_in + k] : 0.0f;
    const float bj = unit ? b1[j] : 0.0f;
    for (int r = 0; r < kL1Ctx; r += 2) {
        // two contexts at a time: two independent fma chains
        float acc0 = bj, acc1 = bj;
        // (the zero weights past n_in add exact zeros)
#pragma unroll
        for (int k = 0; k < NMAX; k++) {
            acc0 = fmaf(xs[r][k], w[k], acc0);
            acc1 = fmaf(xs[r + 1][k], w[k], acc1);
        }
        const float v0 = fmaxf(acc0, 0.0f), v1 = fmaxf(acc1, 0.0f);
        const uint16_t hi0 = f2bf(v0), hi1 = f2bf(v1);
        // the sign bits of the stored values, 32 units per ballot
        const uint32_t pos0 = __ballot_sync(0xffffffffu, unit && hi0 != 0 && (hi0 & 0x8000u) == 0);
        const uint32_t pos1 = __ballot_sync(0xffffffffu, unit && hi1 != 0 && (hi1 & 0x8000u) == 0);
        if (unit) {
            thi[r * h1 + j] = hi0;
            thi[(r + 1) * h1 + j] = hi1;
            if (p1) {
                tlo[r * h1 + j] = f2bf(v0 - bf2f(hi0));
                tlo[(r + 1) * h1 + j] = f2bf(v1 - bf2f(hi1));
            }
        }
        if (lane < 2 && 32 * warp + 16 * lane < h1) {
            smask[r][2 * warp + lane] = (uint16_t)(pos0 >> (16 * lane));
            smask[r + 1][2 * warp + lane] = (uint16_t)(pos1 >> (16 * lane));
        }
    }
    __syncthreads();
    // rows b0.. are contiguous in H1: one block of rows * h1 bf16
    const int rows = min(kL1Ctx, B - b0), n16 = rows * h1 / 8;
    uint4 *dst = reinterpret_cast<uint4 *>(H1 + (size_t)b0 * h1);
    for (int i = tid; i < n16; i += 256) dst[i] = reinterpret_cast<const uint4 *>(thi)[i];
    if (p1) {
        uint4 *dl = reinterpret_cast<uint4 *>(H1 + p1 + (size_t)b0 * h1);
        for (int i = tid; i < n16; i += 256) dl[i] = reinterpret_cast<const uint4 *>(tlo)[i];
    }
    // the sign bits: word (row, g) holds units 16 g .. 16 g + 15
    const int g16 = h1 / 16;
    for (int i = tid; i < rows * g16; i += 256) M1[(size_t)(b0 + i / g16) * g16 + i % g16] = smask[i / g16][i % g16];
}

// out[i] = scale * sum_z part[z * stride + i]: 32 columns per block, the
// partials split over blockDim.y row groups and combined in a fixed order
// (deterministic).  With `kpad` the columns are a [h][kpad] array whose first
// kin entries per row go to a compact [h][kin] output.
__global__ void k_reduce_parts(const float *part, int nparts, size_t stride, int n, float *out, float scale, int kpad,
                               int kin) {
    __shared__ float red[32][33];
    const int x = threadIdx.x, y = threadIdx.y, G = blockDim.y;
    const int i = blockIdx.x * 32 + x;
    float s = 0.0f;
    if (i < n) {
#pragma unroll 4
        for (int z = y; z < nparts; z += G) s += part[(size_t)z * stride + i];
    }
    red[y][x] = s;
    __syncthreads();
    if (y == 0 && i < n) {
        float t = 0.0f;
        for (int k = 0; k < G; k++) t += red[k][x];
        t *= scale;
        if (!kpad) out[i] = t;
        else if (i % kpad < kin) out[(i / kpad) * kin + i % kpad] = t;
    }
}

// The same for wide outputs (n and stride multiples of 4): 128 columns per
// block as float4 columns.
__global__ void k_reduce_parts4(const float *part, int nparts, size_t stride, int n, float *out, float scale) {
    __shared__ float4 red[8][32];
    const int x = threadIdx.x, y = threadIdx.y;
    const int i = (blockIdx.x * 32 + x) * 4;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < n) {
#pragma unroll 4
        for (int z = y; z < nparts; z += 8) {
            const float4 v = *reinterpret_cast<const float4 *>(part + (size_t)z * stride + i);
            s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
        }
    }
    red[y][x] = s;
    __syncthreads();
    if (y == 0 && i < n) {
        float4 t = red[0][x];
        for (int k = 1; k < 8; k++) {
            const float4 v = red[k][x];
            t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w;
        }
        *reinterpret_cast<float4 *>(out + i) = make_float4(t.x * scale, t.y * scale, t.z * scale, t.w * scale);
    }
}

// One shadow entry: bf16 high (and low) planes, or FP32.
__device__ __forceinline__ void shadow_put(void *Wd, size_t idx, size_t plane, float v, int bf16, int split) {
    if (bf16) {
        const uint16_t hi = f2bf(v);
        reinterpret_cast<uint16_t *>(Wd)[idx] = hi;
        if (split) reinterpret_cast<uint16_t *>(Wd)[idx + plane] = f2bf(v - bf2f(hi));
    } else {
        reinterpret_cast<float *>(Wd)[idx] = v;
    }
}

// Adam on the FP32 master weights (bias-corrected, Kingma & Ba) with the
// updated weights written straight into the GEMM operand copies (row-major
// and transposed).  The zero padding of the W1 copy is never touched.
struct ShadowArgs {
    int n_in, k1, h1, h2, n_out, bf16, split;
    void *w1, *w2, *w3, *w2t, *w3t;
};
__global__ void k_adam(float *p, const float *g, float *mo, float *ve, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2, ShadowArgs sa) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float m = b1 * mo[i] + (1.0f - b1) * gi;
    const float v = b2 * ve[i] + (1.0f - b2) * gi * gi;
    mo[i] = m;
    ve[i] = v;
    const float w = p[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    p[i] = w;
    const int h1 = sa.h1, h2 = sa.h2, n_in = sa.n_in;
    const int oW2 = h1 * n_in + h1, oW3 = oW2 + h2 * h1 + h2;
    if (i < h1 * n_in) {
        shadow_put(sa.w1, (size_t)(i / n_in) * sa.k1 + i % n_in, (size_t)h1 * sa.k1, w, sa.bf16, sa.split);
    } else if (i >= oW2 && i < oW2 + h2 * h1) {
        const int j = i - oW2, o = j / h1, k = j % h1;
        shadow_put(sa.w2, j, (size_t)h2 * h1, w, sa.bf16, sa.split);
        shadow_put(sa.w2t, (size_t)k * h2 + o, (size_t)h1 * h2, w, sa.bf16, sa.split);
    } else if (i >= oW3 && i < oW3 + sa.n_out * h2) {
        const int j = i - oW3, o = j / h2, k = j % h2;
        shadow_put(sa.w3, j, (size_t)sa.n_out * h2, w, sa.bf16, sa.split);
        shadow_put(sa.w3t, (size_t)k * sa.n_out + o, (size_t)h2 * sa.n_out, w, sa.bf16, sa.split);
    }
}
__global__ void k_shadow(const float *W, int out, int in, int in_pad, void *Wd, void *WTd, int bf16, int split) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= out * in_pad) return;
    const int o = i / in_pad, k = i % in_pad;
    const float v = k < in ? W[o * in + k] : 0.0f;
    if (bf16) {
        const uint16_t hi = f2bf(v), lo = f2bf(v - bf2f(hi));
        reinterpret_cast<uint16_t *>(Wd)[i] = hi;
        if (split) reinterpret_cast<uint16_t *>(Wd)[i + out * in_pad] = lo;
        if (WTd && k < in) {
            reinterpret_cast<uint16_t *>(WTd)[k * out + o] = hi;
            if (split) reinterpret_cast<uint16_t *>(WTd)[k * out + o + in * out] = lo;
        }
    } else {
        reinterpret_cast<float *>(Wd)[i] = v;
        if (WTd && k < in) reinterpret_cast<float *>(WTd)[k * out + o] = v;
    }
}

}  // namespace dlic

using namespace dlic;

// ===========================================================================
// Trainer object and C ABI
// ===========================================================================
struct dlic_trainer {
    int n_in, k1;                                // network inputs (the window's priors), padded to 16
    int h1, h2, mode, max_batch, num_sms;
    int n_out;                                   // 256 (8-bit samples, u8 batches) or 4096 (12-bit, u16)
    int wide;                                    // n_out = 4096
    int bf, split;                               // bf16 operands; hi + lo planes
    int recompute;                               // two activation buffers, h1 recomputed in the backward
    size_t nparams;
    int step;
    float lr, beta1, beta2, eps;
    float *params, *grads, *mom, *vel;           // FP32 master state
    void *w1, *w2, *w3, *w2t, *w3t;              // operand copies (bf16 or fp32)
    void *X, *H1, *H2, *DZ, *DA2, *DA1;          // row-major [batch][features]
    uint16_t *M1, *M2;                           // BF16 modes: sign bits of H1, H2 [batch][h / 16]
    void *XT, *H1T, *H2T, *DZT, *DA2T, *DA1T;    // FP32 path: transposed [features][batch]
    float *C, *part, *colsum, *losspart;
    float *Z;                     // 4096 outputs: the output layer's products [batch][n_out] (FP32)
    size_t part_floats;           // capacity of the split-K partials
    float *gacc, *closs, *lacc;   // batches above max_batch: gradient and loss sums over chunks
    int weighted;                 // the frequency-weighted loss is on
    float *vw, *wnorm;            // its weights per target value (n_out) and {1 / (W ln 2), 1 / W}
    int *err;
    std::vector<void *> allocs;
};

namespace {

size_t param_count(int n_in, int h1, int h2, int n_out) {
    return (size_t)h1 * n_in + h1 + (size_t)h2 * h1 + h2 + (size_t)n_out * h2 + n_out;
}

struct ParamView {
    float *W1, *b1, *W2, *b2, *W3, *b3;
};
ParamView view(float *p, int n_in, int h1, int h2, int n_out) {
    ParamView v;
    v.W1 = p;
    v.b1 = v.W1 + (size_t)h1 * n_in;
    v.W2 = v.b1 + h1;
    v.b2 = v.W2 + (size_t)h2 * h1;
    v.W3 = v.b2 + h2;
    v.b3 = v.W3 + (size_t)n_out * h2;
    return v;
}

// The driver's tensor-map encoder, looked up through the runtime so that the
// library loads on machines without a CUDA driver (it is only called on a
// GPU).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

CUresult encode_map(CUtensorMap *map, const void *g, int rows, int cols, int pitch, int box_rows) {
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return CUDA_ERROR_NOT_FOUND;
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(g), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

// A GEMM operand in global memory.  K-major: `rows` M (or N) entries of
// `cols` = K values; MN-major: `rows` = K entries of `cols` M (or N) values.
// `pitch` is the row stride and `plane` the element offset of the low plane
// (split mode).
struct Operand {
    const void *p;
    int rows, cols, pitch;
    size_t plane;
    int mn;
};

// C = A[M x K] B[N x K]^T with the given epilogue.  nblk > 1 (EPI_F32, K-major
// B of nblk * N rows, tensor-core path): nblk column blocks of N, one per
// gridDim.y, C's columns offset by the block.
dlic_status gemm(dlic_trainer *t, const Operand &a, const Operand &b, int M, int N, int K, int epi, EpiArgs e,
                 int splits, cudaStream_t st, int nblk = 1) {
    e.M = M;
    e.N = N;
    e.ldT = t->max_batch;
    e.bf16 = t->bf;
    e.split = t->split;
    const int mt = (M + 127) / 128;
    if (t->bf) {
        GemmCfg g;
        g.a_mn = a.mn;
        g.b_mn = b.mn;
        g.n_mma = b.mn ? (N + 63) / 64 * 64 : (N + 15) / 16 * 16;
        g.b_boxes = (N + 63) / 64;
        // Split mode: the activation GEMMs (M = batch) run persistent, one
        // CTA per SM over the m-tiles with two accumulators, so that a tile's
        // epilogue overlaps the next tile's loads and MMAs (its stages are
        // twice as large, so only one CTA fits an SM anyway).  Plain BF16:
        // one tile per CTA and two CTAs per SM (two stages each), whose
        // epilogues run side by side; measured faster than one persistent
        // CTA.  The weight gradients (M = 256 or h, K = batch) take one tile
        // per CTA with split-K over gridDim.z and a deeper pipeline.
        if (nblk > 1 && (epi != EPI_F32 || b.mn)) return fail(DLIC_ERR_INVALID, "column blocks need EPI_F32, K-major B");
        const bool persist = t->split && epi != EPI_F32;
        g.stages = epi == EPI_F32 && !t->split ? 4 : 2;
        CUtensorMap ma, mb, mal, mbl;
        const uint16_t *A16 = static_cast<const uint16_t *>(a.p), *B16 = static_cast<const uint16_t *>(b.p);
        const int abox = a.mn ? 64 : 128, bbox = b.mn ? 64 : N;
        if (encode_map(&ma, A16, a.rows, a.cols, a.pitch, abox) != CUDA_SUCCESS ||
            encode_map(&mb, B16, b.rows, b.cols, b.pitch, bbox) != CUDA_SUCCESS)
            return fail(DLIC_ERR_CUDA, "cuTensorMapEncodeTiled failed (M %d N %d K %d)", M, N, K);
        mal = ma;
        mbl = mb;
        if (t->split && (encode_map(&mal, A16 + a.plane, a.rows, a.cols, a.pitch, abox) != CUDA_SUCCESS ||
                         encode_map(&mbl, B16 + b.plane, b.rows, b.cols, b.pitch, bbox) != CUDA_SUCCESS))
            return fail(DLIC_ERR_CUDA, "cuTensorMapEncodeTiled failed (low planes)");
        const int nkb = (K + 63) / 64;
        const int per = (nkb + splits - 1) / splits;
        const uint32_t stage = 128 * 128 + ((uint32_t)g.n_mma * 128 + 1023) / 1024 * 1024;
        const size_t smem = (size_t)g.stages * (t->split ? 2 : 1) * stage + 1024;
        const int gx = persist ? min(mt, t->num_sms) : mt;
        auto launch = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kern<<<dim3(gx, nblk, splits), kGemmThreads, smem, st>>>(ma, mb, mal, mbl, K, per, epi, g, e, t->err);
        };
        if (persist)
            launch(k_gemm_tc<true, true>);
        else if (t->split)
            launch(k_gemm_tc<true, false>);
        else
            launch(k_gemm_tc<false, false>);
        cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) return cuda_fail(ce, "k_gemm_tc launch");
        return DLIC_OK;
    }
    // FP32 path: raw GEMM into C (or the split-K partials), then the row
    // epilogue; operands K-major (the transposed activations)
    const int per = ((K + splits - 1) / splits + 7) / 8 * 8;
    float *dst = epi == EPI_F32 ? e.c : t->C;
    const int ldc = epi == EPI_F32 ? e.ldc : N;
    k_gemm_f32<<<dim3(mt, (N + 127) / 128, splits), 256, 0, st>>>(static_cast<const float *>(a.p), a.pitch,
                                                                   static_cast<const float *>(b.p), b.pitch, dst, M, N, K,
                                                                   per, ldc);
    if (epi != EPI_F32) k_row_epilogue<<<mt, 128, 4 * N * sizeof(float), st>>>(t->C, epi, e);
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? DLIC_OK : cuda_fail(ce, "fp32 gemm launch");
}

void reduce_parts(const float *part, int nparts, size_t stride, int n, float *out, float scale, int kpad, int kin,
                  cudaStream_t st) {
    if (!kpad && n >= 4096 && n % 4 == 0 && stride % 4 == 0 && nparts < 256) {
        k_reduce_parts4<<<(n + 127) / 128, dim3(32, 8), 0, st>>>(part, nparts, stride, n, out, scale);
        return;
    }
    const int G = nparts >= 256 ? 32 : 8;
    k_reduce_parts<<<(n + 31) / 32, dim3(32, G), 0, st>>>(part, nparts, stride, n, out, scale, kpad, kin);
}

dlic_status refresh_shadows(dlic_trainer *t, cudaStream_t st) {
    ParamView p = view(t->params, t->n_in, t->h1, t->h2, t->n_out);
    const int bf = t->bf, sp = t->split;
    k_shadow<<<(t->h1 * t->k1 + 255) / 256, 256, 0, st>>>(p.W1, t->h1, t->n_in, t->k1, t->w1, nullptr, bf, sp);
    k_shadow<<<(t->h2 * t->h1 + 255) / 256, 256, 0, st>>>(p.W2, t->h2, t->h1, t->h1, t->w2, t->w2t, bf, sp);
    k_shadow<<<(t->n_out * t->h2 + 255) / 256, 256, 0, st>>>(p.W3, t->n_out, t->h2, t->h2, t->w3, t->w3t, bf, sp);
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? DLIC_OK : cuda_fail(ce, "shadow launch");
}

// Forward (and, if `backward`, backward) over one batch.  BF16 modes keep
// every activation row-major [batch][features] and read the weight-gradient
// factors MN-major; the FP32 path also keeps transposed copies [features]
// [batch] for its K-major CUDA-core GEMM.
// Target value b of a batch: u8, or u16 for 12-bit samples; a value past
// the n_out outputs sets DLIC_ERR_INVALID and reads as 0.
__device__ __forceinline__ int batch_target(const void *tgt, int wide, int b, int n_out, int *err) {
    const int y = wide ? (int)static_cast<const uint16_t *>(tgt)[b] : (int)static_cast<const uint8_t *>(tgt)[b];
    if (y < n_out) return y;
    atomicExch(err, (int)DLIC_ERR_INVALID);
    return 0;
}

// W = sum_b vw[tgt[b]] in a fixed order (one CTA), and {1 / (W ln 2), 1 / W}.
__global__ void __launch_bounds__(1024) k_wsum(const void *tgt, int wide, int B, int n_out, const float *vw,
                                               float *wnorm, int *err) {
    __shared__ float red[1024];
    const int tid = threadIdx.x;
    float s = 0.0f;
    for (int b = tid; b < B; b += 1024) s += vw[batch_target(tgt, wide, b, n_out, err)];
    red[tid] = s;
    __syncthreads();
    for (int off = 512; off > 0; off >>= 1) {
        if (tid < off) red[tid] += red[tid + off];
        __syncthreads();
    }
    if (tid == 0) {
        wnorm[0] = 1.0f / (red[0] * kLn2);
        wnorm[1] = 1.0f / red[0];
    }
}

// Softmax cross-entropy over the 4096 outputs of a 12-bit network (Sec. IV
// "Higher Bit Depth"), a row too long for one tensor-memory tile: the output
// layer's GEMM first writes z - b3 to Z [B][4096] (FP32), then this kernel
// does what the fused epilogue of the 256-output layer does (maximum, sum
// of expf, lse = m + logf(sum), loss (lse - z_y) / ln 2 weighted as there,
// dz = (softmax - onehot) * scale) with every logit read from HBM once.
// One CTA of 512 threads per 32-row tile (two CTAs per SM); thread t owns
// the columns 4t .. 4t + 3 and 2048 + 4t .. 2048 + 4t + 3 of every row, so
// that a row's loads are two fully coalesced 8 KB sweeps; rows go four at a
// time through two block reductions (warp trees, then the 16 warp values in
// a fixed order), so every sum has the same order on every run.  The thread
// keeps its columns' dz sums over the tile (the db3 partials) in registers;
// the tiles' loss and column partials are added in a fixed order afterwards.
constexpr int kWideOut = 4096, kWideRows = 32, kWideThreads = 512, kWideGroup = 2;
__global__ void __launch_bounds__(kWideThreads, 2) k_softmax_wide(const float *Z, const float *b3, const uint16_t *tgt,
                                                                  int B, float inv_batch_ln2, const float *vw,
                                                                  const float *wnorm, void *DZ, size_t dz_plane,
                                                                  int bf16, int split, float *colsum, float *losspart,
                                                                  int *err) {
    __shared__ float s_max[kWideGroup][kWideThreads / 32], s_sum[kWideGroup][kWideThreads / 32];
    __shared__ float s_loss[kWideThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = blockIdx.x * kWideRows;
    const int cA = 4 * tid, cB = kWideOut / 2 + 4 * tid;
    float cs[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float loss_acc = 0.0f;
    for (int g0 = 0; g0 < kWideRows; g0 += kWideGroup) {
        // v: the row's logits, then exp(z - m), then dz, in place
        float v[kWideGroup][8], mx[kWideGroup], zy[kWideGroup];
        int ys[kWideGroup];
#pragma unroll
        for (int i = 0; i < kWideGroup; i++) {
            const int row = r0 + g0 + i;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), c = a;
            int y = 0;
            if (row < B) {
                const float *z = Z + (size_t)row * kWideOut;
                a = *reinterpret_cast<const float4 *>(z + cA);
                c = *reinterpret_cast<const float4 *>(z + cB);
                y = tgt[row];
                if (y >= kWideOut) {
                    atomicExch(err, (int)DLIC_ERR_INVALID);
                    y = 0;
                }
            }
            const float4 bA = *reinterpret_cast<const float4 *>(b3 + cA), bB = *reinterpret_cast<const float4 *>(b3 + cB);
            v[i][0] = a.x + bA.x; v[i][1] = a.y + bA.y; v[i][2] = a.z + bA.z; v[i][3] = a.w + bA.w;
            v[i][4] = c.x + bB.x; v[i][5] = c.y + bB.y; v[i][6] = c.z + bB.z; v[i][7] = c.w + bB.w;
            ys[i] = y;
            mx[i] = -INFINITY;
            zy[i] = 0.0f;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                mx[i] = fmaxf(mx[i], v[i][q]);
                if ((q < 4 ? cA : cB - 4) + q == y) zy[i] = v[i][q];
            }
#pragma unroll
            for (int off = 16; off; off >>= 1) mx[i] = fmaxf(mx[i], __shfl_xor_sync(0xffffffffu, mx[i], off));
            if (lane == 0) s_max[i][warp] = mx[i];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kWideGroup; i++) {
            float m = s_max[i][0];
#pragma unroll
            for (int w = 1; w < kWideThreads / 32; w++) m = fmaxf(m, s_max[i][w]);
            mx[i] = m;
            float l = 0.0f;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                v[i][q] = expf(v[i][q] - m);
                l += v[i][q];
            }
#pragma unroll
            for (int off = 16; off; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
            if (lane == 0) s_sum[i][warp] = l;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kWideGroup; i++) {
            const int row = r0 + g0 + i;
            float se = s_sum[i][0];
#pragma unroll
            for (int w = 1; w < kWideThreads / 32; w++) se += s_sum[i][w];
            if (row >= B) continue;
            const int y = ys[i];
            const float lse = mx[i] + logf(se), inv = 1.0f / se;
            const float rw = vw ? vw[y] : 1.0f;
            const float gscale = vw ? rw * wnorm[0] : inv_batch_ln2, lw = vw ? rw * wnorm[1] : 1.0f;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                float g = v[i][q] * inv;
                if ((q < 4 ? cA : cB - 4) + q == y) {
                    g -= 1.0f;
                    loss_acc += lw * ((lse - zy[i]) / kLn2);
                }
                g *= gscale;
                v[i][q] = g;
                cs[q] += g;
            }
            const size_t o = (size_t)row * kWideOut;
            if (bf16) {
                uint16_t *d = static_cast<uint16_t *>(DZ);
                const uint2 hA = make_uint2(pack_bf16x2(v[i][0], v[i][1]), pack_bf16x2(v[i][2], v[i][3]));
                const uint2 hB = make_uint2(pack_bf16x2(v[i][4], v[i][5]), pack_bf16x2(v[i][6], v[i][7]));
                *reinterpret_cast<uint2 *>(d + o + cA) = hA;
                *reinterpret_cast<uint2 *>(d + o + cB) = hB;
                if (split) {
                    const uint32_t h[4] = {hA.x, hA.y, hB.x, hB.y};
                    uint32_t lo[4];
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        lo[k] = pack_bf16x2(v[i][2 * k] - __uint_as_float(h[k] << 16),
                                            v[i][2 * k + 1] - __uint_as_float(h[k] & 0xFFFF0000u));
                    *reinterpret_cast<uint2 *>(d + dz_plane + o + cA) = make_uint2(lo[0], lo[1]);
                    *reinterpret_cast<uint2 *>(d + dz_plane + o + cB) = make_uint2(lo[2], lo[3]);
                }
            } else {
                float *d = static_cast<float *>(DZ);
                *reinterpret_cast<float4 *>(d + o + cA) = make_float4(v[i][0], v[i][1], v[i][2], v[i][3]);
                *reinterpret_cast<float4 *>(d + o + cB) = make_float4(v[i][4], v[i][5], v[i][6], v[i][7]);
            }
        }
    }
    float *cp = colsum + (size_t)blockIdx.x * kWideOut;
    *reinterpret_cast<float4 *>(cp + cA) = make_float4(cs[0], cs[1], cs[2], cs[3]);
    *reinterpret_cast<float4 *>(cp + cB) = make_float4(cs[4], cs[5], cs[6], cs[7]);
#pragma unroll
    for (int off = 16; off; off >>= 1) loss_acc += __shfl_down_sync(0xffffffffu, loss_acc, off);
    if (lane == 0) s_loss[warp] = loss_acc;
    __syncthreads();
    if (tid == 0) {
        float l = 0.0f;
        for (int w = 0; w < kWideThreads / 32; w++) l += s_loss[w];
        losspart[blockIdx.x] = l;
    }
}

// out[c][r] = in[r][c] for an R x Cn FP32 array (row pitch Cn; out pitch
// ldo): 32 x 32 tiles through shared memory, both sides coalesced.
__global__ void k_transpose_f32(const float *in, int R, int Cn, float *out, int ldo) {
    __shared__ float tile[32][33];
    const int x = threadIdx.x, y = threadIdx.y;   // 32 x 8
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = y; k < 32; k += 8)
        if (r0 + k < R && c0 + x < Cn) tile[k][x] = in[(size_t)(r0 + k) * Cn + c0 + x];
    __syncthreads();
    for (int k = y; k < 32; k += 8)
        if (c0 + k < Cn && r0 + x < R) out[(size_t)(c0 + k) * ldo + r0 + x] = tile[x][k];
}

dlic_status run(dlic_trainer *t, const void *ctx, const void *tgt, int B, float *d_loss, bool backward,
                cudaStream_t st, bool wnorm_ready = false) {
    const int h1 = t->h1, h2 = t->h2, mt = (B + 127) / 128, n_in = t->n_in, k1 = t->k1, n_out = t->n_out;
    const int bf = t->bf;
    ParamView p = view(t->params, n_in, h1, h2, n_out);
    ParamView g = view(t->grads, n_in, h1, h2, n_out);
    const int P = t->max_batch;   // capacity: pitch of the transposed arrays, offset of the low planes
    const size_t Bm = (size_t)P;
    const size_t sp = t->split ? 1 : 0;
    // row-major [B][n] activation (K-major as the A factor of the next layer)
    auto rowmaj = [&](const void *q, int n) { return Operand{q, B, n, n, Bm * n, 0}; };
    // weights [out][in] (K-major B factor of a forward or backward GEMM)
    auto wmat = [&](const void *q, int out, int in) { return Operand{q, out, in, in, (size_t)out * in, 0}; };
    // weight-gradient factors: MN-major row-major activations (BF16) or
    // K-major transposed copies (FP32)
    auto wgrad = [&](const void *rm, const void *tr, int n) {
        return bf ? Operand{rm, B, n, n, Bm * n, 1} : Operand{tr, n, B, P, (size_t)n * Bm, 0};
    };
    k_features<<<(B + 255) / 256, 256, 0, st>>>(ctx, t->wide, B, n_in, k1, P, t->X, bf ? nullptr : t->XT, bf,
                                                sp * Bm * k1, t->err);
    EpiArgs e{};
    // layer 1, 2: bias + ReLU
    e.bias = p.b1; e.out = t->H1; e.outT = t->H1T; e.out_plane = Bm * h1; e.outT_plane = (size_t)h1 * Bm;
    dlic_status s = DLIC_OK;
    // the first layer on the CUDA cores (BF16 modes): h1 rows and their sign bits
    auto layer1 = [&]() {
        const int nb = (B + kL1Ctx - 1) / kL1Ctx;
        uint16_t *H1 = static_cast<uint16_t *>(t->H1);
        if (n_in <= 12)
            k_layer1<12><<<nb, 256, 0, st>>>(ctx, t->wide, B, n_in, p.W1, p.b1, h1, H1, sp * Bm * h1, t->M1, t->err);
        else if (n_in <= 16)
            k_layer1<16><<<nb, 256, 0, st>>>(ctx, t->wide, B, n_in, p.W1, p.b1, h1, H1, sp * Bm * h1, t->M1, t->err);
        else if (n_in <= 32)
            k_layer1<32><<<nb, 256, 0, st>>>(ctx, t->wide, B, n_in, p.W1, p.b1, h1, H1, sp * Bm * h1, t->M1, t->err);
        else if (n_in <= 64)
            k_layer1<64><<<nb, 256, 0, st>>>(ctx, t->wide, B, n_in, p.W1, p.b1, h1, H1, sp * Bm * h1, t->M1, t->err);
        else
            k_layer1<96><<<nb, 256, 0, st>>>(ctx, t->wide, B, n_in, p.W1, p.b1, h1, H1, sp * Bm * h1, t->M1, t->err);
    };
    if (bf) {
        layer1();
    } else if ((s = gemm(t, rowmaj(t->X, k1), wmat(t->w1, h1, k1), B, h1, k1, EPI_BIAS_RELU, e, 1, st))) {
        return s;
    }
    e = EpiArgs{}; e.bias = p.b2; e.out = t->H2; e.outT = t->H2T; e.out_plane = Bm * h2; e.outT_plane = (size_t)h2 * Bm;
    e.mask_out = bf ? t->M2 : nullptr;
    if ((s = gemm(t, rowmaj(t->H1, h1), wmat(t->w2, h2, h1), B, h2, h1, EPI_BIAS_RELU, e, 1, st))) return s;
    // layer 3 + softmax cross-entropy: loss partials, dz, db3 partials
    // the frequency-weighted loss: the batch's weight total first
    if (t->weighted && !wnorm_ready) k_wsum<<<1, 1024, 0, st>>>(tgt, t->wide, B, n_out, t->vw, t->wnorm, t->err);
    if (!t->wide) {
        // 256 outputs: one tensor-memory tile per row, softmax fused into the
        // GEMM's epilogue
        e = EpiArgs{}; e.bias = p.b3; e.out = t->DZ; e.outT = t->DZT; e.tgt = static_cast<const uint8_t *>(tgt);
        e.out_plane = Bm * n_out; e.outT_plane = (size_t)n_out * Bm;
        e.inv_batch_ln2 = 1.0f / ((float)B * kLn2);
        if (t->weighted) {
            e.vw = t->vw;
            e.wnorm = t->wnorm;
        }
        e.colsum = t->colsum; e.loss = t->losspart;
        if ((s = gemm(t, rowmaj(t->H2, h2), wmat(t->w3, n_out, h2), B, n_out, h2, EPI_SOFTMAX, e, 1, st)))
            return s;
    } else {
        // 4096 outputs: the products z - b3 to Z (the tensor-core GEMM takes
        // 256 columns, one accumulator tile, per launch), then the row-wise
        // softmax kernel
        e = EpiArgs{}; e.c = t->Z; e.ldc = n_out;
        if (bf) {
            if ((s = gemm(t, rowmaj(t->H2, h2), wmat(t->w3, n_out, h2), B, 256, h2, EPI_F32, e, 1, st, n_out / 256)))
                return s;
        } else if ((s = gemm(t, rowmaj(t->H2, h2), wmat(t->w3, n_out, h2), B, n_out, h2, EPI_F32, e, 1, st))) {
            return s;
        }
        k_softmax_wide<<<(B + kWideRows - 1) / kWideRows, kWideThreads, 0, st>>>(
            t->Z, p.b3, static_cast<const uint16_t *>(tgt), B, 1.0f / ((float)B * kLn2),
            t->weighted ? t->vw : nullptr, t->wnorm, t->DZ, Bm * n_out, bf, t->split, t->colsum, t->losspart, t->err);
        if (!bf && backward)
            k_transpose_f32<<<dim3(n_out / 32, (B + 31) / 32), dim3(32, 8), 0, st>>>(
                static_cast<const float *>(t->DZ), B, n_out, static_cast<float *>(t->DZT), P);
    }
    const int lt = t->wide ? (B + kWideRows - 1) / kWideRows : mt;   // tiles of the loss and db3 partials
    reduce_parts(t->losspart, lt, 1, 1, d_loss, t->weighted ? 1.0f : 1.0f / (float)B, 0, 0, st);
    if (!backward) {
        cudaError_t ce = cudaGetLastError();
        return ce == cudaSuccess ? DLIC_OK : cuda_fail(ce, "forward launch");
    }
    reduce_parts(t->colsum, lt, n_out, n_out, g.b3, 1.0f, 0, 0, st);
    // weight gradients dW = dY^T X: K = batch, split-K partials summed in a
    // fixed order; enough splits to cover every SM, as many as the partial
    // buffer holds
    auto splits_for = [&](int M, int N) {
        const int nkb = (B + 63) / 64;
        int want = bf ? max(1, t->num_sms / ((M + 127) / 128)) : max(1, min(64, (B + 1023) / 1024));
        want = max(1, min(want, (int)(t->part_floats / ((size_t)M * N))));
        const int per = (nkb + min(want, nkb) - 1) / min(want, nkb);
        return (nkb + per - 1) / per;
    };
    int sk = 0;
    if (t->recompute) {
        // Two activation buffers: A held h1, then dz (the layer-3 GEMM
        // overwrote h1, which it no longer needs); B holds h2.  Each buffer
        // is reused once its contents are dead: dW3 = dz^T h2 first, da2
        // into B (over h2), then h1 recomputed from the batch into A (over
        // dz), dW2 = da2^T h1, da1 into A (over h1), dW1 = da1^T x.  The
        // same kernels in the same arithmetic: the gradient equals the
        // stored-activation one bit for bit.
        sk = splits_for(n_out, h2);
        e = EpiArgs{}; e.c = t->part; e.ldc = h2;
        if ((s = gemm(t, wgrad(t->DZ, t->DZT, n_out), wgrad(t->H2, t->H2T, h2), n_out, h2, B, EPI_F32, e, sk, st)))
            return s;
        reduce_parts(t->part, sk, (size_t)n_out * h2, n_out * h2, g.W3, 1.0f, 0, 0, st);
        e = EpiArgs{}; e.mask = t->M2; e.out = t->DA2; e.colsum = t->colsum; e.out_plane = Bm * h2;
        if ((s = gemm(t, rowmaj(t->DZ, n_out), wmat(t->w3t, h2, n_out), B, h2, n_out, EPI_RELU_GRAD, e, 1, st)))
            return s;
        reduce_parts(t->colsum, mt, h2, h2, g.b2, 1.0f, 0, 0, st);
        layer1();
        sk = splits_for(h2, h1);
        e = EpiArgs{}; e.c = t->part; e.ldc = h1;
        if ((s = gemm(t, wgrad(t->DA2, t->DA2T, h2), wgrad(t->H1, t->H1T, h1), h2, h1, B, EPI_F32, e, sk, st)))
            return s;
        reduce_parts(t->part, sk, (size_t)h2 * h1, h2 * h1, g.W2, 1.0f, 0, 0, st);
        e = EpiArgs{}; e.mask = t->M1; e.out = t->DA1; e.colsum = t->colsum; e.out_plane = Bm * h1;
        if ((s = gemm(t, rowmaj(t->DA2, h2), wmat(t->w2t, h1, h2), B, h1, h2, EPI_RELU_GRAD, e, 1, st))) return s;
        reduce_parts(t->colsum, mt, h1, h1, g.b1, 1.0f, 0, 0, st);
        sk = splits_for(h1, k1);
        e = EpiArgs{}; e.c = t->part; e.ldc = k1;
        if ((s = gemm(t, wgrad(t->DA1, t->DA1T, h1), wgrad(t->X, t->XT, k1), h1, k1, B, EPI_F32, e, sk, st))) return s;
        reduce_parts(t->part, sk, (size_t)h1 * k1, h1 * k1, g.W1, 1.0f, k1, n_in, st);
        cudaError_t ce = cudaGetLastError();
        return ce == cudaSuccess ? DLIC_OK : cuda_fail(ce, "backward launch");
    }
    // dh2 = dz W3 (B operand W3^T), da2 = dh2 * [h2 > 0]; db2
    e = EpiArgs{}; e.act = t->H2; e.mask = t->M2; e.out = t->DA2; e.outT = t->DA2T; e.colsum = t->colsum;
    e.out_plane = Bm * h2; e.outT_plane = (size_t)h2 * Bm;
    if ((s = gemm(t, rowmaj(t->DZ, n_out), wmat(t->w3t, h2, n_out), B, h2, n_out, EPI_RELU_GRAD, e, 1, st)))
        return s;
    reduce_parts(t->colsum, mt, h2, h2, g.b2, 1.0f, 0, 0, st);
    // dh1 = da2 W2, da1 = dh1 * [h1 > 0]; db1
    e = EpiArgs{}; e.act = t->H1; e.mask = t->M1; e.out = bf ? t->DA1 : nullptr; e.outT = t->DA1T; e.colsum = t->colsum;
    e.out_plane = Bm * h1; e.outT_plane = (size_t)h1 * Bm;
    if ((s = gemm(t, rowmaj(t->DA2, h2), wmat(t->w2t, h1, h2), B, h1, h2, EPI_RELU_GRAD, e, 1, st))) return s;
    reduce_parts(t->colsum, mt, h1, h1, g.b1, 1.0f, 0, 0, st);
    sk = splits_for(n_out, h2);
    e = EpiArgs{}; e.c = t->part; e.ldc = h2;
    if ((s = gemm(t, wgrad(t->DZ, t->DZT, n_out), wgrad(t->H2, t->H2T, h2), n_out, h2, B, EPI_F32, e, sk, st)))
        return s;
    reduce_parts(t->part, sk, (size_t)n_out * h2, n_out * h2, g.W3, 1.0f, 0, 0, st);
    sk = splits_for(h2, h1);
    e = EpiArgs{}; e.c = t->part; e.ldc = h1;
    if ((s = gemm(t, wgrad(t->DA2, t->DA2T, h2), wgrad(t->H1, t->H1T, h1), h2, h1, B, EPI_F32, e, sk, st))) return s;
    reduce_parts(t->part, sk, (size_t)h2 * h1, h2 * h1, g.W2, 1.0f, 0, 0, st);
    sk = splits_for(h1, k1);
    e = EpiArgs{}; e.c = t->part; e.ldc = k1;
    if ((s = gemm(t, wgrad(t->DA1, t->DA1T, h1), wgrad(t->X, t->XT, k1), h1, k1, B, EPI_F32, e, sk, st))) return s;
    reduce_parts(t->part, sk, (size_t)h1 * k1, h1 * k1, g.W1, 1.0f, k1, n_in, st);
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? DLIC_OK : cuda_fail(ce, "backward launch");
}

}  // namespace

extern "C" size_t dlic_train_param_count(int n_in, int h1, int h2) { return param_count(n_in, h1, h2, kSymbols); }

extern "C" size_t dlic_train_param_count_k(int n_in, int h1, int h2, int n_out) {
    return param_count(n_in, h1, h2, n_out);
}

extern "C" dlic_status dlic_trainer_create(int n_in, int h1, int h2, int mode, int max_batch, const float *h_params,
                                           dlic_trainer **out) {
    return dlic_trainer_create_k(n_in, h1, h2, kSymbols, mode, max_batch, h_params, out);
}

extern "C" dlic_status dlic_trainer_create_k(int n_in, int h1, int h2, int n_out, int mode, int max_batch,
                                             const float *h_params, dlic_trainer **out) {
    if (!out) return fail(DLIC_ERR_INVALID, "null output");
    *out = nullptr;
    if (n_out != kSymbols && n_out != kWideOut)
        return fail(DLIC_ERR_INVALID, "n_out must be 256 (8-bit samples) or 4096 (12-bit samples)");
    if (n_in < 1 || n_in > kMaxPriors) return fail(DLIC_ERR_INVALID, "network inputs must be in [1, %d]", kMaxPriors);
    if (h1 < 16 || h1 > 256 || h1 % 16 || h2 < 16 || h2 > 256 || h2 % 16)
        return fail(DLIC_ERR_UNSUPPORTED, "hidden widths must be multiples of 16 in [16, 256]");
    const int recompute = (mode & DLIC_TRAIN_RECOMPUTE) != 0;
    mode &= ~DLIC_TRAIN_RECOMPUTE;
    if (mode != DLIC_TRAIN_BF16 && mode != DLIC_TRAIN_FP32 && mode != DLIC_TRAIN_BF16X3)
        return fail(DLIC_ERR_INVALID, "unknown training mode %d", mode);
    if (recompute && mode == DLIC_TRAIN_FP32)
        return fail(DLIC_ERR_INVALID, "DLIC_TRAIN_RECOMPUTE takes a BF16 mode");
    if (max_batch < 1 || max_batch > (1 << 22)) return fail(DLIC_ERR_INVALID, "max_batch must be in [1, 2^22]");
    if (!h_params) return fail(DLIC_ERR_INVALID, "null initial parameters");
    dlic_trainer *t = new dlic_trainer();
    t->n_in = n_in;
    t->k1 = (n_in + 15) / 16 * 16;
    t->h1 = h1; t->h2 = h2; t->mode = mode;
    t->n_out = n_out;
    t->wide = n_out == kWideOut;
    t->bf = mode != DLIC_TRAIN_FP32;
    t->split = mode == DLIC_TRAIN_BF16X3;
    t->recompute = recompute;
    t->max_batch = (max_batch + 127) / 128 * 128;
    t->nparams = param_count(n_in, h1, h2, n_out);
    t->step = 0;
    t->lr = 1e-3f; t->beta1 = 0.9f; t->beta2 = 0.999f; t->eps = 1e-8f;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t es = t->bf ? (t->split ? 4 : 2) : 4;   // bytes per element, both planes
    const size_t Bm = (size_t)t->max_batch;
    const int hmax = h1 > h2 ? h1 : h2;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes < 256 ? 256 : bytes) != cudaSuccess) return nullptr;
        t->allocs.push_back(p);
        return p;
    };
    bool ok = true;
    auto A = [&](size_t bytes) { void *p = alloc(bytes); ok = ok && p; return p; };
    t->params = (float *)A(4 * t->nparams);
    t->grads = (float *)A(4 * t->nparams);
    t->mom = (float *)A(4 * t->nparams);
    t->vel = (float *)A(4 * t->nparams);
    t->w1 = A(es * h1 * t->k1);
    t->w2 = A(es * h2 * h1);
    t->w3 = A(es * n_out * h2);
    t->w2t = A(es * h1 * h2);
    t->w3t = A(es * h2 * n_out);
    t->X = A(es * Bm * t->k1);
    if (recompute) {
        // two activation buffers (h1, dz, h1 again, da1 in turn; h2, da2)
        t->H1 = t->DZ = t->DA1 = A(es * Bm * (n_out > h1 ? n_out : h1));
        t->H2 = t->DA2 = A(es * Bm * h2);
    } else {
        t->H1 = A(es * Bm * h1);
        t->H2 = A(es * Bm * h2);
        t->DZ = A(es * Bm * n_out);
        t->DA2 = A(es * Bm * h2);
    }
    if (t->wide) t->Z = (float *)A(4 * Bm * n_out);
    if (t->bf) {
        if (!recompute) t->DA1 = A(es * Bm * h1);
        t->M1 = (uint16_t *)A(2 * Bm * (h1 / 16) + 16);   // (+16: the L2 prefetch rounds up)
        t->M2 = (uint16_t *)A(2 * Bm * (h2 / 16) + 16);
    } else {
        t->XT = A(es * t->k1 * Bm);
        t->H1T = A(es * h1 * Bm);
        t->H2T = A(es * h2 * Bm);
        t->DZT = A(es * n_out * Bm);
        t->DA2T = A(es * h2 * Bm);
        t->DA1T = A(es * h1 * Bm);
        t->C = (float *)A(4 * Bm * kSymbols);
    }
    // split-K partials: up to one split per SM (BF16) or 64 (FP32)
    t->part_floats = (size_t)(t->num_sms > 64 ? t->num_sms : 64) * kSymbols * hmax;
    t->part = (float *)A(4 * t->part_floats);
    // one row per m-tile (or per 32-row tile of the 4096-way softmax), the last one ragged
    const size_t ntile = t->wide ? (Bm + kWideRows - 1) / kWideRows : (Bm + 127) / 128;
    t->colsum = (float *)A(4 * ntile * n_out);
    t->losspart = (float *)A(4 * ntile);
    t->gacc = (float *)A(4 * t->nparams);
    t->vw = (float *)A(4 * (size_t)n_out);
    t->wnorm = (float *)A(8);
    t->closs = (float *)A(8);
    t->lacc = (float *)A(8);
    t->err = (int *)A(4);
    if (!ok) {
        dlic_trainer_destroy(t);
        return fail(DLIC_ERR_CUDA, "cudaMalloc failed while creating the trainer");
    }
    cudaMemcpy(t->params, h_params, 4 * t->nparams, cudaMemcpyHostToDevice);
    cudaMemset(t->mom, 0, 4 * t->nparams);
    cudaMemset(t->vel, 0, 4 * t->nparams);
    cudaMemset(t->err, 0, 4);
    dlic_status s = refresh_shadows(t, nullptr);
    cudaError_t ce = cudaDeviceSynchronize();
    if (s != DLIC_OK || ce != cudaSuccess) {
        dlic_trainer_destroy(t);
        return s != DLIC_OK ? s : cuda_fail(ce, "trainer set-up");
    }
    *out = t;
    return DLIC_OK;
}

extern "C" dlic_status dlic_trainer_destroy(dlic_trainer *t) {
    if (!t) return DLIC_OK;
    for (void *p : t->allocs) cudaFree(p);
    delete t;
    return DLIC_OK;
}

static dlic_status check_batch(dlic_trainer *t, const void *ctx, const void *tgt, int B) {
    if (!t) return fail(DLIC_ERR_INVALID, "null trainer");
    if (!ctx || !tgt) return fail(DLIC_ERR_INVALID, "null batch");
    if (B < 1) return fail(DLIC_ERR_CAPACITY, "batch %d < 1", B);
    return DLIC_OK;
}

// acc = w g (first) or acc + w g, element by element.
__global__ void k_accum(float *acc, const float *g, int n, float w, int first) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) acc[i] = first ? w * g[i] : fmaf(w, g[i], acc[i]);
}

// A batch larger than the trainer's capacity, in chunks of max_batch
// contexts: each chunk's forward (and backward) runs on its own, and its
// mean loss (and gradient) is added with weight B_c / B, so that the
// activations held at any time are one chunk's, whatever the batch.  The
// result lands where the one-pass run puts it (d_loss, t->grads).
static dlic_status run_chunked(dlic_trainer *t, const void *ctx, const void *tgt, int B, float *d_loss,
                               bool backward, cudaStream_t st) {
    const int n = (int)t->nparams, nb = (n + 255) / 256;
    const size_t es = t->wide ? 2 : 1;   // bytes per sample
    // with value weights every chunk's terms are normalised by the whole
    // batch's weight total, and the chunks simply add up
    if (t->weighted) k_wsum<<<1, 1024, 0, st>>>(tgt, t->wide, B, t->n_out, t->vw, t->wnorm, t->err);
    for (int c0 = 0; c0 < B; c0 += t->max_batch) {
        const int bc = min(t->max_batch, B - c0);
        dlic_status s = run(t, static_cast<const char *>(ctx) + (size_t)c0 * t->n_in * es,
                            static_cast<const char *>(tgt) + (size_t)c0 * es, bc, t->closs, backward, st, t->weighted);
        if (s) return s;
        const float w = t->weighted ? 1.0f : (float)bc / (float)B;
        k_accum<<<1, 32, 0, st>>>(t->lacc, t->closs, 1, w, c0 == 0);
        if (backward) k_accum<<<nb, 256, 0, st>>>(t->gacc, t->grads, n, w, c0 == 0);
    }
    cudaError_t ce = cudaMemcpyAsync(d_loss, t->lacc, 4, cudaMemcpyDeviceToDevice, st);
    if (ce == cudaSuccess && backward)
        ce = cudaMemcpyAsync(t->grads, t->gacc, 4ull * n, cudaMemcpyDeviceToDevice, st);
    return ce == cudaSuccess ? DLIC_OK : cuda_fail(ce, "chunk sums");
}

static dlic_status run_any(dlic_trainer *t, const void *ctx, const void *tgt, int B, float *d_loss,
                           bool backward, cudaStream_t st) {
    return B <= t->max_batch ? run(t, ctx, tgt, B, d_loss, backward, st)
                             : run_chunked(t, ctx, tgt, B, d_loss, backward, st);
}

extern "C" dlic_status dlic_train_forward(dlic_trainer *t, const void *d_ctx, const void *d_tgt, int B,
                                          float *d_loss_bits, void *stream) {
    dlic_status s = check_batch(t, d_ctx, d_tgt, B);
    if (s) return s;
    if (!d_loss_bits) return fail(DLIC_ERR_INVALID, "null loss output");
    return run_any(t, d_ctx, d_tgt, B, d_loss_bits, false, static_cast<cudaStream_t>(stream));
}

extern "C" dlic_status dlic_train_backward(dlic_trainer *t, const void *d_ctx, const void *d_tgt, int B,
                                           float *d_loss_bits, float *d_grads, void *stream) {
    dlic_status s = check_batch(t, d_ctx, d_tgt, B);
    if (s) return s;
    if (!d_loss_bits) return fail(DLIC_ERR_INVALID, "null loss output");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = run_any(t, d_ctx, d_tgt, B, d_loss_bits, true, st);
    if (s) return s;
    if (d_grads) {
        cudaError_t ce = cudaMemcpyAsync(d_grads, t->grads, 4 * t->nparams, cudaMemcpyDeviceToDevice, st);
        if (ce != cudaSuccess) return cuda_fail(ce, "gradient copy");
    }
    return DLIC_OK;
}

extern "C" dlic_status dlic_train_step(dlic_trainer *t, const void *d_ctx, const void *d_tgt, int B,
                                       float *d_loss_bits, void *stream) {
    dlic_status s = check_batch(t, d_ctx, d_tgt, B);
    if (s) return s;
    if (!d_loss_bits) return fail(DLIC_ERR_INVALID, "null loss output");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = run_any(t, d_ctx, d_tgt, B, d_loss_bits, true, st);
    if (s) return s;
    t->step += 1;
    const float c1 = 1.0f - powf(t->beta1, (float)t->step), c2 = 1.0f - powf(t->beta2, (float)t->step);
    const ShadowArgs sa{t->n_in, t->k1, t->h1, t->h2, t->n_out, t->bf, t->split, t->w1, t->w2, t->w3, t->w2t, t->w3t};
    k_adam<<<(int)((t->nparams + 255) / 256), 256, 0, st>>>(t->params, t->grads, t->mom, t->vel, (int)t->nparams, t->lr,
                                                             t->beta1, t->beta2, t->eps, c1, c2, sa);
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? DLIC_OK : cuda_fail(ce, "adam launch");
}

extern "C" dlic_status dlic_train_apply(dlic_trainer *t, const float *d_grads, void *stream) {
    if (!t || !d_grads) return fail(DLIC_ERR_INVALID, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    t->step += 1;
    const float c1 = 1.0f - powf(t->beta1, (float)t->step), c2 = 1.0f - powf(t->beta2, (float)t->step);
    const ShadowArgs sa{t->n_in, t->k1, t->h1, t->h2, t->n_out, t->bf, t->split, t->w1, t->w2, t->w3, t->w2t, t->w3t};
    k_adam<<<(int)((t->nparams + 255) / 256), 256, 0, st>>>(t->params, d_grads, t->mom, t->vel, (int)t->nparams, t->lr,
                                                             t->beta1, t->beta2, t->eps, c1, c2, sa);
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? DLIC_OK : cuda_fail(ce, "adam launch");
}

extern "C" dlic_status dlic_trainer_set_value_weights(dlic_trainer *t, const float *h_weights) {
    if (!t) return fail(DLIC_ERR_INVALID, "null trainer");
    if (!h_weights) {
        t->weighted = 0;
        return DLIC_OK;
    }
    double total = 0.0;
    for (int v = 0; v < t->n_out; v++) {
        if (!(h_weights[v] >= 0.0f) || !isfinite(h_weights[v]))
            return fail(DLIC_ERR_INVALID, "value weight %d is negative or not finite", v);
        total += h_weights[v];
    }
    if (!(total > 0.0)) return fail(DLIC_ERR_INVALID, "every value weight is zero");
    cudaError_t ce = cudaMemcpy(t->vw, h_weights, 4 * (size_t)t->n_out, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return cuda_fail(ce, "value weights");
    t->weighted = 1;
    return DLIC_OK;
}

extern "C" dlic_status dlic_trainer_params(dlic_trainer *t, float *d_params, int write, void *stream) {
    if (!t || !d_params) return fail(DLIC_ERR_INVALID, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t ce = write ? cudaMemcpyAsync(t->params, d_params, 4 * t->nparams, cudaMemcpyDeviceToDevice, st)
                           : cudaMemcpyAsync(d_params, t->params, 4 * t->nparams, cudaMemcpyDeviceToDevice, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "parameter copy");
    return write ? refresh_shadows(t, st) : DLIC_OK;
}

extern "C" dlic_status dlic_trainer_status(dlic_trainer *t, int32_t *h_status) {
    if (!t || !h_status) return fail(DLIC_ERR_INVALID, "null argument");
    cudaError_t ce = cudaMemcpy(h_status, t->err, 4, cudaMemcpyDeviceToHost);
    return ce == cudaSuccess ? DLIC_OK : cuda_fail(ce, "status copy");
}
