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
// cores.  Every product is a GEMM C = A B^T with both operands K-major
// (row-major, K contiguous); the backward pass uses transposed copies of the
// activations (written by the producing epilogues) and of the weights.
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
    const void *act;            // RELU_GRAD: activation [M][N] whose sign masks the gradient
    const uint8_t *tgt;         // SOFTMAX: targets
    float inv_batch_ln2;        // SOFTMAX: 1 / (B ln 2)
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

// Adds 16 column values of this thread's row into the shared column sums:
// a reduce-scatter across the warp (each lane ends with one column's warp
// total for lanes 0..15 after four halving steps) and one shared atomic per
// column and warp.
__device__ __forceinline__ void colsum_add(float *cs, float (&v)[16]) {
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
    if (lane < 16) atomicAdd(cs + (lane & 15), a[0]);
}

// Column sums go through shared memory: `cs` holds N floats zeroed by the
// caller; each warp adds its rows' values (colsum_add).
template <class Row>
__device__ void row_epilogue(int epi, const EpiArgs &e, const Row &row, int m, bool valid, float *cs,
                             float *loss_acc) {
    const int N = e.N;
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
                    colsum_add(cs + n0, v);
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
            if (cs) colsum_add(cs + n0, v);
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
    for (int n0 = 0; n0 < N; n0 += 16) {
        float v[16];
        row.load16(n0, v);
        if (!valid) {
            if (cs) {
#pragma unroll
                for (int j = 0; j < 16; j++) v[j] = 0.0f;
                colsum_add(cs + n0, v);
            }
            continue;
        }
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const float zz = v[j] + e.bias[n0 + j];
            float g = expf(zz - mx) * inv;
            if (n0 + j == y) {
                g -= 1.0f;
                *loss_acc += (lse - zz) / kLn2;
            }
            g *= e.inv_batch_ln2;
            store_val(e, e.out, (size_t)m * N + n0 + j, g, e.out_plane);
            store_val(e, e.outT, (size_t)(n0 + j) * e.ldT + m, g, e.outT_plane);
            v[j] = g;
        }
        if (cs) colsum_add(cs + n0, v);
    }
}

// ---------------------------------------------------------------------------
// tcgen05 GEMM: C[M x N] = A[M x K] * B[N x K]^T, bf16 operands fed by TMA
// (128-byte swizzle, 64-element K blocks), FP32 accumulators in tensor
// memory, a fused epilogue.  One 128 x N tile per CTA (N <= 256); split-K
// over gridDim.z for EPI_F32.  Warp 0 loads, warp 1 issues MMAs, warps 2..9
// run the epilogue: two warps per tensor-memory lane quarter, each on half of
// the columns of its 32 rows.  Row-major outputs leave as 16-byte vectors;
// transposed outputs are staged in shared memory (the drained pipeline
// stages) and written as coalesced 16-byte rows.  Two stages keep a CTA at
// 96 KB so that two CTAs share an SM (BF16 mode).
// ---------------------------------------------------------------------------
constexpr int kGemmThreads = 320;
constexpr int kEpiThreads = 256;
constexpr int kGemmStages = 2;

__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
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
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 2, %0;" ::"r"(kEpiThreads) : "memory"); }

// 16 values as bf16 (and their low parts) in the two layouts: row-major
// vectors to global memory, transposed 2-byte entries to the staging tile.
__device__ __forceinline__ void emit16(const EpiArgs &e, const float (&v)[16], int m, int row, int n0, bool valid,
                                       uint16_t *Thi, uint16_t *Tlo, bool rowmajor) {
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint16_t a = f2bf(v[2 * j]), b = f2bf(v[2 * j + 1]);
        hi[j] = a | ((uint32_t)b << 16);
        lo[j] = f2bf(v[2 * j] - bf2f(a)) | ((uint32_t)f2bf(v[2 * j + 1] - bf2f(b)) << 16);
        Thi[(n0 + 2 * j) * 128 + row] = a;
        Thi[(n0 + 2 * j + 1) * 128 + row] = b;
        if (e.split) {
            Tlo[(n0 + 2 * j) * 128 + row] = (uint16_t)lo[j];
            Tlo[(n0 + 2 * j + 1) * 128 + row] = (uint16_t)(lo[j] >> 16);
        }
    }
    if (rowmajor && valid) {
        uint4 *o = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(e.out) + (size_t)m * e.N + n0);
        o[0] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        o[1] = make_uint4(hi[4], hi[5], hi[6], hi[7]);
        if (e.split) {
            uint4 *ol = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(e.out) + e.out_plane + (size_t)m * e.N + n0);
            ol[0] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            ol[1] = make_uint4(lo[4], lo[5], lo[6], lo[7]);
        }
    }
}

// SPLIT: operands come as high and low bf16 planes (x = hi + lo) and every K
// step issues hi*hi + lo*hi + hi*lo, which keeps about 16 significant bits of
// each operand.
template <bool SPLIT>
__global__ void __launch_bounds__(kGemmThreads, SPLIT ? 1 : 2)
    k_gemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const __grid_constant__ CUtensorMap mapAl, const __grid_constant__ CUtensorMap mapBl, int K,
              int kb_per_split, int epi, EpiArgs e, int *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[kGemmStages], empty[kGemmStages], accum;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    __shared__ float cs[256];
    __shared__ float red[2][2][128];
    __shared__ float s_loss[kGemmThreads / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = e.N;
    const uint32_t a_bytes = 128 * 128, b_bytes = (uint32_t)N * 128;
    const uint32_t b_al = (b_bytes + 1023) & ~1023u;
    const uint32_t stage_bytes = SPLIT ? 2 * (a_bytes + b_al) : a_bytes + b_al;
    const int nkb_total = (K + 63) / 64;
    const int kb0 = blockIdx.z * kb_per_split;
    const int kb1 = min(nkb_total, kb0 + kb_per_split);
    const int nkb = max(0, kb1 - kb0);
    const int m0 = blockIdx.x * 128;

    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 256);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < kGemmStages; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(&accum, 1);
        tc::fence_mbar_init();
        s_fail = 0;
    }
    for (int n = tid; n < 256; n += kGemmThreads) cs[n] = 0.0f;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = tmem_base;

    if (warp == 0 && lane == 0) {
        // producer
        for (int i = 0; i < nkb; i++) {
            const int s = i % kGemmStages;
            if (!tc::mbar_wait(&empty[s], ((i / kGemmStages) & 1) ^ 1, kGemmWaitLimit)) { s_fail = 1; break; }
            uint8_t *st = smem + s * stage_bytes;
            mbar_expect_tx(&full[s], SPLIT ? 2 * (a_bytes + b_bytes) : a_bytes + b_bytes);
            tma_load_2d(tc::smem_addr(st), &mapA, (kb0 + i) * 64, m0, tc::smem_addr(&full[s]));
            tma_load_2d(tc::smem_addr(st + a_bytes), &mapB, (kb0 + i) * 64, 0, tc::smem_addr(&full[s]));
            if (SPLIT) {
                tma_load_2d(tc::smem_addr(st + a_bytes + b_al), &mapAl, (kb0 + i) * 64, m0, tc::smem_addr(&full[s]));
                tma_load_2d(tc::smem_addr(st + 2 * a_bytes + b_al), &mapBl, (kb0 + i) * 64, 0, tc::smem_addr(&full[s]));
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = tc::idesc_bf16_f32(128, N);
        for (int i = 0; i < nkb; i++) {
            const int s = i % kGemmStages;
            if (!tc::mbar_wait(&full[s], (i / kGemmStages) & 1, kGemmWaitLimit)) { s_fail = 1; break; }
            tc::fence_after_sync();
            uint8_t *st = smem + s * stage_bytes;
            const uint64_t da = desc_sw128(tc::smem_addr(st)), db = desc_sw128(tc::smem_addr(st + a_bytes));
#pragma unroll
            for (int ks = 0; ks < 4; ks++) tc::mma_bf16(tm, da + 2u * ks, db + 2u * ks, idesc, (i | ks) != 0);
            if (SPLIT) {
                const uint64_t dal = desc_sw128(tc::smem_addr(st + a_bytes + b_al));
                const uint64_t dbl = desc_sw128(tc::smem_addr(st + 2 * a_bytes + b_al));
#pragma unroll
                for (int ks = 0; ks < 4; ks++) {
                    tc::mma_bf16(tm, dal + 2u * ks, db + 2u * ks, idesc, 1u);
                    tc::mma_bf16(tm, da + 2u * ks, dbl + 2u * ks, idesc, 1u);
                }
            }
            tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(&accum);
    } else if (warp >= 2) {
        if (lane == 0 && !tc::mbar_wait(&accum, 0, kGemmWaitLimit)) s_fail = 1;
        __syncwarp();
        tc::mbar_wait(&accum, 0, 1000);   // every lane observes the completed phase
        tc::fence_after_sync();
    }
    // all loads and MMAs are done: the pipeline stages become the staging tiles
    __syncwarp();
    asm volatile("bar.sync 1, %0;" ::"r"(kGemmThreads) : "memory");
    uint16_t *Thi = reinterpret_cast<uint16_t *>(smem);
    uint16_t *Tlo = Thi + (size_t)N * 128;
    float loss_acc = 0.0f;
    const bool staged = epi != EPI_F32;
    if (warp >= 2) {
        const int q = warp & 3, hf = (warp - 2) >> 2;
        const int row = 32 * q + lane, m = m0 + row;
        const bool valid = m < e.M;
        // the two halves split the 16-column chunks (the first takes the odd one)
        const int nch = N / 16, first = (nch + 1) / 2;
        const int n_lo = hf ? 16 * first : 0, n_hi = hf ? N : 16 * first;
        const bool active = !s_fail && n_lo < n_hi;
        TmemRow src{tm + ((uint32_t)(32 * q) << 16)};
        if (epi == EPI_F32) {
            if (active && valid) {
                float *c = e.c + (size_t)blockIdx.z * e.M * e.ldc + (size_t)m * e.ldc;
                for (int n0 = n_lo; n0 < n_hi; n0 += 16) {
                    float v[16];
                    if (nkb > 0) {
                        src.load16(n0, v);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; j++) v[j] = 0.0f;
                    }
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4 *>(c + n0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
            }
        } else if (epi == EPI_BIAS_RELU) {
            if (active)
                for (int n0 = n_lo; n0 < n_hi; n0 += 16) {
                    float v[16];
                    src.load16(n0, v);
#pragma unroll
                    for (int j = 0; j < 16; j++) v[j] = fmaxf(v[j] + e.bias[n0 + j], 0.0f);
                    emit16(e, v, m, row, n0, valid, Thi, Tlo, true);
                }
        } else if (epi == EPI_RELU_GRAD) {
            if (active)
                for (int n0 = n_lo; n0 < n_hi; n0 += 16) {
                    float v[16];
                    src.load16(n0, v);
                    uint4 a0 = make_uint4(0, 0, 0, 0), a1 = a0;
                    if (valid) {
                        const uint4 *ap = reinterpret_cast<const uint4 *>(static_cast<const uint16_t *>(e.act) + (size_t)m * N + n0);
                        a0 = ap[0];
                        a1 = ap[1];
                    }
                    const uint32_t aw[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const uint32_t bits = (aw[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
                        const bool pos = valid && bits != 0 && (bits & 0x8000u) == 0;   // bf16 > 0
                        v[j] = pos ? v[j] : 0.0f;
                    }
                    emit16(e, v, m, row, n0, valid, Thi, Tlo, e.out != nullptr);
                    if (e.colsum) colsum_add(cs + n0, v);
                }
        } else {
            // EPI_SOFTMAX over the full row: halves combine through shared memory
            float mx = -INFINITY;
            if (active)
                for (int n0 = n_lo; n0 < n_hi; n0 += 16) {
                    float v[16];
                    src.load16(n0, v);
#pragma unroll
                    for (int j = 0; j < 16; j++) mx = fmaxf(mx, v[j] + e.bias[n0 + j]);
                }
            red[0][hf][row] = mx;
            epi_sync();
            mx = fmaxf(red[0][0][row], red[0][1][row]);
            float se = 0.0f;
            if (active)
                for (int n0 = n_lo; n0 < n_hi; n0 += 16) {
                    float v[16];
                    src.load16(n0, v);
#pragma unroll
                    for (int j = 0; j < 16; j++) se += expf(v[j] + e.bias[n0 + j] - mx);
                }
            red[1][hf][row] = se;
            epi_sync();
            se = red[1][0][row] + red[1][1][row];
            const float lse = mx + logf(se), inv = 1.0f / se;
            const int y = valid ? e.tgt[m] : -1;
            if (active)
                for (int n0 = n_lo; n0 < n_hi; n0 += 16) {
                    float v[16];
                    src.load16(n0, v);
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const float zz = v[j] + e.bias[n0 + j];
                        float g = expf(zz - mx) * inv;
                        if (n0 + j == y) {
                            g -= 1.0f;
                            loss_acc += (lse - zz) / kLn2;
                        }
                        v[j] = valid ? g * e.inv_batch_ln2 : 0.0f;
                    }
                    emit16(e, v, m, row, n0, valid, Thi, Tlo, true);
                    if (e.colsum) colsum_add(cs + n0, v);
                }
        }
        if (staged && !s_fail) {
            // transposed tile -> outT[n][m0 ..] as 16-byte rows
            epi_sync();
            const int et = tid - 64;
            for (int idx = et; idx < N * 16; idx += kEpiThreads) {
                const int n = idx >> 4, ml = (idx & 15) * 8, gm = m0 + ml;
                uint16_t *dst = static_cast<uint16_t *>(e.outT) + (size_t)n * e.ldT + gm;
                const uint4 vh = *reinterpret_cast<const uint4 *>(Thi + n * 128 + ml);
                if (gm + 8 <= e.M) {
                    *reinterpret_cast<uint4 *>(dst) = vh;
                    if (e.split) *reinterpret_cast<uint4 *>(dst + e.outT_plane) = *reinterpret_cast<const uint4 *>(Tlo + n * 128 + ml);
                } else {
                    for (int j = 0; j < 8 && gm + j < e.M; j++) {
                        dst[j] = Thi[n * 128 + ml + j];
                        if (e.split) dst[j + e.outT_plane] = Tlo[n * 128 + ml + j];
                    }
                }
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
    if (lane == 0) s_loss[warp] = loss_acc;
    tc::fence_before_sync();
    __syncthreads();
    if (e.colsum)
        for (int n = tid; n < N; n += kGemmThreads) e.colsum[(size_t)blockIdx.x * N + n] = cs[n];
    if (e.loss && tid == 0) {
        float t = 0.0f;
        for (int w = 0; w < kGemmThreads / 32; w++) t += s_loss[w];
        e.loss[blockIdx.x] = t;
    }
    if (tid == 0 && s_fail) atomicExch(err, DLIC_ERR_TIMEOUT);
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tm, 256);
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
    extern __shared__ float cs[];
    const int tid = threadIdx.x;
    for (int n = tid; n < e.N; n += 128) cs[n] = 0.0f;
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
        for (int n = tid; n < e.N; n += 128) e.colsum[(size_t)blockIdx.x * e.N + n] = cs[n];
    if (e.loss && tid == 0) e.loss[blockIdx.x] = s_loss[0] + s_loss[1] + s_loss[2] + s_loss[3];
}

// ---------------------------------------------------------------------------
// Small kernels: features, reductions, Adam, weight shadows.
// ---------------------------------------------------------------------------
// v / 128 - 1 has at most 8 significant bits: exact in bf16, low plane 0.
__global__ void k_features(const uint8_t *ctx, int B, int ldT, void *X, void *XT, int bf16, size_t xplane,
                           size_t xtplane) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    for (int k = 0; k < 16; k++) {
        const float x = k < kPriors ? (float)ctx[(size_t)b * kPriors + k] * 0.0078125f - 1.0f : 0.0f;
        if (bf16) {
            reinterpret_cast<uint16_t *>(X)[(size_t)b * 16 + k] = f2bf(x);
            reinterpret_cast<uint16_t *>(XT)[(size_t)k * ldT + b] = f2bf(x);
            if (xplane) {
                reinterpret_cast<uint16_t *>(X)[(size_t)b * 16 + k + xplane] = 0;
                reinterpret_cast<uint16_t *>(XT)[(size_t)k * ldT + b + xtplane] = 0;
            }
        } else {
            reinterpret_cast<float *>(X)[(size_t)b * 16 + k] = x;
            reinterpret_cast<float *>(XT)[(size_t)k * ldT + b] = x;
        }
    }
}

// First layer in FP32 on the CUDA cores (K = 12): h1 = relu(W1 x + b1),
// written as split bf16 (hi and lo planes), row-major and transposed, through
// a shared-memory tile so both stores are coalesced.  The split mode uses it
// because a1 sums only 12 products and often sits near the ReLU kink, where
// 16-bit operand precision would flip masks relative to exact arithmetic.
__global__ void __launch_bounds__(256) k_layer1_f32(const uint8_t *ctx, int B, const float *W1, const float *b1,
                                                    int h1, uint16_t *H1, uint16_t *H1T, int ldT, size_t p1,
                                                    size_t p1T) {
    __shared__ float tile[32][257];
    __shared__ float xs[32][kPriors];
    const int tid = threadIdx.x, b0 = blockIdx.x * 32;
    for (int i = tid; i < 32 * kPriors; i += 256) {
        const int r = i / kPriors, k = i % kPriors;
        xs[r][k] = b0 + r < B ? (float)ctx[(size_t)(b0 + r) * kPriors + k] * 0.0078125f - 1.0f : 0.0f;
    }
    __syncthreads();
    for (int j = tid; j < h1; j += 256) {
        float w[kPriors];
#pragma unroll
        for (int k = 0; k < kPriors; k++) w[k] = W1[j * kPriors + k];
        const float bj = b1[j];
        for (int r = 0; r < 32; r++) {
            float acc = bj;
#pragma unroll
            for (int k = 0; k < kPriors; k++) acc = fmaf(xs[r][k], w[k], acc);
            tile[r][j] = fmaxf(acc, 0.0f);
        }
    }
    __syncthreads();
    for (int i = tid; i < 32 * h1; i += 256) {
        const int r = i / h1, j = i % h1;
        if (b0 + r >= B) continue;
        const float v = tile[r][j];
        const uint16_t hi = f2bf(v), lo = f2bf(v - bf2f(hi));
        H1[(size_t)(b0 + r) * h1 + j] = hi;
        H1[(size_t)(b0 + r) * h1 + j + p1] = lo;
    }
    for (int i = tid; i < 32 * h1; i += 256) {
        const int j = i / 32, r = i % 32;
        if (b0 + r >= B) continue;
        const float v = tile[r][j];
        const uint16_t hi = f2bf(v), lo = f2bf(v - bf2f(hi));
        H1T[(size_t)j * ldT + b0 + r] = hi;
        H1T[(size_t)j * ldT + b0 + r + p1T] = lo;
    }
}

// out[i] = sum_z part[z * stride + i] (fixed order: deterministic)
// out[i] = scale * sum_z part[z * stride + i]: 32 columns per block, the
// partials split over blockDim.y row groups and combined in a fixed order
// (deterministic).  With `pad16` the columns are a [h][16] array whose first
// kPriors entries per row go to a compact [h][kPriors] output.
__global__ void k_reduce_parts(const float *part, int nparts, size_t stride, int n, float *out, float scale, int pad16) {
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
        if (!pad16) out[i] = t;
        else if (i % 16 < kPriors) out[(i / 16) * kPriors + i % 16] = t;
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
    int h1, h2, bf16, split;
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
    const int h1 = sa.h1, h2 = sa.h2;
    const int oW2 = h1 * kPriors + h1, oW3 = oW2 + h2 * h1 + h2;
    if (i < h1 * kPriors) {
        shadow_put(sa.w1, (size_t)(i / kPriors) * 16 + i % kPriors, (size_t)h1 * 16, w, sa.bf16, sa.split);
    } else if (i >= oW2 && i < oW2 + h2 * h1) {
        const int j = i - oW2, o = j / h1, k = j % h1;
        shadow_put(sa.w2, j, (size_t)h2 * h1, w, sa.bf16, sa.split);
        shadow_put(sa.w2t, (size_t)k * h2 + o, (size_t)h1 * h2, w, sa.bf16, sa.split);
    } else if (i >= oW3 && i < oW3 + kSymbols * h2) {
        const int j = i - oW3, o = j / h2, k = j % h2;
        shadow_put(sa.w3, j, (size_t)kSymbols * h2, w, sa.bf16, sa.split);
        shadow_put(sa.w3t, (size_t)k * kSymbols + o, (size_t)h2 * kSymbols, w, sa.bf16, sa.split);
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
    int h1, h2, mode, max_batch, num_sms;
    int bf, split;                               // bf16 operands; hi + lo planes
    size_t nparams;
    int step;
    float lr, beta1, beta2, eps;
    float *params, *grads, *mom, *vel;           // FP32 master state
    void *w1, *w2, *w3, *w2t, *w3t;              // operand copies (bf16 or fp32)
    void *X, *XT, *H1, *H1T, *H2, *H2T, *DZ, *DZT, *DA2, *DA2T, *DA1T;
    float *C, *part, *colsum, *losspart;
    int *err;
    std::vector<void *> allocs;
};

namespace {

size_t param_count(int h1, int h2) {
    return (size_t)h1 * kPriors + h1 + (size_t)h2 * h1 + h2 + (size_t)kSymbols * h2 + kSymbols;
}

struct ParamView {
    float *W1, *b1, *W2, *b2, *W3, *b3;
};
ParamView view(float *p, int h1, int h2) {
    ParamView v;
    v.W1 = p;
    v.b1 = v.W1 + (size_t)h1 * kPriors;
    v.W2 = v.b1 + h1;
    v.b2 = v.W2 + (size_t)h2 * h1;
    v.W3 = v.b2 + h2;
    v.b3 = v.W3 + (size_t)kSymbols * h2;
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

// C = A[M x K] B[N x K]^T with the given epilogue; A and B K-major with row
// pitches lda and ldb (elements).
dlic_status gemm(dlic_trainer *t, const void *A, int lda, size_t aplane, const void *Bm, int ldb, size_t bplane, int M,
                 int N, int K, int epi, EpiArgs e, int splits, cudaStream_t st) {
    e.M = M;
    e.N = N;
    e.ldT = t->max_batch;
    e.bf16 = t->bf;
    e.split = t->split;
    const int mt = (M + 127) / 128;
    if (t->bf) {
        CUtensorMap ma, mb, mal, mbl;
        const uint16_t *A16 = static_cast<const uint16_t *>(A), *B16 = static_cast<const uint16_t *>(Bm);
        if (encode_map(&ma, A16, M, K, lda, 128) != CUDA_SUCCESS || encode_map(&mb, B16, N, K, ldb, N) != CUDA_SUCCESS)
            return fail(DLIC_ERR_CUDA, "cuTensorMapEncodeTiled failed (M %d N %d K %d)", M, N, K);
        mal = ma;
        mbl = mb;
        if (t->split && (encode_map(&mal, A16 + aplane, M, K, lda, 128) != CUDA_SUCCESS ||
                         encode_map(&mbl, B16 + bplane, N, K, ldb, N) != CUDA_SUCCESS))
            return fail(DLIC_ERR_CUDA, "cuTensorMapEncodeTiled failed (low planes)");
        const int nkb = (K + 63) / 64;
        const int per = (nkb + splits - 1) / splits;
        const uint32_t stage = 128 * 128 + ((uint32_t)N * 128 + 1023) / 1024 * 1024;
        const size_t smem = (size_t)kGemmStages * (t->split ? 2 : 1) * stage + 1024;
        if (t->split) {
            cudaFuncSetAttribute(k_gemm_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_gemm_tc<true><<<dim3(mt, 1, splits), kGemmThreads, smem, st>>>(ma, mb, mal, mbl, K, per, epi, e, t->err);
        } else {
            cudaFuncSetAttribute(k_gemm_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_gemm_tc<false><<<dim3(mt, 1, splits), kGemmThreads, smem, st>>>(ma, mb, mal, mbl, K, per, epi, e, t->err);
        }
        cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) return cuda_fail(ce, "k_gemm_tc launch");
        return DLIC_OK;
    }
    // FP32 path: raw GEMM into C (or the split-K partials), then the row epilogue
    const int per = ((K + splits - 1) / splits + 7) / 8 * 8;
    float *dst = epi == EPI_F32 ? e.c : t->C;
    const int ldc = epi == EPI_F32 ? e.ldc : N;
    k_gemm_f32<<<dim3(mt, (N + 127) / 128, splits), 256, 0, st>>>(static_cast<const float *>(A), lda,
                                                                   static_cast<const float *>(Bm), ldb, dst, M, N, K, per, ldc);
    if (epi != EPI_F32) k_row_epilogue<<<mt, 128, N * sizeof(float), st>>>(t->C, epi, e);
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? DLIC_OK : cuda_fail(ce, "fp32 gemm launch");
}

void reduce_parts(const float *part, int nparts, size_t stride, int n, float *out, float scale, int pad16,
                  cudaStream_t st) {
    const int G = nparts >= 256 ? 32 : 8;
    k_reduce_parts<<<(n + 31) / 32, dim3(32, G), 0, st>>>(part, nparts, stride, n, out, scale, pad16);
}

dlic_status refresh_shadows(dlic_trainer *t, cudaStream_t st) {
    ParamView p = view(t->params, t->h1, t->h2);
    const int bf = t->bf, sp = t->split;
    k_shadow<<<(t->h1 * 16 + 255) / 256, 256, 0, st>>>(p.W1, t->h1, kPriors, 16, t->w1, nullptr, bf, sp);
    k_shadow<<<(t->h2 * t->h1 + 255) / 256, 256, 0, st>>>(p.W2, t->h2, t->h1, t->h1, t->w2, t->w2t, bf, sp);
    k_shadow<<<(kSymbols * t->h2 + 255) / 256, 256, 0, st>>>(p.W3, kSymbols, t->h2, t->h2, t->w3, t->w3t, bf, sp);
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? DLIC_OK : cuda_fail(ce, "shadow launch");
}

// Forward (and, if `grads`, backward) over one batch.
dlic_status run(dlic_trainer *t, const uint8_t *ctx, const uint8_t *tgt, int B, float *d_loss, bool backward,
                cudaStream_t st) {
    const int h1 = t->h1, h2 = t->h2, mt = (B + 127) / 128;
    const int bf = t->bf;
    ParamView p = view(t->params, h1, h2);
    ParamView g = view(t->grads, h1, h2);
    const int P = t->max_batch;   // pitch of every transposed [N][batch] array
    const size_t Bm = (size_t)P;  // low planes follow each buffer at its full capacity
    const size_t sp = t->split ? 1 : 0;
    k_features<<<(B + 255) / 256, 256, 0, st>>>(ctx, B, P, t->X, t->XT, bf, sp * Bm * 16, sp * 16 * Bm);
    EpiArgs e{};
    // layer 1, 2: bias + ReLU, row-major and transposed activations
    e.bias = p.b1; e.out = t->H1; e.outT = t->H1T; e.out_plane = Bm * h1; e.outT_plane = (size_t)h1 * Bm;
    dlic_status s = DLIC_OK;
    if (t->split)
        k_layer1_f32<<<(B + 31) / 32, 256, 0, st>>>(ctx, B, p.W1, p.b1, h1, static_cast<uint16_t *>(t->H1),
                                                     static_cast<uint16_t *>(t->H1T), P, Bm * h1, (size_t)h1 * Bm);
    else if ((s = gemm(t, t->X, 16, Bm * 16, t->w1, 16, (size_t)h1 * 16, B, h1, 16, EPI_BIAS_RELU, e, 1, st)))
        return s;
    e = EpiArgs{}; e.bias = p.b2; e.out = t->H2; e.outT = t->H2T; e.out_plane = Bm * h2; e.outT_plane = (size_t)h2 * Bm;
    if ((s = gemm(t, t->H1, h1, Bm * h1, t->w2, h1, (size_t)h2 * h1, B, h2, h1, EPI_BIAS_RELU, e, 1, st))) return s;
    // layer 3 + softmax cross-entropy: loss partials, dz, db3 partials
    e = EpiArgs{}; e.bias = p.b3; e.out = t->DZ; e.outT = t->DZT; e.tgt = tgt;
    e.out_plane = Bm * kSymbols; e.outT_plane = (size_t)kSymbols * Bm;
    e.inv_batch_ln2 = 1.0f / ((float)B * kLn2);
    e.colsum = t->colsum; e.loss = t->losspart;
    if ((s = gemm(t, t->H2, h2, Bm * h2, t->w3, h2, (size_t)kSymbols * h2, B, kSymbols, h2, EPI_SOFTMAX, e, 1, st)))
        return s;
    reduce_parts(t->losspart, mt, 1, 1, d_loss, 1.0f / (float)B, 0, st);
    if (!backward) {
        cudaError_t ce = cudaGetLastError();
        return ce == cudaSuccess ? DLIC_OK : cuda_fail(ce, "forward launch");
    }
    reduce_parts(t->colsum, mt, kSymbols, kSymbols, g.b3, 1.0f, 0, st);
    // dh2 = dz W3 (B operand W3^T), da2 = dh2 * [h2 > 0]; db2
    e = EpiArgs{}; e.act = t->H2; e.out = t->DA2; e.outT = t->DA2T; e.colsum = t->colsum;
    e.out_plane = Bm * h2; e.outT_plane = (size_t)h2 * Bm;
    if ((s = gemm(t, t->DZ, kSymbols, Bm * kSymbols, t->w3t, kSymbols, (size_t)h2 * kSymbols, B, h2, kSymbols,
                  EPI_RELU_GRAD, e, 1, st)))
        return s;
    reduce_parts(t->colsum, mt, h2, h2, g.b2, 1.0f, 0, st);
    // dh1 = da2 W2, da1 = dh1 * [h1 > 0]; db1
    e = EpiArgs{}; e.act = t->H1; e.out = nullptr; e.outT = t->DA1T; e.colsum = t->colsum;
    e.outT_plane = (size_t)h1 * Bm;
    if ((s = gemm(t, t->DA2, h2, Bm * h2, t->w2t, h2, (size_t)h1 * h2, B, h1, h2, EPI_RELU_GRAD, e, 1, st))) return s;
    reduce_parts(t->colsum, mt, h1, h1, g.b1, 1.0f, 0, st);
    // weight gradients: K = batch, split-K partials summed in a fixed order
    const int splits = max(1, min(64, (B + 1023) / 1024));
    e = EpiArgs{}; e.c = t->part; e.ldc = h2;
    if ((s = gemm(t, t->DZT, P, (size_t)kSymbols * Bm, t->H2T, P, (size_t)h2 * Bm, kSymbols, h2, B, EPI_F32, e, splits,
                  st)))
        return s;
    reduce_parts(t->part, splits, (size_t)kSymbols * h2, kSymbols * h2, g.W3, 1.0f, 0, st);
    e = EpiArgs{}; e.c = t->part; e.ldc = h1;
    if ((s = gemm(t, t->DA2T, P, (size_t)h2 * Bm, t->H1T, P, (size_t)h1 * Bm, h2, h1, B, EPI_F32, e, splits, st)))
        return s;
    reduce_parts(t->part, splits, (size_t)h2 * h1, h2 * h1, g.W2, 1.0f, 0, st);
    e = EpiArgs{}; e.c = t->part; e.ldc = 16;
    if ((s = gemm(t, t->DA1T, P, (size_t)h1 * Bm, t->XT, P, 16 * Bm, h1, 16, B, EPI_F32, e, splits, st))) return s;
    reduce_parts(t->part, splits, (size_t)h1 * 16, h1 * 16, g.W1, 1.0f, 1, st);
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? DLIC_OK : cuda_fail(ce, "backward launch");
}

}  // namespace

extern "C" size_t dlic_train_param_count(int h1, int h2) { return param_count(h1, h2); }

extern "C" dlic_status dlic_trainer_create(int h1, int h2, int mode, int max_batch, const float *h_params,
                                           dlic_trainer **out) {
    if (!out) return fail(DLIC_ERR_INVALID, "null output");
    *out = nullptr;
    if (h1 < 16 || h1 > 256 || h1 % 16 || h2 < 16 || h2 > 256 || h2 % 16)
        return fail(DLIC_ERR_UNSUPPORTED, "hidden widths must be multiples of 16 in [16, 256]");
    if (mode != DLIC_TRAIN_BF16 && mode != DLIC_TRAIN_FP32 && mode != DLIC_TRAIN_BF16X3)
        return fail(DLIC_ERR_INVALID, "unknown training mode %d", mode);
    if (max_batch < 1 || max_batch > (1 << 22)) return fail(DLIC_ERR_INVALID, "max_batch must be in [1, 2^22]");
    if (!h_params) return fail(DLIC_ERR_INVALID, "null initial parameters");
    dlic_trainer *t = new dlic_trainer();
    t->h1 = h1; t->h2 = h2; t->mode = mode;
    t->bf = mode != DLIC_TRAIN_FP32;
    t->split = mode == DLIC_TRAIN_BF16X3;
    t->max_batch = (max_batch + 127) / 128 * 128;
    t->nparams = param_count(h1, h2);
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
    t->w1 = A(es * h1 * 16);
    t->w2 = A(es * h2 * h1);
    t->w3 = A(es * kSymbols * h2);
    t->w2t = A(es * h1 * h2);
    t->w3t = A(es * h2 * kSymbols);
    t->X = A(es * Bm * 16);
    t->XT = A(es * 16 * Bm);
    t->H1 = A(es * Bm * h1);
    t->H1T = A(es * h1 * Bm);
    t->H2 = A(es * Bm * h2);
    t->H2T = A(es * h2 * Bm);
    t->DZ = A(es * Bm * kSymbols);
    t->DZT = A(es * kSymbols * Bm);
    t->DA2 = A(es * Bm * h2);
    t->DA2T = A(es * h2 * Bm);
    t->DA1T = A(es * h1 * Bm);
    t->C = (float *)A(4 * Bm * kSymbols);
    t->part = (float *)A(4 * 64 * (size_t)kSymbols * hmax);
    t->colsum = (float *)A(4 * (Bm / 128) * kSymbols);
    t->losspart = (float *)A(4 * (Bm / 128));
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

static dlic_status check_batch(dlic_trainer *t, const uint8_t *ctx, const uint8_t *tgt, int B) {
    if (!t) return fail(DLIC_ERR_INVALID, "null trainer");
    if (!ctx || !tgt) return fail(DLIC_ERR_INVALID, "null batch");
    if (B < 1 || B > t->max_batch) return fail(DLIC_ERR_CAPACITY, "batch %d outside [1, %d]", B, t->max_batch);
    return DLIC_OK;
}

extern "C" dlic_status dlic_train_forward(dlic_trainer *t, const uint8_t *d_ctx, const uint8_t *d_tgt, int B,
                                          float *d_loss_bits, void *stream) {
    dlic_status s = check_batch(t, d_ctx, d_tgt, B);
    if (s) return s;
    if (!d_loss_bits) return fail(DLIC_ERR_INVALID, "null loss output");
    return run(t, d_ctx, d_tgt, B, d_loss_bits, false, static_cast<cudaStream_t>(stream));
}

extern "C" dlic_status dlic_train_backward(dlic_trainer *t, const uint8_t *d_ctx, const uint8_t *d_tgt, int B,
                                           float *d_loss_bits, float *d_grads, void *stream) {
    dlic_status s = check_batch(t, d_ctx, d_tgt, B);
    if (s) return s;
    if (!d_loss_bits) return fail(DLIC_ERR_INVALID, "null loss output");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = run(t, d_ctx, d_tgt, B, d_loss_bits, true, st);
    if (s) return s;
    if (d_grads) {
        cudaError_t ce = cudaMemcpyAsync(d_grads, t->grads, 4 * t->nparams, cudaMemcpyDeviceToDevice, st);
        if (ce != cudaSuccess) return cuda_fail(ce, "gradient copy");
    }
    return DLIC_OK;
}

extern "C" dlic_status dlic_train_step(dlic_trainer *t, const uint8_t *d_ctx, const uint8_t *d_tgt, int B,
                                       float *d_loss_bits, void *stream) {
    dlic_status s = check_batch(t, d_ctx, d_tgt, B);
    if (s) return s;
    if (!d_loss_bits) return fail(DLIC_ERR_INVALID, "null loss output");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = run(t, d_ctx, d_tgt, B, d_loss_bits, true, st);
    if (s) return s;
    t->step += 1;
    const float c1 = 1.0f - powf(t->beta1, (float)t->step), c2 = 1.0f - powf(t->beta2, (float)t->step);
    const ShadowArgs sa{t->h1, t->h2, t->bf, t->split, t->w1, t->w2, t->w3, t->w2t, t->w3t};
    k_adam<<<(int)((t->nparams + 255) / 256), 256, 0, st>>>(t->params, t->grads, t->mom, t->vel, (int)t->nparams, t->lr,
                                                             t->beta1, t->beta2, t->eps, c1, c2, sa);
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? DLIC_OK : cuda_fail(ce, "adam launch");
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
