// INT8 dense layers of the wide networks on the tensor cores (encode).
//
// Sec. II-B ("Neural Network Architecture") allows hidden layers of up to
// 4096 neurons; a 4096 x 4096 layer is 16.8M multiply-adds per pixel, a
// dense contraction over all the pixels of a pass.  The INT8 layer's sum
// acc_j = sum_k x_k q_jk (x_k in [0, 255] the previous layer's units, q_jk
// in [-127, 127]) is an exact integer.  tcgen05 has no integer MMA on this
// GPU, so the sum runs as BF16 MMAs (both operands exact in bf16) with FP32
// accumulation, kept exact by chunks: K is cut into chunks of 256, whose
// partial sums are integers of magnitude at most 256 * 255 * 127 < 2^23, so
// every FP32 addition inside a chunk is exact in any order; the epilogue
// converts each chunk's accumulator to int32 and adds the chunks.  It then
// applies the layer's requantisation (hidden units, written as bf16 for the
// next layer) or its logit map (output layer), exactly as the CUDA-core
// kernels do, so the bitstreams do not change.
//
// Persistent CTAs over 128-pixel x 256-unit tiles: warp 0 issues the TMA
// loads of the activations and the weight rows (128-byte swizzle, K blocks
// of 64) through a ring of stages, warp 1 issues the MMAs of each chunk into
// one of two tensor-memory accumulators, and warps 2..9 drain the other one
// into int32 sums held in registers, so the MMAs never wait for the
// epilogue.  The tile is as wide as one MMA allows (N = 256), so that every
// byte the loads bring from L2 feeds as many multiply-adds as the tensor
// memory's two accumulators permit: the feed from L2 into shared memory,
// not the tensor pipe, is what bounds narrower tiles.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "coder_device.cuh"
#include "tc.cuh"

#include <algorithm>

namespace dlic {

constexpr int kWtThreads = 320;
constexpr int kWtEpiWarps = 8;
constexpr int kWtM = 128, kWtKB = 64;
constexpr int kWtChunkKB = 4;                           // K blocks per exact chunk (K = 256)
constexpr uint32_t kWtABytes = kWtM * kWtKB * 2;        // 16 KB: the activations' K block
constexpr long long kWtWaitLimit = 4000000000LL;
// Tiles of TN units (256, or 128 for a layer whose 256-wide tiles would
// leave most SMs idle): the weight rows of a K block and the stage count
// that fills about 192 KB of shared memory.
template <int TN>
struct WtShape {
    static constexpr uint32_t kBBytes = TN * kWtKB * 2;
    static constexpr uint32_t kStageBytes = kWtABytes + kBBytes;
    static constexpr int kStages = TN == 256 ? 4 : 6;
};

// K-major operand tile with 128-byte swizzle as TMA writes it: 8-row groups
// 1024 bytes apart; a K step of 16 advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void wt_tma_load(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void wt_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_addr(bar)), "r"(bytes) : "memory");
}

// Y = layer(X) for np pixels: X bf16 [np][K] at mapX (the first layer's
// priors v - 128, or the previous layer's u8 units, all exact in bf16), W
// bf16 [N][K] at mapW.  Hidden layer (logits == 0): Y[p * ldy + j] =
// bf16(requant(acc)) (uint16).  Output layer: Y[p * ldy + j] =
// fma(float(acc), s_j, o_j) (FP32).
template <int TN>
__global__ void __launch_bounds__(kWtThreads, 1)
    k_wide_tc(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapW, int K, int N, int np,
              const float *__restrict__ s, const float *__restrict__ o, void *Y, int ldy, int logits, int *err) {
    constexpr int kWtN = TN, kWtStages = WtShape<TN>::kStages;
    constexpr uint32_t kWtStageBytes = WtShape<TN>::kStageBytes;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[kWtStages], empty[kWtStages], cfull[2], cempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    __shared__ __align__(16) float s_so[kWtEpiWarps][2][128];   // an epilogue warp's scales and offsets
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // tile t: n-tile t mod nt, m-tile t / nt, so that the CTAs resident at
    // one time share their activation tiles (each read from DRAM once) and
    // the weights stay in L2
    const int nt = (N + kWtN - 1) / kWtN, tiles = nt * ((np + kWtM - 1) / kWtM);
    const int nkb = (K + kWtKB - 1) / kWtKB, nch = (nkb + kWtChunkKB - 1) / kWtChunkKB;

    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 2 * kWtN);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < kWtStages; q++) {
            tc::mbar_init(&full[q], 1);
            tc::mbar_init(&empty[q], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&cfull[b], 1);
            tc::mbar_init(&cempty[b], kWtEpiWarps);   // one arrival per epilogue warp
        }
        tc::fence_mbar_init();
        s_fail = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = tmem_base;
    auto failed = [&]() { return *reinterpret_cast<volatile int *>(&s_fail) != 0; };

    if (warp == 0 && lane == 0) {
        // producer: every K block of every tile of this CTA through the
        // stages (boxes reaching past the tensor's extent are zero-filled
        // and still deliver their full size)
        int it = 0;
        for (int t = blockIdx.x; t < tiles && !failed(); t += gridDim.x) {
            const int m0 = (t / nt) * kWtM, n0 = (t % nt) * kWtN;
            for (int i = 0; i < nkb; i++, it++) {
                const int q = it % kWtStages;
                if (!tc::mbar_wait(&empty[q], ((it / kWtStages) & 1) ^ 1, kWtWaitLimit)) {
                    s_fail = 1;
                    break;
                }
                uint8_t *st = smem + q * kWtStageBytes;
                const uint32_t bar = tc::smem_addr(&full[q]);
                wt_expect_tx(&full[q], kWtStageBytes);
                wt_tma_load(tc::smem_addr(st), &mapX, i * kWtKB, m0, bar);
                wt_tma_load(tc::smem_addr(st + kWtABytes), &mapW, i * kWtKB, n0, bar);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: chunk g of this CTA goes to accumulator g mod 2 once the
        // epilogue has drained chunk g - 2 from it
        const uint32_t idesc = tc::idesc_bf16_f32(kWtM, kWtN);
        int it = 0, g = 0;
        for (int t = blockIdx.x; t < tiles && !failed(); t += gridDim.x) {
            for (int c = 0; c < nch && !failed(); c++, g++) {
                const int b = g & 1;
                if (g >= 2 && !tc::mbar_wait(&cempty[b], ((g >> 1) - 1) & 1, kWtWaitLimit)) {
                    s_fail = 1;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t acc = tm + (uint32_t)(kWtN * b);
                const int i1 = min(nkb, (c + 1) * kWtChunkKB);
                for (int i = c * kWtChunkKB; i < i1; i++, it++) {
                    const int q = it % kWtStages;
                    if (!tc::mbar_wait(&full[q], (it / kWtStages) & 1, kWtWaitLimit)) {
                        s_fail = 1;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t st = tc::smem_addr(smem + q * kWtStageBytes);
                    const uint64_t dx = desc_sw128(st), dw = desc_sw128(st + kWtABytes);
#pragma unroll
                    for (int ks = 0; ks < kWtKB / 16; ks++)
                        tc::mma_bf16(acc, dx + 2u * ks, dw + 2u * ks, idesc, (i > c * kWtChunkKB || ks > 0) ? 1u : 0u);
                    tc::mma_commit(&empty[q]);
                }
                tc::mma_commit(&cfull[b]);
            }
        }
    } else if (warp >= 2) {
        // epilogue: warp w reads lanes 32 (w mod 4) .. + 31 (one pixel per
        // thread); the two warps of a lane quarter take half the columns each
        constexpr int kHalf = kWtN / 2;
        const int qd = warp & 3, hf = (warp - 2) >> 2;
        const uint32_t lanes = (uint32_t)(32 * qd) << 16;
        const int cb = kHalf * hf;
        float *sw = s_so[warp - 2][0], *ow = s_so[warp - 2][1];
        int g = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
            const int m0 = (t / nt) * kWtM, n0 = (t % nt) * kWtN;
            // this tile's scales and offsets of the warp's columns (its last
            // reads of the previous tile's are done: same warp)
            for (int i = lane; i < kHalf; i += 32) {
                const int j = n0 + cb + i;
                sw[i] = j < N ? s[j] : 0.0f;
                ow[i] = j < N ? o[j] : 0.0f;
            }
            __syncwarp();
            int R[kHalf];
            bool ok = true;
            for (int c = 0; c < nch; c++, g++) {
                const int b = g & 1;
                if (lane == 0 && !failed() && !tc::mbar_wait(&cfull[b], (g >> 1) & 1, kWtWaitLimit)) s_fail = 1;
                __syncwarp();
                // (warp-uniform: the accumulator loads are warp-collective)
                ok = __shfl_sync(0xffffffffu, failed() ? 0 : 1, 0) != 0;
                if (!ok) break;
                tc::mbar_wait(&cfull[b], (g >> 1) & 1, 1000);   // every lane observes the phase
                tc::fence_after_sync();
#pragma unroll
                for (int h = 0; h < kHalf / 16; h++) {
                    uint32_t v[16];
                    tc::tmem_ld16(tm + lanes + (uint32_t)(kWtN * b + cb + 16 * h), v);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 16; e++) {
                        const int x = __float2int_rn(__uint_as_float(v[e]));
                        R[16 * h + e] = c == 0 ? x : R[16 * h + e] + x;
                    }
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(&cempty[b])) : "memory");
            }
            if (!ok) break;
            const int p = m0 + 32 * qd + lane;
            if (p >= np) continue;
#pragma unroll
            for (int h = 0; h < kHalf / 16; h++) {
                const int j0 = n0 + cb + 16 * h;   // N is a multiple of 4
                if (j0 >= N) break;
                const int nv = min(16, N - j0);
                float sv[16], ov[16];
#pragma unroll
                for (int e = 0; e < 16; e += 4) {
                    const float4 a = *reinterpret_cast<const float4 *>(sw + 16 * h + e);
                    const float4 c = *reinterpret_cast<const float4 *>(ow + 16 * h + e);
                    sv[e] = a.x; sv[e + 1] = a.y; sv[e + 2] = a.z; sv[e + 3] = a.w;
                    ov[e] = c.x; ov[e + 1] = c.y; ov[e + 2] = c.z; ov[e + 3] = c.w;
                }
                if (logits) {
                    float *z = static_cast<float *>(Y) + (size_t)p * ldy + j0;
#pragma unroll
                    for (int e = 0; e < 16; e += 4)
                        if (e < nv)
                            *reinterpret_cast<float4 *>(z + e) =
                                make_float4(__fmaf_rn(__int2float_rn(R[16 * h + e]), sv[e], ov[e]),
                                            __fmaf_rn(__int2float_rn(R[16 * h + e + 1]), sv[e + 1], ov[e + 1]),
                                            __fmaf_rn(__int2float_rn(R[16 * h + e + 2]), sv[e + 2], ov[e + 2]),
                                            __fmaf_rn(__int2float_rn(R[16 * h + e + 3]), sv[e + 3], ov[e + 3]));
                } else {
                    // u = clamp(rint(fma(acc, s, o)), 0, 255) in the float
                    // domain (the same value as the integer requantisation),
                    // then its bf16 bits
                    uint32_t pk[8];
#pragma unroll
                    for (int e = 0; e < 8; e++) {
                        float u0 = rintf(__fmaf_rn(__int2float_rn(R[16 * h + 2 * e]), sv[2 * e], ov[2 * e]));
                        float u1 = rintf(__fmaf_rn(__int2float_rn(R[16 * h + 2 * e + 1]), sv[2 * e + 1], ov[2 * e + 1]));
                        u0 = fminf(fmaxf(u0, 0.0f), 255.0f);
                        u1 = fminf(fmaxf(u1, 0.0f), 255.0f);
                        pk[e] = __byte_perm(__float_as_uint(u0), __float_as_uint(u1), 0x7632);
                    }
                    uint16_t *y = static_cast<uint16_t *>(Y) + (size_t)p * ldy + j0;
                    if (nv == 16) {
                        reinterpret_cast<uint4 *>(y)[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        reinterpret_cast<uint4 *>(y)[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; e++)
                            if (2 * e < nv) reinterpret_cast<uint32_t *>(y)[e] = pk[e];
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && s_fail) atomicExch(err, DLIC_ERR_TIMEOUT);
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tm, 2 * kWtN);
    }
}

// Tensor map of a bf16 matrix [rows][cols] with a row pitch of `pitch`
// elements: boxes of 64 columns (128 bytes, swizzled) x box_rows rows,
// zero fill past the extent.  The driver's encoder is looked up through the
// runtime, so the library loads on machines without a CUDA driver.
static CUresult wide_map(CUtensorMap *map, const void *g, int rows, int cols, int pitch, int box_rows) {
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    if (!enc) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return CUDA_ERROR_NOT_FOUND;
        enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
    cuuint32_t box[2] = {(cuuint32_t)kWtKB, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(g), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

template <int TN>
static cudaError_t launch_tn(const DevLayer &ly, const uint16_t *X, int ldx, int np, void *Y, int ldy, bool logits,
                             int num_sms, int *err, cudaStream_t st) {
    CUtensorMap mx, mw;
    if (wide_map(&mx, X, np, ly.n_in, ldx, kWtM) != CUDA_SUCCESS ||
        wide_map(&mw, ly.wtc, ly.n_out, ly.n_in, ly.wtc_pitch, TN) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)WtShape<TN>::kStages * WtShape<TN>::kStageBytes + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_wide_tc<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int tiles = ((np + kWtM - 1) / kWtM) * ((ly.n_out + TN - 1) / TN);
    k_wide_tc<TN><<<std::min(tiles, std::max(1, num_sms)), kWtThreads, smem, st>>>(mx, mw, ly.n_in, ly.n_out, np, ly.a,
                                                                                    ly.o, Y, ldy, logits ? 1 : 0, err);
    return cudaGetLastError();
}

// One layer of a pass: X bf16 [np][ldx], the layer's bf16 weights
// [n_out][wtc_pitch]; one persistent CTA per SM (or per tile, if fewer).
// Tiles are 256 units wide unless that leaves more than half the SMs
// without a tile (the 256 logits of a pass, say).
cudaError_t launch_wide_tc(const DevLayer &ly, const uint16_t *X, int ldx, int np, void *Y, int ldy, bool logits,
                           int num_sms, int *err, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    const int wide_tiles = ((np + kWtM - 1) / kWtM) * ((ly.n_out + 255) / 256);
    return 2 * wide_tiles >= num_sms ? launch_tn<256>(ly, X, ldx, np, Y, ldy, logits, num_sms, err, st)
                                     : launch_tn<128>(ly, X, ldx, np, Y, ldy, logits, num_sms, err, st);
}

}  // namespace dlic
