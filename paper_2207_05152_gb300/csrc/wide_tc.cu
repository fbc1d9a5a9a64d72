// INT8 dense layers of the wide networks on the tensor cores (encode).
//
// Sec. II-B ("Neural Network Architecture") allows hidden layers of up to
// 4096 neurons; a 4096 x 4096 layer is 16.8M multiply-adds per pixel, a
// dense contraction over all the pixels of a pass.  The INT8 layer's sum
// acc_j = sum_k x_k q_jk (x_k in [0, 255] the previous layer's units, q_jk
// in [-127, 127]) is an exact integer.  tcgen05 has no integer MMA on this
// GPU, so the sum runs as BF16 MMAs with FP32 accumulation, kept exact:
//   x = 16 xh + xl with xh, xl in [0, 15], both exact in bf16,
//   acc_h = sum_k xh_k q_jk,  acc_l = sum_k xl_k q_jk,
// each partial sum an integer of magnitude at most K * 15 * 127 < 2^23 for
// K <= 4096, so every FP32 addition is exact in any order, and
//   acc = 16 acc_h + acc_l   (integer arithmetic).
// The epilogue then applies the layer's requantisation (hidden units: the
// next layer's xh and xl planes) or its logit map (output layer), exactly as
// the CUDA-core kernels do, so the bitstreams do not change.
//
// One CTA per 128-pixel x 256-unit tile: warp 0 issues the TMA loads of the
// two activation planes and the weight rows (128-byte swizzle, K blocks of
// 64) through a ring of stages, warp 1 issues the MMAs (two accumulators of
// 256 tensor-memory columns), warps 2..9 read the accumulators back.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "coder_device.cuh"
#include "tc.cuh"

namespace dlic {

constexpr int kWtThreads = 320;
constexpr int kWtEpi = 256;
constexpr int kWtStages = 3;
constexpr int kWtM = 128, kWtN = 256, kWtKB = 64;
constexpr uint32_t kWtPlaneBytes = kWtM * kWtKB * 2;   // 16 KB: one activation plane's K block
constexpr uint32_t kWtWBytes = kWtN * kWtKB * 2;       // 32 KB: the tile's weight rows, one K block
constexpr uint32_t kWtStageBytes = 2 * kWtPlaneBytes + kWtWBytes;
constexpr long long kWtWaitLimit = 4000000000LL;

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

// Y = layer(X) for np pixels: X as two bf16 planes (xh at mapXh, xl at
// mapXl: [np][K]), W bf16 [N][K] at mapW.  Hidden layer (logits == 0):
// u = requant(acc) goes to the output planes Y[p][j] = bf16(u >> 4) and
// Y[plane + p * ldy + j] = bf16(u & 15).  Output layer: Y[p * ldy + j] =
// fma(float(acc), s_j, o_j) (FP32).
__global__ void __launch_bounds__(kWtThreads, 1)
    k_wide_tc(const __grid_constant__ CUtensorMap mapXh, const __grid_constant__ CUtensorMap mapXl,
              const __grid_constant__ CUtensorMap mapW, int K, int N, int np, const float *__restrict__ s,
              const float *__restrict__ o, void *Y, int ldy, size_t plane, int logits, int *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[kWtStages], empty[kWtStages], tfull;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    __shared__ float s_s[kWtN], s_o[kWtN];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kWtM, n0 = blockIdx.y * kWtN;
    const int nkb = (K + kWtKB - 1) / kWtKB;

    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 2 * kWtN);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < kWtStages; q++) {
            tc::mbar_init(&full[q], 1);
            tc::mbar_init(&empty[q], 1);
        }
        tc::mbar_init(&tfull, 1);
        tc::fence_mbar_init();
        s_fail = 0;
    }
    for (int j = tid; j < kWtN; j += kWtThreads) {
        const bool in = n0 + j < N;
        s_s[j] = in ? s[n0 + j] : 0.0f;
        s_o[j] = in ? o[n0 + j] : 0.0f;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = tmem_base;

    if (warp == 0 && lane == 0) {
        // producer: the K blocks through the stages (boxes reaching past the
        // tensor's extent are zero-filled and still deliver their full size)
        for (int i = 0; i < nkb; i++) {
            const int q = i % kWtStages;
            if (!tc::mbar_wait(&empty[q], ((i / kWtStages) & 1) ^ 1, kWtWaitLimit)) {
                s_fail = 1;
                break;
            }
            uint8_t *st = smem + q * kWtStageBytes;
            const uint32_t bar = tc::smem_addr(&full[q]);
            wt_expect_tx(&full[q], kWtStageBytes);
            wt_tma_load(tc::smem_addr(st), &mapXh, i * kWtKB, m0, bar);
            wt_tma_load(tc::smem_addr(st + kWtPlaneBytes), &mapXl, i * kWtKB, m0, bar);
            wt_tma_load(tc::smem_addr(st + 2 * kWtPlaneBytes), &mapW, i * kWtKB, n0, bar);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: acc_h in columns [0, 256), acc_l in [256, 512)
        const uint32_t idesc = tc::idesc_bf16_f32(kWtM, kWtN);
        for (int i = 0; i < nkb; i++) {
            const int q = i % kWtStages;
            if (!tc::mbar_wait(&full[q], (i / kWtStages) & 1, kWtWaitLimit)) {
                s_fail = 1;
                break;
            }
            tc::fence_after_sync();
            const uint32_t st = tc::smem_addr(smem + q * kWtStageBytes);
            const uint64_t dh = desc_sw128(st), dl = desc_sw128(st + kWtPlaneBytes),
                           dw = desc_sw128(st + 2 * kWtPlaneBytes);
#pragma unroll
            for (int ks = 0; ks < kWtKB / 16; ks++) {
                tc::mma_bf16(tm, dh + 2u * ks, dw + 2u * ks, idesc, (i | ks) != 0);
                tc::mma_bf16(tm + kWtN, dl + 2u * ks, dw + 2u * ks, idesc, (i | ks) != 0);
            }
            tc::mma_commit(&empty[q]);
        }
        tc::mma_commit(&tfull);
    } else if (warp >= 2) {
        // epilogue: warp w reads lanes 32 (w mod 4) .. + 31 (one pixel per
        // thread); the two warps of a lane quarter split the 256 columns
        if (lane == 0 && !*reinterpret_cast<volatile int *>(&s_fail) && !tc::mbar_wait(&tfull, 0, kWtWaitLimit))
            s_fail = 1;
        __syncwarp();
        if (!*reinterpret_cast<volatile int *>(&s_fail)) tc::mbar_wait(&tfull, 0, 1000);   // every lane sees the phase
        tc::fence_after_sync();
        // (warp-uniform: the accumulator loads below are warp-collective)
        const bool ok = __shfl_sync(0xffffffffu, *reinterpret_cast<volatile int *>(&s_fail) == 0 ? 1 : 0, 0) != 0;
        const int qd = warp & 3, hf = (warp - 2) >> 2;
        const int row = 32 * qd + lane, p = m0 + row;
        const uint32_t taddr = tm + ((uint32_t)(32 * qd) << 16);
        const int c_lo = hf * (kWtN / 2), c_hi = min(c_lo + kWtN / 2, N - n0);
        for (int c0 = c_lo; ok && c0 < c_hi; c0 += 16) {
            uint32_t vh[16], vl[16];
            tc::tmem_ld16(taddr + (uint32_t)c0, vh);
            tc::tmem_ld16(taddr + (uint32_t)(kWtN + c0), vl);
            tc::tmem_wait_ld();
            if (p >= np) continue;
            int acc[16];
#pragma unroll
            for (int e = 0; e < 16; e++)
                acc[e] = 16 * __float2int_rn(__uint_as_float(vh[e])) + __float2int_rn(__uint_as_float(vl[e]));
            const int nv = min(16, c_hi - c0);   // N is a multiple of 4
            if (logits) {
                float *z = static_cast<float *>(Y) + (size_t)p * ldy + n0 + c0;
                if (nv == 16) {
#pragma unroll
                    for (int e = 0; e < 16; e += 4)
                        *reinterpret_cast<float4 *>(z + e) =
                            make_float4(__fmaf_rn(__int2float_rn(acc[e]), s_s[c0 + e], s_o[c0 + e]),
                                        __fmaf_rn(__int2float_rn(acc[e + 1]), s_s[c0 + e + 1], s_o[c0 + e + 1]),
                                        __fmaf_rn(__int2float_rn(acc[e + 2]), s_s[c0 + e + 2], s_o[c0 + e + 2]),
                                        __fmaf_rn(__int2float_rn(acc[e + 3]), s_s[c0 + e + 3], s_o[c0 + e + 3]));
                } else {
#pragma unroll
                    for (int e = 0; e < 16; e++)
                        if (e < nv) z[e] = __fmaf_rn(__int2float_rn(acc[e]), s_s[c0 + e], s_o[c0 + e]);
                }
            } else {
                uint32_t hi[8], lo[8];
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    const uint32_t u0 = requant_u8(acc[2 * e], s_s[c0 + 2 * e], s_o[c0 + 2 * e]);
                    const uint32_t u1 = requant_u8(acc[2 * e + 1], s_s[c0 + 2 * e + 1], s_o[c0 + 2 * e + 1]);
                    hi[e] = (uint32_t)tc::bf16_of_int((int)(u0 >> 4)) | ((uint32_t)tc::bf16_of_int((int)(u1 >> 4)) << 16);
                    lo[e] = (uint32_t)tc::bf16_of_int((int)(u0 & 15u)) | ((uint32_t)tc::bf16_of_int((int)(u1 & 15u)) << 16);
                }
                uint16_t *yh = static_cast<uint16_t *>(Y) + (size_t)p * ldy + n0 + c0, *yl = yh + plane;
                if (nv == 16) {
                    reinterpret_cast<uint4 *>(yh)[0] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    reinterpret_cast<uint4 *>(yh)[1] = make_uint4(hi[4], hi[5], hi[6], hi[7]);
                    reinterpret_cast<uint4 *>(yl)[0] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                    reinterpret_cast<uint4 *>(yl)[1] = make_uint4(lo[4], lo[5], lo[6], lo[7]);
                } else {
#pragma unroll
                    for (int e = 0; e < 8; e++)
                        if (2 * e < nv) {
                            reinterpret_cast<uint32_t *>(yh)[e] = hi[e];
                            reinterpret_cast<uint32_t *>(yl)[e] = lo[e];
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

// One layer of a pass: X planes [np][ldx] (the low plane plane_in elements
// after the high one), the layer's bf16 weights [n_out][wtc_pitch].
cudaError_t launch_wide_tc(const DevLayer &ly, const uint16_t *X, int ldx, size_t plane_in, int np, void *Y,
                           int ldy, size_t plane_out, bool logits, int *err, cudaStream_t st) {
    CUtensorMap mh, ml, mw;
    if (wide_map(&mh, X, np, ly.n_in, ldx, kWtM) != CUDA_SUCCESS ||
        wide_map(&ml, X + plane_in, np, ly.n_in, ldx, kWtM) != CUDA_SUCCESS ||
        wide_map(&mw, ly.wtc, ly.n_out, ly.n_in, ly.wtc_pitch, kWtN) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)kWtStages * kWtStageBytes + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_wide_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((np + kWtM - 1) / kWtM, (ly.n_out + kWtN - 1) / kWtN);
    k_wide_tc<<<grid, kWtThreads, smem, st>>>(mh, ml, mw, ly.n_in, ly.n_out, np, ly.a, ly.o, Y, ldy, plane_out,
                                               logits ? 1 : 0, err);
    return cudaGetLastError();
}

}  // namespace dlic
