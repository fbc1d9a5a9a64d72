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
//   2. runs the first layer (12 inputs) on the CUDA cores with dp4a, and
//      the two wide layers as tcgen05 MMAs with the weights as the A
//      operand (M = 128 units) and the wave's pixels as the B operand
//      (N = pixels, padded to 16), so a handful of pixels still fills the
//      M dimension; FP32 accumulators in tensor memory are exact integers,
//   3. turns the 256 logits of each pixel into its frequency table with one
//      warp per pixel (warp max, prefix sum, ballot search) and performs the
//      rANS decoding step of the pixel's stream,
//   4. writes the decoded pixel to the image and, through distributed shared
//      memory, to the ring buffers of the CTAs that read it,
// then, unless neighbour-to-neighbour rings are in use, the cluster
// synchronises once before the next wave.
#include "coder_device.cuh"
#include "tc.cuh"

namespace dlic {

constexpr int kDecThreads = 512;
constexpr int kDecWarps = kDecThreads / 32;
constexpr int kDecHidden = 128;
constexpr long long kDecWaitLimit = 4000000000LL;
// The INT8 network's two wide layers (128 x 128 and 256 x 128 against a
// chunk of pixels per wave) run either as tcgen05 MMAs (weights = A, the
// chunk's pixels = B, accumulators in tensor memory) or, for chunks of up to
// kSmmaMaxChunk pixels, as warp-level bf16 MMAs (mma.sync m16n8k16 with FP32
// accumulation, exact for these integer-valued operands: every partial sum
// is an integer below 2^23): a few tens of cycles per MMA with the
// accumulators in registers, against a tcgen05 round trip (issue, commit,
// mbarrier, tensor-memory load) of 0.7-1.0K cycles per layer; past about 32
// pixels the warp MMAs' rate (about 0.32 per cycle per SM) loses to the
// tensor core.  The warp MMAs' operands sit row-major in shared memory with
// rows of kActPitch bf16, so that every fragment load is free of bank
// conflicts.
constexpr int kSmmaMaxChunk = 32;
constexpr int kActPitch = kDecHidden + 8;
// Row pitch (floats) of the INT8 decoder's logits: the layer-3 fragments'
// stores (four pixels x eight units per instruction) fall in distinct banks.
constexpr int kZPitch = kSymbols + 4;

struct DecTcLayout {
    // INT8 network: bf16 operand tiles, s8 priors, bf16 activations
    uint32_t w1, w2, w3, pri, b23, shid;
    // FP32 network: W1^T | b1 | b2 | b3, W2^T, the W3^T staging ring, FP32
    // inputs and activations (the logits z overlay xs and h1t)
    uint32_t wf, w2f, w3s, xs, h1t, h2t;
    uint32_t z, ring, tring, rows, pg, dsym, lut, st_x, st_pos, st_end, pay, zpre, total;
};

struct DecTcParams {
    int P;            // CTAs per image (cluster size)
    int h1, h2;       // hidden widths (FP32 network)
    int nt;           // pixels per chunk (multiple of 16, <= 128)
    int ring_rows;    // byte-ring rows (power of two); 0 with gimg
    int list_rows;    // capacity of the per-wave row list and decoded-pixel buffer
    int tq;           // tagged ring: row rounds kept (power of two)
    int max_g;        // owned streams per CTA (upper bound)
    int pay_words;    // staged payload capacity per CTA (words); 0 = read from global
    int k1;           // network inputs per pixel: the window's priors padded to 16
    int tslots;       // tagged-ring slots per row round: one per row distance 0..rows above
    int tcols;        // tagged-ring columns kept per row (power of two)
    int rcols;        // byte-ring columns kept per row (power of two)
    int gimg;         // 1: priors are read back from the output image (no ring; one
                      // cluster barrier per wave), for waves too long for the rings
    int depth;        // slices per image (volumes); stream states are kept per slice
    int zlist;        // grid decoder: capacity of the per-wave table of active slices (and,
                      // for a batch, of the per-image stream count, flags and wave count)
    int T;            // grid decoder of a batch: waves of the longest image
    int lut2;         // 1: the table's powers of two expanded to kTableSteps entries
    int smma;         // INT8: 1 = the wide layers as warp-level MMAs, 0 = tcgen05
    int deep;         // INT8 networks of 1..5 hidden layers of widths up to 128 from the
                      // layer table (warp-level MMAs, every layer zero-padded to 128 units)
    int nhh;          // deep: hidden-to-hidden layers (the hidden layers less one)
};

// FP32 network parameters kept in shared memory (floats): W1^T [12][h1],
// b1, b2, b3, then W2^T [h1][h2].  W3^T [h2][256] streams through a ring of
// kW3Stages buffers of kW3Rows rows, refilled by bulk copies from L2.
constexpr int kW3Rows = 16, kW3Stages = 5;
__host__ __device__ inline uint32_t dec_f32_weight_floats(int n_in, int h1, int h2) {
    return (uint32_t)(n_in * h1 + h1 + h2 + kSymbols);
}

// Shared-memory plan of a CTA: chunks of up to nt pixels, the byte ring
// (ring_rows x rcols), the tagged ring (tq rounds x tslots x tcols words),
// the wave's row list, max_g owned streams and pay_words staged payload
// words, for the INT8 tensor-core network or (f32) the FP32 network of
// widths h1, h2.
__host__ __device__ inline DecTcLayout dec_layout(const DecTcParams &prm, bool f32) {
    const int nt = prm.nt, rows = prm.ring_rows, g = prm.max_g, pay_words = prm.pay_words, h1 = prm.h1, h2 = prm.h2;
    DecTcLayout L{};
    uint32_t off = 0;
    auto take = [&](uint32_t bytes) {
        const uint32_t o = off;
        off += (bytes + 127u) & ~127u;
        return o;
    };
    if (f32) {
        L.wf = take(4u * dec_f32_weight_floats(prm.k1, h1, h2));
        L.w2f = take(4u * h1 * h2);
        L.w3s = take(4u * kW3Stages * kW3Rows * kSymbols);
        // xs, then h1t [unit][nt + 4] (conflict-free float4 rows); z
        // overlays both once the second layer has consumed them
        const uint32_t xs_bytes = 4u * prm.k1 * nt, h1t_bytes = 4u * h1 * (nt + 4), z_bytes = 4u * nt * kSymbols;
        const uint32_t region = xs_bytes + h1t_bytes > z_bytes ? xs_bytes + h1t_bytes : z_bytes;
        const uint32_t base = take(region);
        L.xs = base;
        L.h1t = base + xs_bytes;
        L.z = base;
        L.h2t = take(4u * h2 * (nt + 4));
    } else if (prm.smma && prm.deep) {
        // deep: W1 words, nhh hidden-to-hidden layers [unit][k] bf16 with their
        // scales and offsets; the output layer's weights live in registers
        L.w1 = take((uint32_t)prm.k1 * kDecHidden);
        L.w2 = take(2u * kDecHidden * kActPitch * (uint32_t)prm.nhh);
        L.shid = take(4u * 2u * kDecHidden * (uint32_t)prm.nhh);
        L.pri = take((uint32_t)prm.k1 * nt);
        L.b23 = take(2u * 2u * nt * kActPitch);
    } else if (prm.smma) {
        L.w1 = take((uint32_t)prm.k1 * kDecHidden);   // W1 as s8 words [k1 / 4][128] (the first layer runs as dp4a)
        L.w2 = take(2u * kDecHidden * kActPitch);     // W2 [unit][k], bf16
        L.w3 = take(2u * kSymbols * kActPitch);       // W3 [unit][k], bf16
        L.pri = take((uint32_t)prm.k1 * nt);
        L.b23 = take(2u * 2u * nt * kActPitch);       // the two hidden layers' outputs [pixel][unit], bf16
    } else {
        L.w1 = take((uint32_t)prm.k1 * kDecHidden);   // W1 as s8 words [k1 / 4][128] (the first layer runs as dp4a)
        L.w2 = take(2u * kDecHidden * kDecHidden);
        L.w3 = take(512u * kDecHidden);
        L.pri = take((uint32_t)prm.k1 * nt);
        L.b23 = take(2u * nt * kDecHidden);
    }
    // warp-level MMAs: the logits overlay the W3 rows, which are read into
    // registers before the first wave (4 nt 260 <= 2 x 256 x 136 for nt <= 64)
    if (!f32) L.z = prm.smma && !prm.deep ? L.w3 : take(4u * nt * (prm.smma ? kZPitch : kSymbols));
    L.ring = take(prm.gimg ? 0u : (uint32_t)prm.rcols * rows);
    L.tring = take(prm.gimg ? 0u : 4u * prm.tcols * prm.tslots * prm.tq);
    L.rows = take(4u * prm.list_rows);
    L.pg = take(4u * nt);
    L.zpre = take(4u * prm.zlist);
    L.dsym = take(prm.gimg ? 0u : (uint32_t)prm.list_rows);   // decoded pixels held back until the barrier
    L.lut = take(prm.lut2 ? 4u * kTableSteps : 4u * 64);
    L.st_x = take(4u * g * prm.depth);
    L.st_pos = take(4u * g * prm.depth);
    L.st_end = take(4u * g * prm.depth);
    L.pay = take(2u * pay_words);
    L.total = off;
    return L;
}


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
__device__ __forceinline__ void st_cluster_u32(uint32_t addr, uint32_t v) {
    asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_gpu_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}


__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.volatile.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(tc::smem_addr(p)) : "memory");
    return v;
}

// Tagged ring entry of pixel (r, c) with value v: a valid bit, 11 bits of the
// row and 12 of the column, then the pixel.  A reader knows which (r, c) it
// wants, so a single 32-bit store both delivers the value and says that it
// has arrived: no fence or barrier is needed between CTAs.
__device__ __forceinline__ uint32_t ring_tag(int r, int c) {
    return 0x80000000u | ((uint32_t)(r & 0x7FF) << 20) | ((uint32_t)(c & 0xFFF) << 8);
}

// floor(65280 * 2^32 / W) for 2^23 <= W <= 2^31, exactly.  A reciprocal
// estimate gives q within a few units of the quotient (q < 2^25); one
// correction step from the exact 64-bit remainder, then a final +-1 fix-up,
// lands on the floor.
__device__ __forceinline__ uint32_t table_q_fast(uint32_t W) {
    const long long num = 65280LL << 32;
    float rw;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rw) : "f"(__uint2float_rn(W)));
    long long q = (long long)__float2uint_rz(__fmul_rz(280375465082880.0f, rw));
    long long rem = num - q * (long long)W;
    q += (long long)__float2int_rz(__fmul_rz(__ll2float_rn(rem), rw));
    rem = num - q * (long long)W;
#pragma unroll 1
    for (int k = 0; k < 4 && rem < 0; k++) {
        q -= 1;
        rem += W;
    }
#pragma unroll 1
    for (int k = 0; k < 4 && rem >= (long long)W; k++) {
        q += 1;
        rem -= W;
    }
    return (uint32_t)q;
}

// r mod S for 0 <= r < 2^24, 1 <= S <= 65535: a single-precision quotient
// estimate (off by at most one) and an exact correction.
__device__ __forceinline__ int fast_mod(int r, int S, float invS) {
    int q = __float2int_rz(__fmul_rz(__int2float_rn(r), invS));
    int m = r - q * S;
    if (m < 0) m += S;
    if (m >= S) m -= S;
    return m;
}

// 8 consecutive 32-bit tensor-memory columns of this thread's lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr)
                 : "memory");
}


// FP32 network helpers of the wavefront decoder.  Activations are stored
// [unit][pitch PT] so that a k row of consecutive pixels is one broadcast
// load.  Each unit starts from its bias and accumulates fma(x_k, w_jk, acc)
// for k ascending, the order the encoder uses.

// The logits phase: thread = (2 units, 4 pixels) over `groups` pixel
// groups; the threads consume w3_chunks staging loads in sequence (rows
// k0 .. k0 + rows - 1 of W3^T each, k ascending) with the accumulators in
// registers, and after each chunk every thread synchronises and thread 0
// refills the buffer just read with the load kW3Stages further on.
template <class Issue>
__device__ __forceinline__ void f32_logits(int tid, int groups, int w3_chunks, int &w3_seq, Issue &w3_issue, int h2,
                                           const float *b3s, const float *h2t, int PT, const uint8_t *w3buf,
                                           uint64_t *w3bar, float *zb, int &s_fail, int &s_cfail) {
    const bool l3 = tid < (kSymbols / 2) * groups;   // at most 128 x 3 < kDecThreads
    const int up = tid % (kSymbols / 2), p0 = 4 * (tid / (kSymbols / 2));
    float a[2][4];
    if (l3) {
        const float2 bb = *reinterpret_cast<const float2 *>(b3s + 2 * up);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            a[0][j] = bb.x;
            a[1][j] = bb.y;
        }
    }
    for (int c = 0; c < w3_chunks; c++, w3_seq++) {
        const int stg = w3_seq % kW3Stages;
        const int rows = min(kW3Rows, h2 - c * kW3Rows);
        if (l3) {
            // every issued copy is waited for, also after a peer wait ran
            // out (a copy from L2 always lands); only a copy that did not
            // land stops the waits and the refills
            if (!*reinterpret_cast<volatile int *>(&s_cfail) &&
                !tc::mbar_wait(&w3bar[stg], (uint32_t)(w3_seq / kW3Stages) & 1u, kDecWaitLimit)) {
                s_cfail = 1;
                s_fail = 1;
            }
            const float *w3c = reinterpret_cast<const float *>(w3buf) + stg * kW3Rows * kSymbols;
#pragma unroll 4
            for (int kr = 0; kr < rows; kr++) {
                const float2 w = *reinterpret_cast<const float2 *>(w3c + kr * kSymbols + 2 * up);
                const float4 x = *reinterpret_cast<const float4 *>(h2t + (c * kW3Rows + kr) * PT + p0);
                a[0][0] = __fmaf_rn(x.x, w.x, a[0][0]);
                a[0][1] = __fmaf_rn(x.y, w.x, a[0][1]);
                a[0][2] = __fmaf_rn(x.z, w.x, a[0][2]);
                a[0][3] = __fmaf_rn(x.w, w.x, a[0][3]);
                a[1][0] = __fmaf_rn(x.x, w.y, a[1][0]);
                a[1][1] = __fmaf_rn(x.y, w.y, a[1][1]);
                a[1][2] = __fmaf_rn(x.z, w.y, a[1][2]);
                a[1][3] = __fmaf_rn(x.w, w.y, a[1][3]);
            }
        }
        __syncthreads();   // every reader is done with this buffer
        if (tid == 0 && !s_cfail) w3_issue(w3_seq + kW3Stages);
    }
    if (l3) {
#pragma unroll
        for (int j = 0; j < 4; j++)
            *reinterpret_cast<float2 *>(zb + (p0 + j) * kSymbols + 2 * up) = make_float2(a[0][j], a[1][j]);
    }
}

// Grid decoder of a volume, before the wave kernel: walks the slices'
// containers (back to back; each header checked against the model and the
// volume), and writes every stream's initial state, read position and end
// to the volume's state block.  One CTA.
__global__ void __launch_bounds__(kDecThreads) k_volume_setup(DevModel m, DecBatch b) {
    __shared__ uint32_t s_part[kDecThreads];
    __shared__ int s_ok;
    __shared__ uint64_t s_next;
    const int tid = threadIdx.x;
    const DecImage &im = b.img[0];
    const uint8_t *in = b.in + im.in_off;
    const VolState vs = vol_state(b, im);
    const int S = im.S, H = im.H, W = im.W;
    if (tid == 0) {
        s_ok = 1;
        s_next = 0;
        vs.hdr[0] = (uint32_t)S;
        vs.hdr[2] = 0u;   // wave-barrier arrivals
        vs.hdr[3] = 0u;   // a wait ran out
    }
    __syncthreads();
    for (int z = 0; z < im.D; z++) {
        const uint64_t off = s_next;
        const uint8_t *sin = in + off;
        if (tid == 0) {
            int ok = im.in_bytes >= off + (uint64_t)kHeaderBytes;
            if (ok) {
                uint64_t hash = 0;
                for (int q = 0; q < 8; q++) hash |= (uint64_t)sin[16 + q] << (8 * q);
                const uint32_t hh = sin[4] | (sin[5] << 8) | (sin[6] << 16) | ((uint32_t)sin[7] << 24);
                const uint32_t ww = sin[8] | (sin[9] << 8) | (sin[10] << 16) | ((uint32_t)sin[11] << 24);
                ok = sin[0] == 'D' && sin[1] == 'L' && sin[2] == 'C' && sin[3] == '1' && hh == (uint32_t)H &&
                     ww == (uint32_t)W && sin[12] == (m.wu | 0x80) && sin[13] == m.precision && hash == m.hash &&
                     (sin[14] | (sin[15] << 8)) == S && im.in_bytes >= off + (uint64_t)kHeaderBytes + 4ull * S;
            }
            if (!ok) s_ok = 0;
        }
        __syncthreads();
        if (!s_ok) break;
        const uint8_t *cnt = sin + kHeaderBytes;
        const uint16_t *pay = reinterpret_cast<const uint16_t *>(sin + kHeaderBytes + 4 * S);
        const int per = (S + kDecThreads - 1) / kDecThreads;
        const int s0 = min(S, tid * per), s1 = min(S, s0 + per);
        // 64-bit sums, each bounded by the input's word count (below 2^32,
        // checked on the host), so the 32-bit prefix sums are exact
        uint64_t sum = 0;
        int bad = 0;
        for (int s = s0; s < s1; s++) {
            const uint32_t c = cnt[4 * s] | (cnt[4 * s + 1] << 8) | (cnt[4 * s + 2] << 16) | ((uint32_t)cnt[4 * s + 3] << 24);
            bad |= c < 2;
            sum += c;
        }
        bad |= sum > im.in_bytes / 2;
        s_part[tid] = (uint32_t)sum;
        if (bad) s_ok = 0;
        __syncthreads();
        if (tid == 0) {
            uint64_t acc = 0;
            for (int q = 0; q < kDecThreads; q++) {
                const uint32_t v = s_part[q];
                s_part[q] = (uint32_t)acc;
                acc += v;
            }
            const uint64_t next = off + (uint64_t)kHeaderBytes + 4ull * S + 2ull * acc;
            if (z == im.D - 1 ? next != im.in_bytes : next > im.in_bytes) s_ok = 0;
            s_next = next;
        }
        __syncthreads();
        if (s_ok) {
            // positions count 16-bit words from the start of the volume
            const uint32_t word0 = (uint32_t)((off + kHeaderBytes + 4ull * S) / 2);
            uint32_t start = s_part[tid];
            for (int s = s0; s < s1; s++) {
                const uint32_t c = cnt[4 * s] | (cnt[4 * s + 1] << 8) | (cnt[4 * s + 2] << 16) | ((uint32_t)cnt[4 * s + 3] << 24);
                const size_t g = (size_t)z * S + s;
                const uint32_t x = ((uint32_t)pay[start] << 16) | pay[start + 1];
                if (x < kRansL) s_ok = 0;
                vs.x[g] = x;
                vs.pos[g] = word0 + start + 2;
                vs.end[g] = word0 + start + c;
                start += c;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        vs.hdr[1] = (uint32_t)s_ok;
        if (!s_ok) atomicMax(b.status + im.sidx, (int)DLIC_ERR_CORRUPT);
    }
}

// Grid decoder of a volume, after the wave kernel: every stream must be back
// at the initial state with every word read.  One CTA.
__global__ void __launch_bounds__(kDecThreads) k_volume_finish(DecBatch b) {
    const DecImage &im = b.img[0];
    const VolState vs = vol_state(b, im);
    if (!vs.hdr[1]) return;   // the setup found a bad header (already reported)
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    const size_t n = (size_t)im.D * im.S;
    for (size_t g = threadIdx.x; g < n; g += kDecThreads)
        if (vs.x[g] != kRansL || vs.pos[g] != vs.end[g]) s_bad = 1;
    __syncthreads();
    if (threadIdx.x == 0 && (s_bad || vs.hdr[3]))
        atomicMax(b.status + im.sidx, vs.hdr[3] ? (int)DLIC_ERR_TIMEOUT : (int)DLIC_ERR_CORRUPT);
}

// Grid decoder of a batch of 2D images, before the wave kernel: CTA i
// checks image i's header and writes its streams' states to the image's
// state block (positions count 16-bit words from the start of the input
// buffer), with the stream count and whether no wave holds two rows of one
// stream ("spread"; the other images go whole to one CTA per wave).  The
// state block of image 0 also carries the grid's wave-barrier counter.
__global__ void __launch_bounds__(kDecThreads) k_batch_setup(DevModel m, DecBatch b) {
    __shared__ uint32_t s_part[kDecThreads];
    __shared__ int s_ok, s_S;
    const int tid = threadIdx.x;
    const DecImage &im = b.img[blockIdx.x];
    const uint8_t *in = b.in + im.in_off;
    const VolState vs = vol_state(b, im);
    const int H = im.H, W = im.W;
    if (tid == 0) {
        int ok = im.in_bytes >= (uint64_t)kHeaderBytes, S = 0;
        if (ok) {
            uint64_t hash = 0;
            for (int q = 0; q < 8; q++) hash |= (uint64_t)in[16 + q] << (8 * q);
            S = in[14] | (in[15] << 8);
            const uint32_t hh = in[4] | (in[5] << 8) | (in[6] << 16) | ((uint32_t)in[7] << 24);
            const uint32_t ww = in[8] | (in[9] << 8) | (in[10] << 16) | ((uint32_t)in[11] << 24);
            ok = in[0] == 'D' && in[1] == 'L' && in[2] == 'C' && in[3] == '1' && hh == (uint32_t)H &&
                 ww == (uint32_t)W && in[12] == m.wu && in[13] == m.precision && hash == m.hash && S >= 1 &&
                 S <= H && im.in_bytes >= (uint64_t)kHeaderBytes + 4ull * S;
        }
        s_ok = ok;
        s_S = ok ? S : 1;
        if (blockIdx.x == 0) {
            vs.hdr[2] = 0u;   // wave-barrier arrivals
            vs.hdr[3] = 0u;   // a wait ran out
        }
    }
    __syncthreads();
    const int S = s_S;
    if (s_ok) {
        const uint8_t *cnt = in + kHeaderBytes;
        const uint16_t *pay = reinterpret_cast<const uint16_t *>(in + kHeaderBytes + 4 * S);
        const int per = (S + kDecThreads - 1) / kDecThreads;
        const int s0 = min(S, tid * per), s1 = min(S, s0 + per);
        // 64-bit sums, each bounded by the input's word count (below 2^32,
        // checked on the host), so the 32-bit prefix sums are exact
        uint64_t sum = 0;
        int bad = 0;
        for (int s = s0; s < s1; s++) {
            const uint32_t c = cnt[4 * s] | (cnt[4 * s + 1] << 8) | (cnt[4 * s + 2] << 16) | ((uint32_t)cnt[4 * s + 3] << 24);
            bad |= c < 2;
            sum += c;
        }
        bad |= sum > im.in_bytes / 2;
        s_part[tid] = (uint32_t)sum;
        if (bad) s_ok = 0;
        __syncthreads();
        if (tid == 0) {
            uint64_t acc = 0;
            for (int q = 0; q < kDecThreads; q++) {
                const uint32_t v = s_part[q];
                s_part[q] = (uint32_t)acc;
                acc += v;
            }
            if ((uint64_t)kHeaderBytes + 4ull * S + 2ull * acc != im.in_bytes) s_ok = 0;
        }
        __syncthreads();
        if (s_ok) {
            const uint32_t word0 = (uint32_t)((im.in_off + kHeaderBytes + 4ull * S) / 2);
            uint32_t start = s_part[tid];
            for (int s = s0; s < s1; s++) {
                const uint32_t c = cnt[4 * s] | (cnt[4 * s + 1] << 8) | (cnt[4 * s + 2] << 16) | ((uint32_t)cnt[4 * s + 3] << 24);
                const uint32_t x = ((uint32_t)pay[start] << 16) | pay[start + 1];
                if (x < kRansL) s_ok = 0;
                vs.x[s] = x;
                vs.pos[s] = word0 + start + 2;
                vs.end[s] = word0 + start + c;
                start += c;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        vs.hdr[0] = (uint32_t)S;
        vs.hdr[1] = (uint32_t)s_ok;
        vs.hdr[4] = (uint32_t)(min(H, (W + 2) / 3) <= S);
        if (!s_ok) atomicMax(b.status + im.sidx, (int)DLIC_ERR_CORRUPT);
    }
}

// After the grid decoder of a batch: CTA i checks image i's final states.
__global__ void __launch_bounds__(kDecThreads) k_batch_finish(DecBatch b) {
    const DecImage &im = b.img[blockIdx.x];
    const VolState vs = vol_state(b, im);
    const uint32_t failed = vol_state(b, b.img[0]).hdr[3];
    if (!vs.hdr[1]) return;
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    const int S = (int)vs.hdr[0];
    for (int g = threadIdx.x; g < S; g += kDecThreads)
        if (vs.x[g] != kRansL || vs.pos[g] != vs.end[g]) s_bad = 1;
    __syncthreads();
    if (threadIdx.x == 0 && (s_bad || failed))
        atomicMax(b.status + im.sidx, failed ? (int)DLIC_ERR_TIMEOUT : (int)DLIC_ERR_CORRUPT);
}

// The wavefront decoder for one image per cluster; F32 selects the FP32
// network on the CUDA cores instead of the INT8 network on the tensor cores.
// DEF compiles the default window (the 12 priors of Fig. 2: two rows above,
// two columns either side) with its sizes and offsets as constants.  GRID
// decodes one volume with every CTA of a cooperative grid (no cluster):
// each wave's pixels are split evenly over the CTAs, stream states live in
// the workspace and the waves are separated by a grid-wide barrier.
// DEEP (with SMMA, 2D, default window): an INT8 network of 1..5 hidden
// layers of widths up to 128 from the layer table, each layer zero-padded to
// 128 units (a padded unit has zero weights in and out and requantises to 0,
// so the sums are those of the unpadded network).
template <bool F32, bool DEF, bool GRID, bool SMMA, bool DEEP = false>
__device__ __forceinline__ void decode_wave(const DevModel &m, const DecBatch &b, const DecTcParams &prm) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar;
    __shared__ uint64_t w3bar[kW3Stages];   // FP32: W3^T staging buffers filled
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok, s_S, s_err, s_fail, s_cfail;
    __shared__ uint64_t s_next;   // byte offset of the next slice's container

    __shared__ char4 s_woff[kMaxPriors];   // (row, column) offset of every prior of the window
    __shared__ uint32_t s_part[kDecThreads];
    __shared__ uint32_t s_gpart[kDecThreads];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = prm.P, NT = prm.nt;
    const int lgP = __ffs(P) - 1;                 // P is a power of two
    const uint32_t k = P > 1 ? cluster_rank() : 0u;
    const int img_idx = GRID ? 0 : blockIdx.x / P;
    const DecImage &im = b.img[img_idx];
    const uint8_t *in = b.in + im.in_off;
    const int H = im.H, W = im.W;
    const int h1 = prm.h1, h2 = prm.h2;
    // (the layout with this instance's MMA kind as a constant)
    DecTcParams pl = prm;
    pl.smma = SMMA ? 1 : 0;
    pl.deep = DEEP ? 1 : 0;
    const DecTcLayout L = dec_layout(pl, F32);
    const int K1 = DEF ? 16 : prm.k1, NPRI = DEF ? kPriors : m.n_in;
    const int TSLOTS = DEF ? 3 : prm.tslots, TCOLS = DEF ? 32 : prm.tcols, RCOLS = DEF ? 16 : prm.rcols;

    // --- set-up: weights, parameters, tensor memory, header and streams ---
    {
        if constexpr (F32) {
            float *wf = reinterpret_cast<float *>(smem + L.wf);
            for (int i = tid; i < NPRI * h1; i += kDecThreads) wf[i] = m.w1t[i];
            for (int i = tid; i < h1; i += kDecThreads) wf[NPRI * h1 + i] = m.b1[i];
            for (int i = tid; i < h2; i += kDecThreads) wf[NPRI * h1 + h1 + i] = m.b2[i];
            for (int i = tid; i < kSymbols; i += kDecThreads) wf[NPRI * h1 + h1 + h2 + i] = m.b3[i];
            for (int i = tid; i < h1 * h2 / 4; i += kDecThreads)
                reinterpret_cast<float4 *>(smem + L.w2f)[i] = __ldg(reinterpret_cast<const float4 *>(m.w2t) + i);
        } else if (DEEP) {
            // the hidden-to-hidden layers as bf16 rows [unit][k] (128 x 128,
            // zero-padded) from their packed s8 words [k / 4][n_out], with
            // their scales and offsets (0 for padded units); W1 as s8 words
            // [k1 / 4][128]
            uint16_t *w2s = reinterpret_cast<uint16_t *>(smem + L.w2);
            float *sh = reinterpret_cast<float *>(smem + L.shid);
            for (int l = 0; l < prm.nhh; l++) {
                const DevLayer ly = m.layers[1 + l];
                const uint32_t *q = static_cast<const uint32_t *>(ly.w);
                const int k4n = (ly.n_in + 3) / 4;
                for (int i = tid; i < (kDecHidden / 4) * kDecHidden; i += kDecThreads) {
                    const int j = i % kDecHidden, k4 = i / kDecHidden;
                    const uint32_t v = j < ly.n_out && k4 < k4n ? __ldg(q + k4 * ly.n_out + j) : 0u;
                    uint32_t lo = 0, hi = 0;
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const uint32_t h = tc::bf16_of_int((int)(int8_t)(uint8_t)(v >> (8 * e)));
                        if (e < 2) lo |= h << (16 * e); else hi |= h << (16 * (e - 2));
                    }
                    *reinterpret_cast<uint2 *>(w2s + ((size_t)l * kDecHidden + j) * kActPitch + 4 * k4) = make_uint2(lo, hi);
                }
                for (int j = tid; j < kDecHidden; j += kDecThreads) {
                    sh[(2 * l) * kDecHidden + j] = j < ly.n_out ? ly.a[j] : 0.0f;
                    sh[(2 * l + 1) * kDecHidden + j] = j < ly.n_out ? ly.o[j] : 0.0f;
                }
            }
            const DevLayer l0 = m.layers[0];
            const uint32_t *q0 = static_cast<const uint32_t *>(l0.w);
            uint32_t *w1q = reinterpret_cast<uint32_t *>(smem + L.w1);
            for (int i = tid; i < (K1 / 4) * kDecHidden; i += kDecThreads) {
                const int j = i % kDecHidden, k4 = i / kDecHidden;
                w1q[i] = j < l0.n_out && k4 < (l0.n_in + 3) / 4 ? __ldg(q0 + k4 * l0.n_out + j) : 0u;
            }
        } else if (SMMA) {
            // W2, W3 as bf16 rows [unit][k] from the packed s8 words [k / 4][unit]
            auto unpack = [&](const uint32_t *q, int units, uint16_t *dst) {
                for (int i = tid; i < (kDecHidden / 4) * units; i += kDecThreads) {
                    const int j = i % units, k4 = i / units;
                    const uint32_t v = __ldg(q + i);
                    uint32_t lo = 0, hi = 0;
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const uint32_t h = tc::bf16_of_int((int)(int8_t)(uint8_t)(v >> (8 * e)));
                        if (e < 2) lo |= h << (16 * e); else hi |= h << (16 * (e - 2));
                    }
                    *reinterpret_cast<uint2 *>(dst + (size_t)j * kActPitch + 4 * k4) = make_uint2(lo, hi);
                }
            };
            unpack(m.q2t, kDecHidden, reinterpret_cast<uint16_t *>(smem + L.w2));
            unpack(m.q3t, kSymbols, reinterpret_cast<uint16_t *>(smem + L.w3));
            uint32_t *w1q = reinterpret_cast<uint32_t *>(smem + L.w1);
            for (int i = tid; i < (K1 / 4) * kDecHidden; i += kDecThreads)
                w1q[i] = i < ((NPRI + 3) / 4) * kDecHidden ? __ldg(m.q1t + i) : 0u;
        } else {
            // W2 | W3 of the weight image (after the k1 x 128 bf16 W1 tile)
            const uint4 *src = reinterpret_cast<const uint4 *>(m.tc_w) + 16 * K1;
            uint4 *dst = reinterpret_cast<uint4 *>(smem + L.w2);
            const int n16 = (int)(m.tc_w_bytes / 16) - 16 * K1;
            for (int i = tid; i < n16; i += kDecThreads) dst[i] = __ldg(src + i);
            // W1 as s8 words [k1 / 4][128] for the dp4a first layer
            uint32_t *w1q = reinterpret_cast<uint32_t *>(smem + L.w1);
            for (int i = tid; i < (K1 / 4) * kDecHidden; i += kDecThreads)
                w1q[i] = i < ((NPRI + 3) / 4) * kDecHidden ? __ldg(m.q1t + i) : 0u;
        }
        uint32_t *lut = reinterpret_cast<uint32_t *>(smem + L.lut);
        if (prm.lut2)
            expand_lut(m.lut, lut, tid, kDecThreads);   // lut2[u] = lut[u mod 64] >> (u div 64)
        else if (tid < 64)
            lut[tid] = m.lut[tid];
        if (tid < m.n_in) {
            int dz, dr, dc;
            window_offset(m, tid, dz, dr, dc);
            s_woff[tid] = make_char4((signed char)dr, (signed char)dc, (signed char)dz, 0);
        }
        uint32_t *ring = reinterpret_cast<uint32_t *>(smem + L.ring);
        for (int i = tid; i < prm.ring_rows * prm.rcols / 4; i += kDecThreads) ring[i] = 0u;
        uint32_t *tring = reinterpret_cast<uint32_t *>(smem + L.tring);
        for (int i = tid; i < prm.tq * prm.tslots * prm.tcols; i += kDecThreads) tring[i] = 0u;
    }
    if constexpr (!F32 && !SMMA) {
        if (warp == 0) {
            tc::tmem_alloc(&tmem_base, 256);
            tc::tmem_relinquish();
        }
    }
    if (tid == 0) {
        if constexpr (!F32) {
            if (!SMMA) tc::mbar_init(&bar, 1);
        } else {
            for (int q = 0; q < kW3Stages; q++) tc::mbar_init(&w3bar[q], 1);
        }
        tc::fence_mbar_init();
        s_err = 0;
        s_fail = 0;
        s_cfail = 0;
        s_ok = 1;
        s_S = 0;
        s_next = 0;
    }
    __syncthreads();
    // Headers and streams of every slice: a 2D image is one slice; the
    // slices of a volume (3D window) are back-to-back containers with the
    // same stream count, their stream states kept at z * GS + g.
    const bool vol = !DEF && m.vol != 0;
    const int D = vol ? im.D : 1, GS = prm.max_g;
    uint32_t *st_x = reinterpret_cast<uint32_t *>(smem + L.st_x);
    uint32_t *st_pos = reinterpret_cast<uint32_t *>(smem + L.st_pos);
    uint32_t *st_end = reinterpret_cast<uint32_t *>(smem + L.st_end);
    const uint16_t *wsrc = nullptr;
    // grid decoder of a batch of 2D images: per image its stream count,
    // flags (1: header good, 2: spread) and wave count, after zpre
    const bool gb = GRID && !vol;
    int *itS = reinterpret_cast<int *>(smem + L.zpre) + (b.n + 1);
    int *itflag = itS + (b.n + 1), *itT2 = itflag + (b.n + 1);
    if constexpr (GRID) {
        if (gb) {
            // states written by k_batch_setup; a bad image just has no pixels
            for (int i = tid; i < b.n; i += kDecThreads) {
                const VolState vi = vol_state(b, b.img[i]);
                itS[i] = (int)__ldcg(vi.hdr);
                itflag[i] = (int)(__ldcg(vi.hdr + 1) | (__ldcg(vi.hdr + 4) << 1));
                itT2[i] = 3 * (b.img[i].H - 1) + b.img[i].W;
            }
            if (tid == 0) {
                s_S = 1;
                s_ok = 1;
            }
            wsrc = reinterpret_cast<const uint16_t *>(b.in);
        } else {
            // states written by k_volume_setup; every CTA reads the same flag
            const VolState vs = vol_state(b, im);
            if (tid == 0) {
                s_S = (int)__ldcg(vs.hdr);
                s_ok = (int)__ldcg(vs.hdr + 1);
            }
            st_x = vs.x;
            st_pos = vs.pos;
            st_end = vs.end;
            wsrc = reinterpret_cast<const uint16_t *>(in);
        }
        __syncthreads();
    }
    for (int z = 0; z < (GRID ? 0 : D); z++) {
        const uint64_t slice_off = s_next;
        const uint8_t *sin = in + slice_off;
        if (tid == 0) {
            int ok = s_ok && im.in_bytes >= slice_off + (uint64_t)kHeaderBytes;
            if (ok) {
                uint64_t hash = 0;
                for (int q = 0; q < 8; q++) hash |= (uint64_t)sin[16 + q] << (8 * q);
                const int Sz = sin[14] | (sin[15] << 8);
                const uint32_t hh = sin[4] | (sin[5] << 8) | (sin[6] << 16) | ((uint32_t)sin[7] << 24);
                const uint32_t ww = sin[8] | (sin[9] << 8) | (sin[10] << 16) | ((uint32_t)sin[11] << 24);
                ok = sin[0] == 'D' && sin[1] == 'L' && sin[2] == 'C' && sin[3] == '1' && hh == (uint32_t)H &&
                     ww == (uint32_t)W && sin[12] == (m.wu | (vol ? 0x80 : 0)) && sin[13] == m.precision &&
                     hash == m.hash && Sz >= 1 && Sz <= H && (Sz + P - 1) / P <= prm.max_g &&
                     (z == 0 || Sz == s_S) && (!vol || Sz % P == 0) &&
                     im.in_bytes >= slice_off + (uint64_t)kHeaderBytes + 4ull * Sz;
                s_S = Sz;
            }
            if (!ok) s_ok = 0;
        }
        __syncthreads();
        if (!s_ok) break;   // uniform: every thread reads the same flag
        const int S = s_S;
        const uint16_t *pay = reinterpret_cast<const uint16_t *>(sin + kHeaderBytes + 4 * S);
        // exclusive scan of the word counts of all streams (chunked per thread)
        const uint8_t *cnt = sin + kHeaderBytes;
        const int per = (S + kDecThreads - 1) / kDecThreads;
        const int s0 = min(S, tid * per), s1 = min(S, s0 + per);
        // 64-bit sums, each bounded by the input's word count (below 2^32,
        // checked on the host), so the 32-bit prefix sums are exact
        uint64_t sum = 0, gsum = 0;
        int bad = 0;
        for (int s = s0; s < s1; s++) {
            const uint32_t c = cnt[4 * s] | (cnt[4 * s + 1] << 8) | (cnt[4 * s + 2] << 16) | ((uint32_t)cnt[4 * s + 3] << 24);
            bad |= c < 2;
            sum += c;
            if (s % P == (int)k) gsum += c;
        }
        bad |= sum > im.in_bytes / 2;
        s_part[tid] = (uint32_t)sum;
        s_gpart[tid] = (uint32_t)gsum;
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
            // the slices fill the input exactly
            const uint64_t next = slice_off + (uint64_t)kHeaderBytes + 4ull * S + 2ull * acc;
            if (z == D - 1 ? next != im.in_bytes : next > im.in_bytes) s_ok = 0;
            s_next = next;
            // payload of the owned streams staged in shared memory if it fits
            // (2D images; a volume's streams read the input through L1)
            s_fail = !vol && gacc <= (uint64_t)prm.pay_words ? 1 : 0;
        }
        __syncthreads();
        const bool staged = s_fail != 0;
        // word index of this slice's payload relative to the stream source
        const uint32_t word0 = vol ? (uint32_t)((slice_off + kHeaderBytes + 4ull * S) / 2) : 0u;
        if (s_ok) {
            uint16_t *spay = reinterpret_cast<uint16_t *>(smem + L.pay);
            uint32_t start = s_part[tid], lstart = s_gpart[tid];
            for (int s = s0; s < s1; s++) {
                const uint32_t c = cnt[4 * s] | (cnt[4 * s + 1] << 8) | (cnt[4 * s + 2] << 16) | ((uint32_t)cnt[4 * s + 3] << 24);
                if (s % P == (int)k) {
                    const int g = z * GS + s / P;
                    const uint32_t base = staged ? lstart : word0 + start;
                    st_x[g] = ((uint32_t)pay[start] << 16) | pay[start + 1];
                    st_pos[g] = base + 2;
                    st_end[g] = base + c;
                    if (staged)
                        for (uint32_t q = 0; q < c; q++) spay[lstart + q] = pay[start + q];
                    lstart += c;
                }
                start += c;
            }
            wsrc = vol ? reinterpret_cast<const uint16_t *>(in) : (staged ? spay : pay);
        }
        __syncthreads();
        const int G = (S - (int)k + P - 1) / P;    // streams owned by this CTA: s = k + P g
        if (s_ok)
            for (int g = tid; g < G; g += kDecThreads)
                if (st_x[z * GS + g] < kRansL) s_err = 1;
        if (tid == 0) s_fail = 0;
        __syncthreads();
    }
    const int S = s_S;
    const float invS = 1.0f / (float)(S > 0 ? S : 1);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // Every CTA of the cluster reads the same header, so this exit is uniform.
    if (!s_ok) {
        if (tid == 0 && k == 0) atomicMax(b.status + im.sidx, (int)DLIC_ERR_CORRUPT);
        if constexpr (!F32 && !SMMA) {
            if (warp == 0) tc::tmem_dealloc(tmem_base, 256);
        }
        return;
    }
    // When every CTA owns the rows k mod P (P divides S), a pixel's priors
    // come from rows r - d, d = 0 .. rows above, owned by CTAs k - d, which
    // push each decoded pixel into a tagged ring slot per row distance
    // (tcols columns of every row they own): CTAs then wait for the very
    // values they read instead of for each other, and no cluster barrier
    // runs per wave.  A CTA can run at most P - 1 waves ahead of a reader;
    // the launcher sizes tcols above 3 (rows above) + left reach + P, so an
    // entry outlives its last reader, and tq so that rows sharing a slot are
    // more than a wave's rows apart.
    // (the tags hold 11 bits of the row and 12 of the column: wider images
    // use the byte ring)
    const bool gimg = prm.gimg != 0;
    const bool p2p = !gimg && prm.tq > 0 && P >= 2 && P <= 16 && (S % P) == 0 && W <= 4096;
    uint32_t *tring = reinterpret_cast<uint32_t *>(smem + L.tring);
    const uint32_t tring_addr = tc::smem_addr(tring);
    const int tqmask = prm.tq - 1, tcmask = TCOLS - 1, rcmask = RCOLS - 1;
    // gather threads per pixel: the priors and one more, rounded to a power of two
    const int lg_slot = DEF || NPRI + 1 <= 16 ? 4 : (NPRI + 1 <= 32 ? 5 : (NPRI + 1 <= 64 ? 6 : 7));
    const int slot_px = 1 << lg_slot;
    if (P > 1) cluster_sync_all();   // every CTA's rings are initialised

    // FP32: W3^T streams through kW3Stages staging buffers in a fixed cycle
    // of chunks (k rows [kW3Rows c, kW3Rows (c + 1))); load number q goes to
    // buffer q mod kW3Stages and holds chunk q mod w3_chunks.  Every thread
    // counts the loads it has consumed in w3_seq.
    const int w3_chunks = (h2 + kW3Rows - 1) / kW3Rows;
    int w3_seq = 0;
    auto w3_issue = [&](int q) {
        const int stg = q % kW3Stages, c = q % w3_chunks;
        const uint32_t bytes = (uint32_t)min(kW3Rows, h2 - c * kW3Rows) * kSymbols * 4u;
        const uint32_t bar_a = tc::smem_addr(&w3bar[stg]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         tc::smem_addr(smem + L.w3s + (uint32_t)stg * kW3Rows * kSymbols * 4u)),
                     "l"(m.w3t + (size_t)c * kW3Rows * kSymbols), "r"(bytes), "r"(bar_a)
                     : "memory");
    };
    if constexpr (F32) {
        if (tid == 0)
            for (int q = 0; q < kW3Stages; q++) w3_issue(q);
    }

    const uint32_t tm = tmem_base;
    const int q4 = warp & 3, cg = warp >> 2;                 // lane quarter, column group (0..3)
    const int unit = 32 * q4 + lane;                          // hidden / output unit of this thread
    const uint32_t tm_q = tm + ((uint32_t)(32 * q4) << 16);
    float s1r = 0.f, o1r = 0.f, s2r = 0.f, o2r = 0.f, s3a = 0.f, o3a = 0.f, s3b = 0.f, o3b = 0.f;
    // warp-level MMAs: the output units of this thread's accumulator rows,
    // 16 w' + g and 16 w' + g + 8 (w' = warp mod 8 for layer 2, the warp for
    // layer 3, g = lane / 4)
    float s2lo = 0.f, o2lo = 0.f, s2hi = 0.f, o2hi = 0.f, s3lo = 0.f, o3lo = 0.f, s3hi = 0.f, o3hi = 0.f;
    if constexpr (DEEP) {
        // the first layer's unit `unit` (0 past its width) and the output
        // layer's units 16 warp + g and 16 warp + g + 8
        const DevLayer l0 = m.layers[0], lo = m.layers[m.nl - 1];
        s1r = unit < l0.n_out ? l0.a[unit] : 0.0f;
        o1r = unit < l0.n_out ? l0.o[unit] : 0.0f;
        const int u3 = 16 * warp + (lane >> 2);
        s3lo = lo.a[u3]; o3lo = lo.o[u3]; s3hi = lo.a[u3 + 8]; o3hi = lo.o[u3 + 8];
    } else if constexpr (!F32) {
        s1r = m.s1[unit]; o1r = m.o1[unit]; s2r = m.s2[unit]; o2r = m.o2[unit];
        s3a = m.s3[unit]; o3a = m.o3[unit]; s3b = m.s3[128 + unit]; o3b = m.o3[128 + unit];
        const int u2 = 16 * (warp & 7) + (lane >> 2), u3 = 16 * warp + (lane >> 2);   // (layer 2: warps 0..7)
        s2lo = m.s2[u2]; o2lo = m.o2[u2]; s2hi = m.s2[u2 + 8]; o2hi = m.o2[u2 + 8];
        s3lo = m.s3[u3]; o3lo = m.o3[u3]; s3hi = m.s3[u3 + 8]; o3hi = m.o3[u3 + 8];
    }
    uint8_t *ring = smem + L.ring;
    const uint32_t ring_addr = tc::smem_addr(ring);
    // the ring bases of the CTAs this lane stores to (the cluster window is
    // linear within a CTA, so the mapping is computed once)
    const uint32_t tring_dst =
        (P > 1 && lane < TSLOTS) ? map_shared(tring_addr, (k + (uint32_t)lane) % (uint32_t)P) : tring_addr;
    const uint32_t ring_dst = (P > 1 && lane < P) ? map_shared(ring_addr, (k + (uint32_t)lane) % (uint32_t)P) : ring_addr;
    const uint32_t *lut = reinterpret_cast<const uint32_t *>(smem + L.lut);
    const bool use_lut2 = prm.lut2 != 0;
    uint8_t *pri = smem + L.pri;   // priors of the chunk's pixels as s8 (x - 128), 16 bytes each
    uint8_t *b23 = smem + L.b23;
    float *zb = reinterpret_cast<float *>(smem + L.z);
    const uint32_t sb23 = tc::smem_addr(b23);
    const uint32_t sw2 = tc::smem_addr(smem + L.w2), sw3 = tc::smem_addr(smem + L.w3);
    // this thread's row of the first layer's INT8 weights, 4 inputs per word
    // (from the zero-padded copy in shared memory)
    uint32_t w1a = 0, w1b = 0, w1c = 0;
    if constexpr (!F32) {
        const uint32_t *w1q0 = reinterpret_cast<const uint32_t *>(smem + L.w1);
        w1a = w1q0[unit];
        w1b = w1q0[kDecHidden + unit];
        w1c = w1q0[2 * kDecHidden + unit];
    }
    const int rmask = prm.ring_rows - 1;
    uint32_t phase = 0;
    // Operand descriptors of K step 0; K step ks starts 256 bytes further,
    // i.e. 16 more in the descriptor's start-address field.
    const uint64_t dw2 = tc::make_desc(sw2, 128u, 16u * kDecHidden);
    const uint64_t dw3 = tc::make_desc(sw3, 128u, 16u * kDecHidden);
    const uint64_t dw3b = tc::make_desc(sw3 + 16u * 16u * kDecHidden, 128u, 16u * kDecHidden);
    const uint64_t db23 = tc::make_desc(sb23, 128u, 16u * kDecHidden);

    // Issues one layer's MMAs (thread 0), waits for them, and synchronises the
    // CTA.  After a timeout no further MMAs are issued; the wave loop still
    // runs to the end so that every cluster barrier is met.
    auto run_layer = [&](int layer, int NP) {
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0 && !s_fail) {
            tc::fence_after_sync();
            const uint32_t idesc = tc::idesc_bf16_f32(128, NP);
            if (layer == 2) {
                // two independent accumulation chains (K halves), summed in
                // the epilogue: exact, since every partial sum is an integer
                for (int j = 0; j < kDecHidden / 32; j++)
                    for (int part = 0; part < 2; part++) {
                        const int ks = part * (kDecHidden / 32) + j;
                        tc::mma_bf16(tm + (uint32_t)(part * NP), dw2 + 16u * ks, db23 + 16u * ks, idesc, j > 0);
                    }
            } else {
                // four chains: output half x K half
                for (int j = 0; j < kDecHidden / 32; j++)
                    for (int half = 0; half < 2; half++)
                        for (int part = 0; part < 2; part++) {
                            const int ks = part * (kDecHidden / 32) + j;
                            tc::mma_bf16(tm + (uint32_t)((2 * half + part) * NP), (half ? dw3b : dw3) + 16u * ks,
                                         db23 + 16u * ks, idesc, j > 0);
                        }
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
    auto hidden_epilogue = [&](int NP, float s, float o, bool two) {
        for (int c0 = 8 * cg; c0 < NP; c0 += 32) {
            uint32_t v[8], v2[8];
            tmem_ld8(tm_q + (uint32_t)c0, v);
            if (two) tmem_ld8(tm_q + (uint32_t)(NP + c0), v2);
            tc::tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const float acc = two ? __fadd_rn(__uint_as_float(v[e]), __uint_as_float(v2[e])) : __uint_as_float(v[e]);
                float h = rintf(__fmaf_rn(acc, s, o));
                h = fminf(fmaxf(h, 0.0f), 255.0f);
                const uint32_t mine = __float_as_uint(h) >> 16;
                const uint32_t other = __shfl_xor_sync(0xffffffffu, mine, 1);
                if ((lane & 1) == 0)
                    *reinterpret_cast<uint32_t *>(b23 + tc::kmajor_offset(c0 + e, unit, kDecHidden)) = mine | (other << 16);
            }
        }
    };

    // Warp-level MMAs of the two wide layers (SMMA).  A fragment rows
    // are units (W [unit][k]), B fragment columns are pixels (the activations
    // [pixel][k]); K = 128 in eight steps of 16.  Shared-memory bandwidth is
    // what these layers spend (every fragment is a shared-memory read), so
    // layer 3's weights, 16 units per warp, stay in registers across waves,
    // and layer 2 runs on warps 0..7 (units 16 w .. 16 w + 15), each taking
    // pixel octets in pairs so that one weight fragment feeds two MMAs.
    // Activation fragments come in by ldmatrix (two 8 x 8 matrices: the
    // octet's 8 pixel rows, k 0..7 and 8..15 of the step).
    uint16_t *act1 = reinterpret_cast<uint16_t *>(b23), *act2 = act1 + (size_t)NT * kActPitch;
    auto ld32 = [](const uint16_t *p) { return *reinterpret_cast<const uint32_t *>(p); };
    auto ldsm2 = [](const uint16_t *row, uint32_t &r0, uint32_t &r1) {
        asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];"
                     : "=r"(r0), "=r"(r1) : "r"(tc::smem_addr(row)));
    };
    const int mg = lane >> 2, mt4 = lane & 3;
    // this lane's row address within an 8-row ldmatrix block: row lane % 8,
    // k half (lane / 8) & 1
    const int lrow = lane & 7, lk = 8 * ((lane >> 3) & 1);
    uint32_t w3f[kDecHidden / 16][4];
    if constexpr (DEEP) {
        // the output layer's fragments straight from its packed s8 words
        // [k / 4][256]: W[u][k], W[u][k + 1] for even k (0 past its inputs)
        const DevLayer lo = m.layers[m.nl - 1];
        const uint32_t *q = static_cast<const uint32_t *>(lo.w);
        auto pair = [&](int u, int k) -> uint32_t {
            if (k >= lo.n_in) return 0u;
            const uint32_t v = __ldg(q + (k >> 2) * kSymbols + u) >> (8 * (k & 3));
            return (uint32_t)tc::bf16_of_int((int)(int8_t)(uint8_t)v) |
                   ((uint32_t)tc::bf16_of_int((int)(int8_t)(uint8_t)(v >> 8)) << 16);
        };
        const int u = 16 * warp + mg;
#pragma unroll
        for (int ks = 0; ks < kDecHidden / 16; ks++) {
            w3f[ks][0] = pair(u, 16 * ks + 2 * mt4);
            w3f[ks][1] = pair(u + 8, 16 * ks + 2 * mt4);
            w3f[ks][2] = pair(u, 16 * ks + 2 * mt4 + 8);
            w3f[ks][3] = pair(u + 8, 16 * ks + 2 * mt4 + 8);
        }
    } else if constexpr (!F32 && SMMA) {
        const uint16_t *W = reinterpret_cast<const uint16_t *>(smem + L.w3) + (size_t)(16 * warp + mg) * kActPitch + 2 * mt4;
#pragma unroll
        for (int ks = 0; ks < kDecHidden / 16; ks++) {
            w3f[ks][0] = ld32(W + 16 * ks);
            w3f[ks][1] = ld32(W + 8 * kActPitch + 16 * ks);
            w3f[ks][2] = ld32(W + 16 * ks + 8);
            w3f[ks][3] = ld32(W + 8 * kActPitch + 16 * ks + 8);
        }
    }
    auto mma_layer2 = [&](int NP) {
        if (warp >= 8) return;
        const uint16_t *W = reinterpret_cast<const uint16_t *>(smem + L.w2);
        const int u = 16 * warp + mg;
        const uint16_t *wa = W + (size_t)u * kActPitch + 2 * mt4;
        for (int n0 = 0; n0 < NP / 8; n0 += 2) {
            const uint16_t *xa = act1 + (size_t)(8 * n0 + lrow) * kActPitch + lk, *xb = xa + 8 * kActPitch;
            float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < kDecHidden / 16; ks++) {
                const uint32_t a0 = ld32(wa + 16 * ks), a1 = ld32(wa + 8 * kActPitch + 16 * ks),
                               a2 = ld32(wa + 16 * ks + 8), a3 = ld32(wa + 8 * kActPitch + 16 * ks + 8);
                uint32_t b0, b1, b2, b3;
                ldsm2(xa + 16 * ks, b0, b1);
                ldsm2(xb + 16 * ks, b2, b3);
                tc::mma_sync_bf16(c0, a0, a1, a2, a3, b0, b1);
                tc::mma_sync_bf16(c1, a0, a1, a2, a3, b2, b3);
            }
            auto q = [](float acc, float s, float o) {
                float h = rintf(__fmaf_rn(acc, s, o));
                h = fminf(fmaxf(h, 0.0f), 255.0f);
                return (uint16_t)(__float_as_uint(h) >> 16);   // bf16 of the integer
            };
            const int p = 8 * n0 + 2 * mt4;
            act2[(size_t)p * kActPitch + u] = q(c0[0], s2lo, o2lo);
            act2[(size_t)(p + 1) * kActPitch + u] = q(c0[1], s2lo, o2lo);
            act2[(size_t)p * kActPitch + u + 8] = q(c0[2], s2hi, o2hi);
            act2[(size_t)(p + 1) * kActPitch + u + 8] = q(c0[3], s2hi, o2hi);
            act2[(size_t)(p + 8) * kActPitch + u] = q(c1[0], s2lo, o2lo);
            act2[(size_t)(p + 9) * kActPitch + u] = q(c1[1], s2lo, o2lo);
            act2[(size_t)(p + 8) * kActPitch + u + 8] = q(c1[2], s2hi, o2hi);
            act2[(size_t)(p + 9) * kActPitch + u + 8] = q(c1[3], s2hi, o2hi);
        }
    };
    // DEEP: hidden-to-hidden layer l (weights and scales in shared memory)
    // from activations `in` to `out`, as mma_layer2 does for the fixed network
    auto mma_hidden = [&](int NP, int l, const uint16_t *in, uint16_t *out) {
        if (warp >= 8) return;
        const uint16_t *W = reinterpret_cast<const uint16_t *>(smem + L.w2) + (size_t)l * kDecHidden * kActPitch;
        const float *sh = reinterpret_cast<const float *>(smem + L.shid) + (size_t)(2 * l) * kDecHidden;
        const int u = 16 * warp + mg;
        const float slo = sh[u], shi = sh[u + 8], olo = sh[kDecHidden + u], ohi = sh[kDecHidden + u + 8];
        const uint16_t *wa = W + (size_t)u * kActPitch + 2 * mt4;
        for (int n0 = 0; n0 < NP / 8; n0 += 2) {
            const uint16_t *xa = in + (size_t)(8 * n0 + lrow) * kActPitch + lk, *xb = xa + 8 * kActPitch;
            float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < kDecHidden / 16; ks++) {
                const uint32_t a0 = ld32(wa + 16 * ks), a1 = ld32(wa + 8 * kActPitch + 16 * ks),
                               a2 = ld32(wa + 16 * ks + 8), a3 = ld32(wa + 8 * kActPitch + 16 * ks + 8);
                uint32_t b0, b1, b2, b3;
                ldsm2(xa + 16 * ks, b0, b1);
                ldsm2(xb + 16 * ks, b2, b3);
                tc::mma_sync_bf16(c0, a0, a1, a2, a3, b0, b1);
                tc::mma_sync_bf16(c1, a0, a1, a2, a3, b2, b3);
            }
            auto q = [](float acc, float sc, float of) {
                float h = rintf(__fmaf_rn(acc, sc, of));
                h = fminf(fmaxf(h, 0.0f), 255.0f);
                return (uint16_t)(__float_as_uint(h) >> 16);   // bf16 of the integer
            };
            const int p = 8 * n0 + 2 * mt4;
            out[(size_t)p * kActPitch + u] = q(c0[0], slo, olo);
            out[(size_t)(p + 1) * kActPitch + u] = q(c0[1], slo, olo);
            out[(size_t)p * kActPitch + u + 8] = q(c0[2], shi, ohi);
            out[(size_t)(p + 1) * kActPitch + u + 8] = q(c0[3], shi, ohi);
            out[(size_t)(p + 8) * kActPitch + u] = q(c1[0], slo, olo);
            out[(size_t)(p + 9) * kActPitch + u] = q(c1[1], slo, olo);
            out[(size_t)(p + 8) * kActPitch + u + 8] = q(c1[2], shi, ohi);
            out[(size_t)(p + 9) * kActPitch + u + 8] = q(c1[3], shi, ohi);
        }
    };
    auto mma_layer3 = [&](int NP, const uint16_t *act_in) {
        const int u = 16 * warp + mg;
        for (int n0 = 0; n0 < NP / 8; n0 += 2) {   // NP is a multiple of 16: octets in pairs
            const uint16_t *xa = act_in + (size_t)(8 * n0 + lrow) * kActPitch + lk, *xb = xa + 8 * kActPitch;
            float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < kDecHidden / 16; ks++) {
                uint32_t b0, b1, b2, b3;
                ldsm2(xa + 16 * ks, b0, b1);
                ldsm2(xb + 16 * ks, b2, b3);
                tc::mma_sync_bf16(c0, w3f[ks][0], w3f[ks][1], w3f[ks][2], w3f[ks][3], b0, b1);
                tc::mma_sync_bf16(c1, w3f[ks][0], w3f[ks][1], w3f[ks][2], w3f[ks][3], b2, b3);
            }
            const int p = 8 * n0 + 2 * mt4;
            zb[(size_t)p * kZPitch + u] = __fmaf_rn(c0[0], s3lo, o3lo);
            zb[(size_t)(p + 1) * kZPitch + u] = __fmaf_rn(c0[1], s3lo, o3lo);
            zb[(size_t)p * kZPitch + u + 8] = __fmaf_rn(c0[2], s3hi, o3hi);
            zb[(size_t)(p + 1) * kZPitch + u + 8] = __fmaf_rn(c0[3], s3hi, o3hi);
            zb[(size_t)(p + 8) * kZPitch + u] = __fmaf_rn(c1[0], s3lo, o3lo);
            zb[(size_t)(p + 9) * kZPitch + u] = __fmaf_rn(c1[1], s3lo, o3lo);
            zb[(size_t)(p + 8) * kZPitch + u + 8] = __fmaf_rn(c1[2], s3hi, o3hi);
            zb[(size_t)(p + 9) * kZPitch + u + 8] = __fmaf_rn(c1[3], s3hi, o3hi);
        }
    };

    int *rowlist = reinterpret_cast<int *>(smem + L.rows);
    int *zpre = reinterpret_cast<int *>(smem + L.zpre);   // grid decoder: first index of each active slice
    int *pixg = reinterpret_cast<int *>(smem + L.pg);
    uint8_t *dsym = smem + L.dsym;   // this wave's decoded pixels, by row-list index
    __shared__ int s_wcnt[kDecWarps];
    // exclusive prefix of v over the CTA's threads (total of all in `total`)
    auto block_scan = [&](int v, int &total) {
        int incl = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        if (lane == 31) s_wcnt[warp] = incl;
        __syncthreads();
        int before = incl - v;
        total = 0;
#pragma unroll
        for (int w2 = 0; w2 < kDecWarps; w2++) {
            const int cw = s_wcnt[w2];
            before += w2 < warp ? cw : 0;
            total += cw;
        }
        __syncthreads();
        return before;
    };
    // A volume's slices run as one 3D wavefront (Sec. IV "3D Wavefront"):
    // pixel (z, r, c) is on wave 3r + c + VSH z, every slice VSH waves behind
    // the one before it, so that the lower layer of its window is decoded.
    const int T2 = 3 * (H - 1) + W;
    const int VSH = vol ? volume_shift(m) : 0;
    const int T = gb ? prm.T : T2 + VSH * (D - 1);
    // When P divides S the owned rows of a wave are r0, r0 + P, ... and no
    // row list is built (a volume lists (slice, row) pairs, with P | S).
    const bool modrows = (S % P) == 0 && !vol;
    // Without a per-wave cluster barrier a decoded pixel goes to the image
    // at once; otherwise the stores wait until the barrier has been arrived at.
    const bool direct = p2p || P == 1 || gimg;
    for (int t = 0; t < T; t++) {
        const int r_lo = t - W + 1 > 0 ? (t - W + 3) / 3 : 0;
        const int r_hi = min(H - 1, t / 3);
        // rows of this wave owned by this CTA, in increasing order
        int nk = 0;
        const int r0 = r_lo + (((int)k - r_lo) & (P - 1));
        int nd = 0;   // grid batch: pixels of this CTA's whole (not spread) images, listed first
        if (gb) {
            const int NB = (int)gridDim.x, kb = (int)blockIdx.x;
            // images whose waves hold two rows of one stream go whole to CTA
            // i mod NB, in row order (n <= kMaxBatch < kDecThreads: thread = image)
            {
                const int i = tid;
                int cnt = 0, rl = 0;
                if (i < b.n && itflag[i] == 1 && i % NB == kb && t < itT2[i]) {
                    rl = t - b.img[i].W + 1 > 0 ? (t - b.img[i].W + 3) / 3 : 0;
                    cnt = min(b.img[i].H - 1, t / 3) - rl + 1;
                }
                int total;
                const int before = block_scan(cnt, total);
                for (int j = 0; j < cnt; j++) rowlist[before + j] = (i << 20) | (rl + j);
                nd = total;
            }
            // the spread images' rows split evenly over the grid
            {
                const int i = tid;
                int cnt = 0;
                if (i < b.n && itflag[i] == 3 && t < itT2[i]) {
                    const int rl = t - b.img[i].W + 1 > 0 ? (t - b.img[i].W + 3) / 3 : 0;
                    cnt = min(b.img[i].H - 1, t / 3) - rl + 1;
                }
                int n;
                const int before = block_scan(cnt, n);
                if (i < b.n) zpre[i] = before;
                __syncthreads();
                const int i0 = (int)((long long)n * kb / NB), i1 = (int)((long long)n * (kb + 1) / NB);
                for (int j = tid; j < i1 - i0; j += kDecThreads) {
                    const int gi = i0 + j;
                    int lo = 0, hi = b.n - 1;   // the last image whose first index is <= gi
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (zpre[mid] <= gi) lo = mid; else hi = mid - 1;
                    }
                    const int rl = t - b.img[lo].W + 1 > 0 ? (t - b.img[lo].W + 3) / 3 : 0;
                    rowlist[nd + j] = (lo << 20) | (rl + gi - zpre[lo]);
                }
                nk = nd + (i1 - i0);
                __syncthreads();
            }
        } else if (GRID) {
            // every row of the slices on this wave, in slice order; this CTA
            // takes the indices [kb n / NB, (kb + 1) n / NB): thread = slice,
            // block-wide exclusive scan of the row counts into zpre
            const int z_lo = t >= T2 ? (t - T2) / VSH + 1 : 0, z_hi = min(D - 1, t / VSH);
            const int nz = z_hi - z_lo + 1;
            int n = 0;
            for (int zb = 0; zb < nz; zb += kDecThreads) {
                const int zi = zb + tid;
                int cnt = 0;
                if (zi < nz) {
                    const int tz = t - VSH * (z_lo + zi);
                    const int rl = tz - W + 1 > 0 ? (tz - W + 3) / 3 : 0, rh = min(H - 1, tz / 3);
                    cnt = rh - rl + 1;
                }
                int incl = cnt;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int o = __shfl_up_sync(0xffffffffu, incl, off);
                    if (lane >= off) incl += o;
                }
                if (lane == 31) s_wcnt[warp] = incl;
                __syncthreads();
                int before = n + incl - cnt, total = 0;
#pragma unroll
                for (int w2 = 0; w2 < kDecWarps; w2++) {
                    const int cw = s_wcnt[w2];
                    before += w2 < warp ? cw : 0;
                    total += cw;
                }
                if (zi < nz) zpre[zi] = before;
                n += total;
                __syncthreads();
            }
            const int NB = (int)gridDim.x, kb = (int)blockIdx.x;
            const int i0 = (int)((long long)n * kb / NB), i1 = (int)((long long)n * (kb + 1) / NB);
            nk = i1 - i0;
            for (int j = tid; j < nk; j += kDecThreads) {
                const int gi = i0 + j;
                int lo = 0, hi = nz - 1;   // the last slice whose first index is <= gi
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (zpre[mid] <= gi) lo = mid; else hi = mid - 1;
                }
                const int z = z_lo + lo, tz = t - VSH * z;
                const int rl = tz - W + 1 > 0 ? (tz - W + 3) / 3 : 0;
                rowlist[j] = (z << 20) | (rl + gi - zpre[lo]);
            }
            __syncthreads();
        } else if (vol) {
            // the slices on this wave (t - VSH z in [0, T2)), in slice
            // order, each with its owned rows r0(z), r0(z) + P, ...:
            // thread = slice, block-wide exclusive scan of the counts
            const int z_lo = t >= T2 ? (t - T2) / VSH + 1 : 0, z_hi = min(D - 1, t / VSH);
            for (int zb = z_lo; zb <= z_hi; zb += kDecThreads) {
                const int z = zb + tid;
                int cnt = 0, rz = 0;
                if (z <= z_hi) {
                    const int tz = t - VSH * z;
                    const int rl = tz - W + 1 > 0 ? (tz - W + 3) / 3 : 0, rh = min(H - 1, tz / 3);
                    rz = rl + (((int)k - rl) & (P - 1));
                    cnt = rz <= rh ? ((rh - rz) >> lgP) + 1 : 0;
                }
                int incl = cnt;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int o = __shfl_up_sync(0xffffffffu, incl, off);
                    if (lane >= off) incl += o;
                }
                if (lane == 31) s_wcnt[warp] = incl;
                __syncthreads();
                int before = nk + incl - cnt, total = 0;
#pragma unroll
                for (int w2 = 0; w2 < kDecWarps; w2++) {
                    const int cw = s_wcnt[w2];
                    before += w2 < warp ? cw : 0;
                    total += cw;
                }
                for (int j = 0; j < cnt; j++) rowlist[before + j] = (z << 20) | (rz + (j << lgP));
                nk += total;
                __syncthreads();
            }
        } else if (modrows) {
            nk = r0 <= r_hi ? ((r_hi - r0) >> lgP) + 1 : 0;
        } else {
            for (int seg = r_lo; seg <= r_hi; seg += kDecThreads) {
                const int r = seg + tid;
                const bool own = r <= r_hi && (fast_mod(r, S, invS) & (P - 1)) == (int)k;
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
        }
        auto row_of = [&](int i) { return modrows ? r0 + (i << lgP) : rowlist[i]; };
        // (slice or image, row, column) of the wave's i-th owned pixel
        auto pix_of = [&](int i, int &z, int &r, int &c) {
            if (gb) {
                const int e = rowlist[i];
                z = e >> 20;
                r = e & 0xFFFFF;
                c = t - 3 * r;
            } else if (vol) {
                const int e = rowlist[i];
                z = e >> 20;
                r = e & 0xFFFFF;
                c = t - VSH * z - 3 * r;
            } else {
                z = 0;
                r = row_of(i);
                c = t - 3 * r;
            }
        };
        // no two rows of a slice's wave share a stream
        const bool spread = gb ? nd == 0 : (GRID || (vol ? min(H, (W + 2) / 3) <= S : r_hi - r_lo < S));
        for (int base = 0; base < nk; base += NT) {
            const int nc = min(NT, nk - base);
            const int NP = (nc + 15) & ~15;
            // 1. priors of the chunk's pixels, one thread per (pixel, prior)
            //    so that every ring read is in flight at once; the spare
            //    thread after a pixel's priors records its stream and table
            //    warp.  Pad pixels up to NP get arbitrary inputs.
            const int NPin = F32 ? (nc + 3) & ~3 : NP;   // pixels whose inputs are written
            for (int idx = tid; idx < slot_px * NPin; idx += kDecThreads) {
                const int px = idx >> lg_slot, q = idx & (slot_px - 1);
                if (q > NPRI) continue;
                uint32_t v = 0x80u;
                if (px < nc) {
                    int z, r, c;
                    pix_of(base + px, z, r, c);
                    if (q == NPRI) {
                        // local stream of the pixel and the warp that runs its
                        // table: by pixel when no two rows of the wave share a
                        // stream, else by stream so that they run in row order
                        int g;
                        bool own_warp = spread;   // warp by pixel, else by stream (row order)
                        if (gb) {
                            const int Si = itS[z];
                            g = (z << 16) | fast_mod(r, Si, 1.0f / (float)Si);
                            own_warp = itflag[z] == 3;
                        } else {
                            g = GRID ? z * S + fast_mod(r, S, invS) : z * GS + (fast_mod(r, S, invS) >> lgP);
                        }
                        pixg[px] = g | ((own_warp ? px % kDecWarps : g % kDecWarps) << 24);
                        continue;
                    }
                    int dr, dc, dz = 0;
                    if (DEF) {
                        dr = q < 5 ? -2 : (q < 10 ? -1 : 0);
                        dc = q < 5 ? q - 2 : (q < 10 ? q - 7 : q - 12);
                    } else {
                        const char4 o = s_woff[q];
                        dr = o.x;
                        dc = o.y;
                        dz = o.z;
                    }
                    const int rr = r + dr, cc = c + dc, zz = z + dz;
                    const int Wz = gb ? b.img[z].W : W;
                    // (a 3D window's lower layer may reach below the row and
                    // off the first slice)
                    if (rr < 0 || cc < 0 || cc >= Wz || (vol && (zz < 0 || rr >= H))) {
                        v = 0u;
                    } else if (p2p) {
                        // entry (round of rr, row distance, column mod tcols)
                        const int slot = ((rr >> lgP) & tqmask) * TSLOTS - dr;
                        const uint32_t *e = tring + slot * TCOLS + (cc & tcmask);
                        const uint32_t want = ring_tag(rr, cc);
                        v = ld_volatile_u32(e);
                        if ((v & 0xFFFFFF00u) != want) {
                            // bounded wait; after any timeout no wait blocks again
                            const long long t0 = clock64();
                            do {
                                v = ld_volatile_u32(e);
                                if (clock64() - t0 > m.peer_wait_limit || *reinterpret_cast<volatile int *>(&s_fail)) {
                                    s_fail = 1;
                                    break;
                                }
                            } while ((v & 0xFFFFFF00u) != want);
                        }
                        v &= 0xFFu;
                    } else if (gimg) {
                        // stored to the image before the last wave's barrier
                        v = gb ? __ldcg(b.img[z].pixels + (int64_t)rr * b.img[z].pitch + cc)
                               : __ldcg(im.pixels + (int64_t)zz * im.slice_pitch + (int64_t)rr * im.pitch + cc);
                    } else {
                        v = ring[(rr & rmask) * RCOLS + (cc & rcmask)];
                    }
                } else if (q == NPRI) {
                    continue;
                }
                // network input: x/128 - 1 (FP32) or x - 128 as s8; out-of-image
                // priors are 0
                if constexpr (F32)
                    reinterpret_cast<float *>(smem + L.xs)[K1 * px + q] = __fmaf_rn((float)v, 0.0078125f, -1.0f);
                else
                    pri[K1 * px + q] = (uint8_t)(v ^ 0x80u);
            }
            __syncthreads();   // every prior of the chunk is in place
            // the stream state (and the next payload word) of this warp's
            // first pixel, read now rather than on the table's dependency
            // chain (one pixel per stream in the wave: only this warp updates
            // that state before its table step)
            uint32_t pf_x = 0, pf_pos = 0, pf_end = 0, pf_word = 0;
            int pf_i = -1;
            if (!F32 && !GRID && spread && warp < nc) {   // (the FP32 decoder measured no gain)
                const int pg = pixg[warp];
                if ((pg >> 24) == warp) {
                    const int g = pg & 0xFFFFFF;
                    pf_x = st_x[g];
                    pf_pos = st_pos[g];
                    pf_end = st_end[g];
                    pf_word = pf_pos < pf_end ? wsrc[pf_pos] : 0u;
                    pf_i = warp;
                }
            }
            if constexpr (F32) {
                // 2. the FP32 network on the CUDA cores, fixed order per unit:
                //    bias first, then fma(x_k, w_jk, acc) for k ascending.
                //    Thread = (unit, 4 pixels); activations [unit][pitch PT].
                const float *xs = reinterpret_cast<const float *>(smem + L.xs);
                const float *wf = reinterpret_cast<const float *>(smem + L.wf);
                const float *w1s = wf, *b1s = wf + NPRI * h1, *b2s = b1s + h1, *b3s = b2s + h2;
                const float *w3s = b3s + kSymbols;
                float *h1t = reinterpret_cast<float *>(smem + L.h1t);
                float *h2t = reinterpret_cast<float *>(smem + L.h2t);
                const int PT = NT + 4;
                const int NG = (nc + 3) >> 2;
                for (int it = tid; it < h1 * NG; it += kDecThreads) {
                    const int u = it % h1, p0 = 4 * (it / h1);
                    float a[4];
#pragma unroll
                    for (int j = 0; j < 4; j++) a[j] = b1s[u];
#pragma unroll 4
                    for (int kk = 0; kk < NPRI; kk++) {
                        const float w = w1s[kk * h1 + u];
#pragma unroll
                        for (int j = 0; j < 4; j++) a[j] = __fmaf_rn(xs[K1 * (p0 + j) + kk], w, a[j]);
                    }
                    *reinterpret_cast<float4 *>(h1t + u * PT + p0) =
                        make_float4(a[0] > 0.0f ? a[0] : 0.0f, a[1] > 0.0f ? a[1] : 0.0f, a[2] > 0.0f ? a[2] : 0.0f,
                                    a[3] > 0.0f ? a[3] : 0.0f);
                }
                __syncthreads();
                // second layer: thread = (4 units, 2 pixels), W2^T in shared memory
                const int NPP = (nc + 1) >> 1;
                const float *w2s = reinterpret_cast<const float *>(smem + L.w2f);
                for (int it = tid; it < (h2 / 4) * NPP; it += kDecThreads) {
                    const int uq = it % (h2 / 4), p0 = 2 * (it / (h2 / 4));
                    const float4 bb = *reinterpret_cast<const float4 *>(b2s + 4 * uq);
                    float a0[4] = {bb.x, bb.y, bb.z, bb.w}, a1[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll 4
                    for (int kk = 0; kk < h1; kk++) {
                        const float4 w = *reinterpret_cast<const float4 *>(w2s + kk * h2 + 4 * uq);
                        const float2 x = *reinterpret_cast<const float2 *>(h1t + kk * PT + p0);
                        a0[0] = __fmaf_rn(x.x, w.x, a0[0]);
                        a0[1] = __fmaf_rn(x.x, w.y, a0[1]);
                        a0[2] = __fmaf_rn(x.x, w.z, a0[2]);
                        a0[3] = __fmaf_rn(x.x, w.w, a0[3]);
                        a1[0] = __fmaf_rn(x.y, w.x, a1[0]);
                        a1[1] = __fmaf_rn(x.y, w.y, a1[1]);
                        a1[2] = __fmaf_rn(x.y, w.z, a1[2]);
                        a1[3] = __fmaf_rn(x.y, w.w, a1[3]);
                    }
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        *reinterpret_cast<float2 *>(h2t + (4 * uq + i) * PT + p0) =
                            make_float2(a0[i] > 0.0f ? a0[i] : 0.0f, a1[i] > 0.0f ? a1[i] : 0.0f);
                }
                __syncthreads();
                // logits: W3^T arrives chunk by chunk in the staging buffers;
                // z overlays the inputs and the first layer's activations
                f32_logits(tid, NG, w3_chunks, w3_seq, w3_issue, h2, b3s, h2t, PT, smem + L.w3s, w3bar, zb, s_fail,
                           s_cfail);
                __syncthreads();
            } else {
                // 2. the three layers: the first (K = the window's priors) as
                //    dp4a on the CUDA cores, exact integer sums requantised like
                //    the tensor-core epilogues.  Thread = (unit, pixel group):
                //    four pixels of the group at a time (NP is a multiple of 16),
                //    their dot products interleaved
                const uint32_t *w1q = reinterpret_cast<const uint32_t *>(smem + L.w1);
                const uint32_t w1d = K1 == 16 && NPRI > 12 ? w1q[3 * kDecHidden + unit] : 0u;
                for (int p0 = cg; p0 < NP; p0 += 16) {
                    int acc[4];
                    if (K1 == 16) {
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            const uint4 xv = *reinterpret_cast<const uint4 *>(pri + 16 * (p0 + 4 * j));
                            acc[j] = dp4a_ss(xv.z, w1c, dp4a_ss(xv.y, w1b, dp4a_ss(xv.x, w1a, 0)));
                            if (NPRI > 12) acc[j] = dp4a_ss(xv.w, w1d, acc[j]);
                        }
                    } else {
                        // a wider window: its priors as words, W1 words from shared memory
#pragma unroll
                        for (int j = 0; j < 4; j++) acc[j] = 0;
                        for (int k16 = 0; k16 < K1 / 16; k16++) {
                            uint32_t w[4];
#pragma unroll
                            for (int e = 0; e < 4; e++) w[e] = w1q[(4 * k16 + e) * kDecHidden + unit];
#pragma unroll
                            for (int j = 0; j < 4; j++) {
                                const uint4 xv = *reinterpret_cast<const uint4 *>(pri + K1 * (p0 + 4 * j) + 16 * k16);
                                acc[j] = dp4a_ss(xv.w, w[3], dp4a_ss(xv.z, w[2], dp4a_ss(xv.y, w[1], dp4a_ss(xv.x, w[0], acc[j]))));
                            }
                        }
                    }
                    uint32_t mine[4];
#pragma unroll
                    for (int j = 0; j < 4; j++) mine[j] = __float_as_uint((float)requant_u8(acc[j], s1r, o1r)) >> 16;   // bf16 of the integer
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const uint32_t other = __shfl_xor_sync(0xffffffffu, mine[j], 1);
                        if ((lane & 1) == 0) {
                            if (SMMA)
                                *reinterpret_cast<uint32_t *>(act1 + (size_t)(p0 + 4 * j) * kActPitch + unit) =
                                    mine[j] | (other << 16);
                            else
                                *reinterpret_cast<uint32_t *>(b23 + tc::kmajor_offset(p0 + 4 * j, unit, kDecHidden)) =
                                    mine[j] | (other << 16);
                        }
                    }
                }
                if (DEEP) {
                    // the hidden-to-hidden layers, act1 and act2 in turn, then
                    // the output layer from the last of them
                    uint16_t *ain = act1, *aout = act2;
                    for (int l = 0; l < prm.nhh; l++) {
                        __syncthreads();   // the previous layer's outputs are in place
                        mma_hidden(NP, l, ain, aout);
                        uint16_t *tsw = ain;
                        ain = aout;
                        aout = tsw;
                    }
                    __syncthreads();
                    mma_layer3(NP, ain);
                    __syncthreads();   // the logits are in place
                } else if (SMMA) {
                    __syncthreads();   // the first layer's outputs are in place
                    mma_layer2(NP);
                    __syncthreads();
                    mma_layer3(NP, act2);
                    __syncthreads();   // the logits are in place
                } else {
                run_layer(2, NP);
                hidden_epilogue(NP, s2r, o2r, true);
                run_layer(3, NP);
                for (int c0 = 8 * cg; c0 < NP; c0 += 32) {
                    uint32_t va[8], va2[8], vb[8], vb2[8];
                    tmem_ld8(tm_q + (uint32_t)c0, va);
                    tmem_ld8(tm_q + (uint32_t)(NP + c0), va2);
                    tmem_ld8(tm_q + (uint32_t)(2 * NP + c0), vb);
                    tmem_ld8(tm_q + (uint32_t)(3 * NP + c0), vb2);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 8; e++) {
                        const float a = __fadd_rn(__uint_as_float(va[e]), __uint_as_float(va2[e]));
                        const float bsum = __fadd_rn(__uint_as_float(vb[e]), __uint_as_float(vb2[e]));
                        zb[(c0 + e) * kSymbols + unit] = __fmaf_rn(a, s3a, o3a);
                        zb[(c0 + e) * kSymbols + 128 + unit] = __fmaf_rn(bsum, s3b, o3b);
                    }
                }
                tc::fence_before_sync();
                __syncthreads();
                }
            }
            // 3. tables and rANS steps, one warp per pixel; pixels that share a
            //    stream go to the same warp (by local stream index), in row
            //    order.
            for (int i = spread ? warp : 0; i < nc; i += spread ? kDecWarps : 1) {
                const int pg = pixg[i];
                if ((pg >> 24) != warp) continue;
                const int g = pg & 0xFFFFFF;
                int zs, r, c;
                pix_of(base + i, zs, r, c);
                // (the grid decoder's states were last written by other CTAs:
                // read them from L2; a batch keeps them per image)
                uint32_t *sx = st_x, *sp = st_pos, *se = st_end;
                int gs = g;
                if (gb) {
                    const VolState vi = vol_state(b, b.img[g >> 16]);
                    sx = vi.x;
                    sp = vi.pos;
                    se = vi.end;
                    gs = g & 0xFFFF;
                }
                const bool pre = i == pf_i;
                const uint32_t x = pre ? pf_x : GRID ? __ldcg(sx + gs) : sx[gs];
                // the stream's next word, fetched before it is known to be needed
                const uint32_t pos = pre ? pf_pos : GRID ? __ldcg(sp + gs) : sp[gs];
                const uint32_t pend = pre ? pf_end : GRID ? __ldcg(se + gs) : se[gs];
                const uint32_t next_word = pre ? pf_word : pos < pend ? wsrc[pos] : 0u;
                const int zp = F32 || !SMMA ? kSymbols : kZPitch;
                const float4 za = *reinterpret_cast<const float4 *>(zb + i * zp + 8 * lane);
                const float4 zc = *reinterpret_cast<const float4 *>(zb + i * zp + 8 * lane + 4);
                const float z[8] = {za.x, za.y, za.z, za.w, zc.x, zc.y, zc.z, zc.w};
                // the lane's maximum, then the warp's through an order-preserving
                // integer key (a zero maximum's sign changes no weight)
                float lmax = z[0];
#pragma unroll
                for (int q = 1; q < 8; q++) lmax = fmaxf(lmax, z[q]);
                const float mx = key_float(__reduce_max_sync(0xffffffffu, float_key(lmax)));
                uint32_t w[8], lsum = 0;
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    w[q] = use_lut2 ? table_weight2(mx, z[q], m.tscale, lut) : table_weight(mx, z[q], m.tscale, lut);
                    lsum += w[q];
                }
                // the total (and from it Q) runs beside the prefix scan
                const uint32_t Wsum = __reduce_add_sync(0xffffffffu, lsum);
                const uint32_t Q = table_q_fast(Wsum);
                uint32_t incl = lsum;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
                    if (lane >= off) incl += o;
                }
                const uint32_t excl = incl - lsum;
                const uint32_t slot = x & 0xFFFFu;
                const uint32_t cs = 8u * lane + __umulhi(excl, Q);
                const uint32_t ball = __ballot_sync(0xffffffffu, cs <= slot);
                const int Lh = 31 - __clz(ball);
                // c at the 9 unit boundaries of this lane; the symbol is the
                // last unit whose lower boundary does not exceed the slot
                uint32_t cb[9];
                uint32_t Pp = excl;
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    cb[q] = 8u * lane + q + __umulhi(Pp, Q);
                    Pp += w[q];
                }
                cb[8] = lane == 31 ? kTotal : 8u * lane + 8u + __umulhi(Pp, Q);
                uint32_t sym = 8u * lane, f = cb[1] - cb[0], clo = cb[0];
#pragma unroll
                for (int q = 1; q < 8; q++)
                    if (cb[q] <= slot) {
                        sym = 8u * lane + q;
                        f = cb[q + 1] - cb[q];
                        clo = cb[q];
                    }
                sym = __shfl_sync(0xffffffffu, sym, Lh);
                // the decoded pixel goes out first: the next waves of this CTA
                // and of the CTAs owning the rows below it read it
                if (p2p) {
                    if (lane < TSLOTS) {
                        // row distance d = lane: the CTA k + d reads this row as r - d
                        const int slot = ((r >> lgP) & tqmask) * TSLOTS + lane;
                        const uint32_t off = 4u * (uint32_t)(slot * TCOLS + (c & tcmask));
                        if (lane == 0)
                            asm volatile("st.shared::cta.u32 [%0], %1;" ::"r"(tring_addr + off), "r"(ring_tag(r, c) | sym)
                                         : "memory");
                        else
                            st_cluster_u32(tring_dst + off, ring_tag(r, c) | sym);
                    }
                } else if (!gimg && lane < P) {
                    const uint32_t off = (uint32_t)((r & rmask) * RCOLS + (c & rcmask));
                    if (P > 1)
                        st_cluster_u8(ring_dst + off, sym);
                    else
                        ring[off] = (uint8_t)sym;
                }
                f = __shfl_sync(0xffffffffu, f, Lh);
                clo = __shfl_sync(0xffffffffu, clo, Lh);
                if (lane == 0) {
                    uint32_t xn = f * (x >> 16) + slot - clo;
                    if (xn < kRansL) {
                        if (pos < pend) {
                            xn = (xn << 16) | next_word;
                            sp[gs] = pos + 1;
                        } else {
                            s_err = 1;
                        }
                    }
                    sx[gs] = xn;
                    if (direct)
                        (gb ? b.img[zs].pixels + (int64_t)r * b.img[zs].pitch
                            : im.pixels + (int64_t)zs * im.slice_pitch + (int64_t)r * im.pitch)[c] = (uint8_t)sym;
                    else
                        dsym[base + i] = (uint8_t)sym;
                }
                __syncwarp();
            }
            __syncthreads();
        }
        if (!direct) {
            // The cluster barrier is arrived at before this wave's pixels go
            // to the image, so its release waits only for the ring writes; the
            // image stores complete during the next wave.
            __syncthreads();   // every ring write of this wave precedes the barrier arrival
            asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
            for (int i = tid; i < nk; i += kDecThreads) {
                const int r = row_of(i);
                im.pixels[(int64_t)r * im.pitch + (t - 3 * r)] = dsym[i];
            }
            __syncthreads();   // the row list is rebuilt only after every image store
            asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
        } else if (GRID) {
            // grid-wide barrier: arrivals accumulate in the volume's header,
            // wave t is complete at (t + 1) NB; a wait that runs out marks
            // the volume so that every other CTA stops waiting too
            const VolState vs = vol_state(b, im);
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                atomicAdd(vs.hdr + 2, 1u);
                const uint32_t target = (uint32_t)(t + 1) * gridDim.x;
                const long long t0 = clock64();
                while (ld_acquire_gpu_u32(vs.hdr + 2) < target) {
                    if (ld_acquire_gpu_u32(vs.hdr + 3) || clock64() - t0 > m.peer_wait_limit) {
                        atomicExch(vs.hdr + 3, 1u);
                        s_fail = 1;
                        break;
                    }
                }
                __threadfence();
            }
            __syncthreads();
            if (s_fail) break;
        } else if (gimg && P > 1) {
            // every CTA's image stores of this wave before any CTA's next gather
            cluster_sync_all();
        } else if (!modrows) {
            __syncthreads();   // the row list is rebuilt only after every reader is done
        }
    }
    // FP32: the loads issued ahead for a next wave complete before the CTA
    // leaves (its shared memory must not be written after it exits)
    if constexpr (F32) {
        if (tid == 0 && !s_cfail)
            for (int q = w3_seq; q < w3_seq + kW3Stages; q++)
                if (!tc::mbar_wait(&w3bar[q % kW3Stages], (uint32_t)(q / kW3Stages) & 1u, kDecWaitLimit)) {
                    s_cfail = 1;
                    s_fail = 1;
                    break;
                }
    }
    // final states must be back at the initial value with every word read
    // (the grid decoder's are checked by k_volume_finish)
    if (!GRID) {
        const int G = (S - (int)k + P - 1) / P;
        for (int i = tid; i < D * G; i += kDecThreads) {
            const int g = (i / G) * GS + i % G;
            if (st_x[g] != kRansL || st_pos[g] != st_end[g]) s_err = 1;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && (s_err || s_fail))
        atomicMax(b.status + im.sidx, s_fail ? (int)DLIC_ERR_TIMEOUT : (int)DLIC_ERR_CORRUPT);
    if constexpr (!F32 && !SMMA) {
        if (warp == 0) {
            tc::fence_after_sync();
            tc::tmem_dealloc(tm, 256);
        }
    }
    if (P > 1) cluster_sync_all();   // no CTA leaves while others may still write its ring
}

template <bool DEF, bool SMMA>
__global__ void __launch_bounds__(kDecThreads, 1) k_decode_tc(DevModel m, DecBatch b, DecTcParams prm) {
    decode_wave<false, DEF, false, SMMA>(m, b, prm);
}
// INT8 networks of 1..5 hidden layers of widths up to 128 (the default window)
__global__ void __launch_bounds__(kDecThreads, 1) k_decode_tc_deep(DevModel m, DecBatch b, DecTcParams prm) {
    decode_wave<false, true, false, true, true>(m, b, prm);
}
template <bool DEF>
__global__ void __launch_bounds__(kDecThreads, 1) k_decode_f32(DevModel m, DecBatch b, DecTcParams prm) {
    decode_wave<true, DEF, false, false>(m, b, prm);
}
// one volume over a cooperative grid
template <bool SMMA>
__global__ void __launch_bounds__(kDecThreads, 1) k_decode_grid_tc(DevModel m, DecBatch b, DecTcParams prm) {
    decode_wave<false, false, true, SMMA>(m, b, prm);
}
__global__ void __launch_bounds__(kDecThreads, 1) k_decode_grid_f32(DevModel m, DecBatch b, DecTcParams prm) {
    decode_wave<true, false, true, false>(m, b, prm);
}

// Chunks of up to kSmmaMaxChunk pixels take the warp-level MMAs (INT8).
static inline bool smma_chunk(const DevModel &m, int per_cta) {
    return m.precision == DLIC_INT8 && min(64, (per_cta + 15) & ~15) <= kSmmaMaxChunk;
}
static inline int wave_per_cta(int maxH, int maxW, int P) { return (min(maxH, (maxW + 2) / 3) + P - 1) / P + 1; }

// Cluster sizes for a batch (the decode autotuner).  A wave of an image
// whose CTAs hold p pixels costs about kWaveFixed cycles (gather, MMA round
// trips, epilogues) plus kWavePerPixelWarp per round of 16 table warps and
// kWavePerPixel per pixel, over chunks of at most 64 pixels (constants from
// clock64 phase timings on GB300); an image takes waves x that.  Starting
// from one CTA per image, the image with the longest estimate gets its
// cluster doubled while the clusters of the whole batch still fit on the
// GPU at once (up to 16 CTAs per image).
constexpr double kWaveFixed = 4200.0, kWavePerPixelWarp = 1900.0, kWavePerPixel = 65.0;
// FP32 network: the CUDA cores' multiply-adds (about 50K per pixel at
// 128 a cycle) add to the table rounds, in chunks of 16 pixels.
constexpr double kWaveFixedF32 = 5000.0, kWavePerPixelF32 = 420.0;

static double est_cycles(int H, int W, int P, bool f32) {
    const double waves = 3.0 * (H - 1) + W;
    const int wave_px = min(H, (W + 2) / 3);
    int per = (wave_px + P - 1) / P;
    double per_wave = 0.0;
    while (per > 0) {
        const int chunk = min(per, f32 ? 16 : 64);
        per_wave += f32 ? kWaveFixedF32 + kWavePerPixelF32 * ((chunk + 3) & ~3) + kWavePerPixelWarp
                        : kWaveFixed + kWavePerPixelWarp * ((chunk + kDecWarps - 1) / kDecWarps) + kWavePerPixel * chunk;
        per -= chunk;
    }
    return waves * per_wave;
}

double decode_estimate(int H, int W, int P, bool f32) { return est_cycles(H, W, P, f32); }

void choose_clusters(const int *H, const int *W, int n, int num_sms, bool f32, int *P) {
    int used = 0;
    for (int i = 0; i < n; i++) {
        P[i] = 1;
        used += 1;
    }
    for (;;) {
        int best = -1;
        double worst = 0.0;
        for (int i = 0; i < n; i++) {
            if (P[i] >= 16 || used + P[i] > num_sms) continue;
            const double t = est_cycles(H[i], W[i], P[i], f32);
            if (t > worst) {
                worst = t;
                best = i;
            }
        }
        if (best < 0) break;
        // stop when the longest image no longer gains from a larger cluster
        if (est_cycles(H[best], W[best], 2 * P[best], f32) >= worst) break;
        used += P[best];
        P[best] *= 2;
    }
}

// The cluster wavefront decoder runs the INT8 network of widths 128 on the
// tensor cores, and FP32 networks whose W3^T fits in 128 KB of shared memory
// on the CUDA cores; other networks use the one-CTA-per-image decoder.
bool wave_decode_supported(const DevModel &m) {
    if (m.precision == DLIC_INT8) return m.tc_w != nullptr && m.h1 == kDecHidden && m.h2 == kDecHidden;
    return m.precision == DLIC_FP32 && m.h1 >= 4 && m.h1 <= kMaxHidden && m.h2 >= 4 && m.h2 <= 128 && m.h1 % 4 == 0 &&
           m.h2 % 4 == 0;
}

// INT8 networks of 1..5 hidden layers (other than two) of widths up to 128
// with the default 2D window: the cluster wavefront decoder's warp-level
// MMAs chained over the layer table (each layer padded to 128 units); the
// hidden-to-hidden layers' weights fill up to 139 KB of shared memory.
bool deep_wave_supported(const DevModel &m) {
    return m.precision == DLIC_INT8 && m.bits == 8 && m.layers != nullptr && !m.vol && default_window(m) &&
           m.nl != 3 && m.nl >= 2 && m.nl <= 6 && m.hmax <= kDecHidden;
}

static void (*wave_kernel(const DevModel &m, bool smma))(DevModel, DecBatch, DecTcParams) {
    if (deep_wave_supported(m)) return k_decode_tc_deep;
    // the default window runs the instance with its sizes as constants
    const bool def = default_window(m);
    if (m.precision == DLIC_FP32) return def ? k_decode_f32<true> : k_decode_f32<false>;
    if (smma) return def ? k_decode_tc<true, true> : k_decode_tc<false, true>;
    return def ? k_decode_tc<true, false> : k_decode_tc<false, false>;
}

// Dynamic shared memory a CTA of the kernel may take next to its static arrays.
static cudaError_t smem_limit(void (*kern)(DevModel, DecBatch, DecTcParams), uint32_t &limit) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    limit = (uint32_t)optin > fa.sharedSizeBytes ? (uint32_t)optin - (uint32_t)fa.sharedSizeBytes : 0u;
    return cudaSuccess;
}

// Shared-memory plan for images up to maxH x maxW in clusters of P CTAs
// within `limit` bytes.  In order of preference: the tagged ring; (INT8)
// smaller pixel chunks; the byte ring with one cluster barrier per wave;
// priors read back from the output image.  False when none fits.
static bool plan_wave(const DevModel &m, int maxH, int maxW, int maxD, int P, uint32_t limit, int plan,
                      DecTcParams &prm, bool smma_ok = true) {
    const bool f32 = m.precision == DLIC_FP32;
    const int wave_px = min(maxH, (maxW + 2) / 3);   // rows of the longest wave (per slice)
    const int per_cta = (wave_px + P - 1) / P + 1;
    prm = DecTcParams{};
    prm.P = P;
    prm.h1 = m.h1;
    prm.h2 = m.h2;
    prm.nt = f32 ? 12 : min(64, (per_cta + 15) & ~15);
    prm.smma = smma_ok && smma_chunk(m, per_cta) ? 1 : 0;
    if (deep_wave_supported(m)) {
        // (warp-level MMAs only, on chunks of up to kSmmaMaxChunk pixels)
        prm.deep = 1;
        prm.nhh = m.nl - 2;
        prm.smma = 1;
        prm.nt = min(kSmmaMaxChunk, prm.nt);
    }
    prm.k1 = (m.n_in + 15) / 16 * 16;
    prm.tslots = m.wu + 1;
    // ring columns kept per row: an entry must outlive its last reader,
    // 3 (rows above) + left reach waves later (plus a writer's lead of up
    // to P - 1 waves in the tagged ring)
    prm.tcols = 3 * m.wu + m.wl + P + 2 <= 32 ? 32 : 64;
    prm.rcols = 3 * m.wu + m.wl + 2 <= 16 ? 16 : 32;
    int rows = 1;
    while (rows < wave_px + m.wu + 2) rows <<= 1;
    prm.ring_rows = rows;
    prm.list_rows = (wave_px + 15) & ~15;
    prm.depth = 1;
    if (m.vol) {
        // a volume's wave holds the slices t - VSH z in [0, 3(H-1) + W), each
        // with at most ceil(wave_px / P) rows of a CTA (P divides S)
        const int active = min(maxD, (3 * (maxH - 1) + maxW) / volume_shift(m) + 1);
        prm.depth = maxD;
        prm.list_rows = (active * ((wave_px + P - 1) / P) + 15) & ~15;
    }
    // Tagged ring (neighbour-to-neighbour mode) only when it stays small.
    // Rows sharing a tagged-ring slot are P * tq apart: more than the rows
    // of a wave plus the rows above and a writer's lead (P - 1 waves), with
    // a round to spare.
    int tq = 0;
    if (P >= 2) {
        tq = 1;
        while (tq < (wave_px + m.wu + P + P - 1) / P + 1) tq <<= 1;
        if (4 * prm.tcols * prm.tslots * tq > 48 * 1024) tq = 0;
    }
    prm.tq = plan == DLIC_PLAN_AUTO && !m.vol ? tq : 0;
    prm.max_g = (min(maxH, 65535) + P - 1) / P;
    prm.pay_words = 0;
    auto size = [&] { return dec_layout(prm, f32).total; };
    // the expanded power-of-two table (6 KB) only where it costs no chunk size
    prm.lut2 = 1;
    if (size() > limit) prm.lut2 = 0;
    while (!f32 && size() > limit && prm.nt > 16) prm.nt -= 16;   // (chunks stay multiples of 16)
    if (size() > limit) prm.tq = 0;
    // volumes read every prior back from the output volume
    if (size() > limit || plan == DLIC_PLAN_IMAGE || m.vol) {
        prm.gimg = 1;
        prm.ring_rows = 0;
    }
    if (size() > limit) return false;
    // the payload of the owned streams is staged in what shared memory is
    // left (INT8; the FP32 decoder leaves it to the L1 cache)
    const uint32_t base = size(), budget = limit > 4096u ? limit - 4096u : 0u;
    prm.pay_words = !f32 && base < budget ? (int)((budget - base) / 2) & ~63 : 0;
    if (prm.pay_words > 65536) prm.pay_words = 65536;
    return true;
}

bool wave_decode_fits(const DevModel &m, int H, int W, int D, int P, int plan) {
    if (m.precision == DLIC_FP32 && default_window(m)) return true;   // the one-CTA decoder takes the rest
    uint32_t limit = 0;
    DecTcParams prm;
    // (the tcgen05 layout is the larger one, so it decides for both instances)
    return smem_limit(wave_kernel(m, false), limit) == cudaSuccess && plan_wave(m, H, W, D, P, limit, plan, prm, false);
}

// Launches one cluster of `cluster` CTAs per image of the batch (stepping
// down when a cluster that large cannot be scheduled).
cudaError_t launch_decode_tc(const DevModel &m, const DecBatch &b, int cluster, int num_sms, int plan,
                             cudaStream_t st, bool latency) {
    const bool f32 = m.precision == DLIC_FP32;
    if (b.n == 0) return cudaSuccess;
    int maxH = 1, maxW = 1, maxD = 1;
    for (int i = 0; i < b.n; i++) {
        maxH = max(maxH, b.img[i].H);
        maxW = max(maxW, b.img[i].W);
        maxD = max(maxD, b.img[i].D);
    }
    int P = cluster > 0 ? cluster : 1;
    // Warp-level MMAs when the call's clusters leave most SMs idle (a wave's
    // latency decides); when they fill the GPU, every SM's throughput does
    // and the tensor core's MMAs win at any chunk size.
    const bool smma = deep_wave_supported(m) || (latency && smma_chunk(m, wave_per_cta(maxH, maxW, P)));
    void (*kern)(DevModel, DecBatch, DecTcParams) = wave_kernel(m, smma);
    uint32_t limit = 0;
    cudaError_t e = smem_limit(kern, limit);
    if (e != cudaSuccess) return e;
    DecTcParams prm;
    if (!plan_wave(m, maxH, maxW, maxD, P, limit, plan, prm, smma))
        return f32 && default_window(m) ? launch_decode_cc(m, b, st) : cudaErrorNotSupported;
    const DecTcLayout L = dec_layout(prm, f32);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kDecThreads);
    cfg.dynamicSmemBytes = L.total;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // a 16-CTA cluster needs 16 free SMs in one GPC; step down if it cannot run
    for (;;) {
        attr[0].val.clusterDim.x = (unsigned)P;
        cfg.gridDim = dim3((unsigned)(b.n * P));
        int nclusters = 0;
        if (P == 1 || (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters > 0))
            break;
        cudaGetLastError();
        P >>= 1;
        if (P < 1) return cudaErrorInvalidConfiguration;
    }
    if (P != prm.P) {
        // smaller clusters hold more streams and pixels per CTA
        return launch_decode_tc(m, b, P, num_sms, plan, st, latency);
    }
    return cudaLaunchKernelEx(&cfg, kern, m, b, prm);
}

// One volume decoded by every SM: k_volume_setup, the wave kernel as a
// cooperative grid of one CTA per SM (co-residency is what makes its
// grid-wide barrier safe), then k_volume_finish.  Needs no two rows of a
// slice's wave on one stream (the wave's pixels go to any CTA) and fewer
// than 2^24 streams in the volume.
bool grid_decode_eligible(const DevModel &m, int H, int W, int D, int S) {
    return m.vol && min(H, (W + 2) / 3) <= S && (long long)D * S < (1ll << 24) && wave_decode_supported(m);
}

// Shared-memory plan of the grid decoder for a volume (b.img[0]) or a batch
// of 2D images; false when none fits.
static bool plan_grid(const DevModel &m, const DecBatch &b, int NB, uint32_t limit, DecTcParams &prm) {
    const bool f32 = m.precision == DLIC_FP32;
    prm = DecTcParams{};
    prm.P = 1;
    prm.h1 = m.h1;
    prm.h2 = m.h2;
    prm.k1 = (m.n_in + 15) / 16 * 16;
    prm.tslots = m.wu + 1;
    prm.tcols = 32;
    prm.rcols = 16;
    prm.gimg = 1;
    prm.max_g = 0;   // stream states live in the workspace
    long long wave = 0;   // pixels of the longest wave
    int designated = 0;   // pixels a CTA may get from whole (not spread) images
    if (m.vol) {
        const DecImage &im = b.img[0];
        const int wave_px = min(im.H, (im.W + 2) / 3), T2 = 3 * (im.H - 1) + im.W;
        const int active = min(im.D, T2 / volume_shift(m) + 1);
        wave = (long long)active * wave_px;
        prm.depth = im.D;
        prm.zlist = active + 1;
    } else {
        int maxw = 0;
        for (int i = 0; i < b.n; i++) {
            const int w = min(b.img[i].H, (b.img[i].W + 2) / 3);
            wave += w;
            maxw = max(maxw, w);
            prm.T = max(prm.T, 3 * (b.img[i].H - 1) + b.img[i].W);
        }
        designated = ((b.n + NB - 1) / NB) * maxw;
        prm.depth = 1;
        prm.zlist = 4 * (b.n + 1);
    }
    const int per_cta = (int)((wave + NB - 1) / NB);
    prm.nt = f32 ? 12 : min(64, max(16, (per_cta + 15) & ~15));
    prm.smma = smma_chunk(m, per_cta) ? 1 : 0;
    prm.list_rows = (per_cta + designated + 15) & ~15;
    prm.lut2 = 1;
    if (dec_layout(prm, f32).total > limit) prm.lut2 = 0;
    while (!f32 && dec_layout(prm, f32).total > limit && prm.nt > 16) prm.nt -= 16;   // (multiples of 16)
    return dec_layout(prm, f32).total <= limit;
}

// (both INT8 instances have the same static shared memory, so the plan is
// made against either's limit and then picks the instance)
static void (*grid_kernel(const DevModel &m, bool smma))(DevModel, DecBatch, DecTcParams) {
    return m.precision == DLIC_FP32 ? k_decode_grid_f32 : smma ? k_decode_grid_tc<true> : k_decode_grid_tc<false>;
}

bool grid_decode_fits(const DevModel &m, const DecBatch &b, int num_sms) {
    uint32_t limit = 0;
    DecTcParams prm;
    return wave_decode_supported(m) && smem_limit(grid_kernel(m, true), limit) == cudaSuccess &&
           plan_grid(m, b, num_sms, limit, prm);
}

cudaError_t launch_decode_grid(const DevModel &m, const DecBatch &b, int num_sms, cudaStream_t st) {
    uint32_t limit = 0;
    cudaError_t e = smem_limit(grid_kernel(m, true), limit);
    if (e != cudaSuccess) return e;
    const int NB = num_sms;
    DecTcParams prm;
    if (!plan_grid(m, b, NB, limit, prm)) return cudaErrorNotSupported;
    void (*kern)(DevModel, DecBatch, DecTcParams) = grid_kernel(m, prm.smma != 0);
    const DecTcLayout L = dec_layout(prm, m.precision == DLIC_FP32);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDecThreads, L.total);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorNotSupported;
    if (m.vol)
        k_volume_setup<<<1, kDecThreads, 0, st>>>(m, b);
    else
        k_batch_setup<<<b.n, kDecThreads, 0, st>>>(m, b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    DevModel ma = m;
    DecBatch ba = b;
    void *args[] = {&ma, &ba, &prm};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(kern), dim3((unsigned)NB), dim3(kDecThreads), args,
                                    L.total, st);
    if (e != cudaSuccess) return e;
    if (m.vol)
        k_volume_finish<<<1, kDecThreads, 0, st>>>(b);
    else
        k_batch_finish<<<b.n, kDecThreads, 0, st>>>(b);
    return cudaGetLastError();
}

// The grid decoder's set-up and final check of a 2D batch, for the other
// decoders that keep their stream states in the workspace.
cudaError_t launch_batch_setup(const DevModel &m, const DecBatch &b, cudaStream_t st) {
    k_batch_setup<<<b.n, kDecThreads, 0, st>>>(m, b);
    return cudaGetLastError();
}
cudaError_t launch_batch_finish(const DecBatch &b, cudaStream_t st) {
    k_batch_finish<<<b.n, kDecThreads, 0, st>>>(b);
    return cudaGetLastError();
}

}  // namespace dlic
