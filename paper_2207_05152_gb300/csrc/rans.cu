// Interleaved rANS encoding and bitstream packing (Sec. II-B "rANS": many
// coder instances with their own bitstreams, at most one per pixel row,
// 32-bit arithmetic on the GPU).
//
// Coder constants: state x in [2^16, 2^32), 16-bit renormalisation words,
// tables summing to M = 2^16.  Encoding a symbol with frequency f and
// cumulative count c:
//     if x >= f * 2^16: emit x & 0xFFFF, x >>= 16     (at most one word)
//     x = (x / f) * 2^16 + (x mod f) + c
// A stream starts from x = 2^16 and its pixels are encoded in the reverse
// of the order the decoder meets them: waves t = 3r + c descending, rows
// descending within a wave.
#include "internal.cuh"

namespace dlic {

// One rANS step.  The quotient x / f comes from a single-precision
// reciprocal estimate corrected to the exact value: x < f * 2^16 after
// renormalisation, so the estimate is within one of the quotient.
__device__ __forceinline__ uint32_t rans_put(uint32_t x, uint32_t v, uint16_t *words, uint32_t &ne) {
    const uint32_t f = v & 0xFFFFu, c = v >> 16;
    const float rf = __frcp_rn((float)f);
    if (x >= (f << 16)) {
        words[ne++] = (uint16_t)(x & 0xFFFFu);
        x >>= 16;
    }
    int q = __float2int_rz(__fmul_rz(__uint2float_rz(x), rf));
    int rem = (int)(x - (uint32_t)q * f);
    if (rem < 0) {
        q -= 1;
        rem += (int)f;
    } else if (rem >= (int)f) {
        q += 1;
        rem -= (int)f;
    }
    return ((uint32_t)q << 16) + (uint32_t)rem + c;
}

// One thread per (image, stream).  The stream's (f, c) entries are stored
// in stream order, so the thread walks them backwards from the last symbol
// with the next batch of loads in flight.  Words are written in emission
// order to the stream's scratch region; pack reverses them.
__global__ void k_rans_encode(EncBatch b, int total_streams) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total_streams) return;
    int ii = 0, first = 0;
    while (ii < b.n && g >= first + b.img[ii].S) {
        first += b.img[ii].S;
        ii++;
    }
    const EncImage &im = b.img[ii];
    const int s = g - first;
    const int H = im.H, W = im.W, S = im.S;
    const uint32_t *fc = reinterpret_cast<const uint32_t *>(b.ws + im.fc_off) + stream_pix_base(H, W, S, s);
    uint16_t *words = reinterpret_cast<uint16_t *>(b.ws + im.words_off) + stream_word_base(H, W, S, s);
    const int64_t n = stream_rows(H, S, s) * W;
    uint32_t x = kRansL;
    uint32_t ne = 0;
    constexpr int B = 8;
    uint32_t cur[B], nxt[B];
    int64_t j = n - 1;
#pragma unroll
    for (int u = 0; u < B; u++) cur[u] = j - u >= 0 ? __ldg(fc + j - u) : 0u;
    while (j >= 0) {
        const int64_t jn = j - B;
#pragma unroll
        for (int u = 0; u < B; u++) nxt[u] = jn - u >= 0 ? __ldg(fc + jn - u) : 0u;
#pragma unroll
        for (int u = 0; u < B; u++)
            if (j - u >= 0) x = rans_put(x, cur[u], words, ne);
#pragma unroll
        for (int u = 0; u < B; u++) cur[u] = nxt[u];
        j = jn;
    }
    reinterpret_cast<uint32_t *>(b.ws + im.cnt_off)[s] = ne + 2;
    reinterpret_cast<uint32_t *>(b.ws + im.xfin_off)[s] = x;
}

// Per image: exclusive scan of the stream word counts -> payload offsets,
// and the image's bitstream size.
__global__ void k_stream_offsets(EncBatch b) {
    __shared__ uint32_t part[256];
    const EncImage &im = b.img[blockIdx.x];
    const int S = im.S, tid = threadIdx.x, nth = blockDim.x;
    const uint32_t *cnt = reinterpret_cast<const uint32_t *>(b.ws + im.cnt_off);
    uint32_t *soff = reinterpret_cast<uint32_t *>(b.ws + im.soff_off);
    const int per = (S + nth - 1) / nth;
    const int s0 = min(S, tid * per), s1 = min(S, s0 + per);
    uint32_t sum = 0;
    for (int s = s0; s < s1; s++) sum += cnt[s];
    part[tid] = sum;
    __syncthreads();
    if (tid == 0) {
        uint32_t acc = 0;
        for (int k = 0; k < nth; k++) {
            const uint32_t v = part[k];
            part[k] = acc;
            acc += v;
        }
        b.sizes[blockIdx.x] = (uint64_t)kHeaderBytes + 4ull * S + 2ull * acc;
    }
    __syncthreads();
    uint32_t acc = part[tid];
    for (int s = s0; s < s1; s++) {
        soff[s] = acc;
        acc += cnt[s];
    }
}

// Byte offsets of the images in the output (one CTA, n <= kMaxBatch).
__global__ void k_image_offsets(EncBatch b, uint64_t *out_offsets) {
    if (threadIdx.x == 0) {
        // a later chunk continues after the previous chunk's last bitstream
        uint64_t acc = b.chunk_start ? out_offsets[0] : 0;
        for (int i = 0; i < b.n; i++) {
            out_offsets[i] = acc;
            acc += b.sizes[i];
        }
        out_offsets[b.n] = acc;
    }
}

// Writes header, word counts and payloads; one CTA per image, one warp per
// stream at a time.
// Container assembly: blockIdx.y = image; block x = 0 writes the header and
// the word counts; every block's warps copy whole streams (one warp per
// stream, strided over the blocks of the image).
__global__ void k_pack(DevModel m, EncBatch b, uint8_t *out, const uint64_t *out_offsets) {
    const EncImage &im = b.img[blockIdx.y];
    const int S = im.S, tid = threadIdx.x;
    uint8_t *o = out + out_offsets[blockIdx.y];
    const uint32_t *cnt = reinterpret_cast<const uint32_t *>(b.ws + im.cnt_off);
    const uint32_t *xfin = reinterpret_cast<const uint32_t *>(b.ws + im.xfin_off);
    const uint32_t *soff = reinterpret_cast<const uint32_t *>(b.ws + im.soff_off);
    const uint16_t *words = reinterpret_cast<const uint16_t *>(b.ws + im.words_off);
    if (blockIdx.x == 0 && tid < kHeaderBytes) {
        uint8_t v;
        if (tid < 4) v = "DLC1"[tid];
        else if (tid < 8) v = (uint8_t)((uint32_t)im.H >> (8 * (tid - 4)));
        else if (tid < 12) v = (uint8_t)((uint32_t)im.W >> (8 * (tid - 8)));
        else if (tid == 12) v = (uint8_t)(m.wu | (m.vol ? 0x80 : 0));   // window rows above; bit 7: a volume's slice
        else if (tid == 13) v = (uint8_t)(m.precision | (m.bits == 12 ? 0x10 : 0));   // bit 4: 12-bit pixels
        else if (tid < 16) v = (uint8_t)((uint32_t)S >> (8 * (tid - 14)));
        else v = (uint8_t)(m.hash >> (8 * (tid - 16)));
        o[tid] = v;
    }
    for (int s = tid; blockIdx.x == 0 && s < S; s += blockDim.x) {
        const uint32_t c = cnt[s];
        o[kHeaderBytes + 4 * s + 0] = (uint8_t)c;
        o[kHeaderBytes + 4 * s + 1] = (uint8_t)(c >> 8);
        o[kHeaderBytes + 4 * s + 2] = (uint8_t)(c >> 16);
        o[kHeaderBytes + 4 * s + 3] = (uint8_t)(c >> 24);
    }
    uint16_t *pay = reinterpret_cast<uint16_t *>(o + kHeaderBytes + 4 * S);
    const int lane = tid & 31, nwarp = blockDim.x >> 5;
    for (int s = blockIdx.x * nwarp + (tid >> 5); s < S; s += gridDim.x * nwarp) {
        const uint32_t n = cnt[s] - 2, base = soff[s];
        const uint16_t *src = words + stream_word_base(im.H, im.W, S, s);
        if (lane == 0) {
            pay[base] = (uint16_t)(xfin[s] >> 16);
            pay[base + 1] = (uint16_t)(xfin[s] & 0xFFFFu);
        }
        for (uint32_t k = lane; k < n; k += 32) pay[base + 2 + k] = src[n - 1 - k];
    }
}

cudaError_t launch_rans_encode(const EncBatch &b, int total_streams, cudaStream_t st) {
    if (total_streams == 0) return cudaSuccess;
    k_rans_encode<<<(total_streams + 63) / 64, 64, 0, st>>>(b, total_streams);
    return cudaGetLastError();
}

cudaError_t launch_pack(const DevModel &m, const EncBatch &b, uint8_t *out, uint64_t *out_offsets,
                        cudaStream_t st) {
    if (b.n == 0) return cudaSuccess;
    k_stream_offsets<<<b.n, 256, 0, st>>>(b);
    k_image_offsets<<<1, 32, 0, st>>>(b, out_offsets);
    int max_s = 1;
    for (int i = 0; i < b.n; i++) max_s = max_s > b.img[i].S ? max_s : b.img[i].S;
    // up to 8 streams per block; at most 1024 blocks per image
    const int nblk = (max_s + 7) / 8 < 1024 ? (max_s + 7) / 8 : 1024;
    k_pack<<<dim3(nblk, b.n), 256, 0, st>>>(m, b, out, out_offsets);
    return cudaGetLastError();
}

}  // namespace dlic
