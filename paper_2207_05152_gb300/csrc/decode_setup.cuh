// Stream set-up of the one-CTA-per-image wavefront decoders (8-bit and
// 12-bit): the container header check and every stream's initial state.
#pragma once

#include "internal.cuh"

namespace dlic {

constexpr int kSetupThreads = 512;   // largest CTA that calls decode_setup

struct StreamState {
    uint32_t x, pos, end, pad;
};

__device__ __forceinline__ uint32_t rd_le32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

// Parses and checks the header, then sets up every stream's state from the
// word counts (CTAs of at most kSetupThreads threads).  Returns false
// (uniformly across the CTA) for a corrupt header.
__device__ inline bool decode_setup(const DevModel &m, const DecImage &im, const uint8_t *in, StreamState *st,
                                    int *S_out, const uint16_t **pay_out) {
    __shared__ int s_ok, s_S;
    __shared__ uint32_t s_part[kSetupThreads];
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
                 rd_le32(h + 4) == (uint32_t)im.H && rd_le32(h + 8) == (uint32_t)im.W && h[12] == m.wu &&
                 h[13] == (m.precision | (m.bits == 12 ? 0x10 : 0)) && hash == m.hash && S >= 1 && S <= im.H &&
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
    // 64-bit sums: no count, and no thread's share of the counts, may exceed
    // the input's word count (the host keeps that below 2^32), so the 32-bit
    // prefix sums below are exact for every header that passes
    const uint64_t max_words = im.in_bytes / 2;
    uint64_t sum = 0;
    int bad = 0;
    for (int s = s0; s < s1; s++) {
        const uint32_t c = rd_le32(cnt + 4 * s);
        bad |= c < 2;
        sum += c;
    }
    bad |= sum > max_words;
    s_part[tid] = (uint32_t)sum;
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

}  // namespace dlic
