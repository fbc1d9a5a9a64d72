// Internal declarations shared by the translation units of libdlic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/dlic.h"

namespace dlic {

constexpr int kPriors = 12;        // priors of the default radius-2 causal window
constexpr int kMaxPriors = 96;     // largest window: rows up <= 8, left reach <= 8, right reach <= 2
constexpr int kSymbols = 256;      // 8-bit alphabet
constexpr int kSymbols12 = 4096;   // 12-bit alphabet (Sec. IV "Higher Bit Depth")
constexpr uint32_t kRansL = 1u << 16;
constexpr uint32_t kTotal = 1u << 16;
constexpr uint32_t kQuantTotal = 65280u;   // 2^16 - 256: mass shared out by the PDF
constexpr int kHeaderBytes = 24;
constexpr int kMaxHidden = 256;

// Device-side view of a model (passed to kernels by value).
// One dense layer of a network of other than two hidden layers, transposed
// like the fixed-depth arrays below: FP32 w = W^T [in][out] (f32), a = bias;
// INT8 w = [in / 4][out] (u32, 4 inputs per word), a = scale s, o = offset.
struct DevLayer {
    const void *w;
    const float *a, *o;
    int32_t n_in, n_out;
    // wide INT8 networks, layers after the first: the weights as bf16
    // [n_out][wtc_pitch] for the tensor-core encoder (wide_tc.cu), else null
    const uint16_t *wtc;
    int32_t wtc_pitch;
};
constexpr int kMaxLayers = 9;     // deeper networks: up to 8 hidden layers and the output layer

struct DevModel {
    int precision;   // DLIC_FP32 / DLIC_INT8
    int h1, h2;      // first and last hidden widths
    // dense layers (3 for two hidden layers); a network of other depth runs
    // on the one-pixel-per-thread kernels from the layer table, whose widest
    // hidden layer has hmax units
    int nl, hmax;
    const DevLayer *layers;       // device array of nl entries (other depths, 12-bit models)
    int bits;                     // 8, or 12: u16 samples, 4096 outputs, FP32 layer-table kernels
    // causal window: rows r-wu..r-1 at columns c-wl..c+wr, then row r at
    // columns c-wl..c-1 (n2 priors in that order); (2, 2, 2) by default.
    // A 3D window (vol = 1) adds the previous slice's rows r-pu..r+pd at
    // columns c-pl..c+pr (Sec. IV "3D Dependencies"): n_in = n2 + n3.
    int wu, wl, wr, n_in;
    int vol, pu, pd, pl, pr, n2;
    float tscale;
    const uint32_t *lut;          // 64 entries
    // FP32 network, transposed: WkT[k * out + j] = W[j][k] (a 12-bit model
    // keeps here its output layer in the decoder's 16 x 256 tiles)
    const float *w1t, *b1, *w2t, *b2, *w3t, *b3;
    // INT8 network, packed 4 inputs per u32 and transposed:
    // QkT[k4 * out + j] = bytes W[j][4*k4 .. 4*k4+3]
    const uint32_t *q1t, *q2t, *q3t;
    const float *s1, *o1, *s2, *o2, *s3, *o3;
    // INT8 network as bf16 (integer-valued) in tcgen05 shared-memory layout
    const uint16_t *tc_w;         // packed image of W1|W2|W3 operand tiles
    uint32_t tc_w_bytes;
    uint64_t hash;
    // clock cycles a wavefront decoder waits for another CTA (a tagged-ring
    // entry of a neighbour, the grid-wide wave barrier) before it gives up
    // with DLIC_ERR_TIMEOUT; waits on the CTA's own tensor-core work and
    // bulk copies keep their own, fixed limit
    long long peer_wait_limit;
};

constexpr long long kDefaultPeerWaitLimit = 4000000000LL;   // about 2 s at 2 GHz

// Per-image encode descriptor.
struct EncImage {
    const uint8_t *pixels;
    const uint8_t *below;         // previous slice of a volume (3D window), or null
    int64_t pitch;
    int32_t H, W, S;
    int32_t tile_begin;           // first 128-pixel tile of this image
    uint64_t fc_off;              // u32 (f | c << 16) per pixel, stream order
    uint64_t words_off;           // u16 renormalisation words, per stream region
    uint64_t cnt_off;             // u32 words per stream (incl. 2 flush words)
    uint64_t xfin_off;            // u32 final state per stream
    uint64_t soff_off;            // u32 payload offset of each stream (words)
};

constexpr int kMaxBatch = 192;    // images per launch (kernel-parameter space)
constexpr int kMaxSlices = 2047;  // slices per volume (11 bits in the decoder's row list)
// a 2D batch goes to the grid decoder when its clusters would fill at most
// half the SMs with more than this many pixels per CTA and wave
constexpr int kGridMinChunkPixels = 64;
constexpr int kPredictTile = 64;  // pixels per CUDA-core prediction CTA

struct EncBatch {
    int n;
    int chunk_start;              // index of img[0] in the caller's batch
    int tile_px;                  // pixels per prediction tile
    int total_tiles;
    uint8_t *ws;                  // workspace base
    uint64_t *sizes;              // per image bitstream bytes (in workspace)
    int raster;                   // 1: (f, c) per pixel in raster order (dlic_predict), else stream order
    EncImage img[kMaxBatch];
};

struct DecImage {
    uint8_t *pixels;
    int64_t pitch;
    int64_t slice_pitch;          // volumes: bytes between slices
    int32_t H, W;
    int32_t D;                    // slices (1 for a 2D image)
    int32_t S;                    // volumes: the caller's stream count per slice
    uint64_t in_off;              // byte offset of the bitstream in d_in
    uint64_t in_bytes;
    uint64_t st_off;              // per-stream state (x, pos, end) in workspace
    int32_t sidx;                 // index of the image's status word
};

struct DecBatch {
    int n;
    const uint8_t *in;
    uint8_t *ws;
    int32_t *status;
    DecImage img[kMaxBatch];
};

// Stream states of a decode in the workspace, at im.st_off: a 256-byte
// header (stream count, ok flag, wave-barrier counter, failure flag, whether
// no wave holds two rows of one stream), then x, position (16-bit words from
// the start of the input) and end of every stream (z S + s).
struct VolState {
    uint32_t *hdr, *x, *pos, *end;
};
__host__ __device__ inline size_t vol_state_bytes(int D, int S) { return 256 + 12ull * D * S; }
__device__ __forceinline__ VolState vol_state(const DecBatch &b, const DecImage &im) {
    VolState v;
    v.hdr = reinterpret_cast<uint32_t *>(b.ws + im.st_off);
    v.x = v.hdr + 64;
    v.pos = v.x + (size_t)im.D * im.S;
    v.end = v.pos + (size_t)im.D * im.S;
    return v;
}

// Sets the thread-local error text and returns the code.
dlic_status fail(dlic_status code, const char *fmt, ...);
dlic_status cuda_fail(cudaError_t e, const char *what);

// Kernel launchers (coder_cc.cu, coder_tc.cu, rans.cu)
cudaError_t launch_predict_cc(const DevModel &m, const EncBatch &b, cudaStream_t st);
cudaError_t launch_predict_tc(const DevModel &m, const EncBatch &b, int *err, int num_sms, cudaStream_t st);
bool tc_supported(const DevModel &m);
size_t tc_weight_bytes(int h1, int h2, int k1);
void tc_pack_weights(int h1, int h2, int n_in, int k1, const int8_t *q1, const int8_t *q2, const int8_t *q3,
                     uint16_t *out);
bool f32_predict_supported(const DevModel &m);
cudaError_t launch_rans_encode(const EncBatch &b, int total_streams, cudaStream_t st);
cudaError_t launch_pack(const DevModel &m, const EncBatch &b, uint8_t *out,
                        uint64_t *out_offsets, cudaStream_t st);
cudaError_t launch_decode(const DevModel &m, const DecBatch &b, cudaStream_t st);
// Decoders (coder_cc.cu: one CTA per image; decode_tc.cu: one cluster per
// image, wavefront)
cudaError_t launch_decode_cc(const DevModel &m, const DecBatch &b, cudaStream_t st);
// 12-bit pixels (coder12.cu): warp-per-pixel FP32 kernels over the layer table
cudaError_t launch_predict12(const DevModel &m, const EncBatch &b, int *err, cudaStream_t st);
cudaError_t launch_decode12(const DevModel &m, const DecBatch &b, cudaStream_t st);
// Networks with hidden layers wider than 256 (wide.cu): one layer at a time
// over sets of pixels, activations in a workspace scratch of
// wide_scratch_bytes (encode: INT8 activations as the tensor-core layers'
// bf16 inputs); hl is the host copy of the layer table
bool wide_supported(const DevModel &m);
size_t wide_scratch_bytes(const DevModel &m, bool encode);
cudaError_t launch_predict_wide(const DevModel &m, const DevLayer *hl, const EncBatch &b, uint8_t *scratch,
                                int *err, cudaStream_t st);
// one INT8 layer of a wide network's encode pass on the tensor cores
// (wide_tc.cu): X the previous layer's u8 units as bf16 [np][ldx]
cudaError_t launch_wide_tc(const DevLayer &ly, const uint16_t *X, int ldx, int np, void *Y, int ldy, bool logits,
                           int num_sms, int *err, cudaStream_t st);
cudaError_t launch_decode_wide(const DevModel &m, const DevLayer *hl, const DecBatch &b, uint8_t *scratch,
                               cudaStream_t st);
// the grid decoder's stream-state set-up and final check (decode_tc.cu)
cudaError_t launch_batch_setup(const DevModel &m, const DecBatch &b, cudaStream_t st);
cudaError_t launch_batch_finish(const DecBatch &b, cudaStream_t st);
// latency: the call's clusters leave most SMs idle (warp-level MMAs for small chunks)
cudaError_t launch_decode_tc(const DevModel &m, const DecBatch &b, int cluster, int num_sms, int plan, cudaStream_t st,
                             bool latency);
bool wave_decode_supported(const DevModel &m);
// INT8 networks of 1..5 hidden layers of widths up to 128 on the same decoder
bool deep_wave_supported(const DevModel &m);
// whether an H x W image decodes in clusters of P CTAs (some shared-memory plan fits)
bool wave_decode_fits(const DevModel &m, int H, int W, int D, int P, int plan);
// a volume on every SM at once (cooperative grid) instead of one cluster
bool grid_decode_eligible(const DevModel &m, int H, int W, int D, int S);
cudaError_t launch_decode_grid(const DevModel &m, const DecBatch &b, int num_sms, cudaStream_t st);
// whether a batch of 2D images (or one volume) fits the grid decoder's shared-memory plan
bool grid_decode_fits(const DevModel &m, const DecBatch &b, int num_sms);
void choose_clusters(const int *H, const int *W, int n, int num_sms, bool f32, int *P);
double decode_estimate(int H, int W, int P, bool f32);   // cycles, the autotuner's cost model

// Rows of stream s (rows s, s + S, ...) and the first entry of its region in
// stream-ordered per-pixel buffers: every earlier stream holds W pixels per
// row.  Word scratch regions add the two flush words of each earlier stream.
__host__ __device__ inline int64_t stream_rows(int H, int S, int s) {
    return (H - s + S - 1) / S;
}
__host__ __device__ inline int64_t stream_pix_base(int H, int W, int S, int s) {
    const int64_t rows_before = (int64_t)(H / S) * s + (s < H % S ? s : H % S);
    return rows_before * W;
}
__host__ __device__ inline int64_t stream_word_base(int H, int W, int S, int s) {
    return stream_pix_base(H, W, S, s) + 2 * (int64_t)s;
}

// Position of pixel (r, c) within its stream s = r mod S, whose pixels are
// ordered by wave t = 3r + c, then by row.  The pixels before it are, for
// every row r_k = s + kS of the stream, those of its columns that lie on an
// earlier wave (clamp(t - 3 r_k, 0, W) of them), plus the pixels of earlier
// rows of the stream on the same wave.
__host__ __device__ inline int64_t stream_pos(int H, int W, int S, int r, int c) {
    const int s = r % S;
    const int64_t kr = r / S;
    const int64_t n = stream_rows(H, S, s);
    const int64_t D = 3LL * S;
    const int64_t a0 = 3LL * r + c - 3LL * s;
    int64_t k1 = 0, k2 = 0;
    if (a0 >= W) {
        k1 = (a0 - W) / D + 1;
        k1 = k1 < n ? k1 : n;
    }
    if (a0 >= 1) {
        k2 = (a0 - 1) / D + 1;
        k2 = k2 < n ? k2 : n;
    }
    const int64_t before = (int64_t)W * k1 + (k2 - k1) * a0 - D * (k2 * (k2 - 1) / 2 - k1 * (k1 - 1) / 2);
    const int64_t same_wave = (W - c - 1) / D;
    return before + (kr < same_wave ? kr : same_wave);
}

// Offsets (dr, dc) of prior q of the model's window.
// (slice, row, column) offset of prior q: dz = -1 for the previous slice
__host__ __device__ inline void window_offset(const DevModel &m, int q, int &dz, int &dr, int &dc) {
    const int wid = m.wl + m.wr + 1;
    dz = 0;
    if (q < m.wu * wid) {
        dr = -m.wu + q / wid;
        dc = -m.wl + q % wid;
    } else if (q < m.n2) {
        dr = 0;
        dc = -m.wl + (q - m.wu * wid);
    } else {
        const int wid3 = m.pl + m.pr + 1, k = q - m.n2;
        dz = -1;
        dr = -m.pu + k / wid3;
        dc = -m.pl + k % wid3;
    }
}
__host__ __device__ inline bool default_window(const DevModel &m) {
    return m.wu == 2 && m.wl == 2 && m.wr == 2 && !m.vol;
}
// waves by which a slice lags the one before in the 3D wavefront
__host__ __device__ inline int volume_shift(const DevModel &m) { return 3 * m.pd + m.pr + 1; }

// Index of pixel (r, c) in the stream-ordered per-pixel table buffer.
__host__ __device__ inline int64_t stream_index(int H, int W, int S, int r, int c) {
    return stream_pix_base(H, W, S, r % S) + stream_pos(H, W, S, r, c);
}

}  // namespace dlic
