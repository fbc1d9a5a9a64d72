/*
 * dlic.h - C ABI of the DLIC coding library (CUDA, sm_103a).
 *
 * DLIC (Barzen, Glazov, Geistert, Sikora, "Accelerated Deep Lossless Image
 * Coding with Unified Parallelized GPU Coding Architecture") codes an 8-bit
 * grayscale image pixel by pixel: a small dense network estimates the PDF of
 * each pixel from its causal neighbours (Eq. 1, Sec. II-A), the PDF drives
 * an rANS entropy coder (Sec. II-B "rANS"), and encoding and decoding run on
 * the GPU as wavefronts so that every pixel whose neighbours are known is
 * coded in parallel (Sec. II-B "Preprocessor", Fig. 1 right).  The whole
 * coder runs on the device; the host only moves the image in and the
 * bitstream out (Sec. II-B, last paragraph of "Preprocessor").
 *
 * Conventions shared by every call:
 *  - Pointers named d_* are device pointers (cudaMalloc'd or equivalent) on
 *    the current CUDA device; pointers named h_* are host pointers.  The
 *    caller owns all of them.  The library allocates device memory only in
 *    dlic_model_create and dlic_trainer_create and frees it in the matching
 *    destroy call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue work on it and return without synchronising.
 *  - Errors the host can see (bad arguments, too small buffers) are returned
 *    at once and nothing is enqueued; dlic_last_error() then describes them.
 *    Errors found by the device (a corrupt bitstream, a wait that timed out)
 *    are written to the per-image d_status array of the decoding call.
 *  - Every call is thread-safe for distinct output buffers; a model may be
 *    shared by concurrent calls on different streams.
 */
#ifndef DLIC_H
#define DLIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DLIC_API __attribute__((visibility("default")))
#else
#define DLIC_API
#endif

typedef enum {
    DLIC_OK = 0,
    DLIC_ERR_INVALID = 1,      /* bad argument or malformed model blob */
    DLIC_ERR_CAPACITY = 2,     /* output or workspace buffer too small */
    DLIC_ERR_CORRUPT = 3,      /* bitstream does not decode (device status) */
    DLIC_ERR_TIMEOUT = 4,      /* a device-side wait ran out (device status) */
    DLIC_ERR_CUDA = 5,         /* a CUDA runtime call failed */
    DLIC_ERR_UNSUPPORTED = 6   /* valid request this build does not support */
} dlic_status;

enum { DLIC_FP32 = 0, DLIC_INT8 = 1 };

typedef struct dlic_model dlic_model;
typedef struct dlic_trainer dlic_trainer;

/* One grayscale image in device memory: row r starts at pixels + r * pitch
 * (pitch in bytes).  With a model of 256 outputs the samples are 8-bit
 * (uint8_t, pitch >= width); with a model of 4096 outputs (12-bit pixels,
 * Sec. IV "Higher Bit Depth") they are uint16_t values 0..4095, pixels
 * 2-byte aligned, pitch even and >= 2 * width; dlic_encode refuses an
 * image with a sample above 4095 by writing DLIC_ERR_INVALID to its status
 * word).  dlic_encode only reads the pixels, dlic_decode writes them. */
typedef struct {
    uint8_t *pixels;
    int32_t height;
    int32_t width;
    int64_t pitch;
} dlic_image;

/* A volume of `depth` slices of height x width 8-bit pixels in device memory
 * (Sec. IV: scans coded with a 3D window): slice z starts at
 * pixels + z * slice_pitch (slice_pitch >= pitch * height), its row r at
 * + r * pitch.  streams: the rANS streams of every slice, at most one per
 * row (0 = dlic_auto_streams when encoding; when decoding, the count in the
 * slices' headers, from dlic_read_header).  depth <= 2047. */
typedef struct {
    uint8_t *pixels;
    int32_t depth;
    int32_t height;
    int32_t width;
    int32_t streams;
    int64_t pitch;
    int64_t slice_pitch;
} dlic_volume;

/* Thread-local description of the last error returned by this thread. */
DLIC_API const char *dlic_last_error(void);

/* ---------------------------------------------------------------------- */
/* Models                                                                 */
/* ---------------------------------------------------------------------- */

/* Creates a coder model from a model blob (host memory, little-endian):
 *   "DLM1", u32 precision (DLIC_FP32 / DLIC_INT8), u32 n_in, u32 h1, u32 h2,
 *   u32 256, u32 window, f32 tscale, u32 lut[64], then the three dense
 *   layers (FP32: W f32[out][in] and b f32[out] per layer; INT8: W i8[out][in],
 *   s f32[out], o f32[out] per layer).
 * The network maps the causal priors of a pixel to 256 logits (Sec. II-B,
 * "Neural Network Architecture": dense layers, a 256-way softmax output).
 * The window ("any window shape", Sec. II-A) is window = 2 for the default
 * 12 priors (rows r-2, r-1 at columns c-2..c+2, then (r, c-2), (r, c-1)), or
 * 1 << 24 | u | l << 8 | rr << 16 for rows r-u..r-1 at columns c-l..c+rr,
 * then row r at columns c-l..c-1 (1 <= u <= 8, l <= 8, rr <= 2, so that
 * wave t = 3r + c stays valid), with n_in = u (l + rr + 1) + l priors; the
 * 9 x 9 window of Fig. 6 is (8, 6, 2), 78 priors.  A 3D window (see the
 * volume calls below) adds a layer from the previous slice.  Windows other
 * than the default need the tensor-core INT8 kernels (h1, h2 <= 128 to
 * encode, h1 = h2 = 128 to decode) or the FP32 tiled kernels (h2 <= 128)
 * (DLIC_ERR_UNSUPPORTED otherwise).
 * h1 and h2 must be multiples of 16 in [16, 256].
 * Networks of other depths (Sec. II-B: the paper's network has six dense
 * layers) come as
 *   "DLM2", u32 precision, u32 n_in, u32 L (hidden layers, 1..8),
 *   u32 widths[8] (the L hidden widths, then zeros), u32 256, u32 window,
 *   f32 tscale, u32 0, u32 lut[64], then the L + 1 dense layers as above.
 * With L = 2 it is the same network as the "DLM1" blob and runs the same
 * kernels.  Other L run on the CUDA-core one-pixel-per-thread encoder and
 * decoder, with the default window only and hidden widths that are
 * multiples of 4 in [4, 256] (DLIC_ERR_UNSUPPORTED otherwise).
 * 12-bit pixels (Sec. IV "Higher Bit Depth"): n_out = 4096 in either blob,
 * an FP32 network (DLIC_ERR_INVALID for INT8), network inputs v / 2048 - 1,
 * the frequency tables of 2^16 with 4096 values (each f >= 1); the default
 * window and hidden widths that are multiples of 4 in [4, 256]
 * (DLIC_ERR_UNSUPPORTED otherwise); CUDA-core warp-per-pixel kernels.
 * The blob is copied; the model owns device copies of the weights in the
 * layouts the kernels use.
 * The model hash (FNV-1a 64 of the blob) is written into every bitstream and
 * checked by the decoder.  Returns DLIC_ERR_INVALID for a malformed blob. */
DLIC_API dlic_status dlic_model_create(const void *h_blob, size_t blob_bytes, dlic_model **out);

/* Frees the model's device memory.  No call using the model may still be in
 * flight on any stream. */
DLIC_API dlic_status dlic_model_destroy(dlic_model *model);

/* How the wavefront decoder keeps the priors of the pixels it decodes
 * (Sec. II-B: a pixel's priors are pixels of earlier waves).
 *  DLIC_PLAN_AUTO        the fastest plan whose shared memory fits: a
 *                        tagged ring that CTAs of a cluster write into one
 *                        another's shared memory (no per-wave barrier), else
 *                        a byte ring with one cluster barrier per wave, else
 *                        the priors read back from the output image;
 *  DLIC_PLAN_BYTE_RING   the byte ring, or the image when it does not fit;
 *  DLIC_PLAN_IMAGE       always the image (one cluster barrier per wave);
 *  DLIC_PLAN_GRID        the whole batch on every SM at once: one cooperative
 *                        grid of one CTA per SM, each wave's pixels (of all
 *                        images) split evenly over the CTAs, priors read back
 *                        from the images, stream states in the workspace, one
 *                        grid-wide barrier per wave.  AUTO takes it for
 *                        volumes (when no slice's wave holds two rows of one
 *                        stream) and for 2D batches whose clusters would fill
 *                        at most half the SMs with more than 64 pixels per CTA
 *                        and wave (a few very wide images).
 * Every plan gives the same decoded pixels; the forced plans exist to test
 * and measure the ones AUTO takes for long waves.  Applies to later
 * dlic_decode and dlic_decode_volume calls with this model;
 * DLIC_ERR_INVALID for another value. */
enum { DLIC_PLAN_AUTO = 0, DLIC_PLAN_BYTE_RING = 1, DLIC_PLAN_IMAGE = 2, DLIC_PLAN_GRID = 3 };
DLIC_API dlic_status dlic_model_set_decode_plan(dlic_model *model, int plan);

/* How long (in SM clock cycles) the wavefront decoders of this model wait
 * for another CTA before giving up: a pixel that a neighbouring CTA of the
 * cluster pushes into the tagged ring, or the grid-wide wave barrier of
 * DLIC_PLAN_GRID.  The default, 4e9 cycles (about 2 s), is restored by
 * cycles <= 0.  A wait that runs out makes the decoder stop waiting for the
 * rest of the call, finish every wave without further waits on other CTAs
 * (still waiting for its own tensor-core work and bulk copies, which always
 * complete), and report DLIC_ERR_TIMEOUT in the image's d_status; the
 * decoded pixels are then invalid and the device stays usable.  A limit of a
 * few hundred cycles makes such waits run out on purpose, which is how the
 * error path is tested.  Not part of the paper's method: a diagnostic of
 * this library.  Applies to later decode calls with this model. */
DLIC_API dlic_status dlic_model_set_peer_wait_limit(dlic_model *model, long long cycles);

/* Precision tag, first and last hidden widths and hash of a model. */
DLIC_API dlic_status dlic_model_info(const dlic_model *model, int *precision, int *h1, int *h2,
                            uint64_t *hash);

/* ---------------------------------------------------------------------- */
/* Encoding (Sec. II-A Fig. 2 left; Sec. II-B)                             */
/* ---------------------------------------------------------------------- */

/* Upper bound, in bytes, of the bitstream of one height x width image coded
 * with `streams` rANS streams (clipped to the height): a 24-byte header,
 * 4 bytes per stream, and at most one 16-bit word per pixel plus two flush
 * words per stream. */
DLIC_API size_t dlic_max_encoded_bytes(int height, int width, int streams);

/* Stream count the library picks when the caller passes none: at least one
 * stream per pixel a wave can hold, ceil(width / 3) rounded up to a multiple
 * of 16, but at most one per row (Sec. II-B "rANS": at most one coder
 * instance per row): min(height, 16 * ceil(ceil(width / 3) / 16)).  No two
 * pixels of a wave share a stream, and the decoder can split the streams
 * evenly over clusters of up to 16 CTAs. */
DLIC_API int dlic_auto_streams(int height, int width);

/* Device workspace, in bytes, that dlic_encode needs for this batch. */
DLIC_API dlic_status dlic_encode_workspace_size(const dlic_model *model, const dlic_image *h_images, int n,
                                       const int *h_streams, size_t *bytes);

/* Encodes n images (descriptors in host memory, pixels on the device).
 *  h_streams:     n stream counts, or NULL for dlic_auto_streams; each is
 *                 clipped to its image height (at most one stream per row,
 *                 Sec. II-B "rANS") and must be in [1, 65535].
 *  d_out:         receives the n bitstreams back to back; out_capacity must
 *                 be at least the sum of dlic_max_encoded_bytes over the
 *                 batch (checked on the host: DLIC_ERR_CAPACITY).
 *  d_out_offsets: n + 1 u64 byte offsets written by the device; bitstream i
 *                 occupies [d_out_offsets[i], d_out_offsets[i + 1]).
 *  d_status:      one int32 on the device, or NULL; receives DLIC_OK,
 *                 DLIC_ERR_TIMEOUT if a tensor-core wait ran out, or
 *                 DLIC_ERR_INVALID if a 12-bit sample exceeds 4095 (the
 *                 output is then invalid).
 *  d_workspace:   at least dlic_encode_workspace_size bytes, 256-aligned.
 * Bitstream layout (little-endian): "DLC1", u32 height, u32 width,
 * u8 window rows u (2 for the default window), u8 precision, u16 S, u64
 * model hash, u32 words[S], then S
 * payloads of u16 words; each payload opens with the final rANS state (high
 * half first) and continues with the renormalisation words in the order the
 * decoder reads them.  Row r is coded by stream r mod S; a stream's pixels
 * are ordered by wave t = 3r + c, then by row. */
DLIC_API dlic_status dlic_encode(const dlic_model *model, const dlic_image *h_images, int n,
                                 const int *h_streams, void *d_out, size_t out_capacity,
                                 uint64_t *d_out_offsets, int32_t *d_status, void *d_workspace,
                                 size_t workspace_bytes, void *stream);

/* The model's prediction for every pixel, without coding: the frequency-
 * table entry of the pixel's own value, f | c << 16 (uint32; f the
 * frequency, c the cumulative frequency below the value, the table summing
 * to 2^16), computed by the same kernels and bits as dlic_encode (Sec. II-B:
 * the network predicts a PDF per pixel, which is quantised to the table the
 * rANS coder uses; Eq. 1).  The ideal code length of an image is the sum of
 * -log2(f / 2^16) over its pixels, the "bits per pixel" a trained model is
 * judged by (Sec. III-A).
 *  d_fc:        device, image i's H_i x W_i entries in raster order at
 *               element offset sum_{j<i} H_j W_j; 4-byte aligned.
 *  d_status:    one int32 on the device, or NULL; DLIC_OK, DLIC_ERR_TIMEOUT
 *               (a tensor-core wait ran out) or DLIC_ERR_INVALID (a 12-bit
 *               sample above 4095).
 *  d_workspace: when d_status is NULL, at least 4 bytes of device memory for
 *               the status word; otherwise unused (may be NULL).
 * Models with a 3D window are refused (DLIC_ERR_INVALID). */
DLIC_API dlic_status dlic_predict(const dlic_model *model, const dlic_image *h_images, int n, uint32_t *d_fc,
                                  int32_t *d_status, void *d_workspace, size_t workspace_bytes, void *stream);

/* Size of the fixed scratch block of dlic_encode_noalloc (16 MiB). */
#define DLIC_NOALLOC_SCRATCH_BYTES (16u << 20)

/* dlic_encode without a caller-provided workspace, for callers that cannot
 * allocate device memory: a plug-in or callback inside another framework
 * that owns every device allocation, a service whose device memory is all
 * reserved in advance, or a loop that must avoid the device-wide
 * synchronisation that cudaMalloc and cudaFree can cause.  The paper has no
 * counterpart; it is a deployment convenience of this library.
 *
 * The call allocates nothing.  Its workspace is one block of
 * DLIC_NOALLOC_SCRATCH_BYTES of device memory declared inside the library,
 * which every GPU that loads the library keeps until the process exits.
 * Arguments and results are those of dlic_encode minus the workspace pair;
 * the output bitstreams are identical.  A batch whose workspace
 * (dlic_encode_workspace_size) exceeds the block is rejected with
 * DLIC_ERR_CAPACITY before anything is enqueued.
 *  - Every call looks up the block's device address on the current device
 *    (a host-side query, no allocation).  The first lookup on a device may
 *    load the library's device code there; make the first call on each
 *    device before any stream capture.
 *  - All calls share the one block and it keeps the previous call's data.
 *    Nothing in it needs to start at zero: each call writes every word it
 *    reads before reading it.  Calls whose work overlaps on the GPU (two
 *    streams, two host threads) race on the block and corrupt each other's
 *    output; serialise them. */
DLIC_API dlic_status dlic_encode_noalloc(const dlic_model *model, const dlic_image *h_images, int n,
                                         const int *h_streams, void *d_out, size_t out_capacity,
                                         uint64_t *d_out_offsets, int32_t *d_status, void *stream);

/* ---------------------------------------------------------------------- */
/* Decoding (Sec. II-A Fig. 2 right; Sec. II-B "Preprocessor" wavefront)   */
/* ---------------------------------------------------------------------- */

/* Parses a bitstream header held in host memory (at least 24 bytes): a 2D
 * image's container or one slice's container of a volume (byte 12 with bit
 * 7 set); DLIC_ERR_CORRUPT when it is neither.  precision receives header
 * byte 13: the model's precision, with bit 4 (0x10) set for 12-bit pixels. */
DLIC_API dlic_status dlic_read_header(const void *h_bitstream, size_t bytes, int *height, int *width,
                             int *streams, int *precision, uint64_t *model_hash);

/* Device workspace, in bytes, that dlic_decode needs for this batch. */
DLIC_API dlic_status dlic_decode_workspace_size(const dlic_model *model, const dlic_image *h_images, int n,
                                       size_t *bytes);

/* Decodes n bitstreams held back to back in device memory d_in; bitstream i
 * occupies bytes [h_in_offsets[i], h_in_offsets[i + 1]) (host array of
 * n + 1 offsets, each even).  h_images[i] gives the destination buffer and
 * the dimensions the caller expects (from dlic_read_header).  Pixels are
 * decoded as a wavefront: wave t holds the pixels with 3r + c = t, all of
 * whose causal priors lie on earlier waves, and each wave's pixels are
 * predicted and decoded in parallel.  Each image is decoded by a cluster of
 * 1 to 16 CTAs chosen by a cost model (larger images get larger clusters
 * while the batch fits on the GPU); images with different cluster sizes run
 * concurrently on internal streams forked from and joined back to `stream`.
 * INT8 networks of widths 128 run on the tensor cores, FP32 networks with
 * h2 <= 128 on the CUDA cores, other networks in one CTA per image.
 * An image whose waves (min(height, ceil(width / 3)) pixels) leave no
 * shared-memory plan room on the cluster decoder (about 20000 pixels for
 * INT8 networks) returns DLIC_ERR_UNSUPPORTED before anything is enqueued;
 * the default-window FP32 decoder falls back to one CTA per image.
 * d_status (n int32, device) receives DLIC_OK or DLIC_ERR_CORRUPT per image
 * (header mismatch, model hash mismatch, stream overrun, or a final state
 * other than the initial one), or DLIC_ERR_TIMEOUT when a bounded wait of
 * the decoder ran out. */
DLIC_API dlic_status dlic_decode(const dlic_model *model, const void *d_in, const uint64_t *h_in_offsets,
                        int n, const dlic_image *h_images, int32_t *d_status, void *d_workspace,
                        size_t workspace_bytes, void *stream);

/* ---------------------------------------------------------------------- */
/* Volumes (Sec. IV "3D Dependencies", "3D Wavefront")                      */
/* ---------------------------------------------------------------------- */

/* A model whose window field is 3D (2 << 28 | u | l << 4 | r << 8 | pu << 10 |
 * pd << 14 | pl << 18 | pr << 22) predicts pixel (z, r, c) from its slice's
 * causal window (u, l, r) and, from slice z - 1, rows r-pu..r+pd at columns
 * c-pl..c+pr (row by row; zeros for the first slice and outside the slice).
 * Such a model codes volumes only (dlic_encode and dlic_decode refuse it
 * with DLIC_ERR_INVALID, and the volume calls refuse 2D models). */

/* Device workspace, in bytes, that dlic_encode_volume needs for these volumes. */
DLIC_API dlic_status dlic_encode_volume_workspace_size(const dlic_model *model, const dlic_volume *h_volumes, int n,
                                              size_t *bytes);

/* Encodes n volumes.  Every slice is coded on its own, with its own streams,
 * into a "DLC1" container whose byte 12 is u | 0x80; the containers follow
 * one another slice by slice, volume by volume, in d_out.  d_out_offsets
 * (device, sum of depths + 1 entries) receives the byte offset of every
 * slice's container and the total.  Capacity, workspace and status as for
 * dlic_encode (each slice needs dlic_max_encoded_bytes). */
DLIC_API dlic_status dlic_encode_volume(const dlic_model *model, const dlic_volume *h_volumes, int n, void *d_out,
                               size_t out_capacity, uint64_t *d_out_offsets, int32_t *d_status,
                               void *d_workspace, size_t workspace_bytes, void *stream);

/* Device workspace, in bytes, that dlic_decode_volume needs. */
DLIC_API dlic_status dlic_decode_volume_workspace_size(const dlic_model *model, const dlic_volume *h_volumes, int n,
                                              size_t *bytes);

/* Decodes n volumes; volume i is the bytes [h_in_offsets[i], h_in_offsets[i + 1])
 * of d_in (host array of n + 1 even offsets): its slices' containers back to
 * back, as dlic_encode_volume wrote them.  All slices of a volume decode at
 * once as a 3D wavefront: pixel (z, r, c) is on wave
 * 3r + c + (3 pd + pr + 1) z, so every prior from slice z - 1 is decoded
 * before it is read (priors are read back from the output volume); the first
 * slice is complete after 3(H-1) + W waves, the volume after
 * (3 pd + pr + 1)(depth - 1) more.  When no slice's wave holds two rows of
 * one stream (min(height, ceil(width / 3)) <= streams) and depth x streams
 * < 2^24, the whole GPU decodes the volume: one CTA per SM in a cooperative
 * launch, each wave's pixels split evenly over the CTAs, stream states in the
 * workspace, one grid-wide barrier per wave (volumes one after another).
 * Otherwise, or under a forced decode plan, one cluster of up to 16 CTAs
 * (the largest power of two dividing the streams) decodes it with one
 * cluster barrier per wave.  h_volumes[i].streams must equal the slices'
 * stream count.  Networks as for the cluster decoder (INT8 of widths 128,
 * FP32 with h2 <= 128).
 * d_status (n int32, device): DLIC_OK, DLIC_ERR_CORRUPT (a slice's header,
 * sizes or final states) or DLIC_ERR_TIMEOUT. */
DLIC_API dlic_status dlic_decode_volume(const dlic_model *model, const void *d_in, const uint64_t *h_in_offsets,
                               int n, const dlic_volume *h_volumes, int32_t *d_status, void *d_workspace,
                               size_t workspace_bytes, void *stream);

/* ---------------------------------------------------------------------- */
/* Training (Sec. III-A: categorical cross-entropy reported in bits)        */
/* ---------------------------------------------------------------------- */

enum { DLIC_TRAIN_BF16 = 0, DLIC_TRAIN_FP32 = 1, DLIC_TRAIN_BF16X3 = 2 };
/* OR'ed into a BF16 mode at dlic_trainer_create(_k): activations recomputed
 * rather than stored.  The trainer then holds two activation buffers of
 * max_batch rows instead of five: the first hidden layer's output is
 * recomputed from the batch in the backward pass (one more first-layer
 * launch per step) and every gradient buffer reuses the memory of an
 * activation that is no longer needed.  Losses, gradients and updates are
 * bit for bit those of the mode without it.  With DLIC_TRAIN_FP32 the call
 * returns DLIC_ERR_INVALID. */
enum { DLIC_TRAIN_RECOMPUTE = 0x100 };

/* Number of FP32 parameters of an n_in -> h1 -> h2 -> 256 network (n_in:
 * the priors of the model's window, 12 for the default window), laid out as
 * W1 [h1][n_in], b1 [h1], W2 [h2][h1], b2 [h2], W3 [256][h2], b3 [256] (the
 * layer order of an FP32 model blob). */
DLIC_API size_t dlic_train_param_count(int n_in, int h1, int h2);

/* The same for an n_in -> h1 -> h2 -> n_out network: n_out = 256 for 8-bit
 * samples, 4096 for 12-bit ones (Sec. IV "Higher Bit Depth": one output
 * neuron per value); W3 is [n_out][h2] and b3 [n_out]. */
DLIC_API size_t dlic_train_param_count_k(int n_in, int h1, int h2, int n_out);

/* Creates a trainer: FP32 master weights (copied from h_params, host),
 * Adam moments (lr 1e-3, betas 0.9 / 0.999, eps 1e-8, bias-corrected) and
 * device buffers for batches of up to max_batch contexts.  mode
 * DLIC_TRAIN_BF16 runs the two wide layers and every backward product on
 * the tensor cores with bf16 operands and FP32 accumulation (the first
 * layer, n_in <= 96 inputs, in FP32 on the CUDA cores); DLIC_TRAIN_BF16X3 stores every
 * tensor-core operand as two bf16 planes (x = hi + lo) and accumulates
 * hi*hi + lo*hi + hi*lo (about 16 significant bits per operand, three times
 * the MMAs); DLIC_TRAIN_FP32 runs every product in FP32 on the CUDA cores.
 * Allocates its device memory here and frees it in dlic_trainer_destroy.
 * The calls below take any batch B >= 1: a batch above max_batch runs in
 * chunks of max_batch contexts (each chunk's forward and backward on its
 * own, the chunks' mean losses and gradients added with weights B_c / B),
 * so the activations held at any time are one chunk's whatever B is; the
 * result equals the one-pass result up to FP32 rounding of the sums. */
DLIC_API dlic_status dlic_trainer_create(int n_in, int h1, int h2, int mode, int max_batch, const float *h_params,
                                         dlic_trainer **out);

/* dlic_trainer_create for n_out outputs: 256 (the call above; batches of u8
 * samples, inputs v/128 - 1) or 4096 (12-bit samples, Sec. IV "Higher Bit
 * Depth": batches of u16 samples 0..4095, inputs v/2048 - 1, the 4096-way
 * cross-entropy in bits).  With 4096 outputs the output layer's products
 * go to an FP32 buffer of max_batch x 4096 (16 KB per context, allocated
 * here) and a row-wise kernel takes the softmax; every mode is available.
 * A 12-bit sample or target above 4095 sets DLIC_ERR_INVALID in the
 * trainer's device status (dlic_trainer_status, which keeps it for the
 * trainer's life); that call's loss and gradient are then meaningless.
 * Any other n_out is DLIC_ERR_INVALID. */
DLIC_API dlic_status dlic_trainer_create_k(int n_in, int h1, int h2, int n_out, int mode, int max_batch,
                                           const float *h_params, dlic_trainer **out);
DLIC_API dlic_status dlic_trainer_destroy(dlic_trainer *trainer);

/* The frequency-weighted loss (Sec. IV "Color Frequencies": the loss is
 * weighted by value frequency so that rare values count more): h_weights
 * (host, n_out floats: 256, or 4096 for 12-bit samples; finite, >= 0, not
 * all zero) gives each target value v a
 * weight w_v, and every later loss and gradient of this trainer become
 *     sum_b w_{y_b} * -log2 softmax(z_b)[y_b] / sum_b w_{y_b},
 * the plain mean when every w_v is 1; an integer weight k counts a context
 * like k copies of it.  A batch must hold a context whose value has a
 * positive weight.  h_weights NULL restores the plain loss. */
DLIC_API dlic_status dlic_trainer_set_value_weights(dlic_trainer *trainer, const float *h_weights);

/* Loss of a batch: d_ctx holds B x n_in causal priors (the window's order,
 * as the coder gathers them), d_tgt B target pixels, both u8 for a trainer
 * of 256 outputs and u16 for one of 4096; *d_loss_bits (device float)
 * receives mean_b -log2 softmax(z_b)[y_b]. */
DLIC_API dlic_status dlic_train_forward(dlic_trainer *trainer, const void *d_ctx, const void *d_tgt, int B,
                                        float *d_loss_bits, void *stream);

/* Loss and its gradient with respect to every parameter (the adjoint of the
 * forward pass).  The activations are recomputed from the batch: nothing
 * is kept from an earlier dlic_train_forward.  d_grads (device,
 * dlic_train_param_count floats, may be NULL) receives the gradient in the
 * parameter layout. */
DLIC_API dlic_status dlic_train_backward(dlic_trainer *trainer, const void *d_ctx, const void *d_tgt, int B,
                                         float *d_loss_bits, float *d_grads, void *stream);

/* Forward, backward and one Adam update of the master weights. */
DLIC_API dlic_status dlic_train_step(dlic_trainer *trainer, const void *d_ctx, const void *d_tgt, int B,
                                     float *d_loss_bits, void *stream);

/* One Adam update of the master weights (and their bf16 operand copies)
 * with a gradient the caller supplies: d_grads (device, in the parameter
 * layout of dlic_train_param_count floats).  With data-parallel training
 * over several GPUs each rank computes its batch's gradient with
 * dlic_train_backward, the ranks average them (weighted by batch size) with
 * one all-reduce, and every rank applies the same average here, so the
 * replicas stay identical (Sec. III-A: the network is trained on the loss in
 * bits; data parallelism is this library's way of spreading that work).
 * dlic_train_backward followed by dlic_train_apply of its own gradient is
 * exactly dlic_train_step. */
DLIC_API dlic_status dlic_train_apply(dlic_trainer *trainer, const float *d_grads, void *stream);

/* Copies the FP32 master weights out of (write = 0) or into (write = 1) the
 * trainer; d_params is a device buffer of dlic_train_param_count floats. */
DLIC_API dlic_status dlic_trainer_params(dlic_trainer *trainer, float *d_params, int write, void *stream);

/* Device status of the trainer's kernels (DLIC_OK, DLIC_ERR_TIMEOUT when a
 * tensor-core wait ran out, DLIC_ERR_INVALID after a 12-bit sample above
 * 4095); synchronises with the device. */
DLIC_API dlic_status dlic_trainer_status(dlic_trainer *trainer, int32_t *h_status);

#ifdef __cplusplus
}
#endif

#endif /* DLIC_H */
