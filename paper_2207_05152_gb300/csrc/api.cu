// C ABI of libdlic: model set-up, workspace planning and the encode / decode
// entry points declared in include/dlic.h.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "tc.cuh"

namespace dlic {

static thread_local char g_err[512] = "";

dlic_status fail(dlic_status code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

dlic_status cuda_fail(cudaError_t e, const char *what) {
    return fail(DLIC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr int kDecodeGroups = 5;   // cluster sizes 1, 2, 4, 8, 16

static inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

static uint32_t le32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

static float lef32(const uint8_t *p) {
    uint32_t u = le32(p);
    float f;
    memcpy(&f, &u, 4);
    return f;
}

static uint64_t fnv1a64(const uint8_t *p, size_t n) {
    uint64_t h = 0xCBF29CE484222325ull;
    for (size_t i = 0; i < n; i++) {
        h ^= p[i];
        h *= 0x100000001B3ull;
    }
    return h;
}

}  // namespace dlic

using namespace dlic;

struct dlic_model {
    DevModel dev;
    void *mem = nullptr;
    int device = 0;
    int num_sms = 0;
    // streams and events of the batched decoder: one stream per cluster size,
    // forked from and joined back to the caller's stream
    cudaStream_t group_stream[kDecodeGroups] = {};
    cudaEvent_t fork_event = nullptr, join_event[kDecodeGroups] = {};
    int decode_plan = DLIC_PLAN_AUTO;
    DevLayer hl[kMaxLayers] = {};   // host copy of the layer table (networks wider than 256)
};

extern "C" const char *dlic_last_error(void) { return g_err; }

extern "C" dlic_status dlic_model_create(const void *h_blob, size_t n, dlic_model **out) {
    if (!h_blob || !out) return fail(DLIC_ERR_INVALID, "null argument");
    *out = nullptr;
    const uint8_t *b = static_cast<const uint8_t *>(h_blob);
    // "DLM1": two hidden layers, 288-byte header (u32 precision, n_in, h1,
    // h2, n_out, window, f32 tscale, u32 lut[64]).  "DLM2": 1..8 hidden
    // layers, 320-byte header (u32 precision, n_in, L, widths[8], n_out,
    // window, f32 tscale, u32 0, u32 lut[64]).  Then the dense layers.
    const bool dlm2 = n >= 320 && memcmp(b, "DLM2", 4) == 0;
    if (!dlm2 && (n < 288 || memcmp(b, "DLM1", 4) != 0)) return fail(DLIC_ERR_INVALID, "not a DLIC model blob");
    const uint32_t prec = le32(b + 4), n_in = le32(b + 8);
    uint32_t widths[kMaxLayers - 1] = {0}, n_out, radius;
    int L = 2;
    size_t hdr = 288, tscale_at = 28, lut_at = 32;
    if (dlm2) {
        L = (int)le32(b + 12);
        if (L < 1 || L > kMaxLayers - 1) return fail(DLIC_ERR_INVALID, "a network has 1..%d hidden layers", kMaxLayers - 1);
        for (int l = 0; l < kMaxLayers - 1; l++) {
            widths[l] = le32(b + 16 + 4 * l);
            if ((l < L) != (widths[l] != 0)) return fail(DLIC_ERR_INVALID, "exactly the first %d hidden widths are nonzero", L);
        }
        n_out = le32(b + 48);
        radius = le32(b + 52);
        hdr = 320;
        tscale_at = 56;
        lut_at = 64;
    } else {
        widths[0] = le32(b + 12);
        widths[1] = le32(b + 16);
        n_out = le32(b + 20);
        radius = le32(b + 24);
    }
    const uint32_t h1 = widths[0], h2 = widths[L - 1];
    // 4096 outputs: 12-bit pixels (Sec. IV "Higher Bit Depth"), on the
    // layer-table FP32 kernels like networks of other depths
    const bool twelve = n_out == (uint32_t)kSymbols12;
    uint32_t wmax = 0;
    for (int l = 0; l < L; l++) wmax = std::max(wmax, widths[l]);
    // hidden layers wider than 256 (8-bit): one layer at a time (wide.cu)
    const bool wide = !twelve && wmax > (uint32_t)kMaxHidden;
    const bool deep = L != 2 || twelve || wide;   // the layer-table kernels
    if (prec > 1) return fail(DLIC_ERR_INVALID, "unknown precision %u", prec);
    // window field: 2 = the default radius-2 window, else 1 << 24 | u | l << 8 | r << 16,
    // or a 3D window 2 << 28 | u | l << 4 | r << 8 | pu << 10 | pd << 14 | pl << 18 | pr << 22
    int wu = 2, wl = 2, wr = 2, vol = 0, pu = 0, pd = 0, pl = 0, pr = 0;
    if (radius != 2) {
        if ((radius >> 24) == 1) {
            wu = (int)(radius & 0xFF);
            wl = (int)((radius >> 8) & 0xFF);
            wr = (int)((radius >> 16) & 0xFF);
        } else if ((radius >> 28) == 2 && ((radius >> 26) & 3) == 0) {
            vol = 1;
            wu = (int)(radius & 0xF);
            wl = (int)((radius >> 4) & 0xF);
            wr = (int)((radius >> 8) & 3);
            pu = (int)((radius >> 10) & 0xF);
            pd = (int)((radius >> 14) & 0xF);
            pl = (int)((radius >> 18) & 0xF);
            pr = (int)((radius >> 22) & 0xF);
            if (pu > 8 || pd > 8 || pl > 8 || pr > 8)
                return fail(DLIC_ERR_INVALID, "3D window reaches must be <= 8");
        } else {
            return fail(DLIC_ERR_INVALID, "unknown window field 0x%x", radius);
        }
        if (wu < 1 || wu > 8 || wl > 8 || wr > 2)
            return fail(DLIC_ERR_INVALID, "window must have 1..8 rows above, left reach <= 8, right reach <= 2");
    }
    const int n2 = wu * (wl + wr + 1) + wl;
    const int npri = n2 + (vol ? (pu + pd + 1) * (pl + pr + 1) : 0);
    if (npri > kMaxPriors || (int)n_in != npri || (n_out != kSymbols && !twelve))
        return fail(DLIC_ERR_INVALID, "model must map the %d priors of its window to 256 (or 4096) logits", npri);
    if (twelve && prec != DLIC_FP32)
        return fail(DLIC_ERR_INVALID, "a 12-bit model (4096 outputs) has an FP32 network");
    for (int l = 0; l < L; l++)
        if (widths[l] > 4096) return fail(DLIC_ERR_INVALID, "hidden widths must be <= 4096");
    if (!deep) {
        if (h1 < 16 || h1 > kMaxHidden || h1 % 16 || h2 < 16 || h2 > kMaxHidden || h2 % 16)
            return fail(DLIC_ERR_UNSUPPORTED, "hidden widths must be multiples of 16 in [16, 256]");
    } else {
        for (int l = 0; l < L; l++)
            if (widths[l] < 4 || widths[l] > (twelve ? (uint32_t)kMaxHidden : 4096u) || widths[l] % 4)
                return fail(DLIC_ERR_UNSUPPORTED, twelve ? "hidden widths of a 12-bit network must be multiples of 4 in "
                                                           "[4, 256]"
                                                         : "hidden widths of a network of %d hidden layers (or wider "
                                                           "than 256) must be multiples of 4 in [4, 4096]", L);
        if (radius != 2)
            return fail(DLIC_ERR_UNSUPPORTED, "12-bit networks and networks of other than two hidden layers run with "
                                              "the default window only");
    }
    const float tscale = lef32(b + tscale_at);
    if (!(tscale > 0.0f)) return fail(DLIC_ERR_INVALID, "tscale must be positive");
    uint32_t lut[64];
    for (int k = 0; k < 64; k++) {
        lut[k] = le32(b + lut_at + 4 * k);
        if (lut[k] > (1u << 23)) return fail(DLIC_ERR_INVALID, "lut entries must be <= 2^23");
    }
    if (lut[0] != (1u << 23)) return fail(DLIC_ERR_INVALID, "lut[0] must be 2^23");
    const int nl = L + 1;
    int din[kMaxLayers], dout[kMaxLayers], hmax = 0;
    for (int l = 0; l < nl; l++) {
        din[l] = l == 0 ? npri : (int)widths[l - 1];
        dout[l] = l == nl - 1 ? (int)n_out : (int)widths[l];
        if (l < L) hmax = std::max(hmax, (int)widths[l]);
    }
    const int k1 = (npri + 15) / 16 * 16;   // first-layer K of the tensor-core operands
    size_t need = hdr;
    for (int l = 0; l < nl; l++)
        need += prec == 0 ? 4ull * din[l] * dout[l] + 4ull * dout[l] : (size_t)din[l] * dout[l] + 8ull * dout[l];
    if (need != n) return fail(DLIC_ERR_INVALID, "blob size %zu does not match its header (%zu)", n, need);

    // Host image of the device buffer.
    std::vector<uint8_t> host;
    auto put = [&](const void *src, size_t bytes) {
        size_t off = align256(host.size());
        host.resize(off + bytes);
        memcpy(host.data() + off, src, bytes);
        return off;
    };
    DevModel d{};
    d.precision = (int)prec;
    d.h1 = (int)h1;
    d.h2 = (int)h2;
    d.nl = nl;
    d.hmax = hmax;
    d.bits = twelve ? 12 : 8;
    d.wu = wu;
    d.wl = wl;
    d.wr = wr;
    d.n_in = npri;
    d.n2 = n2;
    d.vol = vol;
    d.pu = pu;
    d.pd = pd;
    d.pl = pl;
    d.pr = pr;
    d.tscale = tscale;
    d.hash = fnv1a64(b, n);
    d.peer_wait_limit = kDefaultPeerWaitLimit;
    size_t off_lut = put(lut, sizeof(lut));
    // offs[3 l .. 3 l + 2]: layer l's weights and its bias (FP32) or scale
    // and offset (INT8); offs[3 kMaxLayers]: the tensor-core operand image
    size_t offs[3 * kMaxLayers + 1] = {0};
    const int kTcImage = 3 * kMaxLayers;
    const size_t off_table = deep ? put(std::vector<DevLayer>(nl).data(), sizeof(DevLayer) * nl) : 0;
    size_t off_w3tiles = 0;   // 12-bit: the output layer tiled for the decoder
    size_t off_wtc[kMaxLayers] = {0};   // wide INT8: bf16 weight rows of the tensor-core layers
    int wtc_pitch[kMaxLayers] = {0};
    const uint8_t *p = b + hdr;
    if (prec == DLIC_FP32) {
        for (int l = 0; l < nl; l++) {
            std::vector<float> wt((size_t)din[l] * dout[l]), bias(dout[l]);
            for (int j = 0; j < dout[l]; j++)
                for (int k = 0; k < din[l]; k++) wt[(size_t)k * dout[l] + j] = lef32(p + 4 * ((size_t)j * din[l] + k));
            p += 4ull * din[l] * dout[l];
            for (int j = 0; j < dout[l]; j++) bias[j] = lef32(p + 4 * j);
            p += 4ull * dout[l];
            offs[3 * l] = put(wt.data(), wt.size() * 4);
            offs[3 * l + 1] = put(bias.data(), bias.size() * 4);
            if (twelve && l == nl - 1) {
                // the 12-bit decoder's copy of the output layer in 16 x 256
                // tiles (block q of 256 values, k tile kt of 16 rows, rows past
                // the layer's inputs zero), one bulk copy each
                const int KT = (din[l] + 15) / 16;
                std::vector<float> tiles((size_t)kSymbols12 * 16 * KT, 0.0f);
                for (int q = 0; q < kSymbols12 / 256; q++)
                    for (int kt = 0; kt < KT; kt++)
                        for (int r = 0; r < 16 && 16 * kt + r < din[l]; r++)
                            for (int j = 0; j < 256; j++)
                                tiles[(((size_t)q * KT + kt) * 16 + r) * 256 + j] =
                                    wt[(size_t)(16 * kt + r) * dout[l] + 256 * q + j];
                off_w3tiles = put(tiles.data(), tiles.size() * 4);
            }
        }
    } else {
        const int8_t *raw[kMaxLayers];
        const uint8_t *pp = p;
        for (int l = 0; l < nl; l++) {
            raw[l] = reinterpret_cast<const int8_t *>(pp);
            pp += (size_t)din[l] * dout[l] + 8ull * dout[l];
        }
        if (!deep && h1 <= 128 && h2 <= 128) {
            std::vector<uint16_t> img(tc_weight_bytes((int)h1, (int)h2, k1) / 2);
            tc_pack_weights((int)h1, (int)h2, npri, k1, raw[0], raw[1], raw[2], img.data());
            offs[kTcImage] = put(img.data(), img.size() * 2);
            d.tc_w_bytes = (uint32_t)(img.size() * 2);
        }
        for (int l = 0; l < nl; l++) {
            const int k4n = (din[l] + 3) / 4;
            std::vector<uint32_t> qt((size_t)k4n * dout[l], 0u);
            for (int j = 0; j < dout[l]; j++)
                for (int k = 0; k < din[l]; k++)
                    qt[(size_t)(k / 4) * dout[l] + j] |= (uint32_t)p[(size_t)j * din[l] + k] << (8 * (k % 4));
            p += (size_t)din[l] * dout[l];
            std::vector<float> s(dout[l]), o(dout[l]);
            for (int j = 0; j < dout[l]; j++) s[j] = lef32(p + 4 * j);
            p += 4ull * dout[l];
            for (int j = 0; j < dout[l]; j++) o[j] = lef32(p + 4 * j);
            p += 4ull * dout[l];
            offs[3 * l] = put(qt.data(), qt.size() * 4);
            offs[3 * l + 1] = put(s.data(), s.size() * 4);
            offs[3 * l + 2] = put(o.data(), o.size() * 4);
        }
        // a wide network's layers after the first (inputs: u8 units) also as
        // bf16 rows [n_out][K padded to 64] for the tensor-core encoder; the
        // integer weights are exact in bf16
        if (wide)
            for (int l = 1; l < nl; l++) {
                const int kp = (din[l] + 63) / 64 * 64;
                std::vector<uint16_t> wb((size_t)dout[l] * kp, 0);
                for (int j = 0; j < dout[l]; j++)
                    for (int k = 0; k < din[l]; k++) wb[(size_t)j * kp + k] = tc::bf16_of_int(raw[l][(size_t)j * din[l] + k]);
                off_wtc[l] = put(wb.data(), wb.size() * 2);
                wtc_pitch[l] = kp;
            }
    }
    host.resize(align256(host.size()));
    dlic_model *m = new dlic_model();
    cudaGetDevice(&m->device);
    cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
    if (m->num_sms < 1) m->num_sms = 1;
    cudaError_t e = cudaMalloc(&m->mem, host.size());
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail(e, "cudaMalloc(model)");
    }
    uint8_t *base = static_cast<uint8_t *>(m->mem);
    if (deep) {
        // the layer table holds device addresses: written once they are known
        std::vector<DevLayer> table(nl);
        for (int l = 0; l < nl; l++) {
            table[l].w = base + offs[3 * l];
            table[l].a = reinterpret_cast<const float *>(base + offs[3 * l + 1]);
            table[l].o = prec == DLIC_INT8 ? reinterpret_cast<const float *>(base + offs[3 * l + 2]) : nullptr;
            table[l].n_in = din[l];
            table[l].n_out = dout[l];
            table[l].wtc = wtc_pitch[l] ? reinterpret_cast<const uint16_t *>(base + off_wtc[l]) : nullptr;
            table[l].wtc_pitch = wtc_pitch[l];
        }
        memcpy(host.data() + off_table, table.data(), sizeof(DevLayer) * nl);
        d.layers = reinterpret_cast<const DevLayer *>(base + off_table);
        for (int l = 0; l < nl; l++) m->hl[l] = table[l];
    }
    e = cudaMemcpy(m->mem, host.data(), host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(m->mem);
        delete m;
        return cuda_fail(e, "cudaMemcpy(model)");
    }
    for (int g = 0; g < kDecodeGroups && e == cudaSuccess; g++) {
        e = cudaStreamCreateWithFlags(&m->group_stream[g], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->join_event[g], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->fork_event, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        dlic_model_destroy(m);
        return cuda_fail(e, "stream / event creation");
    }
    d.lut = reinterpret_cast<const uint32_t *>(base + off_lut);
    if (deep) {
        // the kernels read the layer table only (and the 12-bit decoder the
        // tiled output layer)
        if (twelve) d.w3t = reinterpret_cast<const float *>(base + off_w3tiles);
    } else if (prec == DLIC_FP32) {
        d.w1t = reinterpret_cast<const float *>(base + offs[0]);
        d.b1 = reinterpret_cast<const float *>(base + offs[1]);
        d.w2t = reinterpret_cast<const float *>(base + offs[3]);
        d.b2 = reinterpret_cast<const float *>(base + offs[4]);
        d.w3t = reinterpret_cast<const float *>(base + offs[6]);
        d.b3 = reinterpret_cast<const float *>(base + offs[7]);
    } else {
        d.q1t = reinterpret_cast<const uint32_t *>(base + offs[0]);
        d.s1 = reinterpret_cast<const float *>(base + offs[1]);
        d.o1 = reinterpret_cast<const float *>(base + offs[2]);
        d.q2t = reinterpret_cast<const uint32_t *>(base + offs[3]);
        d.s2 = reinterpret_cast<const float *>(base + offs[4]);
        d.o2 = reinterpret_cast<const float *>(base + offs[5]);
        d.q3t = reinterpret_cast<const uint32_t *>(base + offs[6]);
        d.s3 = reinterpret_cast<const float *>(base + offs[7]);
        d.o3 = reinterpret_cast<const float *>(base + offs[8]);
        if (d.tc_w_bytes) d.tc_w = reinterpret_cast<const uint16_t *>(base + offs[kTcImage]);
    }
    m->dev = d;
    if (!default_window(d)) {
        // other windows run on the tensor-core INT8 kernels and the FP32
        // tiled / cluster kernels only
        const bool enc_ok = prec == DLIC_INT8 ? (h1 <= 128 && h2 <= 128) : f32_predict_supported(d);
        if (!enc_ok || !wave_decode_supported(d)) {
            dlic_model_destroy(m);
            return fail(DLIC_ERR_UNSUPPORTED, "a window other than the default needs INT8 widths 128/128 or an FP32 "
                                              "network with h2 <= 128");
        }
    }
    *out = m;
    return DLIC_OK;
}

extern "C" dlic_status dlic_model_set_decode_plan(dlic_model *m, int plan) {
    if (!m) return fail(DLIC_ERR_INVALID, "null model");
    if (plan != DLIC_PLAN_AUTO && plan != DLIC_PLAN_BYTE_RING && plan != DLIC_PLAN_IMAGE && plan != DLIC_PLAN_GRID)
        return fail(DLIC_ERR_INVALID, "unknown decode plan %d", plan);
    m->decode_plan = plan;
    return DLIC_OK;
}

extern "C" dlic_status dlic_model_set_peer_wait_limit(dlic_model *m, long long cycles) {
    if (!m) return fail(DLIC_ERR_INVALID, "null model");
    m->dev.peer_wait_limit = cycles > 0 ? cycles : kDefaultPeerWaitLimit;
    return DLIC_OK;
}

extern "C" dlic_status dlic_model_destroy(dlic_model *m) {
    if (!m) return DLIC_OK;
    for (int g = 0; g < kDecodeGroups; g++) {
        if (m->group_stream[g]) cudaStreamDestroy(m->group_stream[g]);
        if (m->join_event[g]) cudaEventDestroy(m->join_event[g]);
    }
    if (m->fork_event) cudaEventDestroy(m->fork_event);
    cudaError_t e = m->mem ? cudaFree(m->mem) : cudaSuccess;
    delete m;
    return e == cudaSuccess ? DLIC_OK : cuda_fail(e, "cudaFree(model)");
}

extern "C" dlic_status dlic_model_info(const dlic_model *m, int *precision, int *h1, int *h2,
                                       uint64_t *hash) {
    if (!m) return fail(DLIC_ERR_INVALID, "null model");
    if (precision) *precision = m->dev.precision;
    if (h1) *h1 = m->dev.h1;
    if (h2) *h2 = m->dev.h2;
    if (hash) *hash = m->dev.hash;
    return DLIC_OK;
}

extern "C" size_t dlic_max_encoded_bytes(int height, int width, int streams) {
    if (height < 1 || width < 1 || streams < 1) return 0;
    const int S = streams < height ? streams : height;
    return (size_t)kHeaderBytes + 4ull * S + 2ull * ((size_t)height * width + 2ull * S);
}

extern "C" int dlic_auto_streams(int height, int width) {
    if (height < 1 || width < 1) return 0;
    int s = ((width + 2) / 3 + 15) / 16 * 16;
    if (s > height) s = height;
    if (s > 65520) s = 65520;
    return s < 1 ? 1 : s;
}

// bps: bytes per sample, 1 (8-bit) or 2 (12-bit: u16 samples, 2-byte aligned rows)
static dlic_status check_images(const dlic_image *im, int n, const int *streams, bool writable, int bps) {
    if (n < 0) return fail(DLIC_ERR_INVALID, "negative image count");
    if (n > 0 && !im) return fail(DLIC_ERR_INVALID, "null image array");
    for (int i = 0; i < n; i++) {
        if (!im[i].pixels) return fail(DLIC_ERR_INVALID, "image %d: null pixels", i);
        if (im[i].height < 1 || im[i].width < 1)
            return fail(DLIC_ERR_INVALID, "image %d: empty image (%d x %d)", i, im[i].height, im[i].width);
        if (im[i].height > (1 << 20) || im[i].width > (1 << 20))
            return fail(DLIC_ERR_UNSUPPORTED, "image %d: dimension above 2^20", i);
        if (im[i].pitch < (int64_t)bps * im[i].width)
            return fail(DLIC_ERR_INVALID, "image %d: pitch < width x %d bytes", i, bps);
        if (bps == 2 && ((reinterpret_cast<uintptr_t>(im[i].pixels) | (uintptr_t)im[i].pitch) & 1))
            return fail(DLIC_ERR_INVALID, "image %d: 12-bit samples need 2-byte aligned pixels and an even pitch", i);
        if (streams && (streams[i] < 1 || streams[i] > 65535))
            return fail(DLIC_ERR_INVALID, "image %d: stream count %d outside [1, 65535]", i, streams[i]);
    }
    (void)writable;
    return DLIC_OK;
}

static int clip_streams(const dlic_image &im, const int *streams, int i) {
    int s = streams ? streams[i] : dlic_auto_streams(im.height, im.width);
    return s < im.height ? s : im.height;
}

static size_t enc_image_bytes(int H, int W, int S) {
    const size_t N = (size_t)H * W;
    return align256(4 * N) + align256(2 * (N + 2ull * S)) + 3 * align256(4ull * S);
}

// One image, or one slice of a volume (with the slice before it), to encode.
struct EncItem {
    const uint8_t *pixels, *below;
    int H, W, S;
    int64_t pitch;
};

static size_t enc_ws_bytes(const std::vector<EncItem> &it) {
    size_t total = align256(8ull * (it.size() + 1)) + 256;
    for (const EncItem &e : it) total += enc_image_bytes(e.H, e.W, e.S);
    return total;
}

static std::vector<EncItem> image_items(const dlic_image *im, int n, const int *streams) {
    std::vector<EncItem> it((size_t)n);
    for (int i = 0; i < n; i++) it[i] = {im[i].pixels, nullptr, im[i].height, im[i].width, clip_streams(im[i], streams, i), im[i].pitch};
    return it;
}

extern "C" dlic_status dlic_encode_workspace_size(const dlic_model *m, const dlic_image *im, int n,
                                                  const int *streams, size_t *bytes) {
    if (!m || !bytes) return fail(DLIC_ERR_INVALID, "null argument");
    dlic_status st = check_images(im, n, streams, false, m->dev.bits == 12 ? 2 : 1);
    if (st) return st;
    *bytes = enc_ws_bytes(image_items(im, n, streams)) + wide_scratch_bytes(m->dev, true);
    return DLIC_OK;
}

// Predicts, rANS-codes and packs every item into its own container, back to
// back in d_out; d_out_offsets gets items + 1 byte offsets.
static dlic_status encode_items(const dlic_model *m, const std::vector<EncItem> &it, void *d_out, size_t out_capacity,
                                uint64_t *d_out_offsets, int32_t *d_status, void *d_ws, size_t ws_bytes, void *stream) {
    const int n = (int)it.size();
    if (n == 0) return DLIC_OK;
    if (!d_out || !d_out_offsets || !d_ws) return fail(DLIC_ERR_INVALID, "null buffer");
    if (reinterpret_cast<uintptr_t>(d_ws) & 255) return fail(DLIC_ERR_INVALID, "workspace must be 256-byte aligned");
    size_t need_out = 0;
    const size_t need_ws = enc_ws_bytes(it) + wide_scratch_bytes(m->dev, true);
    for (const EncItem &e : it) need_out += dlic_max_encoded_bytes(e.H, e.W, e.S);
    if (ws_bytes < need_ws) return fail(DLIC_ERR_CAPACITY, "workspace %zu < %zu bytes", ws_bytes, need_ws);
    if (out_capacity < need_out) return fail(DLIC_ERR_CAPACITY, "output capacity %zu < %zu bytes", out_capacity, need_out);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    size_t off = align256(8ull * (n + 1));
    uint64_t *sizes = reinterpret_cast<uint64_t *>(ws);
    int32_t *err = d_status ? d_status : reinterpret_cast<int32_t *>(ws + off);
    off += 256;
    uint8_t *out = static_cast<uint8_t *>(d_out);
    // networks of other than two hidden layers: the one-pixel-per-thread kernels
    const bool use_tc = m->dev.nl == 3 && m->dev.bits == 8 && tc_supported(m->dev);
    const int tile_px = use_tc ? 128 : kPredictTile;
    {
        cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int32_t), cs);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(status)");
    }
    for (int c0 = 0; c0 < n; c0 += kMaxBatch) {
        const int cn = n - c0 < kMaxBatch ? n - c0 : kMaxBatch;
        EncBatch *b = new EncBatch();
        b->n = cn;
        b->ws = ws;
        b->sizes = sizes + c0;
        b->chunk_start = c0;
        b->tile_px = tile_px;
        int tiles = 0, total_streams = 0;
        for (int k = 0; k < cn; k++) {
            const EncItem &g = it[c0 + k];
            EncImage &e = b->img[k];
            e.pixels = g.pixels;
            e.below = g.below;
            e.pitch = g.pitch;
            e.H = g.H;
            e.W = g.W;
            e.S = g.S;
            e.tile_begin = tiles;
            const size_t N = (size_t)e.H * e.W;
            tiles += (int)((N + tile_px - 1) / tile_px);
            total_streams += e.S;
            e.fc_off = off;
            off += align256(4 * N);
            e.words_off = off;
            off += align256(2 * (N + 2ull * e.S));
            e.cnt_off = off;
            off += align256(4ull * e.S);
            e.xfin_off = off;
            off += align256(4ull * e.S);
            e.soff_off = off;
            off += align256(4ull * e.S);
        }
        b->total_tiles = tiles;
        cudaError_t e = use_tc                       ? launch_predict_tc(m->dev, *b, err, m->num_sms, cs)
                        : m->dev.bits == 12          ? launch_predict12(m->dev, *b, err, cs)
                        : wide_supported(m->dev) ? launch_predict_wide(m->dev, m->hl, *b, ws + enc_ws_bytes(it), err, cs)
                                                     : launch_predict_cc(m->dev, *b, cs);
        if (e == cudaSuccess) e = launch_rans_encode(*b, total_streams, cs);
        if (e == cudaSuccess) e = launch_pack(m->dev, *b, out, d_out_offsets + c0, cs);
        delete b;
        if (e != cudaSuccess) return cuda_fail(e, "encode launch");
    }
    return DLIC_OK;
}

extern "C" dlic_status dlic_predict(const dlic_model *m, const dlic_image *im, int n, uint32_t *d_fc, int32_t *d_status,
                                    void *d_ws, size_t ws_bytes, void *stream) {
    if (!m) return fail(DLIC_ERR_INVALID, "null model");
    if (m->dev.vol) return fail(DLIC_ERR_INVALID, "the model has a 3D window: its priors span slices");
    dlic_status st = check_images(im, n, nullptr, false, m->dev.bits == 12 ? 2 : 1);
    if (st) return st;
    if (n == 0) return DLIC_OK;
    if (!d_fc) return fail(DLIC_ERR_INVALID, "null output");
    if (wide_supported(m->dev)) return fail(DLIC_ERR_UNSUPPORTED, "dlic_predict takes hidden widths up to 256");
    if (!d_status && (!d_ws || ws_bytes < 4)) return fail(DLIC_ERR_INVALID, "a status word or 4 bytes of workspace is needed");
    if (reinterpret_cast<uintptr_t>(d_fc) & 3) return fail(DLIC_ERR_INVALID, "d_fc must be 4-byte aligned");
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    int32_t *err = d_status ? d_status : static_cast<int32_t *>(d_ws);
    {
        cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int32_t), cs);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(status)");
    }
    const bool use_tc = m->dev.nl == 3 && m->dev.bits == 8 && tc_supported(m->dev);
    const int tile_px = use_tc ? 128 : kPredictTile;
    uint64_t px0 = 0;   // element offset of the chunk's first image in d_fc
    for (int c0 = 0; c0 < n; c0 += kMaxBatch) {
        const int cn = n - c0 < kMaxBatch ? n - c0 : kMaxBatch;
        EncBatch *b = new EncBatch();
        b->n = cn;
        b->ws = reinterpret_cast<uint8_t *>(d_fc);
        b->chunk_start = c0;
        b->tile_px = tile_px;
        b->raster = 1;
        int tiles = 0;
        for (int k = 0; k < cn; k++) {
            const dlic_image &g = im[c0 + k];
            EncImage &e = b->img[k];
            e.pixels = g.pixels;
            e.pitch = g.pitch;
            e.H = g.height;
            e.W = g.width;
            e.S = g.height;
            e.tile_begin = tiles;
            const size_t N = (size_t)e.H * e.W;
            tiles += (int)((N + tile_px - 1) / tile_px);
            e.fc_off = 4 * px0;
            px0 += N;
        }
        b->total_tiles = tiles;
        cudaError_t e = use_tc                  ? launch_predict_tc(m->dev, *b, err, m->num_sms, cs)
                        : m->dev.bits == 12 ? launch_predict12(m->dev, *b, err, cs)
                                            : launch_predict_cc(m->dev, *b, cs);
        delete b;
        if (e != cudaSuccess) return cuda_fail(e, "predict launch");
    }
    return DLIC_OK;
}

extern "C" dlic_status dlic_encode(const dlic_model *m, const dlic_image *im, int n, const int *streams,
                                   void *d_out, size_t out_capacity, uint64_t *d_out_offsets,
                                   int32_t *d_status, void *d_ws, size_t ws_bytes, void *stream) {
    if (!m) return fail(DLIC_ERR_INVALID, "null model");
    if (m->dev.vol) return fail(DLIC_ERR_INVALID, "the model has a 3D window: use dlic_encode_volume");
    dlic_status st = check_images(im, n, streams, false, m->dev.bits == 12 ? 2 : 1);
    if (st) return st;
    return encode_items(m, image_items(im, n, streams), d_out, out_capacity, d_out_offsets, d_status, d_ws, ws_bytes,
                        stream);
}

static dlic_status check_volumes(const dlic_volume *v, int n, bool decode) {
    if (n < 0) return fail(DLIC_ERR_INVALID, "negative volume count");
    if (n > 0 && !v) return fail(DLIC_ERR_INVALID, "null volume array");
    for (int i = 0; i < n; i++) {
        const dlic_volume &g = v[i];
        if (!g.pixels) return fail(DLIC_ERR_INVALID, "volume %d: null pixels", i);
        if (g.depth < 1 || g.height < 1 || g.width < 1)
            return fail(DLIC_ERR_INVALID, "volume %d: empty volume (%d x %d x %d)", i, g.depth, g.height, g.width);
        if (g.height > (1 << 20) || g.width > (1 << 20) || g.depth > kMaxSlices)
            return fail(DLIC_ERR_UNSUPPORTED, "volume %d: above 2^20 rows or columns or %d slices", i, kMaxSlices);
        if (g.pitch < g.width) return fail(DLIC_ERR_INVALID, "volume %d: pitch < width", i);
        if (g.slice_pitch < g.pitch * (int64_t)g.height) return fail(DLIC_ERR_INVALID, "volume %d: slices overlap", i);
        if (g.streams < (decode ? 1 : 0) || g.streams > 65535)
            return fail(DLIC_ERR_INVALID, "volume %d: stream count %d outside [%d, 65535]", i, g.streams, decode ? 1 : 0);
    }
    return DLIC_OK;
}

static int volume_streams(const dlic_volume &v) {
    const int s = v.streams ? v.streams : dlic_auto_streams(v.height, v.width);
    return s < v.height ? s : v.height;
}

static std::vector<EncItem> volume_items(const dlic_volume *v, int n) {
    std::vector<EncItem> it;
    for (int i = 0; i < n; i++)
        for (int z = 0; z < v[i].depth; z++) {
            const uint8_t *slice = v[i].pixels + (int64_t)z * v[i].slice_pitch;
            it.push_back({slice, z ? slice - v[i].slice_pitch : nullptr, v[i].height, v[i].width, volume_streams(v[i]),
                          v[i].pitch});
        }
    return it;
}

extern "C" dlic_status dlic_encode_volume_workspace_size(const dlic_model *m, const dlic_volume *v, int n,
                                                         size_t *bytes) {
    if (!m || !bytes) return fail(DLIC_ERR_INVALID, "null argument");
    dlic_status st = check_volumes(v, n, false);
    if (st) return st;
    *bytes = enc_ws_bytes(volume_items(v, n));
    return DLIC_OK;
}

extern "C" dlic_status dlic_encode_volume(const dlic_model *m, const dlic_volume *v, int n, void *d_out,
                                          size_t out_capacity, uint64_t *d_out_offsets, int32_t *d_status,
                                          void *d_ws, size_t ws_bytes, void *stream) {
    if (!m) return fail(DLIC_ERR_INVALID, "null model");
    if (!m->dev.vol) return fail(DLIC_ERR_INVALID, "the model has a 2D window: use dlic_encode");
    dlic_status st = check_volumes(v, n, false);
    if (st) return st;
    return encode_items(m, volume_items(v, n), d_out, out_capacity, d_out_offsets, d_status, d_ws, ws_bytes, stream);
}

extern "C" dlic_status dlic_read_header(const void *h_bits, size_t bytes, int *height, int *width,
                                        int *streams, int *precision, uint64_t *hash) {
    const uint8_t *h = static_cast<const uint8_t *>(h_bits);
    // byte 12: window rows above (1..8), bit 7 set in the slices of a volume
    if (!h || bytes < (size_t)kHeaderBytes || memcmp(h, "DLC1", 4) != 0 || (h[12] & 0x7F) < 1 || (h[12] & 0x7F) > 8)
        return fail(DLIC_ERR_CORRUPT, "not a DLIC bitstream");
    if (height) *height = (int)le32(h + 4);
    if (width) *width = (int)le32(h + 8);
    if (precision) *precision = h[13];
    if (streams) *streams = h[14] | (h[15] << 8);
    if (hash) {
        uint64_t v = 0;
        for (int k = 0; k < 8; k++) v |= (uint64_t)h[16 + k] << (8 * k);
        *hash = v;
    }
    return DLIC_OK;
}

// One image, or one volume, to decode.
struct DecItem {
    uint8_t *pixels;
    int H, W, D, S;
    int64_t pitch, slice_pitch;
};

// per item: stream states (a volume's: header, x, position, end per stream)
static size_t dec_item_bytes(const DecItem &e) {
    // a 2D image: up to H streams of 16 bytes (one CTA per image) or of 12
    // bytes after a 256-byte header (grid decoder)
    return e.D > 1 || e.S ? align256(256 + 12ull * e.D * e.S) : align256(256 + 16ull * e.H);
}

static size_t dec_ws_bytes(const std::vector<DecItem> &it) {
    size_t total = 0;
    for (const DecItem &e : it) total += dec_item_bytes(e);
    return total < 256 ? 256 : total;
}

static std::vector<DecItem> dec_image_items(const dlic_image *im, int n) {
    std::vector<DecItem> it((size_t)n);
    for (int i = 0; i < n; i++) it[i] = {im[i].pixels, im[i].height, im[i].width, 1, 0, im[i].pitch, 0};
    return it;
}

static std::vector<DecItem> dec_volume_items(const dlic_volume *v, int n) {
    std::vector<DecItem> it((size_t)n);
    for (int i = 0; i < n; i++)
        it[i] = {v[i].pixels, v[i].height, v[i].width, v[i].depth, volume_streams(v[i]), v[i].pitch, v[i].slice_pitch};
    return it;
}

extern "C" dlic_status dlic_decode_workspace_size(const dlic_model *m, const dlic_image *im, int n,
                                                  size_t *bytes) {
    if (!m || !bytes) return fail(DLIC_ERR_INVALID, "null argument");
    dlic_status st = check_images(im, n, nullptr, true, m->dev.bits == 12 ? 2 : 1);
    if (st) return st;
    *bytes = dec_ws_bytes(dec_image_items(im, n)) + wide_scratch_bytes(m->dev, false);
    return DLIC_OK;
}

extern "C" dlic_status dlic_decode_volume_workspace_size(const dlic_model *m, const dlic_volume *v, int n,
                                                         size_t *bytes) {
    if (!m || !bytes) return fail(DLIC_ERR_INVALID, "null argument");
    dlic_status st = check_volumes(v, n, true);
    if (st) return st;
    *bytes = dec_ws_bytes(dec_volume_items(v, n));
    return DLIC_OK;
}

// Decodes item i from bytes [h_in_offsets[i], h_in_offsets[i + 1]) of d_in
// (a volume: its slices' containers back to back).
static dlic_status decode_items(const dlic_model *m, const void *d_in, const uint64_t *h_in_offsets,
                                const std::vector<DecItem> &it, int32_t *d_status, void *d_ws, size_t ws_bytes,
                                void *stream) {
    const int n = (int)it.size();
    if (n == 0) return DLIC_OK;
    if (!d_in || !h_in_offsets || !d_status || !d_ws) return fail(DLIC_ERR_INVALID, "null buffer");
    const size_t need = dec_ws_bytes(it) + wide_scratch_bytes(m->dev, false);
    if (ws_bytes < need) return fail(DLIC_ERR_CAPACITY, "workspace %zu < %zu bytes", ws_bytes, need);
    // networks wider than 256: the layers' scratch after the stream states
    uint8_t *wide_scratch = static_cast<uint8_t *>(d_ws) + dec_ws_bytes(it);
    for (int i = 0; i < n; i++) {
        if (h_in_offsets[i + 1] < h_in_offsets[i]) return fail(DLIC_ERR_INVALID, "offsets must not decrease");
        if (h_in_offsets[i] & 1) return fail(DLIC_ERR_INVALID, "bitstream %d starts at an odd offset", i);
    }
    // stream read positions are 32-bit counts of 16-bit words
    if (h_in_offsets[n] >= (1ull << 33))
        return fail(DLIC_ERR_INVALID, "input of %llu bytes: at most 8 GiB per decode call",
                    (unsigned long long)h_in_offsets[n]);
    const bool vol = m->dev.vol != 0;
    const bool deep_wave = deep_wave_supported(m->dev);
    const bool use_wave = (m->dev.nl == 3 && m->dev.bits == 8 && wave_decode_supported(m->dev)) || deep_wave;
    if (vol && !use_wave) return fail(DLIC_ERR_UNSUPPORTED, "volumes decode on the cluster wavefront kernels only");
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    {
        cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(int32_t) * (size_t)n, cs);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(status)");
    }
    // workspace offsets of every image's stream states
    std::vector<size_t> st_off(n);
    {
        size_t off = 0;
        for (int i = 0; i < n; i++) {
            st_off[i] = off;
            off += dec_item_bytes(it[i]);
        }
    }
    // cluster size of every image (1 on the CUDA-core path)
    std::vector<int> P(n, 1), Hs(n), Ws(n);
    for (int i = 0; i < n; i++) {
        Hs[i] = it[i].H;
        Ws[i] = it[i].W;
    }
    auto fill = [&](DecImage &e, int i) {
        const DecItem &g = it[i];
        e.pixels = g.pixels;
        e.pitch = g.pitch;
        e.slice_pitch = g.slice_pitch;
        e.H = g.H;
        e.W = g.W;
        e.D = g.D;
        e.S = g.S ? g.S : g.H;   // 2D: the stream capacity of the grid decoder's state block
        e.in_off = h_in_offsets[i];
        e.in_bytes = h_in_offsets[i + 1] - h_in_offsets[i];
        e.st_off = st_off[i];
        e.sidx = i;
    };
    auto new_batch = [&]() {
        DecBatch *b = new DecBatch();
        b->in = static_cast<const uint8_t *>(d_in);
        b->ws = static_cast<uint8_t *>(d_ws);
        b->status = d_status;
        return b;
    };
    // Items that the whole GPU decodes as one cooperative grid (cluster size
    // 0: in no group): volumes one after another, or a 2D batch in chunks.
    std::vector<char> on_grid(n, 0);
    const int plan = m->decode_plan;
    if (use_wave) {
        if (vol) {
            // a volume's wave spans its slices: every SM (cooperative grid),
            // else the largest cluster that divides its stream count (each
            // CTA owns the rows k mod P)
            for (int i = 0; i < n; i++) {
                on_grid[i] = (plan == DLIC_PLAN_AUTO || plan == DLIC_PLAN_GRID) &&
                             grid_decode_eligible(m->dev, it[i].H, it[i].W, it[i].D, it[i].S);
                P[i] = 16;
                while (it[i].S % P[i]) P[i] >>= 1;
            }
        } else {
            choose_clusters(Hs.data(), Ws.data(), n, m->num_sms, m->dev.precision == DLIC_FP32, P.data());
            // The grid spreads every wave over all SMs but waits for its
            // slowest CTA at each wave; clusters run their images without a
            // common barrier.  AUTO takes the grid when the clusters would
            // leave most SMs idle while their CTAs hold several chunks of
            // pixels per wave (a few very wide images).
            int used = 0, per = 0;
            for (int i = 0; i < n; i++) {
                used += P[i];
                per = std::max(per, (std::min(it[i].H, (it[i].W + 2) / 3) + P[i] - 1) / P[i]);
            }
            // (deeper networks decode on clusters only)
            bool grid = !deep_wave && (plan == DLIC_PLAN_GRID ||
                                       (plan == DLIC_PLAN_AUTO && 2 * used <= m->num_sms && per > kGridMinChunkPixels));
            for (int c0 = 0; grid && c0 < n; c0 += kMaxBatch) {
                DecBatch *b = new_batch();
                b->n = std::min(kMaxBatch, n - c0);
                for (int k = 0; k < b->n; k++) fill(b->img[k], c0 + k);
                grid = grid_decode_fits(m->dev, *b, m->num_sms);
                delete b;
            }
            if (grid)
                for (int i = 0; i < n; i++) on_grid[i] = 1;
        }
        // checked before anything is enqueued
        for (int i = 0; i < n; i++)
            if (!on_grid[i] && !wave_decode_fits(m->dev, Hs[i], Ws[i], it[i].D, P[i], plan))
                return fail(DLIC_ERR_UNSUPPORTED, "image %d: %d x %d (x %d) needs more shared memory than the "
                            "decoder's plans allow", i, Hs[i], Ws[i], it[i].D);
    }
    for (int c0 = 0; c0 < n;) {
        if (!on_grid[c0]) {
            c0++;
            continue;
        }
        DecBatch *b = new_batch();
        b->n = 0;
        // a volume alone; 2D images in chunks of up to kMaxBatch
        for (int i = c0; i < n && on_grid[i] && b->n < (vol ? 1 : kMaxBatch); i++) fill(b->img[b->n++], i);
        for (int k = 0; k < b->n; k++) P[c0 + k] = 0;
        cudaError_t e = launch_decode_grid(m->dev, *b, m->num_sms, cs);
        const int first = c0;
        c0 += b->n;
        delete b;
        if (e != cudaSuccess)
            return e == cudaErrorNotSupported ? fail(DLIC_ERR_UNSUPPORTED, "item %d: the grid decoder does not fit", first)
                                              : cuda_fail(e, "grid decode launch");
    }
    int groups_used = 0;
    for (int gi = 0; gi < kDecodeGroups; gi++)
        for (int i = 0; i < n; i++)
            if (P[i] == (1 << gi)) {
                groups_used++;
                break;
            }
    const bool fork = groups_used > 1;
    int cluster_ctas = 0;   // CTAs of every cluster of the call
    for (int i = 0; i < n; i++) cluster_ctas += P[i];
    if (fork) {
        cudaError_t e = cudaEventRecord(m->fork_event, cs);
        if (e != cudaSuccess) return cuda_fail(e, "fork event");
    }
    // the largest clusters (the longest images) are launched first, and within
    // a group the longest images first, so that CTAs beyond one per SM queue
    // behind them
    const bool f32 = m->dev.precision == DLIC_FP32;
    dlic_status err = DLIC_OK;
    for (int gi = kDecodeGroups - 1; gi >= 0; gi--) {
        const int cluster = 1 << gi;
        std::vector<int> members;
        for (int i = 0; i < n; i++)
            if (P[i] == cluster) members.push_back(i);
        if (members.empty()) continue;
        if (use_wave)
            std::stable_sort(members.begin(), members.end(), [&](int a, int b) {
                return decode_estimate(Hs[a], Ws[a], cluster, f32) * it[a].D >
                       decode_estimate(Hs[b], Ws[b], cluster, f32) * it[b].D;
            });
        cudaStream_t gs = fork ? m->group_stream[gi] : cs;
        if (fork) {
            cudaError_t e = cudaStreamWaitEvent(gs, m->fork_event, 0);
            if (e != cudaSuccess) return cuda_fail(e, "fork wait");
        }
        for (size_t c0 = 0; c0 < members.size(); c0 += kMaxBatch) {
            const int cn = (int)std::min<size_t>(kMaxBatch, members.size() - c0);
            DecBatch *b = new DecBatch();
            b->n = cn;
            b->in = static_cast<const uint8_t *>(d_in);
            b->ws = static_cast<uint8_t *>(d_ws);
            b->status = d_status;
            for (int k = 0; k < cn; k++) fill(b->img[k], members[c0 + k]);
            cudaError_t e = use_wave              ? launch_decode_tc(m->dev, *b, cluster, m->num_sms, m->decode_plan, gs,
                                                                  2 * cluster_ctas <= m->num_sms)
                            : m->dev.bits == 12 ? launch_decode12(m->dev, *b, gs)
                            : wide_supported(m->dev) ? launch_decode_wide(m->dev, m->hl, *b, wide_scratch, gs)
                                                : launch_decode_cc(m->dev, *b, gs);
            delete b;
            if (e != cudaSuccess && err == DLIC_OK)
                err = e == cudaErrorNotSupported ? fail(DLIC_ERR_UNSUPPORTED, "decode launch: no shared-memory plan fits")
                                                 : cuda_fail(e, "decode launch");
            if (err != DLIC_OK) break;
        }
        // a forked group joins the caller's stream even after an error, so
        // that nothing launched outlives the call's ordering
        if (fork) {
            cudaError_t e = cudaEventRecord(m->join_event[gi], gs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, m->join_event[gi], 0);
            if (e != cudaSuccess && err == DLIC_OK) err = cuda_fail(e, "join");
        }
        if (err != DLIC_OK) break;
    }
    return err;
}

extern "C" dlic_status dlic_decode(const dlic_model *m, const void *d_in, const uint64_t *h_in_offsets,
                                   int n, const dlic_image *im, int32_t *d_status, void *d_ws,
                                   size_t ws_bytes, void *stream) {
    if (!m) return fail(DLIC_ERR_INVALID, "null model");
    if (m->dev.vol) return fail(DLIC_ERR_INVALID, "the model has a 3D window: use dlic_decode_volume");
    dlic_status st = check_images(im, n, nullptr, true, m->dev.bits == 12 ? 2 : 1);
    if (st) return st;
    return decode_items(m, d_in, h_in_offsets, dec_image_items(im, n), d_status, d_ws, ws_bytes, stream);
}

extern "C" dlic_status dlic_decode_volume(const dlic_model *m, const void *d_in, const uint64_t *h_in_offsets,
                                          int n, const dlic_volume *v, int32_t *d_status, void *d_ws,
                                          size_t ws_bytes, void *stream) {
    if (!m) return fail(DLIC_ERR_INVALID, "null model");
    if (!m->dev.vol) return fail(DLIC_ERR_INVALID, "the model has a 2D window: use dlic_decode");
    dlic_status st = check_volumes(v, n, true);
    if (st) return st;
    return decode_items(m, d_in, h_in_offsets, dec_volume_items(v, n), d_status, d_ws, ws_bytes, stream);
}
