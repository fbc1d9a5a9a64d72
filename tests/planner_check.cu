// Host-only check of the wavefront decoder's shared-memory planner: compiled
// with nvcc by tests/test_planner.py (no GPU needed); prints one line per
// case: name ok nt tq gimg ring_rows list_rows lut2 total.
#include "../paper_2207_05152_gb300/csrc/decode_tc.cu"

#include <cstdio>

namespace dlic {
cudaError_t launch_decode_cc(const DevModel &, const DecBatch &, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace dlic

using namespace dlic;

static DevModel model(int prec, int u, int l, int r, int vol, int pu, int pd, int pl, int pr, int h) {
    DevModel m{};
    m.precision = prec;
    m.wu = u;
    m.wl = l;
    m.wr = r;
    m.n2 = u * (l + r + 1) + l;
    m.vol = vol;
    m.pu = pu;
    m.pd = pd;
    m.pl = pl;
    m.pr = pr;
    m.n_in = m.n2 + (vol ? (pu + pd + 1) * (pl + pr + 1) : 0);
    m.h1 = m.h2 = h;
    m.nl = 3;
    m.hmax = h;
    return m;
}

static void show(const char *name, bool ok, const DecTcParams &p, bool f32) {
    printf("%s %d %d %d %d %d %d %d %u\n", name, ok ? 1 : 0, p.nt, p.tq, p.gimg, p.ring_rows, p.list_rows, p.lut2,
           ok ? dec_layout(p, f32).total : 0u);
}

int main() {
    const uint32_t limit = 232448 - 5120;   // opt-in shared memory minus the kernel's static arrays
    struct C { const char *name; int prec, u, l, r, vol, pu, pd, pl, pr, h, H, W, D, P, plan; } cs[] = {
        {"int8_default_512", DLIC_INT8, 2, 2, 2, 0, 0, 0, 0, 0, 128, 512, 512, 1, 16, DLIC_PLAN_AUTO},
        {"fp32_default_512", DLIC_FP32, 2, 2, 2, 0, 0, 0, 0, 0, 128, 512, 512, 1, 16, DLIC_PLAN_AUTO},
        {"fp32_fig6_512", DLIC_FP32, 8, 6, 2, 0, 0, 0, 0, 0, 128, 512, 512, 1, 16, DLIC_PLAN_AUTO},
        {"int8_byte_ring_512", DLIC_INT8, 2, 2, 2, 0, 0, 0, 0, 0, 128, 512, 512, 1, 16, DLIC_PLAN_BYTE_RING},
        {"int8_image_512", DLIC_INT8, 2, 2, 2, 0, 0, 0, 0, 0, 128, 512, 512, 1, 16, DLIC_PLAN_IMAGE},
        {"int8_wide_4096x12288", DLIC_INT8, 2, 2, 2, 0, 0, 0, 0, 0, 128, 4096, 12288, 1, 16, DLIC_PLAN_AUTO},
        {"int8_huge_30000x90000", DLIC_INT8, 2, 2, 2, 0, 0, 0, 0, 0, 128, 30000, 90000, 1, 16, DLIC_PLAN_AUTO},
        {"int8_volume_35x256", DLIC_INT8, 2, 2, 2, 1, 1, 1, 1, 1, 128, 256, 256, 35, 16, DLIC_PLAN_AUTO},
    };
    for (const C &c : cs) {
        const DevModel m = model(c.prec, c.u, c.l, c.r, c.vol, c.pu, c.pd, c.pl, c.pr, c.h);
        DecTcParams p{};
        const bool ok = plan_wave(m, c.H, c.W, c.D, c.P, limit, c.plan, p);
        show(c.name, ok, p, c.prec == DLIC_FP32);
    }
    // the grid decoder: one volume, and the 64-image batch's largest sizes
    {
        const DevModel m = model(DLIC_INT8, 2, 2, 2, 1, 1, 1, 1, 1, 128);
        DecBatch *b = new DecBatch();
        b->n = 1;
        b->img[0].H = 512;
        b->img[0].W = 512;
        b->img[0].D = 128;
        DecTcParams p{};
        const bool ok = plan_grid(m, *b, 152, limit, p);
        show("grid_volume_128x512", ok, p, false);
        delete b;
    }
    {
        const DevModel m = model(DLIC_INT8, 2, 2, 2, 0, 0, 0, 0, 0, 128);
        DecBatch *b = new DecBatch();
        b->n = 64;
        for (int i = 0; i < 64; i++) {
            b->img[i].H = 1536;
            b->img[i].W = 2048;
            b->img[i].D = 1;
        }
        DecTcParams p{};
        const bool ok = plan_grid(m, *b, 152, limit, p);
        show("grid_batch_64x1536x2048", ok, p, false);
        delete b;
    }
    // INT8 networks of 1..5 hidden layers up to 128 wide (the deep instance:
    // up to four 128 x 128 bf16 hidden-to-hidden layers in shared memory)
    {
        static DevLayer table[kMaxLayers];   // (the planner reads only whether there is a table)
        struct D { const char *name; int nl, H, W, P; } ds[] = {
            {"six_layers_512", 6, 512, 512, 16}, {"six_layers_512_one_cta", 6, 512, 512, 1},
            {"one_hidden_512", 2, 512, 512, 16}, {"six_layers_4096x12288", 6, 4096, 12288, 16},
        };
        for (const D &d : ds) {
            DevModel m = model(DLIC_INT8, 2, 2, 2, 0, 0, 0, 0, 0, 128);
            m.bits = 8;
            m.nl = d.nl;
            m.layers = table;
            DecTcParams p{};
            const bool ok = deep_wave_supported(m) && plan_wave(m, d.H, d.W, 1, d.P, limit, DLIC_PLAN_AUTO, p);
            printf("deep %s %d %d %d %d %d %d %u\n", d.name, ok ? 1 : 0, p.deep, p.nhh, p.smma, p.nt, p.gimg,
                   ok ? dec_layout(p, false).total : 0u);
        }
    }
    // the decode autotuner: cluster sizes for a few batches
    {
        const int H1[1] = {512}, W1[1] = {512};
        int P1[1];
        choose_clusters(H1, W1, 1, 152, false, P1);
        printf("clusters single_512 %d\n", P1[0]);
        int H64[64], W64[64], P64[64];
        for (int i = 0; i < 64; i++) {
            H64[i] = 192 + (i * 37) % 1345;
            W64[i] = 256 + (i * 53) % 1793;
        }
        choose_clusters(H64, W64, 64, 152, false, P64);
        printf("clusters batch64");
        for (int i = 0; i < 64; i++) printf(" %d", P64[i]);
        printf("\n");
        int Ht[200], Wt[200], Pt[200];
        for (int i = 0; i < 200; i++) {
            Ht[i] = 16;
            Wt[i] = 16;
        }
        choose_clusters(Ht, Wt, 200, 152, false, Pt);
        printf("clusters tiny200 %d %d\n", Pt[0], Pt[199]);
    }
    return 0;
}
