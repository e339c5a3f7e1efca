// Host-only helper of tests/test_plan_host.py: prints the light-cone plans
// the library's planner (csrc/tc_fwd.cu, included whole) builds, one line per
// plan and one per layer, for the test to check against a model of the
// kernel's shared-memory accesses.  No kernel is launched.
#include "../paper_2108_13830_gb300/csrc/tc_fwd.cu"
#include <cstdio>

// the planner's error and workspace hooks, defined by the library proper
int vmc_fail(vmc_ctx *, int code, const char *, ...) { return code; }
int vmc_cuda_check(vmc_ctx *, cudaError_t e, const char *) { return e == cudaSuccess ? 0 : VMC_ERR_CUDA; }
int vmc_ensure_ws(vmc_ctx *, void **, size_t *, size_t) { return 0; }
cudaEvent_t vmc_timing_event(vmc_ctx *, bool, const char *) { return nullptr; }
namespace vmc {
namespace tc {
int launch_store_var(vmc_ctx *, const Plan &, const Params &, cudaStream_t) { return 0; }
int launch_cone_var(vmc_ctx *, const Plan &, const Params &, cudaStream_t) { return 0; }
}  // namespace tc
}  // namespace vmc

static void dump(const char *kind, const vmc::tc::Plan &q, int L, int C, int D, const vmc::tc::LayerGeo *g)
{
    printf("%s L %d C %d D %d S %d P %d G %d BUF %u smem %zu limit %d\n", kind, L, C, D, q.S, q.P,
           q.geo[L >> 1].G, q.BUF, q.smem, vmc::tc::SMEM_LIMIT);
    for (int l = 0; l <= D; ++l)
        printf("  l %d w %d T %d PW %d RW %d NRm %d\n", l, g[l].w, g[l].T, g[l].PW, g[l].RW, g[l].NRm);
}

static vmc_ctx make_ctx(int L, int C, int D)
{
    vmc_ctx ctx;
    ctx.L = L;
    ctx.arch.channels = C;
    ctx.arch.n_layers_cc = D;
    ctx.arch.precision = VMC_BF16;
    ctx.sm_count = 152;
    return ctx;
}

int main()
{
    // every light-cone candidate of the uniform planner (the autotuner's
    // search space, explicit tiles included)
    const int cases[][3] = {{6, 16, 1}, {6, 32, 1}, {8, 32, 2}, {8, 16, 2}, {10, 16, 6}, {10, 32, 3},
                            {12, 32, 4}, {12, 16, 8}, {14, 32, 5}, {16, 32, 8}, {16, 16, 6}, {20, 16, 8},
                            {24, 32, 10}, {32, 32, 14}};
    for (const auto &cs : cases) {
        vmc_ctx ctx = make_ctx(cs[0], cs[1], cs[2]);
        std::vector<vmc::tc::ConeCand> cands;
        vmc::tc::cone_cands(&ctx, cands);
        for (const auto &k : cands) {
            ctx.cone_tiles.slabs = k.S;
            ctx.cone_tiles.lane_cells = k.P;
            ctx.cone_tiles.slab_configs = k.G;
            vmc::tc::Plan q;
            if (vmc::tc::make_cone_plan(&ctx, &q) == VMC_OK) dump("uniform", q, cs[0], cs[1], cs[2], q.cone);
        }
    }
    // ragged plans: the cost model's, and every explicit slab count and P
    const int rcases[][3] = {{16, 16, 6}, {16, 32, 6}, {12, 32, 4}, {24, 32, 10}, {20, 16, 8}, {10, 16, 3}};
    for (const auto &cs : rcases) {
        for (int S = 0; S <= 2; ++S)
            for (int P = 0; P <= vmc::tc::MAX_P; ++P) {
                if ((S == 0) != (P == 0)) continue;
                vmc_ctx ctx = make_ctx(cs[0], cs[1], cs[2]);
                ctx.cone_tiles.slabs = S;
                ctx.cone_tiles.lane_cells = P;
                vmc::tc::Plan q;
                std::vector<vmc::tc::LayerGeo> tab;
                if (vmc::tc::make_cone_plan_ragged(&ctx, cs[0], &q, tab) != VMC_OK) continue;
                for (int L = 4; L <= cs[0]; L += 2)
                    if (q.geo[L >> 1].G > 0) dump("ragged", q, L, cs[1], cs[2], &tab[(L >> 1) * 17]);
            }
    }
    return 0;
}
