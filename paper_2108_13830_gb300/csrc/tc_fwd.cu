// Host side of the tensor-core forward: slab planning, launches, the tile
// autotuner and diagnostics.  The kernel itself is in tc_kern.cuh.
#include <algorithm>
#include <cstring>
#include <vector>
#include "tc_kern.cuh"

namespace vmc {
namespace tc {


// ------------------------------------------------------------------ planning

// control block, spins, bond list, biases
static size_t ctrl_bytes(int L_max, int C, int D)
{
    return sizeof(Ctrl) + ((L_max * L_max + 15) & ~15) + (((size_t)8 * L_max * L_max + 15) & ~(size_t)15) +
           (size_t)(D + 1) * C * 4 + 64;
}

// Slab of G lattices of side L with P cells per TMEM lane: tiles per layer,
// grid row width, and the rows per plane any MMA or store of the slab
// touches (row 0 is a spare row in front of the grid).
static int geo_rows(int L, int G, int P, int *T_out, int *PW_out)
{
    const int PW = (G * (L + 2) + P - 1) / P * P;
    const int RW = PW / P;
    const int NR = L * RW;
    const int T = (NR + 127) / 128;
    const int r_last = RW + std::min(128 * (T - 1), std::max(NR - 128, 0));
    *T_out = T;
    *PW_out = PW;
    return std::max((L + 2) * RW, r_last + 128 + RW + 1) + 1;
}

// issue cycles of one 128 x N x 16 MMA (measured on sm_103a: flat below
// N = 64, then limited by the shared-memory operand reads)
static double mma_cycles(int N) { return N <= 64 ? 50.0 : (N <= 96 ? 56.0 : 64.0 + (N - 128) * 0.5); }

// modelled MMA cycles per tile of a C -> C layer
static double tile_cycles(int C, int P)
{
    double per = 2 * mma_cycles(C);
    for (int i = 0; i < P; ++i) {
        const int jlo = std::max(0, 1 - i), jhi = std::min(2, P - i);
        per += mma_cycles((jhi - jlo + 1) * C);
    }
    return per * 3 * (C / 16);
}

// P C <= 128 keeps at most 64 accumulator values per epilogue thread and
// at least four TMEM slots
static bool p_allowed(int C, int P)
{
    if (P < 1 || P > MAX_P || P * C > 128) return false;
    return (P * C) % 32 == 0;
}

struct Cand {
    Geo g;
    double score;   // modelled cycles per useful lattice cell
};

// every geometry of lattice L within `buf` bytes per buffer, with its score
static void geo_cands(int C, int L, uint32_t buf, int S, std::vector<Cand> &out)
{
    for (int P = 1; P <= MAX_P; ++P) {
        if (!p_allowed(C, P)) continue;
        for (int G = 1; G <= MAX_SLOTS; ++G) {
            int T, PW;
            const int rows = geo_rows(L, G, P, &T, &PW);
            if ((size_t)rows * P * C * 2 > buf) break;
            double sc = T * tile_cycles(C, P) / ((double)G * L * L);
            if (S == 1) sc *= 1.0 + 0.5 / T;   // one slab: the layer barrier is not overlapped
            out.push_back(Cand{Geo{G, P, T, PW}, sc});
        }
    }
}


static uint32_t buf_bytes(int C, int S, int L_max, int D)
{
    const size_t wb = 2 * (size_t)(18 * C * C);
    const size_t avail = SMEM_LIMIT - wb - ctrl_bytes(L_max, C, D) - 1024;
    return (uint32_t)((avail / (2 * (size_t)S)) & ~(size_t)127);
}

// best geometry of lattice L under the tile choice `tc` (0 fields free)
static Geo pick_geo(int C, int L, int S, uint32_t buf, const TileChoice &tc, double *score)
{
    std::vector<Cand> cs;
    geo_cands(C, L, buf, S, cs);
    Geo best{0, 0, 0, 0};
    double bs = 1e300;
    for (const Cand &cd : cs) {
        if (tc.slab_configs && cd.g.G != tc.slab_configs) continue;
        if (tc.lane_cells && cd.g.P != tc.lane_cells) continue;
        if (cd.score < bs - 1e-12) { bs = cd.score; best = cd.g; }
    }
    if (score) *score = bs;
    return best;
}

static int make_plan(const vmc_ctx *ctx, int L_main, int L_max, bool ragged, Plan *pl)
{
    const int C = ctx->arch.channels, D = ctx->arch.n_layers_cc;
    TileChoice tc;
    auto it = ctx->tiles.find(L_main);
    if (it != ctx->tiles.end()) tc = it->second;
    int S = tc.slabs;
    if (!S) {
        // the slab count with the better modelled geometry for L_main
        double s1 = 0, s2 = 0;
        const Geo g1 = pick_geo(C, L_main, 1, buf_bytes(C, 1, L_max, D), tc, &s1);
        const Geo g2 = pick_geo(C, L_main, 2, buf_bytes(C, 2, L_max, D), tc, &s2);
        if (g2.G && (s2 <= s1 || !g1.G)) S = 2;
        else S = 1;
    }
    const uint32_t buf = buf_bytes(C, S, L_max, D);
    pl->S = S;
    pl->BUF = buf;
    for (int i = 0; i < 17; ++i) pl->geo[i] = Geo{0, 0, 0, 0};
    // one lane packing per launch (the epilogue is compiled for it): that of
    // L_main; every other lattice side of a mixed launch takes its best G
    // under the same P
    const Geo gmain = pick_geo(C, L_main, S, buf, tc, nullptr);
    if (!gmain.G) return VMC_ERR_UNSUPPORTED;
    const int P = gmain.P;
    for (int L = 4; L <= L_max; L += 2) {
        if (!ragged && L != L_main) continue;
        TileChoice tl;
        auto jt = ctx->tiles.find(L);
        if (jt != ctx->tiles.end()) tl = jt->second;
        tl.lane_cells = P;
        pl->geo[L >> 1] = (L == L_main) ? gmain : pick_geo(C, L, S, buf, tl, nullptr);
    }
    pl->P = P;
    pl->slotc = P * C;
    pl->smem = 2 * (size_t)(18 * C * C) + (size_t)2 * S * buf + ctrl_bytes(L_max, C, D);
    if (pl->smem > SMEM_LIMIT) return VMC_ERR_UNSUPPORTED;
    return VMC_OK;
}

// ------------------------------------------------------------------ light cone

// Side of the window of layer l: after layer l the activations of sigma'
// that differ from the parent's lie within l + 1 cells (3 x 3 filters) of
// the exchanged pair, a (2l+4) x (2l+3) box for a horizontal J1 pair, its
// transpose for a vertical one and (2l+4)^2 for a diagonal J2 pair.  Every
// pair takes the square of side 2l + 4, capped at L (the whole lattice).
static int cone_w(int L, int l) { return std::min(2 * l + 4, L); }

static LayerGeo cone_layer(int L, int l, int G, int P, int *rows)
{
    LayerGeo g;
    g.w = cone_w(L, l);
    int T, PW;
    *rows = geo_rows(g.w, G, P, &T, &PW);
    g.T = T;
    g.PW = PW;
    g.RW = PW / P;
    g.NRm = std::max(g.w * g.RW - 128, 0);
    g.mRW = udiv_magic((uint32_t)g.RW);
    g.mLP = udiv_magic((uint32_t)(g.w + 2));
    g.mRing = udiv_magic((uint32_t)(8 * g.w + 16));
    g.mW4 = udiv_magic((uint32_t)(g.w + 4));
    return g;
}

// Modelled cycles of one neighbour through every layer with G windows per
// slab, shared by the G windows.  A layer whose windows fit one tile is a
// strict chain (its MMAs, then its drain, then the next layer's MMAs; two
// slabs overlap two such chains); a wider layer costs its tiles' epilogue
// drains (the tile-level hand-off hides its MMAs); every slab pays the
// pooling and the next fill.  The constants are fitted to measured launch
// times over C = 16 and 32, L = 8 .. 24, one and two slabs, P = 1 .. 8:
// the model's pick is within 0-6 % of the fastest measured choice at each
// size (vmc_autotune times the best-modelled plans).
static double cone_cost(int C, int L, int D, int G, int P, int S)
{
    const double nm = P * C / 32.0;                           // accumulator chunks per epilogue thread
    const double mma = 312.0 * 3 * (C / 16) * (P + 2);        // one tile's MMAs
    const double drain = 1070.0 + 1220.0 * nm;                // one tile's epilogue
    const double chain = mma + drain;                         // a one-tile layer: MMAs, then the drain
    double cyc = 170.0 + drain;                               // the embedding layer
    for (int l = 1; l <= D; ++l) {
        int rows;
        const LayerGeo g = cone_layer(L, l, G, P, &rows);
        if (g.T == 1) cyc += S == 1 ? chain : std::max(chain / 2, drain);
        else cyc += g.T * drain + (S == 1 ? 1240.0 : 0.0);
    }
    cyc += 11900.0 + 680.0 * G;                               // pooling and the next fill
    return cyc / G;
}

// Applies when the window covers the lattice by the last layer (the pooling
// then runs over whole lattices) and starts smaller than it.
bool cone_applies_impl(const vmc_ctx *ctx)
{
    const int L = ctx->L, D = ctx->arch.n_layers_cc;
    return vmc_is_tc(ctx->arch.precision) && L >= 6 && cone_w(L, D) == L;
}

// every (slabs, lane cells, windows per slab) of the light-cone pass that
// fits shared memory, with its modelled cost
struct ConeCand {
    int S, P, G;
    double score;
};

static void cone_cands(const vmc_ctx *ctx, std::vector<ConeCand> &out)
{
    const int C = ctx->arch.channels, D = ctx->arch.n_layers_cc, L = ctx->L;
    for (int S = 1; S <= 2; ++S) {
        const uint32_t buf = buf_bytes(C, S, L, D);
        for (int P = 1; P <= MAX_P; ++P) {
            if (!p_allowed(C, P)) continue;
            for (int G = 1; G <= MAX_SLOTS; ++G) {
                int rows_max = 0;
                for (int l = 0; l <= D; ++l) {
                    int rows;
                    cone_layer(L, l, G, P, &rows);
                    rows_max = std::max(rows_max, rows);
                }
                if ((size_t)rows_max * P * C * 2 > buf) break;
                out.push_back(ConeCand{S, P, G, cone_cost(C, L, D, G, P, S)});
            }
        }
    }
}

static int make_cone_plan(const vmc_ctx *ctx, Plan *pl)
{
    const int C = ctx->arch.channels, D = ctx->arch.n_layers_cc, L = ctx->L;
    const TileChoice &tc = ctx->cone_tiles;
    double best = 1e300;
    int bS = 0, bG = 0, bP = 0;
    for (int S = 1; S <= 2; ++S) {
        if (tc.slabs && S != tc.slabs) continue;
        const uint32_t buf = buf_bytes(C, S, L, D);
        for (int P = 1; P <= MAX_P; ++P) {
            if (!p_allowed(C, P)) continue;
            if (tc.lane_cells && P != tc.lane_cells) continue;
            for (int G = 1; G <= MAX_SLOTS; ++G) {
                int rows_max = 0;
                for (int l = 0; l <= D; ++l) {
                    int rows;
                    cone_layer(L, l, G, P, &rows);
                    rows_max = std::max(rows_max, rows);
                }
                if ((size_t)rows_max * P * C * 2 > buf) break;
                if (tc.slab_configs && G != tc.slab_configs) continue;
                const double sc = cone_cost(C, L, D, G, P, S);
                if (sc < best - 1e-9) { best = sc; bS = S; bG = G; bP = P; }
            }
        }
    }
    if (!bG) return VMC_ERR_UNSUPPORTED;
    pl->S = bS;
    pl->P = bP;
    pl->BUF = buf_bytes(C, bS, L, D);
    pl->slotc = bP * C;
    for (int i = 0; i < 17; ++i) { pl->geo[i] = Geo{0, 0, 0, 0}; pl->cone[i] = LayerGeo{}; }
    for (int l = 0; l <= D; ++l) {
        int rows;
        pl->cone[l] = cone_layer(L, l, bG, bP, &rows);
    }
    pl->geo[L >> 1] = Geo{bG, bP, pl->cone[D].T, pl->cone[D].PW};
    pl->smem = 2 * (size_t)(18 * C * C) + (size_t)2 * bS * pl->BUF + ctrl_bytes(L, C, D);
    if (pl->smem > SMEM_LIMIT) return VMC_ERR_UNSUPPORTED;
    return VMC_OK;
}

// Light-cone plan for a ragged batch of sides 4 .. L_max: one slab count and
// lane packing P for the launch (its kernel is compiled for one P), the
// best number of windows per slab for each side, and the per-side layer
// geometry as a [L / 2][layer] table.  (S, P) minimise the summed modelled
// cost of the sides, each weighted by its neighbour count 2 L^2.
static int make_cone_plan_ragged(const vmc_ctx *ctx, int L_max, Plan *pl, std::vector<LayerGeo> &tab)
{
    const int C = ctx->arch.channels, D = ctx->arch.n_layers_cc;
    if (cone_w(L_max, D) != L_max) return VMC_ERR_UNSUPPORTED;
    // explicit light-cone tiles: slabs and P for the launch, windows per slab
    // as every side's upper bound
    const TileChoice &tc = ctx->cone_tiles;
    const int gmax = tc.slab_configs ? std::min(tc.slab_configs, MAX_SLOTS) : MAX_SLOTS;
    double best = 1e300;
    int bS = 0, bP = 0;
    for (int S = 1; S <= 2; ++S) {
        if (tc.slabs && S != tc.slabs) continue;
        const uint32_t buf = buf_bytes(C, S, L_max, D);
        for (int P = 1; P <= MAX_P; ++P) {
            if (!p_allowed(C, P)) continue;
            if (tc.lane_cells && P != tc.lane_cells) continue;
            double tot = 0;
            bool ok = true;
            for (int L = 4; L <= L_max && ok; L += 2) {
                double bl = 1e300;
                for (int G = 1; G <= gmax; ++G) {
                    int rows_max = 0;
                    for (int l = 0; l <= D; ++l) {
                        int rows;
                        cone_layer(L, l, G, P, &rows);
                        rows_max = std::max(rows_max, rows);
                    }
                    if ((size_t)rows_max * P * C * 2 > buf) break;
                    bl = std::min(bl, cone_cost(C, L, D, G, P, S));
                }
                if (bl >= 1e299) ok = false;
                else tot += bl * 2.0 * L * L;
            }
            if (ok && tot < best - 1e-9) { best = tot; bS = S; bP = P; }
        }
    }
    if (!bS) return VMC_ERR_UNSUPPORTED;
    pl->S = bS;
    pl->P = bP;
    pl->BUF = buf_bytes(C, bS, L_max, D);
    pl->slotc = bP * C;
    for (int i = 0; i < 17; ++i) { pl->geo[i] = Geo{0, 0, 0, 0}; pl->cone[i] = LayerGeo{}; }
    tab.assign(17 * 17, LayerGeo{});
    for (int L = 4; L <= L_max; L += 2) {
        double bl = 1e300;
        int bG = 0;
        for (int G = 1; G <= gmax; ++G) {
            int rows_max = 0;
            for (int l = 0; l <= D; ++l) {
                int rows;
                cone_layer(L, l, G, bP, &rows);
                rows_max = std::max(rows_max, rows);
            }
            if ((size_t)rows_max * bP * C * 2 > pl->BUF) break;
            const double sc = cone_cost(C, L, D, G, bP, bS);
            if (sc < bl - 1e-9) { bl = sc; bG = G; }
        }
        for (int l = 0; l <= D; ++l) {
            int rows;
            tab[(L >> 1) * 17 + l] = cone_layer(L, l, bG, bP, &rows);
        }
        pl->geo[L >> 1] = Geo{bG, bP, tab[(L >> 1) * 17 + D].T, tab[(L >> 1) * 17 + D].PW};
    }
    pl->smem = 2 * (size_t)(18 * C * C) + (size_t)2 * bS * pl->BUF + ctrl_bytes(L_max, C, D);
    if (pl->smem > SMEM_LIMIT) return VMC_ERR_UNSUPPORTED;
    return VMC_OK;
}

// Parameters of one launch that do not depend on the variant.
static Params base_params(const vmc_ctx *ctx, const Plan &pl, int mode, const int8_t *sigma, const int64_t *offs,
                          const int32_t *Ls, int64_t B, int L_max, double *out_a, void *out_b, int32_t *n_nbr)
{
    Params p{};
    p.mode = mode; p.B = B; p.sigma = sigma; p.offs = offs; p.Ls = Ls;
    p.L_uniform = ctx->L; p.L_max = L_max;
    p.D = ctx->arch.n_layers_cc; p.marshall = ctx->arch.marshall_sign;
    p.J1 = ctx->J1; p.J2 = ctx->J2;
    p.wimg = reinterpret_cast<const uint8_t *>(ctx->wimg);
    p.bias32 = ctx->bias32;
    p.S = pl.S; p.BUF = pl.BUF;
    p.slotc = pl.slotc;
    p.nslots = std::min(MAX_TSLOTS, 512 / pl.slotc);
    for (int i = 0; i < 17; ++i) p.geo[i] = pl.geo[i];
    for (int i = 0; i < 17; ++i) p.cone[i] = pl.cone[i];
    p.out_a = out_a; p.out_sign = static_cast<int8_t *>(out_b); p.n_nbr = n_nbr;
    p.status = ctx->status; p.counter = ctx->counter;
    p.budget_ns = ctx->wait_budget_ns;
    return p;
}

static int launch_any(vmc_ctx *ctx, const Plan &pl, int mode, const int8_t *sigma, const int64_t *offs,
                      const int32_t *Ls, int64_t B, int L_max, double *out_a, void *out_b, int32_t *n_nbr,
                      cudaStream_t st)
{
    const Params p = base_params(ctx, pl, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr);
    return launch_var<VAR_PLAIN>(ctx, pl, p, st);
}

// ------------------------------------------------------------------ diagnostics

// One UMMA tile, M = 128, N, K, from row-major BF16 A [128 + shift][K] and
// B [N][K]; D FP32 [128][N].  variant 0: descriptors as used by the
// forward kernel; variant 1: LBO / SBO fields exchanged (layout probe).
__global__ void umma_selftest_kernel(const uint16_t *A, const uint16_t *Bm, float *Dm, int N, int K, int shift,
                                     int variant)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rows = 128 + shift + 8;
    const uint32_t PSA = (uint32_t)rows * 16u;
    uint8_t *As = sm;                   // K/8 planes of `rows` 16-byte rows
    uint8_t *Bs = sm + 65536;           // K/16 chunks of 32 N bytes
    for (int i = tid; i < rows * K; i += blockDim.x) {
        const int r = i / K, k = i - r * K;
        const uint16_t v = (r < 128 + shift) ? A[r * K + k] : (uint16_t)0;
        *reinterpret_cast<uint16_t *>(As + (k >> 3) * PSA + r * 16 + (k & 7) * 2) = v;
    }
    for (int i = tid; i < N * K; i += blockDim.x) {
        const int n = i / K, k = i - n * K;
        *reinterpret_cast<uint16_t *>(Bs + (k >> 4) * 32 * N + tc_b_elem_offset(N, n, k & 15)) = Bm[n * K + k];
    }
    if (tid == 0) { mbar_init(&bar, 1); mbar_fence_init(); }
    fence_proxy_async_smem();
    if (warp == 0) tmem_alloc(&tbase, 128);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        const uint32_t idesc = idesc_bf16(128, N);
        for (int kc = 0; kc < K / 16; ++kc) {
            const uint32_t a = smem_u32(As) + 2 * kc * PSA + shift * 16;
            const uint32_t b = smem_u32(Bs) + kc * 32 * N;
            const uint64_t ad = variant ? smem_desc(a, 128, PSA) : smem_desc(a, PSA, 128);
            const uint64_t bd = variant ? smem_desc(b, 128, 16 * N) : smem_desc(b, 16 * N, 128);
            umma_bf16(tbase, ad, bd, idesc, kc > 0);
        }
        umma_commit(&bar);
    }
    __shared__ int abort_flag, fl, site;   // the wait may raise status bits atomically
    if (tid == 0) { abort_flag = 0; fl = 0; site = 0; }
    __syncthreads();
    mbar_wait_bounded(&bar, 0, &abort_flag, 1000000000LL, &fl, &site, 0);
    tc_fence_after();
    if (warp < 4) {
        for (int c0 = 0; c0 < N; c0 += 8) {
            float v[8];
            tmem_ld8(tbase + ((uint32_t)(warp * 32) << 16) + c0, v);
            for (int i = 0; i < 8; ++i) Dm[(warp * 32 + lane) * N + c0 + i] = abort_flag ? -12345.f : v[i];
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tbase, 128);
}

__global__ void wait_timeout_kernel(DevStatus *st, long long budget)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) { mbar_init(&bar, 1); mbar_fence_init(); abort_flag = 0; }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, &abort_flag, budget, &st->flags, &st->timeout_site, 99);
    __syncthreads();
}

// Synthetic probe configurations for the autotuner: the Neel state with a
// counter-hashed set of exchanges (keeps S^z = 0).
__global__ void probe_configs_kernel(int8_t *out, int L, int64_t B)
{
    const int N = L * L;
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        int8_t *s = out + b * N;
        if (threadIdx.x == 0) {
            for (int i = 0; i < N; ++i) s[i] = (((i / L) + (i % L)) & 1) ? -1 : 1;
            uint32_t h = (uint32_t)b * 2654435761u + 12345u;
            for (int k = 0; k < N; ++k) {
                h ^= h << 13; h ^= h >> 17; h ^= h << 5;
                const int i = (int)(h % (uint32_t)N);
                h ^= h << 13; h ^= h >> 17; h ^= h << 5;
                const int j = (int)(h % (uint32_t)N);
                const int8_t t = s[i]; s[i] = s[j]; s[j] = t;
            }
        }
    }
}

}  // namespace tc
}  // namespace vmc



using namespace vmc;

int vmc_tc_default_tiles(const vmc_ctx *ctx, int L, TileChoice *t)
{
    tc::Plan pl;
    const int rc = tc::make_plan(ctx, L, L, false, &pl);
    if (rc) return rc;
    t->slab_configs = pl.geo[L >> 1].G;
    t->slabs = pl.S;
    t->ctas_per_sm = 1;
    t->lane_cells = pl.geo[L >> 1].P;
    return VMC_OK;
}

bool vmc_tc_cone_applies(const vmc_ctx *ctx) { return tc::cone_applies_impl(ctx); }

int vmc_tc_cone_default_tiles(const vmc_ctx *ctx, TileChoice *t)
{
    if (!tc::cone_applies_impl(ctx)) return VMC_ERR_UNSUPPORTED;
    tc::Plan pl;
    const int rc = tc::make_cone_plan(ctx, &pl);
    if (rc) return rc;
    t->slab_configs = pl.geo[ctx->L >> 1].G;
    t->slabs = pl.S;
    t->ctas_per_sm = 1;
    t->lane_cells = pl.P;
    return VMC_OK;
}

// Local energy with light-cone neighbours (uniform L): per chunk of parents,
// a parent pass (log|psi_CNN| and every layer's activations to the store),
// then the neighbour pass, which recomputes only each neighbour's cone and
// takes the rest of every layer from the parent.  The results equal those
// of the plain forward bit for bit: every evaluated cell sums the same taps
// in the same order, and the pooling adds the last layer in lattice order.
static int tc_eloc_cone(vmc_ctx *ctx, const int8_t *sigma, int64_t B, double *out_a, int32_t *n_nbr, cudaStream_t s)
{
    const int L = ctx->L, C = ctx->arch.channels, D = ctx->arch.n_layers_cc, N = L * L;
    tc::Plan pp, pc;
    int rc = tc::make_plan(ctx, L, L, false, &pp);
    if (rc) return vmc_fail(ctx, rc, "no tensor-core plan for L=%d C=%d", L, C);
    rc = tc::make_cone_plan(ctx, &pc);
    if (rc) return vmc_fail(ctx, rc, "no light-cone plan for L=%d C=%d", L, C);
    const long long stride = (long long)D * C * N * 2;
    const int64_t cap = (int64_t)2 << 30;
    const int64_t Bc = std::max<int64_t>(1, std::min<int64_t>(B, cap / stride));
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t need = al((size_t)Bc * stride) + al((size_t)Bc * 8) + al((size_t)Bc);
    rc = vmc_ensure_ws(ctx, &ctx->cone_ws, &ctx->cone_ws_bytes, need);
    if (rc) return rc;
    uint8_t *store = static_cast<uint8_t *>(ctx->cone_ws);
    double *la = reinterpret_cast<double *>(store + al((size_t)Bc * stride));
    int8_t *sg = reinterpret_cast<int8_t *>(reinterpret_cast<uint8_t *>(la) + al((size_t)Bc * 8));
    for (int64_t b0 = 0; b0 < B; b0 += Bc) {
        const int64_t nb = std::min(Bc, B - b0);
        const int8_t *sb = sigma + b0 * N;
        tc::Params p1 = tc::base_params(ctx, pp, 0, sb, nullptr, nullptr, nb, L, la, sg, nullptr);
        p1.act_store = store;
        p1.store_stride = stride;
        rc = tc::launch_store_var(ctx, pp, p1, s);
        if (rc) return rc;
        tc::Params p2 = tc::base_params(ctx, pc, 1, sb, nullptr, nullptr, nb, L, out_a + b0, nullptr,
                                        n_nbr ? n_nbr + b0 : nullptr);
        p2.act_store = store;
        p2.store_stride = stride;
        p2.par_la = la;
        p2.par_sg = sg;
        rc = tc::launch_cone_var(ctx, pc, p2, s);
        if (rc) return rc;
    }
    return VMC_OK;
}

namespace vmc {
namespace tc {

// Work order of a ragged batch: samples grouped by lattice side, largest
// first (the longest work starts first and the small lattices fill the tail;
// slabs hold one lattice side, so grouping also keeps them full), invalid
// sides last.  One CTA: a histogram, a scan from the largest side down, and
// a scatter (the order inside a group is immaterial: every sample's results
// are independent of where it is processed).
__global__ void ragged_order_kernel(const int32_t *__restrict__ Ls, int64_t B, int L_max, int64_t *order)
{
    __shared__ unsigned long long cnt[18];
    const int nb = 18;   // bins 2..16 (L = 4..32), bin 17 invalid
    for (int i = threadIdx.x; i < nb; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    auto bin_of = [&](int L) { return ((L & 1) || L < 4 || L > L_max) ? 17 : (L >> 1); };
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) atomicAdd(&cnt[bin_of(Ls[b])], 1ull);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long acc = 0;
        for (int k = 16; k >= 2; --k) { const unsigned long long c = cnt[k]; cnt[k] = acc; acc += c; }
        const unsigned long long c = cnt[17];
        cnt[17] = acc;
        (void)c;
    }
    __syncthreads();
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
        const unsigned long long pos = atomicAdd(&cnt[bin_of(Ls[b])], 1ull);
        order[pos] = b;
    }
}

}  // namespace tc
}  // namespace vmc

int vmc_tc_eloc(vmc_ctx *ctx, int mode, const int8_t *sigma, const int64_t *offs, const int32_t *Ls,
                int64_t B, int L_max, double *out_a, void *out_b, int32_t *n_nbr, cudaStream_t s)
{
    if (mode == 1 && !Ls && !offs && ctx->light_cone && tc::cone_applies_impl(ctx))
        return tc_eloc_cone(ctx, sigma, B, out_a, n_nbr, s);
    tc::Plan pl;
    const bool ragged = (Ls != nullptr);
    int rc = tc::make_plan(ctx, ragged ? L_max : ctx->L, L_max, ragged, &pl);
    if (rc) return vmc_fail(ctx, rc, "no tensor-core plan for L=%d C=%d", L_max, ctx->arch.channels);
    if (!ragged) return tc::launch_any(ctx, pl, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr, s);
    rc = vmc_ensure_ws(ctx, &ctx->order_ws, &ctx->order_ws_bytes, (size_t)B * sizeof(int64_t));
    if (rc) return rc;
    int64_t *order = static_cast<int64_t *>(ctx->order_ws);
    tc::ragged_order_kernel<<<1, 1024, 0, s>>>(Ls, B, L_max, order);
    ctx->launches += 1;
    rc = vmc_cuda_check(ctx, cudaGetLastError(), "ragged order");
    if (rc) return rc;
    // light cone over the ragged batch: every side shares the launch's P;
    // the parent store is sized for L_max (in one piece, at most 2 GiB)
    const int C = ctx->arch.channels, D = ctx->arch.n_layers_cc;
    const long long stride = (long long)D * C * L_max * L_max * 2;
    tc::Plan pc;
    std::vector<tc::LayerGeo> tab;
    if (mode == 1 && ctx->light_cone && (long long)B * stride <= ((long long)2 << 30) &&
        tc::make_cone_plan_ragged(ctx, L_max, &pc, tab) == VMC_OK) {
        // the per-side table goes to the device once per plan (before any capture)
        const size_t tb = tab.size() * sizeof(tc::LayerGeo);
        const char *th = reinterpret_cast<const char *>(tab.data());
        if (ctx->cone_tab_host.size() != tb || memcmp(ctx->cone_tab_host.data(), th, tb) != 0) {
            rc = vmc_ensure_ws(ctx, &ctx->cone_tab, &ctx->cone_tab_bytes, tb);
            if (rc) return rc;
            rc = vmc_cuda_check(ctx, cudaMemcpy(ctx->cone_tab, th, tb, cudaMemcpyHostToDevice), "cone table");
            if (rc) return rc;
            ctx->cone_tab_host.assign(th, th + tb);
        }
        auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
        const size_t need = al((size_t)B * stride) + al((size_t)B * 8) + al((size_t)B);
        rc = vmc_ensure_ws(ctx, &ctx->cone_ws, &ctx->cone_ws_bytes, need);
        if (rc) return rc;
        uint8_t *store = static_cast<uint8_t *>(ctx->cone_ws);
        double *la = reinterpret_cast<double *>(store + al((size_t)B * stride));
        int8_t *sg = reinterpret_cast<int8_t *>(reinterpret_cast<uint8_t *>(la) + al((size_t)B * 8));
        tc::Params p1 = tc::base_params(ctx, pl, 0, sigma, offs, Ls, B, L_max, la, sg, nullptr);
        p1.order = order;
        p1.act_store = store;
        p1.store_stride = stride;
        rc = tc::launch_store_var(ctx, pl, p1, s);
        if (rc) return rc;
        tc::Params p2 = tc::base_params(ctx, pc, 1, sigma, offs, Ls, B, L_max, out_a, nullptr, n_nbr);
        p2.order = order;
        p2.act_store = store;
        p2.store_stride = stride;
        p2.par_la = la;
        p2.par_sg = sg;
        p2.cone_tab = static_cast<const tc::LayerGeo *>(ctx->cone_tab);
        return tc::launch_cone_var(ctx, pc, p2, s);
    }
    tc::Params p = tc::base_params(ctx, pl, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr);
    p.order = order;
    return tc::launch_var<tc::VAR_PLAIN>(ctx, pl, p, s);
}

int vmc_tc_debug_timeout(vmc_ctx *ctx, int64_t budget_ns, cudaStream_t s)
{
    tc::wait_timeout_kernel<<<1, 32, 0, s>>>(ctx->status, (long long)budget_ns);
    ctx->launches += 1;
    return vmc_cuda_check(ctx, cudaGetLastError(), "wait_timeout launch");
}

extern "C" int vmc_debug_umma_selftest(const uint16_t *A_dev, const uint16_t *B_dev, float *D_dev, int N, int K,
                                       int shift, int variant, void *stream)
{
    if (!A_dev || !B_dev || !D_dev) return VMC_ERR_ARG;
    if (N < 16 || N > 128 || N % 16 || K < 16 || K > 32 || K % 16 || shift < 0 || shift > 64) return VMC_ERR_ARG;
    if (variant && N > 64) return VMC_ERR_ARG;   // exchanged strides would read past the B buffer
    int dev = 0, maj = 0, mnr = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&mnr, cudaDevAttrComputeCapabilityMinor, dev);
    if (!(maj == 10 && mnr == 3)) return VMC_ERR_UNSUPPORTED;
    const size_t smem = 65536 + 16384;
    cudaError_t e = cudaFuncSetAttribute(tc::umma_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return VMC_ERR_CUDA;
    tc::umma_selftest_kernel<<<1, 128, smem, (cudaStream_t)stream>>>(A_dev, B_dev, D_dev, N, K, shift, variant);
    return cudaGetLastError() == cudaSuccess ? VMC_OK : VMC_ERR_CUDA;
}


extern "C" int vmc_autotune(vmc_ctx *ctx, int L, int64_t probe_B, void *stream)
{
    if (!ctx || L < 4 || L > 32 || (L & 1) || probe_B < 1) return VMC_ERR_ARG;
    if (!vmc_is_tc(ctx->arch.precision)) return vmc_fail(ctx, VMC_ERR_STATE, "autotune applies to tensor-core contexts");
    if (!ctx->params_set) return vmc_fail(ctx, VMC_ERR_STATE, "parameters not set");
    ctx->launches = 0;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cfg_bytes = (size_t)probe_B * L * L, out_bytes = (size_t)probe_B * 8;
    char *buf = nullptr;
    if (cudaMalloc(&buf, cfg_bytes + out_bytes + 256) != cudaSuccess) return vmc_fail(ctx, VMC_ERR_CUDA, "autotune alloc");
    int8_t *cfg = reinterpret_cast<int8_t *>(buf);
    double *out = reinterpret_cast<double *>(buf + ((cfg_bytes + 255) & ~size_t(255)));
    tc::probe_configs_kernel<<<(unsigned)std::min<int64_t>(probe_B, 1024), 32, 0, st>>>(cfg, L, probe_B);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const TileChoice saved = ctx->tiles.count(L) ? ctx->tiles[L] : TileChoice{};
    TileChoice best = saved;
    float best_ms = 1e30f;
    int rc = VMC_OK;
    const int saved_L = ctx->L;
    ctx->L = L;
    // candidates: every slab count and geometry, in the order of the MMA
    // cost model; the best few are timed
    std::vector<std::pair<double, TileChoice>> cands;
    for (int S = 1; S <= 2; ++S) {
        std::vector<tc::Cand> cs;
        tc::geo_cands(ctx->arch.channels, L, tc::buf_bytes(ctx->arch.channels, S, L, ctx->arch.n_layers_cc), S, cs);
        for (const tc::Cand &cd : cs) {
            TileChoice t;
            t.slabs = S;
            t.slab_configs = cd.g.G;
            t.lane_cells = cd.g.P;
            t.ctas_per_sm = 1;
            cands.push_back({cd.score, t});
        }
    }
    std::stable_sort(cands.begin(), cands.end(),
                     [](const std::pair<double, TileChoice> &a, const std::pair<double, TileChoice> &b) {
                         return a.first < b.first;
                     });
    if (cands.size() > 8) cands.resize(8);
    for (size_t ci = 0; ci < cands.size() && rc == VMC_OK; ++ci) {
        const TileChoice t = cands[ci].second;
        ctx->tiles[L] = t;
        tc::Plan pl;
        if (tc::make_plan(ctx, L, L, false, &pl) != VMC_OK || pl.geo[L >> 1].G != t.slab_configs ||
            pl.geo[L >> 1].P != t.lane_cells)
            continue;
        float ms = 0.f, best_rep = 1e30f;
        for (int rep = 0; rep < 3 && rc == VMC_OK; ++rep) {
            cudaEventRecord(e0, st);
            rc = tc::launch_any(ctx, pl, 1, cfg, nullptr, nullptr, probe_B, L, out, nullptr, nullptr, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best_rep = std::min(best_rep, ms);
        }
        if (rc == VMC_OK && best_rep < best_ms) { best_ms = best_rep; best = t; }
    }
    ctx->L = saved_L;
    ctx->tiles[L] = best;
    // the light-cone pass (parent pass + neighbour pass, timed together) for
    // the context's own lattice side
    if (rc == VMC_OK && L == ctx->L && ctx->light_cone && tc::cone_applies_impl(ctx)) {
        std::vector<tc::ConeCand> cc;
        tc::cone_cands(ctx, cc);
        std::stable_sort(cc.begin(), cc.end(),
                         [](const tc::ConeCand &a, const tc::ConeCand &b) { return a.score < b.score; });
        if (cc.size() > 8) cc.resize(8);
        const TileChoice saved_c = ctx->cone_tiles;
        TileChoice best_c = saved_c;
        float best_c_ms = 1e30f;
        for (size_t ci = 0; ci < cc.size() && rc == VMC_OK; ++ci) {
            TileChoice t;
            t.slabs = cc[ci].S;
            t.slab_configs = cc[ci].G;
            t.lane_cells = cc[ci].P;
            t.ctas_per_sm = 1;
            ctx->cone_tiles = t;
            float ms = 0.f, best_rep = 1e30f;
            for (int rep = 0; rep < 3 && rc == VMC_OK; ++rep) {
                cudaEventRecord(e0, st);
                rc = tc_eloc_cone(ctx, cfg, probe_B, out, nullptr, st);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) best_rep = std::min(best_rep, ms);
            }
            if (rc == VMC_OK && best_rep < best_c_ms) { best_c_ms = best_rep; best_c = t; }
        }
        ctx->cone_tiles = best_c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(buf);
    DevStatus z{};
    cudaMemcpy(ctx->status, &z, sizeof z, cudaMemcpyHostToDevice);   // probe runs leave no status behind
    return rc;
}
