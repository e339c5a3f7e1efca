// Tensor-core (tcgen05, BF16/FP16 x BF16/FP16 -> FP32) forward pass, log|psi|
// and local energy: the hot loop of Sec. 3.1 ("sprime_batch") on sm_103a.
//
// Persistent CTAs, one per SM.  Each CTA pulls sampled configurations
// sigma from a global counter; for each it lists the antiparallel J1/J2
// bonds (Sec. 3.1, Fig. 2c) and streams sigma itself followed by every
// exchange neighbour sigma' through the network.  Configurations are packed
// into "slabs": G lattices side by side, each as (L+2) x (L+2) circularly
// padded cells, so a slab is a PH x PW grid with PW = G (L+2), PH = L+2.
//
// A C -> C layer is an implicit GEMM over tiles of 128 padded cells
// (row-major, tile t starting at cell 126 t):
//   P[q][kx C + co] = sum_{ky, ci} A[q + ky PW][ci] W[ky][kx][ci][co]
// (the vertical tap is a start-address offset of the A descriptor, the
// three horizontal taps are stacked along N = 3 C), so a tile takes 3 C/16
// MMAs of 128 x 3C x 16.  The output of cell q is
//   z[q][co] = P[q][co] + P[q+1][C + co] + P[q+2][2C + co],
// which the epilogue forms across TMEM lanes with warp shuffles (the last
// two rows of a tile are overlap rows, hence the stride 126).  Outputs at
// the padding columns are computed and dropped.  The embedding layer
// (c_in = 1) uses a small im2col of the nine spins (K = 16, 7 zero).
//
// Warp roles: warps 0-7 (the "epilogue" group) build neighbours, drain
// TMEM tile by tile (shift-add, bias, SiLU -> 16-bit into the next padded
// buffer with the circular halo copies), pool the last layer and keep the
// per-parent FP64 energy sums; warp 8 allocates TMEM and one lane issues
// every MMA and the per-layer weight bulk copies (a two-deep ring).
// Accumulators live in a ring of TMEM slots (one tile each) with full/empty
// mbarriers, and two slabs alternate, so the epilogue of one tile overlaps
// the MMAs of the next.  Every mbarrier wait is bounded by a time budget; on
// expiry the CTA raises VMC_ERR_TIMEOUT, drains its own copies and MMAs,
// frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <algorithm>
#include <vector>
#include "vmc_internal.h"
#include "lattice.cuh"
#include "tc_layout.cuh"
#include "tc_ptx.cuh"

namespace vmc {
namespace tc {

constexpr int NEPI_WARPS = 8;
constexpr int NEPI = NEPI_WARPS * 32;     // epilogue threads
constexpr int MMA_WARP = NEPI_WARPS;
constexpr int NTHREADS = NEPI + 32;
constexpr int MAX_SLOTS = 16;             // configurations per slab
constexpr int RING = 32;                  // parents in flight per CTA
constexpr int TS = 126;                   // tile stride in cells (128-row tiles overlap by 2)
constexpr int MAX_TSLOTS = 16;            // TMEM accumulator slots
constexpr int SMEM_LIMIT = 232448;

struct Geo { int G, T, PW; };

struct Params {
    int mode;                   // 0 logpsi, 1 local energy
    long long B;
    const int8_t *sigma;
    const int64_t *offs;
    const int32_t *Ls;
    int L_uniform, L_max;
    int D, marshall;
    double J1, J2;
    const uint8_t *wimg;
    const float *bias32;
    int S, Rcap;
    int nslots;                 // TMEM slots of 3 C columns
    Geo geo[17];
    double *out_a;
    int8_t *out_sign;
    int32_t *n_nbr;
    DevStatus *status;
    int *counter;
    long long budget_ns;
};

struct Parent {
    long long b;
    double diag, la0, acc;
    int sg0, remaining, nlist, mpar, valid, L;
};

struct SlabMeta {
    int count, L, G, T, PW;
    uint32_t mPW, mLP;          // floor(2^32 / PW) + 1, floor(2^32 / (L+2)) + 1: r / PW = umulhi(r, mPW)
    int parent[MAX_SLOTS];
    int bond[MAX_SLOTS];
};

struct Ctrl {
    uint64_t act_ready[2], w_full[2], w_empty[2], drain;
    uint64_t t_full[MAX_TSLOTS], t_empty[MAX_TSLOTS];
    uint32_t tmem_base;
    int abort;
    int action, ok;
    int okf[2];                 // abort snapshots, indexed by the parity of the check
    long long new_b;
    int new_L;
    int cur_parent, cur_k, cur_nlist, cur_L;
    long long pending_b;
    int no_more, ring_head;
    int seg_first, seg_n;
    int nb_cnt, nb_a1, nb_a2, nb_par;
    SlabMeta slab[2];
    double slot_la[2][MAX_SLOTS];
    int slot_sg[2][MAX_SLOTS];
    Parent ring[RING];
    float xch[2][2][4][3 * 16]; // [tile parity][channel group][lane quarter][x1(lane0), x2(lane0), x2(lane1)]
};

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(2 + g) : "memory"); }

// two FP32 values -> packed 16-bit pair (low half = a), round to nearest even
template <bool F16>
__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    if constexpr (F16) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&h);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
}

// SiLU(z) = z / (1 + e^-z).  BF16 operands: z/2 (1 + tanh(z/2)) with the
// hardware tanh (one MUFU op; its ~2^-11 error is below BF16 rounding for
// the bulk of activations).  FP16 operands: e = exp(-|z|) (one MUFU op),
// r = 1 / (1 + e) by Newton-Raphson from the linear estimate
// 24/17 - 8/17 d on [1, 2] (relative error 1/17 -> (1/17)^4 after two
// steps), sigmoid = r for z >= 0 and e r otherwise.
template <bool F16>
__device__ __forceinline__ float silu(float z)
{
    if constexpr (F16) {
        const float e = __expf(-fabsf(z));
        const float d = 1.0f + e;
        float r = fmaf(-0.47058823529f, d, 1.41176470588f);
        r = r * fmaf(-d, r, 2.0f);
        r = r * fmaf(-d, r, 2.0f);
        return z * (z >= 0.f ? r : e * r);
    } else {
        const float h = 0.5f * z;
        return fmaf(h, tanh_approx(h), h);
    }
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ void st_shared_v2(uint32_t addr, uint32_t a, uint32_t b)
{
    asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}

__device__ __forceinline__ double nan_d() { return __longlong_as_double(0x7ff8000000000000LL); }

template <int N>
__device__ __forceinline__ void tmem_ld_n(uint32_t taddr, float (&v)[N])
{
    if constexpr (N == 8) tmem_ld8(taddr, v);
    else if constexpr (N == 16) tmem_ld16(taddr, v);
    else {
        static_assert(N == 4, "4, 8 or 16 columns");
        uint32_t r[4];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
            : "r"(taddr)
            : "memory");
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
    }
}

template <int C, bool F16>
struct Kern {
    static constexpr uint32_t WB = 18 * C * C;    // bytes of one C -> C layer image
    static constexpr int CPT = C / 2;             // channels per epilogue thread (2 channel groups)
    static constexpr int NCOL = 3 * C;            // TMEM columns per tile slot

    const Params &p;
    uint8_t *smem;
    Ctrl &c;
    int8_t *spins;
    uint16_t *list;
    uint32_t BUF, PS;
    uint32_t tmem;

    __device__ Kern(const Params &p_, uint8_t *smem_, Ctrl &c_, int8_t *sp, uint16_t *li, uint32_t buf, uint32_t tm)
        : p(p_), smem(smem_), c(c_), spins(sp), list(li), BUF(buf), PS(p_.Rcap * 16u), tmem(tm) {}

    __device__ uint8_t *act_buf(int s, int k) const { return smem + 2 * WB + (size_t)(2 * s + k) * BUF; }

    __device__ bool wait_bar(uint64_t *bar, uint32_t parity, int site)
    {
        return mbar_wait_bounded(bar, parity, &c.abort, p.budget_ns, &p.status->flags, &p.status->timeout_site, site);
    }

    // A0 (embedding im2col) rows per plane for a slab of T tiles
    __device__ static int a0_rows(int T) { return TS * (T - 1) + 128; }

    // ---------------------------------------------------------------- MMA
    __device__ void issue_tile(int s, int l, int t, int bsel, uint32_t dcol)
    {
        const SlabMeta &m = c.slab[s];
        const uint32_t wb = smem_u32(smem + bsel * WB);
        if (l == 0) {
            const uint32_t a0 = smem_u32(act_buf(s, 1));
            const uint64_t ad = smem_desc(a0 + (uint32_t)(t * TS) * 16u, (uint32_t)a0_rows(m.T) * 16u, 128);
            umma_bf16(dcol, ad, smem_desc(wb, 16 * C, 128), idesc_f16kind(128, C, F16), 0);
        } else {
            const uint64_t ad0 = smem_desc(smem_u32(act_buf(s, (l - 1) & 1)), PS, 128);
            const uint64_t bd0 = smem_desc(wb, 16 * NCOL, 128);
            const uint32_t idesc = idesc_f16kind(128, NCOL, F16);
            const uint32_t plane2 = (2u * PS) >> 4;
            const uint32_t rt = (uint32_t)(t * TS);
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int h = 0; h < C / 16; ++h)
                    umma_bf16(dcol, ad0 + (uint64_t)(rt + (uint32_t)(ky * m.PW) + h * plane2),
                              bd0 + (uint64_t)((ky * (C / 16) + h) * 2 * NCOL), idesc, (ky | h) != 0);
        }
    }

    __device__ void mma_role()
    {
        const int D = p.D, R = p.nslots;
        int issued[2] = {0, 0}, waited[2] = {0, 0};
        auto issue_w = [&](long long step) {
            const int bsel = (int)(step & 1);
            const int l = (int)(step % (D + 1));
            const uint32_t bytes = (uint32_t)tc_layer_bytes(C, l);
            mbar_expect_tx(&c.w_full[bsel], bytes);
            bulk_g2s(smem + bsel * WB, p.wimg + tc_wimg_offset(C, l), bytes, &c.w_full[bsel]);
            issued[bsel]++;
        };
        issue_w(0);
        issue_w(1);
        bool dead[2] = {false, p.S < 2};
        int cnt[2] = {0, 0};
        uint32_t ph_ar[2] = {0, 0};
        long long step = 0;           // weight step
        int slot = 0;                 // TMEM slot of the next tile, and the parity of its use
        uint32_t use_par = 0;
        bool ok = true;
        while (ok && !(dead[0] && dead[1])) {
            for (int l = 0; l <= D && ok; ++l) {
                bool any = false;
                for (int s = 0; s < 2 && ok; ++s) {
                    if (dead[s]) continue;
                    if (l == 0 || cnt[s] > 0) {
                        if (!wait_bar(&c.act_ready[s], ph_ar[s], 1)) { ok = false; break; }
                        ph_ar[s] ^= 1;
                    }
                    if (l == 0) {
                        cnt[s] = *(volatile int *)&c.slab[s].count;
                        if (cnt[s] == 0) { dead[s] = true; continue; }
                    }
                    if (!any) {
                        const int bsel = (int)(step & 1);
                        if (!wait_bar(&c.w_full[bsel], (uint32_t)((step >> 1) & 1), 2)) { ok = false; break; }
                        waited[bsel]++;
                        any = true;
                    }
                    const int T = *(volatile int *)&c.slab[s].T;
                    for (int t = 0; t < T; ++t) {
                        if (!wait_bar(&c.t_empty[slot], use_par ^ 1u, 3)) { ok = false; break; }
                        tc_fence_after();
                        issue_tile(s, l, t, (int)(step & 1), tmem + (uint32_t)(slot * NCOL));
                        umma_commit(&c.t_full[slot]);
                        if (++slot == R) { slot = 0; use_par ^= 1u; }
                    }
                }
                if (!ok || !any) break;
                umma_commit(&c.w_empty[step & 1]);
                if (step >= 1) {
                    if (!wait_bar(&c.w_empty[(step - 1) & 1], (uint32_t)(((step - 1) >> 1) & 1), 4)) { ok = false; break; }
                    issue_w(step + 1);
                }
                ++step;
            }
        }
        // drain: every weight copy issued and every MMA issued must finish
        const long long cb = p.budget_ns > 1000000000LL ? p.budget_ns : 1000000000LL;
        int dummy_abort = 0;
        for (int bsel = 0; bsel < 2; ++bsel)
            while (waited[bsel] < issued[bsel]) {
                if (!mbar_wait_bounded(&c.w_full[bsel], (uint32_t)(waited[bsel] & 1), &dummy_abort, cb,
                                       &p.status->flags, &p.status->timeout_site, 5))
                    break;
                waited[bsel]++;
            }
        umma_commit(&c.drain);
        mbar_wait_bounded(&c.drain, 0, &dummy_abort, cb, &p.status->flags, &p.status->timeout_site, 6);
    }

    // ---------------------------------------------------------------- epilogue helpers
    // (y, j, x) of padded cell r; j = configuration slot, x column in it
    // (exact for r < 2^16 and divisors < 2^10: umulhi(r, floor(2^32/d) + 1) = floor(r/d))
    __device__ __forceinline__ void cell_coords(int r, const SlabMeta &m, int &y, int &j, int &x) const
    {
        y = (int)__umulhi((uint32_t)r, m.mPW);
        const int X = r - y * m.PW;
        j = (int)__umulhi((uint32_t)X, m.mLP);
        x = X - j * (m.L + 2);
    }

    // Per-(slab, layer) constants of the epilogue threads.
    struct TileCtx {
        int L, PW, count;
        uint32_t mPW, mLP;
        uint32_t out;           // output buffer (shared address)
        float bias[CPT];
    };

    __device__ __forceinline__ void load_tctx(int s, int l, int tid, TileCtx &k) const
    {
        const SlabMeta &m = c.slab[s];
        k.L = m.L; k.PW = m.PW; k.count = m.count; k.mPW = m.mPW; k.mLP = m.mLP;
        k.out = smem_u32(act_buf(s, l & 1));
        const int g = (tid >> 5) >> 2;
        const float *bias = p.bias32 + l * C + g * CPT;
#pragma unroll
        for (int i = 0; i < CPT; ++i) k.bias[i] = __ldg(bias + i);
    }

    // Drain one tile: load the thread's CPT channels of P[q][kx C + co] for
    // kx = 0 (and 1, 2 for C -> C layers) under one wait, release the TMEM
    // slot, and form z[q] = P0[q] + P1[q+1] + P2[q+2] + bias across lanes.
    __device__ __forceinline__ void drain_tile(int l, int t, int slot, int tid, const TileCtx &k, float (&z)[CPT], bool ok)
    {
        const int warp = tid >> 5, lane = tid & 31, g = warp >> 2, wq = warp & 3;
        const uint32_t taddr = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(slot * NCOL + g * CPT);
        float x1[CPT], x2[CPT];
        if (!ok) {
#pragma unroll
            for (int i = 0; i < CPT; ++i) { z[i] = 0.f; x1[i] = 0.f; x2[i] = 0.f; }
        } else if (l > 0) {
            if constexpr (CPT == 16) tmem_ld16x3(taddr, C, z, x1, x2);
            else tmem_ld8x3(taddr, C, z, x1, x2);
        } else {
            tmem_ld_n<CPT>(taddr, z);
        }
        tc_fence_before();
        __syncwarp();
        if (ok && lane == 0) mbar_arrive(&c.t_empty[slot]);
        if (l == 0) {
#pragma unroll
            for (int i = 0; i < CPT; ++i) z[i] += k.bias[i];
            return;
        }
        // rows q+1, q+2 that live in the next lane quarter, through shared memory
        float *xo = c.xch[t & 1][g][wq];
        if (wq > 0 && lane < 2) {
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < CPT; ++i) { xo[i] = x1[i]; xo[CPT + i] = x2[i]; }
            } else {
#pragma unroll
                for (int i = 0; i < CPT; ++i) xo[2 * CPT + i] = x2[i];
            }
        }
        group_sync(g);
        // lanes 30 and 31 take rows q+1 / q+2 from the next quarter; every lane
        // then adds in the same order, so the arithmetic of a cell does not
        // depend on where it sits in the tile
        float a1[CPT], a2[CPT];
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            a1[i] = __shfl_down_sync(0xffffffffu, x1[i], 1);
            a2[i] = __shfl_down_sync(0xffffffffu, x2[i], 2);
        }
        if (lane >= 30) {
            const float *xn = c.xch[t & 1][g][(wq + 1) & 3];
            const bool l31 = (lane == 31);
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                if (l31) a1[i] = xn[i];
                a2[i] = l31 ? xn[2 * CPT + i] : xn[CPT + i];
            }
        }
#pragma unroll
        for (int i = 0; i < CPT; ++i) z[i] = ((z[i] + k.bias[i]) + a1[i]) + a2[i];
    }

    // epilogue of one tile of a hidden layer: SiLU, 16-bit, stores
    __device__ __forceinline__ void store_tile(int l, int t, int slot, int tid, const TileCtx &k, bool ok)
    {
        const int warp = tid >> 5, lane = tid & 31, g = warp >> 2, wq = warp & 3;
        float z[CPT];
        drain_tile(l, t, slot, tid, k, z, ok);
        if (!ok) return;
        const int i_row = wq * 32 + lane;
        const int r = t * TS + i_row;
        const int y = (int)__umulhi((uint32_t)r, k.mPW);
        const int X = r - y * k.PW;
        const int j = (int)__umulhi((uint32_t)X, k.mLP);
        const int x = X - j * (k.L + 2);
        const int L = k.L;
        if (i_row < TS && y < L && x < L && j < k.count) {
            uint32_t w[CPT / 2];
#pragma unroll
            for (int i = 0; i < CPT / 2; ++i) w[i] = pack2<F16>(silu<F16>(z[2 * i]), silu<F16>(z[2 * i + 1]));
            const int R0 = (y + 1) * k.PW + j * (L + 2) + x + 1;
            const int hx = (x == 0) ? L : ((x == L - 1) ? -L : 0);
            const int vy = (y == 0) ? L * k.PW : ((y == L - 1) ? -L * k.PW : 0);
            // channel group g: C = 32 -> planes 2g, 2g + 1; C = 16 -> plane g
            auto put = [&](int row) {
                const uint32_t a = k.out + (uint32_t)row * 16u;
                if constexpr (CPT == 16) {
                    st_shared_v4(a + (2 * g) * PS, w[0], w[1], w[2], w[3]);
                    st_shared_v4(a + (2 * g + 1) * PS, w[4], w[5], w[6], w[7]);
                } else {
                    st_shared_v4(a + g * PS, w[0], w[1], w[2], w[3]);
                }
            };
            put(R0);
            if (hx) put(R0 + hx);
            if (vy) {
                put(R0 + vy);
                if (hx) put(R0 + vy + hx);
            }
        }
    }

    // epilogue of one tile of the last layer: pooling partials
    __device__ __forceinline__ void pool_tile(int t, int slot, int tid, const TileCtx &k, float *partF, int *partI,
                                              int rows, bool ok)
    {
        const int warp = tid >> 5, lane = tid & 31, g = warp >> 2, wq = warp & 3;
        float z[CPT];
        drain_tile(p.D, t, slot, tid, k, z, ok);
        if (!ok) return;
        const int i_row = wq * 32 + lane;
        const int r = t * TS + i_row;
        const int y = (int)__umulhi((uint32_t)r, k.mPW);
        const int X = r - y * k.PW;
        const int j = (int)__umulhi((uint32_t)X, k.mLP);
        const int x = X - j * (k.L + 2);
        if (i_row < TS && y < k.L && x < k.L && j < k.count) {
            float sl = 0.f;
            int neg = 0, zer = 0;
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                sl += __log2f(fabsf(z[i]));
                neg += (z[i] < 0.f);
                zer += (z[i] == 0.f);
            }
            partF[g * rows + r] = sl;
            partI[g * rows + r] = neg | (zer << 16);
        }
    }

    // per-configuration FP64 sums and the per-parent bookkeeping
    __device__ void pool_finish(int s, int tid, const float *partF, const int *partI, int rows)
    {
        SlabMeta &m = c.slab[s];
        const int warp = tid >> 5, lane = tid & 31;
        const int L = m.L, count = m.count, npix = L * L;
        for (int j = warp; j < count; j += NEPI_WARPS) {
            double acc = 0.0;
            int neg = 0, zer = 0;
            for (int idx = lane; idx < 2 * npix; idx += 32) {
                const int gg = idx / npix, pix = idx - gg * npix;
                const int y = pix / L, x = pix - y * L;
                const int r = y * m.PW + j * (L + 2) + x;
                acc += (double)partF[gg * rows + r];
                const int nz = partI[gg * rows + r];
                neg += nz & 0xffff;
                zer += nz >> 16;
            }
            for (int o = 16; o > 0; o >>= 1) {
                acc += __shfl_xor_sync(0xffffffffu, acc, o);
                neg += __shfl_xor_sync(0xffffffffu, neg, o);
                zer += __shfl_xor_sync(0xffffffffu, zer, o);
            }
            if (lane == 0) {
                c.slot_la[s][j] = zer ? -INFINITY : acc * 0.69314718055994530942;
                c.slot_sg[s][j] = zer ? 0 : ((neg & 1) ? -1 : 1);
            }
        }
        epi_sync();
        if (tid == 0) {
            for (int j = 0; j < count; ++j) {
                Parent &P = c.ring[m.parent[j]];
                const double la = c.slot_la[s][j];
                const int sg = c.slot_sg[s][j];
                if (m.bond[j] < 0) {
                    P.la0 = la;
                    P.sg0 = sg;
                } else {
                    const double rho = (double)(sg * P.sg0) * exp(la - P.la0);
                    P.acc += exchange_coef(m.bond[j] & 3, p.J1, p.J2, p.marshall) * rho;
                }
                if (--P.remaining == 0) {
                    finish_parent(P);
                    P.valid = 0;
                }
            }
        }
        epi_sync();
    }

    __device__ void finish_parent(const Parent &P)
    {
        const long long b = P.b;
        if (p.mode == 0) {
            int sg = P.sg0;
            if (p.marshall && P.mpar) sg = -sg;
            p.out_a[b] = P.la0;
            p.out_sign[b] = (int8_t)sg;
            if (P.la0 != P.la0 || P.la0 == INFINITY) {
                atomicOr(&p.status->flags, VMC_STATUS_NONFINITE);
                atomicAdd(&p.status->nonfinite, 1ull);
            }
        } else {
            double e = P.diag + P.acc;
            if (P.sg0 == 0 || !isfinite(P.la0) || !isfinite(e)) {
                e = nan_d();
                atomicOr(&p.status->flags, VMC_STATUS_NONFINITE);
                atomicAdd(&p.status->nonfinite, 1ull);
            }
            p.out_a[b] = e;
            if (p.n_nbr) p.n_nbr[b] = P.nlist;
        }
    }

    // Build the embedding-layer im2col rows of slots [first, first+n):
    // nine spins of sigma' around each cell, 16 values per row in two planes.
    __device__ void build_rows(int s, int first, int n, int tid)
    {
        const SlabMeta &m = c.slab[s];
        const int L = m.L, PW = m.PW, npix = L * L;
        const uint32_t a0 = smem_u32(act_buf(s, 1));
        const uint32_t plane = (uint32_t)a0_rows(m.T) * 16u;
        const uint32_t up = F16 ? 0x3C00u : 0x3F80u, dn = F16 ? 0xBC00u : 0xBF80u;
        for (int idx = tid; idx < n * npix; idx += NEPI) {
            const int jj = first + idx / npix, pix = idx - (idx / npix) * npix;
            const int y = pix / L, x = pix - y * L;
            const int bond = m.bond[jj];
            int bi = -1, bj = -1;
            if (bond >= 0) { bi = bond >> 2; bj = bond_partner(L, bi, bond & 3); }
            uint32_t h[9];
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                int sy = y + ky - 1;
                sy = sy < 0 ? sy + L : (sy >= L ? sy - L : sy);
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    int sx = x + kx - 1;
                    sx = sx < 0 ? sx + L : (sx >= L ? sx - L : sx);
                    const int site = sy * L + sx;
                    int v = spins[site];
                    if (site == bi) v = spins[bj];
                    else if (site == bj) v = spins[bi];
                    h[ky * 3 + kx] = v > 0 ? up : dn;
                }
            }
            const uint32_t q = (uint32_t)(y * PW + jj * (L + 2) + x) * 16u;
            st_shared_v4(a0 + q, h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
            st_shared_v4(a0 + plane + q, h[8], 0u, 0u, 0u);
        }
    }

    // Fill slab s with the next configurations of the stream; returns count.
    __device__ int fill(int s, int tid)
    {
        SlabMeta &m = c.slab[s];
        if (tid == 0) { m.count = 0; m.L = 0; }
        epi_sync();
        for (;;) {
            if (tid == 0) {
                int act = 2;
                if (c.abort) {
                    act = 2;   // stop filling; the caller's next abort check ends the epilogue
                } else if (c.cur_parent >= 0 && c.cur_k <= c.cur_nlist) {
                    act = 0;
                } else {
                    while (!c.no_more) {
                        long long b = c.pending_b >= 0 ? c.pending_b : (long long)atomicAdd(p.counter, 1);
                        c.pending_b = -1;
                        if (b >= p.B) { c.no_more = 1; break; }
                        const int Lb = p.Ls ? p.Ls[b] : p.L_uniform;
                        if ((Lb & 1) || Lb < 4 || Lb > p.L_max || p.geo[Lb >> 1].G == 0) {
                            p.out_a[b] = nan_d();
                            if (p.mode == 0) p.out_sign[b] = 0;
                            if (p.n_nbr) p.n_nbr[b] = 0;
                            atomicOr(&p.status->flags, VMC_STATUS_BADARG);
                            continue;
                        }
                        if (m.count > 0 && Lb != m.L) { c.pending_b = b; break; }
                        c.new_b = b;
                        c.new_L = Lb;
                        act = 1;
                        break;
                    }
                }
                c.action = act;
            }
            epi_sync();
            const int act = c.action;
            if (act == 2) break;
            if (act == 1) {
                const int Lb = c.new_L;
                const long long b = c.new_b;
                const int8_t *sig = p.sigma + (p.offs ? p.offs[b] : b * (long long)Lb * Lb);
                for (int i = tid; i < Lb * Lb; i += NEPI) spins[i] = sig[i];
                epi_sync();
                if (tid < 32) {
                    int a1 = 0, a2 = 0, cnt = 0, par = 0;
                    if (p.mode == 1) cnt = build_bond_list_warp(spins, Lb, list, &a1, &a2);
                    else par = marshall_parity_warp(spins, Lb);
                    if (tid == 0) { c.nb_cnt = cnt; c.nb_a1 = a1; c.nb_a2 = a2; c.nb_par = par; }
                }
                epi_sync();
                if (tid == 0) {
                    const int r = c.ring_head;
                    c.ring_head = (r + 1) % RING;
                    Parent &P = c.ring[r];
                    if (P.valid) { c.abort = 1; atomicOr(&p.status->flags, VMC_STATUS_INTERNAL); }
                    P.b = b;
                    P.diag = (p.mode == 1) ? diag_energy(Lb, c.nb_a1, c.nb_a2, p.J1, p.J2) : 0.0;
                    P.la0 = 0.0; P.acc = 0.0; P.sg0 = 0;
                    P.nlist = c.nb_cnt;
                    P.remaining = 1 + c.nb_cnt;
                    P.mpar = c.nb_par;
                    P.valid = 1;
                    P.L = Lb;
                    c.cur_parent = r;
                    c.cur_k = 0;
                    c.cur_nlist = c.nb_cnt;
                    c.cur_L = Lb;
                }
                epi_sync();
            }
            if (tid == 0) {
                if (m.count == 0) {
                    // the slab takes the geometry of the lattice now at the cursor
                    // (a new parent, or the rest of the previous fill's parent)
                    const int Lc = c.cur_L;
                    m.L = Lc;
                    m.G = p.geo[Lc >> 1].G;
                    m.T = p.geo[Lc >> 1].T;
                    m.PW = p.geo[Lc >> 1].PW;
                    m.mPW = (uint32_t)(0xFFFFFFFFu / (uint32_t)m.PW) + 1u;
                    m.mLP = (uint32_t)(0xFFFFFFFFu / (uint32_t)(Lc + 2)) + 1u;
                }
                if (m.G < 1 || m.G > MAX_SLOTS) { c.abort = 1; atomicOr(&p.status->flags, VMC_STATUS_INTERNAL); m.G = 1; }
                const int n_take = min(m.G - m.count, c.cur_nlist + 1 - c.cur_k);
                for (int i = 0; i < n_take; ++i) {
                    const int kk = c.cur_k + i;
                    m.parent[m.count + i] = c.cur_parent;
                    m.bond[m.count + i] = (kk == 0) ? -1 : (int)list[kk - 1];
                }
                c.seg_first = m.count;
                c.seg_n = n_take;
                m.count += n_take;
                c.cur_k += n_take;
            }
            epi_sync();
            build_rows(s, c.seg_first, c.seg_n, tid);
            epi_sync();
            if (m.count >= m.G) break;
        }
        const int count = m.count;
        if (count > 0) {
            // rows that belong to no configuration: zero (finite) input
            const int L = m.L, rows = a0_rows(m.T);
            const uint32_t a0 = smem_u32(act_buf(s, 1));
            const uint32_t plane = (uint32_t)rows * 16u;
            for (int r = tid; r < rows; r += NEPI) {
                int y, j, x;
                cell_coords(r, m, y, j, x);
                if (!(y < L && x < L && j < count)) {
                    st_shared_v4(a0 + r * 16u, 0u, 0u, 0u, 0u);
                    st_shared_v4(a0 + plane + r * 16u, 0u, 0u, 0u, 0u);
                }
            }
        }
        return count;
    }

    __device__ void signal_ready(int s, int tid)
    {
        fence_proxy_async_smem();
        epi_sync();
        if (tid == 0) mbar_arrive(&c.act_ready[s]);
    }

    // Each warp waits (one lane, bounded) for the accumulator slot of the
    // next tile.  A warp whose wait fails keeps going through the tile loop
    // without touching TMEM, so every named barrier still sees all
    // participants; the whole epilogue returns together at the next CTA-wide
    // check of c.abort.
    __device__ __forceinline__ bool wait_tile(int slot, uint32_t par, int tid)
    {
        int ok = 0;
        if ((tid & 31) == 0) ok = wait_bar(&c.t_full[slot], par, 7) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok) tc_fence_after();
        return ok != 0;
    }

    __device__ void epilogue_role(int tid)
    {
        const int D = p.D, R = p.nslots;
        bool dead[2] = {false, true};
        int slot = 0;
        uint32_t use_par = 0;
        int nchk = 0;
        // CTA-wide abort check: tid 0 snapshots c.abort into okf[parity]; the
        // next write to the same slot comes two barriers later, after every
        // thread has read this one
        auto go_on = [&]() {
            const int kk = (nchk++) & 1;
            if (tid == 0) c.okf[kk] = c.abort ? 0 : 1;
            epi_sync();
            return c.okf[kk] != 0;
        };
        auto next_slot = [&]() { if (++slot == R) { slot = 0; use_par ^= 1u; } };
        for (int s = 0; s < p.S; ++s) {
            const int cnt = fill(s, tid);
            signal_ready(s, tid);
            dead[s] = (cnt == 0);
        }
        while (!(dead[0] && dead[1])) {
            for (int l = 0; l <= D; ++l) {
                for (int s = 0; s < 2; ++s) {
                    if (dead[s]) continue;
                    const int T = c.slab[s].T;
                    TileCtx k;
                    load_tctx(s, l, tid, k);
                    if (l < D) {
                        for (int t = 0; t < T; ++t) {
                            store_tile(l, t, slot, tid, k, wait_tile(slot, use_par, tid));
                            next_slot();
                        }
                        if (!go_on()) return;
                        signal_ready(s, tid);
                    } else {
                        const int rows = TS * T;
                        // pooling partials go to the buffer layer D - 1 read (its MMAs are
                        // done); the layer-D input buffer is still read by later tiles
                        float *partF = reinterpret_cast<float *>(act_buf(s, p.D & 1));
                        int *partI = reinterpret_cast<int *>(partF + 2 * rows);
                        for (int t = 0; t < T; ++t) {
                            pool_tile(t, slot, tid, k, partF, partI, rows, wait_tile(slot, use_par, tid));
                            next_slot();
                        }
                        if (!go_on()) return;
                        pool_finish(s, tid, partF, partI, rows);
                        const int cnt = fill(s, tid);
                        signal_ready(s, tid);
                        dead[s] = (cnt == 0);
                    }
                }
            }
        }
    }
};

template <int C, bool F16>
__global__ void __launch_bounds__(NTHREADS, 1) tc_eloc_kernel(const __grid_constant__ Params p)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t BUF = (uint32_t)(C / 8) * p.Rcap * 16u;
    Ctrl &c = *reinterpret_cast<Ctrl *>(smem + 2 * Kern<C, F16>::WB + (size_t)2 * p.S * BUF);
    int8_t *spins = reinterpret_cast<int8_t *>(&c + 1);
    uint16_t *list = reinterpret_cast<uint16_t *>(spins + ((p.L_max * p.L_max + 15) & ~15));
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&c.act_ready[i], 1);
            mbar_init(&c.w_full[i], 1);
            mbar_init(&c.w_empty[i], 1);
        }
        for (int i = 0; i < MAX_TSLOTS; ++i) {
            mbar_init(&c.t_full[i], 1);
            mbar_init(&c.t_empty[i], NEPI_WARPS);   // one arrival per epilogue warp
        }
        mbar_init(&c.drain, 1);
        c.abort = 0;
        c.cur_parent = -1; c.cur_k = 0; c.cur_nlist = -1; c.cur_L = 0;
        for (int i = 0; i < 2; ++i) { c.slab[i].count = 0; c.slab[i].L = 0; c.slab[i].G = 0; c.slab[i].T = 0; c.slab[i].PW = 0; }
        c.pending_b = -1; c.no_more = 0; c.ring_head = 0;
        for (int r = 0; r < RING; ++r) c.ring[r].valid = 0;
        mbar_fence_init();
        fence_proxy_async_smem();
    }
    if (warp == MMA_WARP) tmem_alloc(&c.tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    Kern<C, F16> k(p, smem, c, spins, list, BUF, c.tmem_base);
    if (warp < MMA_WARP) k.epilogue_role(tid);
    else if ((tid & 31) == 0) k.mma_role();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == MMA_WARP) {
        __syncwarp();
        tmem_dealloc(c.tmem_base, 512);
    }
}

// ------------------------------------------------------------------ planning

static size_t ctrl_bytes(int L_max)
{
    return sizeof(Ctrl) + ((L_max * L_max + 15) & ~15) + (size_t)4 * L_max * L_max * 2 + 64;
}

// tiles and shared-memory rows (per plane) of a slab of G lattices of side L
static int rows_needed(int L, int G, int *T_out)
{
    const int PW = G * (L + 2);
    const int T = (L * PW + TS - 1) / TS;
    *T_out = T;
    const int mma_rows = TS * (T - 1) + 128 + 2 * PW;   // last A row any MMA of the slab reads, + 1
    return (std::max((L + 2) * PW, mma_rows) + 7) & ~7;
}

struct Plan {
    int S, Rcap;
    Geo geo[17];
    size_t smem;
};

// Largest-efficiency G for lattice L under the row capacity.
static Geo best_geo(int L, int Rcap, int Gwant)
{
    Geo best{0, 0, 0};
    double be = -1.0;
    for (int G = 1; G <= MAX_SLOTS; ++G) {
        int T;
        const int R = rows_needed(L, G, &T);
        if (R > Rcap) break;
        const double eff = (double)L * L * G / (double)(TS * T);
        if (Gwant > 0) {
            if (G == Gwant) { best = Geo{G, T, G * (L + 2)}; be = eff; }
            continue;
        }
        if (eff > be + 1e-9) { be = eff; best = Geo{G, T, G * (L + 2)}; }
    }
    return best;
}

static int make_plan(const vmc_ctx *ctx, int L_main, int L_max, bool ragged, Plan *pl)
{
    const int C = ctx->arch.channels;
    TileChoice tc;
    auto it = ctx->tiles.find(L_main);
    if (it != ctx->tiles.end()) tc = it->second;
    const int S = tc.slabs ? tc.slabs : 2;
    const size_t wb = 2 * (size_t)(18 * C * C);
    const size_t ctrl = ctrl_bytes(L_max);
    const size_t avail = SMEM_LIMIT - wb - ctrl - 1024;
    int Rcap = (int)(avail / ((size_t)2 * S * (C / 8) * 16)) & ~7;
    Geo gmain = best_geo(L_main, Rcap, tc.slab_configs);
    if (gmain.G == 0) return VMC_ERR_UNSUPPORTED;
    if (!ragged) {
        int T;
        Rcap = rows_needed(L_main, gmain.G, &T);
    }
    pl->S = S;
    pl->Rcap = Rcap;
    for (int i = 0; i < 17; ++i) pl->geo[i] = Geo{0, 0, 0};
    if (ragged) {
        for (int L = 4; L <= L_max; L += 2) {
            TileChoice tl;
            auto jt = ctx->tiles.find(L);
            if (jt != ctx->tiles.end()) tl = jt->second;
            pl->geo[L >> 1] = best_geo(L, Rcap, tl.slab_configs);
        }
    } else {
        pl->geo[L_main >> 1] = gmain;
    }
    pl->smem = wb + (size_t)2 * S * (C / 8) * Rcap * 16 + ctrl;
    if (pl->smem < 120 * 1024) pl->smem = 120 * 1024;   // keeps one CTA (and one TMEM owner) per SM
    if (pl->smem > SMEM_LIMIT) return VMC_ERR_UNSUPPORTED;
    return VMC_OK;
}

template <int C, bool F16>
static int launch(vmc_ctx *ctx, const Plan &pl, int mode, const int8_t *sigma, const int64_t *offs,
                  const int32_t *Ls, int64_t B, int L_max, double *out_a, void *out_b, int32_t *n_nbr,
                  cudaStream_t st)
{
    Params p;
    p.mode = mode; p.B = B; p.sigma = sigma; p.offs = offs; p.Ls = Ls;
    p.L_uniform = ctx->L; p.L_max = L_max;
    p.D = ctx->arch.n_layers_cc; p.marshall = ctx->arch.marshall_sign;
    p.J1 = ctx->J1; p.J2 = ctx->J2;
    p.wimg = reinterpret_cast<const uint8_t *>(ctx->wimg);
    p.bias32 = ctx->bias32;
    p.S = pl.S; p.Rcap = pl.Rcap;
    p.nslots = std::min(MAX_TSLOTS, 512 / (3 * C));
    for (int i = 0; i < 17; ++i) p.geo[i] = pl.geo[i];
    p.out_a = out_a; p.out_sign = static_cast<int8_t *>(out_b); p.n_nbr = n_nbr;
    p.status = ctx->status; p.counter = ctx->counter;
    p.budget_ns = ctx->wait_budget_ns;
    auto kfn = tc_eloc_kernel<C, F16>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "cudaFuncSetAttribute(tc_eloc)");
    e = cudaMemsetAsync(ctx->counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "counter reset");
    int grid = ctx->sm_count;
    if ((int64_t)grid > B) grid = (int)B;
    kfn<<<grid, NTHREADS, pl.smem, st>>>(p);
    ctx->launches += 1;
    return vmc_cuda_check(ctx, cudaGetLastError(), "tc_eloc launch");
}

static int launch_any(vmc_ctx *ctx, const Plan &pl, int mode, const int8_t *sigma, const int64_t *offs,
                      const int32_t *Ls, int64_t B, int L_max, double *out_a, void *out_b, int32_t *n_nbr,
                      cudaStream_t st)
{
    const bool f16 = ctx->arch.precision == VMC_FP16;
    if (ctx->arch.channels == 32)
        return f16 ? launch<32, true>(ctx, pl, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr, st)
                   : launch<32, false>(ctx, pl, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr, st);
    return f16 ? launch<16, true>(ctx, pl, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr, st)
               : launch<16, false>(ctx, pl, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr, st);
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
    int abort_flag = 0, fl = 0, site = 0;
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
    return VMC_OK;
}

int vmc_tc_eloc(vmc_ctx *ctx, int mode, const int8_t *sigma, const int64_t *offs, const int32_t *Ls,
                int64_t B, int L_max, double *out_a, void *out_b, int32_t *n_nbr, cudaStream_t s)
{
    tc::Plan pl;
    const bool ragged = (Ls != nullptr);
    int rc = tc::make_plan(ctx, ragged ? L_max : ctx->L, L_max, ragged, &pl);
    if (rc) return vmc_fail(ctx, rc, "no tensor-core plan for L=%d C=%d", L_max, ctx->arch.channels);
    return tc::launch_any(ctx, pl, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr, s);
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
    for (int S = 1; S <= 2 && rc == VMC_OK; ++S)
        for (int G = 1; G <= tc::MAX_SLOTS && rc == VMC_OK; ++G) {
            TileChoice t;
            t.slabs = S;
            t.slab_configs = G;
            t.ctas_per_sm = 1;
            ctx->tiles[L] = t;
            tc::Plan pl;
            if (tc::make_plan(ctx, L, L, false, &pl) != VMC_OK || pl.geo[L >> 1].G != G) continue;
            float ms = 0.f;
            for (int rep = 0; rep < 3 && rc == VMC_OK; ++rep) {
                cudaEventRecord(e0, st);
                rc = tc::launch_any(ctx, pl, 1, cfg, nullptr, nullptr, probe_B, L, out, nullptr, nullptr, st);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
            }
            if (rc == VMC_OK && ms < best_ms) { best_ms = ms; best = t; }
        }
    ctx->L = saved_L;
    ctx->tiles[L] = best;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(buf);
    DevStatus z{};
    cudaMemcpy(ctx->status, &z, sizeof z, cudaMemcpyHostToDevice);   // probe runs leave no status behind
    return rc;
}
