// Tensor-core (tcgen05, BF16 x BF16 -> FP32) forward pass, log|psi| and
// local energy: the hot loop of Sec. 3.1 ("sprime_batch") on sm_103a.
//
// Persistent CTAs, one per SM.  Each CTA pulls sampled configurations
// sigma from a global counter; for each it lists the antiparallel J1/J2
// bonds (Sec. 3.1, Fig. 2c) and streams sigma itself followed by every
// exchange neighbour sigma' through the network.  Configurations are packed
// into "slabs": G lattices side by side, each as (L+2) x (L+2) circularly
// padded cells, so a slab is a PH x PW grid with PW = G (L+2), PH = L+2.
//
// A C -> C layer is an implicit GEMM per 128-row tile of the slab:
// D[q][co] = sum_{tap, ci} A[q + ky PW + kx][ci] * W[tap][ci][co], where
// q indexes padded cells row-major (outputs at junk columns are computed
// and dropped).  The tap shift is a start-address offset of the A
// descriptor (tc_layout.cuh), so no im2col copy exists; K = 9 C in chunks
// of 16, N = C, FP32 accumulators in TMEM.  The embedding layer (c_in = 1)
// uses a small im2col of the nine spins (K = 16, 7 zero).
//
// Warp roles: warps 0-7 (the "epilogue" group) build neighbours, drain TMEM
// (bias + SiLU -> BF16 into the next padded buffer, including the circular
// halo copies), pool the last layer and keep the per-parent FP64 energy
// sums; warp 8 allocates TMEM and one lane issues every MMA and the
// per-layer weight bulk copies (a two-deep ring).  Two slabs alternate so
// the epilogue of one overlaps the MMAs of the other.  Every mbarrier wait
// is bounded by a time budget; on expiry the CTA raises VMC_ERR_TIMEOUT,
// drains its own copies and MMAs, frees TMEM and returns.
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

constexpr int NEPI = 256;       // epilogue threads (8 warps)
constexpr int NTHREADS = 288;   // + MMA warp
constexpr int MAX_SLOTS = 16;   // configurations per slab
constexpr int RING = 32;        // parents in flight per CTA
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
    int S, Rcap, Tcap;
    uint32_t tmem_cols;
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
    int parent[MAX_SLOTS];
    int bond[MAX_SLOTS];
};

struct Ctrl {
    uint64_t acc_full[2], act_ready[2], w_full[2], w_empty[2], drain;
    uint32_t tmem_base;
    int abort;
    int action, ok;
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
};

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

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

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ double nan_d() { return __longlong_as_double(0x7ff8000000000000LL); }

template <int C, bool F16>
struct Kern {
    static constexpr uint32_t WB = 9 * (C / 16) * 32 * C;   // bytes of one C -> C layer image
    static constexpr int HALF = C / 2;                       // columns per epilogue thread

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

    // ---------------------------------------------------------------- MMA
    __device__ void issue_slab_layer(int s, int l, int bsel)
    {
        const SlabMeta &m = c.slab[s];
        const int T = m.T, PW = m.PW;
        const uint32_t idesc = idesc_f16kind(128, C, F16);
        const uint32_t wb = smem_u32(smem + bsel * WB);
        const uint32_t dcol0 = tmem + (uint32_t)(s * p.Tcap * C);
        if (l == 0) {
            const uint32_t a0 = smem_u32(act_buf(s, 1));
            const uint64_t ad0 = smem_desc(a0, 128u * T * 16u, 128);
            const uint64_t bdesc = smem_desc(wb, 16 * C, 128);
            for (int t = 0; t < T; ++t)
                umma_bf16(dcol0 + t * C, ad0 + (uint64_t)(t * 128), bdesc, idesc, 0);
        } else {
            // descriptors differ from the base only in the start-address
            // field (16-byte units), so each MMA needs two integer adds
            const uint64_t ad0 = smem_desc(smem_u32(act_buf(s, (l - 1) & 1)), PS, 128);
            const uint64_t bd0 = smem_desc(wb, 16 * C, 128);
            const uint32_t plane2 = (2u * PS) >> 4;
            for (int t = 0; t < T; ++t) {
                const uint32_t d = dcol0 + t * C;
                const uint32_t rt = (uint32_t)(t * 128);
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int ky = tap / 3, kx = tap - 3 * ky;
                    const uint32_t roff = rt + (uint32_t)(ky * PW + kx);
#pragma unroll
                    for (int h = 0; h < C / 16; ++h)
                        umma_bf16(d, ad0 + (uint64_t)(roff + h * plane2),
                                  bd0 + (uint64_t)((tap * (C / 16) + h) * 2 * C), idesc, (tap | h) != 0);
                }
            }
        }
    }

    __device__ void mma_role()
    {
        const int D = p.D;
        int issued[2] = {0, 0}, waited[2] = {0, 0};
        auto issue_w = [&](long long step) {
            const int bsel = (int)(step & 1);
            const int l = (int)(step % (D + 1));
            const uint32_t bytes = (l == 0) ? 32u * C : WB;
            mbar_expect_tx(&c.w_full[bsel], bytes);
            bulk_g2s(smem + bsel * WB, p.wimg + tc_wimg_offset(C, l), bytes, &c.w_full[bsel]);
            issued[bsel]++;
        };
        issue_w(0);
        issue_w(1);
        bool dead[2] = {false, p.S < 2};
        int cnt[2] = {0, 0};
        uint32_t ph_ar[2] = {0, 0};
        long long step = 0;
        bool ok = true;
        while (ok && !(dead[0] && dead[1])) {
            for (int l = 0; l <= D; ++l) {
                bool any = false;
                for (int s = 0; s < 2; ++s) {
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
                    tc_fence_after();
                    issue_slab_layer(s, l, (int)(step & 1));
                    umma_commit(&c.acc_full[s]);
                }
                if (!ok || !any) break;
                umma_commit(&c.w_empty[step & 1]);
                if (step >= 1) {
                    if (!wait_bar(&c.w_empty[(step - 1) & 1], (uint32_t)(((step - 1) >> 1) & 1), 3)) { ok = false; ++step; break; }
                    issue_w(step + 1);
                }
                ++step;
            }
        }
        // drain: every weight copy issued and every MMA committed must finish
        const long long cb = p.budget_ns > 1000000000LL ? p.budget_ns : 1000000000LL;
        int dummy_abort = 0;
        for (int bsel = 0; bsel < 2; ++bsel)
            while (waited[bsel] < issued[bsel]) {
                if (!mbar_wait_bounded(&c.w_full[bsel], (uint32_t)(waited[bsel] & 1), &dummy_abort, cb,
                                       &p.status->flags, &p.status->timeout_site, 4))
                    break;
                waited[bsel]++;
            }
        umma_commit(&c.drain);   // completes once every MMA issued above has finished
        mbar_wait_bounded(&c.drain, 0, &dummy_abort, cb, &p.status->flags, &p.status->timeout_site, 5);
    }

    // ---------------------------------------------------------------- epilogue
    __device__ void row_coords(int r, const SlabMeta &m, int &y, int &j, int &x) const
    {
        y = r / m.PW;
        const int X = r - y * m.PW;
        j = X / (m.L + 2);
        x = X - j * (m.L + 2);
    }

    __device__ void store_layer(int s, int l, int tid)
    {
        const SlabMeta &m = c.slab[s];
        const int warp = tid >> 5, lane = tid & 31, g = warp >> 2, wq = warp & 3;
        const int L = m.L, PW = m.PW, count = m.count;
        const uint32_t out = smem_u32(act_buf(s, l & 1));
        const float *bias = p.bias32 + l * C + g * HALF;
        float bb[HALF];
#pragma unroll
        for (int i = 0; i < HALF; ++i) bb[i] = __ldg(bias + i);
        for (int t = 0; t < m.T; ++t) {
            const int r = t * 128 + wq * 32 + lane;
            const uint32_t taddr = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(s * p.Tcap * C + t * C + g * HALF);
            float v[HALF];
            if constexpr (HALF == 16) tmem_ld16(taddr, v); else tmem_ld8(taddr, v);
            int y, j, x;
            row_coords(r, m, y, j, x);
            if (y < L && x < L && j < count) {
                uint32_t w[HALF / 2];
#pragma unroll
                for (int i = 0; i < HALF / 2; ++i) {
                    const float h0 = 0.5f * (v[2 * i] + bb[2 * i]), h1 = 0.5f * (v[2 * i + 1] + bb[2 * i + 1]);
                    const float a0 = fmaf(h0, tanh_approx(h0), h0);   // SiLU(z) = (z/2)(1 + tanh(z/2))
                    const float a1 = fmaf(h1, tanh_approx(h1), h1);
                    w[i] = pack2<F16>(a0, a1);
                }
                const int R0 = (y + 1) * PW + j * (L + 2) + x + 1;
                int rows[4];
                int nr = 1;
                rows[0] = R0;
                const int hx = (x == 0) ? L : ((x == L - 1) ? -L : 0);
                const int vy = (y == 0) ? L * PW : ((y == L - 1) ? -L * PW : 0);
                if (hx) rows[nr++] = R0 + hx;
                if (vy) {
                    rows[nr++] = R0 + vy;
                    if (hx) rows[nr++] = R0 + vy + hx;
                }
                for (int q = 0; q < nr; ++q) {
                    const uint32_t a = out + (uint32_t)rows[q] * 16u;
                    if constexpr (HALF == 16) {
                        st_shared_v4(a + (2 * g) * PS, w[0], w[1], w[2], w[3]);
                        st_shared_v4(a + (2 * g + 1) * PS, w[4], w[5], w[6], w[7]);
                    } else {
                        st_shared_v4(a + g * PS, w[0], w[1], w[2], w[3]);
                    }
                }
            }
        }
    }

    __device__ void pool(int s, int tid)
    {
        SlabMeta &m = c.slab[s];
        const int warp = tid >> 5, lane = tid & 31, g = warp >> 2, wq = warp & 3;
        const int L = m.L, count = m.count, rows = 128 * m.T;
        float *partF = reinterpret_cast<float *>(act_buf(s, (p.D - 1) & 1));
        int *partI = reinterpret_cast<int *>(partF + 2 * rows);
        const float *bias = p.bias32 + p.D * C + g * HALF;
        float bb[HALF];
#pragma unroll
        for (int i = 0; i < HALF; ++i) bb[i] = __ldg(bias + i);
        for (int t = 0; t < m.T; ++t) {
            const int r = t * 128 + wq * 32 + lane;
            const uint32_t taddr = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(s * p.Tcap * C + t * C + g * HALF);
            float v[HALF];
            if constexpr (HALF == 16) tmem_ld16(taddr, v); else tmem_ld8(taddr, v);
            int y, j, x;
            row_coords(r, m, y, j, x);
            if (y < L && x < L && j < count) {
                float sl = 0.f;
                int neg = 0, zer = 0;
#pragma unroll
                for (int i = 0; i < HALF; ++i) {
                    const float z = v[i] + bb[i];
                    sl += __log2f(fabsf(z));
                    neg += (z < 0.f);
                    zer += (z == 0.f);
                }
                partF[g * rows + r] = sl;
                partI[g * rows + r] = neg | (zer << 16);
            }
        }
        epi_sync();
        // deterministic FP64 sum per configuration
        for (int j = warp; j < count; j += 8) {
            double acc = 0.0;
            int neg = 0, zer = 0;
            const int npix = L * L;
            for (int idx = lane; idx < 2 * npix; idx += 32) {
                const int hh = idx / npix, pix = idx - hh * npix;
                const int y = pix / L, x = pix - y * L;
                const int r = y * m.PW + j * (L + 2) + x;
                acc += (double)partF[hh * rows + r];
                const int nz = partI[hh * rows + r];
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
    // nine spins of sigma' around each cell, 16 BF16 per row in two planes.
    __device__ void build_rows(int s, int first, int n, int tid)
    {
        const SlabMeta &m = c.slab[s];
        const int L = m.L, PW = m.PW, npix = L * L;
        const uint32_t a0 = smem_u32(act_buf(s, 1));
        const uint32_t plane = 128u * m.T * 16u;
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
                    h[ky * 3 + kx] = F16 ? (v > 0 ? 0x3C00u : 0xBC00u) : (v > 0 ? 0x3F80u : 0xBF80u);
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
                if (c.cur_parent >= 0 && c.cur_k <= c.cur_nlist) {
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
                    if (P.valid) { c.abort = 1; atomicOr(&p.status->flags, VMC_STATUS_INTERNAL); }   // cannot happen: RING > parents in flight
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
            if (m.count >= m.G || c.abort) break;
        }
        const int count = m.count;
        if (count > 0) {
            // rows that belong to no configuration: zero (finite) input
            const int L = m.L, rows = 128 * m.T;
            const uint32_t a0 = smem_u32(act_buf(s, 1));
            const uint32_t plane = (uint32_t)rows * 16u;
            for (int r = tid; r < rows; r += NEPI) {
                int y, j, x;
                row_coords(r, m, y, j, x);
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
        tc_fence_before();
        epi_sync();
        if (tid == 0) mbar_arrive(&c.act_ready[s]);
    }

    __device__ void epilogue_role(int tid)
    {
        const int D = p.D;
        bool dead[2] = {false, true};
        uint32_t ph_af[2] = {0, 0};
        for (int s = 0; s < p.S; ++s) {
            const int cnt = fill(s, tid);
            signal_ready(s, tid);
            dead[s] = (cnt == 0);
        }
        while (!(dead[0] && dead[1])) {
            for (int l = 0; l <= D; ++l) {
                for (int s = 0; s < 2; ++s) {
                    if (dead[s]) continue;
                    if (tid == 0) c.ok = wait_bar(&c.acc_full[s], ph_af[s], 6) ? 1 : 0;
                    epi_sync();
                    if (!c.ok) return;
                    ph_af[s] ^= 1;
                    tc_fence_after();
                    if (l < D) {
                        store_layer(s, l, tid);
                        signal_ready(s, tid);
                    } else {
                        pool(s, tid);
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
            mbar_init(&c.acc_full[i], 1);
            mbar_init(&c.act_ready[i], 1);
            mbar_init(&c.w_full[i], 1);
            mbar_init(&c.w_empty[i], 1);
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
    if (warp == 8) tmem_alloc(&c.tmem_base, p.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    Kern<C, F16> k(p, smem, c, spins, list, BUF, c.tmem_base);
    if (warp < 8) k.epilogue_role(tid);
    else if ((tid & 31) == 0) k.mma_role();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 8) {
        __syncwarp();
        tmem_dealloc(c.tmem_base, p.tmem_cols);
    }
}

// ------------------------------------------------------------------ planning

static size_t ctrl_bytes(int L_max)
{
    return sizeof(Ctrl) + ((L_max * L_max + 15) & ~15) + (size_t)4 * L_max * L_max * 2 + 64;
}

static int rows_needed(int L, int G, int *T_out)
{
    const int PW = G * (L + 2);
    const int T = (L * PW + 127) / 128;
    *T_out = T;
    return std::max((L + 2) * PW, 128 * T + 2 * PW + 2);
}

struct Plan {
    int S, Rcap, Tcap;
    uint32_t tmem_cols;
    Geo geo[17];
    size_t smem;
};

// Largest-efficiency G for lattice L under the row / TMEM capacity.
static Geo best_geo(int L, int C, int S, int Rcap, int Tcap, int Gwant)
{
    Geo best{0, 0, 0};
    double be = -1.0;
    for (int G = 1; G <= MAX_SLOTS; ++G) {
        int T;
        const int R = rows_needed(L, G, &T);
        if (R > Rcap || T > Tcap) break;
        const double eff = (double)L * L * G / (128.0 * T);
        if (Gwant > 0) {
            if (G == Gwant) { best = Geo{G, T, G * (L + 2)}; be = eff; }
            continue;
        }
        if (eff > be + 1e-9) { be = eff; best = Geo{G, T, G * (L + 2)}; }
    }
    (void)C; (void)S;
    return best;
}

static int make_plan(const vmc_ctx *ctx, int L_main, int L_max, bool ragged, Plan *pl)
{
    const int C = ctx->arch.channels, D = ctx->arch.n_layers_cc;
    (void)D;
    TileChoice tc;
    auto it = ctx->tiles.find(L_main);
    if (it != ctx->tiles.end()) tc = it->second;
    const int S = tc.slabs ? tc.slabs : 2;
    const size_t wb = 2 * (size_t)(9 * (C / 16) * 32 * C);
    const size_t ctrl = ctrl_bytes(L_max);
    const size_t avail = SMEM_LIMIT - wb - ctrl - 1024;
    // row capacity of one plane from shared memory, tile capacity from TMEM
    int Rcap = (int)(avail / ((size_t)2 * S * (C / 8) * 16));
    int Tcap = 512 / (S * C);
    // For a uniform batch size the buffers to the chosen geometry.
    Geo gmain = best_geo(L_main, C, S, Rcap, Tcap, tc.slab_configs);
    if (gmain.G == 0) return VMC_ERR_UNSUPPORTED;
    if (!ragged) {
        int T;
        Rcap = rows_needed(L_main, gmain.G, &T);
        Tcap = T;
    }
    pl->S = S;
    pl->Rcap = Rcap;
    pl->Tcap = Tcap;
    for (int i = 0; i < 17; ++i) pl->geo[i] = Geo{0, 0, 0};
    if (ragged) {
        for (int L = 4; L <= L_max; L += 2) {
            TileChoice tl;
            auto jt = ctx->tiles.find(L);
            if (jt != ctx->tiles.end()) tl = jt->second;
            pl->geo[L >> 1] = best_geo(L, C, S, Rcap, Tcap, tl.slab_configs);
        }
    } else {
        pl->geo[L_main >> 1] = gmain;
    }
    uint32_t cols = 32;
    while (cols < (uint32_t)(S * Tcap * C)) cols <<= 1;
    if (cols > 512) return VMC_ERR_UNSUPPORTED;
    pl->tmem_cols = cols;
    pl->smem = wb + (size_t)2 * S * (C / 8) * Rcap * 16 + ctrl;
    if (pl->smem < 120 * 1024) pl->smem = 120 * 1024;   // keeps one CTA (and one TMEM owner) per SM
    if (pl->smem > SMEM_LIMIT) return VMC_ERR_UNSUPPORTED;
    return VMC_OK;
}

template <int C, bool F16>
static int launch(vmc_ctx *ctx, const Plan &pl, int mode, const int8_t *sigma, const int64_t *offs,
                  const int32_t *Ls, int64_t B, int L_max, double *out_a, void *out_b, int32_t *n_nbr,
                  cudaStream_t st, int grid_override)
{
    Params p;
    p.mode = mode; p.B = B; p.sigma = sigma; p.offs = offs; p.Ls = Ls;
    p.L_uniform = ctx->L; p.L_max = L_max;
    p.D = ctx->arch.n_layers_cc; p.marshall = ctx->arch.marshall_sign;
    p.J1 = ctx->J1; p.J2 = ctx->J2;
    p.wimg = reinterpret_cast<const uint8_t *>(ctx->wimg);
    p.bias32 = ctx->bias32;
    p.S = pl.S; p.Rcap = pl.Rcap; p.Tcap = pl.Tcap; p.tmem_cols = pl.tmem_cols;
    for (int i = 0; i < 17; ++i) p.geo[i] = pl.geo[i];
    p.out_a = out_a; p.out_sign = static_cast<int8_t *>(out_b); p.n_nbr = n_nbr;
    p.status = ctx->status; p.counter = ctx->counter;
    p.budget_ns = ctx->wait_budget_ns;
    auto kfn = tc_eloc_kernel<C, F16>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "cudaFuncSetAttribute(tc_eloc)");
    e = cudaMemsetAsync(ctx->counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "counter reset");
    int grid = grid_override > 0 ? grid_override : ctx->sm_count;
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
        return f16 ? launch<32, true>(ctx, pl, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr, st, 0)
                   : launch<32, false>(ctx, pl, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr, st, 0);
    return f16 ? launch<16, true>(ctx, pl, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr, st, 0)
               : launch<16, false>(ctx, pl, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr, st, 0);
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
    if (warp == 0) tmem_alloc(&tbase, 64);
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
    if (warp == 0) tmem_dealloc(tbase, 64);
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
    if (N < 16 || N > 64 || N % 16 || K < 16 || K > 64 || K % 16 || shift < 0 || shift > 64) return VMC_ERR_ARG;
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
