// Tensor-core (tcgen05, BF16/FP16 x BF16/FP16 -> FP32) forward pass, log|psi|
// and local energy: the hot loop of Sec. 3.1 ("sprime_batch") on sm_103a.
//
// Persistent CTAs, one per SM.  Each CTA pulls sampled configurations
// sigma from a global counter; for each it lists the antiparallel J1/J2
// bonds (Sec. 3.1, Fig. 2c) and streams sigma itself followed by every
// exchange neighbour sigma' through the network.  Configurations are packed
// into "slabs": G lattices side by side, each as (L+2) x (L+2) circularly
// padded cells, so a slab is an (L+2) x PW grid of cells (PW >= G (L+2)).
//
// Lane packing.  A TMEM lane (an MMA row) holds P consecutive cells of a
// grid row, so an accumulator tile is 128 lanes x P C columns and covers
// 128 P cells; column i C + co of lane r is output channel co of cell
// P r + i.  A C -> C layer (Eq. 5, 3 x 3 circular convolution) is an
// implicit GEMM: for every vertical tap ky (an A start-address offset of
// ky - 1 grid rows) and 16-channel K chunk h, input cell i of lane r feeds
// outputs i - 1, i, i + 1 of the same lane through one MMA whose B operand
// stacks the three horizontal taps along N (N = 3 C, fewer at the ends of
// the lane) and whose D address starts at column (i - 1) C; the last cell of
// lane r - 1 and the first of lane r + 1 feed outputs 0 and P - 1 through
// two N = C MMAs on A shifted by one row.  No data crosses TMEM lanes, so
// the epilogue is a plain per-lane bias + SiLU + store.  The MMAs of a
// tile are issued in the order (previous lane, cells 0..P-1, next lane) for
// every (ky, h): each output then sums its nine taps in the same order for
// every P and every slab geometry, so results do not depend on the tiling.
// Accumulators start from zero: the epilogue clears each TMEM slot as it
// drains it.  The embedding layer (c_in = 1) uses an im2col of the nine
// spins (K = 16, 7 zero), one N = C MMA per cell of the lane.
//
// Warp roles: warps 0-15 (the "epilogue" group) build neighbours, drain
// TMEM tile by tile (bias, SiLU -> 16-bit into the next padded buffer with
// the circular halo copies), pool the last layer and keep the per-parent
// FP64 energy sums; warps 16 and 17 issue the MMAs of alternate tiles (one
// lane each; warp 16 also allocates TMEM); warp 18 issues the per-layer
// weight bulk copies (a two-deep ring) and, in the one-slab light-cone
// pass, stages every slab fill.  Accumulators live in a ring of TMEM slots
// (one tile each) with full/empty mbarriers, and two slabs alternate (or,
// in the light-cone pass, a growing layer is handed to the next tile by
// tile), so the epilogue of one tile overlaps the MMAs of the next.  Every
// mbarrier wait is bounded by a time budget; on expiry the CTA raises
// VMC_ERR_TIMEOUT, drains its own copies and MMAs, frees TMEM and returns.
#pragma once
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

constexpr int NEPI_WARPS = 16;
constexpr int NEPI = NEPI_WARPS * 32;     // epilogue threads
constexpr int MMA_WARP = NEPI_WARPS;       // first of the MMA-issuing warps
constexpr int NMMA = 2;                    // MMA-issuing warps (alternate tiles)
constexpr int WGT_WARP = MMA_WARP + NMMA;  // the warp that issues the weight copies
constexpr int NTHREADS = NEPI + 32 * (NMMA + 1);
constexpr int MAX_SLOTS = 16;             // configurations per slab
constexpr int MAX_P = 8;                  // cells per TMEM lane (P C <= 128 accumulator columns)
constexpr int POOL_PARTS = 16;             // row blocks of a lattice summed separately by the pooling
constexpr int RING = 32;                  // parents in flight per CTA
constexpr int MAX_TSLOTS = 16;            // TMEM accumulator slots
constexpr int SMEM_LIMIT = 232448;

// slab geometry for one lattice side: configurations, cells per lane,
// tiles per layer, grid row width in cells (a multiple of P)
struct Geo { int G, P, T, PW; };

// Slab geometry of one layer: the lattice window its outputs cover (w x w
// cells, w = L for a whole lattice), tiles, grid row width in cells (a
// multiple of P), lanes per grid row, the start of the last tile past the
// first (max(w RW - 128, 0)) and the division magics for RW and w + 2; for
// the light-cone pass also those for the next window's ring (8 w + 16
// cells) and its grid side w + 4.
struct LayerGeo {
    int w, T, PW, RW, NRm;
    uint32_t mRW, mLP;
    uint32_t mRing, mW4;
};

// Kernel variants: the plain forward (log|psi| or E_loc with full forwards
// of every neighbour), the parent pass of the light-cone E_loc (log|psi|
// with the CNN sign only, every layer's activations stored to global
// memory), and the light-cone neighbour pass.
constexpr int VAR_PLAIN = 0, VAR_STORE = 1, VAR_CONE = 2;

struct Params {
    int mode;                   // 0 logpsi, 1 local energy
    long long B;
    const int8_t *sigma;
    const int64_t *offs;
    const int32_t *Ls;
    const int64_t *order;       // ragged batches: sample of each work item (nullable)
    int L_uniform, L_max;
    int D, marshall;
    double J1, J2;
    const uint8_t *wimg;
    const float *bias32;
    int S;
    uint32_t BUF;               // bytes of one activation buffer
    int slotc, nslots;          // TMEM columns per accumulator slot, slots
    Geo geo[17];
    double *out_a;
    int8_t *out_sign;
    int32_t *n_nbr;
    DevStatus *status;
    int *counter;
    long long budget_ns;
    // light-cone path: parent activations [b][layer 0..D-1][channel group][site]
    // (16 bytes each), written by the parent pass and read by the cone pass
    uint8_t *act_store;
    long long store_stride;     // bytes per parent
    const double *par_la;       // cone pass: parent log|psi_CNN|
    const int8_t *par_sg;       // cone pass: parent sign of psi_CNN (no Marshall factor)
    LayerGeo cone[17];          // cone pass: per-layer geometry (uniform lattice side)
    const LayerGeo *cone_tab;   // cone pass over a ragged batch: [L / 2][layer] (device), else null
};

struct Parent {
    long long b;
    double diag, la0, acc;
    int sg0, remaining, nlist, mpar, valid, L;
};

struct SlabMeta {
    int count, L, G, P;
    LayerGeo g;                           // every layer's geometry (plain and store variants)
    uint32_t PS;                          // plane stride (bytes)
    int parent[MAX_SLOTS];
    int bond[MAX_SLOTS];
    int pb[MAX_SLOTS];                    // store and cone variants: the sample index of the parent
    int8_t ox[MAX_SLOTS], oy[MAX_SLOTS];  // cone variant: lattice origin of the layer-0 window
};

struct __align__(16) Ctrl {   // 16-byte size: the arrays placed after it are read as float4
    uint64_t act_ready[2], w_full[2], w_empty[2], drain[NMMA];
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
    float pool_hi[MAX_SLOTS][POOL_PARTS];     // per-configuration pooling partials (double-float)
    float pool_lo[MAX_SLOTS][POOL_PARTS];
    int pool_nz[MAX_SLOTS][POOL_PARTS];
    double pool_la[MAX_SLOTS];                // per-configuration log|psi| and sign
    int pool_sg[MAX_SLOTS];
    Parent ring[RING];
    int mma_steps, mma_done;    // weight steps the MMA issuers ran; issuers finished
    int wpad[2];
    uint64_t staged;            // one-slab light-cone pass: a staged fill is ready
    SlabMeta stage;             // the staged fill
};

static_assert(sizeof(Ctrl) % 16 == 0, "control block size keeps what follows it 16-byte aligned");
static_assert(MAX_SLOTS <= NEPI_WARPS, "the pooling gives every configuration of a slab its own warp");

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 512;" ::: "memory"); }

// x / d for 0 <= x < 2^16, 1 <= d < 2^10: umulhi(x, floor(2^32 / d) + 1) is
// exact there for d >= 2; that multiplier does not fit 32 bits for d = 1,
// which is encoded as 0
__host__ __device__ __forceinline__ uint32_t udiv_magic(uint32_t d) { return d == 1u ? 0u : 0xFFFFFFFFu / d + 1u; }
__device__ __forceinline__ int udiv(int x, uint32_t m) { return m ? (int)__umulhi((uint32_t)x, m) : x; }

// (hi, lo) += x in double-float (TwoSum; lo collects the rounding errors)
__device__ __forceinline__ void df_add(float &hi, float &lo, float x)
{
    const float s = hi + x, bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}

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

// SiLU of z = 2 h, from h (the tensor-core weights and biases are halved).
// BF16 operands: h (1 + tanh h) with the hardware tanh (one MUFU op; its
// ~2^-11 error is below BF16 rounding for the bulk of activations).  FP16
// operands: z / (1 + e^-z) with e = exp(-|z|) (one MUFU op) and
// r = 1 / (1 + e) by Newton-Raphson from the linear estimate
// 24/17 - 8/17 d on [1, 2] (relative error 1/17 -> (1/17)^4 after two
// steps); sigmoid = r for z >= 0 and e r otherwise.
template <bool F16>
__device__ __forceinline__ float silu_h(float h)
{
    if constexpr (F16) {
        const float z = h + h;
        const float e = __expf(-fabsf(z));
        const float d = 1.0f + e;
        float r = fmaf(-0.47058823529f, d, 1.41176470588f);
        r = r * fmaf(-d, r, 2.0f);
        r = r * fmaf(-d, r, 2.0f);
        return z * (z >= 0.f ? r : e * r);
    } else {
        return fmaf(h, tanh_approx(h), h);
    }
}

// SiLU of the pair z = 2 (a, b), packed to 16 bits.  BF16 operands: in FP16
// pairs, h (1 + tanh h) with the paired hardware tanh (one MUFU op per two
// values; the FP16 rounding of h and of the product, 2^-11, is below the
// BF16 rounding of the result, and the tanh error is that of the FP32
// instruction); FP16 operands: silu_h per value.
template <bool F16>
__device__ __forceinline__ uint32_t silu_pack2(float a, float b)
{
    if constexpr (F16) {
        return pack2<true>(silu_h<true>(a), silu_h<true>(b));
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        uint32_t t;
        asm("tanh.approx.f16x2 %0, %1;" : "=r"(t) : "r"(*reinterpret_cast<const uint32_t *>(&h)));
        const __half2 y = __hfma2(h, *reinterpret_cast<const __half2 *>(&t), h);
        const float2 f = __half22float2(y);
        return pack2<false>(f.x, f.y);
    }
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ void st_global_v4(void *ptr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.global.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(ptr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// 16-byte asynchronous copy global -> shared (through L2 only), and the wait
// for every copy this thread has issued
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// stores that happen only where `p` holds (one predicated instruction each)
__device__ __forceinline__ void st_shared_v4_if(bool p, uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.shared.v4.b32 [%1], {%2, %3, %4, %5};\n\t}" ::"r"(
            (uint32_t)p),
        "r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
        : "memory");
}
__device__ __forceinline__ void st_shared_b32_if(bool p, uint32_t addr, uint32_t a)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.shared.b32 [%1], %2;\n\t}" ::"r"((uint32_t)p),
                 "r"(addr), "r"(a)
                 : "memory");
}
__device__ __forceinline__ void st_shared_f32_if(bool p, uint32_t addr, float a)
{
    st_shared_b32_if(p, addr, __float_as_uint(a));
}

__device__ __forceinline__ double nan_d() { return __longlong_as_double(0x7ff8000000000000LL); }

// up to four 8-column TMEM loads (columns c, c + S, c + 2 S, c + 3 S of the
// thread's lane) under one wait
template <int N, uint32_t S>
__device__ __forceinline__ void tmem_ld8_run(uint32_t ta, uint32_t (&r)[N][8])
{
    static_assert(N >= 1 && N <= 4, "1 to 4 chunks");
    if constexpr (N == 1) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[0][4]), "=r"(r[0][5]), "=r"(r[0][6]),
              "=r"(r[0][7])
            : "r"(ta)
            : "memory");
    } else if constexpr (N == 2) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[0][4]), "=r"(r[0][5]), "=r"(r[0][6]),
              "=r"(r[0][7]), "=r"(r[1][0]), "=r"(r[1][1]), "=r"(r[1][2]), "=r"(r[1][3]), "=r"(r[1][4]), "=r"(r[1][5]),
              "=r"(r[1][6]), "=r"(r[1][7])
            : "r"(ta), "r"(ta + S)
            : "memory");
    } else if constexpr (N == 3) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%24];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%25];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%26];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[0][4]), "=r"(r[0][5]), "=r"(r[0][6]),
              "=r"(r[0][7]), "=r"(r[1][0]), "=r"(r[1][1]), "=r"(r[1][2]), "=r"(r[1][3]), "=r"(r[1][4]), "=r"(r[1][5]),
              "=r"(r[1][6]), "=r"(r[1][7]), "=r"(r[2][0]), "=r"(r[2][1]), "=r"(r[2][2]), "=r"(r[2][3]), "=r"(r[2][4]),
              "=r"(r[2][5]), "=r"(r[2][6]), "=r"(r[2][7])
            : "r"(ta), "r"(ta + S), "r"(ta + 2 * S)
            : "memory");
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%32];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%33];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%34];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%35];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[0][4]), "=r"(r[0][5]), "=r"(r[0][6]),
              "=r"(r[0][7]), "=r"(r[1][0]), "=r"(r[1][1]), "=r"(r[1][2]), "=r"(r[1][3]), "=r"(r[1][4]), "=r"(r[1][5]),
              "=r"(r[1][6]), "=r"(r[1][7]), "=r"(r[2][0]), "=r"(r[2][1]), "=r"(r[2][2]), "=r"(r[2][3]), "=r"(r[2][4]),
              "=r"(r[2][5]), "=r"(r[2][6]), "=r"(r[2][7]), "=r"(r[3][0]), "=r"(r[3][1]), "=r"(r[3][2]), "=r"(r[3][3]),
              "=r"(r[3][4]), "=r"(r[3][5]), "=r"(r[3][6]), "=r"(r[3][7])
            : "r"(ta), "r"(ta + S), "r"(ta + 2 * S), "r"(ta + 3 * S)
            : "memory");
    }
}

// NM <= 8 chunks of 8 columns, S columns apart, under at most two waits
template <int NM, uint32_t S>
__device__ __forceinline__ void tmem_ld_chunks(uint32_t ta, float (&v)[NM][8])
{
    if constexpr (NM <= 4) {
        uint32_t r[NM][8];
        tmem_ld8_run<NM, S>(ta, r);
#pragma unroll
        for (int m = 0; m < NM; ++m)
#pragma unroll
            for (int q = 0; q < 8; ++q) v[m][q] = __uint_as_float(r[m][q]);
    } else {
        uint32_t r[4][8], r2[NM - 4][8];
        tmem_ld8_run<4, S>(ta, r);
        tmem_ld8_run<NM - 4, S>(ta + 4 * S, r2);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
#pragma unroll
            for (int m = 0; m < 4; ++m) v[m][q] = __uint_as_float(r[m][q]);
#pragma unroll
            for (int m = 4; m < NM; ++m) v[m][q] = __uint_as_float(r2[m - 4][q]);
        }
    }
}

// clear NM chunks of 8 columns, S columns apart (no wait)
template <int NM, uint32_t S>
__device__ __forceinline__ void tmem_zero_chunks_async(uint32_t ta)
{
    const uint32_t z = 0u;
#pragma unroll
    for (int m = 0; m < NM; ++m)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(ta + S * m),
                     "r"(z)
                     : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// clear NM chunks of 8 columns, S columns apart, and wait for the stores
template <int NM, uint32_t S>
__device__ __forceinline__ void tmem_zero_chunks(uint32_t ta)
{
    const uint32_t z = 0u;
#pragma unroll
    for (int m = 0; m < NM; ++m)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(ta + S * m),
                     "r"(z)
                     : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// NM: 8-column accumulator chunks each epilogue thread drains per tile
// (P C / 32), a compile-time constant so that the epilogue's registers are
// allocated for exactly one shape
template <int C, bool F16, int NM, int VAR>
struct Kern {
    static constexpr uint32_t WB = 18 * C * C;    // bytes of one C -> C layer image
    static constexpr int CP8 = C / 8;             // 16-byte channel planes per cell
    static constexpr int NCOL = 3 * C;            // rows of a C -> C B chunk
    static constexpr int P = NM * 32 / C;         // cells per TMEM lane

    const Params &p;
    uint8_t *smem;
    Ctrl &c;
    int8_t *spins;
    uint16_t *list;
    float *bias_s;              // (D + 1) C halved biases
    uint32_t tmem;

    __device__ Kern(const Params &p_, uint8_t *smem_, Ctrl &c_, int8_t *sp, uint16_t *li, float *bs, uint32_t tm)
        : p(p_), smem(smem_), c(c_), spins(sp), list(li), bias_s(bs), tmem(tm) {}

    __device__ uint8_t *act_buf(int s, int k) const { return smem + 2 * WB + (size_t)(2 * s + k) * p.BUF; }

    __device__ bool wait_bar(uint64_t *bar, uint32_t parity, int site)
    {
        return mbar_wait_bounded(bar, parity, &c.abort, p.budget_ns, &p.status->flags, &p.status->timeout_site, site);
    }

    // Slab geometry for lattice side L.
    __device__ void set_geometry(SlabMeta &m, int L, const Geo &g) const
    {
        m.L = L;
        m.G = g.G;
        m.P = g.P;
        m.g.w = L;
        m.g.T = g.T;
        m.g.PW = g.PW;
        m.g.RW = g.PW / g.P;
        m.g.NRm = max(L * m.g.RW - 128, 0);
        m.g.mRW = udiv_magic((uint32_t)m.g.RW);
        m.g.mLP = udiv_magic((uint32_t)(L + 2));
        m.g.mRing = 0u;
        m.g.mW4 = 0u;
        m.PS = (p.BUF / (uint32_t)(g.P * CP8 * 16)) * 16u;
    }

    // cone pass: the geometry of layer l for lattice side Ls
    __device__ __forceinline__ const LayerGeo &cone_geo(int Ls, int l) const
    {
        return p.cone_tab ? p.cone_tab[(Ls >> 1) * 17 + l] : p.cone[l];
    }

    // Geometry of layer l of slab s: per layer for the cone pass (from the
    // per-side table over a ragged batch), one for all layers otherwise.
    __device__ __forceinline__ const LayerGeo &lg(int s, int l) const
    {
        if constexpr (VAR == VAR_CONE) return cone_geo(c.slab[s].L, l);
        else return c.slab[s].g;
    }

    // first A row (lane 0) of tile t
    __device__ __forceinline__ static int tile_row(const LayerGeo &g, int t) { return g.RW + min(128 * t, g.NRm); }

    // Cone pass, layer l whose next window is wider (g0: layer l, g1: layer
    // l + 1): the last tile of layer l that must be drained before tile t of
    // layer l + 1 may start.  That tile reads its grid up to one grid row and
    // one lane past its own lanes; layer-l output row Y is row Y + 1 of the
    // next grid, and the epilogue drains the tiles of a layer in order, so
    // tiles 0 .. dep_tile hold every layer-l row it reads.
    __device__ __forceinline__ static int dep_tile(const LayerGeo &g0, const LayerGeo &g1, int t)
    {
        const int ymax = udiv(tile_row(g1, t) + 128 + g1.RW, g1.mRW);   // last grid row read
        const int yn = min(ymax - 1, g0.w);                          // last layer-l row needed
        const int x = (yn + 1) * g0.RW - 1 - g0.RW - 127;               // lanes past tile 0's last
        return min(x <= 0 ? 0 : (x + 127) >> 7, g0.T - 1);
    }

    // ---------------------------------------------------------------- MMA
    // One MMA whose descriptors are given as (low, high) words: the high
    // words (stride offset, version) are fixed for a tile, and the entries
    // below move only the 14-bit start-address field of the low words
    // (16-byte units; every address stays below 256 KB, so no carry leaves
    // the field).
    __device__ __forceinline__ static void mma_lh(uint32_t d, uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi,
                                                  uint32_t idesc)
    {
        asm volatile(
            "{\n\t.reg .pred p;\n\t.reg .b64 da, db;\n\t"
            "setp.ne.b32 p, %6, 0;\n\t"
            "mov.b64 da, {%1, %2};\n\t"
            "mov.b64 db, {%3, %4};\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n\t}" ::"r"(d),
            "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(1u)
            : "memory");
    }

    // MMAs of one (ky, h) step, in the order: last cell of the previous lane
    // (tap kx = 0 of output 0), cells 0..P-1 (cell i feeds output
    // i + 1 - kx for the taps kx it reaches inside the lane), first cell of
    // the next lane (tap kx = 2 of output P - 1); every output thus receives
    // kx = 0, 1, 2 in this order.  a / b: low descriptor words of the step.
    __device__ __forceinline__ void issue_step(uint32_t dslot, uint32_t a, uint32_t ahi, uint32_t b, uint32_t bhi,
                                               uint32_t ps16) const
    {
        mma_lh(dslot, a + (uint32_t)((P - 1) * CP8) * ps16 - 1u, ahi, b + 2 * C, bhi, idesc_f16kind(128, C, F16));
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const int jlo = i == 0 ? 1 : 0, jhi = (P - i) < 2 ? (P - i) : 2;
            mma_lh(dslot + (uint32_t)((i - 1 + jlo) * C), a + (uint32_t)(i * CP8) * ps16, ahi, b + (uint32_t)(jlo * C),
                   bhi, idesc_f16kind(128, (jhi - jlo + 1) * C, F16));
        }
        mma_lh(dslot + (uint32_t)((P - 1) * C), a + 1u, ahi, b, bhi, idesc_f16kind(128, C, F16));
    }

    __device__ void issue_tile(int s, int l, int t, int bsel, uint32_t dslot)
    {
        const SlabMeta &m = c.slab[s];
        const LayerGeo &g = lg(s, l);
        const uint32_t wb = smem_u32(smem + bsel * WB);
        const uint32_t PS = m.PS, RW = (uint32_t)g.RW, ps16 = PS >> 4;
        const int r0 = tile_row(g, t);
        if (l == 0) {
            const uint64_t ad = smem_desc(smem_u32(act_buf(s, 1)) + (uint32_t)(r0 + 1) * 16u, PS, 128);
            const uint64_t bd = smem_desc(wb, 16 * C, 128);
            const uint32_t alo = (uint32_t)ad, ahi = (uint32_t)(ad >> 32), blo = (uint32_t)bd, bhi = (uint32_t)(bd >> 32);
#pragma unroll
            for (int i = 0; i < P; ++i)
                mma_lh(dslot + (uint32_t)(i * C), alo + (uint32_t)(2 * i) * ps16, ahi, blo, bhi, idesc_f16kind(128, C, F16));
        } else {
            // descriptors at row r0 of the first plane and at the first chunk;
            // the tile's (ky, h) steps add ky - 1 grid rows, 2 h planes, chunk
            // ky (C/16) + h of 32 * NCOL bytes
            const uint64_t ad = smem_desc(smem_u32(act_buf(s, (l - 1) & 1)) + (uint32_t)(r0 + 1) * 16u, PS, 128);
            const uint64_t bd = smem_desc(wb, 16 * NCOL, 128);
            const uint32_t alo = (uint32_t)ad, ahi = (uint32_t)(ad >> 32), blo = (uint32_t)bd, bhi = (uint32_t)(bd >> 32);
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int h = 0; h < C / 16; ++h)
                    issue_step(dslot, alo + (uint32_t)(ky - 1) * RW + (uint32_t)(2 * h) * ps16, ahi,
                               blo + (uint32_t)((ky * (C / 16) + h) * 2 * NCOL), bhi, ps16);
        }
    }

    // MMA issue.  NMMA warps (one lane each) walk the same tile sequence
    // (layers, slabs, tiles) and issue alternate tiles: tile n goes to
    // warp n % NMMA, into TMEM slot n % nslots.  A single thread issues a
    // tcgen05.mma only every ~55 cycles, slower than the tensor cores
    // consume these narrow MMAs; two issuers reach the shared-memory operand
    // bound.  Each tile's MMAs come from one thread in a fixed order, so the
    // results do not depend on the split.  Both warps wait for the slab and
    // weight barriers; each commits its MMAs of a weight step to w_empty
    // (two arrivals per phase), which the weight warp waits on to reuse the
    // step's buffer.
    //
    // Cone pass, layer l - 1 -> l with a wider window (a "wavefront"
    // hand-off): no slab-wide ready barrier; before issuing tile t of layer
    // l, its issuer waits for the drain of tile dep_tile(t) of layer l - 1
    // (the epilogue publishes each tile of such a layer as it releases its
    // accumulator slot, after the copies of the window's ring), so the
    // first tiles of a layer start while the last ones of the layer before
    // are still being drained.
    __device__ void mma_role(int mw)
    {
        const int D = p.D, R = p.nslots;
        int nseq = 0;                       // sequence number of the next tile
        int first_prev[2] = {0, 0};         // first tile of slab s's previous layer
        int Lsnap[2] = {0, 0};
        bool dead[2] = {false, p.S < 2};
        int cnt[2] = {0, 0};
        uint32_t ph_ar[2] = {0, 0};
        long long step = 0;           // weight step; its layer is l (the loop runs every layer of every step)
        // tile sequence number n, kept as its slot n % R, the slot's use
        // parity (n / R) & 1 and its issuing warp n % NMMA
        int nslot = 0, nwarp = 0;
        uint32_t npar = 0;
        bool ok = true;
        while (ok && !(dead[0] && dead[1])) {
            for (int l = 0; l <= D && ok; ++l) {
                bool any = false;
                for (int s = 0; s < 2 && ok; ++s) {
                    if (dead[s]) continue;
                    const bool wf = VAR == VAR_CONE && l >= 1 && cone_geo(Lsnap[s], l).w > cone_geo(Lsnap[s], l - 1).w;
                    if (!wf && (l == 0 || cnt[s] > 0)) {
                        if (!wait_bar(&c.act_ready[s], ph_ar[s], 1)) { ok = false; break; }
                        ph_ar[s] ^= 1;
                    }
                    if (l == 0) {
                        cnt[s] = *(volatile int *)&c.slab[s].count;
                        // the slab's lattice side, read once per fill: this warp
                        // may still walk the slab's last tiles (issued by the
                        // other warp) after the epilogue has refilled it
                        Lsnap[s] = *(volatile int *)&c.slab[s].L;
                        if (cnt[s] == 0) { dead[s] = true; continue; }
                    }
                    if (!any) {
                        const int bsel = (int)(step & 1);
                        if (!wait_bar(&c.w_full[bsel], (uint32_t)((step >> 1) & 1), 2)) { ok = false; break; }
                        any = true;
                    }
                    int T;
                    if constexpr (VAR == VAR_CONE) T = cone_geo(Lsnap[s], l).T;
                    else T = *(volatile int *)&c.slab[s].g.T;
                    const int fprev = first_prev[s];
                    first_prev[s] = nseq;
                    const LayerGeo *gp = nullptr, *gc = nullptr;
                    if constexpr (VAR == VAR_CONE) {
                        gp = &cone_geo(Lsnap[s], l > 0 ? l - 1 : 0);
                        gc = &cone_geo(Lsnap[s], l);
                    }
                    for (int t = 0; t < T; ++t) {
                        const int slot = nslot;
                        const uint32_t use_par = npar;
                        const bool mine = (nwarp == mw);
                        const int n = nseq++;
                        if (++nslot == R) { nslot = 0; npar ^= 1u; }
                        if (++nwarp == NMMA) nwarp = 0;
                        if (!mine) continue;
                        if (!wait_bar(&c.t_empty[slot], use_par ^ 1u, 3)) { ok = false; break; }
                        if (wf) {
                            // the drain of tile n - back (and, tiles draining in
                            // order, of every tile before it).  Tile n - R is drained
                            // (the wait above), so that tile's slot has finished its
                            // use before it; a tile R or more back is waited for
                            // through a later one, whose slot is not reused before
                            // tile n: the parity then names exactly the phase of its
                            // use.  Its slot and parity follow from tile n's.
                            const int back = min(n - (fprev + dep_tile(*gp, *gc, t)), R - 1);   // >= 1
                            int sd = slot - back;
                            uint32_t pd = use_par;
                            if (sd < 0) { sd += R; pd ^= 1u; }
                            if (!wait_bar(&c.t_empty[sd], pd, 8)) { ok = false; break; }
                        }
                        tc_fence_after();
                        issue_tile(s, l, t, (int)(step & 1), tmem + (uint32_t)(slot * p.slotc));
                        umma_commit(&c.t_full[slot]);
                    }
                }
                if (!ok || !any) break;
                // the step's weight buffer is free once these MMAs complete
                umma_commit(&c.w_empty[step & 1]);
                ++step;
            }
        }
        // tell the weight warp how many steps ran, then drain every MMA issued
        atomicMax(&c.mma_steps, (int)step);
        __threadfence_block();
        atomicAdd(&c.mma_done, 1);
        const long long cb = p.budget_ns > 1000000000LL ? p.budget_ns : 1000000000LL;
        int dummy_abort = 0;
        umma_commit(&c.drain[mw]);
        mbar_wait_bounded(&c.drain[mw], 0, &dummy_abort, cb, &p.status->flags, &p.status->timeout_site, 6);
    }

    // Weight copies (lane 0 of warp WGT_WARP).  Weight step st holds layer
    // st mod (D + 1) (the issuers run every layer of every slab fill) in
    // buffer st & 1; the copy for step st goes out as soon as the MMAs of
    // step st - 2, the last readers of that buffer, have completed (both
    // issuers commit each step to w_empty), independently of where either
    // issuer is in its walk.  With producer_fill() the whole warp also
    // stages each slab fill when the previous slab's last layer has
    // completed.  The warp ends once both issuers have finished and no step
    // that ran is left, after every copy it issued has landed.
    __device__ void weight_role(int lane)
    {
        const int D = p.D;
        const bool prod = producer_fill();
        auto issue = [&](long long st) {
            const int b = (int)(st & 1), l = (int)(st % (D + 1));
            const uint32_t bytes = (uint32_t)tc_layer_bytes(C, l);
            mbar_expect_tx(&c.w_full[b], bytes);
            bulk_g2s(smem + b * WB, p.wimg + tc_wimg_offset(C, l), bytes, &c.w_full[b]);
        };
        // the first fill, staged before the first weights (both are needed
        // before the first MMA)
        bool more = prod ? stage_fill(lane) : false;
        if (lane == 0) {
            issue(0);
            issue(1);
        }
        long long st = 2;
        uint64_t t0 = global_timer_ns();
        for (;;) {
            int done = 0, stop = 0;
            if (lane == 0) {
                if (mbar_try_wait(&c.w_empty[st & 1], (uint32_t)(((st - 2) >> 1) & 1))) {
                    done = 1;
                } else if (*(volatile int *)&c.mma_done == NMMA && st - 2 >= *(volatile int *)&c.mma_steps) {
                    stop = 1;
                } else if (*(volatile int *)&c.abort) {
                    stop = 1;
                } else if ((long long)(global_timer_ns() - t0) > p.budget_ns) {
                    c.abort = 1;
                    atomicOr(&p.status->flags, VMC_STATUS_TIMEOUT);
                    p.status->timeout_site = 4;
                    stop = 1;
                }
            }
            done = __shfl_sync(0xffffffffu, done, 0);
            stop = __shfl_sync(0xffffffffu, stop, 0);
            if (stop) break;
            if (!done) continue;
            if (lane == 0) issue(st);
            // step st - 2 was a slab's last layer: its input buffer is free and
            // the next fill can be staged
            if (more && (st - 2) % (D + 1) == D) more = stage_fill(lane);
            ++st;
            if (lane == 0) t0 = global_timer_ns();
        }
        // the copies of the last two steps (one per buffer, each its buffer's
        // latest phase) may not have been waited for by an issuer
        if (lane == 0) {
            const long long cb = p.budget_ns > 1000000000LL ? p.budget_ns : 1000000000LL;
            int dummy_abort = 0;
            for (long long q = st - 2; q < st; ++q)
                mbar_wait_bounded(&c.w_full[q & 1], (uint32_t)((q >> 1) & 1), &dummy_abort, cb, &p.status->flags,
                                  &p.status->timeout_site, 5);
        }
    }

    // ---------------------------------------------------------------- epilogue
    // Per-(slab, layer) constants of the epilogue threads.  A thread of warp
    // w drains TMEM lane quarter w & 3 and the 8-column chunks k = g4 + 4 m
    // (g4 = w >> 2) of each tile: channel plane g = k % (C/8) of cell
    // k / (C/8), i.e. plane g4 of cell m for C = 32, plane g4 & 1 of cell
    // 2 m + g4 / 2 for C = 16; one bias vector per thread.
    struct TileCtx {
        int L, PW, RW, NRm, T, count, NQ;   // L: side of this layer's window (the lattice side unless a cone)
        uint32_t mRW, mLP, PS;
        uint32_t out;           // output buffer (shared address)
        int l;                  // layer
        int grow;               // cone pass: the next layer's window is 2 cells wider (no halo copies)
        int RWn;                // cone pass, grow: lanes per grid row of the next layer
        const SlabMeta *sm;
        float bias[8];
    };

    __device__ __forceinline__ void load_tctx(int s, int l, int tid, TileCtx &k) const
    {
        const SlabMeta &m = c.slab[s];
        const LayerGeo &g0 = lg(s, l);
        k.L = g0.w; k.PW = g0.PW; k.RW = g0.RW; k.NRm = g0.NRm; k.T = g0.T; k.count = m.count;
        k.NQ = (g0.w + 2) * g0.PW;
        k.mRW = g0.mRW; k.mLP = g0.mLP; k.PS = m.PS;
        k.l = l;
        k.grow = 0;
        k.RWn = 0;
        if constexpr (VAR == VAR_CONE) {
            if (l < p.D) {
                const LayerGeo &g1 = lg(s, l + 1);
                if (g1.w > g0.w) { k.grow = 1; k.RWn = g1.RW; }
            }
        }
        k.sm = &m;
        k.out = smem_u32(act_buf(s, l & 1));
        const int g = ((tid >> 5) >> 2) & (CP8 - 1);
        const float4 *b4 = reinterpret_cast<const float4 *>(bias_s + l * C + g * 8);
        const float4 lo = b4[0], hi = b4[1];
        k.bias[0] = lo.x; k.bias[1] = lo.y; k.bias[2] = lo.z; k.bias[3] = lo.w;
        k.bias[4] = hi.x; k.bias[5] = hi.y; k.bias[6] = hi.z; k.bias[7] = hi.w;
    }

    // Chunks [M0, M0 + N) of a tile, values in v: for each chunk of an
    // interior cell either store SiLU(z) (with its circular halo copies) or,
    // for the last layer, the pooling partials.  Branch-free: every chunk is
    // computed and each store carries its own predicate, so the chunks'
    // arithmetic interleaves.
    template <int M0, int N, bool POOL>
    __device__ __forceinline__ void put_chunks(const float (&v)[N][8], int g4, int r, int Y, int rX, int Yh,
                                               bool fresh, const TileCtx &k, float *partF, int *partI)
    {
        const int L = k.L;
        const bool row_in = (Y >= 1) & (Y <= L) & fresh;
        const int g = g4 & (CP8 - 1);
        // the lane's P cells are consecutive in X: configuration j and column x
        // of the first, then advance (wrapping into the next configuration)
        const int X0 = P * rX + ((CP8 == 4) ? M0 : 2 * M0 + (g4 >> 1));
        int j = udiv(X0, k.mLP);
        int x = X0 - j * (L + 2) - 1;
        const uint32_t outg = k.out + (uint32_t)g * k.PS;
        const int Yv = Yh < 0 ? Y : Yh;
        const uint32_t rowY = (uint32_t)(Y * k.RW + 1) * 16u, rowV = (uint32_t)(Yv * k.RW + 1) * 16u;
#pragma unroll
        for (int mm = 0; mm < N; ++mm) {
            const int m = M0 + mm;
            // chunk k = g4 + 4 m: cell i, channel plane g
            const int i = (CP8 == 4) ? m : 2 * m + (g4 >> 1);
            if (mm > 0) {
                x += (CP8 == 4) ? 1 : 2;
                if (x > L) { x -= L + 2; ++j; }
            }
            const int X = P * rX + i;
            const bool valid = row_in & (x >= 0) & (x < L) & (j < k.count);
            float h[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) h[q] = v[mm][q] + k.bias[q];
            if constexpr (POOL) {
                float sl = 0.f;
                int neg = 0, zer = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    sl += __log2f(fabsf(h[q]));
                    neg += (h[q] < 0.f);
                    zer += (h[q] == 0.f);
                }
                int qc = g * k.NQ + Y * k.PW + X;
                if constexpr (VAR == VAR_CONE) {
                    // the window of the last layer is the whole lattice seen
                    // from its own origin: file the partial at the cell's
                    // lattice position, so the pooling sums in the order of
                    // the plain forward
                    const int jj = j < MAX_SLOTS ? j : 0;
                    const int ls = (L - 4) >> 1;
                    int xl = (int)k.sm->ox[jj] - ls + x, yl = (int)k.sm->oy[jj] - ls + Y - 1;
                    xl += (xl < 0) ? L : 0; xl -= (xl >= L) ? L : 0;
                    yl += (yl < 0) ? L : 0; yl -= (yl >= L) ? L : 0;
                    qc = g * k.NQ + (yl + 1) * k.PW + j * (L + 2) + xl + 1;
                }
                // log2|z| = log2|h| + 1 per channel
                st_shared_f32_if(valid, smem_u32(partF + qc), sl + 8.0f);
                st_shared_b32_if(valid, smem_u32(partI + qc), (uint32_t)(neg | (zer << 16)));
            } else {
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) w[q] = silu_pack2<F16>(h[2 * q], h[2 * q + 1]);
                if constexpr (VAR == VAR_STORE) {
                    // parent pass: the activation also goes to the parent store
                    if (valid) {
                        const int jj = j < MAX_SLOTS ? j : 0;
                        uint8_t *dst = p.act_store + (long long)k.sm->pb[jj] * p.store_stride +
                                       ((long long)(k.l * CP8 + g) * (L * L) + (Y - 1) * L + x) * 16;
                        st_global_v4(dst, w[0], w[1], w[2], w[3]);
                    }
                }
                if constexpr (VAR == VAR_CONE) {
                    if (k.grow) {
                        // output cell (x, Y - 1) of window j moves to cell
                        // (x + 2, Y + 1) of the next layer's window, which is
                        // 4 cells wider including its halo; the ring around
                        // it comes from the parent
                        const int Xn = j * (L + 4) + x + 2;
                        const int qn = Xn / P;
                        const uint32_t dst = outg + (uint32_t)((Xn - qn * P) * CP8) * k.PS +
                                             (uint32_t)((Y + 1) * k.RWn + qn + 1) * 16u;
                        st_shared_v4_if(valid, dst, w[0], w[1], w[2], w[3]);
                        continue;
                    }
                }
                const uint32_t plane = outg + (uint32_t)(i * CP8) * k.PS;
                // circular halo copies: column X -/+ L, row L + 1 / 0, and the corner
                const int hx = (x == 0) ? L : ((x == L - 1) ? -L : 0);
                const int X2 = X + hx;
                const int xr = X2 / P;
                const uint32_t hplane = outg + (uint32_t)((X2 - xr * P) * CP8) * k.PS + (uint32_t)xr * 16u;
                const uint32_t rr = (uint32_t)rX * 16u;
                st_shared_v4_if(valid, plane + (uint32_t)(r + 1) * 16u, w[0], w[1], w[2], w[3]);
                st_shared_v4_if(valid & (hx != 0), hplane + rowY, w[0], w[1], w[2], w[3]);
                st_shared_v4_if(valid & (Yh >= 0), plane + rowV + rr, w[0], w[1], w[2], w[3]);
                st_shared_v4_if(valid & (hx != 0) & (Yh >= 0), hplane + rowV, w[0], w[1], w[2], w[3]);
            }
        }
    }

    // The thread's NM chunks when they are channel planes g0 .. g0 + NM - 1
    // of one cell of the lane (NM divides C/8): the cell's position,
    // validity and addresses are computed once.  Same stores as put_chunks.
    template <bool POOL>
    __device__ __forceinline__ void put_cell(const float (&v)[NM][8], int g4, int r, int Y, int rX, int Yh,
                                             bool fresh, const TileCtx &k, float *partF, int *partI)
    {
        const int L = k.L;
        const int ic = (g4 * NM) / CP8, g0 = (g4 * NM) % CP8;
        const int X = P * rX + ic;
        const int j = udiv(X, k.mLP);
        const int x = X - j * (L + 2) - 1;
        const bool valid = (Y >= 1) & (Y <= L) & fresh & (x >= 0) & (x < L) & (j < k.count);
        const float4 *b4 = reinterpret_cast<const float4 *>(bias_s + k.l * C + g0 * 8);
        if constexpr (POOL) {
            int q0 = Y * k.PW + X;
            if constexpr (VAR == VAR_CONE) {
                // the last layer's window is the whole lattice seen from its
                // own origin: file the partials at the cell's lattice position
                const int jj = j < MAX_SLOTS ? j : 0;
                const int ls = (L - 4) >> 1;
                int xl = (int)k.sm->ox[jj] - ls + x, yl = (int)k.sm->oy[jj] - ls + Y - 1;
                xl += (xl < 0) ? L : 0; xl -= (xl >= L) ? L : 0;
                yl += (yl < 0) ? L : 0; yl -= (yl >= L) ? L : 0;
                q0 = (yl + 1) * k.PW + j * (L + 2) + xl + 1;
            }
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const float4 b0 = b4[2 * m], b1 = b4[2 * m + 1];
                const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                float sl = 0.f;
                int neg = 0, zer = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float h = v[m][q] + bb[q];
                    sl += __log2f(fabsf(h));
                    neg += (h < 0.f);
                    zer += (h == 0.f);
                }
                const int qc = (g0 + m) * k.NQ + q0;
                // log2|z| = log2|h| + 1 per channel
                st_shared_f32_if(valid, smem_u32(partF + qc), sl + 8.0f);
                st_shared_b32_if(valid, smem_u32(partI + qc), (uint32_t)(neg | (zer << 16)));
            }
        } else {
            // destination of plane g0 (the others follow PS apart) and, for the
            // circular halo, the cell's copies
            uint32_t dst0, hdst = 0u;
            bool grow = false;
            if constexpr (VAR == VAR_CONE) grow = k.grow != 0;
            const int hx = (x == 0) ? L : ((x == L - 1) ? -L : 0);
            const int Yv = Yh < 0 ? Y : Yh;
            if (grow) {
                const int Xn = j * (L + 4) + x + 2;
                const int qn = Xn / P;
                dst0 = k.out + (uint32_t)((Xn - qn * P) * CP8 + g0) * k.PS + (uint32_t)((Y + 1) * k.RWn + qn + 1) * 16u;
            } else {
                dst0 = k.out + (uint32_t)(ic * CP8 + g0) * k.PS + (uint32_t)(r + 1) * 16u;
                const int X2 = X + hx;
                const int xr = X2 / P;
                hdst = k.out + (uint32_t)((X2 - xr * P) * CP8 + g0) * k.PS + (uint32_t)xr * 16u;
            }
            const uint32_t rowY = (uint32_t)(Y * k.RW + 1) * 16u, rowV = (uint32_t)(Yv * k.RW + 1) * 16u;
            const uint32_t rr = (uint32_t)rX * 16u;
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const float4 b0 = b4[2 * m], b1 = b4[2 * m + 1];
                uint32_t w[4];
                w[0] = silu_pack2<F16>(v[m][0] + b0.x, v[m][1] + b0.y);
                w[1] = silu_pack2<F16>(v[m][2] + b0.z, v[m][3] + b0.w);
                w[2] = silu_pack2<F16>(v[m][4] + b1.x, v[m][5] + b1.y);
                w[3] = silu_pack2<F16>(v[m][6] + b1.z, v[m][7] + b1.w);
                const uint32_t pm = (uint32_t)m * k.PS;
                if constexpr (VAR == VAR_STORE) {
                    // parent pass: the activation also goes to the parent store
                    if (valid) {
                        const int jj = j < MAX_SLOTS ? j : 0;
                        uint8_t *gd = p.act_store + (long long)k.sm->pb[jj] * p.store_stride +
                                      ((long long)(k.l * CP8 + g0 + m) * (L * L) + (Y - 1) * L + x) * 16;
                        st_global_v4(gd, w[0], w[1], w[2], w[3]);
                    }
                }
                if (grow) {
                    st_shared_v4_if(valid, dst0 + pm, w[0], w[1], w[2], w[3]);
                } else {
                    st_shared_v4_if(valid, dst0 + pm, w[0], w[1], w[2], w[3]);
                    st_shared_v4_if(valid & (hx != 0), hdst + pm + rowY, w[0], w[1], w[2], w[3]);
                    st_shared_v4_if(valid & (Yh >= 0), dst0 + pm + rowV + rr - (uint32_t)(r + 1) * 16u, w[0], w[1], w[2], w[3]);
                    st_shared_v4_if(valid & (hx != 0) & (Yh >= 0), hdst + pm + rowV, w[0], w[1], w[2], w[3]);
                }
            }
        }
    }

    // One tile: load the thread's NM chunks under one wait, start clearing
    // them, put the values, and release the slot once the clearing stores
    // have completed.  PUB (a cone layer whose window grows): the release
    // also publishes the tile's activations to the next layer's MMAs, after
    // the copies of the window's ring (issued before the layer's first tile).
    template <bool POOL, bool PUB>
    __device__ __forceinline__ void epi_tile(int t, int slot, int tid, const TileCtx &k, bool ok, float *partF,
                                             int *partI)
    {
        const int warp = tid >> 5, lane = tid & 31, wq = warp & 3, g4 = warp >> 2;
        // NM dividing C/8: the thread's chunks are consecutive columns (planes
        // of one cell); otherwise chunks g4 + 4 m
        constexpr bool SAMECELL = (CP8 % NM) == 0;
        const uint32_t ta = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(slot * p.slotc + 8 * (SAMECELL ? g4 * NM : g4));
        const int r = k.RW + min(128 * t, k.NRm) + wq * 32 + lane;
        const int Y = udiv(r, k.mRW);
        const int rX = r - Y * k.RW;
        const int L = k.L;
        const int Yh = (Y == 1) ? L + 1 : ((Y == L) ? 0 : -1);
        // the last tile starts early so as not to run past the grid: its
        // first `ov` rows were already drained (and stored, bitwise the same)
        // by the tile before; warps whose rows all lie there skip the work
        const int ov = (t == k.T - 1) ? 128 * t - k.NRm : 0;
        float v[NM][8];
        if (ok) {
            if constexpr (SAMECELL) {
                tmem_ld_chunks<NM, 8>(ta, v);
                tmem_zero_chunks_async<NM, 8>(ta);
                if (wq * 32 + 31 >= ov) put_cell<POOL>(v, g4, r, Y, rX, Yh, wq * 32 + lane >= ov, k, partF, partI);
            } else {
                tmem_ld_chunks<NM, 32>(ta, v);
                tmem_zero_chunks_async<NM, 32>(ta);
                if (wq * 32 + 31 >= ov) put_chunks<0, NM, POOL>(v, g4, r, Y, rX, Yh, wq * 32 + lane >= ov, k, partF, partI);
            }
            __syncwarp();
            tmem_wait_st();
        }
        if constexpr (PUB) {
            if (t == 0) cp_async_wait_all();
            fence_proxy_async_smem();
        }
        tc_fence_before();
        __syncwarp();
        if (ok && lane == 0) mbar_arrive(&c.t_empty[slot]);
    }

    // Per-configuration FP64 sums and the per-parent bookkeeping.  Each
    // configuration's lattice is cut into POOL_PARTS blocks of rows; warps
    // take (configuration, block) tasks, then warp j adds configuration j's
    // blocks in a fixed tree, so the summation order depends on L only, not
    // on the slab; thread 0 applies the configurations to their parents in
    // slab order.
    __device__ void pool_finish(int s, int tid, const float *partF, const int *partI, int NQ)
    {
        SlabMeta &m = c.slab[s];
        const int warp = tid >> 5, lane = tid & 31;
        const int L = m.L, count = m.count, PW = lg(s, p.D).PW;
        for (int task = warp; task < count * POOL_PARTS; task += NEPI_WARPS) {
            const int j = task / POOL_PARTS, part = task - j * POOL_PARTS;
            const int y0 = part * L / POOL_PARTS, y1 = (part + 1) * L / POOL_PARTS;
            // double-float sums (FP32 pairs, ~2^-48 relative): the FP64 pipe of
            // this part is slow, and the block sums need more than FP32
            float hi = 0.f, lo = 0.f;
            int neg = 0, zer = 0;
            if (lane < L) {
                for (int y = y0; y < y1; ++y) {
                    const int q0 = (y + 1) * PW + j * (L + 2) + lane + 1;
#pragma unroll
                    for (int gg = 0; gg < CP8; ++gg) {
                        const int q = gg * NQ + q0;
                        df_add(hi, lo, partF[q]);
                        const int nz = partI[q];
                        neg += nz & 0xffff;
                        zer += nz >> 16;
                    }
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
                df_add(hi, lo, oh);
                lo += ol;
                neg += __shfl_xor_sync(0xffffffffu, neg, o);
                zer += __shfl_xor_sync(0xffffffffu, zer, o);
            }
            if (lane == 0) {
                c.pool_hi[j][part] = hi;
                c.pool_lo[j][part] = lo;
                c.pool_nz[j][part] = (neg & 0xffff) | (zer << 16);
            }
        }
        epi_sync();
        // warp j adds configuration j's blocks (lane = block) in a fixed tree
        if (warp < count) {
            const int j = warp;
            float hi = 0.f, lo = 0.f;
            int neg = 0, zer = 0;
            if (lane < POOL_PARTS) {
                hi = c.pool_hi[j][lane];
                lo = c.pool_lo[j][lane];
                neg = c.pool_nz[j][lane] & 0xffff;
                zer = c.pool_nz[j][lane] >> 16;
            }
            for (int o = POOL_PARTS / 2; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
                df_add(hi, lo, oh);
                lo += ol;
                neg += __shfl_xor_sync(0xffffffffu, neg, o);
                zer += __shfl_xor_sync(0xffffffffu, zer, o);
            }
            if (lane == 0) {
                const double acc = (double)hi + (double)lo;
                c.pool_la[j] = zer ? -INFINITY : acc * 0.69314718055994530942;
                c.pool_sg[j] = zer ? 0 : ((neg & 1) ? -1 : 1);
            }
        }
        epi_sync();
        if (tid == 0) {
            for (int j = 0; j < count; ++j) {
                const double la = c.pool_la[j];
                const int sg = c.pool_sg[j];
                Parent &P = c.ring[m.parent[j]];
                if (m.bond[j] < 0) {
                    P.la0 = la;
                    P.sg0 = sg;
                } else {
                    // the ratio needs the FP64 difference, not an FP64 exponential:
                    // expf's ~1e-7 relative error is far below the tolerance
                    // of the 16-bit network
                    const double rho = (double)(sg * P.sg0) * (double)__expf((float)(la - P.la0));
                    P.acc += exchange_coef(m.bond[j] & 3, p.J1, p.J2, p.marshall) * rho;
                }
                if (--P.remaining == 0) {
                    finish_parent(P);
                    P.valid = 0;
                }
            }
        }
        // no barrier: fill's first step runs on thread 0 too, and the other
        // threads touch the slab only after fill's barrier
    }

    __device__ void finish_parent(const Parent &P)
    {
        const long long b = P.b;
        if (p.mode == 0) {
            int sg = P.sg0;
            if (VAR != VAR_STORE && p.marshall && P.mpar) sg = -sg;
            p.out_a[b] = P.la0;
            p.out_sign[b] = (int8_t)sg;
            // the parent pass of the light-cone E_loc leaves the verdict on a
            // non-finite amplitude to the neighbour pass (one count per sample)
            if (VAR != VAR_STORE && (P.la0 != P.la0 || P.la0 == INFINITY)) {
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

    // Build the embedding-layer im2col rows of slots [first, first+n): nine
    // spins of sigma' around each interior cell, 16 values in two planes
    // (planes 2 i, 2 i + 1 for cell i of its lane).  One warp per lattice
    // row, lane = x (L <= 32), so no per-cell division.
    __device__ void build_rows(int s, int first, int n, int tid)
    {
        const SlabMeta &m = c.slab[s];
        const int L = m.L, PW = m.g.PW;
        const uint32_t a0 = smem_u32(act_buf(s, 1));
        const uint32_t PS = m.PS;
        const uint32_t up = F16 ? 0x3C00u : 0x3F80u, dn = F16 ? 0xBC00u : 0xBF80u;
        const int warp = tid >> 5, x = tid & 31;
        const int xl = x == 0 ? L - 1 : x - 1, xr = x == L - 1 ? 0 : x + 1;
        for (int row = warp; row < n * L; row += NEPI_WARPS) {
            const int jrel = row / L, y = row - jrel * L;
            if (x >= L) continue;
            const int jj = first + jrel;
            const int bond = m.bond[jj];
            int bi = -1, bj = -1;
            if (bond >= 0) { bi = bond >> 2; bj = bond_partner(L, bi, bond & 3); }
            const int ym = y == 0 ? L - 1 : y - 1, yp = y == L - 1 ? 0 : y + 1;
            const int rows3[3] = {ym * L, y * L, yp * L};
            const int cols3[3] = {xl, x, xr};
            uint32_t h[9];
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const int site = rows3[ky] + cols3[kx];
                    const int src = site == bi ? bj : (site == bj ? bi : site);
                    h[ky * 3 + kx] = spins[src] > 0 ? up : dn;
                }
            const int q = (y + 1) * PW + jj * (L + 2) + x + 1;
            const int r = q / P;
            const int i = q - r * P;
            const uint32_t a = a0 + 2u * (uint32_t)i * PS + (uint32_t)(r + 1) * 16u;
            st_shared_v4(a, h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
            st_shared_v4(a + PS, h[8], 0u, 0u, 0u);
        }
    }

    // Cone pass, embedding layer: the im2col rows of the w0 x w0 window of
    // each neighbour sigma' of slots [first, first + n) of meta m (filling
    // slab s), the window's cell (X, Y), 1 <= X, Y <= w0, being lattice site
    // (ox + X - 1, oy + Y - 1) mod L; windows lie side by side, w0 + 2 cells
    // apart.  Threads t0, t0 + nthr, ... of the filling group.
    __device__ void build_rows_cone(const SlabMeta &m, int s, int first, int n, int t0, int nthr)
    {
        const int L = m.L;
        const LayerGeo &g0 = cone_geo(L, 0);
        const int w0 = g0.w, PW = g0.PW;
        const uint32_t a0 = smem_u32(act_buf(s, 1));
        const uint32_t PS = m.PS;
        const uint32_t up = F16 ? 0x3C00u : 0x3F80u, dn = F16 ? 0xBC00u : 0xBF80u;
        for (int it = t0; it < n * w0 * w0; it += nthr) {
            const int jrel = it / (w0 * w0), cell = it - jrel * (w0 * w0);
            const int Y = cell / w0 + 1, X = cell - (Y - 1) * w0 + 1;
            const int jj = first + jrel;
            const int bond = m.bond[jj];
            const int bi = bond >> 2, bj = bond_partner(L, bi, bond & 3);
            int y = (int)m.oy[jj] + Y - 1, x = (int)m.ox[jj] + X - 1;
            y -= (y >= L) ? L : 0;
            x -= (x >= L) ? L : 0;
            const int ym = y == 0 ? L - 1 : y - 1, yp = y == L - 1 ? 0 : y + 1;
            const int xl = x == 0 ? L - 1 : x - 1, xr = x == L - 1 ? 0 : x + 1;
            const int rows3[3] = {ym * L, y * L, yp * L};
            const int cols3[3] = {xl, x, xr};
            uint32_t h[9];
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const int site = rows3[ky] + cols3[kx];
                    const int src = site == bi ? bj : (site == bj ? bi : site);
                    h[ky * 3 + kx] = spins[src] > 0 ? up : dn;
                }
            const int q = Y * PW + jj * (w0 + 2) + X;
            const int r = q / P;
            const int i = q - r * P;
            const uint32_t a = a0 + 2u * (uint32_t)i * PS + (uint32_t)(r + 1) * 16u;
            st_shared_v4(a, h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
            st_shared_v4(a + PS, h[8], 0u, 0u, 0u);
        }
    }

    // Cone pass: the ring of the next layer's windows.  After layer l (window
    // side w, origin o = o0 - l) the next window has side w + 2 and origin
    // o - 1; its input grid, w + 4 cells wide with the halo, holds the
    // layer-l outputs at cells 2 .. w + 1 (written by the epilogue) and, in
    // the two outer rows and columns, activations that equal the parent's:
    // those cells lie outside the cone of the exchanged pair.  They are
    // copied asynchronously from the parent store; the caller waits for the
    // copies before it publishes the layer.
    __device__ void ring_fill(int s, int l, int tid)
    {
        const SlabMeta &m = c.slab[s];
        const int L = m.L, N = L * L, count = m.count;
        const LayerGeo &g = lg(s, l);
        const int w = g.w, W4 = w + 4, RWn = lg(s, l + 1).RW;
        const int per = 8 * w + 16;   // ring cells per window
        // one thread per ring cell (consecutive threads: consecutive cells of
        // a ring row, so the parent-store reads coalesce), its CP8 channel
        // planes in turn; divisions by per and W4 (< 2^10, operands < 2^16)
        // as multiply-high
        const uint32_t mper = g.mRing, mW4 = g.mW4;
        const uint32_t out = smem_u32(act_buf(s, l & 1)) + 16u;
        const uint32_t PS = m.PS;
        const uint8_t *lay = p.act_store + (long long)l * CP8 * N * 16;
        for (int it = tid; it < count * per; it += NEPI) {
            const int j = udiv(it, mper);
            int e = it - j * per;
            int Xp, Yp;
            if (e < 4 * W4) {
                // two rows above the window, then two below
                const int r = udiv(e, mW4);
                Xp = e - r * W4;
                Yp = r < 2 ? r : w + r;
            } else {
                // the two columns either side of rows 2 .. w + 1
                e -= 4 * W4;
                Yp = 2 + (e >> 2);
                const int cc = e & 3;
                Xp = cc < 2 ? cc : w + cc;
            }
            int x = (int)m.ox[j] - l - 2 + Xp, y = (int)m.oy[j] - l - 2 + Yp;
            x += (x < 0) ? L : 0; x += (x < 0) ? L : 0; x -= (x >= L) ? L : 0;
            y += (y < 0) ? L : 0; y += (y < 0) ? L : 0; y -= (y >= L) ? L : 0;
            const uint8_t *src = lay + (long long)m.pb[j] * p.store_stride + (long long)(y * L + x) * 16;
            const int Xg = j * W4 + Xp;
            const int qn = Xg / P;
            const uint32_t dst = out + (uint32_t)((Xg - qn * P) * CP8) * PS + (uint32_t)(Yp * RWn + qn) * 16u;
#pragma unroll
            for (int g = 0; g < CP8; ++g) cp_async16(dst + (uint32_t)g * PS, src + (long long)g * N * 16);
        }
    }

    // The configuration stream's next step for meta m (one thread decides):
    // 0 = configurations of the current parent taken into m (c.seg_first,
    // c.seg_n), 1 = a new parent c.new_b of side c.new_L is to be loaded,
    // 2 = stop (the slab is full, no work is left, or the CTA aborts).
    __device__ int next_step(SlabMeta &m, bool first)
    {
        if (first) { m.count = 0; m.L = 0; }
        int act = 2;
        if (c.abort) {
            act = 2;   // stop filling; the next abort check ends the epilogue
        } else if (c.cur_parent >= 0 && c.cur_k <= c.cur_nlist) {
            act = 0;
        } else {
            while (!c.no_more) {
                long long b = c.pending_b;
                c.pending_b = -1;
                if (b < 0) {
                    // next work item; a ragged batch is walked in the
                    // order of `order` (largest lattices first)
                    const long long idx = (long long)atomicAdd(p.counter, 1);
                    if (idx >= p.B) { c.no_more = 1; break; }
                    b = p.order ? p.order[idx] : idx;
                }
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
        if (act == 0) {
            // the slab takes the geometry of the lattice now at the cursor
            // (a new parent, or the rest of the previous fill's parent)
            if (m.count == 0) set_geometry(m, c.cur_L, p.geo[c.cur_L >> 1]);
            if (m.G < 1 || m.G > MAX_SLOTS || m.P != P) {
                c.abort = 1;
                atomicOr(&p.status->flags, VMC_STATUS_INTERNAL);
                m.G = 1;
            }
            const int n_take = min(m.G - m.count, c.cur_nlist + 1 - c.cur_k);
            for (int i = 0; i < n_take; ++i) {
                const int kk = c.cur_k + i;
                const int jj = m.count + i;
                m.parent[jj] = c.cur_parent;
                m.bond[jj] = (kk == 0) ? -1 : (int)list[kk - 1];
                if constexpr (VAR != VAR_PLAIN) m.pb[jj] = (int)c.ring[c.cur_parent].b;
                if constexpr (VAR == VAR_CONE) {
                    // origin of the layer-0 window: one cell up and left of
                    // the pair's top-left site (the down-left pair's
                    // top-left site is its partner's column)
                    const int L = c.cur_L, k2 = m.bond[jj], si = k2 >> 2, t = k2 & 3;
                    const int y = si / L, x = si - y * L;
                    int ox = (t == 3 ? x - 1 : x) - 1, oy = y - 1;
                    ox += (ox < 0) ? L : 0; ox += (ox < 0) ? L : 0;
                    oy += (oy < 0) ? L : 0;
                    m.ox[jj] = (int8_t)ox;
                    m.oy[jj] = (int8_t)oy;
                }
            }
            c.seg_first = m.count;
            c.seg_n = n_take;
            m.count += n_take;
            c.cur_k += n_take;
        }
        return act;
    }

    // A new parent c.new_b: its spins (threads t, t + nthr, ...), then, in
    // the filling group's first warp (`inwarp`), its bond list (or Marshall
    // parity) and, from the group's thread 0, its ring entry.  `sync` is the
    // group's barrier.
    template <class Sync>
    __device__ void load_parent(int t, int nthr, bool inwarp, Sync sync)
    {
        const int Lb = c.new_L;
        const long long b = c.new_b;
        const int8_t *sig = p.sigma + (p.offs ? p.offs[b] : b * (long long)Lb * Lb);
        for (int i = t; i < Lb * Lb; i += nthr) spins[i] = sig[i];
        sync();
        if (inwarp) {
            int a1 = 0, a2 = 0, cnt = 0, par = 0;
            if (p.mode == 1) cnt = build_bond_list_warp(spins, Lb, list, &a1, &a2);
            else par = marshall_parity_warp(spins, Lb);
            __syncwarp();
            if (t == 0) {
                const int r = c.ring_head;
                c.ring_head = (r + 1) % RING;
                Parent &Q = c.ring[r];
                if (*(volatile int *)&Q.valid) { c.abort = 1; atomicOr(&p.status->flags, VMC_STATUS_INTERNAL); }
                Q.b = b;
                Q.diag = (p.mode == 1) ? diag_energy(Lb, a1, a2, p.J1, p.J2) : 0.0;
                Q.la0 = 0.0; Q.acc = 0.0; Q.sg0 = 0;
                Q.nlist = cnt;
                Q.remaining = 1 + cnt;
                Q.mpar = par;
                Q.valid = 1;
                Q.L = Lb;
                c.cur_parent = r;
                c.cur_k = 0;
                c.cur_nlist = cnt;
                c.cur_L = Lb;
                if constexpr (VAR == VAR_CONE) {
                    // the parent's amplitude comes from the parent pass;
                    // only its neighbours enter slabs
                    Q.la0 = p.par_la[b];
                    Q.sg0 = (int)p.par_sg[b];
                    Q.remaining = cnt;
                    c.cur_k = 1;
                    if (cnt == 0 || Q.sg0 == 0 || !isfinite(Q.la0)) {
                        // nothing to evaluate (no exchange neighbour), or a
                        // parent whose E_loc is NaN whatever they give
                        finish_parent(Q);
                        Q.valid = 0;
                        c.cur_parent = -1;
                    }
                }
            }
        }
    }

    // Fill slab s with the next configurations of the stream; returns count.
    // Thread 0 decides each step (next parent, or more neighbours of the
    // current one) and takes configurations into the slab in the same
    // critical section; the other threads build the im2col rows.  The
    // caller's barrier (the end of pool_finish's task phase, or the
    // kernel's start) orders thread 0's first step after every earlier
    // reader of the slab.
    __device__ int fill(int s, int tid)
    {
        SlabMeta &m = c.slab[s];
        bool first = true;
        for (;;) {
            if (tid == 0) c.action = next_step(m, first);
            first = false;
            epi_sync();
            const int act = c.action;
            if (act == 2) break;
            if (act == 1) {
                load_parent(tid, NEPI, tid < 32, [] { epi_sync(); });
                continue;   // thread 0 takes its configurations next; warp 0's list is
                            // complete before thread 0 reads it (same warp, after __syncwarp)
            }
            if constexpr (VAR == VAR_CONE) build_rows_cone(m, s, c.seg_first, c.seg_n, tid, NEPI);
            else build_rows(s, c.seg_first, c.seg_n, tid);
            if (m.count >= m.G) break;
            epi_sync();     // build_rows reads m.bond; thread 0 writes it next
        }
        // cells of no configuration keep whatever the buffer held: they feed
        // only outputs that are dropped
        return m.count;
    }

    // One-slab light-cone pass with an even number of C -> C layers: the
    // weight warp stages every slab fill (configurations, new parents, the
    // embedding layer's im2col into buffer 1, which the last layer reads and
    // the pooling does not use) as soon as the previous slab's last-layer
    // MMAs have completed, so the epilogue only copies the staged descriptor
    // after its pooling.
    __device__ __forceinline__ bool producer_fill() const
    {
        return VAR == VAR_CONE && p.S == 1 && (p.D & 1) == 0;
    }

    // Weight warp (all lanes): the next fill into c.stage, then the staged
    // barrier; returns whether it holds configurations.
    __device__ bool stage_fill(int lane)
    {
        SlabMeta &m = c.stage;
        bool first = true;
        for (;;) {
            int act = 2;
            if (lane == 0) act = next_step(m, first);
            act = __shfl_sync(0xffffffffu, act, 0);
            first = false;
            __syncwarp();
            if (act == 2) break;
            if (act == 1) {
                load_parent(lane, 32, true, [] { __syncwarp(); });
                __syncwarp();
                continue;
            }
            if constexpr (VAR == VAR_CONE) build_rows_cone(m, 0, c.seg_first, c.seg_n, lane, 32);
            __syncwarp();
            if (m.count >= m.G) break;
        }
        const int cnt = m.count;
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&c.staged);
        return cnt > 0;
    }

    // Epilogue: wait for the staged fill and copy its descriptor into slab
    // s; returns its count (0 when the CTA has aborted).
    __device__ int take_stage(int s, int tid, uint32_t &spar, int &nchk)
    {
        if ((tid & 31) == 0) wait_bar(&c.staged, spar, 9);
        __syncwarp();
        spar ^= 1u;
        if (!cta_check(tid, nchk)) {
            if (tid == 0) c.slab[s].count = 0;
            epi_sync();
            return 0;
        }
        constexpr int NW = (int)(sizeof(SlabMeta) / 4);
        static_assert(sizeof(SlabMeta) % 4 == 0, "slab descriptor copied as words");
        for (int i = tid; i < NW; i += NEPI)
            reinterpret_cast<int *>(&c.slab[s])[i] = reinterpret_cast<const int *>(&c.stage)[i];
        epi_sync();
        return c.slab[s].count;
    }

    // End of a (slab, layer) for this warp: make its shared-memory writes
    // visible to the tensor cores and arrive on the slab's ready barrier
    // (one arrival per epilogue warp), so that no warp waits for the others.
    // A warp cannot arrive for layer l + 1 before every warp has arrived for
    // layer l: its tiles of layer l + 1 need MMAs that wait for that phase.
    __device__ void warp_done(int s, int tid)
    {
        fence_proxy_async_smem();
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&c.act_ready[s]);
    }

    // CTA-wide abort check at a barrier: thread 0 snapshots c.abort into
    // okf[parity] before the barrier; the next write to the same entry comes
    // two checks later, after every thread has read it.
    __device__ bool cta_check(int tid, int &nchk)
    {
        const int kk = (nchk++) & 1;
        if (tid == 0) c.okf[kk] = c.abort ? 0 : 1;
        epi_sync();
        return c.okf[kk] != 0;
    }

    // Each warp waits (one lane, bounded) for the accumulator slot of the
    // next tile.  A warp whose wait fails (timeout or abort) keeps going
    // through the tile loops without touching TMEM, so every named barrier
    // still sees all participants; the whole epilogue returns together at
    // the next CTA-wide check (the pooling step of a slab).
    __device__ __forceinline__ bool wait_tile(int slot, uint32_t par, int tid)
    {
        int ok = 0;
        if ((tid & 31) == 0) ok = wait_bar(&c.t_full[slot], par, 7) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok) tc_fence_after();
        return ok != 0;
    }

    // one (slab, layer) of tiles
    template <bool POOL, bool PUB>
    __device__ __forceinline__ void run_tiles(int T, int &slot, uint32_t &use_par, int tid, const TileCtx &k,
                                              float *partF, int *partI)
    {
        for (int t = 0; t < T; ++t) {
            epi_tile<POOL, PUB>(t, slot, tid, k, wait_tile(slot, use_par, tid), partF, partI);
            if (++slot == p.nslots) { slot = 0; use_par ^= 1u; }
        }
    }

    __device__ void epilogue_role(int tid)
    {
        const int D = p.D;
        bool dead[2] = {false, true};
        int slot = 0;
        uint32_t use_par = 0, spar = 0;
        int nchk = 0;
        const bool prod = producer_fill();
        // all layers' biases into shared memory once
        for (int i = tid; i < (D + 1) * C; i += NEPI) bias_s[i] = p.bias32[i];
        epi_sync();
        for (int s = 0; s < p.S; ++s) {
            const int cnt = prod ? take_stage(s, tid, spar, nchk) : fill(s, tid);
            warp_done(s, tid);
            dead[s] = (cnt == 0);
        }
        while (!(dead[0] && dead[1])) {
            for (int l = 0; l <= D; ++l) {
                for (int s = 0; s < 2; ++s) {
                    if (dead[s]) continue;
                    TileCtx k;
                    load_tctx(s, l, tid, k);
                    const int T = k.T;
                    if (l < D) {
                        if constexpr (VAR == VAR_CONE) {
                            if (k.grow) {
                                // the next window's ring is copied from the parent
                                // while the tiles drain; each tile is published as
                                // it is released (no slab-wide hand-off)
                                ring_fill(s, l, tid);
                                run_tiles<false, true>(T, slot, use_par, tid, k, nullptr, nullptr);
                                continue;
                            }
                        }
                        run_tiles<false, false>(T, slot, use_par, tid, k, nullptr, nullptr);
                        warp_done(s, tid);
                    } else {
                        // pooling partials go to the buffer layer D - 1 read (its MMAs are
                        // done); the layer-D input buffer is still read by later tiles
                        float *partF = reinterpret_cast<float *>(act_buf(s, p.D & 1));
                        int *partI = reinterpret_cast<int *>(partF + CP8 * k.NQ);
                        run_tiles<true, false>(T, slot, use_par, tid, k, partF, partI);
                        // every warp's partials are in place; a timed-out or
                        // failed CTA returns here, all warps together
                        if (!cta_check(tid, nchk)) return;
                        pool_finish(s, tid, partF, partI, k.NQ);
                        const int cnt = prod ? take_stage(s, tid, spar, nchk) : fill(s, tid);
                        warp_done(s, tid);
                        dead[s] = (cnt == 0);
                    }
                }
            }
        }
    }
};

template <int C, bool F16, int NM, int VAR>
__global__ void __launch_bounds__(NTHREADS, 1) tc_eloc_kernel(const __grid_constant__ Params p)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    Ctrl &c = *reinterpret_cast<Ctrl *>(smem + 2 * Kern<C, F16, NM, VAR>::WB + (size_t)2 * p.S * p.BUF);
    // spins, bond list and biases follow the control block, each 16-byte
    // aligned (the biases are read as float4)
    int8_t *spins = reinterpret_cast<int8_t *>((reinterpret_cast<uintptr_t>(&c + 1) + 15) & ~(uintptr_t)15);
    uint16_t *list = reinterpret_cast<uint16_t *>(spins + ((p.L_max * p.L_max + 15) & ~15));
    float *bias_s = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(list) + ((8 * p.L_max * p.L_max + 15) & ~15));
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&c.act_ready[i], NEPI_WARPS);   // one arrival per epilogue warp
            mbar_init(&c.w_full[i], 1);
            mbar_init(&c.w_empty[i], NMMA);   // one commit per MMA-issuing warp
        }
        for (int i = 0; i < MAX_TSLOTS; ++i) {
            mbar_init(&c.t_full[i], 1);
            mbar_init(&c.t_empty[i], NEPI_WARPS);   // one arrival per epilogue warp
        }
        for (int i = 0; i < NMMA; ++i) mbar_init(&c.drain[i], 1);
        mbar_init(&c.staged, 1);
        c.abort = 0;
        c.cur_parent = -1; c.cur_k = 0; c.cur_nlist = -1; c.cur_L = 0;
        for (int i = 0; i < 2; ++i) { c.slab[i].count = 0; c.slab[i].L = 0; c.slab[i].G = 0; c.slab[i].g.T = 0; }
        c.pending_b = -1; c.no_more = 0; c.ring_head = 0;
        c.mma_steps = 0; c.mma_done = 0;
        for (int r = 0; r < RING; ++r) c.ring[r].valid = 0;
        mbar_fence_init();
        fence_proxy_async_smem();
    }
    if (warp == MMA_WARP) tmem_alloc(&c.tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // accumulators start from zero: every MMA accumulates, and the epilogue
    // clears each slot it drains
    if (warp < MMA_WARP) {
        const uint32_t ta = c.tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 128);
#pragma unroll
        for (int q = 0; q < 4; ++q) tmem_zero_chunks<4, 32>(ta + 8u * q);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    Kern<C, F16, NM, VAR> k(p, smem, c, spins, list, bias_s, c.tmem_base);
    if (warp < MMA_WARP) k.epilogue_role(tid);
    else if (warp < WGT_WARP) { if ((tid & 31) == 0) k.mma_role(warp - MMA_WARP); }
    else k.weight_role(tid & 31);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == MMA_WARP) {
        __syncwarp();
        tmem_dealloc(c.tmem_base, 512);
    }
}

// ------------------------------------------------------------------ launch

struct Plan {
    int S, P;
    uint32_t BUF;
    int slotc;
    Geo geo[17];
    size_t smem;
    LayerGeo cone[17];          // light-cone pass only
};

template <int C, bool F16, int NM, int VAR>
static int launch_nm(vmc_ctx *ctx, const Plan &pl, const Params &p, cudaStream_t st)
{
    auto kfn = tc_eloc_kernel<C, F16, NM, VAR>;
    // raise the dynamic shared-memory limit once per device and size, so that
    // repeat launches (and graph captures after a first call) issue only the
    // counter reset and the launch
    static int smem_set[64] = {0};
    cudaError_t e = cudaSuccess;
    if (ctx->device < 0 || ctx->device >= 64 || smem_set[ctx->device] < (int)pl.smem) {
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
        if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "cudaFuncSetAttribute(tc_eloc)");
        if (ctx->device >= 0 && ctx->device < 64) smem_set[ctx->device] = (int)pl.smem;
    }
    e = cudaMemsetAsync(ctx->counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "counter reset");
    int grid = ctx->sm_count;
    if ((int64_t)grid > p.B) grid = (int)p.B;
    static const char *names[3] = {"tc_eloc_kernel", "tc_eloc_kernel<parent pass>", "tc_eloc_kernel<light cone>"};
    if (cudaEvent_t ev = vmc_timing_event(ctx, true, names[VAR])) cudaEventRecord(ev, st);
    kfn<<<grid, NTHREADS, pl.smem, st>>>(p);
    if (cudaEvent_t ev = vmc_timing_event(ctx, false, nullptr)) cudaEventRecord(ev, st);
    ctx->launches += 1;
    return vmc_cuda_check(ctx, cudaGetLastError(), "tc_eloc launch");
}

// one kernel per channel count, operand type and lane packing (P C / 32
// accumulator chunks per epilogue thread)
template <int VAR>
static int launch_var(vmc_ctx *ctx, const Plan &pl, const Params &p, cudaStream_t st)
{
    const bool f16 = ctx->arch.precision == VMC_FP16;
    const int C = ctx->arch.channels, nm = pl.P * C / 32;
    if (pl.P * C % 32 != 0 || nm < 1 || nm > 4 || (C != 16 && C != 32))
        return vmc_fail(ctx, VMC_ERR_UNSUPPORTED, "lane packing P=%d with C=%d", pl.P, C);
#define VMC_TC_NM(CC, FF)                                               \
    switch (nm) {                                                       \
        case 1: return launch_nm<CC, FF, 1, VAR>(ctx, pl, p, st);       \
        case 2: return launch_nm<CC, FF, 2, VAR>(ctx, pl, p, st);       \
        case 3: return launch_nm<CC, FF, 3, VAR>(ctx, pl, p, st);       \
        default: return launch_nm<CC, FF, 4, VAR>(ctx, pl, p, st);      \
    }
    if (C == 32) {
        if (f16) { VMC_TC_NM(32, true) } else { VMC_TC_NM(32, false) }
    }
    if (f16) { VMC_TC_NM(16, true) } else { VMC_TC_NM(16, false) }
#undef VMC_TC_NM
}

// light-cone variants, compiled in their own translation unit
int launch_store_var(vmc_ctx *ctx, const Plan &pl, const Params &p, cudaStream_t st);
int launch_cone_var(vmc_ctx *ctx, const Plan &pl, const Params &p, cudaStream_t st);

}  // namespace tc
}  // namespace vmc
