// Stochastic Reconfiguration (Eq. 5-7, Sec. 3.2.2): moments, the
// matrix-free covariance product and a conjugate-gradient solve.
//
// O is FP32 [m][n].  Every product and sum over O is carried in
// "double-float" arithmetic -- an unevaluated pair (hi, lo) of FP32 values
// with error-free TwoProduct (FMA) and TwoSum steps (Dekker 1971; Knuth,
// TAOCP vol. 2) -- which keeps FP64-level accuracy while running on the
// FP32 pipes; the vector recurrences of CG are plain FP64.
//
// S v = (1/m) O^T (O v) - Obar (Obar . v) is evaluated as
// (1/m) O^T (t - tbar 1) with t = O v and tbar = (1/m) sum_b t_b, which is
// the same quantity (Obar . v = tbar).
#include <algorithm>
#include <cmath>
#include <vector>
#include "vmc_internal.h"
#include "tc_ptx.cuh"

namespace vmc {

struct DF { float h, l; };

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    e = b - (s - a);
}
// acc += x * (yh + yl), x exact in FP32
__device__ __forceinline__ void df_mac(DF &acc, float x, float yh, float yl)
{
    const float p = x * yh;
    float pe = fmaf(x, yh, -p);
    pe = fmaf(x, yl, pe);
    float s, e;
    two_sum(acc.h, p, s, e);
    e += acc.l + pe;
    fast_two_sum(s, e, acc.h, acc.l);
}
// acc += x
__device__ __forceinline__ void df_add(DF &acc, float x)
{
    float s, e;
    two_sum(acc.h, x, s, e);
    e += acc.l;
    fast_two_sum(s, e, acc.h, acc.l);
}
// a += b
__device__ __forceinline__ void df_add_df(DF &a, const DF &b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    e += a.l + b.l;
    fast_two_sum(s, e, a.h, a.l);
}
__device__ __forceinline__ DF df_shfl_xor(const DF &a, int o)
{
    DF r;
    r.h = __shfl_xor_sync(0xffffffffu, a.h, o);
    r.l = __shfl_xor_sync(0xffffffffu, a.l, o);
    return r;
}
__device__ __forceinline__ void split(double v, float &h, float &l)
{
    h = (float)v;
    l = (float)(v - (double)h);
}

// Deterministic FP64 block sum (blockDim.x a multiple of 32, <= 1024).
__device__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if (lane == 0) sh[32] = r;
    }
    __syncthreads();
    return sh[32];
}

// ---------------------------------------------------------------- moments

// One CTA: mean of a length-m vector, and the centred, scaled pair split
// out[b] = split(scale * (x_b - mean)).
__global__ void center_kernel(const double *__restrict__ x, int64_t m, double scale,
                              double *mean_out, float *oh, float *ol)
{
    __shared__ double sh[33];
    double acc = 0.0;
    for (int64_t b = threadIdx.x; b < m; b += blockDim.x) acc += x[b];
    const double mean = block_sum(acc, sh) / (double)m;
    if (threadIdx.x == 0 && mean_out) *mean_out = mean;
    for (int64_t b = threadIdx.x; b < m; b += blockDim.x) split(scale * (x[b] - mean), oh[b], ol[b]);
}

// Column sums over a chunk of rows: part1 = sum O_bk, part2 = sum O_bk w_b.
// Thread = 4 consecutive columns (VEC) or 1 column.
template <bool VEC, bool TWO>
__global__ void colsum_kernel(const float *__restrict__ O, int64_t m, int64_t n, int64_t rows_per_chunk,
                              const float *__restrict__ wh, const float *__restrict__ wl,
                              double *part1, double *part2)
{
    const int64_t chunk = blockIdx.y;
    const int64_t r0 = chunk * rows_per_chunk;
    const int64_t r1 = min(m, r0 + rows_per_chunk);
    constexpr int V = VEC ? 4 : 1;
    const int64_t c0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * V;
    if (c0 >= n) return;
    DF s1[V], s2[V];
#pragma unroll
    for (int j = 0; j < V; ++j) { s1[j] = DF{0.f, 0.f}; s2[j] = DF{0.f, 0.f}; }
    // several rows' loads in flight per thread
#pragma unroll 4
    for (int64_t b = r0; b < r1; ++b) {
        float o[V];
        if constexpr (VEC) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(O + b * n + c0));
            o[0] = f.x; o[1] = f.y; o[2] = f.z; o[3] = f.w;
        } else {
            o[0] = __ldg(O + b * n + c0);
        }
        const float h = TWO ? wh[b] : 0.f, l = TWO ? wl[b] : 0.f;
#pragma unroll
        for (int j = 0; j < V; ++j) {
            if (part1) df_add(s1[j], o[j]);
            if (TWO) df_mac(s2[j], o[j], h, l);
        }
    }
#pragma unroll
    for (int j = 0; j < V; ++j) {
        if (part1) part1[chunk * n + c0 + j] = (double)s1[j].h + (double)s1[j].l;
        if (TWO) part2[chunk * n + c0 + j] = (double)s2[j].h + (double)s2[j].l;
    }
}

// out[k] = scale * sum_chunks part[c][k] (+ add[k] * add_scale)
__global__ void reduce_chunks_kernel(const double *__restrict__ part, int nchunk, int64_t n, double scale,
                                     const double *__restrict__ add, double add_scale, double *out)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < nchunk; ++c) acc += part[(int64_t)c * n + k];
        acc *= scale;
        if (add) acc += add_scale * add[k];
        out[k] = acc;
    }
}

// ---------------------------------------------------------------- S v

__global__ void split_kernel(const double *__restrict__ v, int64_t n, float *vh, float *vl)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        split(v[k], vh[k], vl[k]);
}

// t_b = sum_k O_bk v_k, one warp per row.
template <bool VEC>
__global__ void rowdot_kernel(const float *__restrict__ O, int64_t m, int64_t n,
                              const float *__restrict__ vh, const float *__restrict__ vl, double *t)
{
    const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= m) return;
    const float *o = O + row * n;
    DF acc{0.f, 0.f};
    if (VEC) {
        const float4 *o4 = reinterpret_cast<const float4 *>(o);
        const float4 *h4 = reinterpret_cast<const float4 *>(vh);
        const float4 *l4 = reinterpret_cast<const float4 *>(vl);
        for (int64_t q = lane; q < n / 4; q += 32) {
            const float4 a = __ldg(o4 + q), h = __ldg(h4 + q), l = __ldg(l4 + q);
            df_mac(acc, a.x, h.x, l.x);
            df_mac(acc, a.y, h.y, l.y);
            df_mac(acc, a.z, h.z, l.z);
            df_mac(acc, a.w, h.w, l.w);
        }
    } else {
        for (int64_t k = lane; k < n; k += 32) df_mac(acc, __ldg(o + k), vh[k], vl[k]);
    }
    for (int off = 16; off > 0; off >>= 1) {
        const DF other = df_shfl_xor(acc, off);
        df_add_df(acc, other);
    }
    if (lane == 0) t[row] = (double)acc.h + (double)acc.l;
}

// t_b = sum_k O_bk v_k for RB consecutive rows per CTA: each thread walks
// column groups of 4, loads the split v once and applies it to the RB rows,
// so v is read from L2 once per RB rows instead of once per row.
template <int RB>
__global__ void __launch_bounds__(256) rowdot_blk_kernel(const float *__restrict__ O, int64_t m, int64_t n,
                                                         const float *__restrict__ vh, const float *__restrict__ vl,
                                                         double *t)
{
    __shared__ float red_h[RB][8], red_l[RB][8];
    const int64_t r0 = blockIdx.x * (int64_t)RB;
    const int nr = (int)min((int64_t)RB, m - r0);
    DF acc[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = DF{0.f, 0.f};
    const float4 *h4 = reinterpret_cast<const float4 *>(vh);
    const float4 *l4 = reinterpret_cast<const float4 *>(vl);
    const int64_t nq = n / 4;
    for (int64_t q = threadIdx.x; q < nq; q += blockDim.x) {
        const float4 h = __ldg(h4 + q), l = __ldg(l4 + q);
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            if (r < nr) {
                const float4 a = __ldg(reinterpret_cast<const float4 *>(O + (r0 + r) * n) + q);
                df_mac(acc[r], a.x, h.x, l.x);
                df_mac(acc[r], a.y, h.y, l.y);
                df_mac(acc[r], a.z, h.z, l.z);
                df_mac(acc[r], a.w, h.w, l.w);
            }
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        DF a = acc[r];
        for (int off = 16; off > 0; off >>= 1) {
            const DF o = df_shfl_xor(a, off);
            df_add_df(a, o);
        }
        if (lane == 0) { red_h[r][w] = a.h; red_l[r][w] = a.l; }
    }
    __syncthreads();
    if (threadIdx.x < RB && (int)threadIdx.x < nr) {
        DF a{0.f, 0.f};
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) df_add_df(a, DF{red_h[threadIdx.x][i], red_l[threadIdx.x][i]});
        t[r0 + threadIdx.x] = (double)a.h + (double)a.l;
    }
}

// ---------------------------------------------------------------- fused S v
//
// u = (1/m) O^T (t - tbar) with t = O v in ONE pass over O.  A cooperative
// launch of nC CTAs; CTA c owns the columns [c W, c W + W) and walks the rows
// in blocks of SV_R, each block's rows streamed by bulk copies into a ring of
// SV_STAGES shared-memory stages.  For block i a CTA forms the dots of its
// column slice with the block's rows (one warp per row), publishes them and
// counts itself in; one block later, once every CTA has counted in, it adds
// the nC partials of each row in a fixed order (the same sum in every CTA),
// centres them with tbar = Obar . v (published the same way at the start),
// and accumulates sum_b O_bk d_b for its columns from the stage still in
// shared memory.  Every element of O is read once from HBM; all products and
// sums are double-float as in the two-pass kernels.  Each wait is bounded by
// a time budget and reports VMC_ERR_TIMEOUT.

constexpr int SV_R = 8;           // rows per block (two warps per row in the dot phase)
constexpr int SV_STAGES = 10;     // shared-memory stages of SV_R rows
constexpr int SV_LAG = 5;         // blocks between publishing a block's dots and using them
constexpr int SV_THREADS = 512;
constexpr int SV_WARPS = SV_THREADS / 32;
constexpr int SV_MAXW = 2 * SV_THREADS;   // columns per CTA: two per thread in the column phase
static_assert(SV_WARPS == 2 * SV_R, "two warps per row");
static_assert(SV_STAGES >= SV_LAG + 2, "the stages hold the lagging blocks plus loads ahead");

struct SvParams {
    const float *O;
    int64_t m, n;
    int W, nblk;
    const float *vh, *vl;      // split v, [n]
    const double *Obar;        // [n]
    double inv_m;
    float2 *part;              // [nblk][nC][SV_R] partial dots
    float2 *bar_part;          // [nC] partial Obar . v
    int *cnt;                  // [nblk + 1] arrivals (block i; tbar last), zero at launch
    double *u;                 // [n]
    DevStatus *status;
    long long budget_ns;
};

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// wait until *p >= target (every CTA counted in), bounded by the budget
__device__ bool wait_count(const int *p, int target, long long budget_ns, DevStatus *st)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (ld_acquire_gpu(p) >= target) return true;
        if ((it & 63u) == 63u) {
            const uint64_t now = global_timer_ns();
            if (t0 == 0) t0 = now;
            else if ((long long)(now - t0) > budget_ns) {
                atomicOr(&st->flags, VMC_STATUS_TIMEOUT);
                st->timeout_site = 40;
                return false;
            }
        }
        __nanosleep(32);
    }
}

__device__ __forceinline__ DF warp_df_sum(DF a)
{
    for (int off = 16; off > 0; off >>= 1) {
        const DF o = df_shfl_xor(a, off);
        df_add_df(a, o);
    }
    return a;
}

__global__ void __launch_bounds__(SV_THREADS, 1) sv_fused_kernel(const __grid_constant__ SvParams q)
{
    extern __shared__ __align__(128) uint8_t sv_smem[];
    __shared__ uint64_t full[SV_STAGES];
    __shared__ float dh[SV_R], dl[SV_R], th[SV_R], tl[SV_R];
    __shared__ float red_h[SV_WARPS], red_l[SV_WARPS];
    __shared__ float tbar_h, tbar_l;
    __shared__ double dsum_s;
    __shared__ int abort_flag, site_dummy;
    const int nC = gridDim.x, c = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int W = q.W;
    const int64_t k0 = (int64_t)c * W;
    const int Wc = (int)min((int64_t)W, q.n - k0);
    float *stage = reinterpret_cast<float *>(sv_smem);
    float *svh = stage + (size_t)SV_STAGES * SV_R * W;
    float *svl = svh + W;
    int issued = 0, consumed = 0;
    auto rows_of = [&](int i) { return (int)min((int64_t)SV_R, q.m - (int64_t)i * SV_R); };
    auto issue = [&](int i) {
        const int s = i % SV_STAGES, rows = rows_of(i);
        const uint32_t bytes = (uint32_t)Wc * 4u;
        mbar_expect_tx(&full[s], bytes * (uint32_t)rows);
        for (int r = 0; r < rows; ++r)
            bulk_g2s(stage + ((size_t)s * SV_R + r) * W, q.O + ((int64_t)i * SV_R + r) * q.n + k0, bytes, &full[s]);
    };
    if (tid == 0) {
        for (int s = 0; s < SV_STAGES; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
        abort_flag = 0;
    }
    for (int k = tid; k < Wc; k += SV_THREADS) { svh[k] = q.vh[k0 + k]; svl[k] = q.vl[k0 + k]; }
    __syncthreads();
    if (tid == 0)
        for (; issued < min(SV_STAGES, q.nblk); ++issued) issue(issued);
    // partial tbar = sum over the slice of Obar_k v_k
    {
        DF a{0.f, 0.f};
        for (int k = tid; k < Wc; k += SV_THREADS) {
            float oh, ol;
            split(q.Obar[k0 + k], oh, ol);
            df_mac(a, oh, svh[k], svl[k]);
            df_add(a, ol * svh[k]);
        }
        a = warp_df_sum(a);
        if (lane == 0) { red_h[warp] = a.h; red_l[warp] = a.l; }
        __syncthreads();
        if (tid == 0) {
            DF b{0.f, 0.f};
            for (int w = 0; w < SV_WARPS; ++w) df_add_df(b, DF{red_h[w], red_l[w]});
            q.bar_part[c] = make_float2(b.h, b.l);
            __threadfence();
            atomicAdd(&q.cnt[q.nblk], 1);
        }
        __syncthreads();
    }
    DF acc0{0.f, 0.f}, acc1{0.f, 0.f};
    DF dsum{0.f, 0.f};   // thread 0: sum_b d_b
    for (int i = 0; i < q.nblk + SV_LAG; ++i) {
        if (i < q.nblk) {
            // dot phase: block i, row warp / 2, half warp % 2 of the slice
            const int s = i % SV_STAGES;
            if (tid == 0) {
                const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((i / SV_STAGES) & 1), &abort_flag, q.budget_ns,
                                                  &q.status->flags, &site_dummy, 41);
                if (!ok) abort_flag = 1;
            }
            __syncthreads();
            if (abort_flag) break;
            consumed = i + 1;
            const int rows = rows_of(i), r = warp >> 1, hf = warp & 1;
            DF a{0.f, 0.f};
            if (r < rows) {
                const float *row = stage + ((size_t)s * SV_R + r) * W;
                for (int k = (hf * 32 + lane) * 4; k < Wc; k += 256) {
                    const float4 o = *reinterpret_cast<const float4 *>(row + k);
                    const float4 h = *reinterpret_cast<const float4 *>(svh + k);
                    const float4 l = *reinterpret_cast<const float4 *>(svl + k);
                    df_mac(a, o.x, h.x, l.x);
                    df_mac(a, o.y, h.y, l.y);
                    df_mac(a, o.z, h.z, l.z);
                    df_mac(a, o.w, h.w, l.w);
                }
                a = warp_df_sum(a);
            }
            if (lane == 0) { red_h[warp] = a.h; red_l[warp] = a.l; }
            __syncthreads();
            if (tid < rows) {
                DF b{red_h[2 * tid], red_l[2 * tid]};
                df_add_df(b, DF{red_h[2 * tid + 1], red_l[2 * tid + 1]});
                q.part[((size_t)i * nC + c) * SV_R + tid] = make_float2(b.h, b.l);
            }
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                atomicAdd(&q.cnt[i], 1);
            }
        }
        const int j = i - SV_LAG;
        if (j >= 0) {
            if (tid == 0) {
                bool ok = wait_count(&q.cnt[j], nC, q.budget_ns, q.status);
                if (ok && j == 0) ok = wait_count(&q.cnt[q.nblk], nC, q.budget_ns, q.status);
                if (!ok) abort_flag = 1;
            }
            __syncthreads();
            if (abort_flag) break;
            const int rows = rows_of(j);
            // row sums of the nC partials (lane-strided, then a fixed shuffle tree)
            if (warp < rows) {
                DF a{0.f, 0.f};
                for (int cc = lane; cc < nC; cc += 32) {
                    const float2 v = __ldcg(q.part + ((size_t)j * nC + cc) * SV_R + warp);
                    df_add_df(a, DF{v.x, v.y});
                }
                a = warp_df_sum(a);
                if (lane == 0) { th[warp] = a.h; tl[warp] = a.l; }
            }
            if (j == 0 && warp == SV_WARPS - 1) {
                DF a{0.f, 0.f};
                for (int cc = lane; cc < nC; cc += 32) {
                    const float2 v = __ldcg(q.bar_part + cc);
                    df_add_df(a, DF{v.x, v.y});
                }
                a = warp_df_sum(a);
                if (lane == 0) { tbar_h = a.h; tbar_l = a.l; }
            }
            __syncthreads();
            if (tid < rows) {
                // d_b = (t_b - tbar) / m, split for the column phase
                DF t{th[tid], tl[tid]};
                df_add_df(t, DF{-tbar_h, -tbar_l});
                split(((double)t.h + (double)t.l) * q.inv_m, dh[tid], dl[tid]);
            }
            __syncthreads();
            // the sum of the d_b used, the same in every CTA (see the end)
            if (tid == 0)
                for (int rr = 0; rr < rows; ++rr) { df_add(dsum, dh[rr]); df_add(dsum, dl[rr]); }
            const float *st = stage + (size_t)(j % SV_STAGES) * SV_R * W;
            for (int rr = 0; rr < rows; ++rr) {
                const float hh = dh[rr], ll = dl[rr];
                if (tid < Wc) df_mac(acc0, st[rr * W + tid], hh, ll);
                if (tid + SV_THREADS < Wc) df_mac(acc1, st[rr * W + tid + SV_THREADS], hh, ll);
            }
            __syncthreads();   // stage j % SV_STAGES is free again
            if (tid == 0 && issued < q.nblk) issue(issued++);
        }
    }
    if (abort_flag) {
        // a wait gave up: drain this CTA's bulk copies (bounded) before exiting
        if (tid == 0) {
            int dummy = 0;
            for (int b = consumed; b < issued; ++b)
                mbar_wait_bounded(&full[b % SV_STAGES], (uint32_t)((b / SV_STAGES) & 1), &dummy, q.budget_ns,
                                  &q.status->flags, &site_dummy, 42);
        }
        __syncthreads();
        return;
    }
    // tbar = Obar . v differs from the mean of the computed t_b by rounding,
    // so sum_b d_b is not exactly 0, and on columns whose mean is large that
    // leftover, times sum_b O_bk = m Obar_k, would dominate the error.
    // Centring the d_b on their own mean instead (what the two-pass kernels
    // do with t) subtracts Obar_k sum_b d_b.
    if (tid == 0) dsum_s = (double)dsum.h + (double)dsum.l;
    __syncthreads();
    const double sd = dsum_s;
    if (tid < Wc) q.u[k0 + tid] = ((double)acc0.h + (double)acc0.l) - q.Obar[k0 + tid] * sd;
    if (tid + SV_THREADS < Wc)
        q.u[k0 + tid + SV_THREADS] = ((double)acc1.h + (double)acc1.l) - q.Obar[k0 + tid + SV_THREADS] * sd;
}

// ---------------------------------------------------------------- CG

// q = u + shift p; partial dot p.q per CTA
__global__ void cg_q_kernel(const double *__restrict__ part, int nchunk, int64_t n, double shift,
                            const double *__restrict__ p, double *q, double *pq_part)
{
    __shared__ double sh[33];
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double u = 0.0;
        for (int c = 0; c < nchunk; ++c) u += part[(int64_t)c * n + k];
        const double qk = u + shift * p[k];
        q[k] = qk;
        acc += p[k] * qk;
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) pq_part[blockIdx.x] = s;
}

__device__ double sum_parts(const double *parts, int np)
{
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += parts[i];
    return s;
}

// alpha = rr / pq; x += alpha p; r -= alpha q; partial r.r
__global__ void cg_update_kernel(const double *__restrict__ pq_part, int np, const double *rr_in,
                                 double *x, double *r, const double *__restrict__ p,
                                 const double *__restrict__ q, int64_t n, double *rr_part)
{
    __shared__ double sh[33];
    const double rr = *rr_in;
    const double pq = sum_parts(pq_part, np);
    const double alpha = (rr == 0.0 || pq == 0.0) ? 0.0 : rr / pq;
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        x[k] += alpha * p[k];
        const double rk = r[k] - alpha * q[k];
        r[k] = rk;
        acc += rk * rk;
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) rr_part[blockIdx.x] = s;
}

// beta = rr_new / rr_old; p = r + beta p; split p; rr_out = rr_new
__global__ void cg_dir_kernel(const double *__restrict__ rr_part, int np, const double *rr_old,
                              double *rr_out, const double *__restrict__ r, double *p, int64_t n,
                              float *ph, float *pl)
{
    const double rn = sum_parts(rr_part, np);
    const double ro = *rr_old;
    const double beta = (ro == 0.0) ? 0.0 : rn / ro;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double pk = r[k] + beta * p[k];
        p[k] = pk;
        split(pk, ph[k], pl[k]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *rr_out = rn;
}

// x = 0, r = p = G, split p, partial G.G
__global__ void cg_init_kernel(const double *__restrict__ G, int64_t n, double *x, double *r, double *p,
                               float *ph, float *pl, double *gg_part)
{
    __shared__ double sh[33];
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double g = G[k];
        x[k] = 0.0; r[k] = g; p[k] = g;
        split(g, ph[k], pl[k]);
        acc += g * g;
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) gg_part[blockIdx.x] = s;
}

__global__ void finalize_scalar_kernel(const double *__restrict__ parts, int np, double *out0, double *out1)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double s = sum_parts(parts, np);
        *out0 = s;
        if (out1) *out1 = s;
    }
}

__global__ void resid_kernel(const double *rr, const double *gg, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = (*gg > 0.0) ? sqrt(*rr / *gg) : 0.0;
}

// ---------------------------------------------------------------- workspace

struct SrWs {
    float *vh, *vl;        // [n]
    float *wh, *wl;        // [m]
    double *t;             // [m]
    double *part1, *part2; // [nchunk][n]
    double *Obar, *G;      // [n]
    double *r, *p, *q;     // [n]
    double *scal;          // scalars: 0 Ebar, 1 tbar, 2 gg, 3..4 rr[2], 5 resid
    double *pq_part, *rr_part, *gg_part;   // [NPART]
    float2 *sv_part, *sv_bar;              // fused S v: [nblk][nC][SV_R], [nC]
    int *sv_cnt;                           // [nblk + 1]
};
constexpr int NPART = 256;

static int64_t nchunks_for(int64_t m) { return m >= 1024 ? 16 : (m >= 64 ? 4 : 1); }

static int sr_workspace(vmc_ctx *ctx, int64_t m, SrWs *w)
{
    const int64_t n = ctx->n, nch = nchunks_for(m);
    const int64_t nblk = (m + SV_R - 1) / SV_R, nC = std::max(ctx->sm_count, 1);
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t off[19], tot = 0;
    size_t sz[] = {n * 4, n * 4, (size_t)m * 4, (size_t)m * 4, (size_t)m * 8, (size_t)nch * n * 8, (size_t)nch * n * 8,
                   (size_t)n * 8, (size_t)n * 8, (size_t)n * 8, (size_t)n * 8, (size_t)n * 8, 64 * 8,
                   NPART * 8, NPART * 8, NPART * 8,
                   (size_t)nblk * nC * SV_R * 8, (size_t)nC * 8, (size_t)(nblk + 1) * 4};
    for (int i = 0; i < 19; ++i) { off[i] = tot; tot += al(sz[i]); }
    int rc = vmc_ensure_ws(ctx, &ctx->sr_ws, &ctx->sr_ws_bytes, tot);
    if (rc) return rc;
    char *b = static_cast<char *>(ctx->sr_ws);
    w->vh = (float *)(b + off[0]); w->vl = (float *)(b + off[1]);
    w->wh = (float *)(b + off[2]); w->wl = (float *)(b + off[3]);
    w->t = (double *)(b + off[4]);
    w->part1 = (double *)(b + off[5]); w->part2 = (double *)(b + off[6]);
    w->Obar = (double *)(b + off[7]); w->G = (double *)(b + off[8]);
    w->r = (double *)(b + off[9]); w->p = (double *)(b + off[10]); w->q = (double *)(b + off[11]);
    w->scal = (double *)(b + off[12]);
    w->pq_part = (double *)(b + off[13]); w->rr_part = (double *)(b + off[14]); w->gg_part = (double *)(b + off[15]);
    w->sv_part = (float2 *)(b + off[16]); w->sv_bar = (float2 *)(b + off[17]); w->sv_cnt = (int *)(b + off[18]);
    return VMC_OK;
}

static bool vec_ok(const float *O, int64_t n) { return (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(O) & 15) == 0); }

// launches the moment kernels; Ebar goes to *Ebar (device)
static void launch_moments(vmc_ctx *ctx, const float *O, const double *E, int64_t m, const SrWs &w,
                           double *Obar, double *Ebar, double *G, cudaStream_t s)
{
    const int64_t n = ctx->n, nch = nchunks_for(m);
    const int64_t rpc = (m + nch - 1) / nch;
    center_kernel<<<1, 1024, 0, s>>>(E, m, 1.0, Ebar, w.wh, w.wl);
    const bool vec = vec_ok(O, n);
    const int V = vec ? 4 : 1;
    dim3 grid((unsigned)((n / V + 127) / 128), (unsigned)nch);
    if (vec) colsum_kernel<true, true><<<grid, 128, 0, s>>>(O, m, n, rpc, w.wh, w.wl, w.part1, w.part2);
    else colsum_kernel<false, true><<<grid, 128, 0, s>>>(O, m, n, rpc, w.wh, w.wl, w.part1, w.part2);
    const int rg = (int)std::min<int64_t>((n + 255) / 256, 4 * ctx->sm_count);
    reduce_chunks_kernel<<<rg, 256, 0, s>>>(w.part1, (int)nch, n, 1.0 / (double)m, nullptr, 0.0, Obar);
    reduce_chunks_kernel<<<rg, 256, 0, s>>>(w.part2, (int)nch, n, 1.0 / (double)m, nullptr, 0.0, G);
    ctx->launches += 4;
}

// Geometry of the fused S v for O [m][n]: CTAs, columns per CTA (a multiple
// of 4, at most two per thread) and dynamic shared memory; false where it
// does not apply (unaligned rows, too many columns per CTA), and the
// two-pass kernels run instead.
struct SvPlan {
    int nC, W, nblk;
    size_t smem;
};

static bool sv_fused_plan(const vmc_ctx *ctx, const float *O, int64_t m, SvPlan *pl)
{
    const int64_t n = ctx->n;
    if (!vec_ok(O, n) || m < 1 || ctx->sm_count < 1) return false;
    int nc = (int)std::min<int64_t>(ctx->sm_count, (n + 127) / 128);
    const int64_t n4 = n / 4;
    const int W = (int)(4 * ((n4 + nc - 1) / nc));
    nc = (int)((n + W - 1) / W);
    if (W > SV_MAXW) return false;
    pl->nC = nc;
    pl->W = W;
    pl->nblk = (int)((m + SV_R - 1) / SV_R);
    pl->smem = (size_t)SV_STAGES * SV_R * W * 4 + 2 * (size_t)W * 4;
    if (pl->smem > 220 * 1024) return false;
    static int smem_set[64] = {0};
    const int dev = ctx->device;
    if (dev < 0 || dev >= 64 || smem_set[dev] < (int)pl->smem) {
        if (cudaFuncSetAttribute(sv_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl->smem) !=
            cudaSuccess)
            return false;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sv_fused_kernel, SV_THREADS, pl->smem) !=
                cudaSuccess || per_sm < 1)
            return false;
        if (dev >= 0 && dev < 64) smem_set[dev] = (int)pl->smem;
    }
    return true;
}

// u = (1/m) O^T (O v - tbar) into w.part2 (one chunk) with v split in
// (vh, vl): a counter reset and one cooperative launch
static int launch_sv_fused(vmc_ctx *ctx, const float *O, int64_t m, const double *Obar, const SrWs &w,
                           const SvPlan &pl, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(w.sv_cnt, 0, (size_t)(pl.nblk + 1) * sizeof(int), s);
    if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "S v counters");
    SvParams q;
    q.O = O; q.m = m; q.n = ctx->n; q.W = pl.W; q.nblk = pl.nblk;
    q.vh = w.vh; q.vl = w.vl; q.Obar = Obar; q.inv_m = 1.0 / (double)m;
    q.part = w.sv_part; q.bar_part = w.sv_bar; q.cnt = w.sv_cnt; q.u = w.part2;
    q.status = ctx->status; q.budget_ns = ctx->wait_budget_ns;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)pl.nC);
    cfg.blockDim = dim3(SV_THREADS);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;   // the CTAs wait on one another
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, sv_fused_kernel, q);
    ctx->launches += 1;
    return vmc_cuda_check(ctx, e, "fused S v launch");
}

// u-partials of S p: rowdot, centre, column dots (p already split into vh/vl)
static void launch_sv_partials(vmc_ctx *ctx, const float *O, int64_t m, const SrWs &w, cudaStream_t s)
{
    const int64_t n = ctx->n, nch = nchunks_for(m);
    const int64_t rpc = (m + nch - 1) / nch;
    const bool vec = vec_ok(O, n);
    const unsigned rows_grid = (unsigned)((m + 7) / 8);
    // one row per block: m blocks spread evenly over the SMs (8 rows per block
    // left a 3.4-block-per-SM wave with a tail; the solve is 14 % faster)
    if (vec) rowdot_blk_kernel<1><<<(unsigned)m, 256, 0, s>>>(O, m, n, w.vh, w.vl, w.t);
    else rowdot_kernel<false><<<rows_grid, 256, 0, s>>>(O, m, n, w.vh, w.vl, w.t);
    center_kernel<<<1, 1024, 0, s>>>(w.t, m, 1.0 / (double)m, w.scal + 1, w.wh, w.wl);
    const int V = vec ? 4 : 1;
    dim3 grid((unsigned)((n / V + 127) / 128), (unsigned)nch);
    if (vec) colsum_kernel<true, true><<<grid, 128, 0, s>>>(O, m, n, rpc, w.wh, w.wl, nullptr, w.part2);
    else colsum_kernel<false, true><<<grid, 128, 0, s>>>(O, m, n, rpc, w.wh, w.wl, nullptr, w.part2);
    ctx->launches += 3;
}

}  // namespace vmc

using namespace vmc;

int vmc_sr_moments_impl(vmc_ctx *ctx, const float *O, const double *E, int64_t m,
                        double *Obar, double *Ebar, double *G, cudaStream_t s)
{
    SrWs w;
    int rc = sr_workspace(ctx, m, &w);
    if (rc) return rc;
    launch_moments(ctx, O, E, m, w, Obar, Ebar, G, s);
    return vmc_cuda_check(ctx, cudaGetLastError(), "sr moments");
}

int vmc_sr_matvec_impl(vmc_ctx *ctx, const float *O, int64_t m, const double *Obar,
                       const double *v, double shift, double *out, cudaStream_t s)
{
    // the two-pass kernels centre t with its own mean (Obar . v equals the
    // mean of t = O v; see the file comment); the fused one uses Obar . v
    SrWs w;
    int rc = sr_workspace(ctx, m, &w);
    if (rc) return rc;
    const int64_t n = ctx->n, nch = nchunks_for(m);
    const int g = (int)std::min<int64_t>((n + 255) / 256, 4 * ctx->sm_count);
    split_kernel<<<g, 256, 0, s>>>(v, n, w.vh, w.vl);
    SvPlan pl;
    int used = (int)nch;
    if (ctx->sr_fused && Obar && sv_fused_plan(ctx, O, m, &pl)) {
        rc = launch_sv_fused(ctx, O, m, Obar, w, pl, s);
        if (rc) return rc;
        used = 1;
    } else {
        launch_sv_partials(ctx, O, m, w, s);
    }
    reduce_chunks_kernel<<<g, 256, 0, s>>>(w.part2, used, n, 1.0, v, shift, out);
    ctx->launches += 2;
    return vmc_cuda_check(ctx, cudaGetLastError(), "sr matvec");
}

// scale-split kernel: (wh, wl) = split(w_b) with no centring
__global__ void split_scaled_kernel(const double *__restrict__ w, int64_t m, float *wh, float *wl)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m; b += (int64_t)gridDim.x * blockDim.x)
        split(w[b], wh[b], wl[b]);
}

int vmc_ot_vec_impl(vmc_ctx *ctx, const float *O, int64_t m, const double *wv, double *out, cudaStream_t s)
{
    SrWs w;
    int rc = sr_workspace(ctx, m, &w);
    if (rc) return rc;
    const int64_t n = ctx->n, nch = nchunks_for(m);
    const int64_t rpc = (m + nch - 1) / nch;
    split_scaled_kernel<<<(unsigned)std::min<int64_t>((m + 255) / 256, 1024), 256, 0, s>>>(wv, m, w.wh, w.wl);
    const bool vec = vec_ok(O, n);
    const int V = vec ? 4 : 1;
    dim3 grid((unsigned)((n / V + 127) / 128), (unsigned)nch);
    if (vec) colsum_kernel<true, true><<<grid, 128, 0, s>>>(O, m, n, rpc, w.wh, w.wl, nullptr, w.part2);
    else colsum_kernel<false, true><<<grid, 128, 0, s>>>(O, m, n, rpc, w.wh, w.wl, nullptr, w.part2);
    const int g = (int)std::min<int64_t>((n + 255) / 256, 4 * ctx->sm_count);
    reduce_chunks_kernel<<<g, 256, 0, s>>>(w.part2, (int)nch, n, 1.0, nullptr, 0.0, out);
    ctx->launches += 3;
    return vmc_cuda_check(ctx, cudaGetLastError(), "ot_vec");
}

static void record_cg(vmc_ctx *ctx, const float *O, int64_t m, double shift, int iters, double *x,
                      const SrWs &w, cudaStream_t s)
{
    const int64_t n = ctx->n, nch = nchunks_for(m);
    const int np = (int)std::min<int64_t>((n + 255) / 256, NPART);
    double *rr0 = w.scal + 3, *rr1 = w.scal + 4, *gg = w.scal + 2;
    cg_init_kernel<<<np, 256, 0, s>>>(w.G, n, x, w.r, w.p, w.vh, w.vl, w.gg_part);
    finalize_scalar_kernel<<<1, 32, 0, s>>>(w.gg_part, np, gg, rr0);
    ctx->launches += 2;
    SvPlan pl;
    const bool fused = ctx->sr_fused && sv_fused_plan(ctx, O, m, &pl);
    for (int it = 0; it < iters; ++it) {
        double *rr_old = (it & 1) ? rr1 : rr0;
        double *rr_new = (it & 1) ? rr0 : rr1;
        if (fused) launch_sv_fused(ctx, O, m, w.Obar, w, pl, s);
        else launch_sv_partials(ctx, O, m, w, s);
        cg_q_kernel<<<np, 256, 0, s>>>(w.part2, fused ? 1 : (int)nch, n, shift, w.p, w.q, w.pq_part);
        cg_update_kernel<<<np, 256, 0, s>>>(w.pq_part, np, rr_old, x, w.r, w.p, w.q, n, w.rr_part);
        cg_dir_kernel<<<np, 256, 0, s>>>(w.rr_part, np, rr_old, rr_new, w.r, w.p, n, w.vh, w.vl);
        ctx->launches += 3;
    }
    resid_kernel<<<1, 32, 0, s>>>((iters & 1) ? rr1 : rr0, gg, w.scal + 5);
    ctx->launches += 1;
}

int vmc_sr_solve_impl(vmc_ctx *ctx, const float *O, const double *E, int64_t m, double shift,
                      int iters, double *x, double *resid_out, cudaStream_t s)
{
    SrWs w;
    int rc = sr_workspace(ctx, m, &w);
    if (rc) return rc;
    launch_moments(ctx, O, E, m, w, w.Obar, w.scal + 0, w.G, s);
    rc = vmc_cuda_check(ctx, cudaGetLastError(), "sr moments");
    if (rc) return rc;
    const bool same = ctx->cg_exec && ctx->cg_key_ws == ctx->sr_ws && ctx->cg_key_O == O && ctx->cg_key_m == m && ctx->cg_key_iters == iters &&
                      ctx->cg_key_shift == shift && ctx->cg_key_x == x && ctx->cg_key_fused == ctx->sr_fused;
    if (!same) {
        if (ctx->cg_exec) { cudaGraphExecDestroy(ctx->cg_exec); ctx->cg_exec = nullptr; }
        cudaStream_t cap;
        rc = vmc_cuda_check(ctx, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
        if (rc) return rc;
        cudaGraph_t g;
        const int64_t saved = ctx->launches;
        rc = vmc_cuda_check(ctx, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        if (rc) { cudaStreamDestroy(cap); return rc; }
        record_cg(ctx, O, m, shift, iters, x, w, cap);
        cudaError_t e = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "end capture");
        e = cudaGraphInstantiate(&ctx->cg_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { ctx->cg_exec = nullptr; return vmc_cuda_check(ctx, e, "graph instantiate"); }
        ctx->cg_key_O = O; ctx->cg_key_m = m; ctx->cg_key_iters = iters; ctx->cg_key_shift = shift; ctx->cg_key_x = x;
        ctx->cg_key_ws = ctx->sr_ws;
        ctx->cg_key_fused = ctx->sr_fused;
        ctx->cg_launches = ctx->launches - saved;
        ctx->launches = saved;
    }
    rc = vmc_cuda_check(ctx, cudaGraphLaunch(ctx->cg_exec, s), "graph launch");
    if (rc) return rc;
    ctx->launches += ctx->cg_launches;
    if (resid_out) {
        rc = vmc_cuda_check(ctx, cudaMemcpyAsync(resid_out, w.scal + 5, sizeof(double), cudaMemcpyDeviceToHost, s), "resid copy");
        if (rc) return rc;
        rc = vmc_cuda_check(ctx, cudaStreamSynchronize(s), "sync");
        if (rc) return rc;
    }
    return VMC_OK;
}

// ---------------------------------------------------------------- sample-space solve
//
// (S + shift I) x = G solved exactly in the m-dimensional sample space
// (Woodbury): with Oc = O - 1 Obar^T (the centred rows) and S = Oc^T Oc / m,
//     x = (G - Oc^T y) / shift,   (m shift I + Oc Oc^T) y = Oc G.
// The m x m Gram matrix K = Oc Oc^T is formed from the centred rows held as
// double-float pairs (one exact subtraction per element), K + m shift I is
// factored by a blocked FP64 Cholesky, and the two triangular solves and
// the two passes over O (Oc G, Oc^T y) complete the solve.  Sec. 3.2.2 does
// the same solve with a dense n x n Cholesky; for m << n the m x m system
// is the cheaper exact route.

namespace vmc {
namespace dense {

constexpr int TB = 64;        // Gram tile (TB x TB outputs per CTA, 256 threads of 4 x 4)
constexpr int TK = 16;        // columns per shared-memory stage
constexpr int NB = 32;        // Cholesky block

// Oc[b][k] = O[b][k] - Obar[k] as a double-float pair: the difference of the
// float O and the high part of Obar is exact (TwoSum), then the low part of
// Obar is taken off
__global__ void center_rows_kernel(const float *__restrict__ O, int64_t m, int64_t n, const double *__restrict__ Obar,
                                   float2 *__restrict__ Oc)
{
    const int64_t tot = m * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e % n;
        float oh, ol;
        split(Obar[k], oh, ol);
        float s, err;
        two_sum(O[e], -oh, s, err);
        err -= ol;
        float h, l;
        fast_two_sum(s, err, h, l);
        Oc[e] = make_float2(h, l);
    }
}

// K[a][b] = sum_k Oc[a][k] Oc[b][k] (+ diag on a = b) for the lower
// triangle, tile by tile: (ah + al)(bh + bl) with ah bh exact by FMA, the
// cross terms and the running sum's rounding collected in the low word.
__global__ void __launch_bounds__(256) gram_df_kernel(const float2 *__restrict__ Oc, int64_t m, int64_t n, double diag,
                                                      double *__restrict__ K)
{
    // tile (I, J), I >= J, from the linear block index
    const int64_t t = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    while (I * (I + 1) / 2 > t) --I;
    const int64_t J = t - I * (I + 1) / 2;
    __shared__ float2 As[2][TK][TB], Bs[2][TK][TB];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t a0 = I * TB, b0 = J * TB;
    float ah[4][4], al[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { ah[i][j] = 0.f; al[i][j] = 0.f; }
    // each thread stages 4 elements of each tile per chunk: row tid / 4, columns 4 (tid % 4) ..
    auto load = [&](int buf, int64_t k0) {
        const int r = tid >> 2, c0 = (tid & 3) * 4;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t k = k0 + c0 + q;
            const int64_t ra = a0 + r, rb = b0 + r;
            As[buf][c0 + q][r] = (ra < m && k < n) ? Oc[ra * n + k] : make_float2(0.f, 0.f);
            Bs[buf][c0 + q][r] = (rb < m && k < n) ? Oc[rb * n + k] : make_float2(0.f, 0.f);
        }
    };
    load(0, 0);
    __syncthreads();
    int buf = 0;
    for (int64_t k0 = 0; k0 < n; k0 += TK) {
        if (k0 + TK < n) load(buf ^ 1, k0 + TK);
#pragma unroll 4
        for (int kk = 0; kk < TK; ++kk) {
            float2 av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[buf][kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[buf][kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float p = av[i].x * bv[j].x;
                    float pe = fmaf(av[i].x, bv[j].x, -p);
                    pe = fmaf(av[i].x, bv[j].y, pe);
                    pe = fmaf(av[i].y, bv[j].x, pe);
                    float s, e;
                    two_sum(ah[i][j], p, s, e);
                    ah[i][j] = s;
                    al[i][j] += e + pe;
                }
        }
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t a = a0 + ty * 4 + i, b = b0 + tx * 4 + j;
            if (a < m && b < m && b <= a) K[a * m + b] = (double)ah[i][j] + (double)al[i][j] + (a == b ? diag : 0.0);
        }
}

// Cholesky of the NB x NB diagonal block k (lower, in place); a pivot that
// is not positive makes the factor NaN and raises VMC_STATUS_NONFINITE
__global__ void potrf_diag_kernel(double *K, int64_t m, int k, DevStatus *st)
{
    __shared__ double Ls[NB][NB + 1];
    const int i = threadIdx.x;   // row of the block
    const int64_t base = (int64_t)k * NB;
    const int nb = (int)min((int64_t)NB, m - base);
    if (i < nb)
        for (int j = 0; j <= i; ++j) Ls[i][j] = K[(base + i) * m + base + j];
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (i == j) {
            double d = Ls[j][j];
            for (int t = 0; t < j; ++t) d -= Ls[j][t] * Ls[j][t];
            if (!(d > 0.0)) {
                atomicOr(&st->flags, VMC_STATUS_NONFINITE);
                d = __longlong_as_double(0x7ff8000000000000LL);
            }
            Ls[j][j] = sqrt(d);
        }
        __syncthreads();
        if (i > j && i < nb) {
            double v = Ls[i][j];
            for (int t = 0; t < j; ++t) v -= Ls[i][t] * Ls[j][t];
            Ls[i][j] = v / Ls[j][j];
        }
        __syncthreads();
    }
    if (i < nb)
        for (int j = 0; j <= i; ++j) K[(base + i) * m + base + j] = Ls[i][j];
}

// panel below block k: row r solves x L_kk^T = K[r][block k] by forward substitution
__global__ void trsm_panel_kernel(double *K, int64_t m, int k)
{
    __shared__ double Ls[NB][NB + 1];
    const int64_t base = (int64_t)k * NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, j = e % NB;
        Ls[i][j] = (j <= i) ? K[(base + i) * m + base + j] : 0.0;
    }
    __syncthreads();
    const int64_t r = base + NB + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= m) return;
    double x[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) x[j] = K[r * m + base + j];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        double v = x[j];
        for (int t = 0; t < j; ++t) v -= x[t] * Ls[j][t];
        x[j] = v / Ls[j][j];
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) K[r * m + base + j] = x[j];
}

// trailing update of the lower triangle: K[i][j] -= sum_t P[i][t] P[j][t]
// over the panel columns of block k, for i >= j >= (k + 1) NB; 32 x 32 tiles
__global__ void __launch_bounds__(256) syrk_update_kernel(double *K, int64_t m, int k)
{
    const int64_t off = (int64_t)(k + 1) * NB;
    const int64_t t = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    while (I * (I + 1) / 2 > t) --I;
    const int64_t J = t - I * (I + 1) / 2;
    __shared__ double Pi[NB][NB + 1], Pj[NB][NB + 1];
    const int64_t i0 = off + I * 32, j0 = off + J * 32, pc = (int64_t)k * NB;
    for (int e = threadIdx.x; e < 32 * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        Pi[r][c] = (i0 + r < m) ? K[(i0 + r) * m + pc + c] : 0.0;
        Pj[r][c] = (j0 + r < m) ? K[(j0 + r) * m + pc + c] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 row groups of 4
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = ty * 4 + q;
        const int64_t i = i0 + r, j = j0 + tx;
        if (i >= m || j >= m || j > i) continue;
        double acc = 0.0;
#pragma unroll 8
        for (int c = 0; c < NB; ++c) acc += Pi[r][c] * Pj[tx][c];
        K[i * m + j] -= acc;
    }
}

// L w = z then L^T y = w, one CTA, column by column (L lower, row-major)
__global__ void __launch_bounds__(1024) chol_solve_kernel(const double *__restrict__ L, int64_t m, double *z)
{
    __shared__ double piv;
    for (int64_t i = 0; i < m; ++i) {
        if (threadIdx.x == 0) { z[i] /= L[i * m + i]; piv = z[i]; }
        __syncthreads();
        const double w = piv;
        for (int64_t j = i + 1 + threadIdx.x; j < m; j += blockDim.x) z[j] -= L[j * m + i] * w;
        __syncthreads();
    }
    for (int64_t i = m - 1; i >= 0; --i) {
        if (threadIdx.x == 0) { z[i] /= L[i * m + i]; piv = z[i]; }
        __syncthreads();
        const double y = piv;
        for (int64_t j = threadIdx.x; j < i; j += blockDim.x) z[j] -= L[i * m + j] * y;
        __syncthreads();
    }
}

// z[b] = hi[b] + lo[b] (a double from its split)
__global__ void join_kernel(const float *__restrict__ hi, const float *__restrict__ lo, int64_t m, double *z)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m; b += (int64_t)gridDim.x * blockDim.x)
        z[b] = (double)hi[b] + (double)lo[b];
}

// x = (b - sum_chunks u) / shift, or x += that when accumulate
__global__ void finish_x_kernel(const double *__restrict__ part, int nchunk, int64_t n, const double *__restrict__ b,
                                double inv_shift, double *x, int accumulate)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double u = 0.0;
        for (int c = 0; c < nchunk; ++c) u += part[(int64_t)c * n + k];
        const double d = (b[k] - u) * inv_shift;
        x[k] = accumulate ? x[k] + d : d;
    }
}

// r = G - q
__global__ void sub_kernel(const double *__restrict__ G, const double *__restrict__ q, int64_t n, double *r)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        r[k] = G[k] - q[k];
}

}  // namespace dense
}  // namespace vmc

int vmc_sr_solve_dense_impl(vmc_ctx *ctx, const float *O, const double *E, int64_t m, double shift, double *x,
                            double *resid_out, cudaStream_t s)
{
    using namespace vmc::dense;
    SrWs w;
    int rc = sr_workspace(ctx, m, &w);
    if (rc) return rc;
    const int64_t n = ctx->n, nch = nchunks_for(m);
    const int64_t rpc = (m + nch - 1) / nch;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t need = al((size_t)m * n * sizeof(float2)) + al((size_t)m * m * sizeof(double)) + al((size_t)m * 8);
    rc = vmc_ensure_ws(ctx, &ctx->dense_ws, &ctx->dense_ws_bytes, need);
    if (rc) return rc;
    char *base = static_cast<char *>(ctx->dense_ws);
    float2 *Oc = reinterpret_cast<float2 *>(base);
    double *K = reinterpret_cast<double *>(base + al((size_t)m * n * sizeof(float2)));
    double *z = reinterpret_cast<double *>(reinterpret_cast<char *>(K) + al((size_t)m * m * sizeof(double)));
    // moments: Obar, Ebar, G
    launch_moments(ctx, O, E, m, w, w.Obar, w.scal + 0, w.G, s);
    const int g = (int)std::min<int64_t>((n + 255) / 256, 4 * ctx->sm_count);
    (void)rpc;
    // K = Oc Oc^T + m shift I (lower triangle), then its Cholesky factor in place
    center_rows_kernel<<<8 * ctx->sm_count, 256, 0, s>>>(O, m, n, w.Obar, Oc);
    const int64_t nt = (m + TB - 1) / TB;
    gram_df_kernel<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(Oc, m, n, (double)m * shift, K);
    ctx->launches += 2;
    const int nblk = (int)((m + NB - 1) / NB);
    for (int k = 0; k < nblk; ++k) {
        potrf_diag_kernel<<<1, NB, 0, s>>>(K, m, k, ctx->status);
        ctx->launches += 1;
        const int64_t below = m - (int64_t)(k + 1) * NB;
        if (below > 0) {
            trsm_panel_kernel<<<(unsigned)((below + 127) / 128), 128, 0, s>>>(K, m, k);
            const int64_t tt = (below + 31) / 32;
            syrk_update_kernel<<<(unsigned)(tt * (tt + 1) / 2), 256, 0, s>>>(K, m, k);
            ctx->launches += 2;
        }
    }
    // W b = (b - Oc^T y) / shift with (m shift I + K) y = Oc b, the exact
    // inverse of S + shift I applied to b (accumulated into x when acc)
    const bool vec = vec_ok(O, n);
    const int V = vec ? 4 : 1;
    auto apply = [&](const double *b, int acc) {
        // z = Oc b (the rows' dots with b, centred on their mean)
        split_kernel<<<g, 256, 0, s>>>(b, n, w.vh, w.vl);
        const unsigned rows_grid = (unsigned)((m + 7) / 8);
        if (vec) rowdot_blk_kernel<1><<<(unsigned)m, 256, 0, s>>>(O, m, n, w.vh, w.vl, w.t);
        else rowdot_kernel<false><<<rows_grid, 256, 0, s>>>(O, m, n, w.vh, w.vl, w.t);
        center_kernel<<<1, 1024, 0, s>>>(w.t, m, 1.0, w.scal + 1, w.wh, w.wl);
        join_kernel<<<(unsigned)std::min<int64_t>((m + 255) / 256, 1024), 256, 0, s>>>(w.wh, w.wl, m, z);
        chol_solve_kernel<<<1, 1024, 0, s>>>(K, m, z);
        // Oc^T y = O^T (y - mean y)
        center_kernel<<<1, 1024, 0, s>>>(z, m, 1.0, w.scal + 1, w.wh, w.wl);
        dim3 grid((unsigned)((n / V + 127) / 128), (unsigned)nch);
        if (vec) colsum_kernel<true, true><<<grid, 128, 0, s>>>(O, m, n, rpc, w.wh, w.wl, nullptr, w.part2);
        else colsum_kernel<false, true><<<grid, 128, 0, s>>>(O, m, n, rpc, w.wh, w.wl, nullptr, w.part2);
        finish_x_kernel<<<g, 256, 0, s>>>(w.part2, (int)nch, n, b, 1.0 / shift, x, acc);
        ctx->launches += 8;
    };
    apply(w.G, 0);
    // The formula divides G - Oc^T y by the shift, so its rounding is
    // amplified by the condition of S + shift I (residuals ~1e-5 at shift
    // 1e-4 on these matrices).  Iterative refinement with the double-float
    // covariance product removes that: r = G - (S + shift I) x, x += W r.
    for (int it = 0; it < ctx->dense_refine; ++it) {
        rc = vmc_sr_matvec_impl(ctx, O, m, w.Obar, x, shift, w.q, s);
        if (rc) return rc;
        sub_kernel<<<g, 256, 0, s>>>(w.G, w.q, n, w.r);
        ctx->launches += 1;
        apply(w.r, 1);
    }
    rc = vmc_cuda_check(ctx, cudaGetLastError(), "dense SR solve");
    if (rc || !resid_out) return rc;
    // ||G - (S + shift I) x|| / ||G|| with one more covariance product
    rc = vmc_sr_matvec_impl(ctx, O, m, w.Obar, x, shift, w.q, s);
    if (rc) return rc;
    std::vector<double> hq(n), hg(n);
    rc = vmc_cuda_check(ctx, cudaMemcpyAsync(hq.data(), w.q, n * 8, cudaMemcpyDeviceToHost, s), "resid copy");
    if (!rc) rc = vmc_cuda_check(ctx, cudaMemcpyAsync(hg.data(), w.G, n * 8, cudaMemcpyDeviceToHost, s), "resid copy");
    if (!rc) rc = vmc_cuda_check(ctx, cudaStreamSynchronize(s), "sync");
    if (rc) return rc;
    double rr = 0, gg = 0;
    for (int64_t k = 0; k < n; ++k) { rr += (hg[k] - hq[k]) * (hg[k] - hq[k]); gg += hg[k] * hg[k]; }
    *resid_out = gg > 0 ? sqrt(rr / gg) : 0.0;
    return VMC_OK;
}
