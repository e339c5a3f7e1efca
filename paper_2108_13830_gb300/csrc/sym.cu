// Rotationally symmetrised amplitude (arXiv:2108.13830 Sec. 2.2, Eq. 10;
// Sec. 3.3 applies it in the last fine-tuning stage):
// W~(S) = sum_{i=0..3} W(T^i S), T the 90-degree rotation of the L x L
// lattice, W = (-1)^{M_A} W_CNN.
//
// Every configuration whose W~ is needed is expanded into its four
// rotations in device memory; the batched forward of the context (the
// tensor-core or SIMT log|psi| path, signs included) evaluates them, and a
// combine kernel forms log|W~| and its sign in FP64 after factoring out the
// largest of the four amplitudes.  The local energy expands each sample's
// exchange neighbours (bond order of Sec. 3.1 / Fig. 2c) the same way; the
// log-derivatives weight the four rotations' O rows by W(T^i S) / W~(S).
// Samples are processed in chunks so that the expanded configurations and
// rows stay within a fixed workspace.
#include <algorithm>
#include <cmath>
#include <vector>
#include "vmc_internal.h"
#include "lattice.cuh"

namespace vmc {
namespace sym {

constexpr size_t WS_BUDGET = (size_t)1 << 30;   // bytes of expanded data per chunk

// site of S that T^i S shows at (y, x); T^1 (y, x) <- (x, L - 1 - y)
__device__ __forceinline__ int rot_src(int L, int i, int y, int x)
{
    switch (i) {
        case 0: return y * L + x;
        case 1: return x * L + (L - 1 - y);
        case 2: return (L - 1 - y) * L + (L - 1 - x);
        default: return (L - 1 - x) * L + y;
    }
}

// out[4 b + i] = T^i sigma_b
__global__ void rotate_kernel(const int8_t *__restrict__ sigma, int64_t B, int L, int8_t *__restrict__ out)
{
    const int N = L * L;
    const int64_t total = B * 4 * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / N;
        const int p = (int)(e - row * N);
        const int64_t b = row >> 2;
        const int i = (int)(row & 3);
        out[e] = sigma[b * N + rot_src(L, i, p / L, p % L)];
    }
}

// (log|W~|, sign) of four (log|W|, sign) entries; FP64, the largest factored out
__device__ __forceinline__ void combine4(const double *la, const int8_t *sg, double *out_la, int *out_sg)
{
    double m = -INFINITY;
    for (int i = 0; i < 4; ++i)
        if (sg[i] != 0 && la[i] > m) m = la[i];
    double t = 0.0;
    for (int i = 0; i < 4; ++i)
        if (sg[i] != 0) t += (double)sg[i] * exp(la[i] - m);
    if (t == 0.0 || !(m > -INFINITY)) {
        *out_la = -INFINITY;
        *out_sg = 0;
    } else {
        *out_la = m + log(fabs(t));
        *out_sg = t > 0.0 ? 1 : -1;
    }
}

__global__ void combine_logpsi_kernel(const double *__restrict__ la4, const int8_t *__restrict__ sg4, int64_t B,
                                      double *logabs, int8_t *sign, DevStatus *st)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= B) return;
    double l;
    int s;
    combine4(la4 + 4 * b, sg4 + 4 * b, &l, &s);
    logabs[b] = l;
    sign[b] = (int8_t)s;
    if (l != l || l == INFINITY) {
        atomicOr(&st->flags, VMC_STATUS_NONFINITE);
        atomicAdd(&st->nonfinite, 1ull);
    }
}

// antiparallel J1 + J2 bonds of each sample, and its diagonal energy (Eq. 3)
__global__ void count_kernel(const int8_t *__restrict__ sigma, int64_t B, int L, double J1, double J2,
                             int32_t *cnt, double *diag)
{
    const int lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= B) return;
    const int N = L * L;
    const int8_t *s = sigma + b * N;
    int a1 = 0, a2 = 0;
    for (int k = lane; k < 4 * N; k += 32) {
        const int i = k >> 2, t = k & 3;
        if (s[i] != s[bond_partner(L, i, t)]) {
            if (t < 2) ++a1;
            else ++a2;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (lane == 0) {
        cnt[b] = a1 + a2;
        diag[b] = diag_energy(L, a1, a2, J1, J2);
    }
}

// Expanded configurations of samples [b0, b0 + Bc): rows 4 j + i hold T^i of
// sample b0 + j, rows 4 (Bc + off[j] + q) + i T^i of its q-th exchange
// neighbour (bond order); coef[off[j] + q] is the neighbour's matrix
// element J/2.  One warp per sample.
__global__ void build_kernel(const int8_t *__restrict__ sigma, int64_t b0, int64_t Bc, int L, double J1, double J2,
                             const int64_t *__restrict__ off, int8_t *__restrict__ cfg, double *coef)
{
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= Bc) return;
    const int N = L * L;
    const int8_t *s = sigma + (b0 + j) * N;
    for (int e = lane; e < 4 * N; e += 32) {
        const int i = e / N, p = e - i * N;
        cfg[(4 * j + i) * N + p] = s[rot_src(L, i, p / L, p % L)];
    }
    int64_t q = off[j];
    for (int base = 0; base < 4 * N; base += 32) {
        const int k = base + lane;
        int si = 0, sj = 0;
        bool f = false;
        if (k < 4 * N) {
            si = k >> 2;
            sj = bond_partner(L, si, k & 3);
            f = s[si] != s[sj];
        }
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (f) coef[q + __popc(m & ((1u << lane) - 1u))] = 0.5 * ((k & 3) < 2 ? J1 : J2);
        // the chunk's neighbours one after another, each written by the whole
        // warp: 4 N bytes as N words of four consecutive bytes, lane-strided
        // (coalesced); N = L^2 is a multiple of 4 for even L
        unsigned mm = m;
        for (int idx = 0; mm; ++idx) {
            const int src_lane = __ffs(mm) - 1;
            mm &= mm - 1u;
            const int bi = __shfl_sync(0xffffffffu, si, src_lane), bj = __shfl_sync(0xffffffffu, sj, src_lane);
            uint32_t *dst = reinterpret_cast<uint32_t *>(cfg + 4 * (Bc + q + idx) * N);
            for (int wd = lane; wd < N; wd += 32) {
                uint32_t word = 0;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int e = 4 * wd + t, i = e / N, p = e - i * N;
                    const int src = rot_src(L, i, p / L, p % L);
                    const int8_t v = src == bi ? s[bj] : (src == bj ? s[bi] : s[src]);
                    word |= (uint32_t)(uint8_t)v << (8 * t);
                }
                dst[wd] = word;
            }
        }
        q += __popc(m);
    }
}

// E_loc = diag + sum_q coef_q W~(S'_q) / W~(S), summed in bond order
__global__ void combine_eloc_kernel(const double *__restrict__ la4, const int8_t *__restrict__ sg4, int64_t b0,
                                    int64_t Bc, const int64_t *__restrict__ off, const int32_t *__restrict__ cnt,
                                    const double *__restrict__ diag, const double *__restrict__ coef, double *eloc,
                                    int32_t *n_nbr, DevStatus *st)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= Bc) return;
    double l0;
    int s0;
    combine4(la4 + 4 * j, sg4 + 4 * j, &l0, &s0);
    const int n = cnt[b0 + j];
    double acc = 0.0;
    for (int q = 0; q < n; ++q) {
        const int64_t row = Bc + off[j] + q;
        double l;
        int s;
        combine4(la4 + 4 * row, sg4 + 4 * row, &l, &s);
        if (s != 0) acc += coef[off[j] + q] * (double)(s * s0) * exp(l - l0);
    }
    double e = diag[b0 + j] + acc;
    if (s0 == 0 || !isfinite(l0) || !isfinite(e)) {
        e = NAN;
        atomicOr(&st->flags, VMC_STATUS_NONFINITE);
        atomicAdd(&st->nonfinite, 1ull);
    }
    eloc[b0 + j] = e;
    if (n_nbr) n_nbr[b0 + j] = n;
}

// O[b0 + j][k] = sum_i (W(T^i S) / W~(S)) Orot[4 j + i][k]
template <typename Tin, typename Tout>
__global__ void combine_O_kernel(const Tin *__restrict__ Orot, const double *__restrict__ la4,
                                 const int8_t *__restrict__ sg4, int64_t b0, int64_t Bc, int64_t n, Tout *O)
{
    const int64_t j = blockIdx.y;
    double l;
    int s;
    combine4(la4 + 4 * j, sg4 + 4 * j, &l, &s);
    double w[4];
    for (int i = 0; i < 4; ++i) w[i] = (sg4[4 * j + i] != 0) ? (double)(sg4[4 * j + i] * s) * exp(la4[4 * j + i] - l) : 0.0;
    const Tin *r = Orot + 4 * j * n;
    Tout *o = O + (b0 + j) * n;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        o[k] = (Tout)(w[0] * (double)r[k] + w[1] * (double)r[n + k] + w[2] * (double)r[2 * n + k] + w[3] * (double)r[3 * n + k]);
}

static int forward(vmc_ctx *ctx, const int8_t *cfg, int64_t M, double *la, int8_t *sg, cudaStream_t s)
{
    return vmc_is_tc(ctx->arch.precision) ? vmc_tc_eloc(ctx, 0, cfg, nullptr, nullptr, M, ctx->L, la, sg, nullptr, s)
                                          : vmc_simt_eloc(ctx, 0, cfg, nullptr, nullptr, M, ctx->L, la, sg, nullptr, s);
}

static inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace sym
}  // namespace vmc

using namespace vmc::sym;

int vmc_logpsi_sym_impl(vmc_ctx *ctx, const int8_t *sigma, int64_t B, double *logabs, int8_t *sign, cudaStream_t s)
{
    const int N = ctx->L * ctx->L;
    const int64_t Bc = std::max<int64_t>(1, std::min<int64_t>(B, (int64_t)(WS_BUDGET / (4 * (size_t)(N + 9)))));
    const size_t o_la = up256((size_t)4 * Bc * N), o_sg = o_la + up256((size_t)32 * Bc);
    int rc = vmc_ensure_ws(ctx, &ctx->sym_ws, &ctx->sym_ws_bytes, o_sg + up256((size_t)4 * Bc));
    if (rc) return rc;
    char *w = static_cast<char *>(ctx->sym_ws);
    int8_t *cfg = reinterpret_cast<int8_t *>(w);
    double *la = reinterpret_cast<double *>(w + o_la);
    int8_t *sg = reinterpret_cast<int8_t *>(w + o_sg);
    for (int64_t b0 = 0; b0 < B; b0 += Bc) {
        const int64_t nb = std::min(Bc, B - b0);
        rotate_kernel<<<2 * ctx->sm_count, 256, 0, s>>>(sigma + b0 * N, nb, ctx->L, cfg);
        ctx->launches += 1;
        if ((rc = vmc_cuda_check(ctx, cudaGetLastError(), "rotate"))) return rc;
        if ((rc = forward(ctx, cfg, 4 * nb, la, sg, s))) return rc;
        combine_logpsi_kernel<<<(unsigned)((nb + 127) / 128), 128, 0, s>>>(la, sg, nb, logabs + b0, sign + b0, ctx->status);
        ctx->launches += 1;
        if ((rc = vmc_cuda_check(ctx, cudaGetLastError(), "combine logpsi"))) return rc;
    }
    return VMC_OK;
}

int vmc_local_energy_sym_impl(vmc_ctx *ctx, const int8_t *sigma, int64_t B, double *eloc, int32_t *n_nbr,
                              cudaStream_t s)
{
    const int L = ctx->L, N = L * L;
    // per-sample neighbour counts and diagonal energies
    size_t o_diag = up256((size_t)4 * B), o_off = o_diag + up256((size_t)8 * B);
    int rc = vmc_ensure_ws(ctx, &ctx->sym_cnt, &ctx->sym_cnt_bytes, o_off + up256((size_t)8 * B));
    if (rc) return rc;
    int32_t *cnt = reinterpret_cast<int32_t *>(ctx->sym_cnt);
    double *diag = reinterpret_cast<double *>(static_cast<char *>(ctx->sym_cnt) + o_diag);
    int64_t *off_dev = reinterpret_cast<int64_t *>(static_cast<char *>(ctx->sym_cnt) + o_off);
    count_kernel<<<(unsigned)((B + 7) / 8), 256, 0, s>>>(sigma, B, L, ctx->J1, ctx->J2, cnt, diag);
    ctx->launches += 1;
    if ((rc = vmc_cuda_check(ctx, cudaGetLastError(), "count"))) return rc;
    std::vector<int32_t> hc((size_t)B);
    cudaError_t e = cudaMemcpyAsync(hc.data(), cnt, (size_t)B * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "neighbour counts");
    // chunks of samples whose expanded rows (4 per configuration: N spins,
    // log|psi|, sign) and coefficients fit the budget
    const size_t per_row = 4 * ((size_t)N + 9) + 8;
    const int64_t max_rows = (int64_t)(WS_BUDGET / per_row);
    std::vector<int64_t> hoff((size_t)B);
    int64_t b0 = 0;
    while (b0 < B) {
        int64_t rows = 0, b1 = b0;
        while (b1 < B && (b1 == b0 || rows + 1 + hc[(size_t)b1] <= max_rows)) {
            hoff[(size_t)b1] = rows - (b1 - b0);     // offset among the chunk's neighbours
            rows += 1 + hc[(size_t)b1];
            ++b1;
        }
        const int64_t Bc = b1 - b0, nnb = rows - Bc;
        const size_t o_la = up256((size_t)4 * rows * N), o_sg = o_la + up256((size_t)32 * rows);
        const size_t o_cf = o_sg + up256((size_t)4 * rows);
        if ((rc = vmc_ensure_ws(ctx, &ctx->sym_ws, &ctx->sym_ws_bytes, o_cf + up256((size_t)8 * std::max<int64_t>(nnb, 1)))))
            return rc;
        char *w = static_cast<char *>(ctx->sym_ws);
        int8_t *cfg = reinterpret_cast<int8_t *>(w);
        double *la = reinterpret_cast<double *>(w + o_la);
        int8_t *sg = reinterpret_cast<int8_t *>(w + o_sg);
        double *coef = reinterpret_cast<double *>(w + o_cf);
        e = cudaMemcpyAsync(off_dev, hoff.data() + b0, (size_t)Bc * 8, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "neighbour offsets");
        build_kernel<<<(unsigned)((Bc + 7) / 8), 256, 0, s>>>(sigma, b0, Bc, L, ctx->J1, ctx->J2, off_dev, cfg, coef);
        ctx->launches += 1;
        if ((rc = vmc_cuda_check(ctx, cudaGetLastError(), "build"))) return rc;
        if ((rc = forward(ctx, cfg, 4 * rows, la, sg, s))) return rc;
        combine_eloc_kernel<<<(unsigned)((Bc + 127) / 128), 128, 0, s>>>(la, sg, b0, Bc, off_dev, cnt, diag, coef,
                                                                          eloc, n_nbr, ctx->status);
        ctx->launches += 1;
        if ((rc = vmc_cuda_check(ctx, cudaGetLastError(), "combine eloc"))) return rc;
        // the next chunk's copies and kernels follow in stream order
        b0 = b1;
    }
    return VMC_OK;
}

int vmc_log_derivs_sym_impl(vmc_ctx *ctx, const int8_t *sigma, int64_t B, void *O, int dtype, cudaStream_t s)
{
    const int N = ctx->L * ctx->L;
    const int64_t n = ctx->n;
    const bool f64 = (ctx->arch.precision == VMC_FP64) && dtype == VMC_FP64;
    const size_t esz = f64 ? 8 : 4;
    const int64_t Bc = std::max<int64_t>(1, std::min<int64_t>(B, (int64_t)(WS_BUDGET / (4 * ((size_t)n * esz + N + 9)))));
    const size_t o_la = up256((size_t)4 * Bc * N), o_sg = o_la + up256((size_t)32 * Bc);
    const size_t o_O = o_sg + up256((size_t)4 * Bc);
    int rc = vmc_ensure_ws(ctx, &ctx->sym_ws, &ctx->sym_ws_bytes, o_O + (size_t)4 * Bc * n * esz);
    if (rc) return rc;
    char *w = static_cast<char *>(ctx->sym_ws);
    int8_t *cfg = reinterpret_cast<int8_t *>(w);
    double *la = reinterpret_cast<double *>(w + o_la);
    int8_t *sg = reinterpret_cast<int8_t *>(w + o_sg);
    void *Orot = w + o_O;
    for (int64_t b0 = 0; b0 < B; b0 += Bc) {
        const int64_t nb = std::min(Bc, B - b0);
        rotate_kernel<<<2 * ctx->sm_count, 256, 0, s>>>(sigma + b0 * N, nb, ctx->L, cfg);
        ctx->launches += 1;
        if ((rc = vmc_cuda_check(ctx, cudaGetLastError(), "rotate"))) return rc;
        if ((rc = forward(ctx, cfg, 4 * nb, la, sg, s))) return rc;
        if ((rc = vmc_simt_log_derivs(ctx, cfg, 4 * nb, Orot, f64 ? VMC_FP64 : VMC_FP32, s))) return rc;
        const dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)nb);
        if (f64)
            combine_O_kernel<double, double><<<grid, 256, 0, s>>>(static_cast<const double *>(Orot), la, sg, b0, nb, n,
                                                                 static_cast<double *>(O));
        else if (dtype == VMC_FP64)
            combine_O_kernel<float, double><<<grid, 256, 0, s>>>(static_cast<const float *>(Orot), la, sg, b0, nb, n,
                                                                static_cast<double *>(O));
        else
            combine_O_kernel<float, float><<<grid, 256, 0, s>>>(static_cast<const float *>(Orot), la, sg, b0, nb, n,
                                                               static_cast<float *>(O));
        ctx->launches += 1;
        if ((rc = vmc_cuda_check(ctx, cudaGetLastError(), "combine O"))) return rc;
    }
    return VMC_OK;
}
