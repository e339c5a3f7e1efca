// Per-sample log-derivatives O_bk = d log|psi(sigma_b)| / d theta_k (Eq. 5).
//
// Persistent CTAs; each takes samples b = blockIdx.x, + gridDim.x, ...  For
// a sample the CTA recomputes the forward pass, keeping the pre-activations
// z_l of every layer in its own global scratch slot ((D+1) C N values per
// resident CTA -- bounded by the grid, not by the batch), then runs reverse
// mode:
//   g_D = d log|psi| / d z_D = 1 / z_D                     (product pooling)
//   dW_l[co][ci][ky][kx] = sum_p g_l[co][p] a_{l-1}[ci][p + (ky-1, kx-1)]
//   db_l[co]             = sum_p g_l[co][p]
//   g_{l-1} = (W_l^T * g_l) SiLU'(z_{l-1}),
// where W_l^T * g is the 3x3 circular convolution of g with the flipped,
// transposed kernel W'[ci][co][ky][kx] = W[co][ci][2-ky][2-kx].
#include "vmc_internal.h"
#include "lattice.cuh"
#include "simt_common.cuh"

namespace vmc {

struct BwdParams {
    int L, C, D;
    int64_t B, n;
    const int8_t *sigma;
    const void *W, *WT, *bias;
    void *scratch;       // [gridDim][(D+1)][C][N]
    void *O;             // [B][n]
};

template <typename T>
struct StoreZSilu {
    T *zg;               // global z of this layer, [C][N]
    T *out;              // shared padded planes (nullptr for the last layer)
    int PP, LP, L;
    template <int CO>
    __device__ __forceinline__ void operator()(int, int, int c0, int y, int x0, T (&acc)[CO][2]) const
    {
#pragma unroll
        for (int co = 0; co < CO; ++co)
#pragma unroll
            for (int px = 0; px < 2; ++px) {
                const T z = acc[co][px];
                zg[(c0 + co) * L * L + y * L + x0 + px] = z;
                if (out) out[(c0 + co) * PP + (y + 1) * LP + x0 + px + 1] = silu_f(z);
            }
    }
};

template <typename T>
struct StoreGradSilu {
    T *out;              // shared padded planes
    const T *zprev;      // global z_{l-1}, [C][N]
    int PP, LP, L;
    template <int CO>
    __device__ __forceinline__ void operator()(int, int, int c0, int y, int x0, T (&acc)[CO][2]) const
    {
#pragma unroll
        for (int co = 0; co < CO; ++co)
#pragma unroll
            for (int px = 0; px < 2; ++px) {
                const T z = zprev[(c0 + co) * L * L + y * L + x0 + px];
                const T sg = T(1) / (T(1) + (sizeof(T) == 4 ? (T)expf(-(float)z) : (T)exp(-(double)z)));
                out[(c0 + co) * PP + (y + 1) * LP + x0 + px + 1] = acc[co][px] * sg * (T(1) + z * (T(1) - sg));
            }
    }
};

// 512 threads: one CTA per SM fits (two C-channel planes of shared memory),
// and the per-sample work is latency-bound at fewer warps
constexpr int BWD_THREADS = 512;

template <typename T, int CO, typename OutT>
__global__ void __launch_bounds__(BWD_THREADS) simt_bwd_kernel(BwdParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int8_t *s = reinterpret_cast<int8_t *>(smem);
    const int L = p.L, C = p.C, D = p.D, N = L * L, LP = L + 2;
    const int PP = plane_pitch(L);
    T *gbuf = reinterpret_cast<T *>(smem + 1024);
    T *ibuf = gbuf + (size_t)C * PP;
    T *zs = static_cast<T *>(p.scratch) + (size_t)blockIdx.x * (D + 1) * C * N;
    const T *W = static_cast<const T *>(p.W);
    const T *WT = static_cast<const T *>(p.WT);
    const T *bias = static_cast<const T *>(p.bias);

    for (int64_t b = blockIdx.x; b < p.B; b += gridDim.x) {
        const int8_t *sig = p.sigma + b * N;
        OutT *Ob = static_cast<OutT *>(p.O) + b * p.n;
        for (int i = threadIdx.x; i < N; i += blockDim.x) s[i] = sig[i];
        __syncthreads();
        // forward, keeping z_l of every layer
        for (int c = threadIdx.x; c < LP * LP; c += blockDim.x) {
            const int Y = c / LP, X = c - Y * LP;
            ibuf[c] = (T)s[(wrap_pad(Y, L) - 1) * L + wrap_pad(X, L) - 1];
        }
        __syncthreads();
        T *cur = ibuf, *nxt = gbuf;
        for (int l = 0; l <= D; ++l) {
            const int cin = (l == 0) ? 1 : C;
            conv_layer<T, CO>(cur, C * PP, cin, W + simt_w_offset(C, l), bias + l * C, C, L, PP, 1,
                              StoreZSilu<T>{zs + (size_t)l * C * N, l < D ? nxt : nullptr, PP, LP, L});
            __syncthreads();
            if (l < D) {
                halo_fill(nxt, C, L, PP);
                __syncthreads();
                T *t = cur; cur = nxt; nxt = t;
            }
        }
        // g_D = 1 / z_D
        const T *zD = zs + (size_t)D * C * N;
        for (int i = threadIdx.x; i < C * N; i += blockDim.x) {
            const int c = i / N, q = i - c * N, y = q / L, x = q - y * L;
            gbuf[c * PP + (y + 1) * LP + x + 1] = T(1) / zD[i];
        }
        __syncthreads();
        halo_fill(gbuf, C, L, PP);
        __syncthreads();
        for (int l = D; l >= 0; --l) {
            const int cin = (l == 0) ? 1 : C;
            // input activations of layer l
            if (l == 0) {
                for (int c = threadIdx.x; c < LP * LP; c += blockDim.x) {
                    const int Y = c / LP, X = c - Y * LP;
                    ibuf[c] = (T)s[(wrap_pad(Y, L) - 1) * L + wrap_pad(X, L) - 1];
                }
            } else {
                const T *zp = zs + (size_t)(l - 1) * C * N;
                for (int i = threadIdx.x; i < C * N; i += blockDim.x) {
                    const int c = i / N, q = i - c * N, y = q / L, x = q - y * L;
                    ibuf[c * PP + (y + 1) * LP + x + 1] = silu_f(zp[i]);
                }
                __syncthreads();
                halo_fill(ibuf, C, L, PP);
            }
            __syncthreads();
            // per-sample weight gradient: item = (block of 4 output channels, input
            // channel), on two adjacent lanes that take the even and odd rows
            OutT *dW = Ob + vmc_woffset(C, l);
            const int nitems = (C / 4) * cin;
            for (int it2 = threadIdx.x; it2 < 2 * nitems; it2 += blockDim.x) {
                const int it = it2 >> 1, half = it2 & 1;
                const int cb = it / cin, ci = it - cb * cin;
                T acc[4][9];
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int t = 0; t < 9; ++t) acc[j][t] = T(0);
                const T *ip = ibuf + ci * PP;
                const T *gp = gbuf + cb * 4 * PP;
                for (int y = half; y < L; y += 2)
                    for (int x = 0; x < L; ++x) {
                        T a[9];
#pragma unroll
                        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                            for (int kx = 0; kx < 3; ++kx) a[ky * 3 + kx] = ip[(y + ky) * LP + x + kx];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const T g = gp[j * PP + (y + 1) * LP + x + 1];
#pragma unroll
                            for (int t = 0; t < 9; ++t) acc[j][t] = fma(g, a[t], acc[j][t]);
                        }
                    }
                // both lanes of the pair are active (2 nitems is even)
                const unsigned pm = __activemask();
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int t = 0; t < 9; ++t) acc[j][t] += __shfl_xor_sync(pm, acc[j][t], 1);
                if (half == 0) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int t = 0; t < 9; ++t)
                            dW[((cb * 4 + j) * cin + ci) * 9 + t] = (OutT)acc[j][t];
                }
            }
            for (int c = threadIdx.x; c < C; c += blockDim.x) {
                T acc = T(0);
                for (int y = 0; y < L; ++y)
                    for (int x = 0; x < L; ++x) acc += gbuf[c * PP + (y + 1) * LP + x + 1];
                dW[9 * C * cin + c] = (OutT)acc;
            }
            __syncthreads();
            if (l == 0) break;
            // g_{l-1} = (W^T * g_l) SiLU'(z_{l-1}), into ibuf, then swap
            conv_layer<T, CO>(gbuf, C * PP, C, WT + simt_w_offset(C, l), (const T *)nullptr, C, L, PP, 1,
                              StoreGradSilu<T>{ibuf, zs + (size_t)(l - 1) * C * N, PP, LP, L});
            __syncthreads();
            halo_fill(ibuf, C, L, PP);
            __syncthreads();
            T *t = gbuf; gbuf = ibuf; ibuf = t;
        }
        __syncthreads();
        // restore buffer roles for the next sample
        gbuf = reinterpret_cast<T *>(smem + 1024);
        ibuf = gbuf + (size_t)C * PP;
    }
}

template <typename T, int CO, typename OutT>
static int launch_bwd(vmc_ctx *ctx, const int8_t *sigma, int64_t B, void *O, cudaStream_t st)
{
    const int L = ctx->L, C = ctx->arch.channels, D = ctx->arch.n_layers_cc;
    const int PP = plane_pitch(L);
    const size_t smem = 1024 + 2 * (size_t)C * PP * sizeof(T);
    auto kfn = simt_bwd_kernel<T, CO, OutT>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "cudaFuncSetAttribute(simt_bwd)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, BWD_THREADS, smem);
    if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "occupancy(simt_bwd)");
    if (per_sm < 1) return vmc_fail(ctx, VMC_ERR_UNSUPPORTED, "backward does not fit on an SM (L=%d, C=%d)", L, C);
    int64_t grid = (int64_t)per_sm * ctx->sm_count;
    if (grid > B) grid = B;
    const size_t scratch = (size_t)grid * (D + 1) * C * L * L * sizeof(T);
    int rc = vmc_ensure_ws(ctx, &ctx->ws, &ctx->ws_bytes, scratch);
    if (rc) return rc;
    BwdParams p;
    p.L = L; p.C = C; p.D = D; p.B = B; p.n = ctx->n;
    p.sigma = sigma; p.W = ctx->wsimt; p.WT = ctx->wsimtT; p.bias = ctx->bias;
    p.scratch = ctx->ws; p.O = O;
    kfn<<<(unsigned)grid, BWD_THREADS, smem, st>>>(p);
    ctx->launches += 1;
    return vmc_cuda_check(ctx, cudaGetLastError(), "simt_bwd launch");
}

}  // namespace vmc

int vmc_simt_log_derivs(vmc_ctx *ctx, const int8_t *sigma, int64_t B, void *O, int dtype, cudaStream_t s)
{
    const int C = ctx->arch.channels;
    const bool co8 = (C % 8 == 0);
    if (ctx->arch.precision == VMC_FP64) {
        if (dtype == VMC_FP64)
            return co8 ? vmc::launch_bwd<double, 8, double>(ctx, sigma, B, O, s)
                       : vmc::launch_bwd<double, 4, double>(ctx, sigma, B, O, s);
        return co8 ? vmc::launch_bwd<double, 8, float>(ctx, sigma, B, O, s)
                   : vmc::launch_bwd<double, 4, float>(ctx, sigma, B, O, s);
    }
    if (dtype != VMC_FP32) return vmc_fail(ctx, VMC_ERR_ARG, "FP64 O output needs an FP64 context");
    return co8 ? vmc::launch_bwd<float, 8, float>(ctx, sigma, B, O, s)
               : vmc::launch_bwd<float, 4, float>(ctx, sigma, B, O, s);
}
