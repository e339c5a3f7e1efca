// Parameter preparation: the flat vector theta (layout of vmc.h) becomes
// an FP64 master copy, an FP32 copy, SIMT weight images (forward and
// flipped/transposed for the backward), bias arrays and, for BF16
// contexts, the tcgen05 B-operand images.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include "vmc_internal.h"
#include "simt_common.cuh"
#include "tc_layout.cuh"

namespace vmc {

template <typename Tin>
__global__ void cvt_theta_kernel(const Tin *__restrict__ in, double *t64, float *t32, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)in[i];
        t64[i] = v;
        t32[i] = (float)v;
    }
}

// The SR update of Eq. 6 on the master copy: theta <- theta - eta x, one
// product and one difference, each rounded (no fused multiply-add), so
// that the result is the plain FP64 expression.
__global__ void theta_step_kernel(double *t64, float *t32, const double *__restrict__ x, double eta, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = __dsub_rn(t64[i], __dmul_rn(eta, x[i]));
        t64[i] = v;
        t32[i] = (float)v;
    }
}

// SIMT images.  Forward: out[l][cb][ci][t][co'] = W_l[cb*CO+co'][ci][t].
// Transposed (l >= 1): out[l][cb][co][t][ci'] = W_l[co][cb*CO+ci'][8 - t].
template <typename T>
__global__ void simt_image_kernel(const double *__restrict__ theta, T *fwd, T *bwd, T *bias,
                                  int C, int D, int CO)
{
    const int64_t per_cc = 9LL * C * C;
    const int64_t total = 9LL * C + D * per_cc;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int l, cin;
        int64_t r;
        if (e < 9LL * C) { l = 0; cin = 1; r = e; }
        else { l = 1 + (int)((e - 9LL * C) / per_cc); cin = C; r = (e - 9LL * C) - (int64_t)(l - 1) * per_cc; }
        // r indexes [cb][ci][t][j] of this layer's image
        const int j = (int)(r % CO);
        const int t = (int)((r / CO) % 9);
        const int ci = (int)((r / (CO * 9)) % cin);
        const int cb = (int)(r / ((int64_t)CO * 9 * cin));
        const double *W = theta + vmc_woffset(C, l);
        fwd[e] = (T)W[((cb * CO + j) * cin + ci) * 9 + t];
        if (l > 0) {
            // image "output channel" = ci' = cb*CO + j of W, "input channel" = ci = co of W
            bwd[e] = (T)W[(ci * C + (cb * CO + j)) * 9 + (8 - t)];
        }
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)(D + 1) * C; i += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(i / C), c = (int)(i % C);
        bias[i] = (T)theta[vmc_woffset(C, l) + 9LL * C * (l == 0 ? 1 : C) + c];
    }
}

__global__ void tc_image_kernel(const double *__restrict__ theta, uint16_t *img, float *bias32, int C, int D, int f16)
{
    const int64_t total = tc_wimg_bytes(C, D) / 2;
    const int64_t l0 = tc_layer_bytes(C, 0), l1 = tc_layer_bytes(C, 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t byte = 2 * e;
        int l;
        int64_t rb;
        if (byte < l0) { l = 0; rb = byte; }
        else { l = 1 + (int)((byte - l0) / l1); rb = (byte - l0) - (int64_t)(l - 1) * l1; }
        const int N = tc_chunk_n(C, l);
        const int64_t cb = tc_chunk_bytes(C, l);
        const int chunk = (int)(rb / cb);
        const int off = (int)(rb % cb);
        // invert tc_b_elem_offset: off = kg*16N + ng*128 + nr*16 + kr*2
        const int kg = off / (16 * N);
        const int rem = off % (16 * N);
        const int n = (rem / 128) * 8 + (rem % 128) / 16;
        const int k = kg * 8 + (rem % 16) / 2;
        double w = 0.0;
        const double *W = theta + vmc_woffset(C, l);
        if (l == 0) {
            if (k < 9) w = W[n * 9 + k];
        } else {
            const int ky = chunk / (C / 16), h = chunk % (C / 16);
            // column block j of the B chunk holds horizontal tap kx = 2 - j
            const int kx = 2 - n / C, co = n % C;
            const int ci = 16 * h + k;
            w = W[(co * C + ci) * 9 + ky * 3 + kx];
        }
        // the tensor-core path computes h = z / 2 (SiLU(z) = h + h tanh h), so
        // weights and biases are stored halved (exact: a power of two)
        w *= 0.5;
        img[e] = f16 ? __half_as_ushort(__double2half(w)) : __bfloat16_as_ushort(__double2bfloat16(w));
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)(D + 1) * C; i += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(i / C), c = (int)(i % C);
        bias32[i] = (float)(0.5 * theta[vmc_woffset(C, l) + 9LL * C * (l == 0 ? 1 : C) + c]);
    }
}

}  // namespace vmc

int vmc_prepare_params(vmc_ctx *ctx, const void *theta, int dtype, cudaStream_t s)
{
    const int C = ctx->arch.channels, D = ctx->arch.n_layers_cc;
    const int64_t n = ctx->n;
    const int grid = 2 * ctx->sm_count, blk = 256;
    if (dtype == VMC_FP64)
        vmc::cvt_theta_kernel<double><<<grid, blk, 0, s>>>(static_cast<const double *>(theta), ctx->theta64, ctx->theta32, n);
    else
        vmc::cvt_theta_kernel<float><<<grid, blk, 0, s>>>(static_cast<const float *>(theta), ctx->theta64, ctx->theta32, n);
    ctx->launches += 1;
    return vmc_derive_images(ctx, s);
}

int vmc_derive_images(vmc_ctx *ctx, cudaStream_t s)
{
    const int C = ctx->arch.channels, D = ctx->arch.n_layers_cc;
    const int grid = 2 * ctx->sm_count, blk = 256;
    const int CO = vmc::simt_co(C);
    if (ctx->arch.precision == VMC_FP64)
        vmc::simt_image_kernel<double><<<grid, blk, 0, s>>>(ctx->theta64, (double *)ctx->wsimt, (double *)ctx->wsimtT,
                                                            (double *)ctx->bias, C, D, CO);
    else
        vmc::simt_image_kernel<float><<<grid, blk, 0, s>>>(ctx->theta64, (float *)ctx->wsimt, (float *)ctx->wsimtT,
                                                           (float *)ctx->bias, C, D, CO);
    ctx->launches += 1;
    if (vmc_is_tc(ctx->arch.precision)) {
        vmc::tc_image_kernel<<<grid, blk, 0, s>>>(ctx->theta64, ctx->wimg, ctx->bias32, C, D,
                                                  ctx->arch.precision == VMC_FP16);
        ctx->launches += 1;
    }
    return vmc_cuda_check(ctx, cudaGetLastError(), "prepare params");
}

int vmc_sr_update_impl(vmc_ctx *ctx, const double *x, double eta, cudaStream_t s)
{
    vmc::theta_step_kernel<<<2 * ctx->sm_count, 256, 0, s>>>(ctx->theta64, ctx->theta32, x, eta, ctx->n);
    ctx->launches += 1;
    const int rc = vmc_cuda_check(ctx, cudaGetLastError(), "theta step");
    return rc ? rc : vmc_derive_images(ctx, s);
}
