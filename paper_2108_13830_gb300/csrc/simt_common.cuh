// Building blocks of the SIMT (FP32 / FP64) convolution path.
//
// Activations live in shared memory as circularly padded planes: plane c of
// a configuration holds (L+2) x (L+2) cells, cell (Y, X) = a[(Y-1) mod L][(X-1) mod L],
// so the 3x3 tap (ky, kx) of output (y, x) is cell (y+ky, x+kx).  Planes are
// PP = (L+2)^2 + 1 elements apart (odd, so per-channel strides fall on
// distinct banks).
//
// SIMT weight image of layer l: [cblk][ci][ky*3+kx][CO], CO output channels
// of block cblk contiguous, so one thread loads them with vector loads and
// all threads of a warp (same cblk) read the same address.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vmc {

__host__ __device__ __forceinline__ int plane_pitch(int L) { return (L + 2) * (L + 2) + 1; }

__host__ __device__ __forceinline__ int simt_co(int C) { return (C % 8 == 0) ? 8 : 4; }

// offset of layer l in the SIMT weight image (same element count as W_l)
__host__ __device__ __forceinline__ int64_t simt_w_offset(int C, int l)
{
    return l == 0 ? 0 : (int64_t)9 * C + (int64_t)(l - 1) * 9 * C * C;
}

// padded coordinate -> interior padded coordinate it copies (1..L)
__device__ __forceinline__ int wrap_pad(int Y, int L) { return Y == 0 ? L : (Y == L + 1 ? 1 : Y); }

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ double silu_f(double z) { return z / (1.0 + exp(-z)); }
__device__ __forceinline__ float log_abs(float z) { return logf(fabsf(z)); }
__device__ __forceinline__ double log_abs(double z) { return log(fabs(z)); }

template <typename T, int CO>
__device__ __forceinline__ void load_w(const T *__restrict__ w, T (&out)[CO])
{
    if constexpr (sizeof(T) == 4) {
        const float4 *v = reinterpret_cast<const float4 *>(w);
#pragma unroll
        for (int q = 0; q < CO / 4; ++q) {
            const float4 f = __ldg(v + q);
            out[4 * q + 0] = f.x; out[4 * q + 1] = f.y; out[4 * q + 2] = f.z; out[4 * q + 3] = f.w;
        }
    } else {
        const double2 *v = reinterpret_cast<const double2 *>(w);
#pragma unroll
        for (int q = 0; q < CO / 2; ++q) {
            const double2 f = __ldg(v + q);
            out[2 * q + 0] = f.x; out[2 * q + 1] = f.y;
        }
    }
}

// One 3x3 circular convolution layer over `nconf` configurations.
// in: shared, [nconf][cin][PP] padded planes (conf stride in_cs elements).
// Work item = (conf, output-channel block, row y, pixel pair x0): CO x 2
// outputs.  FP64: one FMA chain (bias, then ci, ky, kx in order).  FP32:
// for each input channel the nine taps form a short FMA chain, and the
// per-channel partial sums are added with Kahan compensation (Kahan 1965),
// so the rounding of a K = 9 c_in term sum stays at the level of a single
// FP32 rounding instead of growing with sqrt(K).  epi(it, conf, c0, y, x0,
// acc) consumes the result; items are numbered conf-major.
template <typename T, int CO, class Epi>
__device__ __forceinline__ void conv_layer(const T *__restrict__ in, int in_cs, int cin,
                                           const T *__restrict__ W, const T *__restrict__ bias,
                                           int cout, int L, int PP, int nconf, Epi epi)
{
    constexpr bool KAHAN = (sizeof(T) == 4);
    const int LP = L + 2, hx = L >> 1;
    const int nblk = cout / CO;
    const int per_row = hx, per_blk = L * hx, per_conf = nblk * per_blk;
    const int total = nconf * per_conf;
    for (int it = threadIdx.x; it < total; it += blockDim.x) {
        const int conf = it / per_conf;
        int r = it - conf * per_conf;
        const int cb = r / per_blk;
        r -= cb * per_blk;
        const int y = r / per_row;
        const int x0 = (r - y * per_row) * 2;
        T acc[CO][2], comp[CO][2];
#pragma unroll
        for (int co = 0; co < CO; ++co) {
            const T bv = bias ? bias[cb * CO + co] : T(0);
            acc[co][0] = bv;
            acc[co][1] = bv;
            comp[co][0] = T(0);
            comp[co][1] = T(0);
        }
        const T *ip = in + conf * in_cs + y * LP + x0;
        const T *wp = W + (size_t)cb * cin * 9 * CO;
        for (int ci = 0; ci < cin; ++ci) {
            T part[CO][2];
#pragma unroll
            for (int co = 0; co < CO; ++co) {
                part[co][0] = KAHAN ? T(0) : acc[co][0];
                part[co][1] = KAHAN ? T(0) : acc[co][1];
            }
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                const T *rp = ip + ci * PP + ky * LP;
                const T a0 = rp[0], a1 = rp[1], a2 = rp[2], a3 = rp[3];
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    T w[CO];
                    load_w<T, CO>(wp + (ci * 9 + ky * 3 + kx) * CO, w);
                    const T i0 = (kx == 0) ? a0 : ((kx == 1) ? a1 : a2);
                    const T i1 = (kx == 0) ? a1 : ((kx == 1) ? a2 : a3);
#pragma unroll
                    for (int co = 0; co < CO; ++co) {
                        part[co][0] = fma(w[co], i0, part[co][0]);
                        part[co][1] = fma(w[co], i1, part[co][1]);
                    }
                }
            }
#pragma unroll
            for (int co = 0; co < CO; ++co)
#pragma unroll
                for (int px = 0; px < 2; ++px) {
                    if constexpr (KAHAN) {
                        const T yk = part[co][px] - comp[co][px];
                        const T tk = acc[co][px] + yk;
                        comp[co][px] = (tk - acc[co][px]) - yk;
                        acc[co][px] = tk;
                    } else {
                        acc[co][px] = part[co][px];
                    }
                }
        }
        if constexpr (KAHAN) {
#pragma unroll
            for (int co = 0; co < CO; ++co) {
                acc[co][0] -= comp[co][0];
                acc[co][1] -= comp[co][1];
            }
        }
        epi(it, conf, cb * CO, y, x0, acc);
    }
}

// Epilogue: SiLU, stored into the interior of padded output planes.
template <typename T>
struct StoreSilu {
    T *out;
    int cs, PP, LP;
    template <int CO>
    __device__ __forceinline__ void operator()(int, int conf, int c0, int y, int x0, T (&acc)[CO][2]) const
    {
        T *o = out + conf * cs + c0 * PP + (y + 1) * LP + x0 + 1;
#pragma unroll
        for (int co = 0; co < CO; ++co) {
            o[co * PP] = silu_f(acc[co][0]);
            o[co * PP + 1] = silu_f(acc[co][1]);
        }
    }
};

// Epilogue of the last layer: product pooling partials, log|z| summed in
// FP64, plus counts of negative and zero outputs.
template <typename T>
struct PoolEpi {
    double *part;
    int *negz;
    int items_per_conf;
    template <int CO>
    __device__ __forceinline__ void operator()(int it, int, int, int, int, T (&acc)[CO][2]) const
    {
        double sacc = 0.0;
        int neg = 0, zer = 0;
#pragma unroll
        for (int co = 0; co < CO; ++co)
#pragma unroll
            for (int px = 0; px < 2; ++px) {
                const T z = acc[co][px];
                neg += (z < T(0));
                zer += (z == T(0));
                sacc += (double)log_abs(z);
            }
        part[it] = sacc;
        negz[it] = neg | (zer << 16);
    }
};

// Fill the 4L+4 halo cells of each of `nplanes` padded planes from the
// interior (circular boundary).
template <typename T>
__device__ __forceinline__ void halo_fill(T *buf, int nplanes, int L, int PP)
{
    const int LP = L + 2, nh = 4 * L + 4;
    for (int idx = threadIdx.x; idx < nplanes * nh; idx += blockDim.x) {
        const int pl = idx / nh;
        const int h = idx - pl * nh;
        int Y, X;
        if (h < LP) { Y = 0; X = h; }
        else if (h < 2 * LP) { Y = L + 1; X = h - LP; }
        else { const int q = h - 2 * LP; Y = 1 + (q >> 1); X = (q & 1) ? L + 1 : 0; }
        T *pb = buf + (size_t)pl * PP;
        pb[Y * LP + X] = pb[wrap_pad(Y, L) * LP + wrap_pad(X, L)];
    }
}

}  // namespace vmc
