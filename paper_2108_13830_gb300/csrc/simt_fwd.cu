// Plain (SIMT) FP32 / FP64 forward pass, log|psi| and local energy.
//
// One CTA per sampled configuration sigma.  The CTA lists the antiparallel
// J1/J2 bonds of sigma in shared memory (Sec. 3.1, Fig. 2c), then evaluates
// sigma itself followed by every exchange neighbour sigma' -- each rebuilt
// from sigma in shared memory, never stored in HBM -- in groups of `nb`
// configurations, through the 3x3 circular convolutions with register tiles
// of CO output channels x 2 pixels.  Product pooling sums log|z| in FP64;
// E_loc = diagonal + sum coef * sgn' sgn exp(log|psi'| - log|psi|) in FP64
// (Eq. 4-5, Marshall factor of Eq. 9 folded into coef).
#include "vmc_internal.h"
#include "lattice.cuh"
#include "simt_common.cuh"

namespace vmc {

struct SimtParams {
    NetDesc net;
    int mode;                 // 0 logpsi, 1 local energy
    const int8_t *sigma;
    const int64_t *offs;      // ragged offsets or nullptr
    const int32_t *Ls;        // ragged sides or nullptr
    int L_max;
    int nb_max;               // configurations per group (for L_max)
    int buf_elems;            // elements per activation buffer
    int part_items;           // capacity of the pooling partial arrays
    const void *W;            // SIMT weight image
    const void *bias;         // [(D+1)][C]
    double *out_a;            // logabs or eloc
    int8_t *out_sign;         // logpsi sign
    int32_t *n_nbr;
    DevStatus *status;
};

template <typename T, int CO>
__global__ void __launch_bounds__(256, 1) simt_eloc_kernel(SimtParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int8_t *s = reinterpret_cast<int8_t *>(smem);                       // 1024
    uint16_t *list = reinterpret_cast<uint16_t *>(smem + 1024);         // 4096
    double *part = reinterpret_cast<double *>(smem + 1024 + 8192);      // part_items
    int *negz = reinterpret_cast<int *>(part + p.part_items);           // part_items (neg | zero << 16)
    double *conf_la = reinterpret_cast<double *>(negz + p.part_items);  // 32
    int *conf_sg = reinterpret_cast<int *>(conf_la + 32);                // 32
    int *sh = conf_sg + 32;                                               // 8 ints of scalars
    T *bufA = reinterpret_cast<T *>(
        (reinterpret_cast<uintptr_t>(sh + 8) + 15) & ~uintptr_t(15));
    T *bufB = bufA + p.buf_elems;

    const int b = blockIdx.x;
    const int C = p.net.C, D = p.net.D;
    const int L = p.Ls ? p.Ls[b] : p.net.L;
    if ((L & 1) || L < 4 || L > p.L_max) {
        if (threadIdx.x == 0) {
            if (p.mode == 0) { p.out_a[b] = __longlong_as_double(0x7ff8000000000000LL); p.out_sign[b] = 0; }
            else p.out_a[b] = __longlong_as_double(0x7ff8000000000000LL);
            if (p.n_nbr) p.n_nbr[b] = 0;
            atomicOr(&p.status->flags, VMC_STATUS_BADARG);
        }
        return;
    }
    const int N = L * L, LP = L + 2;
    const int PP = plane_pitch(L);
    const int8_t *sig = p.sigma + (p.offs ? p.offs[b] : (int64_t)b * N);
    for (int i = threadIdx.x; i < N; i += blockDim.x) s[i] = sig[i];
    __syncthreads();

    if (threadIdx.x < 32) {
        int a1 = 0, a2 = 0, cnt = 0, par = 0;
        if (p.mode == 1) cnt = build_bond_list_warp(s, L, list, &a1, &a2);
        else par = marshall_parity_warp(s, L);
        if (threadIdx.x == 0) { sh[0] = cnt; sh[1] = a1; sh[2] = a2; sh[3] = par; }
    }
    __syncthreads();
    const int nlist = sh[0];
    const int nconf_total = (p.mode == 1) ? 1 + nlist : 1;

    const int per_conf_cells = C * PP;
    const int items_last = (C / CO) * L * (L / 2);
    int nb_cap = p.buf_elems / per_conf_cells;
    nb_cap = min(nb_cap, p.part_items / items_last);
    nb_cap = min(nb_cap, 32);

    const T *Wimg = static_cast<const T *>(p.W);
    const T *bias = static_cast<const T *>(p.bias);

    double la0 = 0.0, acc = 0.0;
    int sg0 = 0;
    for (int c0 = 0; c0 < nconf_total; c0 += nb_cap) {
        const int nb = min(nb_cap, nconf_total - c0);
        // layer-0 input: the spin plane of each configuration (1 channel)
        const int cells = LP * LP;
        for (int idx = threadIdx.x; idx < nb * cells; idx += blockDim.x) {
            const int j = idx / cells, cell = idx - j * cells;
            const int Y = cell / LP, X = cell - Y * LP;
            const int site = (wrap_pad(Y, L) - 1) * L + (wrap_pad(X, L) - 1);
            int v = s[site];
            const int k = c0 + j;
            if (k > 0) {
                const int bond = list[k - 1];
                const int bi = bond >> 2, bj = bond_partner(L, bi, bond & 3);
                if (site == bi) v = s[bj];
                else if (site == bj) v = s[bi];
            }
            bufB[j * per_conf_cells + Y * LP + X] = (T)v;
        }
        __syncthreads();
        T *cur = bufB, *nxt = bufA;
        for (int l = 0; l <= D; ++l) {
            const int cin = (l == 0) ? 1 : C;
            const T *Wl = Wimg + simt_w_offset(C, l);
            const T *bl = bias + l * C;
            if (l < D) {
                conv_layer<T, CO>(cur, per_conf_cells, cin, Wl, bl, C, L, PP, nb,
                                  StoreSilu<T>{nxt, per_conf_cells, PP, LP});
                __syncthreads();
                halo_fill(nxt, nb * C, L, PP);
                __syncthreads();
                T *t = cur; cur = nxt; nxt = t;
            } else {
                conv_layer<T, CO>(cur, per_conf_cells, cin, Wl, bl, C, L, PP, nb,
                                  PoolEpi<T>{part, negz, items_last});
                __syncthreads();
            }
        }
        // deterministic per-configuration reduction (warp j sums configuration j)
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int j = warp; j < nb; j += blockDim.x >> 5) {
            double sacc = 0.0;
            int neg = 0, zer = 0;
            for (int it = lane; it < items_last; it += 32) {
                sacc += part[j * items_last + it];
                const int nz = negz[j * items_last + it];
                neg += nz & 0xffff;
                zer += nz >> 16;
            }
            for (int o = 16; o > 0; o >>= 1) {
                sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
                neg += __shfl_xor_sync(0xffffffffu, neg, o);
                zer += __shfl_xor_sync(0xffffffffu, zer, o);
            }
            if (lane == 0) {
                conf_la[j] = zer ? -INFINITY : sacc;
                conf_sg[j] = zer ? 0 : ((neg & 1) ? -1 : 1);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int j = 0; j < nb; ++j) {
                const int k = c0 + j;
                if (k == 0) { la0 = conf_la[j]; sg0 = conf_sg[j]; continue; }
                const int t = list[k - 1] & 3;
                const double rho = (double)(conf_sg[j] * sg0) * exp(conf_la[j] - la0);
                acc += exchange_coef(t, p.net.J1, p.net.J2, p.net.marshall) * rho;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (p.mode == 0) {
            int sg = sg0;
            if (p.net.marshall && sh[3]) sg = -sg;
            p.out_a[b] = la0;
            p.out_sign[b] = (int8_t)sg;
            if (!(la0 < INFINITY) || la0 != la0 || (sg0 == 0 && la0 != -INFINITY)) {
                atomicOr(&p.status->flags, VMC_STATUS_NONFINITE);
                atomicAdd(&p.status->nonfinite, 1ull);
            }
        } else {
            double e = diag_energy(L, sh[1], sh[2], p.net.J1, p.net.J2) + acc;
            if (sg0 == 0 || !isfinite(la0) || !isfinite(e)) {
                e = __longlong_as_double(0x7ff8000000000000LL);
                atomicOr(&p.status->flags, VMC_STATUS_NONFINITE);
                atomicAdd(&p.status->nonfinite, 1ull);
            }
            p.out_a[b] = e;
            if (p.n_nbr) p.n_nbr[b] = nlist;
        }
    }
}

template <typename T, int CO>
static int launch_simt(vmc_ctx *ctx, int mode, const int8_t *sigma, const int64_t *offs,
                       const int32_t *Ls, int64_t B, int L_max, double *out_a, void *out_b,
                       int32_t *n_nbr, cudaStream_t st)
{
    const int C = ctx->arch.channels;
    const int PP = plane_pitch(L_max);
    const size_t per_conf = (size_t)C * PP;              // elements per activation buffer per conf
    const int items = (C / CO) * L_max * (L_max / 2);
    const size_t fixed = 1024 + 8192 + 32 * 12 + 64 + 16;
    const size_t budget = 200 * 1024;
    const size_t per_nb = 2 * per_conf * sizeof(T) + (size_t)items * 12;
    int nb = (int)((budget - fixed) / per_nb);
    if (nb > 32) nb = 32;
    if (nb < 1) return vmc_fail(ctx, VMC_ERR_UNSUPPORTED, "lattice L=%d with C=%d exceeds shared memory", L_max, C);
    SimtParams p;
    p.net = NetDesc{ctx->L, C, ctx->arch.n_layers_cc, ctx->arch.marshall_sign, ctx->J1, ctx->J2};
    p.mode = mode;
    p.sigma = sigma; p.offs = offs; p.Ls = Ls; p.L_max = L_max;
    p.nb_max = nb;
    p.buf_elems = (int)(nb * per_conf);
    p.part_items = nb * items;
    p.W = ctx->wsimt; p.bias = ctx->bias;
    p.out_a = out_a; p.out_sign = static_cast<int8_t *>(out_b); p.n_nbr = n_nbr;
    p.status = ctx->status;
    const size_t smem = fixed + (size_t)p.part_items * 12 + 2 * (size_t)p.buf_elems * sizeof(T) + 16;
    auto kfn = simt_eloc_kernel<T, CO>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "cudaFuncSetAttribute(simt_eloc)");
    if (B > 0x7fffffff) return vmc_fail(ctx, VMC_ERR_ARG, "batch too large");
    kfn<<<(unsigned)B, 256, smem, st>>>(p);
    ctx->launches += 1;
    return vmc_cuda_check(ctx, cudaGetLastError(), "simt_eloc launch");
}

}  // namespace vmc

int vmc_simt_eloc(vmc_ctx *ctx, int mode, const int8_t *sigma, const int64_t *offs, const int32_t *Ls,
                  int64_t B, int L_max, double *out_a, void *out_b, int32_t *n_nbr, cudaStream_t s)
{
    const int C = ctx->arch.channels;
    if (ctx->arch.precision == VMC_FP64) {
        if (C % 8 == 0) return vmc::launch_simt<double, 8>(ctx, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr, s);
        return vmc::launch_simt<double, 4>(ctx, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr, s);
    }
    if (C % 8 == 0) return vmc::launch_simt<float, 8>(ctx, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr, s);
    return vmc::launch_simt<float, 4>(ctx, mode, sigma, offs, Ls, B, L_max, out_a, out_b, n_nbr, s);
}
