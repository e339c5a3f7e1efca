// Batched Metropolis sampling (arXiv:2108.13830 Sec. 3.1, Fig. 2b-c;
// Sec. 3.2.1: many independent chains whose proposals form one batch).
//
// A transition of chain b: list the J1 propose batch of sigma_b (the
// antiparallel pairs among the right and lower nearest-neighbour bonds,
// bond 2 i + d of site i, in increasing order), take pair
// k = floor(u0 n) of the n pairs, exchange its spins into sigma', and
// accept when P = (W(sigma') / W(sigma))^2 >= r with r = u1.  The random
// numbers are the caller's.  One launch of mh_kernel finishes transition
// s - 1 (decision and state update) and prepares transition s (proposal);
// between two such launches the proposals' log|psi| come from one batched
// forward launch (the tensor-core or SIMT path of vmc_logpsi).
#include "vmc_internal.h"

namespace vmc {
namespace mc {

constexpr int WARPS = 8;   // chains per CTA, one warp each

// bond 2 i + d: partner of site i to the right (d = 0) or below (d = 1)
__device__ __forceinline__ int j1_partner(int L, int i, int d)
{
    const int y = i / L, x = i - y * L;
    return d == 0 ? y * L + (x + 1 == L ? 0 : x + 1) : (y + 1 == L ? 0 : y + 1) * L + x;
}

// spin of site x after exchanging sites i and j of s
__device__ __forceinline__ int8_t swapped(const int8_t *s, int x, int i, int j)
{
    return s[x == i ? j : (x == j ? i : x)];
}

struct Args {
    int8_t *sigma;          // [B][N] chains, updated in place
    double *la;             // [B] log|psi| of the chains
    int8_t *prop;           // [B][N] proposals
    const double *la_new;   // [B] log|psi| of the proposals
    int2 *info;             // [B] (n pairs of sigma, n pairs of sigma')
    const double *u;        // [steps][B][2]
    int32_t *acc;           // [B] or null
    int64_t B;
    int L, step, n_steps, hastings;
};

__global__ void __launch_bounds__(WARPS * 32) mh_kernel(Args a)
{
    const int lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (b >= a.B) return;
    const int L = a.L, N = L * L;
    int8_t *s = a.sigma + b * N;
    int8_t *sp = a.prop + b * N;

    // decision of transition step - 1
    if (a.step > 0) {
        const int2 nf = a.info[b];
        bool take = false;
        if (nf.x > 0) {
            const double ln = a.la_new[b];
            double P = exp(2.0 * (ln - a.la[b]));
            if (a.hastings) P = P * ((double)nf.x / (double)nf.y);
            take = P >= a.u[((int64_t)(a.step - 1) * a.B + b) * 2 + 1];
        }
        if (take) {
            for (int x = lane; x < N; x += 32) s[x] = sp[x];
            if (lane == 0) {
                a.la[b] = a.la_new[b];
                if (a.acc) a.acc[b] += 1;
            }
        }
        __syncwarp();
    }
    if (a.step >= a.n_steps) return;

    // proposal of transition step: count the antiparallel J1 pairs
    const int nb = 2 * N;
    int n = 0;
    for (int base = 0; base < nb; base += 32) {
        const int k = base + lane;
        const bool f = k < nb && s[k >> 1] != s[j1_partner(L, k >> 1, k & 1)];
        n += __popc(__ballot_sync(0xffffffffu, f));
    }
    if (n == 0) {
        // no move: the forward evaluates the unchanged configuration
        for (int x = lane; x < N; x += 32) sp[x] = s[x];
        if (lane == 0) a.info[b] = make_int2(0, 0);
        return;
    }
    const double u0 = a.u[((int64_t)a.step * a.B + b) * 2];
    int k = (int)floor(u0 * (double)n);
    k = k < 0 ? 0 : (k > n - 1 ? n - 1 : k);
    // the k-th antiparallel pair, in bond order
    int bond = -1, seen = 0;
    for (int base = 0; base < nb && bond < 0; base += 32) {
        const int kk = base + lane;
        const bool f = kk < nb && s[kk >> 1] != s[j1_partner(L, kk >> 1, kk & 1)];
        const unsigned m = __ballot_sync(0xffffffffu, f);
        const int c = __popc(m);
        if (seen + c > k) {
            // lane holding the (k - seen)-th set bit of m
            unsigned mm = m;
            for (int r = 0; r < k - seen; ++r) mm &= mm - 1;
            bond = base + __ffs(mm) - 1;
        }
        seen += c;
    }
    const int i = bond >> 1, j = j1_partner(L, i, bond & 1);
    for (int x = lane; x < N; x += 32) sp[x] = swapped(s, x, i, j);
    // pairs of sigma' (for the Hastings factor), from sigma with i, j exchanged
    int n2 = 0;
    for (int base = 0; base < nb; base += 32) {
        const int kk = base + lane;
        bool f = false;
        if (kk < nb) {
            const int ii = kk >> 1;
            f = swapped(s, ii, i, j) != swapped(s, j1_partner(L, ii, kk & 1), i, j);
        }
        n2 += __popc(__ballot_sync(0xffffffffu, f));
    }
    if (lane == 0) a.info[b] = make_int2(n, n2);
}

}  // namespace mc
}  // namespace vmc

int vmc_metropolis_impl(vmc_ctx *ctx, int8_t *sigma, double *logabs, int64_t B, const double *u, int n_steps,
                        int hastings, int32_t *accepted, cudaStream_t s)
{
    using namespace vmc::mc;
    const int L = ctx->L, N = L * L;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_la = up((size_t)B * N), o_sg = o_la + up((size_t)B * 8), o_info = o_sg + up((size_t)B);
    const size_t need = o_info + up((size_t)B * sizeof(int2));
    int rc = vmc_ensure_ws(ctx, &ctx->mc_ws, &ctx->mc_ws_bytes, need);
    if (rc) return rc;
    char *w = static_cast<char *>(ctx->mc_ws);
    Args a;
    a.sigma = sigma; a.la = logabs; a.u = u; a.acc = accepted; a.B = B; a.L = L;
    a.prop = reinterpret_cast<int8_t *>(w);
    a.la_new = reinterpret_cast<double *>(w + o_la);
    a.info = reinterpret_cast<int2 *>(w + o_info);
    a.n_steps = n_steps; a.hastings = hastings ? 1 : 0;
    int8_t *sign = reinterpret_cast<int8_t *>(w + o_sg);
    const unsigned grid = (unsigned)((B + WARPS - 1) / WARPS);
    for (int step = 0; step <= n_steps; ++step) {
        a.step = step;
        mh_kernel<<<grid, WARPS * 32, 0, s>>>(a);
        ctx->launches += 1;
        rc = vmc_cuda_check(ctx, cudaGetLastError(), "mh_kernel launch");
        if (rc) return rc;
        if (step == n_steps) break;
        double *la_new = reinterpret_cast<double *>(w + o_la);
        rc = vmc_is_tc(ctx->arch.precision)
                 ? vmc_tc_eloc(ctx, 0, a.prop, nullptr, nullptr, B, L, la_new, sign, nullptr, s)
                 : vmc_simt_eloc(ctx, 0, a.prop, nullptr, nullptr, B, L, la_new, sign, nullptr, s);
        if (rc) return rc;
    }
    return VMC_OK;
}
