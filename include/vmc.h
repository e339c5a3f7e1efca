/*
 * vmc.h -- C ABI of libvmc: the data-parallel hot path of CNN variational
 * Monte Carlo for the spin-1/2 J1-J2 Heisenberg model on an L x L periodic
 * square lattice (arXiv:2108.13830), on one sm_103a GPU.
 *
 * Model (Sec. 2.1, Eq. 3):  H = J1/4 sum_<ij> sigma_i.sigma_j
 *                             + J2/4 sum_<<ij>> sigma_i.sigma_j.
 * Wavefunction (Sec. 2.2, Eq. 8-9): W(S) = (-1)^{M_A} W_CNN(S), with
 * W_CNN a stack of 3x3 circular-padded convolutions -- a 1 -> C embedding,
 * then D layers C -> C, SiLU after every layer but the last -- and product
 * pooling of the last layer: log|W_CNN| = sum_{c,p} log|z_{c,p}|,
 * sgn W_CNN = prod sgn z_{c,p}.  M_A counts up spins on the sublattice
 * x + y even.
 *
 * Conventions shared by every call:
 *  - Spin configurations are int8 in {+1, -1}, row-major [B][L][L]
 *    (site i = y * L + x).  L must be even and 4 <= L <= 32.
 *  - The flat parameter vector theta holds, for l = 0..D, the weights
 *    W_l[c_out][c_in][ky][kx] followed by the biases b_l[c_out]; c_in = 1 for
 *    l = 0 and C otherwise.  n = 10 C + D (9 C^2 + C).
 *    z_l[co][y][x] = b_l[co] + sum W_l[co][ci][ky][kx] a[ci][(y+ky-1) mod L][(x+kx-1) mod L].
 *  - Every pointer named *_dev is device memory owned by the caller; the
 *    library never frees or retains it past the call.  Every call is
 *    asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 *    stream) unless it says otherwise.
 *  - Return values: VMC_OK, or a negative code.  A negative code from an
 *    asynchronous call reports argument or launch errors only; faults found
 *    on the device (non-finite values, timeouts) are read with
 *    vmc_sync_status().  No call throws across the ABI and no call traps on
 *    the device.  vmc_last_error() gives a one-line message.
 *  - The library allocates its own workspaces (cudaMalloc) at vmc_create,
 *    vmc_set_params or the first call at a given batch size; calls made
 *    during CUDA-graph capture must not be the first at their size.
 */
#ifndef VMC_H_
#define VMC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VMC_OK             0
#define VMC_ERR_ARG       -1   /* invalid argument (null pointer, bad size, ...) */
#define VMC_ERR_CUDA      -2   /* a CUDA runtime call failed */
#define VMC_ERR_NONFINITE -3   /* some sample produced a non-finite value */
#define VMC_ERR_TIMEOUT   -4   /* a device-side wait ran out of its time budget */
#define VMC_ERR_STATE     -5   /* call out of order (e.g. parameters not set) */
#define VMC_ERR_UNSUPPORTED -6 /* device or configuration not supported */

/* Arithmetic of the convolutions.  VMC_BF16 runs the C -> C and embedding
 * convolutions on tcgen05 tensor cores with BF16 operands and FP32
 * accumulation; VMC_FP16 is the same tensor-core path with FP16 operands
 * (same rate, 11-bit instead of 8-bit significands).  log|psi| sums,
 * amplitude ratios and E_loc sums are FP64 in every precision. */
#define VMC_FP64 0
#define VMC_FP32 1
#define VMC_BF16 2
#define VMC_FP16 3

typedef struct vmc_ctx vmc_ctx;

typedef struct {
    int n_layers_cc;     /* D >= 1: number of C -> C layers after the 1 -> C embedding */
    int channels;        /* C: 4..64, multiple of 4 (16 or 32 for VMC_BF16 / VMC_FP16) */
    int precision;       /* VMC_FP64 | VMC_FP32 | VMC_BF16 | VMC_FP16 */
    int marshall_sign;   /* 1: include (-1)^{M_A} (Eq. 9) in the sign and E_loc */
} vmc_arch;

/* Tile choices of the tensor-core forward (chosen by vmc_autotune or set
 * explicitly).  0 fields mean "library default". */
typedef struct {
    int slab_configs;    /* configurations laid side by side in one slab */
    int slabs;           /* slabs in flight per CTA (1 or 2) */
    int ctas_per_sm;     /* persistent CTAs per SM */
    int lane_cells;      /* lattice cells per accumulator row (TMEM lane), P:
                            1..4 for C = 32, even 2..8 for C = 16 */
} vmc_tiles;

/* Create a context for L x L lattices with couplings J1, J2 (Eq. 3) and the
 * network `arch`.  Binds the current CUDA device.  *out receives the
 * context; on failure *out is NULL and the return code says why
 * (VMC_ERR_UNSUPPORTED when the device is not sm_103). */
int vmc_create(int L, double J1, double J2, const vmc_arch *arch, vmc_ctx **out);
void vmc_destroy(vmc_ctx *ctx);

/* n, the length of the flat parameter vector. */
int vmc_num_params(const vmc_ctx *ctx, int64_t *n);

/* Copy theta (n values of `dtype`: VMC_FP64 or VMC_FP32, device memory)
 * into the context and derive the per-precision weight images.  Ordered
 * on `stream`; theta_dev may be reused after the call returns only once
 * the stream has passed this point. */
int vmc_set_params(vmc_ctx *ctx, const void *theta_dev, int dtype, void *stream);

/* Copy the context's FP64 parameter vector (n doubles) to theta_dev. */
int vmc_get_params(const vmc_ctx *ctx, double *theta_dev, void *stream);

/* log|psi(sigma_b)| and its sign for B configurations (Sec. 2.2, Eq. 8-9).
 * sigma_dev: int8 [B][L][L].  logabs_dev: double [B].  sign_dev: int8 [B]
 * (+1, -1, or 0 where psi = 0, in which case logabs = -inf).  B = 0 is a
 * no-op. */
int vmc_logpsi(vmc_ctx *ctx, const int8_t *sigma_dev, int64_t B,
               double *logabs_dev, int8_t *sign_dev, void *stream);

/* Local energy E_loc(sigma_b) = sum_{sigma'} H(sigma, sigma') psi(sigma')/psi(sigma)
 * (Eq. 4-5), summed over the diagonal term and every configuration reached
 * by exchanging an antiparallel J1 or J2 bond (Sec. 3.1, Fig. 2c: right and
 * below neighbours for J1, the two lower diagonals for J2).  Each
 * neighbour sigma' is generated on chip from its parent; the parent is
 * evaluated in the same launch and the same arithmetic as its neighbours.
 * eloc_dev: double [B] (total energy, not per site).  n_nbr_dev: int32 [B]
 * number of exchange neighbours, or NULL.  A sample whose psi is 0 or
 * non-finite gets NaN and raises VMC_ERR_NONFINITE in vmc_sync_status. */
int vmc_local_energy(vmc_ctx *ctx, const int8_t *sigma_dev, int64_t B,
                     double *eloc_dev, int32_t *n_nbr_dev, void *stream);

/* The same over a ragged batch of mixed lattice sizes with the context's
 * weights (translation-invariant convolutions apply to any L).  Sample b has
 * side L_dev[b] (even, 4 <= L_dev[b] <= L_max) and spins at
 * packed_dev[offs_dev[b] .. offs_dev[b] + L_dev[b]^2).  L_max is a host
 * value bounding every L_dev[b]; a sample beyond it gets NaN and raises
 * VMC_ERR_ARG in vmc_sync_status.  One persistent launch covers the batch. */
int vmc_local_energy_ragged(vmc_ctx *ctx, const int8_t *packed_dev, const int64_t *offs_dev,
                            const int32_t *L_dev, int64_t B, int L_max,
                            double *eloc_dev, int32_t *n_nbr_dev, void *stream);

/* Rotationally symmetrised amplitude (Sec. 2.2, Eq. 10; Sec. 3.3 applies it
 * in the last fine-tuning stage):
 *     W~(S) = sum_{i=0..3} W(T^i S),  W = (-1)^{M_A} W_CNN,
 * T the 90-degree rotation of the L x L lattice.  Each W~ evaluates the
 * context's forward (the arithmetic of vmc_logpsi, signs included) on the
 * four rotations, i.e. four times the work, and sums the signed amplitudes
 * in FP64 after factoring out the largest.  The rotated configurations are
 * materialised in device memory, a chunk of samples at a time (workspace
 * up to about 1 GiB).
 *  - vmc_logpsi_sym: log|W~| and sgn W~, layouts as vmc_logpsi.
 *  - vmc_local_energy_sym: E_loc of Eq. 4-5 with W~ for sigma and for every
 *    exchange neighbour (the bonds of vmc_local_energy, full signs);
 *    n_nbr_dev as there.  Synchronises `stream` once, to size the chunks
 *    from the neighbour counts.
 *  - vmc_log_derivs_sym: O_bk = d log|W~| / d theta_k
 *    = sum_i (W(T^i sigma_b) / W~(sigma_b)) O_k(T^i sigma_b); O_dev and
 *    dtype as vmc_log_derivs.
 * A sample with W~ = 0 or a non-finite result gets NaN (E_loc) or -inf
 * (log|W~|) and raises VMC_ERR_NONFINITE in vmc_sync_status (E_loc). */
int vmc_logpsi_sym(vmc_ctx *ctx, const int8_t *sigma_dev, int64_t B,
                   double *logabs_dev, int8_t *sign_dev, void *stream);
int vmc_local_energy_sym(vmc_ctx *ctx, const int8_t *sigma_dev, int64_t B,
                         double *eloc_dev, int32_t *n_nbr_dev, void *stream);
int vmc_log_derivs_sym(vmc_ctx *ctx, const int8_t *sigma_dev, int64_t B,
                       void *O_dev, int dtype, void *stream);

/* Batched Metropolis sampling of |W(S)|^2 (Sec. 3.1, Fig. 2b-c; the chains
 * of Sec. 3.2.1 advance together, their proposals forming one batch).  Each
 * of B independent chains makes n_steps transitions.  Transition s of
 * chain b:
 *  - lists the J1 propose batch of sigma_b: the antiparallel pairs among the
 *    bonds of every site i = y L + x to its right and to its lower neighbour
 *    (periodic), in that order, site by site; n_b pairs;
 *  - picks pair k = floor(u[s][b][0] n_b), clamped to 0..n_b - 1, and
 *    exchanges its two spins into sigma';
 *  - accepts sigma' when P >= u[s][b][1], with
 *    P = exp(2 (log|psi(sigma')| - log|psi(sigma)|)) = (W(sigma') / W(sigma))^2,
 *    times n_b / n'_b (the pair counts of sigma and sigma') when
 *    hastings = 1.  The paper's rule is hastings = 0; its stationary law is
 *    |psi|^2 n_b / Z, the corrected one |psi|^2 / Z.
 *  - A chain with n_b = 0 has no move and stays.
 * The log|psi| of the B proposals of a transition come from one batched
 * forward (the arithmetic of vmc_logpsi), so a transition costs one forward
 * per chain; the paper spaces recorded samples by L^2 transitions.
 *  - sigma_dev int8 [B][L][L]: the chains, updated in place.
 *  - logabs_dev double [B]: on entry log|psi(sigma_b)| as vmc_logpsi gives
 *    it; on exit that of the final sigma_b (the accepted forward's value).
 *  - u_dev double [n_steps][B][2]: the caller's uniform numbers in [0, 1).
 *  - accepted_dev int32 [B] or NULL: incremented by each accepted move.
 * B = 0 or n_steps = 0 is a no-op.  Workspace: about B (L^2 + 17) bytes, grown on
 * the first call at a larger B. */
int vmc_metropolis(vmc_ctx *ctx, int8_t *sigma_dev, double *logabs_dev, int64_t B,
                   const double *u_dev, int n_steps, int hastings, int32_t *accepted_dev, void *stream);

/* Per-sample log-derivatives O_bk = d log|psi(sigma_b)| / d theta_k (Eq. 5),
 * by a hand-written backward pass that recomputes the forward activations
 * (workspace bounded by the number of resident CTAs, not by B).
 * O_dev: [B][n] row-major of `dtype` (VMC_FP32; VMC_FP64 also allowed for
 * FP64 contexts).  Runs in FP64 for VMC_FP64 contexts, FP32 otherwise. */
int vmc_log_derivs(vmc_ctx *ctx, const int8_t *sigma_dev, int64_t B,
                   void *O_dev, int dtype, void *stream);

/* SR moments (Eq. 5): Obar_k = (1/m) sum_b O_bk, Ebar = (1/m) sum_b E_b,
 * G_k = (1/m) sum_b O_bk (E_b - Ebar).  O_dev float [m][n], E_dev double [m],
 * outputs double (device).  Sums carry FP64 accuracy. */
int vmc_sr_moments(vmc_ctx *ctx, const float *O_dev, const double *E_dev, int64_t m,
                   double *Obar_dev, double *Ebar_dev, double *G_dev, void *stream);

/* out = (S + shift I) v with S v = (1/m) O^T (O v) - Obar (Obar . v), the
 * covariance of Eq. 7 applied without forming it (Sec. 3.2.2 builds
 * M = O^T O - <O>^T <O> + shift I).  Computed as
 * (1/m) O^T (t - tbar) with t = O v, tbar = (1/m) sum_b t_b. */
int vmc_sr_matvec(vmc_ctx *ctx, const float *O_dev, int64_t m, const double *Obar_dev,
                  const double *v_dev, double shift, double *out_dev, void *stream);

/* out = O^T w, i.e. out_k = sum_b O_bk w_b, with FP64 accuracy.  O_dev
 * float [m][n], w_dev double [m], out_dev double [n].  This is the
 * vector-Jacobian product of log|psi| (the backward of the autograd layer:
 * d/dtheta sum_b w_b log|psi_b| = O^T w). */
int vmc_ot_vec(vmc_ctx *ctx, const float *O_dev, int64_t m, const double *w_dev,
               double *out_dev, void *stream);

/* out = O^T w like vmc_ot_vec, for callers that must not allocate device
 * memory: code running inside an allocator or memory-pool callback, runtimes
 * that forbid cudaMalloc after start-up, or processes with a device-memory
 * budget fixed at load time.  It takes no context (creating one allocates)
 * and calls no cudaMalloc, cudaFree or allocating library routine; its
 * scratch is a 16 MiB array in the library's device image, held by every
 * GPU that loads the library until the process exits.  The paper has no
 * counterpart.
 *  - O_dev float [m][n], w_dev double [m], out_dev double [n] (device,
 *    owned by the caller); asynchronous on `stream`.
 *  - Limit: 8 n c + 8 m <= 16 MiB (m rounded up to a multiple of 32), with
 *    c = 16 row chunks for m >= 1024, 4 for m >= 64, else 1; e.g. m = 4096
 *    allows n <= 130816, m = 1 allows n <= 2097120.  Larger sizes return
 *    VMC_ERR_UNSUPPORTED before any device work; null pointers or m, n < 1
 *    return VMC_ERR_ARG.
 *  - Every call looks up the scratch array's device address with the
 *    caller's device and context current (nothing is cached, so a
 *    cudaDeviceReset or a different driver context is safe).  With lazy
 *    module loading (the CUDA default) the FIRST call on a device loads the
 *    library's device module, which is when the driver reserves the 16 MiB;
 *    make that first call at start-up, outside any allocator hook and before
 *    any stream capture (a call with m = n = 1 serves as a warm-up).
 *  - All calls on a device share the scratch and it keeps the last call's
 *    contents (nothing in it needs to start at zero); calls whose work
 *    overlaps on the GPU (different streams, no ordering) race. */
int vmc_ot_vec_noalloc(const float *O_dev, int64_t m, int64_t n, const double *w_dev,
                       double *out_dev, void *stream);

/* Single-pass covariance product for vmc_sr_matvec and vmc_sr_solve
 * (enable = 1): one cooperative launch whose CTAs each own a slice of
 * columns, stream the rows through shared memory, exchange their partial
 * row dots (O v) through global memory and accumulate O^T (t - tbar) from
 * the rows still on chip, with tbar = Obar . v and the d_b re-centred on
 * their own sum.  It reads O once per product, but the per-block exchange
 * between CTAs and the double-float arithmetic (not the HBM read) bound
 * it: 2.7 ms per product at m = 4096, n = 92,800 against 0.75 ms for the
 * default two passes over O (t = O v, then O^T (t - mean t)).  Applies
 * when n is a multiple of 4, O is 16-byte aligned and the column slice of
 * one CTA fits shared memory; otherwise the two passes run.  Off by
 * default; results agree to double-float rounding, not bit for bit. */
int vmc_set_sr_fused(vmc_ctx *ctx, int enable);

/* Solve (S + shift I) x = G for the SR direction (Eq. 6 with eta = 1:
 * Delta = x; the caller applies theta -= eta x) by conjugate gradient from
 * x = 0, exactly `iters` iterations (fewer only when the residual is exactly
 * zero), the recurrence in FP64 and every S v matrix-free.  The iteration is
 * captured once in a CUDA graph and replayed.  x_dev: double [n].
 * resid_out (host, nullable): ||r|| / ||G|| after the last step; when it is
 * non-NULL the call synchronises `stream`. */
int vmc_sr_solve(vmc_ctx *ctx, const float *O_dev, const double *eloc_dev, int64_t m,
                 double shift, int iters, double *x_dev, double *resid_out, void *stream);

/* The same SR direction x = (S + shift I)^{-1} G solved exactly (no
 * iteration) in the m-dimensional sample space, the choice for m << n
 * (Sec. 2.1, Eq. 6-7; Sec. 3.2.2 factors the covariance by Cholesky): by
 * the Woodbury identity, with Oc = O - 1 Obar^T,
 *     x = (G - Oc^T y) / shift,   (m shift I + Oc Oc^T) y = Oc G.
 * The m x m Gram matrix Oc Oc^T is formed on the device from the centred
 * rows held as double-float pairs (FP64-level accuracy), factored by a
 * blocked FP64 Cholesky and solved; Oc G and Oc^T y are passes over O.
 * Dividing G - Oc^T y by the shift amplifies rounding by the condition of
 * S + shift I, so two steps of iterative refinement follow (r = G -
 * (S + shift I) x with the covariance product of vmc_sr_matvec, x += W r,
 * W the same solve applied to r).
 * Workspace: 8 m n + 8 m^2 bytes (3.2 GB at m = 4096, n = 92,800).  Cost
 * grows as m^2 n: use it where m is well below n.  shift > 0; m <= 65536.
 * x_dev double [n]; resid_out (host, nullable): ||G - (S + shift I) x|| /
 * ||G|| from one more covariance product (synchronises `stream`).  A
 * factorisation that meets a non-positive pivot leaves NaN in x and raises
 * VMC_ERR_NONFINITE in vmc_sync_status. */
int vmc_sr_solve_dense(vmc_ctx *ctx, const float *O_dev, const double *eloc_dev, int64_t m, double shift,
                       double *x_dev, double *resid_out, void *stream);

/* The SR parameter update of Eq. 6, theta <- theta - eta x, on the
 * context's FP64 parameter vector, with x the direction vmc_sr_solve
 * returns (Delta = eta x, x = (S + shift I)^{-1} G).  Each entry is
 * theta_k - (eta x_k), the product and the difference rounded separately
 * in FP64.  The working images of the context's precision are re-derived
 * from the updated vector, so the next forward uses it.  x_dev double [n]
 * (device).  Requires parameters to be set. */
int vmc_sr_update(vmc_ctx *ctx, const double *x_dev, double eta, void *stream);

/* Synchronise `stream` and read (then clear) the device status word:
 * VMC_OK, VMC_ERR_NONFINITE (with *nonfinite = number of samples, if
 * non-NULL), VMC_ERR_TIMEOUT or VMC_ERR_ARG. */
int vmc_sync_status(vmc_ctx *ctx, void *stream, int64_t *nonfinite);

/* Time budget, in nanoseconds, of every device-side wait (mbarrier waits
 * of the tensor-core pipeline).  0 restores the default (2 s).  A wait that
 * runs out sets VMC_ERR_TIMEOUT, releases its resources and returns. */
int vmc_set_wait_budget(vmc_ctx *ctx, int64_t ns);

/* Light-cone evaluation of the exchange neighbours in vmc_local_energy
 * (tensor-core contexts, uniform batches).  The convolutions are 3 x 3
 * (Sec. 2.2; the locality of the filters, Sec. 3.3), so after layer l the
 * activations of a neighbour sigma' differ from its parent's only within
 * l + 1 cells of the exchanged pair.  With it on, a first launch evaluates
 * every parent and keeps all its layers' activations (workspace of
 * 2 C D L^2 bytes per sample, up to 2 GiB, the batch taken in chunks
 * beyond that); a second evaluates each neighbour on a window of side
 * min(2 l + 4, L) per layer, filling the window's border from the parent.
 * E_loc and the neighbour counts are bit for bit those of the plain
 * evaluation.  It applies when 6 <= L <= 2 D + 4 (the window covers the
 * lattice by the last layer); otherwise, for ragged batches and for
 * FP32/FP64 contexts the plain evaluation runs.  On by default.
 *  - vmc_set_light_cone: enable = 1 (default) or 0 (plain evaluation).
 *  - vmc_light_cone_active: *active = 1 if vmc_local_energy uses it. */
int vmc_set_light_cone(vmc_ctx *ctx, int enable);
int vmc_light_cone_active(const vmc_ctx *ctx, int *active);

/* Launch timing of the tensor-core kernels, for measuring a kernel inside
 * a public call: while enabled, every tensor-core launch is bracketed by a
 * pair of CUDA events recorded on its stream.  vmc_set_launch_timing(ctx, 1)
 * enables it and forgets earlier records; vmc_launch_timings synchronises
 * on the recorded events and writes up to `max` durations (ms) in launch
 * order, *count = the number recorded; vmc_launch_timing_name gives the
 * kernel of record i (NULL beyond the count).  Host-side bookkeeping only
 * (events are created on first use); not for use under stream capture. */
int vmc_set_launch_timing(vmc_ctx *ctx, int enable);
int vmc_launch_timings(vmc_ctx *ctx, int max, double *ms, int *count);
const char *vmc_launch_timing_name(const vmc_ctx *ctx, int i);

/* Launch one wait on an mbarrier that nothing arrives on, with the given
 * budget; the wait must give up and report VMC_ERR_TIMEOUT through
 * vmc_sync_status.  Exercises the timeout path without faulting the GPU. */
int vmc_debug_wait_timeout(vmc_ctx *ctx, int64_t budget_ns, void *stream);

/* Tile choice of the tensor-core forward for lattice side L: set, read, or
 * tune (times each candidate on `probe_B` synthetic configurations with
 * CUDA events on `stream`, keeps the fastest; synchronises `stream`). */
int vmc_set_tiles(vmc_ctx *ctx, int L, const vmc_tiles *tiles);
int vmc_get_tiles(const vmc_ctx *ctx, int L, vmc_tiles *tiles);
int vmc_autotune(vmc_ctx *ctx, int L, int64_t probe_B, void *stream);

/* Tile choice of the light-cone pass (vmc_set_light_cone) for the
 * context's lattice side: slabs (1 or 2), slab_configs = neighbour windows
 * per slab, lane_cells = P; 0 fields are left to the cost model.  Set
 * returns VMC_ERR_UNSUPPORTED (and keeps the previous choice) when no plan
 * fits; get reports the plan in use (VMC_ERR_UNSUPPORTED where the light
 * cone does not apply).  vmc_autotune(ctx, ctx's L, ...) also times the
 * best-modelled light-cone plans and keeps the fastest.  The light-cone
 * pass of vmc_local_energy_ragged takes slabs and lane_cells for its
 * launch and slab_configs as the upper bound of every side's windows. */
int vmc_set_cone_tiles(vmc_ctx *ctx, const vmc_tiles *tiles);
int vmc_get_cone_tiles(const vmc_ctx *ctx, vmc_tiles *tiles);

/* Issue-rate probe of the tensor cores: `ctas` CTAs each issue `count`
 * back-to-back 128 x N x 16 BF16 UMMAs (N multiple of 16, <= 256);
 * returns the mean cycles per MMA and the launch time.  Synchronous.
 * Diagnostic: the paper has no counterpart. */
int vmc_debug_umma_rate(int N, int count, int ctas, double *cycles_per_mma, double *ms);

/* One 128 x N x K UMMA tile (N multiple of 16 up to 128, K = 16 or 32)
 * from row-major BF16 A [128 + shift][K] and B [N][K] (device) into FP32 D [128][N] (device), through the shared-memory
 * layout of the convolution kernel (variant 0) or with the two descriptor
 * strides exchanged (variant 1).  Layout self-test; the paper has no
 * counterpart. */
int vmc_debug_umma_selftest(const uint16_t *A_dev, const uint16_t *B_dev, float *D_dev, int N, int K,
                            int shift, int variant, void *stream);

/* Kernel launches issued by the last public call (for launch accounting). */
int64_t vmc_last_launch_count(const vmc_ctx *ctx);

const char *vmc_last_error(const vmc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* VMC_H_ */
