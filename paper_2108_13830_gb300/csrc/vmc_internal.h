// Internal declarations shared by the translation units of libvmc.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <map>
#include <vector>

#include "../../include/vmc.h"

// Device status word (one per context), written by kernels, read and
// cleared by vmc_sync_status.
struct DevStatus {
    int flags;                 // VMC_STATUS_* bits
    int timeout_site;          // which wait gave up (for diagnostics)
    unsigned long long nonfinite;   // samples with a non-finite result
};
#define VMC_STATUS_NONFINITE 1
#define VMC_STATUS_TIMEOUT 2
#define VMC_STATUS_BADARG 4
#define VMC_STATUS_INTERNAL 8

// Everything a forward / local-energy kernel needs to know about the model.
struct NetDesc {
    int L;          // lattice side (uniform batches); ragged batches read L per sample
    int C;          // channels
    int D;          // C -> C layers after the embedding
    int marshall;   // include (-1)^{M_A}
    double J1, J2;
};

// Per-L tile choice of the tensor-core forward.
struct TileChoice {
    int slab_configs = 0;
    int slabs = 0;
    int ctas_per_sm = 0;
    int lane_cells = 0;
};

struct vmc_ctx {
    int L = 0;
    double J1 = 0, J2 = 0;
    vmc_arch arch{};
    int64_t n = 0;
    int device = 0;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    bool params_set = false;

    // parameter images (device)
    double *theta64 = nullptr;   // [n] master copy
    float *theta32 = nullptr;    // [n]
    void *wsimt = nullptr;       // SIMT forward weights, [l][cblk][ci][9][CO] (float or double)
    void *wsimtT = nullptr;      // transposed/flipped weights for the backward grad-input conv
    void *bias = nullptr;        // [(D+1)][C] (float or double, matching the SIMT type)
    uint16_t *wimg = nullptr;    // BF16 / FP16 UMMA B-operand images, all layers
    float *bias32 = nullptr;     // [(D+1)][C] halved FP32 biases for the tensor-core epilogue
    size_t wimg_bytes = 0;

    DevStatus *status = nullptr; // device
    int *counter = nullptr;      // device work counter(s) for persistent launches

    // workspaces
    void *ws = nullptr;
    size_t ws_bytes = 0;
    void *sr_ws = nullptr;
    size_t sr_ws_bytes = 0;
    void *mc_ws = nullptr;       // Metropolis proposals and their log|psi|
    size_t mc_ws_bytes = 0;
    void *sym_ws = nullptr;      // rotated configurations, their log|psi| and O rows
    size_t sym_ws_bytes = 0;
    void *sym_cnt = nullptr;     // per-sample neighbour counts, diagonals, offsets
    size_t sym_cnt_bytes = 0;
    int dense_refine = 2;        // sample-space SR solve: refinement steps
    void *dense_ws = nullptr;    // sample-space SR solve: centred rows, Gram matrix / factor
    size_t dense_ws_bytes = 0;
    void *order_ws = nullptr;    // ragged batches: work order (largest lattices first)
    size_t order_ws_bytes = 0;
    void *cone_tab = nullptr;    // ragged light cone: per-side layer geometry (device)
    size_t cone_tab_bytes = 0;
    std::vector<char> cone_tab_host;   // the table last uploaded
    void *cone_ws = nullptr;     // light-cone E_loc: parent activations, log|psi| and signs
    size_t cone_ws_bytes = 0;
    int light_cone = 1;          // evaluate E_loc neighbours incrementally where it applies
    TileChoice cone_tiles;       // light-cone pass tile choice (0 fields: cost model)
    int sr_fused = 0;            // S v in one pass over O (off: two passes, faster; see vmc.h)

    // launch timing of the tensor-core kernels (vmc_set_launch_timing):
    // an event pair around each launch on its stream, with the kernel's name
    int timing = 0;
    std::vector<cudaEvent_t> tev;
    std::vector<std::string> tname;
    size_t tn = 0;               // pairs recorded since timing was (re)enabled

    int64_t wait_budget_ns = 2000000000LL;
    std::map<int, TileChoice> tiles;

    // SR CG graph cache
    cudaGraphExec_t cg_exec = nullptr;
    const void *cg_key_O = nullptr;
    int64_t cg_key_m = -1;
    int cg_key_iters = -1;
    double cg_key_shift = 0;
    void *cg_key_x = nullptr;
    void *cg_key_ws = nullptr;
    int cg_key_fused = -1;
    int64_t cg_launches = 0;

    int64_t launches = 0;
    std::string last_error;
};

// error helpers (host)
int vmc_fail(vmc_ctx *ctx, int code, const char *fmt, ...);
int vmc_cuda_check(vmc_ctx *ctx, cudaError_t e, const char *what);
int vmc_ensure_ws(vmc_ctx *ctx, void **buf, size_t *cur, size_t need);
// launch timing: the event to record before (start = true) or after a
// kernel launch named `name` (nullptr when timing is off)
cudaEvent_t vmc_timing_event(vmc_ctx *ctx, bool start, const char *name);

// parameter preparation (prep.cu)
int vmc_prepare_params(vmc_ctx *ctx, const void *theta, int dtype, cudaStream_t s);
int vmc_derive_images(vmc_ctx *ctx, cudaStream_t s);           // per-precision images from theta64
int vmc_sr_update_impl(vmc_ctx *ctx, const double *x, double eta, cudaStream_t s);

// SIMT forward / local energy (simt_fwd.cu)
int vmc_simt_eloc(vmc_ctx *ctx, int mode, const int8_t *sigma, const int64_t *offs, const int32_t *Ls,
                  int64_t B, int L_max, double *out_a, void *out_b, int32_t *n_nbr, cudaStream_t s);
// mode: 0 = logpsi (out_a = logabs, out_b = int8 sign), 1 = local energy (out_a = eloc)

// SIMT backward (simt_bwd.cu)
int vmc_simt_log_derivs(vmc_ctx *ctx, const int8_t *sigma, int64_t B, void *O, int dtype, cudaStream_t s);

// tensor-core forward (tc_fwd.cu)
int vmc_tc_eloc(vmc_ctx *ctx, int mode, const int8_t *sigma, const int64_t *offs, const int32_t *Ls,
                int64_t B, int L_max, double *out_a, void *out_b, int32_t *n_nbr, cudaStream_t s);
int vmc_tc_default_tiles(const vmc_ctx *ctx, int L, TileChoice *t);
bool vmc_tc_cone_applies(const vmc_ctx *ctx);
int vmc_tc_cone_default_tiles(const vmc_ctx *ctx, TileChoice *t);
int vmc_tc_debug_timeout(vmc_ctx *ctx, int64_t budget_ns, cudaStream_t s);

// Metropolis sampling (mcmc.cu)
int vmc_metropolis_impl(vmc_ctx *ctx, int8_t *sigma, double *logabs, int64_t B, const double *u, int n_steps,
                        int hastings, int32_t *accepted, cudaStream_t s);

// rotationally symmetrised amplitude (sym.cu)
int vmc_logpsi_sym_impl(vmc_ctx *ctx, const int8_t *sigma, int64_t B, double *logabs, int8_t *sign, cudaStream_t s);
int vmc_local_energy_sym_impl(vmc_ctx *ctx, const int8_t *sigma, int64_t B, double *eloc, int32_t *n_nbr,
                              cudaStream_t s);
int vmc_log_derivs_sym_impl(vmc_ctx *ctx, const int8_t *sigma, int64_t B, void *O, int dtype, cudaStream_t s);

// SR (sr.cu)
int vmc_sr_moments_impl(vmc_ctx *ctx, const float *O, const double *E, int64_t m,
                        double *Obar, double *Ebar, double *G, cudaStream_t s);
int vmc_sr_matvec_impl(vmc_ctx *ctx, const float *O, int64_t m, const double *Obar,
                       const double *v, double shift, double *out, cudaStream_t s);
int vmc_ot_vec_impl(vmc_ctx *ctx, const float *O, int64_t m, const double *w, double *out, cudaStream_t s);
int vmc_sr_solve_impl(vmc_ctx *ctx, const float *O, const double *E, int64_t m, double shift,
                      int iters, double *x, double *resid_out, cudaStream_t s);
int vmc_sr_solve_dense_impl(vmc_ctx *ctx, const float *O, const double *E, int64_t m, double shift, double *x,
                            double *resid_out, cudaStream_t s);

__host__ __device__ static inline bool vmc_is_tc(int precision) { return precision == VMC_BF16 || precision == VMC_FP16; }
__host__ __device__ static inline int64_t vmc_nparams(int C, int D) { return (int64_t)10 * C + (int64_t)D * (9 * C * C + C); }
__host__ __device__ static inline int64_t vmc_woffset(int C, int l) { return l == 0 ? 0 : (int64_t)10 * C + (int64_t)(l - 1) * (9 * C * C + C); }
