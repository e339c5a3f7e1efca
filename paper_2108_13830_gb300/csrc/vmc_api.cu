// C ABI of libvmc (declared in include/vmc.h): argument checking, context
// lifetime, workspace management and dispatch to the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include "vmc_internal.h"

int vmc_fail(vmc_ctx *ctx, int code, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return code;
}

int vmc_cuda_check(vmc_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return VMC_OK;
    return vmc_fail(ctx, VMC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int vmc_ensure_ws(vmc_ctx *ctx, void **buf, size_t *cur, size_t need)
{
    if (*cur >= need && *buf) return VMC_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(cudaStreamLegacy, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return vmc_fail(ctx, VMC_ERR_STATE, "workspace growth during graph capture");
    if (*buf) {
        // previous work may still use it
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "sync before workspace growth");
        cudaFree(*buf);
        *buf = nullptr;
        *cur = 0;
    }
    cudaError_t e = cudaMalloc(buf, need);
    if (e != cudaSuccess) { *buf = nullptr; return vmc_cuda_check(ctx, e, "workspace cudaMalloc"); }
    *cur = need;
    return VMC_OK;
}

static bool arch_ok(int L, const vmc_arch *a, char *why, size_t nw)
{
    if (L < 4 || L > 32 || (L & 1)) { snprintf(why, nw, "L=%d must be even, 4..32", L); return false; }
    if (a->n_layers_cc < 1 || a->n_layers_cc > 64) { snprintf(why, nw, "n_layers_cc=%d out of 1..64", a->n_layers_cc); return false; }
    if (a->channels < 4 || a->channels > 64 || a->channels % 4) { snprintf(why, nw, "channels=%d must be a multiple of 4 in 4..64", a->channels); return false; }
    if (a->precision < VMC_FP64 || a->precision > VMC_FP16) { snprintf(why, nw, "bad precision %d", a->precision); return false; }
    if (vmc_is_tc(a->precision) && (a->channels != 16 && a->channels != 32)) { snprintf(why, nw, "tensor-core path supports channels 16 or 32"); return false; }
    if (a->marshall_sign != 0 && a->marshall_sign != 1) { snprintf(why, nw, "marshall_sign must be 0 or 1"); return false; }
    return true;
}

cudaEvent_t vmc_timing_event(vmc_ctx *ctx, bool start, const char *name)
{
    if (!ctx->timing) return nullptr;
    const size_t i = 2 * ctx->tn + (start ? 0 : 1);
    if (i >= ctx->tev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ctx->tev.push_back(e);
    }
    if (start) {
        if (ctx->tname.size() <= ctx->tn) ctx->tname.resize(ctx->tn + 1);
        ctx->tname[ctx->tn] = name ? name : "";
    } else {
        ctx->tn += 1;
    }
    return ctx->tev[i];
}

extern "C" {

int vmc_create(int L, double J1, double J2, const vmc_arch *arch, vmc_ctx **out)
{
    if (!out) return VMC_ERR_ARG;
    *out = nullptr;
    if (!arch) return VMC_ERR_ARG;
    char why[128];
    if (!arch_ok(L, arch, why, sizeof why)) return VMC_ERR_ARG;
    vmc_ctx *ctx = new (std::nothrow) vmc_ctx();
    if (!ctx) return VMC_ERR_ARG;
    ctx->L = L; ctx->J1 = J1; ctx->J2 = J2; ctx->arch = *arch;
    ctx->n = vmc_nparams(arch->channels, arch->n_layers_cc);
    int rc = VMC_OK;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->cc_major, cudaDevAttrComputeCapabilityMajor, ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->cc_minor, cudaDevAttrComputeCapabilityMinor, ctx->device);
    if (e != cudaSuccess) { delete ctx; return VMC_ERR_CUDA; }
    if (!(ctx->cc_major == 10 && ctx->cc_minor == 3)) { delete ctx; return VMC_ERR_UNSUPPORTED; }
    const int C = arch->channels, D = arch->n_layers_cc;
    const size_t n = (size_t)ctx->n;
    const size_t tsz = (arch->precision == VMC_FP64) ? 8 : 4;
    e = cudaMalloc(&ctx->theta64, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->theta32, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->wsimt, n * tsz);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->wsimtT, n * tsz);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->bias, (size_t)(D + 1) * C * tsz);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->bias32, (size_t)(D + 1) * C * 4);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->status, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->counter, 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->counter, 0, 64 * sizeof(int));
    if (e == cudaSuccess && vmc_is_tc(arch->precision)) {
        ctx->wimg_bytes = (size_t)(32LL * C + (int64_t)D * 9 * (C / 16) * 32LL * C);
        e = cudaMalloc(&ctx->wimg, ctx->wimg_bytes);
    }
    if (e != cudaSuccess) rc = VMC_ERR_CUDA;
    if (rc) { vmc_destroy(ctx); return rc; }
    *out = ctx;
    return VMC_OK;
}

void vmc_destroy(vmc_ctx *ctx)
{
    if (!ctx) return;
    cudaDeviceSynchronize();
    if (ctx->cg_exec) cudaGraphExecDestroy(ctx->cg_exec);
    cudaFree(ctx->theta64); cudaFree(ctx->theta32); cudaFree(ctx->wsimt); cudaFree(ctx->wsimtT);
    cudaFree(ctx->bias); cudaFree(ctx->bias32); cudaFree(ctx->wimg);
    cudaFree(ctx->status); cudaFree(ctx->counter);
    cudaFree(ctx->ws); cudaFree(ctx->sr_ws); cudaFree(ctx->mc_ws); cudaFree(ctx->sym_ws); cudaFree(ctx->sym_cnt); cudaFree(ctx->cone_ws); cudaFree(ctx->order_ws); cudaFree(ctx->cone_tab); cudaFree(ctx->dense_ws);
    for (cudaEvent_t e : ctx->tev) cudaEventDestroy(e);
    delete ctx;
}

int vmc_num_params(const vmc_ctx *ctx, int64_t *n)
{
    if (!ctx || !n) return VMC_ERR_ARG;
    *n = ctx->n;
    return VMC_OK;
}

int vmc_set_params(vmc_ctx *ctx, const void *theta_dev, int dtype, void *stream)
{
    if (!ctx) return VMC_ERR_ARG;
    ctx->launches = 0;
    if (!theta_dev) return vmc_fail(ctx, VMC_ERR_ARG, "theta is NULL");
    if (dtype != VMC_FP64 && dtype != VMC_FP32) return vmc_fail(ctx, VMC_ERR_ARG, "theta dtype must be FP64 or FP32");
    int rc = vmc_prepare_params(ctx, theta_dev, dtype, (cudaStream_t)stream);
    if (rc == VMC_OK) ctx->params_set = true;
    return rc;
}

int vmc_get_params(const vmc_ctx *ctx, double *theta_dev, void *stream)
{
    if (!ctx || !theta_dev) return VMC_ERR_ARG;
    if (!ctx->params_set) return VMC_ERR_STATE;
    cudaError_t e = cudaMemcpyAsync(theta_dev, ctx->theta64, ctx->n * 8, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return e == cudaSuccess ? VMC_OK : VMC_ERR_CUDA;
}

static int check_ready(vmc_ctx *ctx)
{
    if (!ctx) return VMC_ERR_ARG;
    ctx->launches = 0;
    if (!ctx->params_set) return vmc_fail(ctx, VMC_ERR_STATE, "parameters not set");
    return VMC_OK;
}

int vmc_logpsi(vmc_ctx *ctx, const int8_t *sigma_dev, int64_t B, double *logabs_dev, int8_t *sign_dev, void *stream)
{
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (B < 0) return vmc_fail(ctx, VMC_ERR_ARG, "negative batch");
    if (B == 0) return VMC_OK;
    if (!sigma_dev || !logabs_dev || !sign_dev) return vmc_fail(ctx, VMC_ERR_ARG, "null pointer");
    if (vmc_is_tc(ctx->arch.precision))
        return vmc_tc_eloc(ctx, 0, sigma_dev, nullptr, nullptr, B, ctx->L, logabs_dev, sign_dev, nullptr, (cudaStream_t)stream);
    return vmc_simt_eloc(ctx, 0, sigma_dev, nullptr, nullptr, B, ctx->L, logabs_dev, sign_dev, nullptr, (cudaStream_t)stream);
}

int vmc_local_energy(vmc_ctx *ctx, const int8_t *sigma_dev, int64_t B, double *eloc_dev, int32_t *n_nbr_dev, void *stream)
{
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (B < 0) return vmc_fail(ctx, VMC_ERR_ARG, "negative batch");
    if (B == 0) return VMC_OK;
    if (!sigma_dev || !eloc_dev) return vmc_fail(ctx, VMC_ERR_ARG, "null pointer");
    if (vmc_is_tc(ctx->arch.precision))
        return vmc_tc_eloc(ctx, 1, sigma_dev, nullptr, nullptr, B, ctx->L, eloc_dev, nullptr, n_nbr_dev, (cudaStream_t)stream);
    return vmc_simt_eloc(ctx, 1, sigma_dev, nullptr, nullptr, B, ctx->L, eloc_dev, nullptr, n_nbr_dev, (cudaStream_t)stream);
}

int vmc_local_energy_ragged(vmc_ctx *ctx, const int8_t *packed_dev, const int64_t *offs_dev, const int32_t *L_dev,
                            int64_t B, int L_max, double *eloc_dev, int32_t *n_nbr_dev, void *stream)
{
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (B < 0) return vmc_fail(ctx, VMC_ERR_ARG, "negative batch");
    if (B == 0) return VMC_OK;
    if (!packed_dev || !offs_dev || !L_dev || !eloc_dev) return vmc_fail(ctx, VMC_ERR_ARG, "null pointer");
    if (L_max < 4 || L_max > 32 || (L_max & 1)) return vmc_fail(ctx, VMC_ERR_ARG, "L_max=%d must be even, 4..32", L_max);
    if (vmc_is_tc(ctx->arch.precision))
        return vmc_tc_eloc(ctx, 1, packed_dev, offs_dev, L_dev, B, L_max, eloc_dev, nullptr, n_nbr_dev, (cudaStream_t)stream);
    return vmc_simt_eloc(ctx, 1, packed_dev, offs_dev, L_dev, B, L_max, eloc_dev, nullptr, n_nbr_dev, (cudaStream_t)stream);
}

int vmc_logpsi_sym(vmc_ctx *ctx, const int8_t *sigma_dev, int64_t B, double *logabs_dev, int8_t *sign_dev, void *stream)
{
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (B < 0) return vmc_fail(ctx, VMC_ERR_ARG, "negative batch");
    if (B == 0) return VMC_OK;
    if (!sigma_dev || !logabs_dev || !sign_dev) return vmc_fail(ctx, VMC_ERR_ARG, "null pointer");
    return vmc_logpsi_sym_impl(ctx, sigma_dev, B, logabs_dev, sign_dev, (cudaStream_t)stream);
}

int vmc_local_energy_sym(vmc_ctx *ctx, const int8_t *sigma_dev, int64_t B, double *eloc_dev, int32_t *n_nbr_dev,
                         void *stream)
{
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (B < 0) return vmc_fail(ctx, VMC_ERR_ARG, "negative batch");
    if (B == 0) return VMC_OK;
    if (!sigma_dev || !eloc_dev) return vmc_fail(ctx, VMC_ERR_ARG, "null pointer");
    return vmc_local_energy_sym_impl(ctx, sigma_dev, B, eloc_dev, n_nbr_dev, (cudaStream_t)stream);
}

int vmc_log_derivs_sym(vmc_ctx *ctx, const int8_t *sigma_dev, int64_t B, void *O_dev, int dtype, void *stream)
{
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (B < 0) return vmc_fail(ctx, VMC_ERR_ARG, "negative batch");
    if (B == 0) return VMC_OK;
    if (!sigma_dev || !O_dev) return vmc_fail(ctx, VMC_ERR_ARG, "null pointer");
    if (dtype != VMC_FP32 && dtype != VMC_FP64) return vmc_fail(ctx, VMC_ERR_ARG, "O dtype must be FP32 or FP64");
    if (dtype == VMC_FP64 && ctx->arch.precision != VMC_FP64)
        return vmc_fail(ctx, VMC_ERR_ARG, "FP64 O output needs an FP64 context");
    return vmc_log_derivs_sym_impl(ctx, sigma_dev, B, O_dev, dtype, (cudaStream_t)stream);
}

int vmc_metropolis(vmc_ctx *ctx, int8_t *sigma_dev, double *logabs_dev, int64_t B, const double *u_dev,
                   int n_steps, int hastings, int32_t *accepted_dev, void *stream)
{
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (B < 0 || n_steps < 0) return vmc_fail(ctx, VMC_ERR_ARG, "negative batch or step count");
    if (hastings != 0 && hastings != 1) return vmc_fail(ctx, VMC_ERR_ARG, "hastings must be 0 or 1");
    if (B == 0 || n_steps == 0) return VMC_OK;
    if (!sigma_dev || !logabs_dev || !u_dev) return vmc_fail(ctx, VMC_ERR_ARG, "null pointer");
    return vmc_metropolis_impl(ctx, sigma_dev, logabs_dev, B, u_dev, n_steps, hastings, accepted_dev,
                               (cudaStream_t)stream);
}

int vmc_log_derivs(vmc_ctx *ctx, const int8_t *sigma_dev, int64_t B, void *O_dev, int dtype, void *stream)
{
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (B < 0) return vmc_fail(ctx, VMC_ERR_ARG, "negative batch");
    if (B == 0) return VMC_OK;
    if (!sigma_dev || !O_dev) return vmc_fail(ctx, VMC_ERR_ARG, "null pointer");
    if (dtype != VMC_FP32 && dtype != VMC_FP64) return vmc_fail(ctx, VMC_ERR_ARG, "O dtype must be FP32 or FP64");
    return vmc_simt_log_derivs(ctx, sigma_dev, B, O_dev, dtype, (cudaStream_t)stream);
}

int vmc_sr_moments(vmc_ctx *ctx, const float *O_dev, const double *E_dev, int64_t m,
                   double *Obar_dev, double *Ebar_dev, double *G_dev, void *stream)
{
    if (!ctx) return VMC_ERR_ARG;
    ctx->launches = 0;
    if (m < 1) return vmc_fail(ctx, VMC_ERR_ARG, "m must be >= 1");
    if (!O_dev || !E_dev || !Obar_dev || !Ebar_dev || !G_dev) return vmc_fail(ctx, VMC_ERR_ARG, "null pointer");
    return vmc_sr_moments_impl(ctx, O_dev, E_dev, m, Obar_dev, Ebar_dev, G_dev, (cudaStream_t)stream);
}

int vmc_sr_matvec(vmc_ctx *ctx, const float *O_dev, int64_t m, const double *Obar_dev,
                  const double *v_dev, double shift, double *out_dev, void *stream)
{
    if (!ctx) return VMC_ERR_ARG;
    ctx->launches = 0;
    if (m < 1) return vmc_fail(ctx, VMC_ERR_ARG, "m must be >= 1");
    if (!O_dev || !v_dev || !out_dev) return vmc_fail(ctx, VMC_ERR_ARG, "null pointer");
    return vmc_sr_matvec_impl(ctx, O_dev, m, Obar_dev, v_dev, shift, out_dev, (cudaStream_t)stream);
}

int vmc_ot_vec(vmc_ctx *ctx, const float *O_dev, int64_t m, const double *w_dev, double *out_dev, void *stream)
{
    if (!ctx) return VMC_ERR_ARG;
    ctx->launches = 0;
    if (m < 1) return vmc_fail(ctx, VMC_ERR_ARG, "m must be >= 1");
    if (!O_dev || !w_dev || !out_dev) return vmc_fail(ctx, VMC_ERR_ARG, "null pointer");
    return vmc_ot_vec_impl(ctx, O_dev, m, w_dev, out_dev, (cudaStream_t)stream);
}

int vmc_sr_solve(vmc_ctx *ctx, const float *O_dev, const double *eloc_dev, int64_t m,
                 double shift, int iters, double *x_dev, double *resid_out, void *stream)
{
    if (!ctx) return VMC_ERR_ARG;
    ctx->launches = 0;
    if (m < 1) return vmc_fail(ctx, VMC_ERR_ARG, "m must be >= 1");
    if (iters < 0 || iters > 100000) return vmc_fail(ctx, VMC_ERR_ARG, "iters out of range");
    if (!(shift >= 0.0)) return vmc_fail(ctx, VMC_ERR_ARG, "shift must be >= 0");
    if (!O_dev || !eloc_dev || !x_dev) return vmc_fail(ctx, VMC_ERR_ARG, "null pointer");
    return vmc_sr_solve_impl(ctx, O_dev, eloc_dev, m, shift, iters, x_dev, resid_out, (cudaStream_t)stream);
}

int vmc_sr_solve_dense(vmc_ctx *ctx, const float *O_dev, const double *eloc_dev, int64_t m, double shift,
                       double *x_dev, double *resid_out, void *stream)
{
    if (!ctx) return VMC_ERR_ARG;
    ctx->launches = 0;
    if (m < 1) return vmc_fail(ctx, VMC_ERR_ARG, "m must be >= 1");
    if (!(shift > 0.0)) return vmc_fail(ctx, VMC_ERR_ARG, "shift must be > 0");
    if (!O_dev || !eloc_dev || !x_dev) return vmc_fail(ctx, VMC_ERR_ARG, "null pointer");
    if (m > 65536) return vmc_fail(ctx, VMC_ERR_UNSUPPORTED, "m = %lld beyond the dense solve's limit", (long long)m);
    return vmc_sr_solve_dense_impl(ctx, O_dev, eloc_dev, m, shift, x_dev, resid_out, (cudaStream_t)stream);
}

int vmc_sr_update(vmc_ctx *ctx, const double *x_dev, double eta, void *stream)
{
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (!x_dev) return vmc_fail(ctx, VMC_ERR_ARG, "null pointer");
    if (!std::isfinite(eta)) return vmc_fail(ctx, VMC_ERR_ARG, "eta must be finite");
    return vmc_sr_update_impl(ctx, x_dev, eta, (cudaStream_t)stream);
}

int vmc_sync_status(vmc_ctx *ctx, void *stream, int64_t *nonfinite)
{
    if (!ctx) return VMC_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "stream synchronize");
    DevStatus st;
    e = cudaMemcpy(&st, ctx->status, sizeof st, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof st);
    if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "status read");
    if (nonfinite) *nonfinite = (int64_t)st.nonfinite;
    if (st.flags & VMC_STATUS_TIMEOUT) return vmc_fail(ctx, VMC_ERR_TIMEOUT, "device wait timed out (site %d)", st.timeout_site);
    if (st.flags & VMC_STATUS_INTERNAL) return vmc_fail(ctx, VMC_ERR_STATE, "internal scheduling error in the persistent kernel");
    if (st.flags & VMC_STATUS_BADARG) return vmc_fail(ctx, VMC_ERR_ARG, "a sample had an invalid lattice size");
    if (st.flags & VMC_STATUS_NONFINITE) return vmc_fail(ctx, VMC_ERR_NONFINITE, "%llu samples non-finite", st.nonfinite);
    return VMC_OK;
}

int vmc_set_wait_budget(vmc_ctx *ctx, int64_t ns)
{
    if (!ctx || ns < 0) return VMC_ERR_ARG;
    ctx->wait_budget_ns = ns ? ns : 2000000000LL;
    return VMC_OK;
}

int vmc_set_launch_timing(vmc_ctx *ctx, int enable)
{
    if (!ctx || (enable != 0 && enable != 1)) return VMC_ERR_ARG;
    ctx->timing = enable;
    ctx->tn = 0;
    return VMC_OK;
}

int vmc_launch_timings(vmc_ctx *ctx, int max, double *ms, int *count)
{
    if (!ctx || !count || max < 0 || (max > 0 && !ms)) return VMC_ERR_ARG;
    const int n = (int)ctx->tn;
    *count = n;
    for (int i = 0; i < n && i < max; ++i) {
        cudaError_t e = cudaEventSynchronize(ctx->tev[2 * i + 1]);
        if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "timing event");
        float t = 0.f;
        e = cudaEventElapsedTime(&t, ctx->tev[2 * i], ctx->tev[2 * i + 1]);
        if (e != cudaSuccess) return vmc_cuda_check(ctx, e, "timing elapsed");
        ms[i] = t;
    }
    return VMC_OK;
}

const char *vmc_launch_timing_name(const vmc_ctx *ctx, int i)
{
    if (!ctx || i < 0 || (size_t)i >= ctx->tn) return nullptr;
    return ctx->tname[i].c_str();
}

int vmc_set_sr_fused(vmc_ctx *ctx, int enable)
{
    if (!ctx || (enable != 0 && enable != 1)) return VMC_ERR_ARG;
    ctx->sr_fused = enable;
    return VMC_OK;
}

int vmc_set_light_cone(vmc_ctx *ctx, int enable)
{
    if (!ctx || (enable != 0 && enable != 1)) return VMC_ERR_ARG;
    ctx->light_cone = enable;
    return VMC_OK;
}

int vmc_light_cone_active(const vmc_ctx *ctx, int *active)
{
    if (!ctx || !active) return VMC_ERR_ARG;
    *active = (ctx->light_cone && vmc_tc_cone_applies(ctx)) ? 1 : 0;
    return VMC_OK;
}

int vmc_debug_wait_timeout(vmc_ctx *ctx, int64_t budget_ns, void *stream)
{
    if (!ctx || budget_ns < 0 || budget_ns > 10000000000LL) return VMC_ERR_ARG;
    ctx->launches = 0;
    return vmc_tc_debug_timeout(ctx, budget_ns, (cudaStream_t)stream);
}

int vmc_set_tiles(vmc_ctx *ctx, int L, const vmc_tiles *tiles)
{
    if (!ctx || !tiles || L < 4 || L > 32 || (L & 1)) return VMC_ERR_ARG;
    TileChoice t;
    t.slab_configs = tiles->slab_configs;
    t.slabs = tiles->slabs;
    t.ctas_per_sm = tiles->ctas_per_sm;
    t.lane_cells = tiles->lane_cells;
    if (t.slabs < 0 || t.slabs > 2 || t.slab_configs < 0 || t.slab_configs > 64 || t.ctas_per_sm < 0 ||
        t.ctas_per_sm > 4 || t.lane_cells < 0 || t.lane_cells > 8)
        return vmc_fail(ctx, VMC_ERR_ARG, "tile choice out of range");
    ctx->tiles[L] = t;
    return VMC_OK;
}

int vmc_get_tiles(const vmc_ctx *ctx, int L, vmc_tiles *tiles)
{
    if (!ctx || !tiles) return VMC_ERR_ARG;
    TileChoice t;
    auto it = ctx->tiles.find(L);
    if (it != ctx->tiles.end()) t = it->second;
    TileChoice d;
    int rc = vmc_tc_default_tiles(ctx, L, &d);
    if (rc) return rc;
    tiles->slab_configs = t.slab_configs ? t.slab_configs : d.slab_configs;
    tiles->slabs = t.slabs ? t.slabs : d.slabs;
    tiles->ctas_per_sm = t.ctas_per_sm ? t.ctas_per_sm : d.ctas_per_sm;
    tiles->lane_cells = t.lane_cells ? t.lane_cells : d.lane_cells;
    return VMC_OK;
}

int vmc_set_cone_tiles(vmc_ctx *ctx, const vmc_tiles *tiles)
{
    if (!ctx || !tiles) return VMC_ERR_ARG;
    TileChoice t;
    t.slab_configs = tiles->slab_configs;
    t.slabs = tiles->slabs;
    t.ctas_per_sm = tiles->ctas_per_sm;
    t.lane_cells = tiles->lane_cells;
    if (t.slabs < 0 || t.slabs > 2 || t.slab_configs < 0 || t.slab_configs > 16 || t.ctas_per_sm < 0 ||
        t.ctas_per_sm > 1 || t.lane_cells < 0 || t.lane_cells > 8)
        return vmc_fail(ctx, VMC_ERR_ARG, "light-cone tile choice out of range");
    const TileChoice saved = ctx->cone_tiles;
    ctx->cone_tiles = t;
    TileChoice d;
    if (vmc_tc_cone_applies(ctx) && vmc_tc_cone_default_tiles(ctx, &d) != VMC_OK) {
        ctx->cone_tiles = saved;
        return vmc_fail(ctx, VMC_ERR_UNSUPPORTED, "no light-cone plan with these tiles");
    }
    return VMC_OK;
}

int vmc_get_cone_tiles(const vmc_ctx *ctx, vmc_tiles *tiles)
{
    if (!ctx || !tiles) return VMC_ERR_ARG;
    TileChoice d;
    const int rc = vmc_tc_cone_default_tiles(ctx, &d);
    if (rc) return rc;
    tiles->slab_configs = d.slab_configs;
    tiles->slabs = d.slabs;
    tiles->ctas_per_sm = d.ctas_per_sm;
    tiles->lane_cells = d.lane_cells;
    return VMC_OK;
}

int64_t vmc_last_launch_count(const vmc_ctx *ctx) { return ctx ? ctx->launches : 0; }

const char *vmc_last_error(const vmc_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->last_error.c_str();
}

}  // extern "C"
