// out = O^T w without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside an allocator
// callback or a memory-pool hook, embedded runtimes that forbid device
// allocation after start-up, or processes whose memory budget is fixed when
// the module loads.  They cannot create a vmc context either (vmc_create and
// the workspaces allocate), so this entry point takes only plain pointers and
// keeps its scratch in a fixed, file-scope device array that exists from the
// moment the library's module is loaded on a device until the process exits.
//
// The arithmetic is that of vmc_ot_vec: w is split into FP32 (hi, lo) pairs,
// each CTA column block accumulates sum_b O_bk (hi_b + lo_b) over one chunk of
// rows in double-float, and the chunk partials are summed in FP64.
#include "vmc_internal.h"

// Scratch shared by every call on a device: the split w (2 m floats) followed
// by the per-chunk column partials (nchunk n doubles).  Nothing in it has to
// start at zero: every call writes each entry it reads.
#define VMC_NOALLOC_SCRATCH_BYTES (16u << 20)
static __device__ __align__(256) unsigned char g_ot_scratch[VMC_NOALLOC_SCRATCH_BYTES];

namespace {

__device__ __forceinline__ void na_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__global__ void na_split_kernel(const double *__restrict__ w, int64_t m, float *wh, float *wl)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m; b += (int64_t)gridDim.x * blockDim.x) {
        const float h = (float)w[b];
        wh[b] = h;
        wl[b] = (float)(w[b] - (double)h);
    }
}

// part[chunk][k] = sum over the chunk's rows of O_bk (wh_b + wl_b)
__global__ void na_colsum_kernel(const float *__restrict__ O, int64_t m, int64_t n, int64_t rows_per_chunk,
                                 const float *__restrict__ wh, const float *__restrict__ wl, double *part)
{
    const int64_t chunk = blockIdx.y;
    const int64_t r0 = chunk * rows_per_chunk;
    const int64_t r1 = r0 + rows_per_chunk < m ? r0 + rows_per_chunk : m;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    float sh = 0.f, sl = 0.f;
    for (int64_t b = r0; b < r1; ++b) {
        const float x = __ldg(O + b * n + k);
        const float yh = wh[b], yl = wl[b];
        const float p = x * yh;
        float pe = fmaf(x, yh, -p);
        pe = fmaf(x, yl, pe);
        float s, e;
        na_two_sum(sh, p, s, e);
        e += sl + pe;
        sh = s + e;
        sl = e - (sh - s);
    }
    part[chunk * n + k] = (double)sh + (double)sl;
}

__global__ void na_reduce_kernel(const double *__restrict__ part, int nchunk, int64_t n, double *out)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < nchunk; ++c) acc += part[(int64_t)c * n + k];
        out[k] = acc;
    }
}

}  // namespace

extern "C" int vmc_ot_vec_noalloc(const float *O_dev, int64_t m, int64_t n, const double *w_dev,
                                  double *out_dev, void *stream)
{
    if (!O_dev || !w_dev || !out_dev || m < 1 || n < 1) return VMC_ERR_ARG;
    // beyond the fixed scratch: refuse before any byte arithmetic (which could
    // wrap for huge m or n) and before touching the device
    const int64_t cap = (int64_t)VMC_NOALLOC_SCRATCH_BYTES;
    if (m > cap / 8 || n > cap / 8) return VMC_ERR_UNSUPPORTED;
    const int64_t nchunk = m >= 1024 ? 16 : (m >= 64 ? 4 : 1);
    const int64_t w_bytes = (2 * m * (int64_t)sizeof(float) + 255) & ~(int64_t)255;
    if (w_bytes + nchunk * n * 8 > cap) return VMC_ERR_UNSUPPORTED;
    // The device address of the scratch array, looked up on every call with
    // the caller's device and context current (the host-side symbol is only
    // a stand-in).  Once the module is loaded this allocates nothing; a
    // cached address would go stale after cudaDeviceReset or under another
    // driver-API context, each of which has its own copy of the array.
    void *base = nullptr;
    if (cudaGetSymbolAddress(&base, g_ot_scratch) != cudaSuccess || !base) return VMC_ERR_CUDA;
    char *b = static_cast<char *>(base);
    float *wh = reinterpret_cast<float *>(b);
    float *wl = wh + m;
    double *part = reinterpret_cast<double *>(b + w_bytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t rpc = (m + nchunk - 1) / nchunk;
    na_split_kernel<<<(unsigned)((m + 255) / 256 < 1024 ? (m + 255) / 256 : 1024), 256, 0, s>>>(w_dev, m, wh, wl);
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)nchunk);
    na_colsum_kernel<<<grid, 256, 0, s>>>(O_dev, m, n, rpc, wh, wl, part);
    na_reduce_kernel<<<(unsigned)((n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048), 256, 0, s>>>(part, (int)nchunk, n,
                                                                                                  out_dev);
    return cudaGetLastError() == cudaSuccess ? VMC_OK : VMC_ERR_CUDA;
}
