// Diagnostics of the tcgen05 path: issue-rate probe of back-to-back UMMAs.
//
// Each CTA issues `count` MMAs of shape 128 x N x 16 (BF16, FP32 accumulate)
// from zero-filled shared-memory operands into one TMEM accumulator, commits
// once and waits (bounded).  Cycles between the first issue and the commit's
// completion give the per-instruction cost for that N.
#include <vector>
#include "vmc_internal.h"
#include "tc_layout.cuh"
#include "tc_ptx.cuh"

namespace vmc {

__global__ void umma_rate_kernel(int N, int count, unsigned long long *cycles, int *status)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    __shared__ int abort_flag, wfl, wsite;   // the wait may raise status bits atomically
    const int tid = threadIdx.x, warp = tid >> 5;
    // A: 4 K-chunks of 128 rows (plane per 8 channels: 8 planes of 2 KB);
    // B: 4 K-chunks of N rows (32 N bytes each)
    uint8_t *As = sm;
    uint8_t *Bs = sm + 16384;
    for (int i = tid; i < (16384 + 4 * 32 * N) / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) { mbar_init(&bar, 1); mbar_fence_init(); abort_flag = 0; wfl = 0; wsite = 0; }
    fence_proxy_async_smem();
    if (warp == 0) tmem_alloc(&tbase, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        const uint32_t idesc = idesc_bf16(128, N);
        const uint32_t a = smem_u32(As), b = smem_u32(Bs);
        const unsigned long long t0 = clock64();
        for (int i = 0; i < count; ++i) {
            const int kc = i & 3;
            umma_bf16(tbase, smem_desc(a + kc * 4096, 2048, 128), smem_desc(b + kc * 32 * N, 16 * N, 128), idesc,
                      i > 0);
        }
        umma_commit(&bar);
        mbar_wait_bounded(&bar, 0, &abort_flag, 2000000000LL, &wfl, &wsite, 0);
        const int fl = wfl;
        const unsigned long long t1 = clock64();
        cycles[blockIdx.x] = t1 - t0;
        if (fl) atomicOr(status, fl);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tbase, 256);
}

}  // namespace vmc

extern "C" int vmc_debug_umma_rate(int N, int count, int ctas, double *cycles_per_mma, double *ms)
{
    if (N < 16 || N > 256 || N % 16 || count < 1 || count > (1 << 20) || ctas < 1 || ctas > 1024 ||
        !cycles_per_mma || !ms)
        return VMC_ERR_ARG;
    unsigned long long *cyc = nullptr;
    int *st = nullptr;
    if (cudaMalloc(&cyc, sizeof(unsigned long long) * ctas) != cudaSuccess) return VMC_ERR_CUDA;
    if (cudaMalloc(&st, sizeof(int)) != cudaSuccess) { cudaFree(cyc); return VMC_ERR_CUDA; }
    cudaMemset(st, 0, sizeof(int));
    const size_t smem = 16384 + 4 * 32 * (size_t)N;
    cudaFuncSetAttribute(vmc::umma_rate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    vmc::umma_rate_kernel<<<ctas, 128, smem>>>(N, count, cyc, st);   // warm-up
    cudaEventRecord(e0);
    vmc::umma_rate_kernel<<<ctas, 128, smem>>>(N, count, cyc, st);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    std::vector<unsigned long long> h(ctas);
    int hs = 0;
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, sizeof(unsigned long long) * ctas, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&hs, st, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(cyc);
    cudaFree(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return VMC_ERR_CUDA;
    double s = 0;
    for (auto v : h) s += (double)v;
    *cycles_per_mma = s / ctas / count;
    *ms = t;
    return hs ? VMC_ERR_TIMEOUT : VMC_OK;
}
