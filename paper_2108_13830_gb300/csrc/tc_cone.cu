// Kernel instantiations of the light-cone local energy: the parent pass
// (log|psi| with every layer's activations stored) and the neighbour pass.
// Kept apart from the plain forward so the two compile in parallel.
#include "tc_kern.cuh"

namespace vmc {
namespace tc {

int launch_store_var(vmc_ctx *ctx, const Plan &pl, const Params &p, cudaStream_t st)
{
    return launch_var<VAR_STORE>(ctx, pl, p, st);
}

int launch_cone_var(vmc_ctx *ctx, const Plan &pl, const Params &p, cudaStream_t st)
{
    return launch_var<VAR_CONE>(ctx, pl, p, st);
}

}  // namespace tc
}  // namespace vmc
