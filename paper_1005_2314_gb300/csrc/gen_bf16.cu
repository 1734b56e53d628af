// gen_bf16.cu -- the generate kernel instantiated for __nv_bfloat16 output (one
// translation unit per output type and kernel kind, so they compile in parallel).
#include "wn_gen.cuh"

namespace wn {
cudaError_t launch_generate_bf16(const GenArgs &a, const LaunchCfg &c, bool full, bool var, size_t smem,
                               cudaStream_t cs)
{
    return launch_generate_t<__nv_bfloat16>(a, c, full, var, smem, cs);
}

}  // namespace wn
