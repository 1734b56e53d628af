// gen_f16.cu -- the generate kernel instantiated for __half output (one
// translation unit per output type and kernel kind, so they compile in parallel).
#include "wn_gen.cuh"

namespace wn {
cudaError_t launch_generate_f16(const GenArgs &a, const LaunchCfg &c, bool full, bool var, size_t smem,
                               cudaStream_t cs)
{
    return launch_generate_t<__half>(a, c, full, var, smem, cs);
}

}  // namespace wn
