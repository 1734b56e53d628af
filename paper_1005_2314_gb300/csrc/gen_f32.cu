// gen_f32.cu -- the generate kernel instantiated for float output (one
// translation unit per output type and kernel kind, so they compile in parallel).
#include "wn_gen.cuh"

namespace wn {
cudaError_t launch_generate_f32(const GenArgs &a, const LaunchCfg &c, bool full, bool var, size_t smem,
                               cudaStream_t cs)
{
    return launch_generate_t<float>(a, c, full, var, smem, cs);
}

}  // namespace wn
