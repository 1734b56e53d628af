// lat_f16.cu -- the latency-mode generate kernel instantiated for __half output (a
// translation unit of its own, so it compiles in parallel with the others).
#include "wn_gen.cuh"

namespace wn {
cudaError_t launch_latency_f16(const GenArgs &a, const LaunchCfg &c, bool full, size_t smem, cudaStream_t cs)
{
    return launch_latency_t<__half>(a, c, full, smem, cs);
}
}  // namespace wn
