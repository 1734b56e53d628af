// gen_f16.cu -- the generate kernel instantiated for __half output (one
// translation unit per output type, so the three compile in parallel).
#include "wn_gen.cuh"

namespace wn {
cudaError_t launch_generate_f16(const GenArgs &a, const LaunchCfg &c, bool full, bool var, size_t smem,
                               cudaStream_t cs)
{
    return launch_generate_t<__half>(a, c, full, var, smem, cs);
}

cudaError_t launch_persist_f16(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, bool var,
                              size_t smem, int sms, cudaStream_t cs)
{
    return launch_persist_t<__half>(a, bq, c, full, var, smem, sms, cs);
}
}  // namespace wn
