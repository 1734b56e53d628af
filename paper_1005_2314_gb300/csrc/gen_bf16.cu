// gen_bf16.cu -- the generate kernel instantiated for __nv_bfloat16 output (one
// translation unit per output type, so the three compile in parallel).
#include "wn_gen.cuh"

namespace wn {
cudaError_t launch_generate_bf16(const GenArgs &a, const LaunchCfg &c, bool full, bool var, size_t smem,
                               cudaStream_t cs)
{
    return launch_generate_t<__nv_bfloat16>(a, c, full, var, smem, cs);
}

cudaError_t launch_persist_bf16(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, bool var,
                              size_t smem, int sms, cudaStream_t cs)
{
    return launch_persist_t<__nv_bfloat16>(a, bq, c, full, var, smem, sms, cs);
}
}  // namespace wn
