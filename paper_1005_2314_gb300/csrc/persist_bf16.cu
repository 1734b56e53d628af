// persist_bf16.cu -- the persistent batch kernel instantiated for __nv_bfloat16 output (a
// translation unit of its own, so it compiles in parallel with the others).
#include "wn_gen.cuh"

namespace wn {
cudaError_t launch_persist_bf16(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, bool var,
                              size_t smem, int sms, cudaStream_t cs)
{
    return launch_persist_t<__nv_bfloat16>(a, bq, c, full, var, smem, sms, cs);
}
}  // namespace wn
