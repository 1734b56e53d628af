// emit_bf16.cu -- the latency-mode kernels (emitter warp) instantiated for __nv_bfloat16
// output (a translation unit of its own, so it compiles in parallel).
#include "wn_emit.cuh"

namespace wn {
cudaError_t launch_emit_bf16(const GenArgs &a, const LaunchCfg &c, bool full, size_t smem, cudaStream_t cs)
{
    return launch_emit_t<__nv_bfloat16>(a, c, full, smem, cs);
}

cudaError_t launch_persist_emit_bf16(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, size_t smem,
                                    int sms, cudaStream_t cs)
{
    return launch_persist_emit_t<__nv_bfloat16>(a, bq, c, full, smem, sms, cs);
}
}  // namespace wn
