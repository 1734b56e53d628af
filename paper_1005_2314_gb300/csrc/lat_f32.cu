// lat_f32.cu -- the latency-mode generate and persistent kernels for float
// output (a translation unit of its own, so it compiles in parallel).
#include "wn_gen.cuh"

namespace wn {
cudaError_t launch_latency_f32(const GenArgs &a, const LaunchCfg &c, bool full, size_t smem, cudaStream_t cs)
{
    return launch_latency_t<float>(a, c, full, smem, cs);
}

cudaError_t launch_persist_lat_f32(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, size_t smem,
                                  int sms, cudaStream_t cs)
{
    return launch_persist_lat_t<float>(a, bq, c, full, smem, sms, cs);
}
}  // namespace wn
