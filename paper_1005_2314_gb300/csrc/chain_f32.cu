// chain_f32.cu -- the chain-mode kernels (wn_chain.cuh) instantiated for
// float output (a translation unit of its own, so it compiles in parallel).
#include "wn_chain.cuh"

namespace wn {
cudaError_t launch_chain_f32(const GenArgs &a, uint32_t N, uint32_t G, size_t smem, cudaStream_t cs)
{
    return launch_chain_t<float>(a, N, G, smem, cs);
}

cudaError_t launch_persist_chain_f32(const GenArgs &a, const BatchArgs &bq, uint32_t N, uint32_t G, size_t smem,
                                     int sms, cudaStream_t cs)
{
    return launch_persist_chain_t<float>(a, bq, N, G, smem, sms, cs);
}
}  // namespace wn
