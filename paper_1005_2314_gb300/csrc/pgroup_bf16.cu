// pgroup_bf16.cu -- the persistent group-mode batch kernel instantiated for
// __nv_bfloat16 output (a translation unit of its own, so it compiles in parallel).
#include "wn_group.cuh"

namespace wn {
cudaError_t launch_persist_group_bf16(const GenArgs &a, const BatchArgs &bq, uint32_t N, uint32_t G, int sms,
                                     cudaStream_t cs)
{
    return launch_persist_group_t<__nv_bfloat16>(a, bq, N, G, sms, cs);
}
}  // namespace wn
