// pgroup_f16.cu -- the persistent group-mode batch kernel instantiated for
// __half output (a translation unit of its own, so it compiles in parallel).
#include "wn_group.cuh"

namespace wn {
cudaError_t launch_persist_group_f16(const GenArgs &a, const BatchArgs &bq, uint32_t N, uint32_t G, int sms,
                                     cudaStream_t cs)
{
    return launch_persist_group_t<__half>(a, bq, N, G, sms, cs);
}
}  // namespace wn
