// group_f16.cu -- the group-mode generate kernel instantiated for __half output
// (a translation unit of its own, so it compiles in parallel with the others).
#include "wn_group.cuh"

namespace wn {
cudaError_t launch_group_f16(const GenArgs &a, uint32_t N, uint32_t G, int sms, cudaStream_t cs,
                             uint32_t *ctas_per_sm)
{
    return launch_group_t<__half>(a, N, G, sms, cs, ctas_per_sm);
}
}  // namespace wn
