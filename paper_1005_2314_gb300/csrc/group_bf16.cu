// group_bf16.cu -- the group-mode generate kernel instantiated for __nv_bfloat16 output
// (a translation unit of its own, so it compiles in parallel with the others).
#include "wn_group.cuh"

namespace wn {
cudaError_t launch_group_bf16(const GenArgs &a, uint32_t N, uint32_t G, int sms, cudaStream_t cs,
                             uint32_t *ctas_per_sm)
{
    return launch_group_t<__nv_bfloat16>(a, N, G, sms, cs, ctas_per_sm);
}
}  // namespace wn
