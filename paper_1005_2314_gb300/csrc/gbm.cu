// gbm.cu -- the fused GBM consumer kernel (FP32 sums; a translation unit of
// its own, so it compiles in parallel with the others).
#include "wn_gen.cuh"

namespace wn {
template <int QT, int MAXT, int MINB>
static cudaError_t launch_gbm_shape(const GenArgs &a, const GbmArgs &g, uint32_t threads, bool full, size_t smem,
                                    cudaStream_t cs)
{
    auto kern = full ? gbm_kernel<QT, MAXT, MINB, true> : gbm_kernel<QT, MAXT, MINB, false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<a.n_streams, threads + 32, smem, cs>>>(a, g);  // + the control warp
    return cudaGetLastError();
}

cudaError_t launch_gbm(const GenArgs &a, const GbmArgs &g, const LaunchCfg &c, bool full, size_t smem,
                       cudaStream_t cs)
{
    switch (c.qt) {
    case 1: return launch_gbm_shape<1, 1024, 1>(a, g, c.threads, full, smem, cs);
#ifndef WN_DEBUG
    case 4: return launch_gbm_shape<4, 288, 3>(a, g, c.threads, full, smem, cs);
#endif
#ifndef WN_DEBUG
    case 8: return launch_gbm_shape<8, 544, 1>(a, g, c.threads, full, smem, cs);
#endif
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace wn
