// gen_f32.cu -- the generate kernel instantiated for float output (one
// translation unit per output type, so the three compile in parallel).
#include "wn_gen.cuh"

namespace wn {
cudaError_t launch_generate_f32(const GenArgs &a, const LaunchCfg &c, bool full, bool var, size_t smem,
                               cudaStream_t cs)
{
    return launch_generate_t<float>(a, c, full, var, smem, cs);
}

cudaError_t launch_persist_f32(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, bool var,
                              size_t smem, int sms, cudaStream_t cs)
{
    return launch_persist_t<float>(a, bq, c, full, var, smem, sms, cs);
}

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
    case 4: return launch_gbm_shape<4, 288, 3>(a, g, c.threads, full, smem, cs);
    case 8: return launch_gbm_shape<8, 544, 1>(a, g, c.threads, full, smem, cs);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace wn
