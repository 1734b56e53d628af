// boxmuller.cu -- the conventional comparison generator on GB300: Box-Muller
// (named in Section 5 of Brent, arXiv:1005.2314, among the older methods,
// with Section 4 on why transcendental-based methods are slower) fed by the
// counter-based Philox4x32-10 generator of Salmon et al. (SC'11).
//
// Each thread turns one Philox block (four 32-bit words) into four normals:
// words (w0, w1) and (w2, w3) each give u1 = ((w >> 8) + 1) 2^-24 in (0, 1],
// u2 = (w' >> 8) 2^-24 in [0, 1), rho = sqrt(-2 ln u1) and the pair
// (rho cos 2 pi u2, rho sin 2 pi u2).  The kernel is a grid-stride loop over
// each stream's blocks (grid rows are streams); four consecutive outputs go
// out as one 16-byte (FP32) or 8-byte (16-bit types) store when the
// destination allows it.
#include <string>

#include "wallace_gb300.h"
#include "wn_device.cuh"

namespace wn {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ float2 bm_pair(uint32_t wu, uint32_t wv)
{
    const float u1 = (float)((wu >> 8) + 1u) * 0x1p-24f;
    const float u2 = (float)(wv >> 8) * 0x1p-24f;
    const float rho = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    return make_float2(rho * c, rho * s);
}

template <typename OutT> struct Vec4;
template <> struct Vec4<float> {
    __device__ static void store(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
};
template <typename H> __device__ __forceinline__ void store_half4(H *p, float4 v)
{
    union {
        H h[4];
        uint2 u;
    } pk;
    pk.h[0] = to_out<H>(v.x);
    pk.h[1] = to_out<H>(v.y);
    pk.h[2] = to_out<H>(v.z);
    pk.h[3] = to_out<H>(v.w);
    *reinterpret_cast<uint2 *>(p) = pk.u;
}
template <> struct Vec4<__nv_bfloat16> {
    __device__ static void store(__nv_bfloat16 *p, float4 v) { store_half4(p, v); }
};
template <> struct Vec4<__half> {
    __device__ static void store(__half *p, float4 v) { store_half4(p, v); }
};

template <typename OutT>
__global__ void __launch_bounds__(256) boxmuller_kernel(OutT *__restrict__ out, uint64_t count,
                                                        uint32_t n_streams, uint64_t seed)
{
    const uint64_t mb = (count + 3) / 4;  // Philox blocks per stream
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const bool vec_ok = (count % 4 == 0) &&
                        (reinterpret_cast<uintptr_t>(out) % (4 * sizeof(OutT)) == 0);
    for (uint32_t stream = blockIdx.y; stream < n_streams; stream += gridDim.y) {
        OutT *os = out + (uint64_t)stream * count;
        for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < mb;
             m += (uint64_t)gridDim.x * blockDim.x) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)m, (uint32_t)(m >> 32), stream, 0u), key);
            const float2 p0 = bm_pair(w.x, w.y), p1 = bm_pair(w.z, w.w);
            OutT *o = os + 4 * m;
            if (vec_ok) {
                Vec4<OutT>::store(o, make_float4(p0.x, p0.y, p1.x, p1.y));
            } else {
                const float z[4] = {p0.x, p0.y, p1.x, p1.y};
                const uint64_t n = count - 4 * m < 4 ? count - 4 * m : 4;
                for (uint64_t i = 0; i < n; ++i) o[i] = to_out<OutT>(z[i]);
            }
        }
    }
}

}  // namespace wn

namespace wn {
wn_status set_error(wn_status st, const std::string &msg);  // wallace.cu
}

extern "C" wn_status wn_boxmuller(void *out, uint64_t count, uint32_t n_streams, uint64_t seed,
                                  wn_dtype dtype, void *cuda_stream)
{
    if (count == 0 || n_streams == 0) return WN_OK;
    if (!out || reinterpret_cast<uintptr_t>(out) % 16 != 0)
        return wn::set_error(WN_EINVAL, "wn_boxmuller: NULL or misaligned output");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return wn::set_error(WN_ECUDA, "wn_boxmuller: no CUDA device");
    // blocks: one row per stream (up to 65535, then rows loop), and along a
    // row enough blocks that the grid fills the GPU about eight CTAs per SM
    const uint64_t mb = (count + 3) / 4;
    const unsigned gy = n_streams < 65535u ? n_streams : 65535u;
    const uint64_t target = (uint64_t)sms * 8;
    uint64_t gx = (target + gy - 1) / gy;
    const uint64_t gx_max = (mb + 255) / 256;
    if (gx > gx_max) gx = gx_max;
    if (gx < 1) gx = 1;
    const dim3 grid((unsigned)gx, gy);
    switch (dtype) {
    case WN_F32: wn::boxmuller_kernel<float><<<grid, 256, 0, cs>>>((float *)out, count, n_streams, seed); break;
    case WN_BF16:
        wn::boxmuller_kernel<__nv_bfloat16><<<grid, 256, 0, cs>>>((__nv_bfloat16 *)out, count, n_streams, seed);
        break;
    case WN_F16: wn::boxmuller_kernel<__half><<<grid, 256, 0, cs>>>((__half *)out, count, n_streams, seed); break;
    default: return wn::set_error(WN_EINVAL, "wn_boxmuller: unknown dtype");
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return wn::set_error(WN_ECUDA, std::string("wn_boxmuller: ") + cudaGetErrorString(e));
    return WN_OK;
}
