// wallace.cu -- GB300 (sm_103a) kernels and host runtime of Wallace's
// maximum-entropy normal generator (Brent, arXiv:1005.2314, Section 5).
//
// One CTA owns one stream: the stream's pool lives in shared memory for the
// whole call while the CTA runs its blocks back to back.  A pass gathers each
// quadruple through the affine permutation j -> alpha*j + gamma (mod N)
// (Section 5.4), applies y_k = s_k (t - a_k), t = (a_0+a_1+a_2+a_3)/2
// (Sections 5.2-5.3), and stores the four results contiguously (the
// transposed write).  Consecutive lanes take consecutive quadruples, so with
// alpha odd a warp's 32 gathers of one k fall in 32 distinct banks, and its
// 32 float4 stores cover 512 contiguous bytes: both are conflict-free.
// After the R passes of a block, the pool's sum of squares is reduced (FP32
// per warp, FP64 across warps) and one warp forms the output scale
// sqrt(S / sum of squares) in FP64 from the chi-squared approximation (c) of
// Section 5.5, driven by the previous block's reserved value.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "wallace_gb300.h"
#include "wn_device.cuh"

namespace wn {

struct GenArgs {
    StreamHdr *hdr;
    float *pools;
    void *out;
    uint64_t count;          // values per stream
    uint64_t out_stride;     // elements between consecutive streams' outputs
    uint32_t n_streams;
    uint32_t n_max;          // largest pool of the launch (shared-memory layout)
    uint32_t warmup_blocks;  // nonzero: discard this many whole blocks, store nothing
};

// Shared memory of a generate CTA whose launch's largest pool is n_max and
// largest pass count r_max: two pool buffers, 32 warp partial sums, the block
// scale, and the 2 r_max draws of the coming block.
__host__ __device__ inline size_t gen_smem_bytes(uint32_t n_max, uint32_t r_max)
{
    return (size_t)8 * n_max + 128 + 16 + (size_t)16 * r_max;
}

// ---------------------------------------------------------------------------
// Initialisation (Section 5.8): seed, N draws -> v_i = 2 (sum of the four
// 16-bit fields) - 4*65535, scale so that sum v_i^2 = N.  The v_i and their
// squares are integers, so the sum is exact and the FP64 scale is the
// correctly rounded sqrt(N / sum); each pool value is the FP32 rounding of the
// FP64 product.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32) init_kernel(StreamHdr *hdr, float *pools)
{
    extern __shared__ int32_t vsm[];
    StreamHdr *h = hdr + blockIdx.x;
    const uint32_t N = h->N, lane = threadIdx.x;
    uint64_t x = 0, w = 0;
    if (lane == 0) {
        seed_gen(h->x, x, w);
        for (uint32_t i = 0; i < N; ++i) {
            const uint64_t u = draw(x, w);
            const int32_t f = (int32_t)(u & 0xFFFFu) + (int32_t)((u >> 16) & 0xFFFFu) +
                              (int32_t)((u >> 32) & 0xFFFFu) + (int32_t)(u >> 48);
            vsm[i] = 2 * f - 4 * 65535;
        }
    }
    __syncwarp();
    long long ss = 0;
    for (uint32_t i = lane; i < N; i += 32) ss += (long long)vsm[i] * vsm[i];
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const double scale = sqrt((double)N / (double)ss);
    float *P = pools + h->pool_off;
    for (uint32_t i = lane; i < N; i += 32) P[i] = (float)((double)vsm[i] * scale);
    if (lane == 0) {
        const double nu = (double)N;
        const double A = 2.0 * sqrt(nu) * sin(asin(1.0 / sqrt(nu)) / 3.0);
        h->x = x;
        h->w = w;
        h->r = 0.0;
        h->A = A;
        h->B = sqrt(2.0 * (nu - A * A));
        h->blocks = 0;
        h->scale = 1.0f;
        h->k = N - 1;
    }
}

// ---------------------------------------------------------------------------
// One stream's share of a call: return the rest of the last block, then run
// as many whole blocks as `count` needs, then write the state back.
// QT = quadruples per thread (compile-time bound); blockDim.x is a multiple
// of 32 with blockDim.x * QT >= N/4.
// ---------------------------------------------------------------------------
template <int QT, typename OutT>
__device__ __forceinline__ void run_stream(StreamHdr *__restrict__ h, float *__restrict__ pool_g,
                                           OutT *__restrict__ out, uint64_t count, bool store,
                                           uint32_t n_max)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t T = blockDim.x, tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5, nw = T >> 5;
    const uint32_t N = h->N, R = h->R, nq = N >> 2, mask = N - 1;
    float *buf0 = reinterpret_cast<float *>(smem);
    float *buf1 = buf0 + n_max;
    float *red = buf0 + 2 * (size_t)n_max;
    float *sc_sm = red + 32;
    uint64_t *dr = reinterpret_cast<uint64_t *>(sc_sm + 4);

    {
        const float4 *pg4 = reinterpret_cast<const float4 *>(pool_g);
        float4 *b04 = reinterpret_cast<float4 *>(buf0);
        for (uint32_t i = tid; i < nq; i += T) b04[i] = pg4[i];
    }
    const uint32_t k0 = h->k;
    const float sc_prev = h->scale;
    const uint64_t left = (uint64_t)(N - 1 - k0);
    const uint64_t n0 = left < count ? left : count;
    const uint64_t nb = (count - n0 + (N - 2)) / (N - 1);

    // Warp 0 owns the generator, the reserved value and the chi-squared
    // constants; it publishes each block's draws through shared memory.
    uint64_t gx = 0, gw = 0;
    double r = 0.0, A = 0.0, B = 0.0;
    const double invN = 1.0 / (double)N;
    if (warp == 0) {
        gx = h->x;
        gw = h->w;
        r = h->r;
        A = h->A;
        B = h->B;
        if (nb > 0)
            for (uint32_t i = 0; i < 2 * R; ++i) {
                const uint64_t d = draw(gx, gw);
                if (lane == (i & 31u)) dr[i] = d;
            }
    }
    __syncthreads();
    if (store)
        for (uint64_t i = tid; i < n0; i += T) out[i] = to_out<OutT>(sc_prev * buf0[k0 + i]);

    float *cur = buf0, *nxt = buf1;
    uint64_t emitted = n0;
    uint32_t last_n = 0;
    float last_sc = sc_prev;
    const uint32_t sh = 4u * (tid & 15u);  // nibble of quadruple q: q mod 16 = tid mod 16

    for (uint64_t b = 0; b < nb; ++b) {
        float part = 0.f;
        for (uint32_t p = 0; p < R; ++p) {
            const uint64_t wa = dr[2 * p], ws = dr[2 * p + 1];
            const uint32_t alpha = ((uint32_t)(wa >> 32) & mask) | 1u;
            const uint32_t o0 = (uint32_t)wa & mask;
            const uint32_t o1 = (alpha * nq + o0) & mask;
            const uint32_t o2 = (2u * alpha * nq + o0) & mask;
            const uint32_t o3 = (3u * alpha * nq + o0) & mask;
            const uint32_t nib = (uint32_t)(ws >> sh) & 15u;
            const uint32_t s0 = (nib & 1u) << 31, s1 = ((nib >> 1) & 1u) << 31;
            const uint32_t s2 = ((nib >> 2) & 1u) << 31, s3 = (nib >> 3) << 31;
            float4 *n4 = reinterpret_cast<float4 *>(nxt);
            const bool last = (p + 1 == R);
#pragma unroll
            for (int j = 0; j < QT; ++j) {
                const uint32_t q = tid + (uint32_t)j * T;
                if (q < nq) {
                    const uint32_t base = alpha * q;
                    const float a0 = cur[(base + o0) & mask];
                    const float a1 = cur[(base + o1) & mask];
                    const float a2 = cur[(base + o2) & mask];
                    const float a3 = cur[(base + o3) & mask];
                    const float t = 0.5f * ((a0 + a1) + (a2 + a3));
                    float4 y;
                    y.x = __uint_as_float(__float_as_uint(t - a0) ^ s0);
                    y.y = __uint_as_float(__float_as_uint(t - a1) ^ s1);
                    y.z = __uint_as_float(__float_as_uint(t - a2) ^ s2);
                    y.w = __uint_as_float(__float_as_uint(t - a3) ^ s3);
                    n4[q] = y;
                    if (last) part = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, part))));
                }
            }
            float *tmp = cur;
            cur = nxt;
            nxt = tmp;
            if (last) {
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                if (lane == 0) red[warp] = part;
            }
            __syncthreads();
        }
        if (warp == 0) {
            double v = (lane < nw) ? (double)red[lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            const double den = v * invN;                      // pool sum of squares / N
            const double u = fma(A, fma(r, r, -1.0), B * r);  // S - N
            const double num = fma(u, invN, 1.0);             // S / N
            const double s = num * rsqrt_nr(num * den);       // sqrt(S / sum of squares)
            r = s * (double)cur[N - 1];                       // held back for the next block
            if (lane == 0) *sc_sm = (float)s;
            if (b + 1 < nb)
                for (uint32_t i = 0; i < 2 * R; ++i) {
                    const uint64_t d = draw(gx, gw);
                    if (lane == (i & 31u)) dr[i] = d;
                }
        }
        __syncthreads();
        const float sc = *sc_sm;
        const uint64_t rem = count - emitted;
        const uint32_t n = rem < (uint64_t)(N - 1) ? (uint32_t)rem : (N - 1);
        if (store) {
            OutT *o = out + emitted;
            for (uint32_t i = tid; i < n; i += T) o[i] = to_out<OutT>(sc * cur[i]);
        }
        emitted += n;
        last_n = n;
        last_sc = sc;
    }

    {
        float4 *pw4 = reinterpret_cast<float4 *>(pool_g);
        const float4 *c4 = reinterpret_cast<const float4 *>(cur);
        for (uint32_t i = tid; i < nq; i += T) pw4[i] = c4[i];
    }
    if (tid == 0) {
        h->x = gx;
        h->w = gw;
        h->r = r;
        if (nb > 0) {
            h->scale = last_sc;
            h->k = last_n;
        } else {
            h->k = k0 + (uint32_t)n0;
        }
        h->blocks += nb;
    }
}

template <int QT, typename OutT>
__global__ void __launch_bounds__(1024) generate_kernel(GenArgs a)
{
    StreamHdr *h = a.hdr + blockIdx.x;
    const uint32_t N = h->N;
    const uint64_t count = a.warmup_blocks ? (uint64_t)a.warmup_blocks * (N - 1) : a.count;
    OutT *out = a.out ? reinterpret_cast<OutT *>(a.out) + (uint64_t)blockIdx.x * a.out_stride : nullptr;
    run_stream<QT, OutT>(h, a.pools + h->pool_off, out, count, a.warmup_blocks == 0, a.n_max);
}

__global__ void draws_kernel(uint64_t seed, uint64_t n, uint64_t *out)
{
    uint64_t x, w;
    seed_gen(seed, x, w);
    for (uint64_t i = 0; i < n; ++i) out[i] = draw(x, w);
}

}  // namespace wn

// ===========================================================================
// Host runtime and C ABI.
// ===========================================================================

struct wn_stream {
    int device = 0;
    uint32_t n = 0;
    uint32_t n_max = 0, r_max = 0;
    wn::StreamHdr *d_hdr = nullptr;
    float *d_pools = nullptr;
    cudaStream_t cs = nullptr;
    std::vector<uint32_t> N, R;
    // host delivery (wn_generate_host): staging buffers, copy stream, events
    void *d_stage[2] = {nullptr, nullptr};
    size_t stage_bytes = 0;
    cudaStream_t copy_cs = nullptr;
    cudaEvent_t ev_gen[2] = {nullptr, nullptr}, ev_copy[2] = {nullptr, nullptr};
};

namespace {
thread_local std::string g_err;
}  // namespace

namespace wn {
// Records the calling thread's error text for wn_last_error().
wn_status set_error(wn_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}
}  // namespace wn

namespace {

wn_status fail(wn_status st, const std::string &msg) { return wn::set_error(st, msg); }

wn_status cuda_fail(const char *what, cudaError_t e)
{
    return fail(WN_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define WN_CU(call)                                      \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(#call, e_); \
    } while (0)

bool valid_pool(uint32_t N) { return N >= WN_MIN_POOL && N <= WN_MAX_POOL && (N & (N - 1)) == 0; }
bool valid_passes(uint32_t R) { return R >= 1 && R <= WN_MAX_PASSES; }

struct LaunchCfg {
    int qt;
    uint32_t threads;
};

// Threads and quadruples per thread for a launch whose largest pool is n_max:
// one quadruple per thread up to N = 1024 (at least one full warp), four above.
LaunchCfg pick_cfg(uint32_t n_max)
{
    const uint32_t nq = n_max / 4;
    if (nq <= 256) return {1, std::max(32u, (nq + 31u) / 32u * 32u)};
    return {4, nq / 4};
}

template <int QT, typename OutT>
cudaError_t launch_gen(const wn::GenArgs &a, uint32_t threads, size_t smem, cudaStream_t cs)
{
    auto kern = wn::generate_kernel<QT, OutT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<a.n_streams, threads, smem, cs>>>(a);
    return cudaGetLastError();
}

template <typename OutT>
cudaError_t launch_gen_t(const wn::GenArgs &a, const LaunchCfg &c, size_t smem, cudaStream_t cs)
{
    switch (c.qt) {
    case 1: return launch_gen<1, OutT>(a, c.threads, smem, cs);
    case 4: return launch_gen<4, OutT>(a, c.threads, smem, cs);
    default: return cudaErrorInvalidValue;
    }
}

wn_status launch_generate(wn_stream *s, void *out, uint64_t count, uint32_t warmup, wn_dtype dt,
                          cudaStream_t cs)
{
    wn::GenArgs a;
    a.hdr = s->d_hdr;
    a.pools = s->d_pools;
    a.out = out;
    a.count = count;
    a.out_stride = count;
    a.n_streams = s->n;
    a.n_max = s->n_max;
    a.warmup_blocks = warmup;
    const LaunchCfg c = pick_cfg(s->n_max);
    const size_t smem = wn::gen_smem_bytes(s->n_max, s->r_max);
    cudaError_t e;
    switch (dt) {
    case WN_F32: e = launch_gen_t<float>(a, c, smem, cs); break;
    case WN_BF16: e = launch_gen_t<__nv_bfloat16>(a, c, smem, cs); break;
    case WN_F16: e = launch_gen_t<__half>(a, c, smem, cs); break;
    default: return fail(WN_EINVAL, "unknown dtype");
    }
    if (e != cudaSuccess) return cuda_fail("generate launch", e);
    return WN_OK;
}

}  // namespace

extern "C" {

const char *wn_last_error(void) { return g_err.c_str(); }

wn_stream *wn_create_streams(uint32_t n_streams, const uint32_t *pool_N, const uint32_t *passes_R,
                             const uint64_t *seeds, uint32_t warmup_blocks, void *cuda_stream)
{
    g_err.clear();
    if (n_streams == 0 || !pool_N || !passes_R || !seeds) {
        fail(WN_EINVAL, "wn_create_streams: empty stream set or NULL array");
        return nullptr;
    }
    wn_stream *s = new wn_stream();
    s->n = n_streams;
    s->N.assign(pool_N, pool_N + n_streams);
    s->R.assign(passes_R, passes_R + n_streams);
    std::vector<wn::StreamHdr> h(n_streams);
    uint64_t off = 0;
    for (uint32_t i = 0; i < n_streams; ++i) {
        if (!valid_pool(pool_N[i]) || !valid_passes(passes_R[i])) {
            fail(WN_EINVAL, "wn_create_streams: stream " + std::to_string(i) +
                                ": pool_N must be a power of two in [4, 16384] and passes_R in [1, 64]");
            delete s;
            return nullptr;
        }
        std::memset(&h[i], 0, sizeof(h[i]));
        h[i].x = seeds[i];  // consumed by the init kernel
        h[i].N = pool_N[i];
        h[i].R = passes_R[i];
        h[i].pool_off = off;
        off += pool_N[i];
        s->n_max = std::max(s->n_max, pool_N[i]);
        s->r_max = std::max(s->r_max, passes_R[i]);
    }
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_hdr, sizeof(wn::StreamHdr) * n_streams);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_pools, sizeof(float) * off);
    if (e != cudaSuccess) {
        cuda_fail("wn_create_streams: allocation", e);
        wn_destroy(s);
        return nullptr;
    }
    e = cudaMemcpyAsync(s->d_hdr, h.data(), sizeof(wn::StreamHdr) * n_streams, cudaMemcpyHostToDevice, cs);
    const size_t ismem = sizeof(int32_t) * s->n_max;
    if (e == cudaSuccess && ismem > 48 * 1024)
        e = cudaFuncSetAttribute(wn::init_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem);
    if (e == cudaSuccess) {
        wn::init_kernel<<<n_streams, 32, ismem, cs>>>(s->d_hdr, s->d_pools);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cuda_fail("wn_create_streams: init", e);
        wn_destroy(s);
        return nullptr;
    }
    if (warmup_blocks > 0 && launch_generate(s, nullptr, 0, warmup_blocks, WN_F32, cs) != WN_OK) {
        wn_destroy(s);
        return nullptr;
    }
    e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        cuda_fail("wn_create_streams: synchronize", e);
        wn_destroy(s);
        return nullptr;
    }
    return s;
}

wn_stream *wn_create(uint32_t pool_N, uint32_t passes_R, uint64_t seed)
{
    return wn_create_streams(1, &pool_N, &passes_R, &seed, WN_DEFAULT_WARMUP, nullptr);
}

void wn_destroy(wn_stream *s)
{
    if (!s) return;
    if (s->d_hdr || s->d_pools) cudaDeviceSynchronize();
    if (s->d_hdr) cudaFree(s->d_hdr);
    if (s->d_pools) cudaFree(s->d_pools);
    for (int b = 0; b < 2; ++b) {
        if (s->d_stage[b]) cudaFree(s->d_stage[b]);
        if (s->ev_gen[b]) cudaEventDestroy(s->ev_gen[b]);
        if (s->ev_copy[b]) cudaEventDestroy(s->ev_copy[b]);
    }
    if (s->copy_cs) cudaStreamDestroy(s->copy_cs);
    delete s;
}

wn_status wn_set_cuda_stream(wn_stream *s, void *cuda_stream)
{
    if (!s) return fail(WN_EINVAL, "wn_set_cuda_stream: NULL handle");
    s->cs = reinterpret_cast<cudaStream_t>(cuda_stream);
    return WN_OK;
}

uint32_t wn_num_streams(const wn_stream *s) { return s ? s->n : 0; }

wn_status wn_generate_ex(void *out, uint64_t count, wn_stream *s, wn_dtype dtype, void *cuda_stream)
{
    if (!s) return fail(WN_EINVAL, "wn_generate: NULL handle");
    if (dtype != WN_F32 && dtype != WN_BF16 && dtype != WN_F16) return fail(WN_EINVAL, "wn_generate: unknown dtype");
    if (count == 0) return WN_OK;
    if (!out) return fail(WN_EINVAL, "wn_generate: NULL output");
    if (reinterpret_cast<uintptr_t>(out) % 16 != 0) return fail(WN_EINVAL, "wn_generate: output not 16-byte aligned");
    return launch_generate(s, out, count, 0, dtype, reinterpret_cast<cudaStream_t>(cuda_stream));
}

wn_status wn_generate_host(void *host_out, uint64_t count, wn_stream *s, wn_dtype dtype, void *cuda_stream)
{
    if (!s) return fail(WN_EINVAL, "wn_generate_host: NULL handle");
    if (dtype != WN_F32 && dtype != WN_BF16 && dtype != WN_F16) return fail(WN_EINVAL, "wn_generate_host: unknown dtype");
    if (count == 0) return WN_OK;
    if (!host_out) return fail(WN_EINVAL, "wn_generate_host: NULL output");
    const size_t esize = dtype == WN_F32 ? 4 : 2;
    const size_t kStageMax = size_t(256) << 20;
    if (!s->d_stage[0]) {
        // per-stream chunk: a multiple of 8 values so each stream's slice of a
        // staging buffer stays 16-byte aligned
        s->stage_bytes = kStageMax;
        for (int b = 0; b < 2; ++b) {
            WN_CU(cudaMalloc(&s->d_stage[b], s->stage_bytes));
            WN_CU(cudaEventCreateWithFlags(&s->ev_gen[b], cudaEventDisableTiming));
            WN_CU(cudaEventCreateWithFlags(&s->ev_copy[b], cudaEventDisableTiming));
        }
        WN_CU(cudaStreamCreateWithFlags(&s->copy_cs, cudaStreamNonBlocking));
    }
    uint64_t chunk = s->stage_bytes / (esize * (uint64_t)s->n) / 8 * 8;
    if (chunk == 0) return fail(WN_EINVAL, "wn_generate_host: too many streams for the staging buffer");
    if (chunk > count) chunk = count;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(cuda_stream);
    unsigned char *dst = static_cast<unsigned char *>(host_out);
    uint64_t done = 0;
    for (int j = 0; done < count; ++j) {
        const int b = j & 1;
        const uint64_t c = std::min<uint64_t>(chunk, count - done);
        if (j >= 2) WN_CU(cudaStreamWaitEvent(cs, s->ev_copy[b], 0));
        wn_status st = launch_generate(s, s->d_stage[b], c, 0, dtype, cs);
        if (st != WN_OK) return st;
        WN_CU(cudaEventRecord(s->ev_gen[b], cs));
        WN_CU(cudaStreamWaitEvent(s->copy_cs, s->ev_gen[b], 0));
        WN_CU(cudaMemcpy2DAsync(dst + done * esize, count * esize, s->d_stage[b], c * esize, c * esize, s->n,
                                cudaMemcpyDeviceToHost, s->copy_cs));
        WN_CU(cudaEventRecord(s->ev_copy[b], s->copy_cs));
        done += c;
    }
    // later work on cuda_stream (and its synchronisation) follows the copies
    for (int b = 0; b < 2; ++b) WN_CU(cudaStreamWaitEvent(cs, s->ev_copy[b], 0));
    return WN_OK;
}

wn_status wn_generate(void *out, uint64_t count, wn_stream *s)
{
    if (!s) return fail(WN_EINVAL, "wn_generate: NULL handle");
    return wn_generate_ex(out, count, s, WN_F32, s->cs);
}

wn_status wn_get_pool(const wn_stream *s, uint32_t i, float *host_out)
{
    if (!s || !host_out || i >= s->n) return fail(WN_EINVAL, "wn_get_pool: bad handle, index or pointer");
    wn::StreamHdr h;
    WN_CU(cudaDeviceSynchronize());
    WN_CU(cudaMemcpy(&h, s->d_hdr + i, sizeof(h), cudaMemcpyDeviceToHost));
    WN_CU(cudaMemcpy(host_out, s->d_pools + h.pool_off, sizeof(float) * h.N, cudaMemcpyDeviceToHost));
    return WN_OK;
}

wn_status wn_get_state(const wn_stream *s, uint32_t i, uint64_t *host_xw, double *host_r, float *host_scale,
                       uint32_t *host_k, uint64_t *host_blocks)
{
    if (!s || i >= s->n) return fail(WN_EINVAL, "wn_get_state: bad handle or index");
    wn::StreamHdr h;
    WN_CU(cudaDeviceSynchronize());
    WN_CU(cudaMemcpy(&h, s->d_hdr + i, sizeof(h), cudaMemcpyDeviceToHost));
    if (host_xw) {
        host_xw[0] = h.x;
        host_xw[1] = h.w;
    }
    if (host_r) *host_r = h.r;
    if (host_scale) *host_scale = h.scale;
    if (host_k) *host_k = h.k;
    if (host_blocks) *host_blocks = h.blocks;
    return WN_OK;
}

wn_status wn_rng_draws(uint64_t seed, uint64_t n, uint64_t *host_out)
{
    if (n == 0) return WN_OK;
    if (!host_out) return fail(WN_EINVAL, "wn_rng_draws: NULL output");
    uint64_t *d = nullptr;
    WN_CU(cudaMalloc(&d, sizeof(uint64_t) * n));
    wn::draws_kernel<<<1, 1>>>(seed, n, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(host_out, d, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail("wn_rng_draws", e);
    return WN_OK;
}

}  // extern "C"
