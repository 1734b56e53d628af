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
    void *out;               // 16-byte aligned
    uint64_t count;          // values per stream
    uint64_t out_stride;     // elements between consecutive streams' outputs
    uint32_t n_streams;
    uint32_t n_max;          // largest pool of the launch (shared-memory layout)
    uint32_t r_max;          // most passes per block of the launch
    uint32_t warmup_blocks;  // nonzero: discard this many whole blocks, store nothing
};

// Shared memory of a generate CTA: two pool buffers of n_max floats, 32 warp
// partial sums, the block scale, and two sets of 2 r_max draws (this block's
// and the next one's).
__host__ __device__ inline size_t gen_smem_bytes(uint32_t n_max, uint32_t r_max)
{
    return (size_t)8 * n_max + 128 + 16 + (size_t)32 * r_max;
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

// Per-pass constants a thread derives from the pass's two draws (Section 5.4
// index choice, Section 5.2 signs).  Element k of quadruple q is read from
// (alpha q + o_k) mod N with o_k = (alpha k N/4 + gamma) mod N; its sign mask
// is bit k of the nibble (w_s >> 4 (q mod 16)), placed in the float sign bit.
struct PassParams {
    uint32_t alpha, o0, o1, o2, o3, s0, s1, s2, s3;
};

__device__ __forceinline__ PassParams pass_params(uint64_t wa, uint64_t ws, uint32_t nq, uint32_t mask,
                                                  uint32_t nibble_shift)
{
    PassParams pp;
    pp.alpha = ((uint32_t)(wa >> 32) & mask) | 1u;
    pp.o0 = (uint32_t)wa & mask;
    pp.o1 = (pp.alpha * nq + pp.o0) & mask;
    pp.o2 = (2u * pp.alpha * nq + pp.o0) & mask;
    pp.o3 = (3u * pp.alpha * nq + pp.o0) & mask;
    const uint32_t nib = (uint32_t)(ws >> nibble_shift) & 15u;
    pp.s0 = (nib & 1u) << 31;
    pp.s1 = ((nib >> 1) & 1u) << 31;
    pp.s2 = ((nib >> 2) & 1u) << 31;
    pp.s3 = (nib >> 3) << 31;
    return pp;
}

// One pass over this thread's quadruples q = tid + j T: gather, update,
// store the four results contiguously at nxt[4q..4q+3].  The final pass of a
// block also keeps the results in registers and sums their squares.
template <int QT, bool FINAL>
__device__ __forceinline__ void pass_quads(const float *__restrict__ cur, float *__restrict__ nxt,
                                           const PassParams &pp, uint32_t nq, uint32_t mask, uint32_t tid,
                                           uint32_t T, float (&y)[QT][4], float &part)
{
    float4 *n4 = reinterpret_cast<float4 *>(nxt);
#pragma unroll
    for (int j = 0; j < QT; ++j) {
        const uint32_t q = tid + (uint32_t)j * T;
        if (q < nq) {
            const uint32_t base = pp.alpha * q;
            const float a0 = cur[(base + pp.o0) & mask];
            const float a1 = cur[(base + pp.o1) & mask];
            const float a2 = cur[(base + pp.o2) & mask];
            const float a3 = cur[(base + pp.o3) & mask];
            const float t = 0.5f * ((a0 + a1) + (a2 + a3));
            float4 v;
            v.x = __uint_as_float(__float_as_uint(t - a0) ^ pp.s0);
            v.y = __uint_as_float(__float_as_uint(t - a1) ^ pp.s1);
            v.z = __uint_as_float(__float_as_uint(t - a2) ^ pp.s2);
            v.w = __uint_as_float(__float_as_uint(t - a3) ^ pp.s3);
            n4[q] = v;
            if (FINAL) {
                y[j][0] = v.x;
                y[j][1] = v.y;
                y[j][2] = v.z;
                y[j][3] = v.w;
                part = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, part))));
            }
        }
    }
}

template <typename OutT> __device__ __forceinline__ void store1(OutT *p, float v) { *p = to_out<OutT>(v); }

// Four consecutive values to an address aligned to four elements.
__device__ __forceinline__ void store4(float *p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
template <typename H> __device__ __forceinline__ void store4_16(H *p, float a, float b, float c, float d)
{
    union {
        H h[4];
        uint2 u;
    } pk;
    pk.h[0] = to_out<H>(a);
    pk.h[1] = to_out<H>(b);
    pk.h[2] = to_out<H>(c);
    pk.h[3] = to_out<H>(d);
    *reinterpret_cast<uint2 *>(p) = pk.u;
}
__device__ __forceinline__ void store4(__nv_bfloat16 *p, float a, float b, float c, float d) { store4_16(p, a, b, c, d); }
__device__ __forceinline__ void store4(__half *p, float a, float b, float c, float d) { store4_16(p, a, b, c, d); }

// Writes a block's first n values (n <= N-1) from the registers of its final
// pass: value 4q+k is y[j][k] scaled, q = tid + j T, and goes to ob[4q+k].
// `a` = (element offset of ob from a 16-byte boundary) mod 4.  Each thread
// stores the aligned group that holds its first value -- the previous
// quadruple's last a values (from lane - 1, by shuffle) and its own first
// 4 - a -- as one 16-byte (FP32) or 8-byte (16-bit) store.  Where the
// neighbour quadruple sits in another warp (lanes 0 and 31) or past the end,
// the values fall back to single stores; nothing at or beyond n is written.
template <int QT, typename OutT>
__device__ __forceinline__ void emit_regs(OutT *__restrict__ ob, uint32_t a, uint32_t n, float sc,
                                          const float (&y)[QT][4], uint32_t tid, uint32_t T, uint32_t lane,
                                          uint32_t nq)
{
#pragma unroll
    for (int j = 0; j < QT; ++j) {
        const uint32_t q = tid + (uint32_t)j * T;
        const float v0 = sc * y[j][0], v1 = sc * y[j][1], v2 = sc * y[j][2], v3 = sc * y[j][3];
        float p1 = 0.f, p2 = 0.f, p3 = 0.f;  // previous quadruple's values 1..3
        if (a >= 1) p3 = __shfl_up_sync(0xffffffffu, v3, 1);
        if (a >= 2) p2 = __shfl_up_sync(0xffffffffu, v2, 1);
        if (a >= 3) p1 = __shfl_up_sync(0xffffffffu, v1, 1);
        if (q >= nq) continue;
        const uint32_t pos = 4u * q;  // position of v0 in the block
        const bool lead = (a != 0) && (lane == 0);
        const bool trail = (a != 0) && (lane == 31 || q + 1 >= nq);
        const bool vec = !lead && pos + 3u - a < n;
        if (vec) {
            OutT *g = ob + (pos - a);
            switch (a) {
            case 0: store4(g, v0, v1, v2, v3); break;
            case 1: store4(g, p3, v0, v1, v2); break;
            case 2: store4(g, p2, p3, v0, v1); break;
            default: store4(g, p1, p2, p3, v0); break;
            }
        } else if (!lead) {
            // previous quadruple's value i sits at pos - 4 + i; this thread
            // owns the last a of them (i >= 4 - a)
            if (a >= 3 && pos - 3u < n) store1(ob + (pos - 3u), p1);
            if (a >= 2 && pos - 2u < n) store1(ob + (pos - 2u), p2);
            if (a >= 1 && pos - 1u < n) store1(ob + (pos - 1u), p3);
        }
        // own values: the first 4 - a unless the vector store took them, the
        // last a only where the next quadruple's thread cannot (trail)
        if ((0u < 4u - a ? !vec : trail) && pos < n) store1(ob + pos, v0);
        if ((1u < 4u - a ? !vec : trail) && pos + 1u < n) store1(ob + pos + 1u, v1);
        if ((2u < 4u - a ? !vec : trail) && pos + 2u < n) store1(ob + pos + 2u, v2);
        if ((3u < 4u - a ? !vec : trail) && pos + 3u < n) store1(ob + pos + 3u, v3);
    }
}

// ---------------------------------------------------------------------------
// One stream's share of a call: return the rest of the last block, then run
// as many whole blocks as `count` needs, then write the state back.
// QT = quadruples per thread; blockDim.x is a multiple of 32 with
// blockDim.x * QT >= N/4.  Per block: R passes (one barrier each), the sum
// of squares (FP32 within a warp, FP64 across warps), one barrier while warp 0
// forms the scale, then the outputs straight from the final pass's registers.
// ---------------------------------------------------------------------------
template <int QT, typename OutT>
__device__ __forceinline__ void run_stream(StreamHdr *__restrict__ h, float *__restrict__ pool_g,
                                           OutT *__restrict__ out, uint64_t out_off, uint64_t count,
                                           bool store, uint32_t n_max, uint32_t r_max)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t T = blockDim.x, tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5, nw = T >> 5;
    const uint32_t N = h->N, R = h->R, nq = N >> 2, mask = N - 1;
    float *buf0 = reinterpret_cast<float *>(smem);
    float *buf1 = buf0 + n_max;
    float *red = buf0 + 2 * (size_t)n_max;
    float *sc_sm = red + 32;
    uint64_t *dr = reinterpret_cast<uint64_t *>(sc_sm + 4);  // [2][2 r_max]

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
    // constants; it publishes each block's draws through shared memory one
    // block ahead.
    uint64_t gx = 0, gw = 0;
    float r = 0.f, Af = 0.f, Bf = 0.f;
    const double invN = 1.0 / (double)N;
    const float invNf = 1.0f / (float)N;
    if (warp == 0) {
        gx = h->x;
        gw = h->w;
        r = (float)h->r;
        Af = (float)h->A;
        Bf = (float)h->B;
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
    const uint32_t sh = 4u * (tid & 15u);  // quadruple q uses nibble q mod 16 = tid mod 16
    float y[QT][4];
#pragma unroll
    for (int j = 0; j < QT; ++j) y[j][0] = y[j][1] = y[j][2] = y[j][3] = 0.f;

    for (uint64_t b = 0; b < nb; ++b) {
        const uint64_t *dcur = dr + (b & 1) * 2 * r_max;
        if (warp == 0 && b + 1 < nb) {
            uint64_t *dnext = dr + ((b + 1) & 1) * 2 * r_max;
            for (uint32_t i = 0; i < 2 * R; ++i) {
                const uint64_t d = draw(gx, gw);
                if (lane == (i & 31u)) dnext[i] = d;
            }
        }
        float part = 0.f;
        for (uint32_t p = 0; p + 1 < R; ++p) {
            const PassParams pp = pass_params(dcur[2 * p], dcur[2 * p + 1], nq, mask, sh);
            pass_quads<QT, false>(cur, nxt, pp, nq, mask, tid, T, y, part);
            float *tmp = cur;
            cur = nxt;
            nxt = tmp;
            __syncthreads();
        }
        {
            const PassParams pp = pass_params(dcur[2 * (R - 1)], dcur[2 * (R - 1) + 1], nq, mask, sh);
            pass_quads<QT, true>(cur, nxt, pp, nq, mask, tid, T, y, part);
            float *tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (warp == 0) {
            // FP64 across warps: the pool's sum of squares and its deviation
            // from N; the scale sqrt(S / sum) is then formed in FP32 with
            // correctly rounded operations (S from approximation (c)).
            double v = (lane < nw) ? (double)red[lane] : 0.0;
            for (uint32_t o = 1; o < 32; o <<= 1)
                if (o < nw) v += __shfl_xor_sync(0xffffffffu, v, o);
            const float delta = (float)fma(v, invN, -1.0);                  // sum/N - 1
            const float c = __frsqrt_rn(1.0f + delta);                      // sqrt(N / sum)
            const float u = fmaf(Af, fmaf(r, r, -1.0f), Bf * r) * invNf;   // S/N - 1
            const float s = __fsqrt_rn(1.0f + u) * c;                       // sqrt(S / sum)
            r = s * cur[N - 1];                                             // held back
            if (lane == 0) *sc_sm = s;
        }
        __syncthreads();
        const float sc = *sc_sm;
        const uint64_t rem = count - emitted;
        const uint32_t n = rem < (uint64_t)(N - 1) ? (uint32_t)rem : (N - 1);
        if (store) emit_regs<QT, OutT>(out + emitted, (uint32_t)((out_off + emitted) & 3u), n, sc, y, tid, T, lane, nq);
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
        h->r = (double)r;
        if (nb > 0) {
            h->scale = last_sc;
            h->k = last_n;
        } else {
            h->k = k0 + (uint32_t)n0;
        }
        h->blocks += nb;
    }
}

template <int QT, int MAXT, int MINB, typename OutT>
__global__ void __launch_bounds__(MAXT, MINB) generate_kernel(GenArgs a)
{
    StreamHdr *h = a.hdr + blockIdx.x;
    const uint32_t N = h->N;
    const uint64_t count = a.warmup_blocks ? (uint64_t)a.warmup_blocks * (N - 1) : a.count;
    const uint64_t off = (uint64_t)blockIdx.x * a.out_stride;
    OutT *out = a.out ? reinterpret_cast<OutT *>(a.out) + off : nullptr;
    run_stream<QT, OutT>(h, a.pools + h->pool_off, out, off, count, a.warmup_blocks == 0, a.n_max, a.r_max);
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

namespace wn {
struct LaunchCfg {
    int qt;            // quadruples per thread
    int maxt;          // launch bound of the instantiation
    uint32_t threads;  // blockDim.x
};
}  // namespace wn

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
    // launch configuration chosen by wn_set_config (otherwise the default)
    bool has_cfg = false;
    wn::LaunchCfg cfg{};
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

using wn::LaunchCfg;

// Compiled (quadruples per thread, thread bound) pairs; each instantiation
// also carries a minimum of resident CTAs per SM that caps its registers.
constexpr int kCfgs[][2] = {{1, 1024}, {2, 512}, {4, 256}, {4, 1024}, {8, 128}, {8, 512}};

bool cfg_ok(const LaunchCfg &c, uint32_t n_max)
{
    bool compiled = false;
    for (const auto &k : kCfgs) compiled |= (k[0] == c.qt && k[1] == c.maxt);
    return compiled && c.threads >= 32 && c.threads % 32 == 0 && c.threads <= (uint32_t)c.maxt &&
           (uint64_t)c.threads * c.qt >= n_max / 4;
}

// Default threads and quadruples per thread for a launch whose largest pool
// is n_max: one quadruple per thread up to N = 1024 (at least one full
// warp), four above.
LaunchCfg pick_cfg(uint32_t n_max)
{
    const uint32_t nq = n_max / 4;
    if (nq <= 256) return {1, 1024, std::max(32u, (nq + 31u) / 32u * 32u)};
    if (nq <= 1024) return {4, 256, nq / 4};
    return {4, 1024, nq / 4};
}

template <int QT, int MAXT, int MINB, typename OutT>
cudaError_t launch_gen(const wn::GenArgs &a, uint32_t threads, size_t smem, cudaStream_t cs)
{
    auto kern = wn::generate_kernel<QT, MAXT, MINB, OutT>;
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
    const int key = c.qt * 10000 + c.maxt;
    switch (key) {
    case 1 * 10000 + 1024: return launch_gen<1, 1024, 1, OutT>(a, c.threads, smem, cs);
    case 2 * 10000 + 512: return launch_gen<2, 512, 2, OutT>(a, c.threads, smem, cs);
    case 4 * 10000 + 256: return launch_gen<4, 256, 4, OutT>(a, c.threads, smem, cs);
    case 4 * 10000 + 1024: return launch_gen<4, 1024, 1, OutT>(a, c.threads, smem, cs);
    case 8 * 10000 + 128: return launch_gen<8, 128, 6, OutT>(a, c.threads, smem, cs);
    case 8 * 10000 + 512: return launch_gen<8, 512, 1, OutT>(a, c.threads, smem, cs);
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
    a.r_max = s->r_max;
    a.warmup_blocks = warmup;
    const LaunchCfg c = s->has_cfg ? s->cfg : pick_cfg(s->n_max);
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

wn_status wn_set_config(wn_stream *s, uint32_t quads_per_thread, uint32_t threads)
{
    if (!s) return fail(WN_EINVAL, "wn_set_config: NULL handle");
    if (quads_per_thread == 0 && threads == 0) {
        s->has_cfg = false;
        return WN_OK;
    }
    // the instantiation with the smallest thread bound that admits `threads`
    LaunchCfg best{0, 0, threads};
    for (const auto &k : kCfgs) {
        LaunchCfg c{k[0], k[1], threads};
        if (k[0] == (int)quads_per_thread && cfg_ok(c, s->n_max) && (best.qt == 0 || k[1] < best.maxt)) best = c;
    }
    if (best.qt == 0)
        return fail(WN_EINVAL, "wn_set_config: no compiled configuration with " + std::to_string(quads_per_thread) +
                                   " quadruples per thread and " + std::to_string(threads) +
                                   " threads covers pool " + std::to_string(s->n_max));
    s->cfg = best;
    s->has_cfg = true;
    return WN_OK;
}

wn_status wn_get_config(const wn_stream *s, uint32_t *quads_per_thread, uint32_t *threads)
{
    if (!s) return fail(WN_EINVAL, "wn_get_config: NULL handle");
    const LaunchCfg c = s->has_cfg ? s->cfg : pick_cfg(s->n_max);
    if (quads_per_thread) *quads_per_thread = (uint32_t)c.qt;
    if (threads) *threads = c.threads;
    return WN_OK;
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
