// wn_group.cuh -- the group-mode generate kernel for the plain method
// (Brent, arXiv:1005.2314, Section 5: chi-squared approximation (c),
// reserved value from the previous block, the 4x4 update), for launches of
// many streams.
//
// A CTA of G warps owns one stream and nothing else runs beside them: there
// is no control warp.  Every warp keeps its own copy of the stream's
// generator in registers and derives each pass's permutation and signs from
// the pass's two draws itself (Sections 5.2, 5.4, 5.8; the signs a lane needs
// are one nibble of the second draw, since quadruple q uses nibble q mod 16
// and a lane's quadruples are congruent mod 16), so no pass table is stored
// or loaded.  The pool lives in one shared-memory buffer (in place): a pass
// gathers all of its quadruples into registers, the group synchronises, and
// the results overwrite the pool.  With one buffer a pool of 4096 takes 16 KB,
// so nine streams share an SM and 4096 streams fill three whole waves.
//
// Each block's scale (Section 5.5) is formed at the end of the block before
// it, from that block's sum of squares (FP32 within a warp, FP64 across warps
// and for its deviation from N, which for one warp's FP32 sum FP32 computes
// exactly) and its reserved value -- the sum of squares when the block
// starts, which the orthogonal passes preserve exactly in exact arithmetic.  The final pass stores the block's values straight from
// registers as 16-byte (FP32) or 8-byte (16-bit) stores, realigned by warp
// shuffles, as the ordinary kernel does.
#pragma once

#include "wn_gen.cuh"

namespace wn {

// Dynamic shared memory of a group-mode CTA starts at this shared-window
// address (the first KB of the window is reserved on sm_103a; the host
// checks the probed value before it selects this kernel, and the kernel
// checks it again).  The first kGroupSmall bytes hold per-warp partial sums
// and the reserved value; the pool buffer follows, at a fixed window address,
// so that a gather's address is its pool offset plus an immediate.
constexpr uint32_t kGroupBase = 1024;
constexpr uint32_t kGroupSmall = 128;
constexpr uint32_t kGroupPool = kGroupBase + kGroupSmall;

__host__ __device__ inline size_t group_smem_bytes(uint32_t N) { return kGroupSmall + 4 * (size_t)N; }

// Pool accesses at offset o (bytes) from the pool buffer.
__device__ __forceinline__ float gld(uint32_t o)
{
    if (!dbg_shared_ok(o + kGroupPool, 4)) return 0.f;
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(o), "n"(kGroupPool));
    return v;
}
__device__ __forceinline__ float4 gld4(uint32_t o)
{
    if (!dbg_shared_ok(o + kGroupPool, 16)) return make_float4(0.f, 0.f, 0.f, 0.f);
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4+%5];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(o), "n"(kGroupPool));
    return v;
}
__device__ __forceinline__ void gst4(uint32_t o, float2 lo, float2 hi)
{
    if (!dbg_shared_ok(o + kGroupPool, 16)) return;
    asm volatile("st.shared.v4.f32 [%0+%5], {%1, %2, %3, %4};" ::"r"(o), "f"(lo.x), "f"(lo.y), "f"(hi.x), "f"(hi.y),
                 "n"(kGroupPool));
}

template <int G> __device__ __forceinline__ void group_sync()
{
    if (G == 1) __syncwarp();
    else __syncthreads();
}

// One pass's quantities for this thread, from the pass's two draws: gather
// offsets of quadruple q0 (B0, element 1's offset d1, step dq per 32
// quadruples) and the sign multipliers m_k = -s_k, h_k = s_k / 2 of the
// thread's nibble (the same values the ordinary kernel's tables hold).
struct GroupPass {
    uint32_t B0, d1, dq;
    float2 m01, m23, h01, h23;
};

__device__ __forceinline__ GroupPass group_pass(uint64_t &gx, uint64_t &gw, uint32_t N, uint32_t q0, uint32_t lane)
{
    const uint64_t wa = draw(gx, gw);
    const uint64_t ws = draw(gx, gw);
    const uint32_t alpha = ((uint32_t)(wa >> 32) & (N - 1)) | 1u;
    const uint32_t gamma = (uint32_t)wa & (N - 1);
    GroupPass p;
    p.B0 = 4u * (alpha * q0 + gamma);
    p.d1 = (alpha & 3u) * N;
    p.dq = 128u * alpha;
    const uint32_t word = (lane & 8u) ? (uint32_t)(ws >> 32) : (uint32_t)ws;
    const uint32_t nib = (word >> (4u * (lane & 7u))) & 15u;
    p.m01 = make_float2(neg_sign_one(nib & 1u), neg_sign_one((nib >> 1) & 1u));
    p.m23 = make_float2(neg_sign_one((nib >> 2) & 1u), neg_sign_one(nib >> 3));
    p.h01 = fmul2(p.m01, make_float2(-0.5f, -0.5f));
    p.h23 = fmul2(p.m23, make_float2(-0.5f, -0.5f));
    return p;
}

// Block scale sqrt(S / sum) (Section 5.5, approximation (c)): ss the pool's
// sum of squares, r the previous block's reserved value (scaled).  The same
// FP64 deviation and FP32 steps as the ordinary kernel's.
__device__ __forceinline__ float group_scale(double ss, float r, float A, float B, uint32_t N)
{
    const float invNf = 1.0f / (float)N;
    const float delta = (float)fma(ss, (double)invNf, -1.0);
    const float c = __frsqrt_rn(1.0f + delta);
    const float u = fmaf(A, fmaf(r, r, -1.0f), B * r) * invNf;
    return __fsqrt_rn(1.0f + u) * c;
}

// The same scale from a sum of squares held in FP32: ss (1/N) is then exact
// (N a power of two) and ss/N - 1 exact by Sterbenz's lemma (ss/N lies in
// [1/2, 2]), so one FP32 FMA gives the deviation the FP64 route rounds to,
// bit for bit, without FP64's latency.
__device__ __forceinline__ float group_scale_f32(float ss, float r, float A, float B, uint32_t N)
{
    const float invNf = 1.0f / (float)N;
    const float delta = fmaf(ss, invNf, -1.0f);
    const float c = __frsqrt_rn(1.0f + delta);
    const float u = fmaf(A, fmaf(r, r, -1.0f), B * r) * invNf;
    return __fsqrt_rn(1.0f + u) * c;
}

// The final pass's output: y (this thread's quadruples q0 + 32 j, unscaled)
// times sc to ob[4q + k], as in the ordinary kernel's EMIT_WHOLE (A = element
// offset of ob from a 16-byte boundary; for A = 3 the aligned groups take the
// next quadruple's first value instead of the previous one's last three) or,
// with PART, the first n values with single stores.  nq: quadruples of the pool (slot 4 nq - 1 is the
// reserved value and never written).
template <int QT, int A, bool PART, typename OutT>
__device__ __forceinline__ void group_emit(OutT *__restrict__ ob, const float2 (&y)[QT][2], float sc, uint32_t q0,
                                           uint32_t lane, uint32_t nq, uint32_t n, const DbgRange &rg)
{
    const float2 sc2 = make_float2(sc, sc);
    const uint32_t src = (lane + 31u) & 31u;
    const bool l31 = (lane == 31u);
    float l1 = 0.f, l2 = 0.f, l3 = 0.f;  // this thread's values 1..3 of the previous j
#pragma unroll
    for (int j = 0; j < QT; ++j) {
        const uint32_t q = q0 + 32u * j;
        const float2 v01 = fmul2(y[j][0], sc2), v23 = fmul2(y[j][1], sc2);
        const uint32_t pos = 4u * q;
        if (PART) {
            if (pos < n) store1(rg, ob + pos, v01.x);
            if (pos + 1 < n) store1(rg, ob + pos + 1, v01.y);
            if (pos + 2 < n) store1(rg, ob + pos + 2, v23.x);
            if (pos + 3 < n) store1(rg, ob + pos + 3, v23.y);
            continue;
        }
        const bool last = (j == QT - 1) && (q + 1u == nq);  // the quadruple holding the reserved slot
        if (A == 3) {
            // groups start one value into each quadruple: this quadruple's
            // values 1..3 and the next one's value 0 -- one shuffle from the
            // right neighbour (lane 0 lends its next j's value to lane 31)
            // instead of three from the left
            const float lend = (lane == 0 && j + 1 < QT) ? y[j + 1 < QT ? j + 1 : j][0].x * sc : v01.x;
            const float nx = __shfl_sync(0xffffffffu, lend, (lane + 1u) & 31u);
            if (j == 0 && lane == 0) store1(rg, ob + pos, v01.x);  // predecessor in another warp or before the block
            if (!(l31 && j == QT - 1)) {
                store4(rg, ob + pos + 1, v01.y, v23.x, v23.y, nx);
            } else {  // the successor is in another warp, or slot pos + 3 is the reserved one
                store1(rg, ob + pos + 1, v01.y);
                store1(rg, ob + pos + 2, v23.x);
                if (!last) store1(rg, ob + pos + 3, v23.y);
            }
            continue;
        }
        float p1 = 0.f, p2 = 0.f, p3 = 0.f;
        if (A >= 1) p3 = __shfl_sync(0xffffffffu, l31 ? l3 : v23.y, src);
        if (A >= 2) p2 = __shfl_sync(0xffffffffu, l31 ? l2 : v23.x, src);
        if (A >= 3) p1 = __shfl_sync(0xffffffffu, l31 ? l1 : v01.y, src);
        l1 = v01.y;
        l2 = v23.x;
        l3 = v23.y;
        if (A == 0) {
            if (!last) store4(rg, ob + pos, v01.x, v01.y, v23.x, v23.y);
            else {
                store1(rg, ob + pos, v01.x);
                store1(rg, ob + pos + 1, v01.y);
                store1(rg, ob + pos + 2, v23.x);
            }
            continue;
        }
        if (j == 0 && lane == 0) {  // predecessor in another warp (or before the block): own first 4 - A
            store1(rg, ob + pos, v01.x);
            if (A <= 2) store1(rg, ob + pos + 1, v01.y);
            if (A == 1) store1(rg, ob + pos + 2, v23.x);
        } else {
            OutT *g = ob + (pos - A);
            if (A == 1) store4(rg, g, p3, v01.x, v01.y, v23.x);
            else if (A == 2) store4(rg, g, p2, p3, v01.x, v01.y);
            else store4(rg, g, p1, p2, p3, v01.x);
        }
        if ((j == QT - 1 && l31) || last) {  // successor cannot take the last A
            if (A == 3) store1(rg, ob + pos + 1, v01.y);
            if (A >= 2) store1(rg, ob + pos + 2, v23.x);
            if (!last) store1(rg, ob + pos + 3, v23.y);
        }
    }
}

// One stream's share of a call in group mode (the plain method only).  The
// CTA is G warps; warp w, lane l owns quadruples q0 + 32 j (j < QT),
// q0 = 32 QT w + l, and 128 QT G = N.
template <int G, int QT, typename OutT>
__device__ __forceinline__ void run_stream_group(StreamHdr *__restrict__ h, float *__restrict__ pool_g,
                                                 OutT *__restrict__ out, uint64_t out_off, uint64_t count)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t N = 128u * QT * G, nq = N / 4;
    float *red = reinterpret_cast<float *>(wn_smem);  // [2][G] partial sums by block parity; [2][8]: slot N-1
    const DbgRange rg = dbg_range(out, out + count);   // this stream's output (the debug build checks stores)
    if (smem_base() != kGroupBase || h->N != N) {     // not the layout this kernel was built for
        if (tid == 0) h->flags |= 1u;
        return;
    }
    {
        const float4 *pg4 = reinterpret_cast<const float4 *>(pool_g);
        for (uint32_t i = tid; i < nq; i += 32u * G) {
            const float4 v = pg4[i];
            gst4(16u * i, make_float2(v.x, v.y), make_float2(v.z, v.w));
        }
    }
    const uint32_t k0 = h->k;
    const float sc_prev = h->scale;
    const uint64_t left = (uint64_t)(N - 1 - k0);
    const uint64_t n0 = left < count ? left : count;
    const uint64_t nb = (count - n0 + (N - 2)) / (N - 1);
    const uint64_t tail = (count - n0) % (N - 1);  // values of a partial last block (0: whole)
    const uint32_t R = h->R;
    uint64_t gx = h->x, gw = h->w;
    const float A = (float)h->A, B = (float)h->B;
    // block 0's scale: the stored sum of squares and reserved value
    float sc = nb > 0 ? group_scale(h->sumsq, (float)h->r, A, B, N) : sc_prev;
    double ss = h->sumsq;
    group_sync<G>();
    for (uint64_t i = tid; i < n0; i += 32u * G) store1(rg, out + i, sc_prev * gld(4u * (uint32_t)(k0 + i)));

    const uint32_t q0 = warp * 32u * QT + lane;
    const uint32_t m4 = 4u * N - 1u, half = 2u * N;
    OutT *ob = out + n0;
    uint32_t a = (uint32_t)((out_off + n0) & 3u);  // alignment of ob within 16 bytes
    float rv = 0.f;                                // the last block's reserved value, unscaled
    for (uint64_t b = 0; b < nb; ++b) {
        float2 y[QT][2];
        float2 part = make_float2(0.f, 0.f);
        for (uint32_t p = 0; p < R; ++p) {
            const GroupPass gp = group_pass(gx, gw, N, q0, lane);
            float av[QT][4];
#pragma unroll
            for (int j = 0; j < QT; ++j) {
                const uint32_t Bj = gp.B0 + (uint32_t)j * gp.dq;
                const uint32_t o0 = Bj & m4, o1 = (Bj + gp.d1) & m4;
                av[j][0] = gld(o0);
                av[j][2] = gld(o0 ^ half);
                av[j][1] = gld(o1);
                av[j][3] = gld(o1 ^ half);
            }
            group_sync<G>();  // every gather of the pass is done: the pool may be overwritten
            const bool fin = (p + 1 == R);
#pragma unroll
            for (int j = 0; j < QT; ++j) {
                const float2 a01 = make_float2(av[j][0], av[j][1]), a23 = make_float2(av[j][2], av[j][3]);
                const float2 s2 = fadd2(a01, a23);
                const float sum = s2.x + s2.y;
                const float2 SS = make_float2(sum, sum);
                y[j][0] = ffma2(gp.m01, a01, fmul2(gp.h01, SS));
                y[j][1] = ffma2(gp.m23, a23, fmul2(gp.h23, SS));
                gst4(16u * (q0 + 32u * j), y[j][0], y[j][1]);
                if (fin) part = ffma2(y[j][0], y[j][0], ffma2(y[j][1], y[j][1], part));
            }
            if (!fin) group_sync<G>();  // the pass's stores precede the next pass's gathers
        }
        // the block's values (scale sc), then the next block's scale
        const bool whole = (b + 1 < nb) || tail == 0;
        if (!whole) {
            group_emit<QT, 0, true, OutT>(ob, y, sc, q0, lane, nq, (uint32_t)tail, rg);
        } else {
            switch (a) {
            case 0: group_emit<QT, 0, false, OutT>(ob, y, sc, q0, lane, nq, 0, rg); break;
            case 1: group_emit<QT, 1, false, OutT>(ob, y, sc, q0, lane, nq, 0, rg); break;
            case 2: group_emit<QT, 2, false, OutT>(ob, y, sc, q0, lane, nq, 0, rg); break;
            default: group_emit<QT, 3, false, OutT>(ob, y, sc, q0, lane, nq, 0, rg); break;
            }
        }
        float ps = part.x + part.y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ps += __shfl_xor_sync(0xffffffffu, ps, o);
        if (G == 1) {
            ss = (double)ps;
            rv = __shfl_sync(0xffffffffu, y[QT - 1][1].y, 31);
        } else {
            const uint32_t par = (uint32_t)(b & 1u);
            if (lane == 0) red[par * 8u + warp] = ps;
            if (warp == G - 1 && lane == 31) red[16u + par] = y[QT - 1][1].y;
            __syncthreads();  // partial sums published; also ends the pass
            double t4[G];  // the warps' partial sums, added pairwise in FP64
#pragma unroll
            for (int w = 0; w < G; ++w) t4[w] = (double)red[par * 8u + w];
#pragma unroll
            for (int st = 1; st < G; st <<= 1)
#pragma unroll
                for (int w = 0; w + st < G; w += 2 * st) t4[w] += t4[w + st];
            ss = t4[0];
            rv = red[16u + par];
        }
        if (G == 1) __syncwarp();  // the final pass's stores precede the next block's gathers
        const float r = sc * rv;   // this block's reserved value, scaled (Section 5.5, fastnorm2)
        // one warp's sum is an FP32 value, for which the FP32 route gives the
        // FP64 route's bits (group_scale_f32); several warps' partial sums are
        // added in FP64 (pairwise) and take the FP64 route
        if (b + 1 < nb) sc = (G == 1) ? group_scale_f32((float)ss, r, A, B, N) : group_scale(ss, r, A, B, N);
        ob += N - 1;
        a = (a + N - 1) & 3u;
    }

    group_sync<G>();
    {
        float4 *pw4 = reinterpret_cast<float4 *>(pool_g);
        for (uint32_t i = tid; i < nq; i += 32u * G) pw4[i] = gld4(16u * i);
    }
    if (tid == 0) {
        if (nb > 0) {
            h->x = gx;
            h->w = gw;
            h->sumsq = ss;
            h->r = (double)(sc * rv);
            h->scale = sc;
            h->k = tail == 0 ? N - 1 : (uint32_t)tail;
            h->blocks += nb;
        } else {
            h->k = k0 + (uint32_t)n0;
        }
    }
}

// Group-mode generate kernel: one CTA of G warps per stream; MINB resident
// CTAs per SM bound the registers.
template <int G, int QT, int MINB, typename OutT>
__global__ void __launch_bounds__(32 * G, MINB) group_kernel(GenArgs a)
{
    StreamHdr *h = a.hdr + blockIdx.x;
    const uint64_t off = (uint64_t)blockIdx.x * a.out_stride;
    run_stream_group<G, QT, OutT>(h, a.pools + h->pool_off, reinterpret_cast<OutT *>(a.out) + off, off, a.count);
}

// Compiled group-mode shapes {pool N, warps per stream G, quadruples per lane
// QT, minimum CTAs per SM}.
constexpr int kGroupShapes[][4] = {{1024, 1, 8, 16}, {1024, 4, 2, 8},  {2048, 1, 16, 12}, {4096, 1, 32, 9},
                                   {4096, 2, 16, 9},  {4096, 4, 8, 6},  {4096, 8, 4, 4},   {8192, 2, 32, 4},
                                   {16384, 4, 32, 3}, {16384, 8, 16, 2}};

// Resident CTAs per SM for a launch of n_streams streams: the fewest that
// keeps the number of waves the most the SM holds would give (4096 streams on
// 152 SMs are 27 per SM: nine at a time make three whole waves, where twelve
// would leave a third wave of three).  Shared memory is then padded so that
// exactly that many fit.
inline uint32_t group_ctas_per_sm(uint32_t n_streams, int sms, int k_max)
{
    if (k_max < 1 || sms < 1) return 1;
    const uint32_t per_sm = (n_streams + (uint32_t)sms - 1) / (uint32_t)sms;
    const uint32_t waves = (per_sm + (uint32_t)k_max - 1) / (uint32_t)k_max;
    return waves ? (per_sm + waves - 1) / waves : 1u;
}

template <int G, int QT, int MINB, typename OutT>
cudaError_t launch_group_shape(const GenArgs &a, int sms, cudaStream_t cs, uint32_t *ctas_per_sm)
{
    auto kern = group_kernel<G, QT, MINB, OutT>;
    const uint32_t N = 128u * QT * G;
    const size_t need = group_smem_bytes(N);
    int dev = 0, sm_bytes = 0, reserved = 0, optin = 0, k_max = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // the whole opt-in range first: the occupancy query honours the limit
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k_max, kern, 32 * G, need);
    if (e != cudaSuccess) return e;
    if (k_max < 1 || need > (size_t)optin) return cudaErrorInvalidConfiguration;
    const uint32_t k = group_ctas_per_sm(a.n_streams, sms, k_max);
    size_t smem = ((size_t)sm_bytes / k - (size_t)reserved) / 128 * 128;
    if (smem < need) smem = need;
    if (smem > (size_t)optin) smem = (size_t)optin;
    if (ctas_per_sm) *ctas_per_sm = k;
    kern<<<a.n_streams, 32 * G, smem, cs>>>(a);
    return cudaGetLastError();
}

// Launch of the group-mode kernel for pool N with G warps per stream; sms:
// the device's multiprocessors; *ctas_per_sm (may be NULL) receives the CTAs
// per SM the launch was sized for.
template <typename OutT>
cudaError_t launch_group_t(const GenArgs &a, uint32_t N, uint32_t G, int sms, cudaStream_t cs, uint32_t *ctas_per_sm)
{
    switch (N * 16 + G) {
    case 1024 * 16 + 1: return launch_group_shape<1, 8, 16, OutT>(a, sms, cs, ctas_per_sm);
#ifndef WN_DEBUG
    case 2048 * 16 + 1: return launch_group_shape<1, 16, 12, OutT>(a, sms, cs, ctas_per_sm);
#endif
#ifndef WN_DEBUG
    case 4096 * 16 + 1: return launch_group_shape<1, 32, 9, OutT>(a, sms, cs, ctas_per_sm);
#endif
#ifndef WN_DEBUG
    case 4096 * 16 + 2: return launch_group_shape<2, 16, 9, OutT>(a, sms, cs, ctas_per_sm);
#endif
#ifndef WN_DEBUG
    case 4096 * 16 + 4: return launch_group_shape<4, 8, 6, OutT>(a, sms, cs, ctas_per_sm);
#endif
#ifndef WN_DEBUG
    case 4096 * 16 + 8: return launch_group_shape<8, 4, 4, OutT>(a, sms, cs, ctas_per_sm);
#endif
#ifndef WN_DEBUG
    case 1024 * 16 + 4: return launch_group_shape<4, 2, 8, OutT>(a, sms, cs, ctas_per_sm);
#endif
#ifndef WN_DEBUG
    case 16384 * 16 + 8: return launch_group_shape<8, 16, 2, OutT>(a, sms, cs, ctas_per_sm);
#endif
#ifndef WN_DEBUG
    case 8192 * 16 + 2: return launch_group_shape<2, 32, 4, OutT>(a, sms, cs, ctas_per_sm);
#endif
#ifndef WN_DEBUG
    case 16384 * 16 + 4: return launch_group_shape<4, 32, 3, OutT>(a, sms, cs, ctas_per_sm);
#endif
    default: return cudaErrorInvalidValue;
    }
}

// Persistent group-mode kernel for batches (one pool size): each CTA claims
// the next stream from an atomic counter (longest request first), returns
// that stream's request, and claims again until the list is exhausted.  No
// CTA waits on another.  The claimed index passes through the small area
// (word 24), since static shared memory would move the pool's window address.
template <int G, int QT, int MINB, typename OutT>
__global__ void __launch_bounds__(32 * G, MINB) persist_group_kernel(GenArgs a, BatchArgs bq)
{
    uint32_t *slot = reinterpret_cast<uint32_t *>(wn_smem) + 24;
    for (;;) {
        group_sync<G>();  // the previous stream is done with shared memory
        uint32_t it;
        if (G == 1) {
            uint32_t c = 0;
            if (threadIdx.x == 0) c = atomicAdd(bq.queue, 1u);
            it = __shfl_sync(0xffffffffu, c, 0);
        } else {
            if (threadIdx.x == 0) *slot = atomicAdd(bq.queue, 1u);
            __syncthreads();
            it = *slot;
        }
        if (it >= bq.n_items) return;
        const uint32_t si = bq.order[it];
        StreamHdr *h = a.hdr + si;
        const uint64_t off = bq.offsets[si];
        run_stream_group<G, QT, OutT>(h, a.pools + h->pool_off, reinterpret_cast<OutT *>(a.out) + off, off,
                                      bq.counts[si]);
    }
}

template <int G, int QT, int MINB, typename OutT>
cudaError_t launch_persist_group_shape(const GenArgs &a, const BatchArgs &bq, int sms, cudaStream_t cs)
{
    auto kern = persist_group_kernel<G, QT, MINB, OutT>;
    const size_t smem = group_smem_bytes(128u * QT * G);
    int dev = 0, optin = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * G, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1 || smem > (size_t)optin) return cudaErrorInvalidConfiguration;
    const uint32_t grid = std::min<uint32_t>(bq.n_items, (uint32_t)(per_sm * sms));
    if (grid == 0) return cudaSuccess;
    kern<<<grid, 32 * G, smem, cs>>>(a, bq);
    return cudaGetLastError();
}

// Persistent launch of the group-mode kernel for pool N with G warps per
// stream over the batch list bq.
template <typename OutT>
cudaError_t launch_persist_group_t(const GenArgs &a, const BatchArgs &bq, uint32_t N, uint32_t G, int sms,
                                   cudaStream_t cs)
{
    switch (N * 16 + G) {
    case 1024 * 16 + 1: return launch_persist_group_shape<1, 8, 16, OutT>(a, bq, sms, cs);
#ifndef WN_DEBUG
    case 1024 * 16 + 4: return launch_persist_group_shape<4, 2, 8, OutT>(a, bq, sms, cs);
#endif
#ifndef WN_DEBUG
    case 2048 * 16 + 1: return launch_persist_group_shape<1, 16, 12, OutT>(a, bq, sms, cs);
#endif
#ifndef WN_DEBUG
    case 4096 * 16 + 1: return launch_persist_group_shape<1, 32, 9, OutT>(a, bq, sms, cs);
#endif
#ifndef WN_DEBUG
    case 4096 * 16 + 2: return launch_persist_group_shape<2, 16, 9, OutT>(a, bq, sms, cs);
#endif
#ifndef WN_DEBUG
    case 4096 * 16 + 4: return launch_persist_group_shape<4, 8, 6, OutT>(a, bq, sms, cs);
#endif
#ifndef WN_DEBUG
    case 4096 * 16 + 8: return launch_persist_group_shape<8, 4, 4, OutT>(a, bq, sms, cs);
#endif
#ifndef WN_DEBUG
    case 8192 * 16 + 2: return launch_persist_group_shape<2, 32, 4, OutT>(a, bq, sms, cs);
#endif
#ifndef WN_DEBUG
    case 16384 * 16 + 4: return launch_persist_group_shape<4, 32, 3, OutT>(a, bq, sms, cs);
#endif
#ifndef WN_DEBUG
    case 16384 * 16 + 8: return launch_persist_group_shape<8, 16, 2, OutT>(a, bq, sms, cs);
#endif
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_persist_group_f32(const GenArgs &a, const BatchArgs &bq, uint32_t N, uint32_t G, int sms,
                                     cudaStream_t cs);
cudaError_t launch_persist_group_bf16(const GenArgs &a, const BatchArgs &bq, uint32_t N, uint32_t G, int sms,
                                      cudaStream_t cs);
cudaError_t launch_persist_group_f16(const GenArgs &a, const BatchArgs &bq, uint32_t N, uint32_t G, int sms,
                                     cudaStream_t cs);

cudaError_t launch_group_f32(const GenArgs &a, uint32_t N, uint32_t G, int sms, cudaStream_t cs,
                             uint32_t *ctas_per_sm);
cudaError_t launch_group_bf16(const GenArgs &a, uint32_t N, uint32_t G, int sms, cudaStream_t cs,
                              uint32_t *ctas_per_sm);
cudaError_t launch_group_f16(const GenArgs &a, uint32_t N, uint32_t G, int sms, cudaStream_t cs,
                             uint32_t *ctas_per_sm);

}  // namespace wn
