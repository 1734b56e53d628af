// wn_gen.cuh -- the kernels of Wallace's maximum-entropy normal generator for
// sm_103a (Brent, arXiv:1005.2314, Section 5), as templates instantiated per
// output type and kernel kind in gen_*.cu (generate), persist_*.cu (batches),
// lat_*.cu (latency mode) and gbm.cu (the fused Monte Carlo consumer).
//
// One CTA owns one stream for the whole call and keeps its pool of N values
// in shared memory.  A pass gathers each quadruple through the affine
// permutation j -> alpha j + gamma (mod N) (Section 5.4), applies
// y_k = s_k (t - a_k), t = (a_0+a_1+a_2+a_3)/2 (Sections 5.2-5.3) and stores
// the four results contiguously (the transposed write).  After the R passes
// of a block its N-1 values are scaled so that the pool's sum of squares is a
// chi-squared_N sample drawn from the previous block's reserved value
// (Section 5.5, approximation (c)), and written to global memory.
//
// GB300 mapping (measured on this part: the kernel is bound by issue slots
// and by the L1 data pipe, which carries both shared-memory and global-store
// wavefronts, not by HBM):
//  * warp 0 is a control warp: it draws and tabulates the next block's passes
//    and forms each block's scale (FP64 sum of the compute warps' partial sums
//    of squares, then FP32) while the compute warps run passes (the latency
//    mode for few streams splits this between two control warps outside the
//    pass barriers; see run_stream_lat);
//  * gathers are conflict-free (alpha odd: a warp's 32 consecutive
//    quadruples hit 32 banks) and their addresses cost one LOP3 each, because
//    the pool buffers sit at shared-window addresses that are multiples of
//    their size;
//  * the update runs on packed FP32 pairs (f32x2);
//  * the final pass of a block scales its results in registers and stores
//    them straight to global memory as 16-byte (FP32) or 8-byte (16-bit)
//    aligned stores, realigned by warp shuffles (blocks of N-1 values shift
//    the output alignment by one element per block);
//  * large pools can live in one buffer instead of two (the in-place layout:
//    a pass gathers everything into registers before any store), so that two
//    16384-value pools share an SM.
// The block's scale uses the pool's sum of squares measured when the block
// starts, which the orthogonal passes preserve exactly in exact arithmetic
// (Section 5.5); in FP32 the two differ by the rounding of R passes.
#pragma once

#include <algorithm>
#include <cstdint>

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

// Launch shape: `threads` compute threads (plus the control warp) each owning
// `qt` quadruples; `maxt` is the instantiation's thread bound; `ip` selects
// the in-place pool layout (one pool buffer instead of two; see run_stream).
// `grp` selects the group-mode kernel (wn_group.cuh): `threads` / 32 warps
// per stream, `qt` quadruples per lane, no control warp, in place.
struct LaunchCfg {
    int qt;
    int maxt;
    uint32_t threads;
    int ip = 0;
    int grp = 0;
};

// Compiled shapes {quadruples per thread, thread bound (compute threads + 32),
// minimum resident CTAs per SM (caps registers), in-place pool}.  The
// in-place shape halves the pool's shared memory, so that two CTAs with
// 16384-value pools share an SM where the two-buffer layout fits one.
constexpr int kShapes[][4] = {{1, 1024, 1, 0}, {2, 544, 2, 0}, {4, 288, 4, 0}, {8, 160, 4, 0},
                              {8, 544, 1, 0},  {16, 288, 1, 0}, {16, 288, 2, 1}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);
// Launcher switch key of a shape.
constexpr int shape_key(int qt, int maxt, int ip) { return (ip * 100 + qt) * 10000 + maxt; }

// Stream state the control warp keeps in shared memory between blocks.
struct CtlState {
    uint64_t gx, gw;  // generator
    double sumsq;     // pool's sum of squares when the call's first block starts
    float r;          // reserved value of the block before the call
    float A, B;       // chi-squared (c) constants
    float sc[2];      // output scale of block b, by parity of b
    uint32_t item;    // persistent CTAs: the work item just claimed
};
static_assert(sizeof(CtlState) == 48, "CtlState layout");

// Per-pass table the control warp derives from the pass's two draws
// (Section 5.4 index choice, Section 5.2 signs).  Element k of quadruple q is
// P[(alpha q + o_k) mod N], o_k = (alpha k N/4 + gamma) mod N.  Since alpha is
// odd, o_2 = o_0 + N/2 and o_3 = o_1 + N/2 (mod N) and o_1 - o_0 =
// (alpha mod 4) N/4: the four elements share one offset within the pool's
// quarters.  In bytes, with B = 4 (alpha q + gamma): element 0 at B mod 4N,
// element 2 at that XOR 2N, element 1 at (B + d1) mod 4N with
// d1 = (alpha mod 4) N, element 3 at that XOR 2N.  Output k of quadruple q
// takes the sign of bit k of the nibble (w_s >> 4 (q mod 16)); sgn[g] holds
// the four values -s_k of nibble g.
struct PassTab {
    uint32_t a4, g4, d1, dq;  // 4 alpha, 4 gamma, d1, 128 alpha (quadruple q+32)
    float4 sgn[16];
};
static_assert(sizeof(PassTab) == 272, "PassTab layout");

// Shared memory of a generate CTA.  Dynamic shared memory starts at window
// address `base` (1024 on sm_103a: the first KB is reserved).  At its start:
// partial sums [2][32], the control state, and two sets of r_max pass tables
// (this block's and the next one's); then the two pool buffers, each at a
// window address that is a multiple of its size 4 n_max, so that a gather
// address is (offset & (4N-1)) | buffer -- one LOP3.
__host__ __device__ inline uint32_t small_bytes(uint32_t r_max)
{
    return 256 + (uint32_t)sizeof(CtlState) + 2 * r_max * (uint32_t)sizeof(PassTab);
}
__host__ __device__ inline uint32_t pool_window(uint32_t base, uint32_t n_max, uint32_t r_max)
{
    const uint32_t sz = 4 * n_max;
    return (base + small_bytes(r_max) + sz - 1) / sz * sz;
}
__host__ __device__ inline size_t gen_smem_bytes(uint32_t base, uint32_t n_max, uint32_t r_max)
{
    return (size_t)pool_window(base, n_max, r_max) + 8 * (size_t)n_max - base;
}
// The in-place layout: one pool buffer right after the small part (a 16-byte
// multiple); gather addresses are then offset + buffer instead of the OR of
// an aligned window (aligning one 64 KB buffer would cost a whole pool, as the
// window's first KB is reserved).
__host__ __device__ inline uint32_t pool_window_ip(uint32_t base, uint32_t r_max) { return base + small_bytes(r_max); }
__host__ __device__ inline size_t gen_smem_bytes_ip(uint32_t n_max, uint32_t r_max)
{
    return (size_t)small_bytes(r_max) + 4 * (size_t)n_max;
}

// --- shared-memory and packed-FP32 primitives ------------------------------
extern __shared__ __align__(16) unsigned char wn_smem[];
__device__ __forceinline__ uint32_t smem_base() { return (uint32_t)__cvta_generic_to_shared(wn_smem); }

// The debug build checks every pool access against the CTA's dynamic shared
// memory (window address and alignment; see DbgRange).
__device__ __forceinline__ bool dbg_shared_ok(uint32_t a, uint32_t bytes)
{
#ifdef WN_DEBUG
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const uint32_t base = smem_base();
    if (a < base || a + bytes > base + dyn || a % bytes != 0) {
        dbg_fail(1, a);
        return false;
    }
#else
    (void)a;
    (void)bytes;
#endif
    return true;
}

// Pool accesses by shared-window address.  ptxas orders ld/st.shared against
// bar.sync itself, and the volatile asm keeps the compiler from moving them
// across __syncthreads().
__device__ __forceinline__ float lds(uint32_t a)
{
    if (!dbg_shared_ok(a, 4)) return 0.f;
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float4 lds4(uint32_t a)
{
    if (!dbg_shared_ok(a, 16)) return make_float4(0.f, 0.f, 0.f, 0.f);
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ uint4 lds4u(uint32_t a)
{
    if (!dbg_shared_ok(a, 16)) return make_uint4(0u, 0u, 0u, 0u);
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts4(uint32_t a, float2 lo, float2 hi)
{
    if (!dbg_shared_ok(a, 16)) return;
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(lo.x), "f"(lo.y), "f"(hi.x), "f"(hi.y));
}

__device__ __forceinline__ void sts1(uint32_t a, float v)
{
    if (!dbg_shared_ok(a, 4)) return;
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v));
}

// Named barriers of the latency mode (0 is __syncthreads): the compute warps
// end each pass on kBarPass among themselves; once per block the two control
// warps hand over the block's scale and the next block's tables (kBarReady:
// they arrive, the compute warps wait) and take back the block's partial sums
// and reserved slot (kBarDone: the compute warps arrive, they wait).  An
// arrive never waits; the writes before it are fenced for the waiting side.
constexpr uint32_t kBarPass = 1, kBarReady = 2, kBarDone = 3;
// In-place layout: the compute warps finish every gather of a pass before any
// of them overwrites the pool (kBarGather, among themselves).
constexpr uint32_t kBarGather = 4;
__device__ __forceinline__ void bar_wait(uint32_t id, uint32_t n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_signal(uint32_t id, uint32_t n)
{
    __threadfence_block();
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ unsigned long long f2u(float2 v) { return *reinterpret_cast<unsigned long long *>(&v); }
__device__ __forceinline__ float2 u2f(unsigned long long v) { return *reinterpret_cast<float2 *>(&v); }
// Blackwell packed FP32 pairs: one instruction, two IEEE round-to-nearest results.
__device__ __forceinline__ float2 fmul2(float2 a, float2 b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(d);
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(d);
}
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)), "l"(f2u(c)));
    return u2f(d);
}

__device__ __forceinline__ float neg_sign_one(uint32_t bit) { return __uint_as_float(0xbf800000u ^ (bit << 31)); }

// Control warp: draw the R passes' (w_a, w_s) of the coming block from the
// stream generator, in the order the method draws them, and tabulate them.
// With `rot` (the plane-rotation form of Section 5.3) the second draw gives
// t = (2u + 1)/2^24 - 1, u its top 24 bits, and the pass rotates pairs by
// c = (1 - t^2)/(1 + t^2), s = 2t/(1 + t^2) (FP64, rounded to FP32 once); the
// table then describes quadruple q as the pairs 2q and 2q+1: element 0 at
// 8 alpha q + 4 gamma, element 2 its partner N/2 away, elements 1 and 3 the
// next pair (offset 4 alpha), and every sgn entry holds (c, s, c, s).
__device__ __forceinline__ void make_tables(CtlState *ctl, PassTab *tab, uint32_t R, uint32_t N, uint32_t lane,
                                            bool rot)
{
    uint64_t gx = ctl->gx, gw = ctl->gw;
    for (uint32_t p = 0; p < R; ++p) {
        const uint64_t wa = draw(gx, gw);
        const uint64_t ws = draw(gx, gw);
        const uint32_t alpha = ((uint32_t)(wa >> 32) & (N - 1)) | 1u;
        const uint32_t gamma = (uint32_t)wa & (N - 1);
        if (rot) {
            if (lane < 16) {
                const double t = (double)(2u * (uint32_t)(ws >> 40) + 1u) * (1.0 / 16777216.0) - 1.0;
                const double d = 1.0 + t * t;
                const float c = (float)((1.0 - t * t) / d), sn = (float)(2.0 * t / d);
                tab[p].sgn[lane] = make_float4(c, sn, c, sn);
            } else if (lane == 16) {
                tab[p].a4 = 8u * alpha;
                tab[p].g4 = 4u * gamma;
                tab[p].d1 = 4u * alpha;
                tab[p].dq = 256u * alpha;
            }
            continue;
        }
        if (lane < 16) {
            const uint32_t nib = (uint32_t)(ws >> (4u * lane)) & 15u;
            tab[p].sgn[lane] = make_float4(neg_sign_one(nib & 1u), neg_sign_one((nib >> 1) & 1u),
                                           neg_sign_one((nib >> 2) & 1u), neg_sign_one(nib >> 3));
        } else if (lane == 16) {
            tab[p].a4 = 4u * alpha;
            tab[p].g4 = 4u * gamma;
            tab[p].d1 = (alpha & 3u) * N;
            tab[p].dq = 128u * alpha;
        }
    }
    __syncwarp();
    if (lane == 0) {
        ctl->gx = gx;
        ctl->gw = gw;
    }
}

template <typename OutT> __device__ __forceinline__ void store1(const DbgRange &rg, OutT *p, float v)
{
    if (dbg_global_ok(rg, p, sizeof(OutT))) *p = to_out<OutT>(v);
}

// Four consecutive values to an address aligned to four elements.
__device__ __forceinline__ void store4(const DbgRange &rg, float *p, float a, float b, float c, float d)
{
    if (!dbg_global_ok(rg, p, 16)) return;
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void store4(const DbgRange &rg, __nv_bfloat16 *p, float a, float b, float c, float d)
{
    if (!dbg_global_ok(rg, p, 8)) return;
    __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t *>(&lo);
    u.y = *reinterpret_cast<uint32_t *>(&hi);
    *reinterpret_cast<uint2 *>(p) = u;
}
__device__ __forceinline__ void store4(const DbgRange &rg, __half *p, float a, float b, float c, float d)
{
    if (!dbg_global_ok(rg, p, 8)) return;
    __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t *>(&lo);
    u.y = *reinterpret_cast<uint32_t *>(&hi);
    *reinterpret_cast<uint2 *>(p) = u;
}

enum { EMIT_NONE = 0, EMIT_WHOLE = 1, EMIT_PART = 2, EMIT_GBM = 3 };

// Fused Monte Carlo consumer (geometric Brownian motion): the stream's values
// drive paths and never leave the chip.  Path p of a stream takes value
// j ppg + p as its step-j normal; ppg divides N-1, so pool position i of
// every block feeds path i mod ppg.  A compute thread therefore keeps one
// running sum of the (scaled) values per pool position it owns, in
// registers; at the end the k = (N-1)/ppg sums of each path are added and
// S_T = S0 exp(steps (mu - sigma^2/2) dt + sigma sqrt(dt) sum).
struct GbmArgs {
    float *st;          // terminal prices: stream i writes st[i ppg .. i ppg + ppg)
    uint32_t ppg;       // paths per stream
    float S0;           // initial price
    float drift_total;  // steps (mu - sigma^2/2) dt
    float vol;          // sigma sqrt(dt)
};

// One pass over this thread's quadruples q = q0 + 32 j (j < QT): gather from
// the buffer at window address rd, store the four results contiguously into
// the buffer at wr.  All gathers are issued before any arithmetic.  The
// update y_k = s_k (S/2 - a_k), S = a_0 + a_1 + a_2 + a_3, is computed as
// m_k a_k + h_k S with m_k = -s_k and h_k = -m_k/2 (both products exact, so
// the one rounding is that of S/2 - a_k).
//
// The final pass of a block (FINAL) also sums the squares of its results
// (the next block's renormalisation) and, when EMIT is set, writes the
// block's values scaled by sc to ob[4q+k] (value N-1 is the reserved one and
// is never written):
//  * EMIT_WHOLE, A = (element offset of ob from a 16-byte boundary) mod 4:
//    each thread stores, as one aligned 16-byte (FP32) or 8-byte (16-bit)
//    store, the group holding its first value: the previous quadruple's last
//    A values (lane - 1 by shuffle; for lane 0, lane 31's values of the
//    previous j) and its own first 4 - A.  Only a warp's first quadruple
//    (predecessor in another warp) and last one (successor in another warp,
//    or the reserved slot) use single stores;
//  * EMIT_PART: the first n values of a partial last block, single stores.
//  * EMIT_GBM: add the scaled values to the per-position sums `acc`.
// nsync barriers separate the arithmetic (and the pool's stores) from the
// scaled output, so that the control warp's scale for this block is visible:
// one with one pass per block, two when the scale depends on this block's own
// reserved slot (fastnorm's reserved value).
//
// HAND (latency mode): instead of the nsync barriers, the owner of slot N-1
// stores its value at window address rsv and the compute warps take the
// scale from the control warps at kBarReady (nthr threads: the whole CTA).
//
// IP (in-place layout, rd == wr): addresses are offset + rd, the compute
// warps (nthr threads) meet at kBarGather between their gathers and their
// stores, and the final pass also stores slot N-1 at rsv (the control warp
// reads the reserved value there, never from the pool being overwritten).
template <int QT, bool FINAL, bool FULL, int EMIT, int A, typename OutT, bool ROT, bool HAND = false,
          bool IP = false>
__device__ __forceinline__ void pass_quads(uint32_t rd, uint32_t wr, uint32_t tab, uint32_t q0, uint32_t lane,
                                           uint32_t m4, uint32_t half, uint32_t nq, float2 &part, int nsync,
                                           OutT *__restrict__ ob, const float *sc_ptr, uint32_t n,
                                           float2 (&acc)[QT][2], uint32_t rsv = 0, uint32_t nthr = 0,
                                           const DbgRange &rg = DbgRange{})
{
    static_assert(!(HAND && IP), "the latency mode keeps two pool buffers");
    const uint4 P = lds4u(tab);
    const float4 sg = lds4(tab + 16u + 16u * (lane & 15u));
    const float2 m01 = make_float2(sg.x, sg.y), m23 = make_float2(sg.z, sg.w);
    const float2 h01 = fmul2(m01, make_float2(-0.5f, -0.5f)), h23 = fmul2(m23, make_float2(-0.5f, -0.5f));
    const uint32_t B0 = P.x * q0 + P.y;
    float a[QT][4];
#pragma unroll
    for (int j = 0; j < QT; ++j) {
        if (FULL || q0 + 32u * j < nq) {
            const uint32_t B = B0 + (uint32_t)j * P.w;
            if (IP) {
                const uint32_t o0 = B & m4, o1 = (B + P.z) & m4;
                a[j][0] = lds(o0 + rd);
                a[j][2] = lds((o0 ^ half) + rd);
                a[j][1] = lds(o1 + rd);
                a[j][3] = lds((o1 ^ half) + rd);
            } else {
                const uint32_t p0 = (B & m4) | rd;
                const uint32_t p1 = ((B + P.z) & m4) | rd;
                a[j][0] = lds(p0);
                a[j][2] = lds(p0 ^ half);
                a[j][1] = lds(p1);
                a[j][3] = lds(p1 ^ half);
            }
        } else {
            a[j][0] = a[j][1] = a[j][2] = a[j][3] = 0.f;
        }
    }
    if (IP) bar_wait(kBarGather, nthr);  // the pool is read: it may now be overwritten
    float2 y[QT][2];
#pragma unroll
    for (int j = 0; j < QT; ++j) {
        const uint32_t q = q0 + 32u * j;
        if (ROT) {  // pairs (a0, a2) and (a1, a3) rotated by (c, s) = m01
            const float c = m01.x, sn = m01.y;
            y[j][0] = make_float2(fmaf(c, a[j][0], sn * a[j][2]), fmaf(c, a[j][2], -sn * a[j][0]));
            y[j][1] = make_float2(fmaf(c, a[j][1], sn * a[j][3]), fmaf(c, a[j][3], -sn * a[j][1]));
        } else {
            const float2 a01 = make_float2(a[j][0], a[j][1]), a23 = make_float2(a[j][2], a[j][3]);
            const float2 s2 = fadd2(a01, a23);
            const float sum = s2.x + s2.y;
            const float2 SS = make_float2(sum, sum);
            y[j][0] = ffma2(m01, a01, fmul2(h01, SS));
            y[j][1] = ffma2(m23, a23, fmul2(h23, SS));
        }
        if (FULL || q < nq) {
            sts4(wr + 16u * q, y[j][0], y[j][1]);
            if (FINAL) part = ffma2(y[j][0], y[j][0], ffma2(y[j][1], y[j][1], part));
            if (FINAL && (HAND || IP) && (!FULL || j == QT - 1) && q + 1u == nq) sts1(rsv, y[j][1].y);  // slot N-1
        }
    }
    if (FINAL && HAND) bar_wait(kBarReady, nthr);
    if (!FINAL || EMIT == EMIT_NONE) return;
    if (!HAND && nsync > 0) __syncthreads();
    if (!HAND && nsync > 1) __syncthreads();
    const float sc = *sc_ptr;
    const float2 sc2 = make_float2(sc, sc);
    if (EMIT == EMIT_GBM) {
#pragma unroll
        for (int j = 0; j < QT; ++j) {
            acc[j][0] = ffma2(y[j][0], sc2, acc[j][0]);
            acc[j][1] = ffma2(y[j][1], sc2, acc[j][1]);
        }
        return;
    }
    const uint32_t src = (lane + 31u) & 31u;
    const bool l31 = (lane == 31u);
    float l1 = 0.f, l2 = 0.f, l3 = 0.f;  // this thread's values 1..3 of the previous j
#pragma unroll
    for (int j = 0; j < QT; ++j) {
        const uint32_t q = q0 + 32u * j;
        const bool act = FULL || q < nq;
        const float2 v01 = fmul2(y[j][0], sc2), v23 = fmul2(y[j][1], sc2);
        const uint32_t pos = 4u * q;
        if (EMIT == EMIT_PART) {
            if (act) {
                if (pos < n) store1(rg, ob + pos, v01.x);
                if (pos + 1 < n) store1(rg, ob + pos + 1, v01.y);
                if (pos + 2 < n) store1(rg, ob + pos + 2, v23.x);
                if (pos + 3 < n) store1(rg, ob + pos + 3, v23.y);
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
        if (!act) continue;
        // the quadruple holding the reserved slot N-1 (in a FULL launch it can
        // only be the last j)
        const bool last = (FULL && j != QT - 1) ? false : (q + 1u == nq);
        if (A == 0) {
            if (!last) store4(rg, ob + pos, v01.x, v01.y, v23.x, v23.y);
            else {
                store1(rg, ob + pos, v01.x);
                store1(rg, ob + pos + 1, v01.y);
                store1(rg, ob + pos + 2, v23.x);
            }
            continue;
        }
        if (j == 0 && lane == 0) {  // predecessor in another warp: own first 4 - A only
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

// ---------------------------------------------------------------------------
// One stream's share of a call: return the rest of the last block, then run
// as many whole blocks as `count` needs, then write the state back.
//
// Warp 0 is the control warp; warps 1.. are compute warps (T = blockDim.x -
// 32 threads, T QT >= N/4; FULL: equal for every stream of the launch);
// compute thread (warp w, lane l) owns quadruples q0 + 32 j,
// q0 = (w - 1) 32 QT + l.  Phases are passes, separated by barriers.  In the
// first phase of block b the control warp forms block b's scale -- from the
// sum of squares the previous block's final pass left in `red` (or, for the
// call's first block, the one stored with the stream) and the previous
// block's reserved value.  The compute
// warps' final pass of block b then writes the block's values from
// registers, while the control warp tabulates block b+1's passes.  With one
// pass per block the final pass is also the first, so it waits for the scale
// at a mid-phase barrier.
// ---------------------------------------------------------------------------
template <int QT, bool FULL, typename OutT, bool GBM, bool VAR, bool ROT, bool IP = false>
__device__ __forceinline__ void run_stream(StreamHdr *__restrict__ h, float *__restrict__ pool_g,
                                           OutT *__restrict__ out, uint64_t out_off, uint64_t count,
                                           bool store, uint32_t n_max, uint32_t r_max, const GbmArgs &gbm)
{
    static_assert(!(GBM && IP), "the GBM consumer keeps its path sums in the second pool buffer");
    unsigned char *smem = wn_smem;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const bool control = (warp == 0);
    const uint32_t N = h->N, nq = N >> 2;
    const uint32_t base = smem_base();
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const uint32_t W0 = IP ? pool_window_ip(base, r_max) : pool_window(base, n_max, r_max);
    if (W0 + (IP ? 4u : 8u) * n_max > base + dyn) {  // layout does not fit: flag and do nothing
        if (tid == 0) h->flags |= 1u;
        return;
    }
    float *red = reinterpret_cast<float *>(smem);  // [2][32] partial sums, by block parity
    CtlState *ctl = reinterpret_cast<CtlState *>(smem + 256);
    PassTab *tabs = reinterpret_cast<PassTab *>(smem + 256 + sizeof(CtlState));  // [2][r_max]
    const uint32_t tabs_s = base + 256u + (uint32_t)sizeof(CtlState);
    const DbgRange rg = dbg_range(out, out + count);  // this stream's output (the debug build checks stores)
    // bytes per buffer; buffer i at window W0 + i bsz (in place: one buffer)
    const uint32_t bsz = IP ? 0u : 4u * n_max;
    const uint32_t nwc = (blockDim.x >> 5) - 1u;  // compute warps
    const uint32_t ncomp = blockDim.x - 32u;
    const uint32_t q0 = (warp - 1u) * 32u * QT + lane;
    const uint32_t m4 = 4u * N - 1u, half = 2u * N;

    {
        const float4 *pg4 = reinterpret_cast<const float4 *>(pool_g);
        float4 *b04 = reinterpret_cast<float4 *>(smem + (W0 - base));
        for (uint32_t i = tid; i < nq; i += blockDim.x) b04[i] = pg4[i];
    }
    const uint32_t k0 = h->k;
    const float sc_prev = h->scale;
    const uint64_t left = (uint64_t)(N - 1 - k0);
    const uint64_t n0 = left < count ? left : count;
    const uint64_t nb = (count - n0 + (N - 2)) / (N - 1);
    const uint64_t tail = (count - n0) % (N - 1);  // values of a partial last block (0: whole)
    const uint32_t R = h->R;
    const uint32_t variant = VAR ? h->variant : VAR_CHI2_C;  // !VAR: the plain method, folded at compile time
    const bool wh = var_chi2(variant) == VAR_CHI2_B;  // Wilson-Hilferty form of the scale
    const bool late = var_current(variant);           // reserved value from this block's own pool
    const uint32_t dec = (store || GBM) ? var_decimate(variant) : 1u;  // blocks run per returned block
    const uint64_t nrun = nb * dec;

    if (control) {
        if (lane == 0) {
            ctl->gx = h->x;
            ctl->gw = h->w;
            ctl->sumsq = h->sumsq;
            ctl->r = (float)h->r;
            ctl->A = (float)h->A;
            ctl->B = (float)h->B;
            ctl->sc[1] = sc_prev;
        }
        __syncwarp();
        if (nb > 0) make_tables(ctl, tabs, R, N, lane, ROT);
    }
    __syncthreads();
    if (store)
        for (uint64_t i = tid; i < n0; i += blockDim.x)
            store1(rg, out + i, sc_prev * lds(W0 + 4u * (uint32_t)(k0 + i)));
    if (IP && store && n0 > 0) __syncthreads();  // the control warp's reads precede the first pass's stores

    // Control warp: FP64 sum of the compute warps' partial sums of squares of
    // parity `par` (the pool at the end of that block).
    auto sum_partials = [&](uint32_t par) {
        const float *rb = red + par * 32;
        double v = (lane < nwc) ? (double)rb[lane] : 0.0;
        for (uint32_t o = 1; o < 32; o <<= 1)
            if (o < nwc) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
    // Control warp: block b's scale sqrt(S / sum of squares) (Section 5.5).
    // rslot is the window address of a pool's slot N-1 (unscaled): the
    // previous block's (fastnorm2: its reserved value times that block's
    // scale; in place, the copy the final pass left in the partial-sum array,
    // since the first pass may already be overwriting the pool) or, with
    // `late`, this block's own (fastnorm: renormalised).
    auto form_scale = [&](uint64_t b, uint32_t rslot) {
        const double ss = (b == 0) ? ctl->sumsq : sum_partials((uint32_t)((b - 1) & 1));
        const float invNf = 1.0f / (float)N;  // exact: N is a power of two
        const float delta = (float)fma(ss, (double)invNf, -1.0);  // sum/N - 1
        const float c = __frsqrt_rn(1.0f + delta);                // sqrt(N / sum)
        const float r = late ? c * lds(rslot) : (b == 0) ? ctl->r : ctl->sc[(b - 1) & 1] * lds(rslot);
        float u;  // S/N - 1
        if (wh) {
            const float d = fmaf(ctl->A, r, -ctl->B);
            u = d * fmaf(d, d + 3.0f, 3.0f);  // (1 + d)^3 - 1
        } else {
            u = fmaf(ctl->A, fmaf(r, r, -1.0f), ctl->B * r) * invNf;
        }
        const float sv = __fsqrt_rn(1.0f + u) * c;  // sqrt(S / sum)
        __syncwarp();
        if (lane == 0) ctl->sc[b & 1] = sv;
    };

    OutT *ob = out + n0;
    uint32_t a = (uint32_t)((out_off + n0) & 3u);  // alignment of ob within 16 bytes
    uint32_t cb = 0;                               // buffer (0 or 1) holding the current pool
    const bool one_pass = (R == 1);
    const int nsync = late ? 2 : (one_pass ? 1 : 0);  // barriers inside the final pass
    float2 acc[QT][2];  // GBM: running sums of this thread's pool positions
#pragma unroll
    for (int j = 0; j < QT; ++j) acc[j][0] = acc[j][1] = make_float2(0.f, 0.f);
    uint32_t dc = 0;  // blocks run since the last returned one (decimation)
    uint64_t e = 0;   // blocks returned so far
    for (uint64_t b = 0; b < nrun; ++b) {
        const uint32_t tb = tabs_s + (uint32_t)(b & 1) * r_max * (uint32_t)sizeof(PassTab);
        for (uint32_t p = 0; p < R; ++p) {
            const uint32_t rd = W0 + cb * bsz, wr = W0 + (cb ^ 1u) * bsz;
            const uint32_t tp = tb + p * (uint32_t)sizeof(PassTab);
            if (control) {
                // scale in the first phase, the next block's tables in the
                // second (the final pass, which carries the stores): the two
                // serial chains then each overlap a phase of compute work
                if (p == 0 && !late) {
                    form_scale(b, IP ? base + 4u * ((uint32_t)((b - 1) & 1) * 32u + 31u) : rd + 4u * (N - 1u));
                    if (one_pass) __syncthreads();  // pairs with the final pass's mid-phase barrier
                }
                if (p == (one_pass ? 0u : 1u) && b + 1 < nrun)
                    make_tables(ctl, tabs + ((b + 1) & 1) * r_max, R, N, lane, ROT);
                if (late && p + 1 == R) {  // between the final pass's pool stores and its output
                    __syncthreads();
                    form_scale(b, wr + 4u * (N - 1u));
                    __syncthreads();
                }
            } else if (p + 1 < R) {
                float2 part;
                pass_quads<QT, false, FULL, EMIT_NONE, 0, OutT, ROT, false, IP>(
                    rd, wr, tp, q0, lane, m4, half, nq, part, 0, nullptr, nullptr, 0, acc, 0, ncomp);
            } else {
                float2 part = make_float2(0.f, 0.f);
                const float *scp = &ctl->sc[b & 1];
                const uint32_t rsv = base + 4u * ((uint32_t)(b & 1) * 32u + 31u);  // in place: slot N-1's copy
                const bool emit = (dec == 1) || (dc + 1 == dec);  // decimation: a block to return
                const bool whole = ((dec == 1 ? b : e) + 1 < nb) || tail == 0;
                if (GBM && emit) {
                    pass_quads<QT, true, FULL, EMIT_GBM, 0, OutT, ROT, false, IP>(
                        rd, wr, tp, q0, lane, m4, half, nq, part, nsync, ob, scp, 0, acc, rsv, ncomp, rg);
                } else if (!store || !emit) {
                    pass_quads<QT, true, FULL, EMIT_NONE, 0, OutT, ROT, false, IP>(
                        rd, wr, tp, q0, lane, m4, half, nq, part, 0, ob, scp, 0, acc, rsv, ncomp, rg);
                    if (nsync > 0) __syncthreads();
                    if (nsync > 1) __syncthreads();
                } else if (!whole) {
                    pass_quads<QT, true, FULL, EMIT_PART, 0, OutT, ROT, false, IP>(
                        rd, wr, tp, q0, lane, m4, half, nq, part, nsync, ob, scp, (uint32_t)tail, acc, rsv, ncomp, rg);
                } else {
                    switch (a) {
                    case 0:
                        pass_quads<QT, true, FULL, EMIT_WHOLE, 0, OutT, ROT, false, IP>(
                            rd, wr, tp, q0, lane, m4, half, nq, part, nsync, ob, scp, 0, acc, rsv, ncomp, rg);
                        break;
                    case 1:
                        pass_quads<QT, true, FULL, EMIT_WHOLE, 1, OutT, ROT, false, IP>(
                            rd, wr, tp, q0, lane, m4, half, nq, part, nsync, ob, scp, 0, acc, rsv, ncomp, rg);
                        break;
                    case 2:
                        pass_quads<QT, true, FULL, EMIT_WHOLE, 2, OutT, ROT, false, IP>(
                            rd, wr, tp, q0, lane, m4, half, nq, part, nsync, ob, scp, 0, acc, rsv, ncomp, rg);
                        break;
                    default:
                        pass_quads<QT, true, FULL, EMIT_WHOLE, 3, OutT, ROT, false, IP>(
                            rd, wr, tp, q0, lane, m4, half, nq, part, nsync, ob, scp, 0, acc, rsv, ncomp, rg);
                        break;
                    }
                }
                float ps = part.x + part.y;
                for (int o = 16; o > 0; o >>= 1) ps += __shfl_xor_sync(0xffffffffu, ps, o);
                if (lane == 0) red[(b & 1) * 32 + (warp - 1)] = ps;
            }
            cb ^= 1u;
            __syncthreads();
        }
        if ((dec == 1) || (dc + 1 == dec)) {  // the block was returned
            ob += N - 1;
            a = (a + N - 1) & 3u;
            ++e;
            dc = 0;
        } else {
            ++dc;
        }
    }

    {
        float4 *pw4 = reinterpret_cast<float4 *>(pool_g);
        for (uint32_t i = tid; i < nq; i += blockDim.x) pw4[i] = lds4(W0 + cb * bsz + 16u * i);
    }
    if (control && nb > 0) {
        const double ss = sum_partials((uint32_t)((nrun - 1) & 1));
        if (lane == 0) {
            const float sc = ctl->sc[(nrun - 1) & 1];
            h->x = ctl->gx;
            h->w = ctl->gw;
            h->sumsq = ss;
            h->r = (double)(sc * lds(W0 + cb * bsz + 4u * (N - 1)));
            h->scale = sc;
            h->k = tail == 0 ? N - 1 : (uint32_t)tail;
            h->blocks += nrun;
        }
    } else if (tid == 0 && nb == 0) {
        h->k = k0 + (uint32_t)n0;
    }
    if (GBM) {
        // per-position sums into the buffer that does not hold the pool, then
        // each path adds its k = (N-1)/ppg positions
        const uint32_t accb = W0 + (cb ^ 1u) * bsz;
        if (!control) {
#pragma unroll
            for (int j = 0; j < QT; ++j) {
                const uint32_t q = q0 + 32u * j;
                if (FULL || q < nq) sts4(accb + 16u * q, acc[j][0], acc[j][1]);
            }
        }
        __syncthreads();
        const uint32_t k = (N - 1) / gbm.ppg;
        for (uint32_t p = tid; p < gbm.ppg; p += blockDim.x) {
            float tot = 0.f;
            for (uint32_t m = 0; m < k; ++m) tot += lds(accb + 4u * (p + m * gbm.ppg));
            gbm.st[(uint64_t)blockIdx.x * gbm.ppg + p] = gbm.S0 * expf(fmaf(gbm.vol, tot, gbm.drift_total));
        }
    }
}

// ---------------------------------------------------------------------------
// Latency mode (the plain method, launches of few streams: a stream is a
// serial chain, so a lone stream waits on every step of every block).  Two
// control warps run beside the compute warps instead of inside their pass
// barriers: warp 0 forms each block's scale (the FP64 sum of the partial
// sums, Section 5.5), warp 1 draws and tabulates the next block's passes
// (Section 5.4); compute warps 2.. own quadruples q0 + 32 j,
// q0 = (w - 2) 32 QT + l, end each pass on a barrier among themselves, and
// once per block take the scale and the next tables (kBarReady, in the final
// pass between its arithmetic and its output) and return the block's partial
// sums of squares and reserved slot (kBarDone).  The arithmetic is
// run_stream's (passes, per-warp partial sums, FP64 cross-warp sum, scale,
// emission): bit-identical for the same compute-warp layout.
// ---------------------------------------------------------------------------
template <int QT, bool FULL, typename OutT>
__device__ __forceinline__ void run_stream_lat(StreamHdr *__restrict__ h, float *__restrict__ pool_g,
                                               OutT *__restrict__ out, uint64_t out_off, uint64_t count,
                                               uint32_t n_max, uint32_t r_max)
{
    unsigned char *smem = wn_smem;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t N = h->N, nq = N >> 2;
    const uint32_t base = smem_base();
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const uint32_t W0 = pool_window(base, n_max, r_max);
    if (W0 + 8u * n_max > base + dyn) {  // layout does not fit: flag and do nothing
        if (tid == 0) h->flags |= 1u;
        return;
    }
    float *red = reinterpret_cast<float *>(smem);  // [2][32] partial sums by block parity; [par][31]: slot N-1
    const DbgRange rg = dbg_range(out, out + count);
    CtlState *ctl = reinterpret_cast<CtlState *>(smem + 256);
    PassTab *tabs = reinterpret_cast<PassTab *>(smem + 256 + sizeof(CtlState));  // [2][r_max]
    const uint32_t tabs_s = base + 256u + (uint32_t)sizeof(CtlState);
    const uint32_t bsz = 4u * n_max;
    const uint32_t nthr = blockDim.x, ncomp = nthr - 64u, nwc = ncomp >> 5;
    const uint32_t q0 = (warp - 2u) * 32u * QT + lane;
    const uint32_t m4 = 4u * N - 1u, half = 2u * N;

    {
        const float4 *pg4 = reinterpret_cast<const float4 *>(pool_g);
        float4 *b04 = reinterpret_cast<float4 *>(smem + (W0 - base));
        for (uint32_t i = tid; i < nq; i += blockDim.x) b04[i] = pg4[i];
    }
    const uint32_t k0 = h->k;
    const float sc_prev = h->scale;
    const uint64_t left = (uint64_t)(N - 1 - k0);
    const uint64_t n0 = left < count ? left : count;
    const uint64_t nb = (count - n0 + (N - 2)) / (N - 1);
    const uint64_t tail = (count - n0) % (N - 1);
    const uint32_t R = h->R;
    if (warp == 0 && lane == 0) {
        ctl->gx = h->x;
        ctl->gw = h->w;
        ctl->sumsq = h->sumsq;
        ctl->r = (float)h->r;
        ctl->A = (float)h->A;
        ctl->B = (float)h->B;
        ctl->sc[1] = sc_prev;
    }
    __syncthreads();
    if (warp == 1 && nb > 0) make_tables(ctl, tabs, R, N, lane, false);
    for (uint64_t i = tid; i < n0; i += blockDim.x) store1(rg, out + i, sc_prev * lds(W0 + 4u * (uint32_t)(k0 + i)));
    __syncthreads();  // block 0's tables are there and buffer 0 has been read

    uint32_t cb = (uint32_t)((nb * R) & 1u);  // the control warps only need the final buffer
    if (warp == 0) {
        for (uint64_t b = 0; b < nb; ++b) {
            if (b > 0) bar_wait(kBarDone, nthr);
            double ss;
            if (b == 0) {
                ss = ctl->sumsq;
            } else {
                const float *rb = red + ((b - 1) & 1) * 32;
                double v = (lane < nwc) ? (double)rb[lane] : 0.0;
                for (uint32_t o = 1; o < 32; o <<= 1)
                    if (o < nwc) v += __shfl_xor_sync(0xffffffffu, v, o);
                ss = v;
            }
            const float r = (b == 0) ? ctl->r : ctl->sc[(b - 1) & 1] * red[((b - 1) & 1) * 32 + 31];
            const float invNf = 1.0f / (float)N;
            const float delta = (float)fma(ss, (double)invNf, -1.0);
            const float c = __frsqrt_rn(1.0f + delta);
            const float u = fmaf(ctl->A, fmaf(r, r, -1.0f), ctl->B * r) * invNf;
            const float sv = __fsqrt_rn(1.0f + u) * c;
            __syncwarp();
            if (lane == 0) ctl->sc[b & 1] = sv;
            bar_signal(kBarReady, nthr);
        }
    } else if (warp == 1) {
        for (uint64_t b = 0; b < nb; ++b) {
            if (b > 0) bar_wait(kBarDone, nthr);
            if (b + 1 < nb) make_tables(ctl, tabs + ((b + 1) & 1) * r_max, R, N, lane, false);
            bar_signal(kBarReady, nthr);
        }
    } else {
        float2 acc[QT][2];
        cb = 0;
        OutT *ob = out + n0;
        uint32_t a = (uint32_t)((out_off + n0) & 3u);
        for (uint64_t b = 0; b < nb; ++b) {
            const uint32_t tb = tabs_s + (uint32_t)(b & 1) * r_max * (uint32_t)sizeof(PassTab);
            for (uint32_t p = 0; p < R; ++p) {
                const uint32_t rd = W0 + cb * bsz, wr = W0 + (cb ^ 1u) * bsz;
                const uint32_t tp = tb + p * (uint32_t)sizeof(PassTab);
                if (p + 1 < R) {
                    float2 part;
                    pass_quads<QT, false, FULL, EMIT_NONE, 0, OutT, false>(rd, wr, tp, q0, lane, m4, half, nq, part,
                                                                          0, nullptr, nullptr, 0, acc);
                } else {
                    float2 part = make_float2(0.f, 0.f);
                    const float *scp = &ctl->sc[b & 1];
                    const uint32_t rsv = base + 4u * ((uint32_t)(b & 1) * 32u + 31u);
                    const bool whole = (b + 1 < nb) || tail == 0;
                    if (!whole) {
                        pass_quads<QT, true, FULL, EMIT_PART, 0, OutT, false, true>(
                            rd, wr, tp, q0, lane, m4, half, nq, part, 0, ob, scp, (uint32_t)tail, acc, rsv, nthr, rg);
                    } else {
                        switch (a) {
                        case 0:
                            pass_quads<QT, true, FULL, EMIT_WHOLE, 0, OutT, false, true>(
                                rd, wr, tp, q0, lane, m4, half, nq, part, 0, ob, scp, 0, acc, rsv, nthr, rg);
                            break;
                        case 1:
                            pass_quads<QT, true, FULL, EMIT_WHOLE, 1, OutT, false, true>(
                                rd, wr, tp, q0, lane, m4, half, nq, part, 0, ob, scp, 0, acc, rsv, nthr, rg);
                            break;
                        case 2:
                            pass_quads<QT, true, FULL, EMIT_WHOLE, 2, OutT, false, true>(
                                rd, wr, tp, q0, lane, m4, half, nq, part, 0, ob, scp, 0, acc, rsv, nthr, rg);
                            break;
                        default:
                            pass_quads<QT, true, FULL, EMIT_WHOLE, 3, OutT, false, true>(
                                rd, wr, tp, q0, lane, m4, half, nq, part, 0, ob, scp, 0, acc, rsv, nthr, rg);
                            break;
                        }
                    }
                    float ps = part.x + part.y;
                    for (int o = 16; o > 0; o >>= 1) ps += __shfl_xor_sync(0xffffffffu, ps, o);
                    if (lane == 0) red[(b & 1) * 32 + (warp - 2)] = ps;
                    if (b + 1 < nb) bar_signal(kBarDone, nthr);
                }
                cb ^= 1u;
                bar_wait(kBarPass, ncomp);
            }
            ob += N - 1;
            a = (a + N - 1) & 3u;
        }
    }
    __syncthreads();

    {
        float4 *pw4 = reinterpret_cast<float4 *>(pool_g);
        for (uint32_t i = tid; i < nq; i += blockDim.x) pw4[i] = lds4(W0 + cb * bsz + 16u * i);
    }
    if (warp == 0 && nb > 0) {
        const float *rb = red + ((nb - 1) & 1) * 32;
        double v = (lane < nwc) ? (double)rb[lane] : 0.0;
        for (uint32_t o = 1; o < 32; o <<= 1)
            if (o < nwc) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) {
            const float sc = ctl->sc[(nb - 1) & 1];
            h->x = ctl->gx;
            h->w = ctl->gw;
            h->sumsq = v;
            h->r = (double)(sc * red[((nb - 1) & 1) * 32 + 31]);
            h->scale = sc;
            h->k = tail == 0 ? N - 1 : (uint32_t)tail;
            h->blocks += nb;
        }
    } else if (tid == 0 && nb == 0) {
        h->k = k0 + (uint32_t)n0;
    }
}

// Latency-mode generate kernel: one CTA per stream, blockDim = compute
// threads + 64 (two control warps).
template <int QT, int MAXT, int MINB, bool FULL, typename OutT>
__global__ void __launch_bounds__(MAXT, MINB) latency_kernel(GenArgs a)
{
    StreamHdr *h = a.hdr + blockIdx.x;
    const uint64_t off = (uint64_t)blockIdx.x * a.out_stride;
    run_stream_lat<QT, FULL, OutT>(h, a.pools + h->pool_off, reinterpret_cast<OutT *>(a.out) + off, off, a.count,
                                   a.n_max, a.r_max);
}

// FULL: every stream of the launch has exactly (blockDim.x - 32) * QT
// quadruples, so no quadruple index needs a bounds check.  IP: the in-place
// pool layout.
template <int QT, int MAXT, int MINB, bool FULL, typename OutT, bool VAR, bool IP = false>
__global__ void __launch_bounds__(MAXT, MINB) generate_kernel(GenArgs a)
{
    StreamHdr *h = a.hdr + blockIdx.x;
    const uint32_t N = h->N;
    const uint64_t count = a.warmup_blocks ? (uint64_t)a.warmup_blocks * (N - 1) : a.count;
    const uint64_t off = (uint64_t)blockIdx.x * a.out_stride;
    OutT *out = a.out ? reinterpret_cast<OutT *>(a.out) + off : nullptr;
    const GbmArgs none{};
    if (VAR && var_rotation(h->variant))
        run_stream<QT, FULL, OutT, false, VAR, true, IP>(h, a.pools + h->pool_off, out, off, count,
                                                         a.warmup_blocks == 0, a.n_max, a.r_max, none);
    else
        run_stream<QT, FULL, OutT, false, VAR, false, IP>(h, a.pools + h->pool_off, out, off, count,
                                                          a.warmup_blocks == 0, a.n_max, a.r_max, none);
}

// The fused GBM consumer: every stream of the launch returns steps * ppg
// values (a whole number of blocks, starting at a block boundary) into path
// sums instead of memory.
template <int QT, int MAXT, int MINB, bool FULL>
__global__ void __launch_bounds__(MAXT, MINB) gbm_kernel(GenArgs a, GbmArgs g)
{
    StreamHdr *h = a.hdr + blockIdx.x;
    if (var_rotation(h->variant))
        run_stream<QT, FULL, float, true, true, true>(h, a.pools + h->pool_off, nullptr, 0, a.count, false, a.n_max,
                                                      a.r_max, g);
    else
        run_stream<QT, FULL, float, true, true, false>(h, a.pools + h->pool_off, nullptr, 0, a.count, false, a.n_max,
                                                       a.r_max, g);
}

// Work of a batch: per stream an output offset (elements from `out`) and a
// count; `order` lists the streams of one pool size, longest first.
struct BatchArgs {
    const uint32_t *order;
    const uint64_t *offsets;
    const uint64_t *counts;
    uint32_t n_items;
    uint32_t *queue;  // claim counter, zero at launch
};

// Persistent generate kernel for a batch of uneven requests: each CTA claims
// the next stream from an atomic counter (longest first), returns that
// stream's request, and claims again until the list is exhausted.  No CTA
// waits on another.
template <int QT, int MAXT, int MINB, bool FULL, typename OutT, bool VAR, bool IP = false>
__global__ void __launch_bounds__(MAXT, MINB) persist_kernel(GenArgs a, BatchArgs bq)
{
    CtlState *ctl = reinterpret_cast<CtlState *>(wn_smem + 256);
    const GbmArgs none{};
    for (;;) {
        __syncthreads();  // the previous stream is done with shared memory
        if (threadIdx.x == 0) ctl->item = atomicAdd(bq.queue, 1u);
        __syncthreads();
        const uint32_t it = ctl->item;
        if (it >= bq.n_items) return;
        const uint32_t si = bq.order[it];
        StreamHdr *h = a.hdr + si;
        const uint64_t off = bq.offsets[si];
        OutT *o = reinterpret_cast<OutT *>(a.out) + off;
        if (VAR && var_rotation(h->variant))
            run_stream<QT, FULL, OutT, false, VAR, true, IP>(h, a.pools + h->pool_off, o, off, bq.counts[si], true,
                                                             a.n_max, a.r_max, none);
        else
            run_stream<QT, FULL, OutT, false, VAR, false, IP>(h, a.pools + h->pool_off, o, off, bq.counts[si], true,
                                                              a.n_max, a.r_max, none);
    }
}

template <int QT, int MAXT, int MINB, typename OutT, bool IP = false>
cudaError_t launch_persist_shape(const GenArgs &a, const BatchArgs &bq, uint32_t threads, bool full, bool var,
                                 size_t smem, int sms, cudaStream_t cs)
{
    auto kern = full ? (var ? persist_kernel<QT, MAXT, MINB, true, OutT, true, IP>
                            : persist_kernel<QT, MAXT, MINB, true, OutT, false, IP>)
                     : (var ? persist_kernel<QT, MAXT, MINB, false, OutT, true, IP>
                            : persist_kernel<QT, MAXT, MINB, false, OutT, false, IP>);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    // every persistent kernel of a batch prefers the whole shared-memory
    // carveout: an SM's split of L1 and shared memory serves all the CTAs it
    // holds, and one preference lets any batch kernel join an SM the others use
    if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return cudaGetLastError();
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)threads + 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const uint32_t grid = std::min<uint32_t>(bq.n_items, (uint32_t)(per_sm * sms));
    if (grid == 0) return cudaSuccess;
    kern<<<grid, threads + 32, smem, cs>>>(a, bq);
    return cudaGetLastError();
}

template <typename OutT>
cudaError_t launch_persist_t(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, bool var,
                             size_t smem, int sms, cudaStream_t cs)
{
    switch (shape_key(c.qt, c.maxt, c.ip)) {
    case shape_key(1, 1024, 0):
        return launch_persist_shape<1, 1024, 1, OutT>(a, bq, c.threads, full, var, smem, sms, cs);
    case shape_key(2, 544, 0): return launch_persist_shape<2, 544, 2, OutT>(a, bq, c.threads, full, var, smem, sms, cs);
#ifndef WN_DEBUG
    case shape_key(4, 288, 0): return launch_persist_shape<4, 288, 4, OutT>(a, bq, c.threads, full, var, smem, sms, cs);
#endif
#ifndef WN_DEBUG
    case shape_key(8, 160, 0): return launch_persist_shape<8, 160, 4, OutT>(a, bq, c.threads, full, var, smem, sms, cs);
#endif
#ifndef WN_DEBUG
    case shape_key(8, 544, 0): return launch_persist_shape<8, 544, 1, OutT>(a, bq, c.threads, full, var, smem, sms, cs);
#endif
#ifndef WN_DEBUG
    case shape_key(16, 288, 0):
        return launch_persist_shape<16, 288, 1, OutT>(a, bq, c.threads, full, var, smem, sms, cs);
#endif
#ifndef WN_DEBUG
    case shape_key(16, 288, 1):
        return launch_persist_shape<16, 288, 2, OutT, true>(a, bq, c.threads, full, var, smem, sms, cs);
#endif
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_persist_f32(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, bool var,
                              size_t smem, int sms, cudaStream_t cs);
cudaError_t launch_persist_bf16(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, bool var,
                              size_t smem, int sms, cudaStream_t cs);
cudaError_t launch_persist_f16(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, bool var,
                              size_t smem, int sms, cudaStream_t cs);

// Shapes of the GBM consumer {quadruples per thread, thread bound, min CTAs
// per SM}: fewer resident CTAs than generate's, since the per-position sums
// take another 4 QT registers per thread.
constexpr int kGbmShapes[][3] = {{1, 1024, 1}, {4, 288, 3}, {8, 544, 1}};

// Launch of the GBM consumer (defined in gen_f32.cu).
cudaError_t launch_gbm(const GenArgs &a, const GbmArgs &g, const LaunchCfg &c, bool full, size_t smem,
                       cudaStream_t cs);

template <int QT, int MAXT, int MINB, typename OutT, bool IP = false>
cudaError_t launch_shape(const GenArgs &a, uint32_t threads, bool full, bool var, size_t smem, cudaStream_t cs)
{
    auto kern = full ? (var ? generate_kernel<QT, MAXT, MINB, true, OutT, true, IP>
                            : generate_kernel<QT, MAXT, MINB, true, OutT, false, IP>)
                     : (var ? generate_kernel<QT, MAXT, MINB, false, OutT, true, IP>
                            : generate_kernel<QT, MAXT, MINB, false, OutT, false, IP>);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<a.n_streams, threads + 32, smem, cs>>>(a);  // + the control warp
    return cudaGetLastError();
}

// Launch of the generate kernel for one output type (defined in gen_*.cu).
template <typename OutT>
cudaError_t launch_generate_t(const GenArgs &a, const LaunchCfg &c, bool full, bool var, size_t smem, cudaStream_t cs)
{
    switch (shape_key(c.qt, c.maxt, c.ip)) {
    case shape_key(1, 1024, 0): return launch_shape<1, 1024, 1, OutT>(a, c.threads, full, var, smem, cs);
    case shape_key(2, 544, 0): return launch_shape<2, 544, 2, OutT>(a, c.threads, full, var, smem, cs);
#ifndef WN_DEBUG
    case shape_key(4, 288, 0): return launch_shape<4, 288, 4, OutT>(a, c.threads, full, var, smem, cs);
#endif
#ifndef WN_DEBUG
    case shape_key(8, 160, 0): return launch_shape<8, 160, 4, OutT>(a, c.threads, full, var, smem, cs);
#endif
#ifndef WN_DEBUG
    case shape_key(8, 544, 0): return launch_shape<8, 544, 1, OutT>(a, c.threads, full, var, smem, cs);
#endif
#ifndef WN_DEBUG
    case shape_key(16, 288, 0): return launch_shape<16, 288, 1, OutT>(a, c.threads, full, var, smem, cs);
#endif
#ifndef WN_DEBUG
    case shape_key(16, 288, 1): return launch_shape<16, 288, 2, OutT, true>(a, c.threads, full, var, smem, cs);
#endif
    default: return cudaErrorInvalidValue;
    }
}

template <int QT, int MAXT, int MINB, typename OutT>
cudaError_t launch_latency_shape(const GenArgs &a, uint32_t threads, bool full, size_t smem, cudaStream_t cs)
{
    auto kern = full ? latency_kernel<QT, MAXT, MINB, true, OutT> : latency_kernel<QT, MAXT, MINB, false, OutT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<a.n_streams, threads + 64, smem, cs>>>(a);  // + the two control warps
    return cudaGetLastError();
}

// Persistent latency-mode kernel (batches): claims streams like
// persist_kernel and runs each with run_stream_lat.
template <int QT, int MAXT, int MINB, bool FULL, typename OutT>
__global__ void __launch_bounds__(MAXT, MINB) persist_lat_kernel(GenArgs a, BatchArgs bq)
{
    CtlState *ctl = reinterpret_cast<CtlState *>(wn_smem + 256);
    for (;;) {
        __syncthreads();  // the previous stream is done with shared memory
        if (threadIdx.x == 0) ctl->item = atomicAdd(bq.queue, 1u);
        __syncthreads();
        const uint32_t it = ctl->item;
        if (it >= bq.n_items) return;
        const uint32_t si = bq.order[it];
        StreamHdr *h = a.hdr + si;
        const uint64_t off = bq.offsets[si];
        run_stream_lat<QT, FULL, OutT>(h, a.pools + h->pool_off, reinterpret_cast<OutT *>(a.out) + off, off,
                                       bq.counts[si], a.n_max, a.r_max);
    }
}

template <int QT, int MAXT, int MINB, typename OutT>
cudaError_t launch_persist_lat_shape(const GenArgs &a, const BatchArgs &bq, uint32_t threads, bool full,
                                     size_t smem, int sms, cudaStream_t cs)
{
    auto kern = full ? persist_lat_kernel<QT, MAXT, MINB, true, OutT> : persist_lat_kernel<QT, MAXT, MINB, false, OutT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    // every persistent kernel of a batch prefers the whole shared-memory
    // carveout: an SM's split of L1 and shared memory serves all the CTAs it
    // holds, and one preference lets any batch kernel join an SM the others use
    if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return cudaGetLastError();
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)threads + 64, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const uint32_t grid = std::min<uint32_t>(bq.n_items, (uint32_t)(per_sm * sms));
    if (grid == 0) return cudaSuccess;
    kern<<<grid, threads + 64, smem, cs>>>(a, bq);
    return cudaGetLastError();
}

template <typename OutT>
cudaError_t launch_persist_lat_t(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, size_t smem,
                                 int sms, cudaStream_t cs)
{
    if (c.ip || c.threads + 64 > (uint32_t)c.maxt) return cudaErrorInvalidValue;  // two buffers, two control warps
    switch (c.qt * 10000 + c.maxt) {
    case 1 * 10000 + 1024: return launch_persist_lat_shape<1, 1024, 1, OutT>(a, bq, c.threads, full, smem, sms, cs);
    case 2 * 10000 + 544: return launch_persist_lat_shape<2, 544, 2, OutT>(a, bq, c.threads, full, smem, sms, cs);
#ifndef WN_DEBUG
    case 4 * 10000 + 288: return launch_persist_lat_shape<4, 288, 4, OutT>(a, bq, c.threads, full, smem, sms, cs);
#endif
#ifndef WN_DEBUG
    case 8 * 10000 + 160: return launch_persist_lat_shape<8, 160, 4, OutT>(a, bq, c.threads, full, smem, sms, cs);
#endif
#ifndef WN_DEBUG
    case 8 * 10000 + 544: return launch_persist_lat_shape<8, 544, 1, OutT>(a, bq, c.threads, full, smem, sms, cs);
#endif
#ifndef WN_DEBUG
    case 16 * 10000 + 288: return launch_persist_lat_shape<16, 288, 1, OutT>(a, bq, c.threads, full, smem, sms, cs);
#endif
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_persist_lat_f32(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full,
                                   size_t smem, int sms, cudaStream_t cs);
cudaError_t launch_persist_lat_bf16(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full,
                                    size_t smem, int sms, cudaStream_t cs);
cudaError_t launch_persist_lat_f16(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full,
                                   size_t smem, int sms, cudaStream_t cs);

// Latency-mode launch for one output type: the shape's thread bound must
// admit the compute threads plus two control warps.
template <typename OutT>
cudaError_t launch_latency_t(const GenArgs &a, const LaunchCfg &c, bool full, size_t smem, cudaStream_t cs)
{
    if (c.ip || c.threads + 64 > (uint32_t)c.maxt) return cudaErrorInvalidValue;  // two buffers, two control warps
    switch (c.qt * 10000 + c.maxt) {
    case 1 * 10000 + 1024: return launch_latency_shape<1, 1024, 1, OutT>(a, c.threads, full, smem, cs);
    case 2 * 10000 + 544: return launch_latency_shape<2, 544, 2, OutT>(a, c.threads, full, smem, cs);
#ifndef WN_DEBUG
    case 4 * 10000 + 288: return launch_latency_shape<4, 288, 4, OutT>(a, c.threads, full, smem, cs);
#endif
#ifndef WN_DEBUG
    case 8 * 10000 + 160: return launch_latency_shape<8, 160, 4, OutT>(a, c.threads, full, smem, cs);
#endif
#ifndef WN_DEBUG
    case 8 * 10000 + 544: return launch_latency_shape<8, 544, 1, OutT>(a, c.threads, full, smem, cs);
#endif
#ifndef WN_DEBUG
    case 16 * 10000 + 288: return launch_latency_shape<16, 288, 1, OutT>(a, c.threads, full, smem, cs);
#endif
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_latency_f32(const GenArgs &a, const LaunchCfg &c, bool full, size_t smem, cudaStream_t cs);
cudaError_t launch_latency_bf16(const GenArgs &a, const LaunchCfg &c, bool full, size_t smem, cudaStream_t cs);
cudaError_t launch_latency_f16(const GenArgs &a, const LaunchCfg &c, bool full, size_t smem, cudaStream_t cs);

cudaError_t launch_generate_f32(const GenArgs &a, const LaunchCfg &c, bool full, bool var, size_t smem,
                               cudaStream_t cs);
cudaError_t launch_generate_bf16(const GenArgs &a, const LaunchCfg &c, bool full, bool var, size_t smem,
                               cudaStream_t cs);
cudaError_t launch_generate_f16(const GenArgs &a, const LaunchCfg &c, bool full, bool var, size_t smem,
                               cudaStream_t cs);

}  // namespace wn
