// wn_chain.cuh -- the chain mode of the plain method (Brent, arXiv:1005.2314,
// Section 5: chi-squared approximation (c), reserved value from the previous
// block, the 4x4 update) for streams whose serial chain of blocks sets the
// time: lone streams, and the longest requests of a batch.
//
// A stream's blocks form one dependency chain through its pool (Section 5.1),
// but the chain itself is only the passes: a block's scale comes from the
// block before it (Section 5.5), and its values leave the pool untouched.  So
// a CTA runs the passes on G compute warps, and helper warps do the rest
// beside them:
//  * the draw warp draws each pass's permutation and signs (Sections 5.2,
//    5.4, 5.8) from the stream's generator into a ring of pass words, blocks
//    ahead; a compute warp loads the next pass's words during the pass;
//  * a pass reads one shared pool buffer and writes another, so one barrier
//    among the compute warps ends it: the passes of a block alternate
//    between two work buffers, and the final pass writes emission buffer
//    b mod KS (KS = 4, or 2 for pools of 8192), which the next block's first
//    pass reads;
//  * the scale warp (warp G) adds the block's per-lane sums of squares and
//    forms the next block's scale;
//  * NS store warps (warps G+1 .. G+NS, store warp s taking the blocks
//    b = s mod NS) read a block's values from its emission buffer, scale
//    them into a staging buffer laid out like the output (16-byte chunks of
//    the output at 16-byte boundaries), and write the whole chunks with one
//    bulk copy of the tensor-memory-access unit (cp.async.bulk), the partial
//    chunk at each end (shared with the neighbouring block) with plain
//    stores.  Bulk copies belong to the asynchronous proxy, which no barrier
//    waits on.
// Hand-overs: at PART(b) the compute warps arrive with block b's sums of
// squares and reserved value (its emission buffer written), the scale warp,
// block b's store warp and the draw warp wait; at SCALE(b) those three arrive
// (block b's sums read; its emission buffer read; block b + KS + 1's pass
// words written), and the compute warps wait at the end of block b + KS - 1,
// before they next overwrite those buffers -- so a store warp has KS - 1
// blocks for its staging and NS blocks for all of its work; at SC(b) the
// scale warp hands block b+1's scale to block b+1's store warp.  Only the
// store warps wait for a scale.
// Pools above 8192 values leave no room for the emission and staging
// buffers; there the passes alternate between two buffers, the compute warps
// store each block's values themselves early in the next block's first pass
// (realigned by warp shuffles), KS = 2, and the store warps only keep the
// barrier counts.
// Barrier identifiers cycle with the block index (PART, SCALE: b mod
// max(NS, KS); SC: the rest of the 16), so that no barrier ever has two
// phases open; the scales are kept in 2 NS slots (b mod 2 NS) for the same
// reason.  No wait spins: every barrier is a hardware named barrier whose
// arrivals are fixed by the block count all warps share.
#pragma once

#include "wn_group.cuh"

namespace wn {

// Named barriers of the chain mode (0 is __syncthreads): the pass barrier
// among the compute warps, then PART, SCALE and SC (with MP = max(NS, KS):
// PART(b) has identifier 2 + b mod MP, SCALE(b) 2 + MP + b mod MP, SC(b)
// 2 + 2 MP + b mod (14 - 2 MP) -- every one of the 16).
constexpr uint32_t kChPass = 1;
// Store warps: four beside four compute warps (pools of 1024, whose blocks are
// short), two beside eight (the registers allow no more warps).
__host__ __device__ constexpr uint32_t chain_store_warps(uint32_t G) { return G <= 4u ? 4u : 2u; }
// Threads: the compute warps, the scale warp, the store warps, the draw warp.
__host__ __device__ constexpr uint32_t chain_threads(uint32_t G) { return 32u * (G + 2u + chain_store_warps(G)); }

// Small area at the window base: per-lane sums of squares [4][32 G] (by the
// block's index modulo the emission buffers), then the reserved values [4],
// the scales [8], the scale warp's final sum of squares / reserved value, and
// the persistent kernel's claimed item.
__host__ __device__ constexpr uint32_t chain_small(uint32_t G) { return 512u * G + 128u; }
// Window address of the first pool buffer (the others follow): a multiple of
// the buffer size 4N, so that a gather address is one LOP3 of its pool offset.
__host__ __device__ inline uint32_t chain_window(uint32_t base, uint32_t N, uint32_t G)
{
    const uint32_t sz = 4u * N;
    return (base + chain_small(G) + sz - 1u) / sz * sz;
}
// Pools up to 8192 values have two work buffers, the emission buffers and a
// staging buffer per store warp: a block's N - 1 values behind up to 7
// positions of its first 16-byte chunk, at 4 bytes at most.
__host__ __device__ constexpr bool chain_stages(uint32_t N) { return N <= 8192u; }
__host__ __device__ constexpr uint32_t chain_stage_bytes(uint32_t N) { return ((N + 8u) * 4u + 15u) / 16u * 16u; }
// Emission buffers: four up to pools of 4096 (a store warp may finish
// reading a block's values while the compute warps run the next three), two
// for 8192 (shared memory).
__host__ __device__ constexpr uint32_t chain_emit_bufs(uint32_t N) { return N <= 4096u ? 4u : 2u; }
// Blocks from PART(b) to the compute warps' wait at SCALE(b): the emission
// buffers with staging, else 2.  The draw warp keeps this many blocks' pass
// words plus two in its ring.
__host__ __device__ constexpr uint32_t chain_lag(uint32_t N) { return chain_stages(N) ? chain_emit_bufs(N) : 2u; }
__host__ __device__ constexpr uint32_t chain_ring(uint32_t N) { return chain_lag(N) + 2u; }
// Shared memory of a chain-mode CTA for pool N, G compute warps and up to
// r_max passes per block: the pool, emission and staging buffers, then the
// ring of pass words (16 bytes per pass).
__host__ __device__ inline size_t chain_smem_bytes(uint32_t base, uint32_t N, uint32_t G, uint32_t r_max)
{
    return (size_t)chain_window(base, N, G) +
           (chain_stages(N) ? 4u * (size_t)N * (2u + chain_emit_bufs(N)) +
                                  chain_store_warps(G) * (size_t)chain_stage_bytes(N)
                            : 8u * (size_t)N) +
           16u * (size_t)chain_ring(N) * r_max - base;
}

__device__ __forceinline__ void sts4u(uint32_t a, uint4 v)
{
    if (!dbg_shared_ok(a, 16)) return;
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w));
}

// One pass's words: alpha, gamma and the sign word (low, high) from the
// pass's two draws (Sections 5.2, 5.4, 5.8).
__device__ __forceinline__ uint4 pass_words(uint64_t &gx, uint64_t &gw, uint32_t N)
{
    const uint64_t wa = draw(gx, gw);
    const uint64_t ws = draw(gx, gw);
    return make_uint4(((uint32_t)(wa >> 32) & (N - 1)) | 1u, (uint32_t)wa & (N - 1), (uint32_t)ws,
                      (uint32_t)(ws >> 32));
}

// A thread's pass quantities from the pass words (as group_pass derives them
// from the draws).
__device__ __forceinline__ GroupPass pass_from_words(uint4 t, uint32_t N, uint32_t q0, uint32_t lane)
{
    GroupPass p;
    p.B0 = 4u * (t.x * q0 + t.y);
    p.d1 = (t.x & 3u) * N;
    p.dq = 128u * t.x;
    const uint32_t word = (lane & 8u) ? t.w : t.z;
    const uint32_t nib = (word >> (4u * (lane & 7u))) & 15u;
    p.m01 = make_float2(neg_sign_one(nib & 1u), neg_sign_one((nib >> 1) & 1u));
    p.m23 = make_float2(neg_sign_one((nib >> 2) & 1u), neg_sign_one(nib >> 3));
    p.h01 = fmul2(p.m01, make_float2(-0.5f, -0.5f));
    p.h23 = fmul2(p.m23, make_float2(-0.5f, -0.5f));
    return p;
}

__device__ __forceinline__ void bar_arrive_n(uint32_t id, uint32_t n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// The block's values y (unscaled) times sc to ob, whole block with the
// output's alignment a, or the first n values (n > 0: a partial last block).
template <int QT, typename OutT>
__device__ __forceinline__ void chain_emit(OutT *__restrict__ ob, const float2 (&y)[QT][2], float sc, uint32_t q0,
                                           uint32_t lane, uint32_t nq, uint32_t a, uint32_t n, const DbgRange &rg)
{
    if (n) {
        group_emit<QT, 0, true, OutT>(ob, y, sc, q0, lane, nq, n, rg);
        return;
    }
    switch (a) {
    case 0: group_emit<QT, 0, false, OutT>(ob, y, sc, q0, lane, nq, 0, rg); break;
    case 1: group_emit<QT, 1, false, OutT>(ob, y, sc, q0, lane, nq, 0, rg); break;
    case 2: group_emit<QT, 2, false, OutT>(ob, y, sc, q0, lane, nq, 0, rg); break;
    default: group_emit<QT, 3, false, OutT>(ob, y, sc, q0, lane, nq, 0, rg); break;
    }
}


// --- staging and bulk copies ------------------------------------------------
// Bulk copy of `bytes` (a multiple of 16) from shared window address s to
// global address g (both 16-byte aligned), in the calling thread's current
// bulk group; commit closes the group; the waits return once at most n of the
// thread's groups are still reading shared memory (read) or still writing.
__device__ __forceinline__ void bulk_store(void *g, uint32_t s, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(g), "r"(s), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int n> __device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(n) : "memory");
}
template <int n> __device__ __forceinline__ void bulk_wait()
{
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(n) : "memory");
}
// Orders this thread's shared-memory writes before later bulk copies (the
// asynchronous proxy) that read them.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One output value, or four consecutive ones at a 4-value boundary, into the
// staging buffer at window address a, converted to the output type.
template <typename OutT> __device__ __forceinline__ void stage1(uint32_t a, float v);
template <> __device__ __forceinline__ void stage1<float>(uint32_t a, float v)
{
    if (!dbg_shared_ok(a, 4)) return;
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v));
}
template <typename T16> __device__ __forceinline__ void stage1_16(uint32_t a, T16 h)
{
    if (!dbg_shared_ok(a, 2)) return;
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"(*reinterpret_cast<unsigned short *>(&h)));
}
template <> __device__ __forceinline__ void stage1<__nv_bfloat16>(uint32_t a, float v)
{
    stage1_16(a, __float2bfloat16_rn(v));
}
template <> __device__ __forceinline__ void stage1<__half>(uint32_t a, float v) { stage1_16(a, __float2half_rn(v)); }

template <typename OutT> __device__ __forceinline__ void stage4(uint32_t a, float x, float y, float z, float w);
template <> __device__ __forceinline__ void stage4<float>(uint32_t a, float x, float y, float z, float w)
{
    if (!dbg_shared_ok(a, 16)) return;
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x), "f"(y), "f"(z), "f"(w));
}
template <typename T2> __device__ __forceinline__ void stage4_16(uint32_t a, T2 lo, T2 hi)
{
    if (!dbg_shared_ok(a, 8)) return;
    asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a), "r"(*reinterpret_cast<uint32_t *>(&lo)),
                 "r"(*reinterpret_cast<uint32_t *>(&hi)));
}
template <> __device__ __forceinline__ void stage4<__nv_bfloat16>(uint32_t a, float x, float y, float z, float w)
{
    stage4_16(a, __floats2bfloat162_rn(x, y), __floats2bfloat162_rn(z, w));
}
template <> __device__ __forceinline__ void stage4<__half>(uint32_t a, float x, float y, float z, float w)
{
    stage4_16(a, __floats2half2_rn(x, y), __floats2half2_rn(z, w));
}

// A staged value (its output-type bits) read back, and stored to global memory as such.
template <typename OutT> __device__ __forceinline__ uint32_t stage_ld(uint32_t a)
{
    uint32_t v;
    if (sizeof(OutT) == 4) {
        if (!dbg_shared_ok(a, 4)) return 0u;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    } else {
        if (!dbg_shared_ok(a, 2)) return 0u;
        unsigned short h;
        asm volatile("ld.shared.u16 %0, [%1];" : "=h"(h) : "r"(a));
        v = h;
    }
    return v;
}
template <typename OutT> __device__ __forceinline__ void global_st(const DbgRange &rg, OutT *p, uint32_t v)
{
    if (!dbg_global_ok(rg, p, sizeof(OutT))) return;
    if (sizeof(OutT) == 4) *reinterpret_cast<uint32_t *>(p) = v;
    else *reinterpret_cast<unsigned short *>(p) = (unsigned short)v;
}

// Block values from a staging buffer (window address stg, holding output
// positions c .. e + n - 1 from position e on: c = e rounded down to a 16-byte
// chunk, e the block's first position) to global memory (gbase: the
// 16-byte-aligned output base), by the 32 lanes of one warp: the whole
// 16-byte chunks with one bulk copy (lane 0's bulk group), the partial chunks
// at either end (which the neighbouring blocks share) with plain stores.
template <typename OutT>
__device__ __forceinline__ void chain_flush(OutT *__restrict__ gbase, uint32_t stg, uint64_t e, uint32_t n,
                                            uint32_t lane, const DbgRange &rg)
{
    constexpr uint32_t ES = sizeof(OutT), E = 16u / ES;
    const uint64_t c = e / E * E, hi = e + n;
    const uint64_t h = (e + E - 1u) / E * E < hi ? (e + E - 1u) / E * E : hi;  // end of the head
    const uint64_t B = hi / E * E > h ? hi / E * E : h;                         // start of the tail
    if (lane < h - e) global_st<OutT>(rg, gbase + e + lane, stage_ld<OutT>(stg + ES * (uint32_t)(e - c + lane)));
    if (lane < hi - B) global_st<OutT>(rg, gbase + B + lane, stage_ld<OutT>(stg + ES * (uint32_t)(B - c + lane)));
    if (B > h && lane == 0) {
        bool ok = true;
#ifdef WN_DEBUG
        ok = dbg_global_ok(rg, gbase + h, 16) && dbg_global_ok(rg, gbase + B - E, 16) &&
             dbg_shared_ok(stg + ES * (uint32_t)(h - c), 16) && dbg_shared_ok(stg + ES * (uint32_t)(B - c) - 16u, 16);
#endif
        if (ok) bulk_store(gbase + h, stg + ES * (uint32_t)(h - c), ES * (uint32_t)(B - h));
        bulk_commit();
    }
}

// The store warp's staging of one block: values i < n of the emission buffer
// at window address eb (unscaled FP32, value i at eb + 4 i) times sc, as the
// output type, at positions r + i of the staging buffer st.  Lane l writes
// the 4-position groups l, l + 32, ...: groups wholly inside [r, r + n) with
// one vector store of four values read singly (one code path whatever the
// alignment, so that the loop's instructions stay cached), the positions at
// either end value by value.
template <typename OutT>
__device__ __forceinline__ void chain_stage_block(uint32_t st, uint32_t eb, uint32_t r, uint32_t n, float sc,
                                                  uint32_t lane)
{
    constexpr uint32_t ES = sizeof(OutT);
    constexpr int U = 4;
    const uint32_t end = r + n, gA = (r + 3u) / 4u, gB = end / 4u;  // interior groups [gA, gB)
    const float2 sc2 = make_float2(sc, sc);
    const uint32_t e0 = eb - 4u * r;  // value i at e0 + 4 (r + i): position p's value at e0 + 4 p
    for (uint32_t g = gA + lane; g < gB; g += 32u * U) {
        float v[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t a = e0 + 16u * (g + 32u * u);
            if (g + 32u * u < gB) {
#pragma unroll
                for (int k = 0; k < 4; ++k) v[u][k] = lds(a + 4u * k);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (g + 32u * u < gB) {
                const float2 lo = fmul2(make_float2(v[u][0], v[u][1]), sc2);
                const float2 hi = fmul2(make_float2(v[u][2], v[u][3]), sc2);
                stage4<OutT>(st + ES * 4u * (g + 32u * u), lo.x, lo.y, hi.x, hi.y);
            }
        }
    }
    // the ends: positions [r, 4 gA) and [4 gB, end), fewer than four each
    // (with no whole group, all of [r, end): fewer than seven)
    uint32_t pos = r + lane;
    bool mine = lane < 8u && pos < end;
    if (gB > gA) {
        pos = lane < 4u ? r + lane : 4u * gB + (lane - 4u);
        mine = lane < 4u ? pos < 4u * gA : lane < 8u && pos < end;
    }
    if (mine) stage1<OutT>(st + ES * pos, sc * lds(e0 + 4u * pos));
}

// One stream's share of a call in the chain mode.  The CTA is G compute warps,
// the scale warp and NS store warps; compute warp w, lane l owns quadruples
// q0 + 32 j (j < QT), q0 = 32 QT w + l, and 128 QT G = N.  out: the stream's
// output, out_off elements past a 16-byte boundary.
template <int G, int QT, typename OutT>
__device__ __forceinline__ void run_stream_chain(StreamHdr *__restrict__ h, float *__restrict__ pool_g,
                                                 OutT *__restrict__ out, uint64_t out_off, uint64_t count,
                                                 uint32_t r_max)
{
    constexpr uint32_t N = 128u * QT * G, nq = N / 4, NS = chain_store_warps(G), NT = chain_threads(G);
    constexpr bool STAGE = chain_stages(N);
    // KS: blocks from PART(b) to the compute warps' wait at SCALE(b) (the
    // emission buffers with staging, else 2); MP: identifiers of PART and of
    // SCALE; MSC: of SC
    constexpr uint32_t KS = chain_lag(N), MP = NS > KS ? NS : KS, MSC = 14u - 2u * MP, RK = chain_ring(N);
    constexpr uint32_t kPart = 2u, kScale = 2u + MP, kSc = 2u + 2u * MP;
    constexpr uint32_t NH = 32u * (G + 3), ES = sizeof(OutT);  // NH: PART and SCALE (all but NS - 1 store warps)
    static_assert(MSC >= NS + 1u, "SC needs NS + 1 identifiers");
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t base = smem_base();
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    // pool buffers: work W[0], W[1], then (with STAGE) emission E[0 .. KS-1],
    // the staging buffers T[0 .. NS-1]; then the ring of pass words,
    // [RK][r_max] (block b's in slot b mod RK)
    const uint32_t W = chain_window(base, N, G), SB = chain_stage_bytes(N);
    const uint32_t E0 = W + 8u * N, T0 = E0 + 4u * N * KS, TB = STAGE ? T0 + NS * SB : W + 8u * N;
    const uint32_t R = h->R;
    if (dyn < chain_smem_bytes(base, N, G, r_max) || h->N != N || R > r_max) {  // not this kernel's layout
        if (tid == 0) h->flags |= 1u;
        return;
    }
    float *parts = reinterpret_cast<float *>(wn_smem);  // [KS][32 G] per-lane sums of squares, by b mod KS
    float *rvs = parts + 4u * 32u * G;                  // [KS] reserved values (unscaled)
    float *scs = rvs + 4;                               // [2 NS] block scales, by b mod 2 NS
    float *fin = scs + 8;                               // the last block's sum of squares and scaled reserved value
    const DbgRange rg = dbg_range(out, out + count);    // this stream's output (the debug build checks stores)
    const uint32_t P0 = STAGE ? E0 + 4u * N * (KS - 1u) : W;  // the stored pool, as if block -1's output
    {
        const float4 *pg4 = reinterpret_cast<const float4 *>(pool_g);
        for (uint32_t i = tid; i < nq; i += NT) {
            const float4 v = pg4[i];
            sts4(P0 + 16u * i, make_float2(v.x, v.y), make_float2(v.z, v.w));
        }
    }
    const uint32_t k0 = h->k;
    const float sc_prev = h->scale;
    const uint64_t left = (uint64_t)(N - 1 - k0);
    const uint64_t n0 = left < count ? left : count;
    const uint64_t nb = (count - n0 + (N - 2)) / (N - 1);
    const uint64_t tail = (count - n0) % (N - 1);  // values of a partial last block (0: whole)
    const uint64_t g0 = out_off + n0;              // output position of block 0's first value
    // block 0's scale: the stored sum of squares and reserved value
    if (tid == 0) scs[0] = nb > 0 ? group_scale(h->sumsq, (float)h->r, (float)h->A, (float)h->B, N) : sc_prev;
    const uint32_t dw = G + 1u + NS;  // the draw warp
    uint64_t gx = h->x, gw = h->w;    // its generator
    if (warp == dw)                   // the first blocks' pass words
        for (uint64_t b = 0; b < nb && b <= KS; ++b)
            for (uint32_t p = 0; p < R; ++p) {
                const uint4 t = pass_words(gx, gw, N);
                if (lane == (p & 31u)) sts4u(TB + 16u * ((uint32_t)b * r_max + p), t);
            }
    __syncthreads();
    for (uint64_t i = tid; i < n0; i += NT) store1(rg, out + i, sc_prev * lds(P0 + 4u * (uint32_t)(k0 + i)));
    __syncthreads();  // the stored pool is read: it may be overwritten

    if (warp < G) {
        const uint32_t q0 = warp * 32u * QT + lane;
        const uint32_t m4 = 4u * N - 1u, half = 2u * N;
        uint64_t e = g0;  // without STAGE: output position of the block whose values y hold
        float2 y[QT][2];
#pragma unroll
        for (int j = 0; j < QT; ++j) y[j][0] = y[j][1] = make_float2(0.f, 0.f);
        uint32_t cur = P0;            // the buffer holding the pool
        uint32_t kb = 0, kp = 0, kt = 0;  // b mod KS, b mod MP, b mod RK
        GroupPass gp = pass_from_words(lds4u(TB), N, q0, lane);
        for (uint64_t b = 0; b < nb; ++b) {
            const uint32_t kt1 = kt + 1u == RK ? 0u : kt + 1u;
            for (uint32_t p = 0; p < R; ++p) {
                uint32_t wr;
                if (STAGE) wr = p + 1 == R ? E0 + 4u * N * kb : W + 4u * N * (p & 1u);
                else wr = cur == W ? W + 4u * N : W;
                float av[QT][4];
#pragma unroll
                for (int j = 0; j < QT; ++j) {
                    const uint32_t Bj = gp.B0 + (uint32_t)j * gp.dq;
                    const uint32_t o0 = (Bj & m4) | cur, o1 = ((Bj + gp.d1) & m4) | cur;
                    av[j][0] = lds(o0);
                    av[j][2] = lds(o0 ^ half);
                    av[j][1] = lds(o1);
                    av[j][3] = lds(o1 ^ half);
                }
                if (!STAGE && p == 0 && b > 0) {  // the previous block's values, behind this pass's gathers
                    chain_emit<QT, OutT>(out + (e - out_off), y, scs[(uint32_t)((b - 1) % (2u * NS))], q0, lane, nq,
                                         (uint32_t)(e & 3u), 0, rg);
                    e += N - 1;
                }
                // the next pass's words: of pass p+1, or of the next block's first
                const uint32_t tn = p + 1 < R ? TB + 16u * (kt * r_max + p + 1u) : TB + 16u * kt1 * r_max;
                const GroupPass gn = pass_from_words(lds4u(tn), N, q0, lane);
#pragma unroll
                for (int j = 0; j < QT; ++j) {
                    const float2 a01 = make_float2(av[j][0], av[j][1]), a23 = make_float2(av[j][2], av[j][3]);
                    const float2 s2 = fadd2(a01, a23);
                    const float sum = s2.x + s2.y;
                    const float2 SS = make_float2(sum, sum);
                    y[j][0] = ffma2(gp.m01, a01, fmul2(gp.h01, SS));
                    y[j][1] = ffma2(gp.m23, a23, fmul2(gp.h23, SS));
                    sts4(wr + 16u * (q0 + 32u * j), y[j][0], y[j][1]);
                }
                if (p + 1 == R) {
                    // the block's per-lane sums of squares and reserved slot (and
                    // its emission buffer) to the helpers; the block ends once
                    // they are done with block b - KS + 1, whose buffers block
                    // b+1 overwrites
                    float2 part = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < QT; ++j) part = ffma2(y[j][0], y[j][0], ffma2(y[j][1], y[j][1], part));
                    parts[kb * 32u * G + tid] = part.x + part.y;
                    if (warp == G - 1 && lane == 31) rvs[kb] = y[QT - 1][1].y;
                    bar_arrive_n(kPart + kp, NH);
                    if (b + 1 >= KS) bar_wait(kScale + (uint32_t)((b + 1 - KS) % MP), NH);
                    else bar_wait(kChPass, 32u * G);
                    kb = kb + 1 == KS ? 0u : kb + 1;
                    kp = kp + 1 == MP ? 0u : kp + 1;
                    kt = kt1;
                } else {
                    bar_wait(kChPass, 32u * G);  // the pass's stores precede the next pass's gathers
                }
                cur = wr;
                gp = gn;
            }
        }
        if (!STAGE && nb > 0)  // the last block
            chain_emit<QT, OutT>(out + (e - out_off), y, scs[(uint32_t)((nb - 1) % (2u * NS))], q0, lane, nq,
                                 (uint32_t)(e & 3u), (uint32_t)tail, rg);
    } else if (warp == G) {
        // the scale warp: block b's sum of squares (FP32: per lane, pairwise
        // over the warps, then across lanes) and, with the block's reserved
        // value, block b+1's scale (Section 5.5, approximation (c); the FP32
        // route of group_scale_f32, exact for an FP32 sum)
        const float A = (float)h->A, B = (float)h->B;
        float sc = scs[0];
        uint32_t kb = 0;  // b mod KS
        for (uint64_t b = 0; b < nb; ++b) {
            bar_wait(kPart + (uint32_t)(b % MP), NH);
            const float *pp = parts + kb * 32u * G;
            float t[G];
#pragma unroll
            for (int w = 0; w < G; ++w) t[w] = pp[32u * w + lane];
            const float rv = rvs[kb];
            kb = kb + 1 == KS ? 0u : kb + 1;
            // with staging only the store warps wait for a scale: the compute
            // warps need only the sums read
            if (STAGE && b + KS <= nb) bar_arrive_n(kScale + (uint32_t)(b % MP), NH);
#pragma unroll
            for (int st = 1; st < G; st <<= 1)
#pragma unroll
                for (int w = 0; w + st < G; w += 2 * st) t[w] += t[w + st];
            float s = t[0];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            const float r = sc * rv;  // block b's reserved value, scaled (fastnorm2)
            if (b + 1 < nb) {
                sc = group_scale_f32(s, r, A, B, N);
                if (lane == 0) scs[(uint32_t)((b + 1) % (2u * NS))] = sc;
                __syncwarp();
                if (STAGE) bar_arrive_n(kSc + (uint32_t)(b % MSC), 64u);
                else bar_arrive_n(kScale + (uint32_t)(b % MP), NH);
            } else if (lane == 0) {
                fin[0] = s;
                fin[1] = r;
            }
        }
    } else if (warp == dw) {
        // the draw warp: once block b is done, block b + KS + 1's pass words
        // (the compute warps read them after SCALE(b))
        for (uint64_t b = 0; b < nb; ++b) {
            bar_wait(kPart + (uint32_t)(b % MP), NH);
            if (b + KS + 1 < nb) {
                const uint32_t slot = (uint32_t)((b + KS + 1) % RK);
                for (uint32_t p = 0; p < R; ++p) {
                    const uint4 t = pass_words(gx, gw, N);
                    if (lane == (p & 31u)) sts4u(TB + 16u * (slot * r_max + p), t);
                }
            }
            if (b + KS <= nb) bar_arrive_n(kScale + (uint32_t)(b % MP), NH);
        }
        if (nb > 0 && lane == 0) {  // the generator after the call's last pass
            h->x = gx;
            h->w = gw;
        }
    } else {
        // store warp s (warp G+1+s): the blocks b = s mod NS -- block b's
        // values from its emission buffer, scaled (block b's scale: from the
        // scale warp at SC(b-1)), staged in T[s], written out
        const uint32_t sp = warp - (G + 1u);
        OutT *gbase = out - out_off;       // 16-byte aligned
        constexpr uint32_t EL = 16u / ES;  // values per 16-byte chunk
        for (uint64_t b = sp; b < nb; b += NS) {
            bar_wait(kPart + (uint32_t)(b % MP), NH);
            if (!STAGE) {
                if (b + 1 < nb) bar_arrive_n(kScale + (uint32_t)(b % MP), NH);
                continue;
            }
            if (b > 0) bar_wait(kSc + (uint32_t)((b - 1) % MSC), 64u);
            const float sc = scs[(uint32_t)(b % (2u * NS))];
            const uint64_t e = g0 + b * (N - 1);
            const uint32_t n = b + 1 == nb && tail ? (uint32_t)tail : N - 1;
            const uint32_t st = T0 + sp * SB;
            if (lane == 0) bulk_wait_read<0>();  // this warp's previous copy has read T[s]
            __syncwarp();
            chain_stage_block<OutT>(st, E0 + 4u * N * (uint32_t)(b % KS), (uint32_t)(e % EL), n, sc, lane);
            fence_proxy_async();  // the staged values are read by the bulk copy
            __syncwarp();
            if (b + KS <= nb) bar_arrive_n(kScale + (uint32_t)(b % MP), NH);  // block b's emission buffer is read
            chain_flush<OutT>(gbase, st, e, n, lane, rg);
        }
        if (STAGE && lane == 0) bulk_wait<0>();  // every bulk copy complete (and its buffer read)
    }
    __syncthreads();

    {
        const uint32_t fb = STAGE ? (nb > 0 ? E0 + 4u * N * (uint32_t)((nb - 1) % KS) : P0)
                                  : (((nb * R) & 1u) ? W + 4u * N : W);  // the buffer the last pass wrote
        float4 *pw4 = reinterpret_cast<float4 *>(pool_g);
        for (uint32_t i = tid; i < nq; i += NT) pw4[i] = lds4(fb + 16u * i);
    }
    if (tid == 0) {
        if (nb > 0) {
            h->sumsq = (double)fin[0];
            h->r = (double)fin[1];
            h->scale = scs[(uint32_t)((nb - 1) % (2u * NS))];
            h->k = tail == 0 ? N - 1 : (uint32_t)tail;
            h->blocks += nb;
        } else {
            h->k = k0 + (uint32_t)n0;
        }
    }
}

// Chain-mode generate kernel: one CTA of G compute warps and the scale, store
// and draw warps per stream.  One CTA per SM is what a lone stream needs; the register
// bound follows from the thread count alone.
template <int G, int QT, typename OutT>
__global__ void __launch_bounds__(chain_threads(G), 1) chain_kernel(GenArgs a)
{
    StreamHdr *h = a.hdr + blockIdx.x;
    const uint64_t off = (uint64_t)blockIdx.x * a.out_stride;
    run_stream_chain<G, QT, OutT>(h, a.pools + h->pool_off, reinterpret_cast<OutT *>(a.out) + off, off, a.count,
                                  a.r_max);
}

// Persistent chain-mode kernel (a batch's longest requests): each CTA claims
// the next stream from an atomic counter (longest first) and returns its
// request; no CTA waits on another.  The claimed index passes through the
// small area's last word.
template <int G, int QT, typename OutT>
__global__ void __launch_bounds__(chain_threads(G), 1) persist_chain_kernel(GenArgs a, BatchArgs bq)
{
    uint32_t *slot = reinterpret_cast<uint32_t *>(wn_smem + chain_small(G) - 4u);
    for (;;) {
        __syncthreads();  // the previous stream is done with shared memory
        if (threadIdx.x == 0) *slot = atomicAdd(bq.queue, 1u);
        __syncthreads();
        const uint32_t it = *slot;
        if (it >= bq.n_items) return;
        const uint32_t si = bq.order[it];
        StreamHdr *h = a.hdr + si;
        const uint64_t off = bq.offsets[si];
        run_stream_chain<G, QT, OutT>(h, a.pools + h->pool_off, reinterpret_cast<OutT *>(a.out) + off, off,
                                      bq.counts[si], a.r_max);
    }
}

// Compiled chain-mode shapes {pool N, compute warps G, quadruples per lane}.
// (At most eight compute warps: with the helpers no SM sub-partition holds
// more than three warps, and the registers allow 64 values per lane.)
#ifndef WN_DEBUG
constexpr int kChainShapes[][3] = {{1024, 4, 2}, {1024, 8, 1}, {2048, 8, 2},
                                   {4096, 8, 4},  {8192, 8, 8}, {16384, 8, 16}};
#else
constexpr int kChainShapes[][3] = {{1024, 4, 2}};  // the debug build compiles one
#endif

template <int G, int QT, typename OutT>
cudaError_t launch_chain_shape(const GenArgs &a, size_t smem, cudaStream_t cs)
{
    auto kern = chain_kernel<G, QT, OutT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.n_streams, chain_threads(G), smem, cs>>>(a);
    return cudaGetLastError();
}

template <int G, int QT, typename OutT>
cudaError_t launch_persist_chain_shape(const GenArgs &a, const BatchArgs &bq, size_t smem, int sms, cudaStream_t cs)
{
    auto kern = persist_chain_kernel<G, QT, OutT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // every persistent kernel of a batch prefers the whole shared-memory
    // carveout: an SM's split of L1 and shared memory serves all the CTAs it
    // holds, and one preference lets any batch kernel join an SM the others use
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, chain_threads(G), smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const uint32_t grid = std::min<uint32_t>(bq.n_items, (uint32_t)(per_sm * sms));
    if (grid == 0) return cudaSuccess;
    kern<<<grid, chain_threads(G), smem, cs>>>(a, bq);
    return cudaGetLastError();
}

// Launches for one output type: pool N with G compute warps (smem: at least
// chain_smem_bytes of the launch's window base; more pads CTAs per SM).
template <typename OutT>
cudaError_t launch_chain_t(const GenArgs &a, uint32_t N, uint32_t G, size_t smem, cudaStream_t cs)
{
    switch (N * 64u + G) {
    case 1024 * 64 + 4: return launch_chain_shape<4, 2, OutT>(a, smem, cs);
#ifndef WN_DEBUG
    case 1024 * 64 + 8: return launch_chain_shape<8, 1, OutT>(a, smem, cs);
    case 2048 * 64 + 8: return launch_chain_shape<8, 2, OutT>(a, smem, cs);
    case 4096 * 64 + 8: return launch_chain_shape<8, 4, OutT>(a, smem, cs);
    case 8192 * 64 + 8: return launch_chain_shape<8, 8, OutT>(a, smem, cs);
    case 16384 * 64 + 8: return launch_chain_shape<8, 16, OutT>(a, smem, cs);
#endif
    default: return cudaErrorInvalidValue;
    }
}

template <typename OutT>
cudaError_t launch_persist_chain_t(const GenArgs &a, const BatchArgs &bq, uint32_t N, uint32_t G, size_t smem, int sms,
                                   cudaStream_t cs)
{
    switch (N * 64u + G) {
    case 1024 * 64 + 4: return launch_persist_chain_shape<4, 2, OutT>(a, bq, smem, sms, cs);
#ifndef WN_DEBUG
    case 1024 * 64 + 8: return launch_persist_chain_shape<8, 1, OutT>(a, bq, smem, sms, cs);
    case 2048 * 64 + 8: return launch_persist_chain_shape<8, 2, OutT>(a, bq, smem, sms, cs);
    case 4096 * 64 + 8: return launch_persist_chain_shape<8, 4, OutT>(a, bq, smem, sms, cs);
    case 8192 * 64 + 8: return launch_persist_chain_shape<8, 8, OutT>(a, bq, smem, sms, cs);
    case 16384 * 64 + 8: return launch_persist_chain_shape<8, 16, OutT>(a, bq, smem, sms, cs);
#endif
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_chain_f32(const GenArgs &a, uint32_t N, uint32_t G, size_t smem, cudaStream_t cs);
cudaError_t launch_chain_bf16(const GenArgs &a, uint32_t N, uint32_t G, size_t smem, cudaStream_t cs);
cudaError_t launch_chain_f16(const GenArgs &a, uint32_t N, uint32_t G, size_t smem, cudaStream_t cs);
cudaError_t launch_persist_chain_f32(const GenArgs &a, const BatchArgs &bq, uint32_t N, uint32_t G, size_t smem,
                                     int sms, cudaStream_t cs);
cudaError_t launch_persist_chain_bf16(const GenArgs &a, const BatchArgs &bq, uint32_t N, uint32_t G, size_t smem,
                                      int sms, cudaStream_t cs);
cudaError_t launch_persist_chain_f16(const GenArgs &a, const BatchArgs &bq, uint32_t N, uint32_t G, size_t smem,
                                     int sms, cudaStream_t cs);

}  // namespace wn
