// wn_emit.cuh -- the latency mode of the plain method (Brent, arXiv:1005.2314,
// Section 5) for launches of few streams: a stream is a serial chain of
// blocks, so a lone stream waits on every step of every block.
//
// Three roles share a CTA and hand work along through mbarriers:
//  * warp 0 draws and tabulates each block's passes (Sections 5.4, 5.8),
//    into one of two table slots;
//  * warps 2.. (the compute warps) run the block's R passes (Sections
//    5.1-5.3); the final pass writes the block's pool into one of two
//    emission buffers E[b mod 2] instead of storing the block's values;
//  * warp 1 (the emitter) reads E[b mod 2] while the compute warps already
//    run block b+1: it writes the block's N-1 values scaled by the block's
//    scale, sums the pool's squares and forms the next block's scale from
//    that sum and the block's reserved value (Section 5.5, approximation
//    (c), the value held back by the previous block).
// So a block's critical path is its passes alone; emission, the sum of
// squares and the scale overlap the next block.  Work buffers W[0], W[1]
// carry the passes between the emission buffers: pass p reads E[(b-1) mod 2]
// (p = 0) or W[(p-1) mod 2] and writes W[p mod 2], the final pass E[b mod 2].
//
// Every wait on an mbarrier is bounded in time: after kWaitNs without the
// awaited phase (which a correct launch never sees) the waiting warp sets the
// CTA's abort word, every role leaves its loop at its next wait, the stream
// is flagged (StreamHdr::flags bit 1) and its state is left as it was.
#pragma once

#include "wn_group.cuh"

namespace wn {

constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s

// mbarrier primitives on shared-window addresses.
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint32_t a)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(a)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(a), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Named barrier `id` over n threads that also returns, to every one of them,
// whether any of them passed a true predicate.
__device__ __forceinline__ bool bar_red_or(uint32_t id, uint32_t n, bool pred)
{
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r)
                 : "r"((uint32_t)pred), "r"(id), "r"(n)
                 : "memory");
    return r != 0;
}

// Waits until the phase of parity `parity` of the mbarrier at `a` has
// completed: true; false once *abort is set or after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, const volatile uint32_t *abort)
{
    for (int i = 0; i < 64; ++i)
        if (mbar_try(a, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try(a, parity)) return true;
        if (*abort || global_ns() - t0 > kWaitNs) return false;
    }
}

// Shared memory of a latency-mode CTA: at the window base 8 mbarriers
// (tables full/empty, emission buffers full/empty, two slots each), the abort
// word at +64, the emitter's results at +72 (and its sum of squares, FP64, at
// +232), the persistent kernel's claimed item at +88, the control state at
// +256 and
// two slots of r_max pass tables after it; then four pool buffers, E[0],
// E[1], W[0], W[1], at window addresses that are multiples of their size (so
// that a gather address is one LOP3, as in the ordinary kernel).
constexpr uint32_t kMbTabFull = 0, kMbTabEmpty = 16, kMbEFull = 32, kMbEEmpty = 48;
__host__ __device__ inline size_t emit_smem_bytes(uint32_t base, uint32_t n_max, uint32_t r_max)
{
    return (size_t)pool_window(base, n_max, r_max) + 16 * (size_t)n_max - base;
}

// One stream's share of a call in the latency mode (the plain method).
// blockDim = compute threads + 64; compute thread (warp w >= 2, lane l) owns
// quadruples q0 + 32 j, q0 = (w - 2) 32 QT + l.  The emitter reads CH values
// per lane at a time (as many as the instantiation's registers allow).  All
// roles reach the closing __syncthreads, whether they finished their blocks
// or left on abort.
template <int QT, bool FULL, typename OutT, int CH>
__device__ __forceinline__ void run_stream_emit(StreamHdr *__restrict__ h, float *__restrict__ pool_g,
                                                OutT *__restrict__ out, uint64_t count, uint32_t n_max,
                                                uint32_t r_max)
{
    unsigned char *smem = wn_smem;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t N = h->N, nq = N >> 2;
    const uint32_t base = smem_base();
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const uint32_t W0 = pool_window(base, n_max, r_max);
    const uint32_t bsz = 4u * n_max;
    if (W0 + 4u * bsz > base + dyn) {  // layout does not fit: flag and do nothing
        if (tid == 0) h->flags |= 1u;
        return;
    }
    volatile uint32_t *abort = reinterpret_cast<volatile uint32_t *>(smem + 64);
    float *res = reinterpret_cast<float *>(smem + 72);   // the emitter's last sum of squares, reserved value, scale
    CtlState *ctl = reinterpret_cast<CtlState *>(smem + 256);
    PassTab *tabs = reinterpret_cast<PassTab *>(smem + 256 + sizeof(CtlState));  // [2][r_max]
    const uint32_t tabs_s = base + 256u + (uint32_t)sizeof(CtlState);
    const uint32_t nthr = blockDim.x, ncomp = nthr - 64u;
    auto ebuf = [&](uint32_t s) { return W0 + s * bsz; };       // emission buffers E[0], E[1]
    auto wbuf = [&](uint32_t s) { return W0 + (2u + s) * bsz; };  // work buffers W[0], W[1]

    {  // the stored pool goes to E[1], as if it were block -1's
        const float4 *pg4 = reinterpret_cast<const float4 *>(pool_g);
        float4 *e1 = reinterpret_cast<float4 *>(smem + (ebuf(1) - base));
        for (uint32_t i = tid; i < nq; i += nthr) e1[i] = pg4[i];
    }
    const uint32_t k0 = h->k;
    const float sc_prev = h->scale;
    const uint64_t left = (uint64_t)(N - 1 - k0);
    const uint64_t n0 = left < count ? left : count;
    const uint64_t nb = (count - n0 + (N - 2)) / (N - 1);
    const uint64_t tail = (count - n0) % (N - 1);
    const uint32_t R = h->R;
    if (tid == 0) {
        mbar_init(base + kMbTabFull, 1);
        mbar_init(base + kMbTabFull + 8, 1);
        // one arrival per warp: lane 0 arrives after a __syncwarp, which
        // orders its lanes' accesses before lane 0's release
        mbar_init(base + kMbTabEmpty, ncomp / 32u);
        mbar_init(base + kMbTabEmpty + 8, ncomp / 32u);
        mbar_init(base + kMbEFull, ncomp / 32u);
        mbar_init(base + kMbEFull + 8, ncomp / 32u);
        mbar_init(base + kMbEEmpty, 1);
        mbar_init(base + kMbEEmpty + 8, 1);
        *abort = 0u;
        ctl->gx = h->x;
        ctl->gw = h->w;
    }
    __syncthreads();
    const DbgRange rg = dbg_range(out, out + count);  // this stream's output (the debug build checks stores)
    for (uint64_t i = tid; i < n0; i += nthr) store1(rg, out + i, sc_prev * lds(ebuf(1) + 4u * (uint32_t)(k0 + i)));
    __syncthreads();  // E[1] is read: block 1's final pass may overwrite it

    if (warp == 0) {
        // tables of block b into slot b mod 2, once the compute warps are done with block b-2's
        for (uint64_t b = 0; b < nb; ++b) {
            const uint32_t s = (uint32_t)(b & 1u), k = (uint32_t)(b >> 1);
            // the warp leaves or goes on as one (a vote over its lanes' waits)
            if (!__all_sync(0xffffffffu, k == 0 || mbar_wait(base + kMbTabEmpty + 8u * s, (k - 1u) & 1u, abort))) {
                *abort = 1u;
                break;
            }
            make_tables(ctl, tabs + s * r_max, R, N, lane, false);
            __syncwarp();
            if (lane == 0) mbar_arrive(base + kMbTabFull + 8u * s);
        }
    } else if (warp == 1) {
        // the emitter: block b's values from E[b mod 2], its sum of squares and the next scale
        const float A = (float)h->A, B = (float)h->B;
        float sc = nb > 0 ? group_scale(h->sumsq, (float)h->r, A, B, N) : sc_prev;
        double ss = 0.0;
        float r = 0.f;
        OutT *ob = out + n0;
        for (uint64_t b = 0; b < nb; ++b) {
            const uint32_t s = (uint32_t)(b & 1u), k = (uint32_t)(b >> 1);
            if (!__all_sync(0xffffffffu, mbar_wait(base + kMbEFull + 8u * s, k & 1u, abort))) {
                *abort = 1u;
                break;
            }
            const uint32_t eb = ebuf(s);
            const uint32_t n_out = (b + 1 < nb || tail == 0) ? N - 1u : (uint32_t)tail;
            float part[4] = {0.f, 0.f, 0.f, 0.f};
            float rv = 0.f;  // the reserved value, unscaled
            const float sc_b = sc;
            // chunks of CH values per lane: all loads first; E[s] is handed back
            // to the compute warps as soon as its last chunk is in registers
            for (uint32_t c = 0; c < N; c += 32u * CH) {
                float v[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    const uint32_t i = c + lane + 32u * u;
                    v[u] = i < N ? lds(eb + 4u * i) : 0.f;
                }
                if (c + 32u * CH >= N) {
                    rv = lds(eb + 4u * (N - 1u));
                    __syncwarp();
                    if (lane == 0) mbar_arrive(base + kMbEEmpty + 8u * s);  // every lane has read E[s]
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) part[u & 3] = fmaf(v[u], v[u], part[u & 3]);
                if (c + 32u * CH >= N) {  // the next block's scale before this chunk's stores
                    float t = (part[0] + part[1]) + (part[2] + part[3]);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                    ss = t;
                    r = sc_b * rv;  // this block's reserved value, scaled (fastnorm2)
                    if (b + 1 < nb) sc = group_scale_f32(t, r, A, B, N);
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    const uint32_t i = c + lane + 32u * u;
                    if (i < n_out) store1(rg, ob + i, sc_b * v[u]);
                }
            }
            ob += N - 1;
        }
        if (lane == 0) {
            *reinterpret_cast<double *>(smem + 232) = ss;
            res[1] = r;
            res[2] = sc;
        }
    } else {
        const uint32_t q0 = (warp - 2u) * 32u * QT + lane;
        const uint32_t m4 = 4u * N - 1u, half = 2u * N;
        float2 acc[QT][2];
        for (uint64_t b = 0; b < nb; ++b) {
            const uint32_t s = (uint32_t)(b & 1u), k = (uint32_t)(b >> 1);
            // block b needs its tables, and E[s] free of block b-2's emission
            const bool ok = mbar_wait(base + kMbTabFull + 8u * s, k & 1u, abort) &&
                            (k == 0 || mbar_wait(base + kMbEEmpty + 8u * s, (k - 1u) & 1u, abort));
            // one decision for all compute threads (the OR of their failures,
            // reduced by the barrier that also orders the previous block's pool
            // stores before these gathers): they leave together or not at all
            if (bar_red_or(kBarPass, ncomp, !ok || *abort != 0u)) {
                *abort = 1u;
                break;
            }
            const uint32_t tb = tabs_s + s * r_max * (uint32_t)sizeof(PassTab);
            for (uint32_t p = 0; p < R; ++p) {
                const uint32_t rd = p == 0 ? ebuf(s ^ 1u) : wbuf((p - 1u) & 1u);
                const uint32_t wr = p + 1 == R ? ebuf(s) : wbuf(p & 1u);
                float2 part;
                pass_quads<QT, false, FULL, EMIT_NONE, 0, OutT, false>(rd, wr, tb + p * (uint32_t)sizeof(PassTab),
                                                                      q0, lane, m4, half, nq, part, 0, nullptr,
                                                                      nullptr, 0, acc);
                if (p + 1 < R) bar_wait(kBarPass, ncomp);
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(base + kMbTabEmpty + 8u * s);  // this warp is done with the tables
                mbar_arrive(base + kMbEFull + 8u * s);     // and has written its part of E[s]
            }
        }
    }
    __syncthreads();

    const bool failed = *abort != 0u;
    if (!failed) {
        const uint32_t fin = nb > 0 ? ebuf((uint32_t)((nb - 1) & 1u)) : ebuf(1);
        float4 *pw4 = reinterpret_cast<float4 *>(pool_g);
        for (uint32_t i = tid; i < nq; i += nthr) pw4[i] = lds4(fin + 16u * i);
    }
    if (tid == 0) {
        if (failed) {
            h->flags |= 2u;  // a wait timed out: the stream's state was not advanced
        } else if (nb > 0) {
            h->x = ctl->gx;
            h->w = ctl->gw;
            h->sumsq = *reinterpret_cast<const double *>(smem + 232);
            h->r = (double)res[1];
            h->scale = res[2];
            h->k = tail == 0 ? N - 1 : (uint32_t)tail;
            h->blocks += nb;
        } else {
            h->k = k0 + (uint32_t)n0;
        }
        for (uint32_t m = 0; m < 64u; m += 8u) mbar_inval(base + m);
    }
}

// Latency-mode generate kernel: one CTA per stream, blockDim = compute
// threads + 64 (the table warp and the emitter).
// One CTA per SM is all a lone stream needs, so the thread bound MAXT alone
// sets the registers: 192 threads (the defaults: up to 128 compute threads)
// leave room for the emitter's 32-value chunks, wider shapes use 8.
template <int MAXT> __host__ __device__ constexpr int emit_chunk() { return MAXT <= 192 ? 32 : 8; }

template <int QT, int MAXT, bool FULL, typename OutT>
__global__ void __launch_bounds__(MAXT, 1) emit_kernel(GenArgs a)
{
    StreamHdr *h = a.hdr + blockIdx.x;
    const uint64_t off = (uint64_t)blockIdx.x * a.out_stride;
    run_stream_emit<QT, FULL, OutT, emit_chunk<MAXT>()>(h, a.pools + h->pool_off, reinterpret_cast<OutT *>(a.out) + off, a.count, a.n_max,
                                    a.r_max);
}

// Persistent latency-mode kernel (batches): claims streams like
// persist_kernel and runs each with run_stream_emit.
template <int QT, int MAXT, bool FULL, typename OutT>
__global__ void __launch_bounds__(MAXT, 1) persist_emit_kernel(GenArgs a, BatchArgs bq)
{
    uint32_t *slot = reinterpret_cast<uint32_t *>(wn_smem + 88);
    for (;;) {
        __syncthreads();  // the previous stream is done with shared memory
        if (threadIdx.x == 0) *slot = atomicAdd(bq.queue, 1u);
        __syncthreads();
        const uint32_t it = *slot;
        if (it >= bq.n_items) return;
        const uint32_t si = bq.order[it];
        StreamHdr *h = a.hdr + si;
        run_stream_emit<QT, FULL, OutT, emit_chunk<MAXT>()>(h, a.pools + h->pool_off,
                                                          reinterpret_cast<OutT *>(a.out) + bq.offsets[si],
                                        bq.counts[si], a.n_max, a.r_max);
    }
}

template <int QT, int MAXT, typename OutT>
cudaError_t launch_emit_shape(const GenArgs &a, uint32_t threads, bool full, size_t smem, cudaStream_t cs)
{
    auto kern = full ? emit_kernel<QT, MAXT, true, OutT> : emit_kernel<QT, MAXT, false, OutT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<a.n_streams, threads + 64, smem, cs>>>(a);
    return cudaGetLastError();
}

template <int QT, int MAXT, typename OutT>
cudaError_t launch_persist_emit_shape(const GenArgs &a, const BatchArgs &bq, uint32_t threads, bool full, size_t smem,
                                      int sms, cudaStream_t cs)
{
    auto kern = full ? persist_emit_kernel<QT, MAXT, true, OutT> : persist_emit_kernel<QT, MAXT, false, OutT>;
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

// Launches for one output type: the shape's thread bound must admit the
// compute threads plus the two role warps.
// Launches for one output type: quadruples per thread QT in {1, 2, 4, 8, 16}
// and a thread bound of 192 (up to 128 compute threads) or 576 (up to 512).
template <typename OutT>
cudaError_t launch_emit_t(const GenArgs &a, const LaunchCfg &c, bool full, size_t smem, cudaStream_t cs)
{
    if (c.ip || c.grp || c.threads + 64 > 576u) return cudaErrorInvalidValue;
    const bool narrow = c.threads + 64 <= 192u;
    switch (c.qt) {
    case 1: return narrow ? launch_emit_shape<1, 192, OutT>(a, c.threads, full, smem, cs)
                          : launch_emit_shape<1, 576, OutT>(a, c.threads, full, smem, cs);
    case 2: return narrow ? launch_emit_shape<2, 192, OutT>(a, c.threads, full, smem, cs)
                          : launch_emit_shape<2, 576, OutT>(a, c.threads, full, smem, cs);
#ifndef WN_DEBUG
    case 4: return narrow ? launch_emit_shape<4, 192, OutT>(a, c.threads, full, smem, cs)
                          : launch_emit_shape<4, 576, OutT>(a, c.threads, full, smem, cs);
#endif
#ifndef WN_DEBUG
    case 8: return narrow ? launch_emit_shape<8, 192, OutT>(a, c.threads, full, smem, cs)
                          : launch_emit_shape<8, 576, OutT>(a, c.threads, full, smem, cs);
#endif
#ifndef WN_DEBUG
    case 16: return narrow ? launch_emit_shape<16, 192, OutT>(a, c.threads, full, smem, cs)
                           : launch_emit_shape<16, 576, OutT>(a, c.threads, full, smem, cs);
#endif
    default: return cudaErrorInvalidValue;
    }
}

template <typename OutT>
cudaError_t launch_persist_emit_t(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, size_t smem,
                                  int sms, cudaStream_t cs)
{
    if (c.ip || c.grp || c.threads + 64 > 192u) return cudaErrorInvalidValue;
    switch (c.qt) {
    case 1: return launch_persist_emit_shape<1, 192, OutT>(a, bq, c.threads, full, smem, sms, cs);
    case 2: return launch_persist_emit_shape<2, 192, OutT>(a, bq, c.threads, full, smem, sms, cs);
#ifndef WN_DEBUG
    case 4: return launch_persist_emit_shape<4, 192, OutT>(a, bq, c.threads, full, smem, sms, cs);
#endif
#ifndef WN_DEBUG
    case 8: return launch_persist_emit_shape<8, 192, OutT>(a, bq, c.threads, full, smem, sms, cs);
#endif
#ifndef WN_DEBUG
    case 16: return launch_persist_emit_shape<16, 192, OutT>(a, bq, c.threads, full, smem, sms, cs);
#endif
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_emit_f32(const GenArgs &a, const LaunchCfg &c, bool full, size_t smem, cudaStream_t cs);
cudaError_t launch_emit_bf16(const GenArgs &a, const LaunchCfg &c, bool full, size_t smem, cudaStream_t cs);
cudaError_t launch_emit_f16(const GenArgs &a, const LaunchCfg &c, bool full, size_t smem, cudaStream_t cs);
cudaError_t launch_persist_emit_f32(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, size_t smem,
                                    int sms, cudaStream_t cs);
cudaError_t launch_persist_emit_bf16(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, size_t smem,
                                     int sms, cudaStream_t cs);
cudaError_t launch_persist_emit_f16(const GenArgs &a, const BatchArgs &bq, const LaunchCfg &c, bool full, size_t smem,
                                    int sms, cudaStream_t cs);

}  // namespace wn
