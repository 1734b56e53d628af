// wn_device.cuh -- device-side pieces of the Wallace generator for sm_103a.
//
// Brent, arXiv:1005.2314, Section 5: a pool of N normal values renewed by
// random-signed 4x4 orthogonal updates on permuted quadruples, with a
// chi-squared rescale per block.  This header holds the per-stream state
// layout, the integer generator and the small FP64 helpers; the kernels live
// in wallace.cu.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace wn {

// Per-stream state in device memory.  The pool itself lives in a separate
// float array at pools + pool_off (16-byte aligned).
struct __align__(16) StreamHdr {
    uint64_t x;        // xorshift64 state (never 0); holds the seed until init
    uint64_t w;        // Weyl state
    double r;          // scaled reserved value of the last block (Section 5.5)
    double A;          // chi-squared (c) constant for nu = N
    double B;          // sqrt(2 (N - A^2))
    uint64_t pool_off; // float offset of the pool
    uint64_t blocks;   // blocks completed, warm-up included
    float scale;       // output scale of the last block
    uint32_t k;        // values of the last block already returned (N-1: none left)
    uint32_t N;        // pool size, a power of two
    uint32_t R;        // passes per block
    uint32_t flags;    // nonzero: a launch could not run this stream (bit 0: shared-memory layout)
    uint32_t variant;  // bits 0-1 chi-squared approximation (VAR_CHI2_*), bit 2 reserved value from the
                       // current pool (fastnorm), bit 3 plane rotations instead of the 4x4 update
                       // (rann4), bits 8-15 pool decimation d (0 and 1: none)
    double sumsq;      // sum of squares of the stored pool, as the generate kernel forms it
    uint64_t pad2_;
};
static_assert(sizeof(StreamHdr) == 96, "StreamHdr layout");

// StreamHdr::variant (Section 5.5's approximations and reserved value; Section 5.7's decimation)
constexpr uint32_t VAR_CHI2_OFF = 0, VAR_CHI2_A = 1, VAR_CHI2_B = 2, VAR_CHI2_C = 3;
constexpr uint32_t VAR_RESERVE_CURRENT = 4u, VAR_ROTATION = 8u;
__host__ __device__ inline uint32_t var_chi2(uint32_t v) { return v & 3u; }
__host__ __device__ inline bool var_current(uint32_t v) { return (v & VAR_RESERVE_CURRENT) != 0; }
__host__ __device__ inline uint32_t var_decimate(uint32_t v) { return ((v >> 8) & 0xFFu) > 1u ? (v >> 8) & 0xFFu : 1u; }
__host__ __device__ inline bool var_rotation(uint32_t v) { return (v & VAR_ROTATION) != 0; }
__host__ __device__ inline bool var_valid(uint32_t v) { return (v & ~0xFF0Fu) == 0; }

constexpr uint64_t kGoldenGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kWeyl = 0x61C8864680B583EBull;  // 2^64 - kGoldenGamma, odd

// SplitMix64 (Steele, Lea and Flood 2014): one step on `s`.
__device__ __forceinline__ uint64_t splitmix64(uint64_t &s)
{
    s += kGoldenGamma;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One draw: xorshift64 with shifts (13, 7, 17), Weyl step, sum mod 2^64.
__device__ __forceinline__ uint64_t draw(uint64_t &x, uint64_t &w)
{
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    w += kWeyl;
    return x + w;
}

// Seed the generator: first SplitMix64 output is the xorshift state (1 if
// it is 0), the second the Weyl state.
__device__ __forceinline__ void seed_gen(uint64_t seed, uint64_t &x, uint64_t &w)
{
    uint64_t sm = seed;
    x = splitmix64(sm);
    if (x == 0) x = 1;
    w = splitmix64(sm);
}

// --- the debug build (-DWN_DEBUG) -------------------------------------------
// Device bounds checks that never trap: every checked access that would fall
// outside its range (or be misaligned) is counted in wn_dbg_record, the first
// one's kind and address kept, and skipped.  wn_dbg_record[0]: violations;
// [1]: (kind << 56) | address of the first (kind 1: shared window address, 2:
// global address).  The debug build compiles with relocatable device code, so
// that every translation unit counts into the one record.
#ifdef WN_DEBUG
extern __device__ unsigned long long wn_dbg_record[4];
__device__ __forceinline__ void dbg_fail(unsigned long long kind, unsigned long long where)
{
    if (atomicAdd(&wn_dbg_record[0], 1ull) == 0ull)
        atomicExch(&wn_dbg_record[1], (kind << 56) | (where & 0x00FFFFFFFFFFFFFFull));
}
// The bytes [lo, hi) a stream's output may take.
struct DbgRange {
    const void *lo, *hi;
};
#else
struct DbgRange {};
#endif
__device__ __forceinline__ DbgRange dbg_range(const void *lo, const void *hi)
{
#ifdef WN_DEBUG
    return DbgRange{lo, hi};
#else
    (void)lo;
    (void)hi;
    return DbgRange{};
#endif
}
// A global store of `bytes` at p: inside the range and aligned to `bytes`.
__device__ __forceinline__ bool dbg_global_ok(const DbgRange &rg, const void *p, unsigned bytes)
{
#ifdef WN_DEBUG
    const char *c = static_cast<const char *>(p);
    if (c < static_cast<const char *>(rg.lo) || c + bytes > static_cast<const char *>(rg.hi) ||
        reinterpret_cast<uintptr_t>(p) % bytes != 0) {
        dbg_fail(2, reinterpret_cast<uintptr_t>(p));
        return false;
    }
#else
    (void)rg;
    (void)p;
    (void)bytes;
#endif
    return true;
}

template <typename T> __device__ __forceinline__ T to_out(float v);
template <> __device__ __forceinline__ float to_out<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half to_out<__half>(float v) { return __float2half_rn(v); }

}  // namespace wn
