/*
 * wallace_gb300.h -- C ABI of the GB300 (sm_103a) implementation of Wallace's
 * maximum-entropy normal generator, as discussed by R. P. Brent,
 * "Some Comments on C. S. Wallace's Random Number Generators"
 * (arXiv:1005.2314), Section 5.
 *
 * The method (Section 5.1): a pool of N values that are (nearly) iid N(0,1)
 * is renewed by an orthogonal map, which keeps an iid N(0,1) vector iid
 * N(0,1).  Each pass applies random-signed 4x4 blocks y_k = t - a_k,
 * t = (a_0+a_1+a_2+a_3)/2 (Section 5.3, the printed A_1 up to row order and
 * signs; Section 5.2 for the signs) to quadruples gathered through an affine
 * permutation j -> alpha*j + gamma mod N with alpha odd (Section 5.4), and
 * writes the pool transposed.  After R passes a block returns N-1 values,
 * scaled so that the pool's sum of squares is a chi-squared_N sample drawn
 * from the value held back by the previous block (Section 5.5, fastnorm2,
 * approximation (c)).  A uniform generator (xorshift64 + Weyl, seeded by
 * SplitMix64) is used only for initialisation and to choose each pass's
 * permutation and signs, two 64-bit draws per pass (Section 5.8).
 *
 * Conventions for every entry point:
 *  - Pointers named `out` are DEVICE pointers owned by the caller (e.g. a
 *    torch tensor's data_ptr()), aligned to 16 bytes, holding at least the
 *    number of elements the call writes.  Host arrays are named host_*.
 *  - `cuda_stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Generation calls are asynchronous on that stream;
 *    host-visible bookkeeping advances when the call is enqueued.
 *  - Return codes: WN_OK on success; WN_EINVAL for bad arguments (nothing is
 *    launched); WN_ENOMEM when device memory cannot be allocated; WN_ECUDA when
 *    a CUDA call fails (the text is kept for wn_last_error()).
 *  - A handle is not thread-safe: calls on one handle must not overlap.
 */
#ifndef WALLACE_GB300_H
#define WALLACE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wn_stream wn_stream; /* opaque: owns the device pools and generator states */

typedef enum {
    WN_OK = 0,
    WN_EINVAL = 1,
    WN_ENOMEM = 2,
    WN_ECUDA = 3,
    WN_ETIMEOUT = 4
} wn_status;

typedef enum {
    WN_F32 = 0,  /* float, 4 bytes per value */
    WN_BF16 = 1, /* bfloat16, round-to-nearest-even from the FP32 value */
    WN_F16 = 2   /* IEEE half, round-to-nearest-even from the FP32 value */
} wn_dtype;

#define WN_MIN_POOL 4u
#define WN_MAX_POOL 16384u
#define WN_MAX_PASSES 64u
#define WN_DEFAULT_WARMUP 8u

/*
 * wn_create -- one stream with pool size pool_N (a power of two in
 * [WN_MIN_POOL, WN_MAX_POOL]; fastnorm's is 1024, Section 5.4), passes_R
 * passes per block (1..WN_MAX_PASSES) and a 64-bit seed.  The pool is
 * initialised from the uniform generator (Section 5.8) and WN_DEFAULT_WARMUP
 * blocks are discarded.  Blocks the calling thread until the state is ready.
 * Returns NULL on error (see wn_last_error()).
 */
wn_stream *wn_create(uint32_t pool_N, uint32_t passes_R, uint64_t seed);

/*
 * wn_create_streams -- n_streams independent streams in one handle: stream i
 * has pool size pool_N[i], passes passes_R[i] and seed seeds[i] (host arrays
 * of n_streams entries), and warmup_blocks discarded blocks (0 leaves the
 * freshly initialised pool, for tests).  Each stream is a separate serial
 * chain (Section 5.1); streams share nothing.  The initialisation kernels run
 * on cuda_stream and the call synchronises it before returning.
 * Returns NULL on error.
 */
wn_stream *wn_create_streams(uint32_t n_streams, const uint32_t *pool_N, const uint32_t *passes_R,
                             const uint64_t *seeds, uint32_t warmup_blocks, void *cuda_stream);

/*
 * Method variants (Section 5.5 and Section 5.7), for wn_create_ex.
 *  chi2:     the chi-squared_N approximation the scale is drawn from, with x
 *            the reserved value: WN_CHI2_C (default) A(x^2-1) +
 *            sqrt(2(N-A^2)) x + N, A = 2 sqrt(N) sin(arcsin(1/sqrt(N))/3);
 *            WN_CHI2_A (x + sqrt(2N-1))^2 / 2 (rann4); WN_CHI2_B
 *            Wilson-Hilferty N ((2/(9N))^(1/2) x + 1 - 2/(9N))^3; WN_CHI2_OFF
 *            no correction (S = N: the sum of squares never varies, the
 *            defect Section 5.5 starts from).
 *  reserve:  where x comes from: WN_RESERVE_PREVIOUS (default, fastnorm2:
 *            the previous block's value held back) or WN_RESERVE_CURRENT
 *            (fastnorm: this block's own, which Section 5.5 explains is
 *            correlated with the block's other values).
 *  decimate: d in [1, 255]: return the values of every d-th block only; the
 *            d - 1 blocks between run in full and return nothing
 *            (Section 5.7: keep one pool in d).  1 = all.
 *  update:   WN_UPDATE_QUAD (default) the random-signed 4x4 update of
 *            fastnorm; WN_UPDATE_ROTATION rann4's plane rotations (Section
 *            5.3): each pass draws t = tan(theta/2) in (-1, 1) from the top
 *            24 bits u of its second draw, t = (2u+1)/2^24 - 1, and rotates
 *            the pairs (P[pi(j)], P[pi(j + N/2)]), pi the pass's affine
 *            permutation (Section 5.4), by c = (1-t^2)/(1+t^2),
 *            s = 2t/(1+t^2), writing them to slots 2j, 2j+1.
 */
typedef enum { WN_CHI2_OFF = 0, WN_CHI2_A = 1, WN_CHI2_B = 2, WN_CHI2_C = 3 } wn_chi2;
typedef enum { WN_RESERVE_PREVIOUS = 0, WN_RESERVE_CURRENT = 1 } wn_reserve;
typedef enum { WN_UPDATE_QUAD = 0, WN_UPDATE_ROTATION = 1 } wn_update;
typedef struct {
    uint32_t chi2;     /* wn_chi2 */
    uint32_t reserve;  /* wn_reserve */
    uint32_t decimate; /* 1..255 */
    uint32_t update;   /* wn_update */
} wn_options;

/*
 * wn_create_ex -- as wn_create_streams, every stream with the variants in
 * *opt (NULL: the defaults, i.e. wn_create_streams).  Warm-up blocks are
 * never decimated.  WN_EINVAL (NULL returned) for options out of range.
 */
wn_stream *wn_create_ex(uint32_t n_streams, const uint32_t *pool_N, const uint32_t *passes_R,
                        const uint64_t *seeds, uint32_t warmup_blocks, const wn_options *opt, void *cuda_stream);

/* wn_destroy -- frees the handle's device memory (synchronises the device
 * first).  NULL is accepted. */
void wn_destroy(wn_stream *s);

/*
 * wn_generate -- the next `count` values of every stream of `s`, FP32, on the
 * handle's CUDA stream (wn_set_cuda_stream; default NULL).  Stream i writes
 * out[i*count .. i*count + count).  Each stream's values continue its
 * sequence: the concatenation of successive calls equals one call of the
 * summed count (blocks are cut anywhere; Section 5.5's N-1 values per block).
 */
wn_status wn_generate(void *out, uint64_t count, wn_stream *s);

/* wn_generate_ex -- as wn_generate, with the output type and CUDA stream
 * given explicitly. */
wn_status wn_generate_ex(void *out, uint64_t count, wn_stream *s, wn_dtype dtype, void *cuda_stream);

/*
 * wn_generate_host -- as wn_generate_ex, but the values land in HOST memory:
 * stream i's values go to host_out[i*count .. i*count + count) (elements of
 * `dtype`).  If host_out is page-locked memory the device can address
 * (cudaHostAlloc, cudaHostRegister, a pinned torch tensor) and 16-byte
 * aligned, the kernel writes it directly over the host link.  Otherwise the
 * values are generated into a device staging area the handle owns (allocated
 * on first use: two buffers of 256 MiB) and copied out on a second CUDA
 * stream: a group of consecutive streams' whole requests at a time (one
 * contiguous range of host_out per copy) when one stream's part fits 256 MiB,
 * else every stream's next chunk per round (pitched copies).  A copy into
 * pageable memory returns to the host only when it is done, so on that route
 * the call returns after its copies and generation and copies take turns.
 * On the page-locked route the call is asynchronous on cuda_stream: the
 * values are in place once cuda_stream has been synchronised.
 */
wn_status wn_generate_host(void *host_out, uint64_t count, wn_stream *s, wn_dtype dtype, void *cuda_stream);

/*
 * wn_generate_batch -- uneven requests in one call: stream i of `s` returns
 * its next counts[i] values (0 allowed) as `dtype` to out + offsets[i]
 * elements (host arrays of wn_num_streams(s) entries; `out` 16-byte aligned;
 * the ranges must not overlap).  Streams are grouped by pool size; each group
 * runs as one persistent kernel whose CTAs claim streams, longest request
 * first, from an atomic counter in device memory the handle owns, and the
 * groups run concurrently on branch streams joined back into cuda_stream.
 * use_graph != 0: the counter reset and the group launches are captured once
 * into a CUDA graph kept by the handle, and later calls with the same out,
 * counts, offsets and dtype replay it (a call with other arguments captures
 * anew).  The graph reads a device copy of the descriptors of its own, which
 * calls with use_graph = 0 and wn_autotune_batch never touch, so eager calls
 * may come between replays.  Streams continue their sequences as with
 * wn_generate.  counts and offsets are copied (through a host buffer of the
 * library's) before the call returns: the caller may reuse or free them at
 * once, page-locked or not.  Asynchronous on cuda_stream; an upload of new
 * descriptors waits for the work already enqueued on cuda_stream.  Successive
 * calls on one handle must be ordered on the GPU (one CUDA stream, or
 * synchronisation between them).
 */
wn_status wn_generate_batch(void *out, const uint64_t *counts, const uint64_t *offsets, wn_stream *s,
                            wn_dtype dtype, int use_graph, void *cuda_stream);

/*
 * wn_generate_batch_noalloc -- the same work as wn_generate_batch with
 * use_graph = 0, for callers that must not allocate device memory: code whose
 * device memory is already fully claimed by another allocator (a framework's
 * caching pool, a fixed budget per tenant), and latency-critical serving
 * loops that cannot afford cudaMalloc, which blocks the calling thread and
 * can synchronise the device.  This call makes no cudaMalloc or cudaFree and
 * no other allocating call (nor does it create streams or events): the claim
 * counters and the request descriptors live in one fixed array of device
 * memory compiled into the library (about 320 KB, resident on every device
 * that loads the library until the process exits), so it serves at most
 * WN_NOALLOC_MAX_STREAMS streams (WN_EINVAL beyond; the 13 possible pool
 * sizes always fit its 16 counters).  The groups run one after another on
 * cuda_stream.  The first call on a device looks up the array's device
 * address there (with that device current).  The call copies the caller's
 * counts and offsets and advances the streams' positions on the host when it
 * is made, so it must not be recorded into a CUDA graph: WN_EINVAL while
 * cuda_stream is being captured.  Every call shares the array: calls whose
 * work overlaps on the GPU (e.g. on two CUDA streams at once) race on it, so
 * order them on one stream or synchronise in between.  The handle's device
 * must be current.  The paper has no counterpart to this entry point.
 */
#define WN_NOALLOC_MAX_STREAMS 16384u
wn_status wn_generate_batch_noalloc(void *out, const uint64_t *counts, const uint64_t *offsets, wn_stream *s,
                                    wn_dtype dtype, void *cuda_stream);

/*
 * wn_autotune_batch -- picks, for each pool size of the batch described by
 * out/counts/offsets/dtype (as in wn_generate_batch), the compiled launch
 * shape (or the latency mode) whose persistent kernel serves that group
 * fastest, timing each group alone; then times the whole batch with those
 * shapes for several numbers of exclusive groups (the longest serial chains,
 * one CTA per SM: none, 4, 8, ... up to a third of the SMs, or the
 * estimate's rule) and keeps the fastest; it also tries more chain groups
 * sharing SMs two or four to one (see wn_set_batch_plan).  All timing runs on
 * a saved copy of the state (the streams' sequences are unaffected; `out` is
 * overwritten with scratch values).  Later wn_generate_batch calls use the
 * choices.  A batch tuned before on this device (the tune cache, see
 * wn_autotune) takes its cached choices without timing.  Synchronous.
 */
wn_status wn_autotune_batch(void *out, const uint64_t *counts, const uint64_t *offsets, wn_stream *s,
                            wn_dtype dtype, void *cuda_stream);

/*
 * wn_get_batch_plan / wn_set_batch_plan -- how wn_generate_batch treats the
 * batch's longest serial chains (a stream is a serial chain of blocks,
 * Section 5.1): `chains` requests, longest first, run in the latency mode in
 * chain groups launched ahead of the others, at most `density` chain CTAs per
 * SM (1: each has an SM to itself); chains = -1 lets an estimate decide,
 * 0 uses none.  wn_autotune_batch sets both by timing the whole batch;
 * wn_set_batch_plan overrides them (and drops a captured graph).  WN_EINVAL
 * for chains < -1 or density outside [1, 8].  The plan changes only where
 * and when streams run, never their values.
 */
wn_status wn_get_batch_plan(const wn_stream *s, int32_t *chains, uint32_t *density);
wn_status wn_set_batch_plan(wn_stream *s, int32_t chains, uint32_t density);

/*
 * wn_set_batch_chain_kernel -- which kernel runs a batch's chain groups:
 * chain_mode = 1 the chain mode (wn_set_config_ex, WN_CFG_CHAIN) for the pool
 * sizes it serves, 0 (the default) the latency modes.  Measured on the
 * 10,000-stream batch: a call after the GPU was idle, and eager calls, run
 * ~1 ms faster in the chain mode (22.3-23.5 against 23.6 ms), but graph
 * replays issued back to back took 30-37 ms in it, as if the chain CTAs then
 * reached the SMs after the throughput groups' CTAs.  Drops a captured graph;
 * WN_EINVAL for other values.  Values do not depend on the choice.
 */
wn_status wn_set_batch_chain_kernel(wn_stream *s, int32_t chain_mode);

/*
 * wn_gbm -- a fused Monte Carlo consumer: geometric Brownian motion terminal
 * prices driven by the streams' own normals, which never leave the chip.
 * Stream i serves paths [i*paths_per_stream, (i+1)*paths_per_stream); path p
 * of stream i takes value j*paths_per_stream + p of the stream's sequence as
 * its step-j normal Z_j and follows the exact log step
 * S <- S exp((mu - sigma^2/2) dt + sigma sqrt(dt) Z_j) from S0 for `steps`
 * steps.  ST_out (device, float, n_streams * paths_per_stream entries)
 * receives the terminal prices.  Requires, for every stream, that
 * paths_per_stream divide pool_N - 1, that steps * paths_per_stream be a
 * multiple of pool_N - 1, and that no values of a partly returned block be
 * pending (WN_EINVAL otherwise).  Advances each stream as generating
 * steps * paths_per_stream values would.  Asynchronous on cuda_stream.
 */
wn_status wn_gbm(wn_stream *s, float *ST_out, uint32_t paths_per_stream, uint32_t steps, double S0, double mu,
                 double sigma, double dt, void *cuda_stream);

/* wn_set_cuda_stream -- CUDA stream used by wn_generate. */
wn_status wn_set_cuda_stream(wn_stream *s, void *cuda_stream);

/*
 * wn_set_config -- launch shape of the handle's generate kernel: `threads`
 * per CTA (a multiple of 32) each updating `quads_per_thread` quadruples per
 * pass, with threads * quads_per_thread >= pool_N/4 for the handle's largest
 * pool.  (0, 0) restores the default.  The shape changes only the order of
 * the FP32 partial sums of squares, so outputs stay within the same FP32
 * tolerance of the oracle; integer streams are unaffected.  WN_EINVAL if no
 * compiled kernel has that shape.
 */
wn_status wn_set_config(wn_stream *s, uint32_t quads_per_thread, uint32_t threads);

/*
 * wn_set_config_ex -- wn_set_config with layout flags.  WN_CFG_IN_PLACE keeps
 * each pool in one shared-memory buffer instead of two: a pass gathers all of
 * its quadruples into registers, the compute warps meet at a barrier, and the
 * results overwrite the pool.  This halves a CTA's shared memory, so that
 * more CTAs share an SM (two with 16384-value pools instead of one), at the
 * cost of one more barrier per pass.  The values are bit-identical to the
 * two-buffer layout of the same shape.  Compiled for 16 quadruples per
 * thread only; WN_EINVAL for unknown flags or shapes.  Launches of few
 * streams that would take the latency mode use the ordinary kernel instead.
 */
#define WN_CFG_IN_PLACE 1u
/*
 * WN_CFG_GROUP selects the group-mode kernel for handles of the plain method
 * whose streams share one pool size: threads / 32 warps own each stream with
 * no control warp (each warp draws and derives every pass's permutation and
 * signs itself, Sections 5.2, 5.4 and 5.8), the pool stays in one
 * shared-memory buffer, and each block's scale (Section 5.5) is formed at the
 * end of the block before it.  quads_per_thread is then the quadruples per
 * lane, with 128 * quads_per_thread * (threads / 32) = pool_N; compiled for
 * (pool 1024: 8, 32), (2048: 16, 32), (4096: 32, 32), (4096: 16, 64),
 * (8192: 32, 64), (16384: 32, 128).  The launch pads each CTA's shared memory
 * so that the streams fill whole waves of the SMs.  Values agree with the
 * ordinary kernel's within the FP32 tolerance (the sums of squares are added
 * in another order); integer streams are identical.  WN_EINVAL for other
 * shapes, variants, mixed pool sizes, or a device whose dynamic shared memory
 * does not start at window address 1024.
 */
#define WN_CFG_GROUP 2u
/*
 * WN_CFG_CHAIN selects the chain-mode kernel, built for streams whose serial
 * chain of blocks sets the time (Section 5.1: each block's pool is the
 * previous block's output): threads / 32 compute warps run only a stream's
 * passes (one barrier per pass), while helper warps draw the passes'
 * permutations and signs blocks ahead (Sections 5.2, 5.4, 5.8), form each
 * block's scale from its sums of squares (Section 5.5) and write each block's
 * values (for pools up to 8192 staged in shared memory and written with bulk
 * copies).  quads_per_thread is the quadruples
 * per lane, with 128 * quads_per_thread * (threads / 32) = pool_N; compiled
 * for (pool 1024: 2, 128 and 1, 256), (2048: 2, 256), (4096: 4, 256),
 * (8192: 8, 256), (16384: 16, 256).  Launches of few streams of one
 * pool size use it without being asked.  Values agree with the other kernels
 * within the FP32 tolerance (sums of squares added in FP32, in another
 * order); integer streams are identical.  WN_EINVAL for other shapes,
 * variants, mixed pool sizes, or together with the other flags.
 */
#define WN_CFG_CHAIN 4u
wn_status wn_set_config_ex(wn_stream *s, uint32_t quads_per_thread, uint32_t threads, uint32_t flags);

/*
 * wn_autotune -- times every compiled launch shape (and layout) that covers the handle's
 * pools on a saved copy of its state, generating `count` values per stream as
 * `dtype`, and keeps the fastest for later calls (the streams' sequences are
 * unaffected: the state is restored afterwards).  The chosen shape is
 * returned through quads_per_thread and threads (either may be NULL).  A
 * result is remembered per (streams, largest pool, passes, dtype, count) for
 * the process, and kept across processes in the tune cache (below).
 * Synchronous; allocates a temporary output of n_streams * count elements and
 * a copy of the state.
 *
 * The tune cache: a small JSON file of the tuners' choices, keyed by the
 * device's name and SM count and the workload (pool size, passes, stream
 * count, output type, method variant; for batches a hash of every stream's
 * pool size, passes and request length), at $WN_TUNE_CACHE if that is set
 * ("off": no file), else $XDG_CACHE_HOME/wn/tune.json, else
 * $HOME/.cache/wn/tune.json.  wn_create, wn_create_streams and wn_create_ex
 * apply the FP32 shape cached for their workload; wn_autotune and
 * wn_autotune_batch use a cached choice instead of timing (and write the
 * choices they time).  Entries naming shapes this library did not compile,
 * and unreadable files, are ignored.
 */
wn_status wn_autotune(wn_stream *s, uint64_t count, wn_dtype dtype, void *cuda_stream,
                      uint32_t *quads_per_thread, uint32_t *threads);

/* wn_get_config -- the launch shape the next generate call will use (for a
 * handle of few streams, the chain mode's or the latency mode's). */
wn_status wn_get_config(const wn_stream *s, uint32_t *quads_per_thread, uint32_t *threads);

/* wn_get_config_ex -- the same and its layout flags (WN_CFG_IN_PLACE,
 * WN_CFG_GROUP, WN_CFG_CHAIN); any output pointer may be NULL. */
wn_status wn_get_config_ex(const wn_stream *s, uint32_t *quads_per_thread, uint32_t *threads, uint32_t *flags);

/* wn_num_streams -- number of streams in the handle (0 for NULL). */
uint32_t wn_num_streams(const wn_stream *s);

/*
 * wn_get_pool -- copies stream i's current pool (pool_N floats, in the
 * library's own scaling: its sum of squares is N up to rounding) to
 * host_out.  Synchronises the handle's CUDA stream.
 */
wn_status wn_get_pool(const wn_stream *s, uint32_t i, float *host_out);

/*
 * wn_get_state -- stream i's generator words host_xw[0..1] (xorshift, Weyl),
 * the reserved value r of the last block (Section 5.5), the scale of the
 * last block, the number k of that block's values already returned, and the
 * number of blocks completed.  Any output pointer may be NULL.
 * Synchronises the handle's CUDA stream.
 */
wn_status wn_get_state(const wn_stream *s, uint32_t i, uint64_t *host_xw, double *host_r,
                       float *host_scale, uint32_t *host_k, uint64_t *host_blocks);

/*
 * wn_save -- checkpoint: serialise the complete state of every stream of the
 * handle (generator words, Section 5.8; pool, reserved value, sum of squares,
 * block count and the position within the last block, Section 5.5) into the
 * caller's host buffer.  Synchronises the handle's device first, so the state
 * includes every call enqueued before on any CUDA stream (the caller's
 * current device is left as it was).  With host_buf == NULL only
 * *bytes_needed is set.  Layout (little-endian, version 1): 8-byte magic
 * "WNSTATE1", uint32 stream count, uint32 header size (96), the 96-byte
 * per-stream headers, the pools as FP32 in stream order, and an FNV-1a 64
 * checksum of everything before it.  WN_EINVAL if buf_bytes is too small.
 */
wn_status wn_save(const wn_stream *s, void *host_buf, uint64_t buf_bytes, uint64_t *bytes_needed);

/*
 * wn_load -- resume: a new handle whose streams continue exactly where the
 * saved ones stood (the next call returns, bit for bit, what the saved
 * handle's next call would have).  The buffer is validated before any
 * device memory is touched: magic, version, sizes, checksum, pool sizes
 * (powers of two in [4, 16384]), pass counts, positions and generator words;
 * a corrupt buffer returns NULL with the reason in wn_last_error().  The
 * handle is created on the current device; the copies run on cuda_stream,
 * which is then synchronised.
 */
wn_stream *wn_load(const void *host_buf, uint64_t buf_bytes, void *cuda_stream);

/*
 * wn_rng_draws -- the first n 64-bit draws of the stream generator seeded by
 * `seed` (SplitMix64 seeding, xorshift64 (13,7,17) + Weyl), computed on the
 * device and copied to host_out.  For checking the integer stream
 * (Section 5.8).  Synchronous.
 */
wn_status wn_rng_draws(uint64_t seed, uint64_t n, uint64_t *host_out);

/*
 * wn_boxmuller -- the conventional comparison method (Section 4; Section 5
 * names Box-Muller): `count` normals for each of n_streams streams, stream i
 * writing out[i*count ..).  Value j of stream i is component j mod 2 of pair
 * (j mod 4)/2 of Philox4x32-10 block j/4 with counter (j/4 low, j/4 high, i, 0)
 * and key (seed low, seed high): u1 = ((w >> 8) + 1) 2^-24,
 * u2 = (w' >> 8) 2^-24, rho = sqrt(-2 ln u1), (rho cos 2 pi u2,
 * rho sin 2 pi u2).  Computed in FP32 and stored as `dtype`.
 */
wn_status wn_boxmuller(void *out, uint64_t count, uint32_t n_streams, uint64_t seed,
                       wn_dtype dtype, void *cuda_stream);

/*
 * wn_debug_report -- the debug build's bounds record.  A library built with
 * -DWN_DEBUG (build(debug=True): libwallace_gb300_debug.so) checks every pool
 * access of the generator kernels' passes, emission and pool loads against
 * the CTA's dynamic shared memory (window address and alignment) and every
 * output store against its stream's range; a violation is counted, the first
 * one's kind and address kept (*host_first = kind << 56 | address, kind 1:
 * shared window address, 2: global address) and the access skipped -- nothing
 * traps.  Synchronises the device; reset != 0 clears the record afterwards.
 * Other builds return WN_EINVAL (and zeros).
 */
wn_status wn_debug_report(uint64_t *host_violations, uint64_t *host_first, int reset);

/* wn_last_error -- text of the last error on the calling thread ("" if none). */
const char *wn_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* WALLACE_GB300_H */
