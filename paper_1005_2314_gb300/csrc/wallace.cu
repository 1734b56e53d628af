// wallace.cu -- host runtime and C ABI of the GB300 (sm_103a) Wallace
// maximum-entropy normal generator (Brent, arXiv:1005.2314, Section 5), plus
// the stream initialisation kernel.  The generate kernel itself is in
// wn_gen.cuh (instantiated per output type in gen_*.cu).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "wallace_gb300.h"
#include "wn_gen.cuh"
#include "wn_group.cuh"
#include "wn_emit.cuh"
#include "wn_chain.cuh"
#include "tune_cache.h"

namespace wn {

#ifdef WN_DEBUG
// The debug build's violation record (wn_device.cuh, dbg_fail).
__device__ unsigned long long wn_dbg_record[4];
#endif

// ---------------------------------------------------------------------------
// Initialisation (Section 5.8): seed, N draws -> v_i = 2 (sum of the four
// 16-bit fields) - 4*65535, scale so that sum v_i^2 = N.  The v_i and their
// squares are integers, so the sum is exact and the FP64 scale is the
// correctly rounded sqrt(N / sum); each pool value is the FP32 rounding of the
// FP64 product.  The stored sum of squares is that of the FP32 pool.
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
    double ps = 0.0;
    for (uint32_t i = lane; i < N; i += 32) {
        const float v = (float)((double)vsm[i] * scale);
        P[i] = v;
        ps += (double)v * (double)v;
    }
    for (int o = 16; o > 0; o >>= 1) ps += __shfl_xor_sync(0xffffffffu, ps, o);
    if (lane == 0) {
        // constants of the chi-squared approximation (Section 5.5): S/N - 1 is
        // (A (r^2 - 1) + B r) / N for (c), for (a) (A = 1/2, B = sqrt(2N-1))
        // and for no correction (A = B = 0); Wilson-Hilferty (b) uses
        // A = sqrt(2/(9N)) and B = 2/(9N) in (1 + A r - B)^3 - 1
        const double nu = (double)N;
        double A = 0.0, B = 0.0;
        switch (var_chi2(h->variant)) {
        case VAR_CHI2_A: A = 0.5; B = sqrt(2.0 * nu - 1.0); break;
        case VAR_CHI2_B: B = 2.0 / (9.0 * nu); A = sqrt(B); break;
        case VAR_CHI2_C:
            A = 2.0 * sqrt(nu) * sin(asin(1.0 / sqrt(nu)) / 3.0);
            B = sqrt(2.0 * (nu - A * A));
            break;
        default: break;
        }
        h->x = x;
        h->w = w;
        h->r = 0.0;
        h->A = A;
        h->B = B;
        h->blocks = 0;
        h->scale = 1.0f;
        h->k = N - 1;
        h->flags = 0;
        h->sumsq = ps;
    }
}

__global__ void smem_base_kernel(uint32_t *out)
{
    if (threadIdx.x == 0) *out = smem_base();
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


// Device copy of a batch's request descriptors, in one allocation: output
// offsets and counts (uint64 per stream), the claim order (uint32 per
// stream; each pool-size group's streams, longest first) and 16 claim
// counters (one per group).
struct BatchDesc {
    unsigned char *base = nullptr;
    uint64_t *counts = nullptr, *offsets = nullptr;
    uint32_t *order = nullptr, *queue = nullptr;
};

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
    // values of each stream's last block already returned, as of the calls
    // enqueued so far (N-1: at a block boundary)
    std::vector<uint32_t> k_host;
    // window address where dynamic shared memory starts (probed at creation)
    uint32_t smem_base = 0;
    bool uniform_N = true;  // every stream has pool n_max
    int sms = 0;  // multiprocessors of the device
    int smem_optin = 0;  // largest dynamic shared memory a CTA may request
    // batches (wn_generate_batch): per-stream descriptors on the device, one
    // claim counter per pool-size group, branch streams for the groups, the
    // tuned shape per pool size, and the last captured graph.  The graph reads
    // descriptors of its own (bd_graph), which only a new capture rewrites, so
    // that eager calls and the tuner (bd_eager) never change what a cached
    // graph replays.
    BatchDesc bd_eager, bd_graph;
    std::vector<cudaStream_t> branch;
    std::vector<cudaEvent_t> join;
    // branch streams of the greatest priority, for exclusive groups: their
    // few CTAs must reach the SMs before the other groups' persistent CTAs
    // fill them (a persistent CTA leaves its SM only when its queue is empty)
    std::vector<cudaStream_t> branch_hi;
    cudaEvent_t fork = nullptr;
    std::map<uint32_t, wn::LaunchCfg> group_cfg;
    cudaGraphExec_t gexec = nullptr;
    void *g_out = nullptr;
    int g_dtype = -1;
    std::vector<uint64_t> g_counts, g_offsets;
    // batches: latency-mode persistent kernels for exclusive groups (1) or for
    // every group whose pool size has a latency shape (2); 0: never.  The
    // batch tuner's choice per pool size (group_lat) overrides it.
    int batch_lat = 2;
    // batches: how many of the longest serial chains get chain groups (the
    // latency mode), as timed on the whole batch by wn_autotune_batch (-1: the
    // estimate's rule), and how many chain CTAs share an SM (1: exclusive)
    int batch_crit = -1;
    int batch_density = 1;
    // batches: chain groups of pools the chain mode serves run it (else the
    // latency modes); see wn_set_batch_chain_kernel
    bool batch_chain_mode = false;
    int sm_smem = 0, smem_reserved = 0;  // shared memory per SM and reserved per CTA
    std::map<uint32_t, bool> group_lat;
    // some stream runs a method variant (wn_create_ex, wn_load): use the
    // kernels that read StreamHdr::variant (the others compile the plain method)
    bool var = false;
    // launch configuration chosen by wn_set_config (otherwise the default)
    bool has_cfg = false;
    wn::LaunchCfg cfg{};
    // CTAs per SM the last group-mode launch was sized for
    uint32_t group_ctas = 0;
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

// A compiled shape (wn::kShapes) whose thread bound, counting the control
// warp, admits `threads` compute threads covering the largest pool.
bool cfg_ok(const LaunchCfg &c, uint32_t n_max)
{
    bool compiled = false;
    for (const auto &k : wn::kShapes) compiled |= (k[0] == c.qt && k[1] == c.maxt && k[3] == c.ip);
    return compiled && c.grp == 0 && c.threads >= 32 && c.threads % 32 == 0 && c.threads + 32 <= (uint32_t)c.maxt &&
           (uint64_t)c.threads * c.qt >= n_max / 4;
}

// Default compute threads and quadruples per thread for a launch whose
// largest pool is n_max (measured on GB300 for 4096 streams of N = 4096, R = 2:
// 8 quadruples x 128 threads beat 4 x 256 by 13% and 2 x 512 by 50%): one
// quadruple per thread up to N = 1024 (at least one full warp), eight above;
// pools of 16384 in place, 16 quadruples x 256 threads, two CTAs per SM
// (4096 streams, R = 3, BF16 out: 10.6 ms against 11.2 for the same shape
// with two buffers and 11.9 for 8 x 512).
LaunchCfg pick_cfg(uint32_t n_max)
{
    const uint32_t nq = n_max / 4;
    if (nq <= 256) return {1, 1024, std::max(32u, (nq + 31u) / 32u * 32u)};
    if (nq <= 1024) return {8, 160, nq / 8};
    if (nq >= 4096) return {16, 288, nq / 16, 1};
    return {8, 544, nq / 8};
}

// A compiled group-mode shape (wn::kGroupShapes) for pool N with G warps.
bool group_shape_ok(uint32_t N, uint32_t G)
{
    for (const auto &k : wn::kGroupShapes)
        if ((uint32_t)k[0] == N && (uint32_t)k[1] == G) return true;
    return false;
}

// Group mode serves handles of the plain method whose streams all have one
// pool size, when dynamic shared memory starts where the kernel expects it.
bool group_eligible(const wn_stream *s)
{
    return !s->var && s->uniform_N && s->smem_base == wn::kGroupBase;
}

// The group-mode shape of pool N with G warps per stream.
LaunchCfg group_cfg_of(uint32_t N, uint32_t G)
{
    LaunchCfg c{(int)(N / (128u * G)), (int)(32u * G), 32u * G, 1};
    c.grp = 1;
    return c;
}

// A compiled chain-mode shape (wn::kChainShapes) for pool N with G compute warps.
bool chain_shape_ok(uint32_t N, uint32_t G)
{
    for (const auto &k : wn::kChainShapes)
        if ((uint32_t)k[0] == N && (uint32_t)k[1] == G) return true;
    return false;
}

// The chain-mode shape of pool N with G compute warps (plus the scale warp).
LaunchCfg chain_cfg_of(uint32_t N, uint32_t G)
{
    LaunchCfg c{(int)(N / (128u * G)), (int)(32u * (G + 1)), 32u * G, 0};
    c.grp = 2;
    return c;
}

// Compute warps of the chain mode's default shape for pool N (false: none).
bool chain_default(uint32_t N, uint32_t &G)
{
    switch (N) {
    case 1024: G = 4; break;
    case 2048:
    case 4096:
    case 8192:
    case 16384: G = 8; break;
    default: G = 0; return false;
    }
    return chain_shape_ok(N, G);
}

// The chain mode serves the plain method (any number of streams of one pool
// size); its shared memory must fit one CTA.
bool chain_fits(const wn_stream *s, uint32_t N, uint32_t G)
{
    return !s->var && chain_shape_ok(N, G) &&
           wn::chain_smem_bytes(s->smem_base, N, G, s->r_max) <= (size_t)s->smem_optin;
}

// Pool sizes whose default launch is the group mode, with its warps per
// stream (other sizes keep pick_cfg's shapes).  Measured on GB300 against
// the ordinary kernel's defaults: 4096 streams of pool 4096, R = 2, 2^20 FP32
// each, 3.18 ms (one warp per stream) against 3.65; 4864 streams of pool
// 1024, 11.5 -> 3.8 ms; 4096 streams of pool 16384, R = 3, 2^21 BF16 each,
// 10.6 -> 8.3 ms (four warps per stream); two warps per stream of pool 4096
// were slower than one (1.31e12 against 1.36e12 values/s at equal waves).
bool group_default(uint32_t N, uint32_t &G)
{
    switch (N) {
    case 1024:
    case 2048:
    case 4096: G = 1; return true;
    case 8192: G = 2; return true;
    case 16384: G = 4; return true;
    default: G = 0; return false;
    }
}

// The launch shape a generate call of the handle uses when none was set.
LaunchCfg default_cfg(const wn_stream *s)
{
    uint32_t G = 0;
    if (group_eligible(s) && group_default(s->n_max, G) && group_shape_ok(s->n_max, G))
        return group_cfg_of(s->n_max, G);
    return pick_cfg(s->n_max);
}

// The latency mode (two control warps beside the compute warps; see
// run_stream_lat) serves launches of few streams of the plain method, where
// each stream's serial chain of blocks sets the time.  Its shape: the user's
// (or the tuner's) when two control warps fit in its thread bound, else four
// compute warps (measured best for lone streams of pools 1024 and 4096: 2 x
// 128 and 8 x 128), fewer for small pools.  false: no such shape (pools above
// 8192 keep the ordinary kernel).
bool fits_latency(const LaunchCfg &c, uint32_t n_max)
{
    return !c.ip && cfg_ok(c, n_max) && c.threads + 64 <= (uint32_t)c.maxt;
}

// Dynamic shared memory of a launch of shape c over pools of up to n values
// and up to r passes per block: one pool buffer in place, else two.
size_t cfg_smem(const wn_stream *s, const LaunchCfg &c, uint32_t n, uint32_t r)
{
    return c.ip ? wn::gen_smem_bytes_ip(n, r) : wn::gen_smem_bytes(s->smem_base, n, r);
}

bool latency_default(uint32_t n_max, LaunchCfg &out)
{
    const uint32_t nq = n_max / 4;
    const uint32_t t = nq >= 128 ? 128u : std::max(32u, (nq + 31u) / 32u * 32u);
    const int qt = (int)std::max(1u, nq / t);
    for (const auto &k : wn::kShapes) {
        const LaunchCfg c{k[0], k[1], t, k[3]};
        if (k[0] == qt && fits_latency(c, n_max)) {
            out = c;
            return true;
        }
    }
    return false;
}

bool latency_cfg_for(const wn_stream *s, LaunchCfg &out, uint32_t n_launch)
{
    if (s->var || n_launch > (uint32_t)std::max(1, s->sms / 2)) return false;
    if (s->r_max >= 3 && wn::emit_smem_bytes(s->smem_base, s->n_max, s->r_max) > (size_t)s->smem_optin) return false;
    if (s->has_cfg) {
        if (!fits_latency(s->cfg, s->n_max)) return false;
        out = s->cfg;
        return true;
    }
    return latency_default(s->n_max, out);
}

// The chain mode (wn_chain.cuh) for a generate launch of n_launch streams:
// the handle's shape when it is a chain shape; with no shape set, the default
// chain shape of the pool size for launches of few streams (each stream's
// serial chain of blocks then sets the time).
bool chain_cfg_for(const wn_stream *s, LaunchCfg &out, uint32_t n_launch)
{
    if (s->var || !s->uniform_N) return false;
    if (s->has_cfg) {
        if (s->cfg.grp != 2 || !chain_fits(s, s->n_max, s->cfg.threads / 32u)) return false;
        out = s->cfg;
        return true;
    }
    uint32_t G = 0;
    if (n_launch > (uint32_t)std::max(1, s->sms / 2) || !chain_default(s->n_max, G) || !chain_fits(s, s->n_max, G))
        return false;
    out = chain_cfg_of(s->n_max, G);
    return true;
}

// --- the autotuners' choices across processes (tune_cache.cu) -------------
// The device's name and SM count, the first part of every key.
std::string device_tag(const wn_stream *s)
{
    static std::mutex mu;
    static std::map<int, std::string> names;
    std::lock_guard<std::mutex> lock(mu);
    auto it = names.find(s->device);
    if (it == names.end()) {
        cudaDeviceProp p{};
        std::string nm = "unknown";
        if (cudaGetDeviceProperties(&p, s->device) == cudaSuccess) nm = p.name;
        for (char &c : nm)
            if (c == ' ' || c == '"' || c == '|' || c == '\\') c = '_';
        it = names.emplace(s->device, nm).first;
    }
    return it->second + "|sms=" + std::to_string(s->sms);
}

std::string cfg_text(const LaunchCfg &c)
{
    char b[96];
    std::snprintf(b, sizeof b, "%d %d %u %d %d", c.qt, c.maxt, c.threads, c.ip, c.grp);
    return b;
}

bool cfg_from_text(const char *t, LaunchCfg &c)
{
    unsigned th = 0;
    if (std::sscanf(t, "%d %d %u %d %d", &c.qt, &c.maxt, &th, &c.ip, &c.grp) != 5) return false;
    c.threads = th;
    return true;
}

// A shape read from the file is used only if this library compiled it.
bool cached_cfg_ok(const LaunchCfg &c, uint32_t N)
{
    if (c.grp == 2) return c.threads % 32 == 0 && chain_shape_ok(N, c.threads / 32u) && c.ip == 0 &&
                           (uint64_t)128u * c.qt * (c.threads / 32u) == N;
    if (c.grp) return c.grp == 1 && c.threads % 32 == 0 && group_shape_ok(N, c.threads / 32u) && c.ip == 1 &&
                      (uint64_t)128u * c.qt * (c.threads / 32u) == N;
    return cfg_ok(c, N);
}

// Key of a handle's generate shape for output type dt.
std::string gen_key(const wn_stream *s, wn_dtype dt)
{
    return "gen|" + device_tag(s) + "|N=" + std::to_string(s->n_max) + "|R=" + std::to_string(s->r_max) +
           "|uniform=" + std::to_string((int)s->uniform_N) + "|var=" + std::to_string((int)s->var) +
           "|streams=" + std::to_string(s->n) + "|dtype=" + std::to_string((int)dt);
}

// The cached generate shape of the handle for dt, if any and valid.
bool cached_gen_cfg(const wn_stream *s, wn_dtype dt, LaunchCfg &c)
{
    std::string v;
    if (!wn::tune_cache_get(gen_key(s, dt), v) || !cfg_from_text(v.c_str(), c) || !cached_cfg_ok(c, s->n_max))
        return false;
    if (c.grp == 2) return s->uniform_N && chain_fits(s, s->n_max, c.threads / 32u);
    return !c.grp || group_eligible(s);
}

// One generate launch over streams [first, first + len) of the handle (all of
// them by default): stream first + i writes out[i count .. (i+1) count).
wn_status launch_generate(wn_stream *s, void *out, uint64_t count, uint32_t warmup, wn_dtype dt,
                          cudaStream_t cs, uint32_t first = 0, uint32_t len = 0xffffffffu)
{
    wn::GenArgs a;
    a.hdr = s->d_hdr + first;
    a.pools = s->d_pools;
    a.out = out;
    a.count = count;
    a.out_stride = count;
    a.n_streams = std::min(len, s->n - first);
    a.n_max = s->n_max;
    a.r_max = s->r_max;
    a.warmup_blocks = warmup;
    cudaError_t e;
    LaunchCfg lc;
    if (warmup == 0 && count > 0 && chain_cfg_for(s, lc, a.n_streams)) {
        const uint32_t G = lc.threads / 32u;
        const size_t smem = wn::chain_smem_bytes(s->smem_base, s->n_max, G, s->r_max);
        switch (dt) {
        case WN_F32: e = wn::launch_chain_f32(a, s->n_max, G, smem, cs); break;
        case WN_BF16: e = wn::launch_chain_bf16(a, s->n_max, G, smem, cs); break;
        case WN_F16: e = wn::launch_chain_f16(a, s->n_max, G, smem, cs); break;
        default: return fail(WN_EINVAL, "unknown dtype");
        }
        if (e != cudaSuccess) return cuda_fail("generate launch (chain mode)", e);
        return WN_OK;
    }
    if (warmup == 0 && count > 0 && latency_cfg_for(s, lc, a.n_streams)) {
        // the two-control-warp kernel up to two passes per block, the emitter
        // kernel (wn_emit.cuh) above (see launch_persist_latency)
        const bool emit = s->r_max >= 3;
        const size_t smem = emit ? wn::emit_smem_bytes(s->smem_base, s->n_max, s->r_max)
                                 : wn::gen_smem_bytes(s->smem_base, s->n_max, s->r_max);
        const bool full = s->uniform_N && (uint64_t)lc.threads * lc.qt == s->n_max / 4;
        switch (dt) {
        case WN_F32: e = emit ? wn::launch_emit_f32(a, lc, full, smem, cs) : wn::launch_latency_f32(a, lc, full, smem, cs); break;
        case WN_BF16:
            e = emit ? wn::launch_emit_bf16(a, lc, full, smem, cs) : wn::launch_latency_bf16(a, lc, full, smem, cs);
            break;
        case WN_F16: e = emit ? wn::launch_emit_f16(a, lc, full, smem, cs) : wn::launch_latency_f16(a, lc, full, smem, cs); break;
        default: return fail(WN_EINVAL, "unknown dtype");
        }
        if (e != cudaSuccess) return cuda_fail("generate launch (latency mode)", e);
        return WN_OK;
    }
    LaunchCfg c = s->has_cfg && s->cfg.grp != 2 ? s->cfg : default_cfg(s);
    if (c.grp == 1 && warmup == 0 && group_eligible(s)) {
        const uint32_t G = c.threads / 32u;
        switch (dt) {
        case WN_F32: e = wn::launch_group_f32(a, s->n_max, G, s->sms, cs, &s->group_ctas); break;
        case WN_BF16: e = wn::launch_group_bf16(a, s->n_max, G, s->sms, cs, &s->group_ctas); break;
        case WN_F16: e = wn::launch_group_f16(a, s->n_max, G, s->sms, cs, &s->group_ctas); break;
        default: return fail(WN_EINVAL, "unknown dtype");
        }
        if (e != cudaSuccess) return cuda_fail("generate launch (group mode)", e);
        return WN_OK;
    }
    if (c.grp) c = pick_cfg(s->n_max);  // warm-up blocks run in the ordinary kernel
    const size_t smem = cfg_smem(s, c, s->n_max, s->r_max);
    // every stream's quadruples exactly fill the CTA: no per-quadruple checks
    const bool full = s->uniform_N && (uint64_t)c.threads * c.qt == s->n_max / 4;
    switch (dt) {
    case WN_F32: e = wn::launch_generate_f32(a, c, full, s->var, smem, cs); break;
    case WN_BF16: e = wn::launch_generate_bf16(a, c, full, s->var, smem, cs); break;
    case WN_F16: e = wn::launch_generate_f16(a, c, full, s->var, smem, cs); break;
    default: return fail(WN_EINVAL, "unknown dtype");
    }
    if (e != cudaSuccess) return cuda_fail("generate launch", e);
    return WN_OK;
}

// Host mirror of each stream's position within its current block after
// `count` more values (the device state advances the same way).
void advance_k(wn_stream *s, uint64_t count)
{
    for (uint32_t i = 0; i < s->n; ++i) {
        const uint64_t per = s->N[i] - 1, left = per - s->k_host[i];
        if (count <= left) {
            s->k_host[i] += (uint32_t)count;
        } else {
            const uint64_t tail = (count - left) % per;
            s->k_host[i] = tail == 0 ? (uint32_t)per : (uint32_t)tail;
        }
    }
}

// The same for stream i alone.
void advance_k_one(wn_stream *s, uint32_t i, uint64_t count)
{
    const uint64_t per = s->N[i] - 1, left = per - s->k_host[i];
    if (count <= left) {
        s->k_host[i] += (uint32_t)count;
    } else {
        const uint64_t tail = (count - left) % per;
        s->k_host[i] = tail == 0 ? (uint32_t)per : (uint32_t)tail;
    }
}

// One pool-size group of a batch: its streams occupy order[start, start+len).
struct Group {
    uint32_t N = 0, r_max = 0, start = 0, len = 0;
    bool exclusive = false;  // long serial chains: one CTA per SM, lowest-latency shape
};

// The lowest-latency shape for a lone stream (8 quadruples per thread,
// measured on single streams of pools 1024..16384); small pools keep the
// default.
LaunchCfg latency_cfg(uint32_t N)
{
    const uint32_t nq = N / 4;
    if (nq < 256) return pick_cfg(N);
    const LaunchCfg c{8, nq / 8 + 32 <= 160 ? 160 : 544, nq / 8};
    return cfg_ok(c, N) ? c : pick_cfg(N);
}

// Groups streams by pool size and orders each group longest first (cost
// counts[i] (R_i + 1): a block costs R passes plus its stores).  A stream is
// a serial chain of blocks, so a request whose chain alone outlasts the
// whole batch's throughput time -- estimated passes x a per-pass latency of
// about 400 + N/20 ns against 0.34 ps per value-pass over the machine --
// would set the batch's length; up to a third of the SMs' worth of such
// requests (longest first) get exclusive groups instead: one CTA per SM with
// the lowest-latency shape, so that no other CTA shares their SM.  crit_k >= 0
// (after wn_autotune_batch: s->batch_crit) fixes how many of the longest
// chains get them instead of the estimate's threshold.
std::vector<Group> plan_batch(const wn_stream *s, const uint64_t *counts, std::vector<uint32_t> &order, int crit_k)
{
    std::vector<double> chain(s->n);
    double thr = 0.0;
    for (uint32_t i = 0; i < s->n; ++i) {
        const double N = s->N[i];
        chain[i] = std::ceil((double)counts[i] / (N - 1.0)) * s->R[i] * (400.0 + N / 20.0) * 1e-9;
        thr += (double)counts[i] * (s->R[i] + 0.5) * (N >= 16384 ? 1.3 : 1.0) * 0.34e-12;
    }
    std::vector<uint32_t> by_chain(s->n);
    for (uint32_t i = 0; i < s->n; ++i) by_chain[i] = i;
    std::sort(by_chain.begin(), by_chain.end(),
              [&](uint32_t x, uint32_t y) { return chain[x] != chain[y] ? chain[x] > chain[y] : x < y; });
    std::vector<char> crit(s->n, 0);
    std::map<uint32_t, std::vector<uint32_t>> by_n, crit_n;
    for (uint32_t i = 0; i < s->n; ++i) by_n[s->N[i]];
    const uint32_t max_crit = crit_k >= 0 ? (uint32_t)crit_k : (uint32_t)std::max(1, s->sms / 3);
    for (uint32_t k = 0; k < s->n && k < max_crit; ++k) {
        const uint32_t i = by_chain[k];
        if ((crit_k < 0 && !(chain[i] > thr)) || counts[i] == 0) break;
        if (by_n.size() + crit_n.size() + (crit_n.count(s->N[i]) ? 0 : 1) > 16) break;  // one claim counter each
        crit[i] = 1;
        crit_n[s->N[i]].push_back(i);
    }
    for (uint32_t i = 0; i < s->n; ++i)
        if (!crit[i]) by_n[s->N[i]].push_back(i);
    std::vector<Group> groups;
    order.clear();
    for (auto &kv : crit_n) {
        Group g;
        g.N = kv.first;
        g.exclusive = true;
        g.start = (uint32_t)order.size();
        g.len = (uint32_t)kv.second.size();
        for (uint32_t i : kv.second) g.r_max = std::max(g.r_max, s->R[i]);
        order.insert(order.end(), kv.second.begin(), kv.second.end());
        groups.push_back(g);
    }
    for (auto &kv : by_n) {
        if (kv.second.empty()) continue;
        auto &v = kv.second;
        std::stable_sort(v.begin(), v.end(), [&](uint32_t x, uint32_t y) {
            return counts[x] * (s->R[x] + 1ull) > counts[y] * (s->R[y] + 1ull);
        });
        Group g;
        g.N = kv.first;
        g.start = (uint32_t)order.size();
        g.len = (uint32_t)v.size();
        for (uint32_t i : v) g.r_max = std::max(g.r_max, s->R[i]);
        order.insert(order.end(), v.begin(), v.end());
        groups.push_back(g);
    }
    return groups;
}

// Byte layout of a BatchDesc for n streams: counts, offsets, order, counters.
constexpr size_t desc_counters(size_t n) { return (20 * n + 15) / 16 * 16; }

wn_status alloc_desc(wn_stream *s, BatchDesc &d)
{
    if (d.base) return WN_OK;
    const size_t n = s->n;
    WN_CU(cudaMalloc(&d.base, desc_counters(n) + 16 * sizeof(uint32_t)));
    d.counts = reinterpret_cast<uint64_t *>(d.base);
    d.offsets = reinterpret_cast<uint64_t *>(d.base + 8 * n);
    d.order = reinterpret_cast<uint32_t *>(d.base + 16 * n);
    d.queue = reinterpret_cast<uint32_t *>(d.base + desc_counters(n));
    return WN_OK;
}

// Uploads counts, offsets and the claim order into d with one copy from a
// pageable host buffer of the library's own: a copy from pageable memory has
// consumed its source when it returns, so the caller may reuse or free its
// arrays as soon as the call returns, whether they are page-locked or not.
wn_status upload_desc(wn_stream *s, const BatchDesc &d, const uint64_t *counts, const uint64_t *offsets,
                      const std::vector<uint32_t> &order, cudaStream_t cs)
{
    const size_t n = s->n;
    std::vector<unsigned char> host(20 * n);
    std::memcpy(host.data(), counts, 8 * n);
    std::memcpy(host.data() + 8 * n, offsets, 8 * n);
    std::memcpy(host.data() + 16 * n, order.data(), 4 * n);
    WN_CU(cudaMemcpyAsync(d.base, host.data(), host.size(), cudaMemcpyHostToDevice, cs));
    return WN_OK;
}

wn_status ensure_batch_buffers(wn_stream *s, size_t n_groups)
{
    wn_status st = alloc_desc(s, s->bd_eager);
    if (st == WN_OK) st = alloc_desc(s, s->bd_graph);
    if (st != WN_OK) return st;
    if (!s->fork) WN_CU(cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming));
    while (s->branch.size() < n_groups) {
        cudaStream_t b, bh;
        cudaEvent_t j;
        int least = 0, greatest = 0;
        WN_CU(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        WN_CU(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking));
        WN_CU(cudaStreamCreateWithPriority(&bh, cudaStreamNonBlocking, greatest));
        WN_CU(cudaEventCreateWithFlags(&j, cudaEventDisableTiming));
        s->branch.push_back(b);
        s->branch_hi.push_back(bh);
        s->join.push_back(j);
    }
    return WN_OK;
}

// Batch groups of one pool size can run the group mode whenever the handle
// runs the plain method (mixed pool sizes are split into groups anyway).
bool batch_group_ok(const wn_stream *s) { return !s->var && s->smem_base == wn::kGroupBase; }

// The shape a batch group of pool N runs with: the tuner's pick, else the
// group mode's default for N, else the ordinary kernel's.
LaunchCfg batch_cfg(const wn_stream *s, uint32_t N)
{
    auto it = s->group_cfg.find(N);
    if (it != s->group_cfg.end()) return it->second;
    uint32_t G = 0;
    if (batch_group_ok(s) && group_default(N, G) && group_shape_ok(N, G)) return group_cfg_of(N, G);
    return pick_cfg(N);
}

// One persistent launch of a batch group of pool N with shape c (ordinary or
// group mode; smem: the ordinary kernel's shared memory).
cudaError_t launch_persist_cfg(const wn_stream *s, const wn::GenArgs &a, const wn::BatchArgs &bq, const LaunchCfg &c,
                               uint32_t N, wn_dtype dt, size_t smem, cudaStream_t cs)
{
    if (c.grp) {
        const uint32_t G = c.threads / 32u;
        switch (dt) {
        case WN_F32: return wn::launch_persist_group_f32(a, bq, N, G, s->sms, cs);
        case WN_BF16: return wn::launch_persist_group_bf16(a, bq, N, G, s->sms, cs);
        default: return wn::launch_persist_group_f16(a, bq, N, G, s->sms, cs);
        }
    }
    const bool full = (uint64_t)c.threads * c.qt == N / 4;
    switch (dt) {
    case WN_F32: return wn::launch_persist_f32(a, bq, c, full, s->var, smem, s->sms, cs);
    case WN_BF16: return wn::launch_persist_bf16(a, bq, c, full, s->var, smem, s->sms, cs);
    default: return wn::launch_persist_f16(a, bq, c, full, s->var, smem, s->sms, cs);
    }
}

// Shared memory of a chain group's CTA (need: the kernel's own): padded so
// that at most s->batch_density of them share an SM (1: a whole SM each).
size_t chain_smem(const wn_stream *s, size_t need)
{
    size_t pad = (size_t)s->smem_optin;
    if (s->batch_density > 1 && s->sm_smem > 0)
        pad = ((size_t)s->sm_smem / (size_t)s->batch_density - (size_t)s->smem_reserved) / 128 * 128;
    return std::min(std::max(need, pad), (size_t)s->smem_optin);
}

// One persistent latency-mode launch over a batch group of pool N.  A chain
// group (chain: padded to batch_density CTAs per SM) with more than two
// passes per block runs the emitter kernel (wn_emit.cuh; lone streams of
// pool 1024: 700 ns per block at R = 4 against 790), everything else the
// two-control-warp kernel (565 / 574 ns at R = 1 / 2 against 594 / 625),
// which also holds more CTAs per SM: the emitter kernel is built for one CTA
// per SM (its registers), too few for a group of many streams.
cudaError_t launch_persist_latency(const wn_stream *s, const wn::GenArgs &a, const wn::BatchArgs &bq,
                                   const LaunchCfg &lc, uint32_t N, uint32_t r_max, bool chain, wn_dtype dt,
                                   cudaStream_t cs)
{
    const bool lfull = (uint64_t)lc.threads * lc.qt == N / 4;
    const bool emit = chain && r_max >= 3;
    size_t smem = emit ? wn::emit_smem_bytes(s->smem_base, N, r_max) : wn::gen_smem_bytes(s->smem_base, N, r_max);
    if (chain) smem = chain_smem(s, smem);
    if (emit) {
        switch (dt) {
        case WN_F32: return wn::launch_persist_emit_f32(a, bq, lc, lfull, smem, s->sms, cs);
        case WN_BF16: return wn::launch_persist_emit_bf16(a, bq, lc, lfull, smem, s->sms, cs);
        default: return wn::launch_persist_emit_f16(a, bq, lc, lfull, smem, s->sms, cs);
        }
    }
    switch (dt) {
    case WN_F32: return wn::launch_persist_lat_f32(a, bq, lc, lfull, smem, s->sms, cs);
    case WN_BF16: return wn::launch_persist_lat_bf16(a, bq, lc, lfull, smem, s->sms, cs);
    default: return wn::launch_persist_lat_f16(a, bq, lc, lfull, smem, s->sms, cs);
    }
}

// Enqueues a batch whose descriptors are already on the device (in d): reset
// the claim counters, fork one branch per group, launch each group's
// persistent kernel, join.
wn_status enqueue_batch(wn_stream *s, const std::vector<Group> &groups, void *out, wn_dtype dt, cudaStream_t cs,
                        const BatchDesc &d)
{
    WN_CU(cudaMemsetAsync(d.queue, 0, sizeof(uint32_t) * 16, cs));
    WN_CU(cudaEventRecord(s->fork, cs));
    // chain groups in the chain mode (when chosen) first
    std::vector<char> chain_mode(groups.size(), 0);
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        uint32_t cg = 0;
        chain_mode[gi] = s->batch_chain_mode && groups[gi].exclusive && chain_default(groups[gi].N, cg) &&
                         chain_fits(s, groups[gi].N, cg);
    }
    for (int pass = 0; pass < 2; ++pass)
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        if ((pass == 0) != (chain_mode[gi] != 0)) continue;
        const Group &g = groups[gi];
        cudaStream_t b = g.exclusive ? s->branch_hi[gi] : s->branch[gi];
        WN_CU(cudaStreamWaitEvent(b, s->fork, 0));
        wn::GenArgs a;
        a.hdr = s->d_hdr;
        a.pools = s->d_pools;
        a.out = out;
        a.count = 0;
        a.out_stride = 0;
        a.n_streams = g.len;
        a.n_max = g.N;
        a.r_max = g.r_max;
        a.warmup_blocks = 0;
        wn::BatchArgs bq;
        bq.order = d.order + g.start;
        bq.offsets = d.offsets;
        bq.counts = d.counts;
        bq.n_items = g.len;
        bq.queue = d.queue + gi;
        size_t smem = wn::gen_smem_bytes(s->smem_base, g.N, g.r_max);
        if (g.exclusive) smem = chain_smem(s, smem);  // at most batch_density chain CTAs per SM
        cudaError_t e;
        LaunchCfg lc;
        const auto tuned = s->group_lat.find(g.N);
        // untuned groups take the latency mode only where the group mode cannot run
        const bool want_lat = g.exclusive ? s->batch_lat >= 1
                                          : (tuned != s->group_lat.end() ? tuned->second
                                                                         : s->batch_lat >= 2 && !batch_cfg(s, g.N).grp);
        uint32_t cg = 0;
        if (chain_mode[gi] && chain_default(g.N, cg)) {
            // the longest chains: the chain mode, at most batch_density CTAs per SM
            const size_t csm = chain_smem(s, wn::chain_smem_bytes(s->smem_base, g.N, cg, g.r_max));
            switch (dt) {
            case WN_F32: e = wn::launch_persist_chain_f32(a, bq, g.N, cg, csm, s->sms, b); break;
            case WN_BF16: e = wn::launch_persist_chain_bf16(a, bq, g.N, cg, csm, s->sms, b); break;
            default: e = wn::launch_persist_chain_f16(a, bq, g.N, cg, csm, s->sms, b); break;
            }
            if (e != cudaSuccess) return cuda_fail("wn_generate_batch: launch (chain mode)", e);
            WN_CU(cudaEventRecord(s->join[gi], b));
            WN_CU(cudaStreamWaitEvent(cs, s->join[gi], 0));
            continue;
        }
        if (!s->var && want_lat && latency_default(g.N, lc)) {
            e = launch_persist_latency(s, a, bq, lc, g.N, g.r_max, g.exclusive, dt, b);
            if (e != cudaSuccess) return cuda_fail("wn_generate_batch: launch", e);
            WN_CU(cudaEventRecord(s->join[gi], b));
            WN_CU(cudaStreamWaitEvent(cs, s->join[gi], 0));
            continue;
        }
        const LaunchCfg c = g.exclusive ? latency_cfg(g.N) : batch_cfg(s, g.N);
        if (!g.exclusive && !c.grp) smem = cfg_smem(s, c, g.N, g.r_max);
        e = launch_persist_cfg(s, a, bq, c, g.N, dt, smem, b);
        if (e != cudaSuccess) return cuda_fail("wn_generate_batch: launch", e);
        WN_CU(cudaEventRecord(s->join[gi], b));
        WN_CU(cudaStreamWaitEvent(cs, s->join[gi], 0));
    }
    return WN_OK;
}

wn_status check_batch_args(const wn_stream *s, const void *out, const uint64_t *counts, const uint64_t *offsets,
                           wn_dtype dtype)
{
    if (!s) return fail(WN_EINVAL, "wn_generate_batch: NULL handle");
    if (dtype != WN_F32 && dtype != WN_BF16 && dtype != WN_F16) return fail(WN_EINVAL, "wn_generate_batch: unknown dtype");
    if (!counts || !offsets) return fail(WN_EINVAL, "wn_generate_batch: NULL counts or offsets");
    if (!out || reinterpret_cast<uintptr_t>(out) % 16 != 0)
        return fail(WN_EINVAL, "wn_generate_batch: output NULL or not 16-byte aligned");
    return WN_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Scratch for wn_generate_batch_noalloc: a fixed device array instead of
// memory the library allocates.  Layout: 16 claim counters (one per pool-size
// group) in the first 256 bytes, then the claim order (uint32), the output
// offsets and the counts (uint64) of up to WN_NOALLOC_MAX_STREAMS streams.
// Every call shares it.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kNaCounters = 0;
constexpr size_t kNaOrder = 256;
constexpr size_t kNaOffsets = kNaOrder + 4 * (size_t)WN_NOALLOC_MAX_STREAMS;
constexpr size_t kNaCounts = kNaOffsets + 8 * (size_t)WN_NOALLOC_MAX_STREAMS;
constexpr size_t kNaBytes = kNaCounts + 8 * (size_t)WN_NOALLOC_MAX_STREAMS;
}  // namespace

static __device__ __align__(256) unsigned char wn_noalloc_scratch[kNaBytes];

namespace {
// Device address of wn_noalloc_scratch on each device, looked up once per
// device (with that device current) on the first call there.  In host code
// the array's name is only a host-side stand-in, never a device address.
std::mutex g_na_mu;
unsigned char *g_na_ptr[128] = {};
// host-side claim order of the call in progress (static storage: nothing is
// allocated per call); calls are serialised on g_na_plan_mu
std::mutex g_na_plan_mu;
uint32_t g_na_order[WN_NOALLOC_MAX_STREAMS];

wn_status noalloc_scratch(int dev, unsigned char **ptr)
{
    if (dev < 0 || dev >= 128) return fail(WN_EINVAL, "wn_generate_batch_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, wn_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail("wn_generate_batch_noalloc: cudaGetSymbolAddress", e);
        g_na_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *ptr = g_na_ptr[dev];
    return WN_OK;
}
}  // namespace

extern "C" void wn_destroy(wn_stream *s);

// A handle for n streams of the given pool sizes and pass counts: validates
// them, allocates headers and pools (contents unset), probes where dynamic
// shared memory starts and checks that the generate kernel's layout fits.
// NULL (with the error recorded under `who`) on failure.
wn_stream *alloc_handle(uint32_t n_streams, const uint32_t *pool_N, const uint32_t *passes_R, cudaStream_t cs,
                        const char *who)
{
    const std::string w(who);
    for (uint32_t i = 0; i < n_streams; ++i)
        if (!valid_pool(pool_N[i]) || !valid_passes(passes_R[i])) {
            fail(WN_EINVAL, w + ": stream " + std::to_string(i) +
                                ": pool_N must be a power of two in [4, 16384] and passes_R in [1, 64]");
            return nullptr;
        }
    wn_stream *s = new wn_stream();
    s->n = n_streams;
    s->N.assign(pool_N, pool_N + n_streams);
    s->R.assign(passes_R, passes_R + n_streams);
    s->k_host.resize(n_streams);
    uint64_t off = 0;
    for (uint32_t i = 0; i < n_streams; ++i) {
        s->k_host[i] = pool_N[i] - 1;
        off += pool_N[i];
        s->n_max = std::max(s->n_max, pool_N[i]);
        if (pool_N[i] != pool_N[0]) s->uniform_N = false;
        s->r_max = std::max(s->r_max, passes_R[i]);
    }
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&s->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, s->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&s->smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, s->device);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_hdr, sizeof(wn::StreamHdr) * n_streams);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_pools, sizeof(float) * off);
    if (e != cudaSuccess) {
        cuda_fail((w + ": allocation").c_str(), e);
        wn_destroy(s);
        return nullptr;
    }
    {
        // where dynamic shared memory starts in a CTA's shared window: the
        // generate kernel places its pool buffers at multiples of their size
        uint32_t *d_base = nullptr;
        e = cudaMalloc(&d_base, sizeof(uint32_t));
        if (e == cudaSuccess) {
            wn::smem_base_kernel<<<1, 32, 16, cs>>>(d_base);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&s->smem_base, d_base, sizeof(uint32_t), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (d_base) cudaFree(d_base);
        if (e != cudaSuccess) {
            cuda_fail((w + ": shared-memory probe").c_str(), e);
            wn_destroy(s);
            return nullptr;
        }
    }
    if (wn::gen_smem_bytes(s->smem_base, s->n_max, s->r_max) > 227u * 1024u) {
        fail(WN_EINVAL, w + ": pool and pass counts need more shared memory than a CTA has");
        wn_destroy(s);
        return nullptr;
    }
    return s;
}

extern "C" {

const char *wn_last_error(void) { return g_err.c_str(); }

wn_stream *wn_create_ex(uint32_t n_streams, const uint32_t *pool_N, const uint32_t *passes_R,
                        const uint64_t *seeds, uint32_t warmup_blocks, const wn_options *opt, void *cuda_stream)
{
    g_err.clear();
    if (n_streams == 0 || !pool_N || !passes_R || !seeds) {
        fail(WN_EINVAL, "wn_create_streams: empty stream set or NULL array");
        return nullptr;
    }
    uint32_t variant = wn::VAR_CHI2_C;
    if (opt) {
        if (opt->chi2 > WN_CHI2_C || opt->reserve > WN_RESERVE_CURRENT || opt->decimate < 1 || opt->decimate > 255 ||
            opt->update > WN_UPDATE_ROTATION) {
            fail(WN_EINVAL, "wn_create_ex: options out of range (chi2 0..3, reserve 0..1, decimate 1..255, update 0..1)");
            return nullptr;
        }
        variant = opt->chi2 | (opt->reserve ? wn::VAR_RESERVE_CURRENT : 0u) |
                  (opt->update ? wn::VAR_ROTATION : 0u) | (opt->decimate << 8);
    }
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(cuda_stream);
    wn_stream *s = alloc_handle(n_streams, pool_N, passes_R, cs, "wn_create_streams");
    if (!s) return nullptr;
    s->var = (variant != wn::VAR_CHI2_C);
    std::vector<wn::StreamHdr> h(n_streams);
    uint64_t off = 0;
    for (uint32_t i = 0; i < n_streams; ++i) {
        std::memset(&h[i], 0, sizeof(h[i]));
        h[i].x = seeds[i];  // consumed by the init kernel
        h[i].N = pool_N[i];
        h[i].R = passes_R[i];
        h[i].variant = variant;
        h[i].pool_off = off;
        off += pool_N[i];
    }
    cudaError_t e;
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
    LaunchCfg c;
    if (cached_gen_cfg(s, WN_F32, c)) {  // a shape wn_autotune chose for this workload before
        s->cfg = c;
        s->has_cfg = true;
    }
    return s;
}

namespace {
constexpr char kSaveMagic[8] = {'W', 'N', 'S', 'T', 'A', 'T', 'E', '1'};

uint64_t fnv1a64(const unsigned char *p, size_t n)
{
    uint64_t h = 0xcbf29ce484222325ull;
    for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 0x100000001b3ull;
    return h;
}
}  // namespace

wn_status wn_save(const wn_stream *s, void *host_buf, uint64_t buf_bytes, uint64_t *bytes_needed)
{
    if (!s) return fail(WN_EINVAL, "wn_save: NULL handle");
    uint64_t pool_elems = 0;
    for (uint32_t i = 0; i < s->n; ++i) pool_elems += s->N[i];
    const uint64_t need = 16 + (uint64_t)sizeof(wn::StreamHdr) * s->n + 4 * pool_elems + 8;
    if (bytes_needed) *bytes_needed = need;
    if (!host_buf) return WN_OK;
    if (buf_bytes < need) return fail(WN_EINVAL, "wn_save: buffer holds " + std::to_string(buf_bytes) +
                                                     " bytes, the state needs " + std::to_string(need));
    unsigned char *b = static_cast<unsigned char *>(host_buf);
    std::memcpy(b, kSaveMagic, 8);
    const uint32_t n = s->n, hb = (uint32_t)sizeof(wn::StreamHdr);
    std::memcpy(b + 8, &n, 4);
    std::memcpy(b + 12, &hb, 4);
    // every call enqueued before, on whichever CUDA stream (calls take their
    // own streams, and wn_generate_host copies on a second one), has finished
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e == cudaSuccess && cur != s->device) e = cudaSetDevice(s->device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(b + 16, s->d_hdr, (size_t)hb * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(b + 16 + (size_t)hb * n, s->d_pools, 4 * pool_elems, cudaMemcpyDeviceToHost);
    if (cur >= 0 && cur != s->device) cudaSetDevice(cur);  // the caller's device stays current
    if (e != cudaSuccess) return cuda_fail("wn_save: copy", e);
    wn::StreamHdr *h = reinterpret_cast<wn::StreamHdr *>(b + 16);
    for (uint32_t i = 0; i < n; ++i) {
        if (h[i].flags != 0) return fail(WN_EINVAL, "wn_save: stream " + std::to_string(i) + " carries an error flag");
        h[i].pool_off = 0;  // assigned again on load
    }
    const uint64_t sum = fnv1a64(b, need - 8);
    std::memcpy(b + need - 8, &sum, 8);
    return WN_OK;
}

wn_stream *wn_load(const void *host_buf, uint64_t buf_bytes, void *cuda_stream)
{
    g_err.clear();
    const unsigned char *b = static_cast<const unsigned char *>(host_buf);
    if (!b || buf_bytes < 16 + 8) {
        fail(WN_EINVAL, "wn_load: NULL or short buffer");
        return nullptr;
    }
    if (std::memcmp(b, kSaveMagic, 8) != 0) {
        fail(WN_EINVAL, "wn_load: not a saved state (magic)");
        return nullptr;
    }
    uint32_t n = 0, hb = 0;
    std::memcpy(&n, b + 8, 4);
    std::memcpy(&hb, b + 12, 4);
    if (hb != sizeof(wn::StreamHdr) || n == 0 || (uint64_t)n * hb + 24 > buf_bytes) {
        fail(WN_EINVAL, "wn_load: bad header (stream count or header size)");
        return nullptr;
    }
    std::vector<wn::StreamHdr> h(n);
    std::memcpy(h.data(), b + 16, (size_t)hb * n);
    uint64_t pool_elems = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const wn::StreamHdr &x = h[i];
        if (!valid_pool(x.N) || !valid_passes(x.R) || x.k > x.N - 1 || x.x == 0 || x.flags != 0 ||
            !wn::var_valid(x.variant)) {
            fail(WN_EINVAL, "wn_load: stream " + std::to_string(i) + " has an invalid pool size, pass count, "
                            "position or generator word");
            return nullptr;
        }
        pool_elems += x.N;
    }
    const uint64_t need = 16 + (uint64_t)hb * n + 4 * pool_elems + 8;
    if (buf_bytes != need) {
        fail(WN_EINVAL, "wn_load: buffer holds " + std::to_string(buf_bytes) + " bytes, the state it describes " +
                            std::to_string(need));
        return nullptr;
    }
    uint64_t sum = 0;
    std::memcpy(&sum, b + need - 8, 8);
    if (sum != fnv1a64(b, need - 8)) {
        fail(WN_EINVAL, "wn_load: checksum mismatch");
        return nullptr;
    }
    const float *pools = reinterpret_cast<const float *>(b + 16 + (size_t)hb * n);
    for (uint64_t i = 0; i < pool_elems; ++i)
        if (!std::isfinite(pools[i])) {
            fail(WN_EINVAL, "wn_load: non-finite pool value");
            return nullptr;
        }
    std::vector<uint32_t> N(n), R(n);
    for (uint32_t i = 0; i < n; ++i) {
        N[i] = h[i].N;
        R[i] = h[i].R;
    }
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(cuda_stream);
    wn_stream *s = alloc_handle(n, N.data(), R.data(), cs, "wn_load");
    if (!s) return nullptr;
    for (uint32_t i = 0; i < n; ++i) s->var = s->var || h[i].variant != wn::VAR_CHI2_C;
    uint64_t off = 0;
    for (uint32_t i = 0; i < n; ++i) {
        h[i].pool_off = off;
        off += N[i];
        s->k_host[i] = h[i].k;
    }
    cudaError_t e = cudaMemcpyAsync(s->d_hdr, h.data(), sizeof(wn::StreamHdr) * n, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_pools, pools, 4 * pool_elems, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        cuda_fail("wn_load: copy", e);
        wn_destroy(s);
        return nullptr;
    }
    return s;
}

wn_stream *wn_create_streams(uint32_t n_streams, const uint32_t *pool_N, const uint32_t *passes_R,
                             const uint64_t *seeds, uint32_t warmup_blocks, void *cuda_stream)
{
    return wn_create_ex(n_streams, pool_N, passes_R, seeds, warmup_blocks, nullptr, cuda_stream);
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
    if (s->bd_eager.base) cudaFree(s->bd_eager.base);
    if (s->bd_graph.base) cudaFree(s->bd_graph.base);
    for (auto b : s->branch) cudaStreamDestroy(b);
    for (auto b : s->branch_hi) cudaStreamDestroy(b);
    for (auto j : s->join) cudaEventDestroy(j);
    if (s->fork) cudaEventDestroy(s->fork);
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    delete s;
}

wn_status wn_set_config_ex(wn_stream *s, uint32_t quads_per_thread, uint32_t threads, uint32_t flags)
{
    if (!s) return fail(WN_EINVAL, "wn_set_config: NULL handle");
    if (flags & ~(uint32_t)(WN_CFG_IN_PLACE | WN_CFG_GROUP | WN_CFG_CHAIN))
        return fail(WN_EINVAL, "wn_set_config_ex: unknown flags");
    if (quads_per_thread == 0 && threads == 0) {
        s->has_cfg = false;
        return WN_OK;
    }
    if (flags & WN_CFG_CHAIN) {
        const uint32_t G = threads / 32u;
        if ((flags & (WN_CFG_GROUP | WN_CFG_IN_PLACE)) || threads % 32u != 0 || G == 0 ||
            !chain_shape_ok(s->n_max, G) || (uint64_t)128u * quads_per_thread * G != s->n_max)
            return fail(WN_EINVAL, "wn_set_config_ex: no compiled chain-mode shape with " +
                                       std::to_string(quads_per_thread) + " quadruples per lane and " +
                                       std::to_string(threads) + " compute threads covers pool " +
                                       std::to_string(s->n_max));
        if (s->var || !s->uniform_N || !chain_fits(s, s->n_max, G))
            return fail(WN_EINVAL, "wn_set_config_ex: the chain mode needs one pool size, the plain method and "
                                   "room for two pool buffers in one CTA's shared memory");
        s->cfg = chain_cfg_of(s->n_max, G);
        s->has_cfg = true;
        return WN_OK;
    }
    if (flags & WN_CFG_GROUP) {
        const uint32_t G = threads / 32u;
        if (threads % 32u != 0 || G == 0 || !group_shape_ok(s->n_max, G) ||
            (uint64_t)128u * quads_per_thread * G != s->n_max)
            return fail(WN_EINVAL, "wn_set_config_ex: no compiled group-mode shape with " +
                                       std::to_string(quads_per_thread) + " quadruples per lane and " +
                                       std::to_string(threads) + " threads covers pool " + std::to_string(s->n_max));
        if (!group_eligible(s))
            return fail(WN_EINVAL, "wn_set_config_ex: group mode needs one pool size, the plain method and "
                                   "dynamic shared memory at its expected window address");
        s->cfg = group_cfg_of(s->n_max, G);
        s->has_cfg = true;
        return WN_OK;
    }
    // the instantiation of the asked layout with the smallest thread bound
    // that admits `threads`
    const int ip = (flags & WN_CFG_IN_PLACE) ? 1 : 0;
    LaunchCfg best{0, 0, threads};
    for (const auto &k : wn::kShapes) {
        LaunchCfg c{k[0], k[1], threads, k[3]};
        if (k[0] == (int)quads_per_thread && k[3] == ip && cfg_ok(c, s->n_max) && (best.qt == 0 || k[1] < best.maxt))
            best = c;
    }
    if (best.qt == 0)
        return fail(WN_EINVAL, "wn_set_config: no compiled configuration with " + std::to_string(quads_per_thread) +
                                   " quadruples per thread and " + std::to_string(threads) + " threads" +
                                   (ip ? " (in-place layout)" : "") + " covers pool " + std::to_string(s->n_max));
    s->cfg = best;
    s->has_cfg = true;
    return WN_OK;
}

wn_status wn_set_config(wn_stream *s, uint32_t quads_per_thread, uint32_t threads)
{
    return wn_set_config_ex(s, quads_per_thread, threads, 0);
}

wn_status wn_autotune(wn_stream *s, uint64_t count, wn_dtype dtype, void *cuda_stream, uint32_t *quads_per_thread,
                      uint32_t *threads)
{
    if (!s) return fail(WN_EINVAL, "wn_autotune: NULL handle");
    if (count == 0) return fail(WN_EINVAL, "wn_autotune: count must be positive");
    if (dtype != WN_F32 && dtype != WN_BF16 && dtype != WN_F16) return fail(WN_EINVAL, "wn_autotune: unknown dtype");
    using Key = std::tuple<uint32_t, uint32_t, uint32_t, bool, int, uint64_t, int>;
    static std::map<Key, LaunchCfg> cache;
    static std::mutex mu;
    const Key key{s->n, s->n_max, s->r_max, s->uniform_N, (int)dtype, count, s->device};
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            s->cfg = it->second;
            s->has_cfg = true;
            if (quads_per_thread) *quads_per_thread = (uint32_t)s->cfg.qt;
            if (threads) *threads = s->cfg.threads;
            return WN_OK;
        }
    }
    {
        LaunchCfg c;
        if (cached_gen_cfg(s, dtype, c)) {  // chosen for this workload by an earlier process
            s->cfg = c;
            s->has_cfg = true;
            if (quads_per_thread) *quads_per_thread = (uint32_t)c.qt;
            if (threads) *threads = c.threads;
            return WN_OK;
        }
    }
    // candidate shapes: every compiled one whose compute threads cover the
    // largest pool with at most twice the needed quadruple slots
    std::vector<LaunchCfg> cand;
    const uint32_t nq = s->n_max / 4;
    for (const auto &k : wn::kShapes)
        for (uint32_t t = 32; t + 32 <= (uint32_t)k[1]; t += 32) {
            LaunchCfg c{k[0], k[1], t, k[3]};
            const uint64_t slots = (uint64_t)t * k[0];
            if (cfg_ok(c, s->n_max) && slots < 2ull * nq + 32ull * k[0]) {
                bool dup = false;  // same (qt, threads, layout) under a larger bound
                for (auto &o : cand)
                    if (o.qt == c.qt && o.threads == c.threads && o.ip == c.ip) dup = true;
                if (!dup) cand.push_back(c);
            }
        }
    if (group_eligible(s))  // the compiled group-mode shapes of this pool size
        for (const auto &k : wn::kGroupShapes)
            if ((uint32_t)k[0] == s->n_max) cand.push_back(group_cfg_of(s->n_max, (uint32_t)k[1]));
    if (s->uniform_N)  // and the chain-mode ones
        for (const auto &k : wn::kChainShapes)
            if ((uint32_t)k[0] == s->n_max && chain_fits(s, s->n_max, (uint32_t)k[1]))
                cand.push_back(chain_cfg_of(s->n_max, (uint32_t)k[1]));
    if (cand.empty()) return fail(WN_EINVAL, "wn_autotune: no compiled shape fits");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(cuda_stream);
    const size_t esize = dtype == WN_F32 ? 4 : 2;
    size_t pool_floats = 0;
    for (uint32_t i = 0; i < s->n; ++i) pool_floats += s->N[i];
    wn::StreamHdr *hdr_bak = nullptr;
    float *pool_bak = nullptr;
    void *tmp = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (hdr_bak) cudaFree(hdr_bak);
        if (pool_bak) cudaFree(pool_bak);
        if (tmp) cudaFree(tmp);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = cudaMalloc(&hdr_bak, sizeof(wn::StreamHdr) * s->n);
    if (e == cudaSuccess) e = cudaMalloc(&pool_bak, sizeof(float) * pool_floats);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, esize * count * s->n);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    auto save = [&](bool to_backup) {
        cudaError_t r = cudaMemcpyAsync(to_backup ? (void *)hdr_bak : (void *)s->d_hdr,
                                        to_backup ? (void *)s->d_hdr : (void *)hdr_bak,
                                        sizeof(wn::StreamHdr) * s->n, cudaMemcpyDeviceToDevice, cs);
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(to_backup ? (void *)pool_bak : (void *)s->d_pools,
                                to_backup ? (void *)s->d_pools : (void *)pool_bak, sizeof(float) * pool_floats,
                                cudaMemcpyDeviceToDevice, cs);
        return r;
    };
    if (e == cudaSuccess) e = save(true);
    const bool had_cfg = s->has_cfg;
    const LaunchCfg old_cfg = s->cfg;
    LaunchCfg best = cand[0];
    float best_ms = 1e30f;
    for (size_t ci = 0; ci < cand.size() && e == cudaSuccess; ++ci) {
        s->cfg = cand[ci];
        s->has_cfg = true;
        float times[3];
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // first run warms up
            e = save(false);
            if (e == cudaSuccess) e = cudaEventRecord(e0, cs);
            if (e == cudaSuccess && launch_generate(s, tmp, count, 0, dtype, cs) != WN_OK) e = cudaErrorLaunchFailure;
            if (e == cudaSuccess) e = cudaEventRecord(e1, cs);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) times[rep - 1] = ms;
        }
        if (e != cudaSuccess) break;
        std::sort(times, times + 3);
        if (times[1] < best_ms) {
            best_ms = times[1];
            best = cand[ci];
        }
    }
    if (e == cudaSuccess) e = save(false);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    cleanup();
    if (e != cudaSuccess) {
        s->cfg = old_cfg;
        s->has_cfg = had_cfg;
        return cuda_fail("wn_autotune", e);
    }
    s->cfg = best;
    s->has_cfg = true;
    {
        std::lock_guard<std::mutex> lock(mu);
        cache[key] = best;
    }
    wn::tune_cache_put(gen_key(s, dtype), cfg_text(best));
    if (quads_per_thread) *quads_per_thread = (uint32_t)best.qt;
    if (threads) *threads = best.threads;
    return WN_OK;
}

wn_status wn_get_config_ex(const wn_stream *s, uint32_t *quads_per_thread, uint32_t *threads, uint32_t *flags)
{
    if (!s) return fail(WN_EINVAL, "wn_get_config: NULL handle");
    LaunchCfg c = s->has_cfg ? s->cfg : default_cfg(s), lc;
    if (chain_cfg_for(s, lc, s->n)) c = lc;           // few streams of one pool size: the chain mode
    else if (latency_cfg_for(s, lc, s->n)) c = lc;  // few streams: the latency mode's shape
    if (quads_per_thread) *quads_per_thread = (uint32_t)c.qt;
    if (threads) *threads = c.threads;
    if (flags)
        *flags = (c.ip ? (uint32_t)WN_CFG_IN_PLACE : 0u) | (c.grp == 1 ? (uint32_t)WN_CFG_GROUP : 0u) |
                 (c.grp == 2 ? (uint32_t)WN_CFG_CHAIN : 0u);
    return WN_OK;
}

wn_status wn_get_config(const wn_stream *s, uint32_t *quads_per_thread, uint32_t *threads)
{
    return wn_get_config_ex(s, quads_per_thread, threads, nullptr);
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
    const wn_status st = launch_generate(s, out, count, 0, dtype, reinterpret_cast<cudaStream_t>(cuda_stream));
    if (st == WN_OK) advance_k(s, count);
    return st;
}

wn_status wn_generate_host(void *host_out, uint64_t count, wn_stream *s, wn_dtype dtype, void *cuda_stream)
{
    if (!s) return fail(WN_EINVAL, "wn_generate_host: NULL handle");
    if (dtype != WN_F32 && dtype != WN_BF16 && dtype != WN_F16) return fail(WN_EINVAL, "wn_generate_host: unknown dtype");
    if (count == 0) return WN_OK;
    if (!host_out) return fail(WN_EINVAL, "wn_generate_host: NULL output");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(cuda_stream);
    const size_t esize = dtype == WN_F32 ? 4 : 2;
    const size_t kStageMax = size_t(256) << 20;
    const uint64_t per_stream = count * esize;
    // streams whose whole request fits one staging buffer (0: not even one)
    const uint64_t group = per_stream <= kStageMax ? kStageMax / per_stream : 0;
    {
        // page-locked host memory that the device can address (every
        // cudaHostAlloc'd or registered buffer under unified addressing): the
        // kernel stores straight into it over the host link -- 181 GB/s for
        // 16 GiB on GB300, against 163 GB/s for staging groups of streams
        // through the copy engines (which move a plain 1 GiB copy at 192 GB/s)
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, host_out) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer && reinterpret_cast<uintptr_t>(pa.devicePointer) % 16 == 0) {
            const wn_status st = launch_generate(s, pa.devicePointer, count, 0, dtype, cs);
            if (st != WN_OK) return st;
            advance_k(s, count);
            return WN_OK;
        }
        cudaGetLastError();  // an unregistered pointer is not an error here
    }
    if (!s->d_stage[0]) {
        s->stage_bytes = kStageMax;
        for (int b = 0; b < 2; ++b) {
            WN_CU(cudaMalloc(&s->d_stage[b], s->stage_bytes));
            WN_CU(cudaEventCreateWithFlags(&s->ev_gen[b], cudaEventDisableTiming));
            WN_CU(cudaEventCreateWithFlags(&s->ev_copy[b], cudaEventDisableTiming));
        }
        WN_CU(cudaStreamCreateWithFlags(&s->copy_cs, cudaStreamNonBlocking));
    }
    unsigned char *dst = static_cast<unsigned char *>(host_out);
    // a previous call's copies out of the staging buffers come first
    for (int b = 0; b < 2; ++b) WN_CU(cudaStreamWaitEvent(cs, s->ev_copy[b], 0));
    if (group > 0) {
        // whole requests of consecutive streams: each group's output is one
        // contiguous range of host_out, moved by one plain copy.  A copy into
        // pageable memory returns only once it is done, so the next group's
        // kernel is enqueued after it: generation and copies alternate (the
        // copies, not the kernels, set the pace)
        int j = 0;
        for (uint64_t g0 = 0; g0 < s->n; g0 += group, ++j) {
            const int b = j & 1;
            const uint32_t len = (uint32_t)std::min<uint64_t>(group, s->n - g0);
            if (j >= 2) WN_CU(cudaStreamWaitEvent(cs, s->ev_copy[b], 0));
            const wn_status st = launch_generate(s, s->d_stage[b], count, 0, dtype, cs, (uint32_t)g0, len);
            if (st != WN_OK) return st;
            WN_CU(cudaEventRecord(s->ev_gen[b], cs));
            WN_CU(cudaStreamWaitEvent(s->copy_cs, s->ev_gen[b], 0));
            WN_CU(cudaMemcpyAsync(dst + g0 * per_stream, s->d_stage[b], len * per_stream, cudaMemcpyDeviceToHost,
                                  s->copy_cs));
            WN_CU(cudaEventRecord(s->ev_copy[b], s->copy_cs));
        }
        advance_k(s, count);
    } else {
        // requests too long to stage whole: every stream's next chunk per
        // round (a multiple of 8 values, so each stream's slice of a staging
        // buffer stays 16-byte aligned), copied with a pitched copy (which,
        // into pageable memory, also returns once it is done)
        uint64_t chunk = s->stage_bytes / (esize * (uint64_t)s->n) / 8 * 8;
        if (chunk == 0) return fail(WN_EINVAL, "wn_generate_host: too many streams for the staging buffer");
        if (chunk > count) chunk = count;
        uint64_t done = 0;
        for (int j = 0; done < count; ++j) {
            const int b = j & 1;
            const uint64_t c = std::min<uint64_t>(chunk, count - done);
            if (j >= 2) WN_CU(cudaStreamWaitEvent(cs, s->ev_copy[b], 0));
            wn_status st = launch_generate(s, s->d_stage[b], c, 0, dtype, cs);
            if (st != WN_OK) return st;
            advance_k(s, c);
            WN_CU(cudaEventRecord(s->ev_gen[b], cs));
            WN_CU(cudaStreamWaitEvent(s->copy_cs, s->ev_gen[b], 0));
            WN_CU(cudaMemcpy2DAsync(dst + done * esize, count * esize, s->d_stage[b], c * esize, c * esize, s->n,
                                    cudaMemcpyDeviceToHost, s->copy_cs));
            WN_CU(cudaEventRecord(s->ev_copy[b], s->copy_cs));
            done += c;
        }
    }
    // later work on cuda_stream (and its synchronisation) follows the copies
    for (int b = 0; b < 2; ++b) WN_CU(cudaStreamWaitEvent(cs, s->ev_copy[b], 0));
    return WN_OK;
}

wn_status wn_generate_batch(void *out, const uint64_t *counts, const uint64_t *offsets, wn_stream *s, wn_dtype dtype,
                            int use_graph, void *cuda_stream)
{
    wn_status st = check_batch_args(s, out, counts, offsets, dtype);
    if (st != WN_OK) return st;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(cuda_stream);
    std::vector<uint32_t> order;
    const std::vector<Group> groups = plan_batch(s, counts, order, s->batch_crit);
    if (groups.size() > 16) return fail(WN_EINVAL, "wn_generate_batch: more than 16 pool sizes");
    if ((st = ensure_batch_buffers(s, groups.size())) != WN_OK) return st;
    const bool same = use_graph && s->gexec && s->g_out == out && s->g_dtype == (int)dtype &&
                      std::equal(counts, counts + s->n, s->g_counts.begin()) &&
                      std::equal(offsets, offsets + s->n, s->g_offsets.begin());
    if (!use_graph) {
        if ((st = upload_desc(s, s->bd_eager, counts, offsets, order, cs)) != WN_OK) return st;
        if ((st = enqueue_batch(s, groups, out, dtype, cs, s->bd_eager)) != WN_OK) return st;
    } else {
        if (!same) {
            // the graph's own descriptors, then one capture of the counters'
            // reset and the groups' launches reading them (the upload is in
            // stream order before the graph's first launch)
            if (s->gexec) {
                cudaGraphExecDestroy(s->gexec);
                s->gexec = nullptr;
            }
            if ((st = upload_desc(s, s->bd_graph, counts, offsets, order, cs)) != WN_OK) return st;
            cudaStream_t cap = nullptr;
            WN_CU(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                st = enqueue_batch(s, groups, out, dtype, cap, s->bd_graph);
                e = cudaStreamEndCapture(cap, &graph);
            }
            // keep the captured streams' priorities (exclusive groups first)
            if (e == cudaSuccess && st == WN_OK)
                e = cudaGraphInstantiate(&s->gexec, graph, cudaGraphInstantiateFlagUseNodePriority);
            if (graph) cudaGraphDestroy(graph);
            cudaStreamDestroy(cap);
            if (st != WN_OK) return st;
            if (e != cudaSuccess) return cuda_fail("wn_generate_batch: graph capture", e);
            s->g_out = out;
            s->g_dtype = (int)dtype;
            s->g_counts.assign(counts, counts + s->n);
            s->g_offsets.assign(offsets, offsets + s->n);
        }
        WN_CU(cudaGraphLaunch(s->gexec, cs));
    }
    for (uint32_t i = 0; i < s->n; ++i) advance_k_one(s, i, counts[i]);
    return WN_OK;
}

namespace {
// Key of a batch's tuned plan: the device, the output type and a hash of
// every stream's pool size, passes and request length.
std::string batch_key(const wn_stream *s, const uint64_t *counts, wn_dtype dt)
{
    uint64_t h = 0xcbf29ce484222325ull;
    auto mix = [&](uint64_t v) {
        for (int i = 0; i < 8; ++i) h = (h ^ ((v >> (8 * i)) & 0xFF)) * 0x100000001b3ull;
    };
    for (uint32_t i = 0; i < s->n; ++i) {
        mix(s->N[i]);
        mix(s->R[i]);
        mix(counts[i]);
    }
    char hx[32];
    std::snprintf(hx, sizeof hx, "%016llx", (unsigned long long)h);
    return "batch|" + device_tag(s) + "|var=" + std::to_string((int)s->var) + "|dtype=" + std::to_string((int)dt) +
           "|streams=" + std::to_string(s->n) + "|sig=" + hx;
}

// "chains density;N qt maxt threads ip grp lat;..." <-> the handle's batch choices.
std::string batch_text(const wn_stream *s)
{
    std::string t = std::to_string(s->batch_crit) + " " + std::to_string(s->batch_density);
    for (const auto &kv : s->group_cfg) {
        const auto lat = s->group_lat.find(kv.first);
        t += ";" + std::to_string(kv.first) + " " + cfg_text(kv.second) + " " +
             std::to_string(lat != s->group_lat.end() && lat->second ? 1 : 0);
    }
    return t;
}

bool batch_from_text(wn_stream *s, const std::string &t)
{
    int crit = 0, dens = 0;
    if (std::sscanf(t.c_str(), "%d %d", &crit, &dens) != 2 || crit < -1 || dens < 1 || dens > 8) return false;
    std::map<uint32_t, LaunchCfg> cfg;
    std::map<uint32_t, bool> lat;
    for (size_t p = t.find(';'); p != std::string::npos; p = t.find(';', p + 1)) {
        unsigned N = 0;
        int l = 0, used = 0;
        if (std::sscanf(t.c_str() + p + 1, "%u%n", &N, &used) != 1 || !valid_pool(N)) return false;
        LaunchCfg c;
        const char *rest = t.c_str() + p + 1 + used;
        if (!cfg_from_text(rest, c) || !cached_cfg_ok(c, N) || (c.grp && !batch_group_ok(s))) return false;
        if (std::sscanf(rest, "%*d %*d %*u %*d %*d %d", &l) != 1) return false;
        cfg[N] = c;
        lat[N] = l != 0;
    }
    s->batch_crit = crit;
    s->batch_density = dens;
    s->group_cfg = cfg;
    s->group_lat = lat;
    return true;
}
}  // namespace

wn_status wn_autotune_batch(void *out, const uint64_t *counts, const uint64_t *offsets, wn_stream *s, wn_dtype dtype,
                            void *cuda_stream)
{
    wn_status st = check_batch_args(s, out, counts, offsets, dtype);
    if (st != WN_OK) return st;
    {
        std::string v;  // tuned for this batch by an earlier process
        if (wn::tune_cache_get(batch_key(s, counts, dtype), v) && batch_from_text(s, v)) {
            if (s->gexec) {
                cudaGraphExecDestroy(s->gexec);
                s->gexec = nullptr;
            }
            return WN_OK;
        }
    }
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(cuda_stream);
    std::vector<uint32_t> order;
    const std::vector<Group> groups = plan_batch(s, counts, order, -1);
    if (groups.size() > 16) return fail(WN_EINVAL, "wn_autotune_batch: more than 16 pool sizes");
    if ((st = ensure_batch_buffers(s, groups.size())) != WN_OK) return st;
    const BatchDesc &d = s->bd_eager;
    if ((st = upload_desc(s, d, counts, offsets, order, cs)) != WN_OK) return st;
    size_t pool_floats = 0;
    for (uint32_t i = 0; i < s->n; ++i) pool_floats += s->N[i];
    wn::StreamHdr *hdr_bak = nullptr;
    float *pool_bak = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&hdr_bak, sizeof(wn::StreamHdr) * s->n);
    if (e == cudaSuccess) e = cudaMalloc(&pool_bak, sizeof(float) * pool_floats);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hdr_bak, s->d_hdr, sizeof(wn::StreamHdr) * s->n, cudaMemcpyDeviceToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pool_bak, s->d_pools, sizeof(float) * pool_floats, cudaMemcpyDeviceToDevice, cs);
    auto restore = [&]() {
        cudaError_t r = cudaMemcpyAsync(s->d_hdr, hdr_bak, sizeof(wn::StreamHdr) * s->n, cudaMemcpyDeviceToDevice, cs);
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(s->d_pools, pool_bak, sizeof(float) * pool_floats, cudaMemcpyDeviceToDevice, cs);
        return r;
    };
    // the trials below set the handle's shapes; an error restores these
    const std::map<uint32_t, LaunchCfg> old_cfg = s->group_cfg;
    const std::map<uint32_t, bool> old_lat = s->group_lat;
    std::map<uint32_t, LaunchCfg> chosen;
    std::map<uint32_t, bool> chosen_lat;
    for (size_t gi = 0; gi < groups.size() && e == cudaSuccess; ++gi) {
        const Group &g = groups[gi];
        if (g.exclusive) continue;  // fixed lowest-latency shape
        const uint32_t nq = g.N / 4;
        float best_ms = 1e30f;
        LaunchCfg best = pick_cfg(g.N);
        // candidates: the full ordinary shapes and, for the plain method, the
        // group-mode shapes of this pool size
        std::vector<LaunchCfg> cand;
        for (const auto &k : wn::kShapes)
            for (uint32_t t = 32; t + 32 <= (uint32_t)k[1]; t += 32) {
                LaunchCfg c{k[0], k[1], t, k[3]};
                if (cfg_ok(c, g.N) && (uint64_t)t * k[0] == nq) cand.push_back(c);  // full shapes only
            }
        if (batch_group_ok(s))
            for (const auto &k : wn::kGroupShapes)
                if ((uint32_t)k[0] == g.N) cand.push_back(group_cfg_of(g.N, (uint32_t)k[1]));
        for (size_t ci = 0; ci < cand.size() && e == cudaSuccess; ++ci) {
            const LaunchCfg c = cand[ci];
            s->group_cfg[g.N] = c;
            float times[2] = {0.f, 0.f};
            for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
                e = restore();
                if (e == cudaSuccess) e = cudaMemsetAsync(d.queue, 0, sizeof(uint32_t) * 16, cs);
                if (e == cudaSuccess) e = cudaEventRecord(e0, cs);
                if (e == cudaSuccess) {
                    const size_t smem = cfg_smem(s, c, g.N, g.r_max);
                    wn::GenArgs a{s->d_hdr, s->d_pools, out, 0, 0, g.len, g.N, g.r_max, 0};
                    wn::BatchArgs bq{d.order + g.start, d.offsets, d.counts, g.len, d.queue};
                    e = launch_persist_cfg(s, a, bq, c, g.N, dtype, smem, cs);
                }
                if (e == cudaSuccess) e = cudaEventRecord(e1, cs);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) times[rep - 1] = ms;
            }
            const float t_ms = std::min(times[0], times[1]);
            if (e == cudaSuccess && t_ms < best_ms) {
                best_ms = t_ms;
                best = c;
            }
        }
        chosen[g.N] = best;
        // the latency mode with its default shape, if it beats every ordinary shape
        LaunchCfg lc;
        bool lat = false;
        if (e == cudaSuccess && !s->var && latency_default(g.N, lc)) {
            float times[2] = {0.f, 0.f};
            for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
                e = restore();
                if (e == cudaSuccess) e = cudaMemsetAsync(d.queue, 0, sizeof(uint32_t) * 16, cs);
                if (e == cudaSuccess) e = cudaEventRecord(e0, cs);
                if (e == cudaSuccess) {
                    wn::GenArgs a{s->d_hdr, s->d_pools, out, 0, 0, g.len, g.N, g.r_max, 0};
                    wn::BatchArgs bq{d.order + g.start, d.offsets, d.counts, g.len, d.queue};
                    e = launch_persist_latency(s, a, bq, lc, g.N, g.r_max, false, dtype, cs);
                }
                if (e == cudaSuccess) e = cudaEventRecord(e1, cs);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) times[rep - 1] = ms;
            }
            lat = e == cudaSuccess && std::min(times[0], times[1]) < best_ms;
        }
        chosen_lat[g.N] = lat;
    }
    // Then the whole batch with the chosen shapes, for several numbers of
    // exclusive chains (0 .. a third of the SMs, and the estimate's rule):
    // the groups share the machine, which timing them alone cannot show.
    int best_crit = -1, best_density = 1;
    const int old_density = s->batch_density;
    if (e == cudaSuccess) {
        for (auto &kv : chosen) s->group_cfg[kv.first] = kv.second;
        for (auto &kv : chosen_lat) s->group_lat[kv.first] = kv.second;
        // (chains, chain CTAs per SM): the estimate's rule and up to a third of
        // the SMs exclusively, as before; then more chains sharing SMs two or
        // four to one, up to as many as that leaves room for
        std::vector<std::pair<int, int>> cands = {{-1, 1}, {0, 1}};
        const int third = std::max(1, s->sms / 3);
        for (int k = 4; k < third; k *= 2) cands.push_back({k, 1});
        cands.push_back({third, 1});
        for (int dd : {2, 4})
            for (int k = 32; k <= dd * s->sms && k <= (int)s->n; k *= 2) cands.push_back({k, dd});
        // each plan also with every group that has a latency shape in the
        // latency mode: the groups were timed without the estimate's chains,
        // and the requests left in them are serial chains too
        const std::map<uint32_t, bool> tuned_lat = s->group_lat;
        std::map<uint32_t, bool> all_lat = tuned_lat;
        for (const auto &g : groups) {
            LaunchCfg lc;
            if (!s->var && latency_default(g.N, lc)) all_lat[g.N] = true;
        }
        const size_t nplan = cands.size();
        // time of `reps` replays of the batch under plan ci (after one
        // untimed): their median, or with `worst` their slowest.  The groups'
        // CTAs reach the SMs in a different order on every run, and a chain
        // CTA that finds every SM taken waits for one to drain, so a plan can
        // be fast on most replays and much slower on some
        auto score = [&](size_t ci, int reps, float &t_ms, bool worst) {
            const auto &cd = cands[ci % nplan];
            s->group_lat = ci >= nplan ? all_lat : tuned_lat;
            s->batch_density = cd.second;
            std::vector<uint32_t> ord;
            const std::vector<Group> gk = plan_batch(s, counts, ord, cd.first);
            if (gk.size() > 16) return false;
            if ((st = ensure_batch_buffers(s, gk.size())) != WN_OK) return false;
            e = cudaMemcpyAsync(d.order, ord.data(), sizeof(uint32_t) * s->n, cudaMemcpyHostToDevice, cs);
            std::vector<float> times;
            for (int rep = 0; rep <= reps && e == cudaSuccess && st == WN_OK; ++rep) {
                e = restore();
                if (e == cudaSuccess) e = cudaEventRecord(e0, cs);
                if (e == cudaSuccess) st = enqueue_batch(s, gk, out, dtype, cs, d);
                if (e == cudaSuccess) e = cudaEventRecord(e1, cs);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) times.push_back(ms);
            }
            if (e != cudaSuccess || st != WN_OK || times.empty()) return false;
            std::sort(times.begin(), times.end());
            const size_t m = times.size();
            t_ms = worst ? times.back() : (m % 2) ? times[m / 2] : 0.5f * (times[m / 2 - 1] + times[m / 2]);
            return true;
        };
        // every plan on four replays (median); then the best four again on
        // eight, ranked by their slowest replay, so that neither one lucky
        // score nor a plan that is only sometimes fast decides
        std::vector<std::pair<float, size_t>> scored;
        for (size_t ci = 0; ci < 2 * nplan && e == cudaSuccess && st == WN_OK; ++ci) {
            if (ci >= nplan && all_lat == tuned_lat) break;  // nothing different to try
            float t = 0.f;
            if (score(ci, 4, t, false)) scored.push_back({t, ci});
        }
        std::sort(scored.begin(), scored.end());
        float best_ms = 1e30f;
        for (size_t r = 0; r < scored.size() && r < 4 && e == cudaSuccess && st == WN_OK; ++r) {
            float t = 0.f;
            if (!score(scored[r].second, 8, t, true) || t >= best_ms) continue;
            best_ms = t;
            best_crit = cands[scored[r].second % nplan].first;
            best_density = cands[scored[r].second % nplan].second;
            for (auto &kv : s->group_lat) chosen_lat[kv.first] = kv.second;
        }
    }
    s->batch_density = old_density;
    if (e == cudaSuccess) e = restore();
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (hdr_bak) cudaFree(hdr_bak);
    if (pool_bak) cudaFree(pool_bak);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess || st != WN_OK) {
        s->group_cfg = old_cfg;
        s->group_lat = old_lat;
        return e != cudaSuccess ? cuda_fail("wn_autotune_batch", e) : st;
    }
    for (auto &kv : chosen) s->group_cfg[kv.first] = kv.second;
    for (auto &kv : chosen_lat) s->group_lat[kv.first] = kv.second;
    s->batch_crit = best_crit;
    s->batch_density = best_density;
    wn::tune_cache_put(batch_key(s, counts, dtype), batch_text(s));
    if (s->gexec) {  // a captured graph used the old shapes
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
    }
    return WN_OK;
}

wn_status wn_generate_batch_noalloc(void *out, const uint64_t *counts, const uint64_t *offsets, wn_stream *s,
                                    wn_dtype dtype, void *cuda_stream)
{
    wn_status st = check_batch_args(s, out, counts, offsets, dtype);
    if (st != WN_OK) return st;
    if (s->n > WN_NOALLOC_MAX_STREAMS)
        return fail(WN_EINVAL, "wn_generate_batch_noalloc: " + std::to_string(s->n) + " streams exceed the " +
                                   std::to_string(WN_NOALLOC_MAX_STREAMS) + " its fixed scratch array holds");
    int dev = -1;
    WN_CU(cudaGetDevice(&dev));
    if (dev != s->device)
        return fail(WN_EINVAL, "wn_generate_batch_noalloc: the handle's device must be current");
    {
        // the call copies from host arrays and advances host bookkeeping as it
        // is made: a captured copy would replay stale arrays and a replay would
        // not advance the streams' positions
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        WN_CU(cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(cuda_stream), &cap));
        if (cap != cudaStreamCaptureStatusNone)
            return fail(WN_EINVAL, "wn_generate_batch_noalloc: not allowed while cuda_stream is being captured");
    }
    unsigned char *scratch = nullptr;
    if ((st = noalloc_scratch(dev, &scratch)) != WN_OK) return st;
    // Plan without heap allocation: pool sizes are powers of two 4..16384
    // (13 groups, indexed by log2 N - 2); each group's streams in claim order,
    // longest request first (ties by stream index; std::sort sorts in place).
    std::lock_guard<std::mutex> plan_lock(g_na_plan_mu);
    uint32_t *order = g_na_order;
    uint32_t cnt[13] = {}, start[13] = {}, fill[13] = {}, rmax[13] = {};
    auto gidx = [](uint32_t N) {
        uint32_t g = 0;
        while ((4u << g) < N) ++g;
        return g;
    };
    for (uint32_t i = 0; i < s->n; ++i) {
        const uint32_t g = gidx(s->N[i]);
        ++cnt[g];
        rmax[g] = std::max(rmax[g], s->R[i]);
    }
    for (uint32_t g = 1; g < 13; ++g) start[g] = start[g - 1] + cnt[g - 1];
    for (uint32_t i = 0; i < s->n; ++i) {
        const uint32_t g = gidx(s->N[i]);
        order[start[g] + fill[g]++] = i;
    }
    for (uint32_t g = 0; g < 13; ++g)
        std::sort(order + start[g], order + start[g] + cnt[g], [&](uint32_t x, uint32_t y) {
            const uint64_t cx = counts[x] * (s->R[x] + 1ull), cy = counts[y] * (s->R[y] + 1ull);
            return cx != cy ? cx > cy : x < y;
        });
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(cuda_stream);
    uint32_t *d_counters = reinterpret_cast<uint32_t *>(scratch + kNaCounters);
    uint32_t *d_order = reinterpret_cast<uint32_t *>(scratch + kNaOrder);
    uint64_t *d_offsets = reinterpret_cast<uint64_t *>(scratch + kNaOffsets);
    uint64_t *d_counts = reinterpret_cast<uint64_t *>(scratch + kNaCounts);
    WN_CU(cudaMemcpyAsync(d_counts, counts, sizeof(uint64_t) * s->n, cudaMemcpyHostToDevice, cs));
    WN_CU(cudaMemcpyAsync(d_offsets, offsets, sizeof(uint64_t) * s->n, cudaMemcpyHostToDevice, cs));
    WN_CU(cudaMemcpyAsync(d_order, order, sizeof(uint32_t) * s->n, cudaMemcpyHostToDevice, cs));
    // the claim counters must start at zero; the array keeps the last call's values
    WN_CU(cudaMemsetAsync(d_counters, 0, 256, cs));
    for (uint32_t g = 0; g < 13; ++g) {
        if (cnt[g] == 0) continue;
        const uint32_t N = 4u << g;
        wn::GenArgs a{s->d_hdr, s->d_pools, out, 0, 0, cnt[g], N, rmax[g], 0};
        wn::BatchArgs bq{d_order + start[g], d_offsets, d_counts, cnt[g], d_counters + g};
        const LaunchCfg c = batch_cfg(s, N);
        const size_t smem = cfg_smem(s, c, N, rmax[g]);
        const cudaError_t e = launch_persist_cfg(s, a, bq, c, N, dtype, smem, cs);
        if (e != cudaSuccess) return cuda_fail("wn_generate_batch_noalloc: launch", e);
    }
    for (uint32_t i = 0; i < s->n; ++i) advance_k_one(s, i, counts[i]);
    return WN_OK;
}

wn_status wn_get_batch_plan(const wn_stream *s, int32_t *chains, uint32_t *density)
{
    if (!s) return fail(WN_EINVAL, "wn_get_batch_plan: NULL handle");
    if (chains) *chains = s->batch_crit;
    if (density) *density = (uint32_t)s->batch_density;
    return WN_OK;
}

wn_status wn_set_batch_plan(wn_stream *s, int32_t chains, uint32_t density)
{
    if (!s) return fail(WN_EINVAL, "wn_set_batch_plan: NULL handle");
    if (chains < -1 || density < 1 || density > 8)
        return fail(WN_EINVAL, "wn_set_batch_plan: chains must be >= -1 and density in [1, 8]");
    s->batch_crit = chains;
    s->batch_density = (int)density;
    if (s->gexec) {  // a captured graph used the old plan
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
    }
    return WN_OK;
}

wn_status wn_set_batch_chain_kernel(wn_stream *s, int32_t chain_mode)
{
    if (!s) return fail(WN_EINVAL, "wn_set_batch_chain_kernel: NULL handle");
    if (chain_mode != 0 && chain_mode != 1) return fail(WN_EINVAL, "wn_set_batch_chain_kernel: chain_mode must be 0 or 1");
    s->batch_chain_mode = chain_mode == 1;
    if (s->gexec) {  // a captured graph used the other kernels
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
    }
    return WN_OK;
}

wn_status wn_gbm(wn_stream *s, float *ST_out, uint32_t paths_per_stream, uint32_t steps, double S0, double mu,
                 double sigma, double dt, void *cuda_stream)
{
    if (!s) return fail(WN_EINVAL, "wn_gbm: NULL handle");
    if (!ST_out || paths_per_stream == 0 || steps == 0 || !(S0 > 0.0) || !(sigma >= 0.0) || !(dt > 0.0))
        return fail(WN_EINVAL, "wn_gbm: NULL output or non-positive paths, steps, S0, dt, or negative sigma");
    for (uint32_t i = 0; i < s->n; ++i) {
        const uint32_t per = s->N[i] - 1;
        if (per % paths_per_stream != 0 || ((uint64_t)steps * paths_per_stream) % per != 0)
            return fail(WN_EINVAL, "wn_gbm: paths_per_stream must divide pool_N-1 and steps*paths_per_stream "
                                   "must be a multiple of pool_N-1 for every stream");
        if (s->k_host[i] != per)
            return fail(WN_EINVAL, "wn_gbm: stream " + std::to_string(i) +
                                       " has values of a partly returned block pending");
    }
    wn::GenArgs a;
    a.hdr = s->d_hdr;
    a.pools = s->d_pools;
    a.out = nullptr;
    a.count = (uint64_t)steps * paths_per_stream;
    a.out_stride = 0;
    a.n_streams = s->n;
    a.n_max = s->n_max;
    a.r_max = s->r_max;
    a.warmup_blocks = 0;
    wn::GbmArgs g;
    g.st = ST_out;
    g.ppg = paths_per_stream;
    g.S0 = (float)S0;
    g.drift_total = (float)((double)steps * (mu - 0.5 * sigma * sigma) * dt);
    g.vol = (float)(sigma * std::sqrt(dt));
    const uint32_t nq = s->n_max / 4;
    LaunchCfg c;
    if (nq <= 128) c = {1, 1024, std::max(32u, (nq + 31u) / 32u * 32u)};
    else if (nq <= 1024) c = {4, 288, nq / 4};
    else c = {8, 544, nq / 8};
    const bool full = s->uniform_N && (uint64_t)c.threads * c.qt == nq;
    const size_t smem = wn::gen_smem_bytes(s->smem_base, s->n_max, s->r_max);
    const cudaError_t e = wn::launch_gbm(a, g, c, full, smem, reinterpret_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail("wn_gbm launch", e);
    advance_k(s, a.count);
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

wn_status wn_debug_report(uint64_t *host_violations, uint64_t *host_first, int reset)
{
#ifdef WN_DEBUG
    unsigned long long rec[4] = {0, 0, 0, 0};
    WN_CU(cudaDeviceSynchronize());
    WN_CU(cudaMemcpyFromSymbol(rec, wn::wn_dbg_record, sizeof rec));
    if (host_violations) *host_violations = rec[0];
    if (host_first) *host_first = rec[1];
    if (reset) {
        const unsigned long long zero[4] = {0, 0, 0, 0};
        WN_CU(cudaMemcpyToSymbol(wn::wn_dbg_record, zero, sizeof zero));
    }
    return WN_OK;
#else
    (void)reset;
    if (host_violations) *host_violations = 0;
    if (host_first) *host_first = 0;
    return fail(WN_EINVAL, "wn_debug_report: this library was built without WN_DEBUG (no bounds checks)");
#endif
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
