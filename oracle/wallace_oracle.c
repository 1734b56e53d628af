/*
 * wallace_oracle.c -- plain, slow FP64 CPU oracle for Wallace's
 * maximum-entropy normal generator, as discussed by R. P. Brent,
 * "Some Comments on C. S. Wallace's Random Number Generators"
 * (arXiv:1005.2314), Section 5.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library
 * against.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it; the library never calls it and shares no code with it.
 *
 * Everything is FP64 with round-to-nearest and no FMA contraction (it is
 * compiled with -ffp-contract=off).  Each routine follows the method's steps
 * in the paper's order; where the paper leaves a detail to sources it cites
 * but does not reproduce, the routine states the reading it takes.
 *
 * Readings taken here (the paper is silent or defers to absent sources):
 *  - Uniform generator (Sections 3 and 5.8 only ask for a long-period generator
 *    with little state): xorshift64 with shifts (13, 7, 17) plus a Weyl
 *    sequence with increment 0x61C8864680B583EB; each draw advances both and
 *    returns their sum mod 2^64.  Seeded by SplitMix64(seed): the first output
 *    is the xorshift state (replaced by 1 if it is 0), the second the Weyl
 *    state.
 *  - Index choice and mixing (Section 5.4): each pass draws w_a and w_s.
 *    alpha = ((w_a >> 32) mod N) | 1 (odd, so a unit mod N), gamma = w_a mod N.
 *    Quadruple q (0 <= q < N/4) reads a_k = P[(alpha*(q + k*N/4) + gamma) mod N]
 *    for k = 0..3 and writes its outputs to slots 4q+k (the pool, seen as an
 *    (N/4) x 4 matrix, is transposed each pass as in fastnorm).
 *  - Orthogonal update (Section 5.3): y_k = t - a_k with t = (a_0+..+a_3)/2,
 *    i.e. the matrix (1/2)J - I, which equals the printed A_1 up to the order
 *    and signs of its rows.
 *  - Signs (Section 5.2): output k of quadruple q is negated when bit k of
 *    the nibble (w_s >> 4*(q mod 16)) & 15 is set.
 *  - Initialisation (Section 5.8 names it only): v_i = 2*(sum of the four
 *    16-bit fields of one draw) - 4*65535, then scaled so that sum v_i^2 = N.
 *    The first reserved value is r = 0, and W whole blocks are discarded.
 *  - Chi-squared correction (Section 5.5): after the R passes of a block the
 *    pool is renormalised to sum of squares N; the reserved value r of the
 *    previous block (fastnorm2) gives S from approximation (c) with nu = N;
 *    g = sqrt(S/N); the block returns g*P_0 .. g*P_{N-2} and keeps
 *    r = g*P_{N-1} for the next block.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* ---------------------------------------------------------------- */
/* Integer generators (Section 3; Section 5.8).                     */
/* ---------------------------------------------------------------- */

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): add the golden gamma to
 * the state, then mix the new state with Stafford's variant 13 finaliser. */
uint64_t orc_splitmix64(uint64_t *state)
{
    uint64_t z;
    *state = *state + 0x9E3779B97F4A7C15ull;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* One step of Marsaglia's 64-bit xorshift with the triple (13, 7, 17). */
uint64_t orc_xorshift64_step(uint64_t x)
{
    x = x ^ (x << 13);
    x = x ^ (x >> 7);
    x = x ^ (x << 17);
    return x;
}

/* Weyl increment: an odd constant (2^64 minus the golden gamma). */
#define ORC_WEYL 0x61C8864680B583EBull

typedef struct {
    uint64_t x; /* xorshift state, never 0 */
    uint64_t w; /* Weyl state */
} orc_u64gen;

void orc_u64gen_seed(orc_u64gen *g, uint64_t seed)
{
    uint64_t sm = seed;
    g->x = orc_splitmix64(&sm);
    if (g->x == 0)
        g->x = 1;
    g->w = orc_splitmix64(&sm);
}

uint64_t orc_u64gen_next(orc_u64gen *g)
{
    g->x = orc_xorshift64_step(g->x);
    g->w = g->w + ORC_WEYL;
    return g->x + g->w;
}

/* The first n draws of the stream seeded by `seed` (for bit-exact checks). */
void orc_draws(uint64_t seed, uint64_t n, uint64_t *out)
{
    orc_u64gen g;
    uint64_t i;
    orc_u64gen_seed(&g, seed);
    for (i = 0; i < n; i++)
        out[i] = orc_u64gen_next(&g);
}

/* ---------------------------------------------------------------- */
/* One pass: y = Q x with Q built from 4x4 orthogonal blocks         */
/* (Sections 5.1-5.4).                                              */
/* ---------------------------------------------------------------- */

static uint64_t orc_alpha(uint32_t N, uint64_t w_a) { return ((w_a >> 32) & (uint64_t)(N - 1)) | 1u; }
static uint64_t orc_gamma(uint32_t N, uint64_t w_a) { return w_a & (uint64_t)(N - 1); }

/* Read slot of element k of quadruple q: pi(j) = alpha*j + gamma mod N with
 * j = q + k*N/4 (the affine permutations of Section 5.4). */
static uint32_t orc_read_slot(uint32_t N, uint64_t alpha, uint64_t gamma, uint32_t q, uint32_t k)
{
    uint64_t j = (uint64_t)q + (uint64_t)k * (N / 4);
    return (uint32_t)((alpha * j + gamma) % N);
}

/* Read slots of the whole pass, slots[4q+k], for the mixing test. */
void orc_pass_read_slots(uint32_t N, uint64_t w_a, uint32_t *slots)
{
    uint64_t alpha = orc_alpha(N, w_a), gamma = orc_gamma(N, w_a);
    uint32_t q, k;
    for (q = 0; q < N / 4; q++)
        for (k = 0; k < 4; k++)
            slots[4 * q + k] = orc_read_slot(N, alpha, gamma, q, k);
}

static int orc_sign_bit(uint64_t w_s, uint32_t q, uint32_t k)
{
    uint64_t nibble = (w_s >> (4 * (q % 16))) & 15u;
    return (int)((nibble >> k) & 1u);
}

/* New pool Pn from pool P (N a power of two, N >= 4; P and Pn distinct). */
void orc_pass(uint32_t N, const double *P, double *Pn, uint64_t w_a, uint64_t w_s)
{
    uint64_t alpha = orc_alpha(N, w_a), gamma = orc_gamma(N, w_a);
    uint32_t q, k;
    for (q = 0; q < N / 4; q++) {
        double a[4], t, y;
        for (k = 0; k < 4; k++)
            a[k] = P[orc_read_slot(N, alpha, gamma, q, k)];
        t = (a[0] + a[1] + a[2] + a[3]) / 2.0;
        for (k = 0; k < 4; k++) {
            y = t - a[k];
            if (orc_sign_bit(w_s, q, k))
                y = -y;
            Pn[4 * q + k] = y;
        }
    }
}

/* Inverse of orc_pass with the same draws: undo the signs, apply the update
 * again ((1/2)J - I is its own inverse), and scatter back to the read slots. */
void orc_pass_inverse(uint32_t N, const double *Pn, double *P, uint64_t w_a, uint64_t w_s)
{
    uint64_t alpha = orc_alpha(N, w_a), gamma = orc_gamma(N, w_a);
    uint32_t q, k;
    for (q = 0; q < N / 4; q++) {
        double u[4], t;
        for (k = 0; k < 4; k++) {
            u[k] = Pn[4 * q + k];
            if (orc_sign_bit(w_s, q, k))
                u[k] = -u[k];
        }
        t = (u[0] + u[1] + u[2] + u[3]) / 2.0;
        for (k = 0; k < 4; k++)
            P[orc_read_slot(N, alpha, gamma, q, k)] = t - u[k];
    }
}

/* ---------------------------------------------------------------- */
/* The plane-rotation form (rann4, Section 5.3): one rotation        */
/* R(theta) = [c s; -s c] per pass, c = (1-t^2)/(1+t^2),              */
/* s = 2t/(1+t^2), t = tan(theta/2) drawn for the pass (theta itself  */
/* is never formed), applied to pairs gathered through the pass's     */
/* affine permutation (Section 5.4).                                  */
/* ---------------------------------------------------------------- */

/* t in (-1, 1) from the top 24 bits u of the pass's second draw:
 * t = (2u + 1) / 2^24 - 1, exact in FP64 (and in FP32). */
double orc_rot_t(uint64_t w_t)
{
    uint64_t u = w_t >> 40;
    return (double)(2 * u + 1) / 16777216.0 - 1.0;
}

/* Pair j (0 <= j < N/2) takes a = P[pi(j)], b = P[pi(j + N/2)] and writes
 * (c a + s b, -s a + c b) to slots 2j, 2j+1 (the transposed write). */
void orc_pass_rot(uint32_t N, const double *P, double *Pn, uint64_t w_a, uint64_t w_t)
{
    uint64_t alpha = orc_alpha(N, w_a), gamma = orc_gamma(N, w_a);
    double t = orc_rot_t(w_t), c = (1.0 - t * t) / (1.0 + t * t), s = 2.0 * t / (1.0 + t * t);
    uint32_t j;
    for (j = 0; j < N / 2; j++) {
        double a = P[(alpha * j + gamma) % N];
        double b = P[(alpha * (j + N / 2) + gamma) % N];
        Pn[2 * j] = c * a + s * b;
        Pn[2 * j + 1] = -s * a + c * b;
    }
}

/* The inverse of orc_pass_rot (the transposed rotation, gathered back). */
void orc_pass_rot_inverse(uint32_t N, const double *Pn, double *P, uint64_t w_a, uint64_t w_t)
{
    uint64_t alpha = orc_alpha(N, w_a), gamma = orc_gamma(N, w_a);
    double t = orc_rot_t(w_t), c = (1.0 - t * t) / (1.0 + t * t), s = 2.0 * t / (1.0 + t * t);
    uint32_t j;
    for (j = 0; j < N / 2; j++) {
        double y0 = Pn[2 * j], y1 = Pn[2 * j + 1];
        P[(alpha * j + gamma) % N] = c * y0 - s * y1;
        P[(alpha * (j + N / 2) + gamma) % N] = s * y0 + c * y1;
    }
}

/* ---------------------------------------------------------------- */
/* Chi-squared approximations (Section 5.5).                        */
/* ---------------------------------------------------------------- */

#define ORC_CHI2_OFF 0 /* no correction: g = 1 */
#define ORC_CHI2_A 1   /* 2 chi2 ~ (x + sqrt(2 nu - 1))^2 (rann4) */
#define ORC_CHI2_B 2   /* Wilson-Hilferty */
#define ORC_CHI2_C 3   /* A(x^2 - 1) + sqrt(2(nu - A^2)) x + nu */

/* A = 2 sqrt(nu) sin(arcsin(1/sqrt(nu)) / 3), the root of A^3 - 3 nu A + 2 nu = 0. */
double orc_chi2_A(double nu)
{
    return 2.0 * sqrt(nu) * sin(asin(1.0 / sqrt(nu)) / 3.0);
}

double orc_chi2(int kind, double nu, double x)
{
    if (kind == ORC_CHI2_A) {
        double s = x + sqrt(2.0 * nu - 1.0);
        return s * s / 2.0;
    }
    if (kind == ORC_CHI2_B) {
        double h = 2.0 / (9.0 * nu);
        double c = sqrt(h) * x + (1.0 - h);
        return nu * c * c * c;
    }
    if (kind == ORC_CHI2_C) {
        double A = orc_chi2_A(nu);
        return A * (x * x - 1.0) + sqrt(2.0 * (nu - A * A)) * x + nu;
    }
    return nu;
}

/* ---------------------------------------------------------------- */
/* A stream: pool, generator, reserved value, partly consumed block. */
/* ---------------------------------------------------------------- */

#define ORC_RESERVE_PREVIOUS 0 /* fastnorm2: x from the previous pool */
#define ORC_RESERVE_CURRENT 1  /* fastnorm: x from the current pool (test switch) */

typedef struct {
    uint32_t N, R;
    int chi2_kind, reserve_mode;
    orc_u64gen gen;
    double *P;       /* pool, renormalised to sum of squares N after each block */
    double *tmp;     /* second pool for the pass */
    double *blk;     /* the current block's N-1 returned values */
    double r;        /* scaled reserved value of the previous block */
    double g;        /* scale factor of the current block */
    uint32_t k;      /* values of the current block already returned */
    uint64_t blocks; /* blocks completed, warm-up included */
    uint32_t decimate; /* Section 5.7: return the values of every d-th block only */
    int update;        /* 0: the 4x4 form (fastnorm); 1: plane rotations (rann4) */
} orc_stream;

static int orc_valid(uint32_t N, uint32_t R)
{
    return N >= 4 && N <= (1u << 20) && (N & (N - 1)) == 0 && R >= 1;
}

/* One block: R passes, renormalisation, chi-squared scale, N-1 outputs. */
static void orc_block(orc_stream *s)
{
    uint32_t N = s->N, p, i;
    double sumsq, c, S, x;
    for (p = 0; p < s->R; p++) {
        uint64_t w_a = orc_u64gen_next(&s->gen);
        uint64_t w_s = orc_u64gen_next(&s->gen);
        double *t;
        if (s->update)
            orc_pass_rot(N, s->P, s->tmp, w_a, w_s);
        else
            orc_pass(N, s->P, s->tmp, w_a, w_s);
        t = s->P;
        s->P = s->tmp;
        s->tmp = t;
    }
    /* The sum of squares is invariant in exact arithmetic (Section 5.5);
     * renormalising removes rounding drift. */
    sumsq = 0.0;
    for (i = 0; i < N; i++)
        sumsq += s->P[i] * s->P[i];
    c = sqrt((double)N / sumsq);
    for (i = 0; i < N; i++)
        s->P[i] = s->P[i] * c;
    /* Scale so that the pool's sum of squares is a chi-squared_N sample S. */
    x = (s->reserve_mode == ORC_RESERVE_CURRENT) ? s->P[N - 1] : s->r;
    S = orc_chi2(s->chi2_kind, (double)N, x);
    s->g = sqrt(S / (double)N);
    for (i = 0; i + 1 < N; i++)
        s->blk[i] = s->g * s->P[i];
    s->r = s->g * s->P[N - 1];
    s->k = 0;
    s->blocks++;
}

/* A stream whose passes (warm-up included) use the 4x4 update (update 0)
 * or plane rotations (update 1, Section 5.3). */
orc_stream *orc_create_update(uint32_t N, uint32_t R, uint64_t seed, uint32_t warmup,
                              int chi2_kind, int reserve_mode, int update)
{
    orc_stream *s;
    uint32_t i, b, f;
    double sumsq, scale;
    if (!orc_valid(N, R) || (update != 0 && update != 1))
        return NULL;
    s = (orc_stream *)calloc(1, sizeof(*s));
    if (!s)
        return NULL;
    s->P = (double *)malloc(sizeof(double) * N);
    s->tmp = (double *)malloc(sizeof(double) * N);
    s->blk = (double *)malloc(sizeof(double) * N);
    if (!s->P || !s->tmp || !s->blk) {
        free(s->P);
        free(s->tmp);
        free(s->blk);
        free(s);
        return NULL;
    }
    s->N = N;
    s->R = R;
    s->chi2_kind = chi2_kind;
    s->reserve_mode = reserve_mode;
    orc_u64gen_seed(&s->gen, seed);
    /* Initial pool from the uniform generator (Section 5.8). */
    sumsq = 0.0;
    for (i = 0; i < N; i++) {
        uint64_t u = orc_u64gen_next(&s->gen);
        int64_t fields = 0;
        for (f = 0; f < 4; f++)
            fields += (int64_t)((u >> (16 * f)) & 0xFFFFu);
        s->P[i] = (double)(2 * fields - 4 * 65535);
        sumsq += s->P[i] * s->P[i];
    }
    scale = sqrt((double)N / sumsq);
    for (i = 0; i < N; i++)
        s->P[i] = s->P[i] * scale;
    s->r = 0.0;
    s->g = 1.0;
    s->decimate = 1;
    s->update = update;
    s->k = N - 1; /* no block has values left */
    for (b = 0; b < warmup; b++)
        orc_block(s);
    s->k = N - 1;
    return s;
}

orc_stream *orc_create(uint32_t N, uint32_t R, uint64_t seed, uint32_t warmup,
                       int chi2_kind, int reserve_mode)
{
    return orc_create_update(N, R, seed, warmup, chi2_kind, reserve_mode, 0);
}

void orc_destroy(orc_stream *s)
{
    if (!s)
        return;
    free(s->P);
    free(s->tmp);
    free(s->blk);
    free(s);
}

/* Section 5.7's remedy for finite-pool effects, keeping only one pool in
 * three (here one in d): from now on a new block is the d-th of d blocks run back to back,
 * the first d - 1 running in full (passes, scale, reserved value) but
 * returning nothing.  d = 1 is the plain method. */
int orc_set_decimate(orc_stream *s, uint32_t d)
{
    if (d < 1)
        return -1;
    s->decimate = d;
    return 0;
}

static void orc_next_block(orc_stream *s)
{
    uint32_t t;
    for (t = 0; t < s->decimate; t++)
        orc_block(s);
}

/* The next `count` values of the stream's sequence, which is the
 * concatenation of the blocks' returned values; calls may cut it anywhere. */
void orc_generate(orc_stream *s, double *out, uint64_t count)
{
    uint64_t n = 0;
    while (n < count) {
        if (s->k == s->N - 1)
            orc_next_block(s);
        while (s->k < s->N - 1 && n < count)
            out[n++] = s->blk[s->k++];
    }
}

/* Generate without storing (skips `count` values), for timing large samples
 * with bounded memory. Returns the sum of the values so nothing is elided. */
double orc_skip(orc_stream *s, uint64_t count)
{
    uint64_t n = 0;
    double acc = 0.0;
    while (n < count) {
        if (s->k == s->N - 1)
            orc_next_block(s);
        while (s->k < s->N - 1 && n < count) {
            acc += s->blk[s->k++];
            n++;
        }
    }
    return acc;
}

void orc_get_pool(const orc_stream *s, double *out) { memcpy(out, s->P, sizeof(double) * s->N); }
double orc_get_r(const orc_stream *s) { return s->r; }
double orc_get_g(const orc_stream *s) { return s->g; }
uint32_t orc_get_k(const orc_stream *s) { return s->k; }
uint64_t orc_get_blocks(const orc_stream *s) { return s->blocks; }
void orc_get_gen(const orc_stream *s, uint64_t *xw)
{
    xw[0] = s->gen.x;
    xw[1] = s->gen.w;
}

/* ---------------------------------------------------------------- */
/* Conventional comparison: Box-Muller on Philox4x32-10 (Section 4;  */
/* Section 5 names Box-Muller among the older methods).             */
/* ---------------------------------------------------------------- */

/* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11): ten rounds of two
 * 32x32->64 multiplies with the key bumped by the Weyl constants between
 * rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    int round;
    for (round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 = k0 + 0x9E3779B9u;
        k1 = k1 + 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Box-Muller normals z[i], i in [first, first+count), of stream `stream`
 * keyed by `seed`.  Philox block m = i / 4 uses counter (m lo, m hi, stream, 0)
 * and key (seed lo, seed hi); its words (w0, w1) and (w2, w3) each give one
 * pair: u1 = ((w >> 8) + 1) 2^-24 in (0, 1], u2 = (w' >> 8) 2^-24 in [0, 1),
 * rho = sqrt(-2 ln u1), z = (rho cos 2 pi u2, rho sin 2 pi u2). */
void orc_boxmuller(uint64_t seed, uint32_t stream, uint64_t first, uint64_t count, double *z)
{
    const double two_pi = 6.283185307179586476925286766559;
    uint64_t i;
    for (i = 0; i < count; i++) {
        uint64_t idx = first + i, m = idx / 4;
        uint32_t ctr[4], key[2], w[4];
        uint32_t pair = (uint32_t)((idx % 4) / 2), comp = (uint32_t)(idx % 2);
        double u1, u2, rho;
        ctr[0] = (uint32_t)m;
        ctr[1] = (uint32_t)(m >> 32);
        ctr[2] = stream;
        ctr[3] = 0;
        key[0] = (uint32_t)seed;
        key[1] = (uint32_t)(seed >> 32);
        orc_philox4x32_10(ctr, key, w);
        u1 = ((double)(w[2 * pair] >> 8) + 1.0) / 16777216.0;
        u2 = (double)(w[2 * pair + 1] >> 8) / 16777216.0;
        rho = sqrt(-2.0 * log(u1));
        z[i] = comp == 0 ? rho * cos(two_pi * u2) : rho * sin(two_pi * u2);
    }
}

/* ---------------------------------------------------------------- */
/* Monte Carlo consumer: geometric Brownian motion terminal prices.  */
/* ---------------------------------------------------------------- */

/* Path p (0 <= p < n_paths) of group c = p / paths_per_group draws its normal
 * for step j as value j*paths_per_group + (p mod paths_per_group) of the
 * Wallace stream with seed c+1, and takes the exact log step
 * S <- S exp((mu - sigma^2/2) dt + sigma sqrt(dt) Z). */
int orc_gbm(uint64_t n_paths, uint32_t paths_per_group, uint32_t steps, uint32_t N, uint32_t R,
            uint32_t warmup, double S0, double mu, double sigma, double dt, double *ST)
{
    uint64_t groups = (n_paths + paths_per_group - 1) / paths_per_group, c;
    double drift = (mu - 0.5 * sigma * sigma) * dt, vol = sigma * sqrt(dt);
    double *z = (double *)malloc(sizeof(double) * (size_t)paths_per_group);
    if (!z)
        return ORC_ENOMEM;
    for (c = 0; c < groups; c++) {
        orc_stream *s = orc_create(N, R, c + 1, warmup, ORC_CHI2_C, ORC_RESERVE_PREVIOUS);
        uint64_t p0 = c * paths_per_group, np = n_paths - p0, p;
        uint32_t j;
        if (!s) {
            free(z);
            return ORC_EINVAL;
        }
        if (np > paths_per_group)
            np = paths_per_group;
        for (p = 0; p < np; p++)
            ST[p0 + p] = 0.0; /* accumulated log-return */
        for (j = 0; j < steps; j++) {
            orc_generate(s, z, paths_per_group);
            for (p = 0; p < np; p++)
                ST[p0 + p] += drift + vol * z[p];
        }
        for (p = 0; p < np; p++)
            ST[p0 + p] = S0 * exp(ST[p0 + p]);
        orc_destroy(s);
    }
    free(z);
    return ORC_OK;
}
