/*
 * pns_oracle.c -- plain, slow CPU oracle for Rejection-Free Partial Neighbor
 * Search on QUBO targets pi(x) ~ exp(-beta * (x^T Q x + b^T x)), x in {0,1}^n.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, __graft_entry__.smoke() and the cpu_baseline
 * / reference leg of bench.py use it.  It shares no code, header, table or
 * constant with the CUDA library; it restates the paper's algorithms one
 * record at a time, in the order the paper states them:
 *
 *   Metropolis            -- Algorithm 1 (Sec. 1.1)
 *   Rejection-Free (RF)   -- Algorithm 2 (Sec. 1.2), jump chain of Eq. (2)
 *   Basic PNS             -- Algorithm 3 (Sec. 2)
 *   Unbiased PNS          -- Algorithm 6 (Sec. 3.2), alternating partial
 *                            neighbour sets with an L0 original-sample budget
 *   Alg. 11               -- Unbiased PNS without the Rejection-Free technique
 *                            (Appendix A), used only as a statistical check
 *   proportional choice   -- exponential race of Proposition 5 (appendix
 *                            "How to Sample Proportionally")
 *
 * Arithmetic that decides an integer (which neighbour wins the race, the
 * multiplicity M, accept/reject, the replica swap) is taken in IEEE fp32 with
 * the operation order written below, because that is the precision the GPU
 * kernels decide in; fields and energies of integer QUBOs are exact integers.
 * Compile with contraction off:  gcc -O2 -ffp-contract=off -fno-fast-math.
 *
 * Conventions (readings taken where the paper is silent):
 *  - local fields h = Qx + b (Q symmetric); flip delta of bit i:
 *      Delta_i = s_i * (2 h_i - b_i) + Q_ii,  s_i = 1 - 2 x_i
 *    which is E(x xor e_i) - E(x) for E = x^T Q x + b^T x.
 *  - proposal Q(x,y) = 1/n over Hamming-1 neighbours (Sec. 4); inside a
 *    partial neighbour set of size k the normalised proposal is 1/k (Sec. 3.2).
 *  - weights 1/k * min(1, exp(-beta Delta)) (Eq. (1) with the symmetric
 *    proposal cancelling).
 *  - M = 1 + G, G ~ Geometric(p) counting failures before the first success,
 *    so E[M] = 1/p (Sec. 1.2, Example 1: Geom(1) gives E[M] = 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): 10 rounds of the 4x32 Philox S-box with the     */
/* published multipliers and Weyl key increments.                           */
/* ------------------------------------------------------------------------ */
static void philox4x32_10(const uint32_t in[4], uint32_t key0, uint32_t key1, uint32_t out[4])
{
    uint32_t x0 = in[0], x1 = in[1], x2 = in[2], x3 = in[3];
    uint32_t k0 = key0, k1 = key1;
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod_a = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod_b >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod_b;
        uint32_t y2 = (uint32_t)(prod_a >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Stream tags (counter word 3, bits 24..31). */
enum { TAG_RACE = 1, TAG_STEP = 2, TAG_SUBSET = 3, TAG_SWAP = 5, TAG_ALG11 = 7 };

/* Word `index` of the stream (tag, id, step): counter = (index/4, id,
 * step low 32 bits, tag<<24 | step bits 32..55), key = (seed lo, seed hi). */
static uint32_t rng_word(uint64_t seed, uint32_t tag, uint32_t id, uint64_t step, uint32_t index)
{
    uint32_t ctr[4], out[4];
    ctr[0] = index >> 2;
    ctr[1] = id;
    ctr[2] = (uint32_t)step;
    ctr[3] = (tag << 24) | ((uint32_t)(step >> 32) & 0xFFFFFFu);
    philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32), out);
    return out[index & 3u];
}

/* ------------------------------------------------------------------------ */
/* Deterministic fp32 math from basic IEEE operations only.                 */
/* ------------------------------------------------------------------------ */
static float bits_to_float(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t float_to_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* ln 2 split so that e * LN2_HI is exact for |e| < 256. */
#define O_LN2_HI 0x1.62e400p-1f             /* 16 significant bits */
#define O_LN2_LO 0x1.7f7d1cp-20f            /* RN(ln 2 - LN2_HI) */
#define O_INV_LN2 0x1.715476p+0f             /* RN(1/ln 2) */

/* Natural log of a positive normal float.  x = 2^e * m, m in [sqrt(1/2),
 * sqrt(2)); ln m = 2 atanh(s), s = (m-1)/(m+1), by its odd power series
 * s + s^3/3 + ... + s^11/11 (|s| <= 0.1716, truncation < 1e-9 relative). */
float oq_logf(float x)
{
    uint32_t u = float_to_bits(x);
    int e = (int)((u >> 23) & 0xFFu) - 127;
    float m = bits_to_float((u & 0x007FFFFFu) | 0x3F800000u);
    if (m > 0x1.6a09e6p+0f) {           /* RN(sqrt 2) */
        m = m * 0.5f;
        e = e + 1;
    }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float poly = 0x1.745d18p-4f;                 /* 1/11 */
    poly = 0x1.c71c72p-4f + s2 * poly;            /* 1/9  */
    poly = 0x1.24924ap-3f + s2 * poly;            /* 1/7  */
    poly = 0x1.99999ap-3f + s2 * poly;            /* 1/5  */
    poly = 0x1.555556p-2f + s2 * poly;            /* 1/3  */
    poly = s2 * poly;
    float half_ln_m = s + s * poly;
    float ln_m = half_ln_m + half_ln_m;
    float ef = (float)e;
    float lo = ef * O_LN2_LO + ln_m;
    return ef * O_LN2_HI + lo;
}

/* exp(y) for y <= 0 (returns 0 below -87): n = rint(y / ln 2), r = y - n ln 2
 * (Cody-Waite, both products exact), exp(r) by its Taylor series to r^7/7!,
 * scaled by 2^n. */
float oq_expf(float y)
{
    if (!(y >= -87.0f)) return 0.0f;
    float nf = rintf(y * O_INV_LN2);
    float r = y - nf * O_LN2_HI;
    r = r - nf * O_LN2_LO;
    float p = 0x1.a01a02p-13f;                  /* 1/5040 */
    p = 0x1.6c16c2p-10f + r * p;                /* 1/720  */
    p = 0x1.111112p-7f + r * p;                /* 1/120  */
    p = 0x1.555556p-5f + r * p;                /* 1/24   */
    p = 0x1.555556p-3f + r * p;                   /* 1/6    */
    p = 0.5f + r * p;
    p = 1.0f + r * p;
    p = 1.0f + r * p;
    int n = (int)nf;
    float scale = bits_to_float((uint32_t)(n + 127) << 23);
    return p * scale;
}

/* -ln(1 - v) for v in (0, 1): power series v + v^2/2 + ... + v^7/7 below
 * 1/16 (truncation < 5e-10 relative), else -ln of the rounded (1 - v). */
float oq_neg_log1m(float v)
{
    if (v < 0.0625f) {
        float p = 0x1.24924ap-3f;                 /* 1/7 */
        p = 0x1.555556p-3f + v * p;               /* 1/6 */
        p = 0x1.99999ap-3f + v * p;               /* 1/5 */
        p = 0.25f + v * p;
        p = 0x1.555556p-2f + v * p;               /* 1/3 */
        p = 0.5f + v * p;
        p = 1.0f + v * p;
        return v * p;
    }
    return -oq_logf(1.0f - v);
}

/* Uniform in (0,1) with fine resolution near 0: the word is normalised by
 * its leading zeros, 23 bits below the leading one are kept and a half unit
 * is added, v = (2m+1) 2^-24 2^-z.  w = 0 maps to 2^-56. */
float oq_uniform_fine32(uint32_t w)
{
    if (w == 0u) return bits_to_float((uint32_t)(127 - 56) << 23);
    int z = 0;
    while (!(w & 0x80000000u)) { w <<= 1; ++z; }
    uint32_t m = (w >> 9);                      /* in [2^22, 2^23) */
    float mf = (float)(2u * m + 1u) * 0x1p-24f;  /* * 2^-24 */
    float scale = bits_to_float((uint32_t)(127 - z) << 23);
    return mf * scale;
}

/* Same normalisation for a 64-bit word; w = 0 maps to 2^-88. */
float oq_uniform_fine64(uint64_t w)
{
    if (w == 0u) return bits_to_float((uint32_t)(127 - 88) << 23);
    int z = 0;
    while (!(w & 0x8000000000000000ull)) { w <<= 1; ++z; }
    uint32_t m = (uint32_t)(w >> 41);           /* in [2^22, 2^23) */
    float mf = (float)(2u * m + 1u) * 0x1p-24f;
    float scale = bits_to_float((uint32_t)(127 - z) << 23);
    return mf * scale;
}

/* Plain uniform in (0,1) on the grid (2j+1) 2^-24. */
float oq_uniform24(uint32_t w)
{
    return (float)(2u * (w >> 9) + 1u) * 0x1p-24f;
}

/* ------------------------------------------------------------------------ */
/* Problem description (filled from Python through ctypes).                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t n;
    int32_t is_float;        /* 0: integer QUBO, exact int64 arithmetic; 1: fp32 */
    int32_t is_csr;          /* 0: dense n*n row-major; 1: CSR off-diagonal + diag */
    int32_t pad;
    const int32_t *q_i;      /* dense matrix or CSR values (integer) */
    const float *q_f;        /* dense matrix or CSR values (fp32) */
    const int32_t *row_ptr;  /* CSR: n+1 */
    const int32_t *col;      /* CSR: nnz */
    const int32_t *diag_i;   /* CSR diagonal */
    const float *diag_f;
    const int32_t *b_i;      /* linear term, may be NULL (= 0) */
    const float *b_f;
} oq_problem;

enum { V_BASIC = 0, V_UNBIASED = 1, V_RF = 2, V_METROPOLIS = 3 };
enum { SUB_SYSTEMATIC = 0, SUB_RANDOM = 1 };

typedef struct {
    int32_t variant;
    int32_t k;
    int32_t subset;
    int32_t pad;
    int64_t L0;
    uint64_t seed;
    /* Cooling schedule T(k) of Algorithms 8-10 (Sec. 8.1), non-increasing:
     * record k (k = 1, 2, ...) targets pi^{1/T(k)}, i.e. inverse temperature
     * beta / T(k) = beta s_k with s_k = s0^(1 - k/K) for k < K and 1 from
     * k = K on (geometric cooling from T = 1/s0 down to T = 1).
     * anneal_steps = K = 0: T = 1 throughout. */
    float anneal_start;      /* s0, in (0, 1] */
    int32_t pad2;
    int64_t anneal_steps;    /* K */
} oq_config;

/* beta / T(k) for record k of the schedule, in fp32:
 * r = k / K, y = ln(s0) (1 - r), beta exp(y). */
static float anneal_beta(const oq_config *C, float beta, float ln_s0, int64_t k)
{
    if (C->anneal_steps <= 0 || k >= C->anneal_steps) return beta;
    float r = (float)k / (float)C->anneal_steps;
    float y = ln_s0 * (1.0f - r);
    return beta * oq_expf(y);
}

/* Per-chain state (one per chain, owned by the caller). */
typedef struct {
    int64_t step;            /* records emitted so far */
    int64_t L;               /* Unbiased: remaining original samples */
    int64_t period_start;    /* Unbiased random sets: step the set was drawn at */
    int64_t flips;           /* moves */
    int64_t stays;           /* Unbiased period ends, Metropolis rejections */
    int64_t saturated;       /* multiplicities clamped at 2^63 */
    int64_t swaps_accepted;
    int32_t set_start;       /* Unbiased systematic: first bit of the set */
    int32_t beta_idx;
    double E;                /* current energy */
    double sum_m;            /* sum of multiplicities (original samples) */
    double best_E;
} oq_chain;

#define M_SATURATED 9223372036854775808.0   /* 2^63 */

static double q_entry(const oq_problem *P, int64_t idx)
{
    return P->is_float ? (double)P->q_f[idx] : (double)P->q_i[idx];
}

static int64_t qi_entry(const oq_problem *P, int64_t idx) { return (int64_t)P->q_i[idx]; }

static int64_t diag_int(const oq_problem *P, int i)
{
    if (P->is_csr) return (int64_t)P->diag_i[i];
    return (int64_t)P->q_i[(int64_t)i * P->n + i];
}

static float diag_flt(const oq_problem *P, int i)
{
    if (P->is_csr) return P->diag_f[i];
    return P->q_f[(int64_t)i * P->n + i];
}

static int64_t b_int(const oq_problem *P, int i) { return P->b_i ? (int64_t)P->b_i[i] : 0; }
static float b_flt(const oq_problem *P, int i) { return P->b_f ? P->b_f[i] : 0.0f; }

/* h = Qx + b.  Integer: exact.  fp32: h_i starts at b_i and adds the
 * selected entries in a fixed order (dense: column i read as row entries
 * Q[j][i], j ascending; CSR: diagonal first, then row i in stored order). */
void oq_init_fields(const oq_problem *P, const uint8_t *x, int64_t *h_i, float *h_f, double *E)
{
    int n = P->n;
    for (int i = 0; i < n; ++i) {
        if (P->is_float) {
            float acc = b_flt(P, i);
            if (P->is_csr) {
                if (x[i]) acc = acc + P->diag_f[i];
                for (int e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e)
                    if (x[P->col[e]]) acc = acc + P->q_f[e];
            } else {
                for (int j = 0; j < n; ++j)
                    if (x[j]) acc = acc + P->q_f[(int64_t)j * n + i];
            }
            h_f[i] = acc;
        } else {
            int64_t acc = b_int(P, i);
            if (P->is_csr) {
                if (x[i]) acc += P->diag_i[i];
                for (int e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e)
                    if (x[P->col[e]]) acc += P->q_i[e];
            } else {
                for (int j = 0; j < n; ++j)
                    if (x[j]) acc += P->q_i[(int64_t)j * n + i];
            }
            h_i[i] = acc;
        }
    }
    /* E = x^T Q x + b^T x = sum_i x_i h_i, summed in double, i ascending. */
    double e = 0.0;
    for (int i = 0; i < n; ++i)
        if (x[i]) e = e + (P->is_float ? (double)h_f[i] : (double)h_i[i]);
    *E = e;
}

/* Flip delta of bit i (Sec. 4 target, derived from the local fields). */
static int64_t delta_int(const oq_problem *P, const uint8_t *x, const int64_t *h, int i)
{
    int64_t g = 2 * h[i] - b_int(P, i);
    if (x[i]) g = -g;
    return g + diag_int(P, i);
}

static float delta_flt(const oq_problem *P, const uint8_t *x, const float *h, int i)
{
    float g = h[i] + h[i];
    g = g - b_flt(P, i);
    if (x[i]) g = -g;
    return g + diag_flt(P, i);
}

/* Apply the flip of bit j: h += s_j * Q[j,:] (Q symmetric), x_j ^= 1. */
static void apply_flip(const oq_problem *P, uint8_t *x, int64_t *h_i, float *h_f, int j)
{
    int n = P->n;
    int up = (x[j] == 0);      /* s_j = +1 */
    if (P->is_csr) {
        for (int e = P->row_ptr[j]; e < P->row_ptr[j + 1]; ++e) {
            int r = P->col[e];
            if (P->is_float) h_f[r] = up ? h_f[r] + P->q_f[e] : h_f[r] - P->q_f[e];
            else h_i[r] += up ? (int64_t)P->q_i[e] : -(int64_t)P->q_i[e];
        }
        if (P->is_float) h_f[j] = up ? h_f[j] + P->diag_f[j] : h_f[j] - P->diag_f[j];
        else h_i[j] += up ? (int64_t)P->diag_i[j] : -(int64_t)P->diag_i[j];
    } else {
        for (int r = 0; r < n; ++r) {
            int64_t idx = (int64_t)j * n + r;
            if (P->is_float) h_f[r] = up ? h_f[r] + P->q_f[idx] : h_f[r] - P->q_f[idx];
            else h_i[r] += up ? qi_entry(P, idx) : -qi_entry(P, idx);
        }
    }
    x[j] ^= 1u;
}

/* ------------------------------------------------------------------------ */
/* One Rejection-Free decision over k candidates (Algorithms 2, 3, 6).      */
/* ------------------------------------------------------------------------ */
/* Inputs: the k flip deltas (integer or fp32), beta, and the stream ids.
 * Outputs: the race winner (position in 0..k-1), the quantised weight sum
 * S_q, p, and M = 1 + Geometric(p).  Steps:
 *   Delta+_t = max(Delta_t, 0); anchor A = min_t Delta+_t
 *   w_t = exp(-beta (Delta+_t - A))           in (0, 1], w = 1 at the anchor
 *   race (Prop. 5): key_t = E_t / w_t with E_t = -ln(1 - V_t) ~ Exp(1);
 *                   winner = lexicographic min (key_t, t)
 *   S_q = sum_t floor(w_t 2^32)                (uint64, order free)
 *   p = (S_q 2^-32 / k) exp(-beta A)           = sum_t (1/k) min(1, e^{-beta Delta_t})
 *   M = 1 + floor(E1 / -ln(1 - p)),  E1 = -ln(V) ~ Exp(1) from 64 bits.
 */
int oq_decide(int is_float, const int64_t *d_int, const float *d_flt, int32_t k, float beta,
              uint64_t seed, uint32_t chain, uint64_t step,
              int32_t *winner, uint64_t *s_q, float *p_out, double *m_out, int32_t *saturated)
{
    if (k <= 0) return 1;
    /* anchor */
    int64_t a_int = 0;
    float a_flt = 0.0f;
    for (int t = 0; t < k; ++t) {
        if (is_float) {
            float dp = d_flt[t] > 0.0f ? d_flt[t] : 0.0f;
            if (t == 0 || dp < a_flt) a_flt = dp;
        } else {
            int64_t dp = d_int[t] > 0 ? d_int[t] : 0;
            if (t == 0 || dp < a_int) a_int = dp;
        }
    }
    uint64_t sum_q = 0;
    uint32_t best_key = 0xFFFFFFFFu;
    int best_t = -1;
    for (int t = 0; t < k; ++t) {
        float diff;
        if (is_float) {
            float dp = d_flt[t] > 0.0f ? d_flt[t] : 0.0f;
            diff = dp - a_flt;
        } else {
            int64_t dp = d_int[t] > 0 ? d_int[t] : 0;
            diff = (float)(dp - a_int);
        }
        float w = oq_expf(-(beta * diff));
        sum_q += (uint64_t)(w * 0x1p32f);
        uint32_t word = rng_word(seed, TAG_RACE, chain, step, (uint32_t)t);
        float v = oq_uniform_fine32(word);
        float ex = oq_neg_log1m(v);
        float key = ex / w;                      /* w = 0 gives +inf */
        uint32_t kb = float_to_bits(key);
        if (best_t < 0 || kb < best_key) {       /* strict: lowest t wins ties */
            best_key = kb;
            best_t = t;
        }
    }
    float anchor = is_float ? a_flt : (float)a_int;
    float ps = (float)sum_q * 0x1p-32f;   /* * 2^-32 */
    ps = ps / (float)k;
    float f = oq_expf(-(beta * anchor));
    float p = ps * f;
    double m;
    int sat = 0;
    if (p >= 1.0f) {
        m = 1.0;
    } else if (p <= 0.0f) {
        m = M_SATURATED;
        sat = 1;
    } else {
        float lam = oq_neg_log1m(p);
        uint32_t w0 = rng_word(seed, TAG_STEP, chain, step, 0);
        uint32_t w1 = rng_word(seed, TAG_STEP, chain, step, 1);
        uint64_t wide = ((uint64_t)w1 << 32) | (uint64_t)w0;
        float e1 = -oq_logf(oq_uniform_fine64(wide));
        float g = e1 / lam;
        if (!(g < 0x1p63f)) {
            m = M_SATURATED;
            sat = 1;
        } else {
            m = (double)floorf(g) + 1.0;
        }
    }
    *winner = best_t;
    *s_q = sum_q;
    *p_out = p;
    *m_out = m;
    *saturated = sat;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Random partial neighbour set: the first k distinct values of the stream  */
/* v_m = floor(word_m * n / 2^32), m = 0, 1, 2, ... (sequential sampling     */
/* without replacement by rejection; uniform over k-subsets).               */
/* ------------------------------------------------------------------------ */
int oq_random_subset(int32_t n, int32_t k, uint64_t seed, uint32_t chain, uint64_t step, int32_t *out)
{
    if (k <= 0 || k > n) return 1;
    uint8_t *seen = (uint8_t *)calloc((size_t)n, 1);
    if (!seen) return 2;
    int got = 0;
    int64_t cap = 64 * (int64_t)n + 1024;
    for (int64_t m = 0; got < k; ++m) {
        if (m >= cap) { free(seen); return 3; }
        uint32_t w = rng_word(seed, TAG_SUBSET, chain, step, (uint32_t)m);
        int v = (int)(((uint64_t)w * (uint64_t)n) >> 32);
        if (!seen[v]) {
            seen[v] = 1;
            out[got++] = v;
        }
    }
    free(seen);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One chain, one record at a time.                                         */
/* ------------------------------------------------------------------------ */
/* Runs until `max_records` records are emitted, or (when stop_after_periods
 * > 0, Unbiased only) until that many periods have ended.  Records go to the
 * tape (flip index or -1, M) when the tape pointers are non-NULL.  Returns 0,
 * or a positive error code.  *records_out = records emitted by this call. */
int oq_run_chain(const oq_problem *P, const oq_config *C, float beta, uint32_t chain,
                 uint8_t *x, int64_t *h_i, float *h_f, oq_chain *S,
                 int64_t max_records, int64_t stop_after_periods,
                 int32_t *tape_flip, double *tape_m, int64_t *records_out, uint8_t *x_best)
{
    /* x_best (may be NULL): X_max of Algorithms 8-10, the state of lowest
     * energy seen so far (highest pi at any beta > 0); it changes only on a
     * strict improvement, so it stays the initial state until E drops below
     * the initial energy. */
    int n = P->n;
    int k;
    switch (C->variant) {
    case V_RF: k = n; break;
    case V_METROPOLIS: k = 1; break;
    default: k = C->k; break;
    }
    if (k <= 0 || k > n) return 1;
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    int64_t *d_i = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    float *d_f = (float *)malloc(sizeof(float) * (size_t)k);
    if (!cand || !d_i || !d_f) { free(cand); free(d_i); free(d_f); return 2; }
    int rc = 0;
    int64_t rec = 0, periods = 0;
    const float ln_s0 = C->anneal_steps > 0 ? oq_logf(C->anneal_start) : 0.0f;
    const float beta_chain = beta;
    while (rec < max_records) {
        if (stop_after_periods > 0 && periods >= stop_after_periods) break;
        uint64_t step = (uint64_t)S->step;
        int32_t flip = -1;
        double m = 1.0;
        /* the record's inverse temperature: record k = step + 1 of the chain */
        beta = anneal_beta(C, beta_chain, ln_s0, (int64_t)step + 1);
        if (C->variant == V_METROPOLIS) {
            /* Algorithm 1: propose a uniform neighbour, accept w.p. min(1, e^{-beta Delta}). */
            uint32_t w2 = rng_word(C->seed, TAG_STEP, chain, step, 2);
            uint32_t w3 = rng_word(C->seed, TAG_STEP, chain, step, 3);
            int i = (int)(((uint64_t)w2 * (uint64_t)n) >> 32);
            float df = P->is_float ? delta_flt(P, x, h_f, i) : (float)delta_int(P, x, h_i, i);
            float lu = oq_logf(oq_uniform24(w3));
            float y = -(beta * df);
            if (lu < y) {
                double dE = P->is_float ? (double)delta_flt(P, x, h_f, i) : (double)delta_int(P, x, h_i, i);
                apply_flip(P, x, h_i, h_f, i);
                S->E = S->E + dE;
                S->flips += 1;
                flip = i;
            } else {
                S->stays += 1;
            }
            m = 1.0;
        } else {
            /* the partial neighbour set N_i (or all n bits for RF) */
            if (C->variant == V_RF) {
                for (int t = 0; t < k; ++t) cand[t] = t;
            } else if (C->variant == V_BASIC) {
                rc = oq_random_subset(n, k, C->seed, chain, step, cand);
                if (rc) break;
            } else if (C->subset == SUB_SYSTEMATIC) {
                for (int t = 0; t < k; ++t) cand[t] = (int)(((int64_t)S->set_start + t) % n);
            } else {
                rc = oq_random_subset(n, k, C->seed, chain, (uint64_t)S->period_start, cand);
                if (rc) break;
            }
            for (int t = 0; t < k; ++t) {
                if (P->is_float) d_f[t] = delta_flt(P, x, h_f, cand[t]);
                else d_i[t] = delta_int(P, x, h_i, cand[t]);
            }
            int32_t win;
            uint64_t sq;
            float p;
            int32_t sat;
            rc = oq_decide(P->is_float, d_i, d_f, k, beta, C->seed, chain, step, &win, &sq, &p, &m, &sat);
            if (rc) break;
            int move = 1;
            if (C->variant == V_UNBIASED) {
                /* Algorithm 6: spend the budget if m <= L, else stay for the
                 * remaining L samples and switch to the next set. */
                if (m <= (double)S->L) {
                    S->L -= (int64_t)m;
                } else {
                    move = 0;
                    m = (double)S->L;
                    S->L = C->L0;
                    S->stays += 1;
                    periods += 1;
                    S->set_start = (int32_t)(((int64_t)S->set_start + k) % n);
                    S->period_start = (int64_t)step + 1;
                }
            }
            if (move) {
                if (sat) S->saturated += 1;
                int j = cand[win];
                double dE = P->is_float ? (double)d_f[win] : (double)d_i[win];
                apply_flip(P, x, h_i, h_f, j);
                S->E = S->E + dE;
                S->flips += 1;
                flip = j;
            }
        }
        if (tape_flip) tape_flip[rec] = flip;
        if (tape_m) tape_m[rec] = m;
        S->sum_m = S->sum_m + m;
        if (S->E < S->best_E) {
            S->best_E = S->E;
            if (x_best) memcpy(x_best, x, (size_t)n);
        }
        S->step += 1;
        rec += 1;
    }
    free(cand);
    free(d_i);
    free(d_f);
    if (records_out) *records_out = rec;
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Replica exchange between adjacent temperatures (parallel tempering, Sec. */
/* 4's "multiple replicas at different temperatures").  Round r pairs       */
/* temperature indices (a, a+1) for a = r mod 2, r mod 2 + 2, ...; pair q   */
/* swaps with probability min(1, exp((beta_a - beta_b)(E_a - E_b))).        */
/* beta_idx[s] is the temperature index held by replica slot s.             */
/* ------------------------------------------------------------------------ */
int oq_swap_round(int32_t R, const float *betas, const double *E, int32_t *beta_idx,
                  uint64_t seed, uint32_t group, uint64_t round, int64_t *accepted)
{
    int32_t *slot_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
    if (!slot_of) return 2;
    for (int s = 0; s < R; ++s) slot_of[beta_idx[s]] = s;
    int q = 0;
    for (int a = (int)(round & 1u); a + 1 < R; a += 2, ++q) {
        int sa = slot_of[a], sb = slot_of[a + 1];
        float db = betas[a] - betas[a + 1];
        float de = (float)(E[sa] - E[sb]);
        float xr = db * de;
        uint32_t w = rng_word(seed, TAG_SWAP, group, round, (uint32_t)q);
        float lu = oq_logf(oq_uniform24(w));
        if (lu < xr) {
            beta_idx[sa] = a + 1;
            beta_idx[sb] = a;
            slot_of[a] = sb;
            slot_of[a + 1] = sa;
            if (accepted) accepted[sa] += 1, accepted[sb] += 1;
        }
    }
    free(slot_of);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Alg. 11 (Appendix A): Metropolis restricted to the systematic set N_i,   */
/* switching sets every L0 steps.  Writes the state code after each step    */
/* (n <= 31).  Statistical cross-check of Algorithm 6 only.                 */
/* ------------------------------------------------------------------------ */
int oq_run_alg11(const oq_problem *P, int32_t k, int64_t L0, float beta, uint64_t seed, uint32_t chain,
                 uint8_t *x, int64_t *h_i, float *h_f, int64_t n_steps, uint32_t *codes)
{
    int n = P->n;
    if (n > 31 || k <= 0 || k > n) return 1;
    int64_t L = L0;
    int set_start = 0;
    for (int64_t s = 0; s < n_steps; ++s) {
        uint32_t w0 = rng_word(seed, TAG_ALG11, chain, (uint64_t)s, 0);
        uint32_t w1 = rng_word(seed, TAG_ALG11, chain, (uint64_t)s, 1);
        int t = (int)(((uint64_t)w0 * (uint64_t)k) >> 32);   /* uniform in N_i: Q_i = 1/k */
        int i = (set_start + t) % n;
        float df = P->is_float ? delta_flt(P, x, h_f, i) : (float)delta_int(P, x, h_i, i);
        float lu = oq_logf(oq_uniform24(w1));
        if (lu < -(beta * df)) apply_flip(P, x, h_i, h_f, i);
        L -= 1;
        if (L == 0) {
            L = L0;
            set_start = (set_start + k) % n;
        }
        uint32_t code = 0;
        for (int b = 0; b < n; ++b) code |= (uint32_t)x[b] << b;
        codes[s] = code;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Continuous Unbiased PNS (Algorithm 7) and Metropolis on the Donuts target */
/* (Sec. 7): f(x) ~ exp[-(x1^2 + x2^2 - mu0)^2 / (2 sigma^2)], written as    */
/* exp(-E(x)) with E(x) = c (x1^2 + x2^2 - mu0)^2, c = 1 / (2 sigma^2).      */
/* ------------------------------------------------------------------------ */

/* (cos 2 pi u, sin 2 pi u) for u in [0, 1): quadrant q = floor(4u), angle
 * theta = (4u - q) pi / 2 in [0, pi / 2), Taylor series of sin to theta^11
 * and of cos to theta^12 (Horner in theta^2), then the quadrant's rotation. */
void oq_sincos2pi(float u, float *c_out, float *s_out)
{
    float u4 = u * 4.0f;                  /* exact */
    float qf = floorf(u4);
    float f = u4 - qf;                    /* exact */
    int q = (int)qf;
    float t = f * 0x1.921fb6p+0f;         /* pi / 2 */
    float t2 = t * t;
    float ps = -0x1.ae6456p-26f;          /* -1/11! */
    ps = 0x1.71de3ap-19f + t2 * ps;       /* 1/9! */
    ps = -0x1.a01a02p-13f + t2 * ps;      /* -1/7! */
    ps = 0x1.111112p-7f + t2 * ps;        /* 1/5! */
    ps = -0x1.555556p-3f + t2 * ps;       /* -1/3! */
    float sn = t + t * (t2 * ps);
    float pc = 0x1.1eed8ep-29f;           /* 1/12! */
    pc = -0x1.27e4fcp-22f + t2 * pc;      /* -1/10! */
    pc = 0x1.a01a02p-16f + t2 * pc;       /* 1/8! */
    pc = -0x1.6c16c2p-10f + t2 * pc;      /* -1/6! */
    pc = 0x1.555556p-5f + t2 * pc;        /* 1/4! */
    pc = -0.5f + t2 * pc;
    float cs = 1.0f + t2 * pc;
    float co, si;
    switch (q & 3) {
    case 0: co = cs; si = sn; break;
    case 1: co = -sn; si = cs; break;
    case 2: co = -cs; si = -sn; break;
    default: co = sn; si = -cs; break;
    }
    *c_out = co;
    *s_out = si;
}

/* Two independent N(0, 1) variates from two Philox words (Box-Muller):
 * r = sqrt(-2 ln U1) with U1 the fine uniform of w0, angle 2 pi U2 with U2
 * the grid uniform of w1. */
void oq_normal_pair(uint32_t w0, uint32_t w1, float *z1, float *z2)
{
    float lg = oq_logf(oq_uniform_fine32(w0));
    float r = sqrtf(-2.0f * lg);
    float co, si;
    oq_sincos2pi(oq_uniform24(w1), &co, &si);
    *z1 = r * co;
    *z2 = r * si;
}

float oq_donut_energy(float mu0, float c, float x1, float x2)
{
    float sq = x1 * x1 + x2 * x2;
    float u = sq - mu0;
    return c * (u * u);
}

typedef struct {
    float mu0;        /* ring radius squared */
    float c;          /* 1 / (2 sigma^2) */
    int64_t L0;       /* Unbiased budget per partial neighbour set */
    uint64_t seed;
    int32_t variant;  /* V_UNBIASED or V_METROPOLIS */
    int32_t npairs;   /* Unbiased: pairs +-delta per set (the set has 2 npairs points) */
} oq_donuts_cfg;

typedef struct {
    double weight;        /* sum of M: original samples */
    double sum_x[2];      /* sum of M x_i over records (x at the record's start) */
    double sum_x2[2];
    double sum_x4[2];
    double sum_pos[2];    /* sum of M [x_i > 0] */
    int64_t records, moves, budget_left, period_start;
    float x[2];           /* state after the run */
} oq_donuts_stats;

/* One chain for `steps` records from (x1, x2).  Unbiased PNS (Algorithm 7):
 * the partial neighbour set of a period is {x + d_j, x - d_j : j < npairs}
 * with d_j ~ N(0, I) drawn when the period starts (SUBSET stream at the
 * period's first record, Philox block j, words 0 and 1); the proposal is
 * uniform over the set, so each candidate weighs min(1, exp(-Delta)); M,
 * the budget and the choice of the next state are those of Algorithm 6.
 * Metropolis: y = x + d with d ~ N(0, I) from STEP words 0 and 1, accepted
 * iff ln U (grid uniform of STEP word 3) < -Delta. */
int oq_donuts_chain(const oq_donuts_cfg *C, uint32_t chain, int64_t steps, float x1, float x2, oq_donuts_stats *S)
{
    const int np = C->npairs;
    const int k = 2 * np;
    if (C->variant == V_UNBIASED && (np < 1 || np > 64)) return 1;
    float dx[64], dy[64], dl[128];
    memset(S, 0, sizeof(*S));
    int64_t L = C->L0, pstart = 0;
    int need_set = 1;
    for (int64_t step = 0; step < steps; ++step) {
        const float e0 = oq_donut_energy(C->mu0, C->c, x1, x2);
        double m;
        float nx1 = x1, nx2 = x2;
        int moved = 0;
        if (C->variant == V_METROPOLIS) {
            float d1, d2;
            oq_normal_pair(rng_word(C->seed, TAG_STEP, chain, (uint64_t)step, 0),
                           rng_word(C->seed, TAG_STEP, chain, (uint64_t)step, 1), &d1, &d2);
            float y1 = x1 + d1, y2 = x2 + d2;
            float dlt = oq_donut_energy(C->mu0, C->c, y1, y2) - e0;
            float lu = oq_logf(oq_uniform24(rng_word(C->seed, TAG_STEP, chain, (uint64_t)step, 3)));
            if (lu < -dlt) {
                nx1 = y1;
                nx2 = y2;
                moved = 1;
            }
            m = 1.0;
        } else {
            if (need_set) {
                for (int j = 0; j < np; ++j)
                    oq_normal_pair(rng_word(C->seed, TAG_SUBSET, chain, (uint64_t)pstart, 4u * (uint32_t)j),
                                   rng_word(C->seed, TAG_SUBSET, chain, (uint64_t)pstart, 4u * (uint32_t)j + 1u),
                                   &dx[j], &dy[j]);
                need_set = 0;
            }
            for (int j = 0; j < np; ++j) {
                dl[2 * j] = oq_donut_energy(C->mu0, C->c, x1 + dx[j], x2 + dy[j]) - e0;
                dl[2 * j + 1] = oq_donut_energy(C->mu0, C->c, x1 - dx[j], x2 - dy[j]) - e0;
            }
            int32_t win, sat;
            uint64_t sq;
            float p;
            int rc = oq_decide(1, NULL, dl, k, 1.0f, C->seed, chain, (uint64_t)step, &win, &sq, &p, &m, &sat);
            if (rc) return rc;
            if (m <= (double)L) {
                L -= (int64_t)m;
                const int j = win >> 1;
                if (win & 1) {
                    nx1 = x1 - dx[j];
                    nx2 = x2 - dy[j];
                } else {
                    nx1 = x1 + dx[j];
                    nx2 = x2 + dy[j];
                }
                moved = 1;
            } else {
                m = (double)L;
                L = C->L0;
                pstart = step + 1;
                need_set = 1;
            }
        }
        /* the record weighs the state it starts from */
        for (int i = 0; i < 2; ++i) {
            const double xd = (double)(i == 0 ? x1 : x2);
            const double x2d = xd * xd;
            S->sum_x[i] += m * xd;
            S->sum_x2[i] += m * x2d;
            S->sum_x4[i] += m * (x2d * x2d);
            if (xd > 0.0) S->sum_pos[i] += m;
        }
        S->weight += m;
        S->records += 1;
        S->moves += moved;
        x1 = nx1;
        x2 = nx2;
    }
    S->budget_left = L;
    S->period_start = pstart;
    S->x[0] = x1;
    S->x[1] = x2;
    return 0;
}

/* Raw stream access for the RNG pins. */
void oq_philox(const uint32_t ctr[4], uint32_t k0, uint32_t k1, uint32_t out[4])
{
    philox4x32_10(ctr, k0, k1, out);
}

uint32_t oq_rng_word(uint64_t seed, uint32_t tag, uint32_t id, uint64_t step, uint32_t index)
{
    return rng_word(seed, tag, id, step, index);
}

/* Vector helpers for the math pins. */
void oq_logf_vec(const float *x, float *y, int64_t n) { for (int64_t i = 0; i < n; ++i) y[i] = oq_logf(x[i]); }
void oq_expf_vec(const float *x, float *y, int64_t n) { for (int64_t i = 0; i < n; ++i) y[i] = oq_expf(x[i]); }
void oq_neg_log1m_vec(const float *x, float *y, int64_t n) { for (int64_t i = 0; i < n; ++i) y[i] = oq_neg_log1m(x[i]); }
void oq_uniform_fine32_vec(const uint32_t *w, float *y, int64_t n) { for (int64_t i = 0; i < n; ++i) y[i] = oq_uniform_fine32(w[i]); }
void oq_uniform_fine64_vec(const uint64_t *w, float *y, int64_t n) { for (int64_t i = 0; i < n; ++i) y[i] = oq_uniform_fine64(w[i]); }

void oq_sincos2pi_vec(const float *u, float *c, float *s, int64_t n) { for (int64_t i = 0; i < n; ++i) oq_sincos2pi(u[i], &c[i], &s[i]); }
void oq_normal_pair_vec(const uint32_t *w0, const uint32_t *w1, float *z1, float *z2, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) oq_normal_pair(w0[i], w1[i], &z1[i], &z2[i]);
}

/* Unused helper kept private to silence -Wunused for q_entry in some builds. */
double oq_q_entry(const oq_problem *P, int64_t idx) { return q_entry(P, idx); }
