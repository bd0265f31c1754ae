/*
 * pns.h -- C ABI of the GB300 Rejection-Free Partial Neighbor Search sampler.
 *
 * Samples QUBO targets  pi(x) ~ exp(-beta (x^T Q x + b^T x)),  x in {0,1}^n,
 * with the jump-chain samplers of Chen, Rosenthal, Dote, Tamura and
 * Sheikholeslami, "Sampling via Rejection-Free Partial Neighbor Search":
 *
 *   PNS_METROPOLIS  Algorithm 1 (Sec. 1.1): one uniform Hamming-1 proposal,
 *                   accepted w.p. min(1, exp(-beta Delta)); every record has M = 1.
 *   PNS_RF          Algorithm 2 (Sec. 1.2): all n neighbours weighted
 *                   (1/n) min(1, exp(-beta Delta)); the next state is drawn in
 *                   proportion (Proposition 5's exponential race) and the
 *                   current one is recorded with multiplicity M = 1 + Geom(p),
 *                   p = sum of the weights (the jump chain of Eq. (2)).
 *   PNS_BASIC       Algorithm 3 (Sec. 2): as RF over a fresh uniform k-subset
 *                   each step, proposal 1/k on the subset.  Biased (Sec. 2.1-2.2).
 *   PNS_UNBIASED    Algorithm 6 (Sec. 3.2): partial neighbour sets N_i used in
 *                   turn for L0 original samples each; a move is taken only if
 *                   its M fits the remaining budget L, else the state is
 *                   recorded with M = L and the next set starts.  Systematic
 *                   sets are k consecutive bits starting at (i k) mod n
 *                   (Sec. 4-5, wrapping when k does not divide n); random sets
 *                   are a fresh uniform k-subset each period (Sec. 5).
 *
 * Each step reads the flip deltas of the candidate bits from maintained local
 * fields h = Q x + b,
 *     Delta_i = s_i (2 h_i - b_i) + Q_ii,   s_i = 1 - 2 x_i,
 * and a move to bit j updates all fields by the row Q[j,:] (rank-1 update).
 * Integer QUBOs are computed exactly (int32 fields); fp32 QUBOs in fp32 with a
 * fixed operation order.  Random numbers come from Philox4x32-10 with a fixed
 * counter layout, so a chain's records depend only on (seed, chain id, inputs)
 * and not on how chains are mapped onto the GPU.
 *
 * Replica exchange (parallel tempering, named in Sec. 4 as a way to use
 * parallel hardware): when swap_interval > 0, the n_replicas chains of one
 * (instance, chain) group run whole Unbiased periods and, every swap_interval
 * original samples, adjacent temperatures swap with probability
 * min(1, exp((beta_a - beta_b)(E_a - E_b))), alternating even / odd pairs.
 *
 * Pointers: every pointer argument may be host memory (pageable or pinned) or
 * device memory of the context's device; the library detects which.  Nothing
 * is retained after a call returns unless stated.  All functions return a
 * pns_status; none aborts.  pns_last_error() gives a thread-local message for
 * the last failing call.  Calls on one context must not overlap.
 */
#ifndef PNS_H
#define PNS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PNS_OK = 0,
    PNS_ERR_INVALID_ARG = 1,   /* bad size, pointer, enum or combination */
    PNS_ERR_NOT_SYMMETRIC = 2, /* Q != Q^T (dense) or a CSR entry without its mirror */
    PNS_ERR_RANGE = 3,         /* non-finite entry, or an integer field bound
                                  3 * max_i (sum_j |Q_ij| + |b_i|) >= 2^31 */
    PNS_ERR_OOM = 4,           /* device allocation failed */
    PNS_ERR_CUDA = 5,          /* a CUDA call failed (message says which) */
    PNS_ERR_TIMEOUT = 6,       /* a bounded device loop gave up (random subset draw) */
    PNS_ERR_STATE = 7,         /* the context latched a device error: restore or destroy */
    PNS_ERR_UNSUPPORTED = 8    /* valid request this build does not implement */
} pns_status;

typedef enum { PNS_BASIC = 0, PNS_UNBIASED = 1, PNS_RF = 2, PNS_METROPOLIS = 3 } pns_variant;
typedef enum { PNS_Q_I16 = 0, PNS_Q_I32 = 1, PNS_Q_F32 = 2 } pns_qtype;
typedef enum { PNS_DENSE = 0, PNS_CSR = 1 } pns_qformat;
typedef enum { PNS_SUBSET_SYSTEMATIC = 0, PNS_SUBSET_RANDOM = 1 } pns_subset;

/* One QUBO instance.  Q must be symmetric.  All instances of one context
 * share qtype and fmt. */
typedef struct {
    int32_t n;                 /* bits, >= 1 */
    int32_t fmt;               /* pns_qformat */
    int32_t qtype;             /* pns_qtype of q, diag and b */
    int32_t n_replicas;        /* temperatures of this instance (length of betas), >= 1 */
    int32_t k;                 /* subset size for this instance (Basic, Unbiased); 0 = pns_config.k */
    int32_t reserved;          /* must be 0 */
    const void *q;             /* DENSE: n*n row-major; CSR: nnz off-diagonal values */
    const int32_t *row_ptr;    /* CSR: n+1 offsets, row_ptr[0] = 0 */
    const int32_t *col;        /* CSR: nnz column indices, no diagonal, no duplicates in a row */
    int64_t nnz;               /* CSR: number of stored off-diagonal entries */
    const void *diag;          /* CSR: n diagonal entries (NULL = 0); ignored for DENSE */
    const void *b;             /* n linear terms (NULL = 0) */
    const float *betas;        /* n_replicas inverse temperatures, finite, >= 0 */
} pns_problem;

typedef struct {
    int32_t variant;           /* pns_variant */
    int32_t k;                 /* |N_i|: 1..n (Basic, Unbiased); ignored for RF (k = n) and Metropolis */
    int32_t subset;            /* pns_subset, Unbiased only */
    int32_t chains_per_replica;/* independent chains per (instance, temperature), >= 1 */
    int64_t L0;                /* Unbiased budget of original samples per set, >= 1 (paper: 100) */
    int64_t swap_interval;     /* 0: no exchange; else original samples between exchange
                                  rounds (Unbiased: a multiple of L0; Metropolis: any >= 1) */
    uint64_t seed;             /* Philox key */
    int32_t tape;              /* 0: no per-step records; 1: record (flip, M) every step;
                                  2: also the state bits and energy at each record's start */
    int32_t warps_per_chain;   /* 0: choose automatically; else 1, 2, 4, 8, 16 or 32 */
    int32_t chains_per_cta;    /* 0: choose automatically; else at most this many chains
                                  (or exchange groups) per CTA */
    int32_t chain_base;        /* global id of this context's first chain, >= 0: a shard of a larger
                                  job draws the same Philox streams as the whole job would */
    const uint32_t *x0;        /* NULL (all zeros) or initial bit-packed states: chain c,
                                  bit i at word c*W + i/32, bit i%32; W = pns_info.words_per_chain */
    int32_t group_base;        /* global id of this context's first exchange group, >= 0 */
    int32_t graph;             /* 1: pns_run captures its launch into a CUDA graph once per step
                                  count (and stream) and replays it; records are identical to
                                  direct launches.  On the legacy default stream (NULL) the
                                  kernel is launched directly.  The first call for a new step
                                  count captures: make it outside any capture of your own. */
    int32_t autotune;          /* 1: pns_create times the candidate chain-to-CTA mappings
                                  (warps per chain, producer warps, speculation depth, chains
                                  per CTA) on short probe runs and keeps the fastest; results
                                  do not depend on the mapping.  Choices are cached in the file
                                  named by PNS_AUTOTUNE_CACHE when that variable is set. */
    int32_t track_best;        /* 1: keep each chain's lowest-energy state X_max, the output of the
                                  optimisation forms (Algorithms 8-10: with variant BASIC this is
                                  Optimization PNS, with RF Optimization Rejection-Free, at the
                                  constant temperature 1/beta, or on the cooling schedule below);
                                  read it with pns_read_best.  Runs on the per-flip kernel. */
    int32_t reserved;          /* must be 0 */
    float anneal_start;        /* cooling schedule T(k) of Algorithms 8-10 (Sec. 8.1): s0 in (0, 1];
                                  with anneal_steps = K > 0, record k = 1, 2, ... of a chain (k counts
                                  the chain's records from its start) targets pi^{1/T(k)}, i.e. runs at
                                  inverse temperature beta s_k, s_k = s0^(1 - k/K) for k < K and 1 from
                                  k = K on (geometric cooling from T = 1/s0 to T = 1), in fp32:
                                  beta * det_exp(det_log(s0) * (1 - k/K)).  No replica exchange; runs
                                  on the per-flip kernel.  Ignored when anneal_steps = 0. */
    int32_t reserved2;         /* must be 0 */
    int64_t anneal_steps;      /* K >= 0; 0: constant temperature */
} pns_config;

/* Chain numbering: instance p, chain r of each temperature, replica slot s:
 *   id = sum_{p' < p} chains_per_replica * n_replicas(p') + r * n_replicas(p) + s.
 * Slot s starts at temperature index s; exchange moves temperatures, not states. */
typedef struct {
    int64_t chains;            /* total chains */
    int32_t words_per_chain;   /* W: uint32 words per packed state (max n rounded up) */
    int32_t field_stride;      /* elements per chain in pns_fields output */
    int32_t field_bytes;       /* bytes per field element (1, 2, 4) */
    int32_t field_is_float;    /* 1: fp32 fields, 0: signed integers */
    int64_t tape_capacity;     /* records per chain held by the tape of the last pns_run */
    int32_t warps_per_chain;   /* mapping in use: warps that serve one chain (all kinds) */
    int32_t ctas;              /* CTAs of the sampling launch */
    int32_t team_warps;        /* warps evaluating the chain's candidates (non-speculative kernel);
                                  period-blocked kernel: warps serving one exchange group */
    int32_t producer_warps;    /* warps precomputing the next record's random numbers */
    int32_t spec_depth;        /* speculative kernel: records evaluated at once (0: not used) */
    int32_t period_blocked;    /* 1: period-blocked update (Unbiased PNS with exchange): set fields
                                  from the k x k sub-block, other fields once per period */
    int32_t set_sweep;         /* 1: set-sweep kernel (Unbiased PNS, systematic sets): the
                                  spec_depth warps of a chain evaluate every set of the current
                                  state once, then decide up to 32 * spec_depth records at once */
    int32_t chains_per_warp;   /* 2: two chains per warp, one per half (Unbiased PNS on systematic
                                  sets of k <= 16, no exchange, many chains); else 1 */
    int32_t reserved_info;
} pns_info;

typedef struct {
    int64_t steps;             /* records emitted so far (jump steps, stays included) */
    int64_t flips;             /* moves */
    int64_t stays;             /* Unbiased period ends, Metropolis rejections */
    int64_t saturated;         /* moves whose M was clamped at 2^63 */
    int64_t swaps_accepted;    /* exchanges this slot took part in */
    int64_t budget_left;       /* Unbiased: L */
    int64_t tape_records;      /* records written to the tape by the last pns_run */
    int32_t set_start;         /* Unbiased systematic: first bit of the current set */
    int32_t beta_idx;          /* temperature index currently held */
    double energy;             /* E(x) of the current state */
    double sum_m;              /* sum of M: original (Metropolis-equivalent) samples */
    double best_energy;        /* lowest E seen */
} pns_stats;

typedef struct pns_ctx pns_ctx;

/* Copies the instances (host or device memory) into library-owned device
 * memory with padded rows, validates them on the device (symmetry, finiteness,
 * integer field range), sets the initial states and computes h = Qx + b and E
 * for every chain.  Enqueued on `stream` (a cudaStream_t, NULL = default) and
 * synchronised before returning.  The caller may free its buffers afterwards. */
pns_status pns_create(const pns_problem *probs, int32_t n_probs, const pns_config *cfg, void *stream,
                      pns_ctx **out);

/* Runs every chain for `steps` more records (without exchange), or for `steps`
 * more original samples, a multiple of swap_interval (with exchange).
 * Asynchronous on `stream`; returns launch errors only.  With cfg.tape = 1 the
 * records of this run replace the tape. */
pns_status pns_run(pns_ctx *ctx, int64_t steps, void *stream);

/* The plain form of pns_run: the same records, but each CTA of the plan is
 * its own launch, one after another on `stream` (with chains_per_cta = 1,
 * one chain per launch).  Exists to measure what batching buys. */
pns_status pns_run_plain(pns_ctx *ctx, int64_t steps, void *stream);

/* Synchronises `stream` and copies out: states (chains x W words), the tape
 * (chains x tape_capacity M values and flip indices, -1 = stay; entries past a
 * chain's tape_records are undefined) and per-chain statistics (host memory).
 * Any pointer may be NULL.  Returns a device error latched by earlier runs. */
pns_status pns_read(pns_ctx *ctx, uint32_t *states, double *multiplicities, int32_t *flips, pns_stats *stats,
                    void *stream);

/* With cfg.tape = 2, copies the sample tape of the last run: the state bits
 * (chains x tape_capacity x W words) and the energy (chains x tape_capacity)
 * at the start of each record, i.e. the jump-chain state J that the record's
 * multiplicity M weighs (Sec. 1.2, Theorem 3 (5)). */
pns_status pns_read_samples(pns_ctx *ctx, uint32_t *states, double *energies, void *stream);

/* With cfg.track_best = 1, copies every chain's X_max (Algorithms 8-10): the
 * state of lowest energy the chain has visited, which changes only when the
 * energy drops strictly below the best so far and so starts as the initial
 * state; chains x W words, host or device memory.  Its energy is
 * pns_stats.best_energy.  Synchronises `stream`. */
pns_status pns_read_best(pns_ctx *ctx, uint32_t *states, void *stream);

/* Scalars of a multiplicity-weighted sample: weight W = sum M, <E>, Var(E),
 * number of samples. */
typedef struct {
    double weight;
    double mean_energy;
    double var_energy;
    double samples;
} pns_moment_scalars;

/* Multiplicity-weighted moments of the last run's records (cfg.tape = 2, no
 * replica exchange) of the chains of one (instance, temperature index):
 * <x> (n), <x x^T> (n x n), Cov(E, x) (n), Cov(E, x x^T) (n x n), in fp64,
 * with <f> = sum_k M_k f(J_k) / sum_k M_k (Theorem 3 (5)).  The second moments
 * run on tcgen05 tensor cores (bf16 bit tiles, weights split into three bf16
 * parts, fp32 accumulation per 16384 samples, fp64 across).  n <= 64.
 * Outputs may be host or device memory, any may be NULL. */
pns_status pns_moments(pns_ctx *ctx, int32_t instance, int32_t beta_idx, pns_moment_scalars *scalars,
                       double *mean_x, double *mean_xx, double *cov_ex, double *cov_exx, void *stream);

/* Gradients from moments (all pointers device memory, fp64):
 *  data_xx == NULL: of the mean energy <E>:
 *      dQ = <x x^T> - beta Cov(E, x x^T), db = <x> - beta Cov(E, x), dbeta = -Var(E);
 *  else: of the Boltzmann log-likelihood of data with moments data_x, data_xx
 *  and mean energy data_mean_energy:
 *      dQ = -beta (data_xx - <x x^T>), db = -beta (data_x - <x>), dbeta = -data_E + <E>.
 *  `scalars` points to a device pns_moment_scalars. */
pns_status pns_energy_grads(int32_t n, float beta, const pns_moment_scalars *scalars, const double *mean_x,
                            const double *mean_xx, const double *cov_ex, const double *cov_exx, const double *data_x,
                            const double *data_xx, double data_mean_energy, double *dQ, double *db, double *dbeta,
                            void *stream);

/* The data term of the Boltzmann log-likelihood's energy (Sec. 8 target
 * pi ~ exp(-beta E)): the mean energy of data with moments data_x (n) and
 * data_xx (n x n), <E>_D = sum_ij data_xx_ij Q_ij + sum_i data_x_i b_i, in
 * fp64 with a fixed reduction order, written to *out.  q (n x n fp32), b (n
 * fp32, NULL = 0), data_x (required with b), data_xx and out are device
 * memory; asynchronous on `stream`. */
pns_status pns_data_energy(int32_t n, const float *q, const float *b, const double *data_x, const double *data_xx,
                           double *out, void *stream);

/* Copies the maintained local fields h (chains x field_stride elements of
 * field_bytes each, integers or fp32 per pns_info) to `out`. */
pns_status pns_fields(pns_ctx *ctx, void *out, void *stream);

/* Fills `info` (host memory) with the context's sizes and the launch mapping
 * in use (kernel form, CTAs, warps per chain); no device work. */
pns_status pns_get_info(const pns_ctx *ctx, pns_info *info);

/* Serialises every chain's state (statistics, bits, fields, exchange counters)
 * into host memory.  With buf = NULL only *bytes is set.  Restoring it into a
 * context created with the same problems and configuration continues the
 * chains exactly as if they had not stopped. */
pns_status pns_checkpoint(pns_ctx *ctx, void *buf, size_t *bytes);
pns_status pns_restore(pns_ctx *ctx, const void *buf, size_t bytes);

/* Frees the context's device memory and captured graph (cudaFree waits for
 * the device's outstanding work); NULL is ignored. */
void pns_destroy(pns_ctx *ctx);
/* The message of the last failed call on this thread (thread-local storage
 * owned by the library; valid until the thread's next failing call). */
const char *pns_last_error(void);

/* ---- Continuous state space: Unbiased PNS for continuous targets -------------
 * Algorithm 7 (Sec. 6) on the Donuts example of Sec. 7:
 *   pi(x) ~ exp[-(x1^2 + x2^2 - mu0)^2 / (2 sigma^2)] = exp(-E(x)),
 *   E(x) = c (x1^2 + x2^2 - mu0)^2 with c = 1 / (2 sigma^2),
 * evaluated in fp32 in this order: s = x1*x1 + x2*x2, u = s - mu0, E = c*(u*u).
 * PNS_UNBIASED: each period's partial neighbour set is {x + d_j, x - d_j :
 * j < npairs} with d_j ~ N(0, I) (Box-Muller from the SUBSET Philox stream at
 * the period's first record, block j, words 0 and 1), so that the set is
 * reversible; the proposal is uniform over the set, the multiplicity, the
 * budget L0 and the next state follow Algorithm 6.  PNS_METROPOLIS: the
 * paper's comparison, y = x + d with d ~ N(0, I), accepted w.p.
 * min(1, e^{-Delta}).  The chains' records are reduced on the fly to the
 * multiplicity-weighted sums the paper's bias measures need (Sec. 7). */
typedef struct {
    float mu0;                 /* mu0 (the paper: 9) */
    float c;                   /* 1 / (2 sigma^2) (sigma = 0.1: 50) */
    int64_t L0;                /* Unbiased: original samples per partial neighbour set (the paper: 1000) */
    uint64_t seed;             /* Philox key */
    int32_t variant;           /* PNS_UNBIASED or PNS_METROPOLIS */
    int32_t npairs;            /* Unbiased: 1..32 pairs +-d per set (the paper: 25, 50 neighbours) */
    int32_t chain_base;        /* global id of chain 0 (Philox stream id = chain_base + chain), >= 0 */
    int32_t reserved;          /* must be 0 */
} pns_donuts_config;

typedef struct {
    double weight;             /* sum of M over the records: original samples */
    double sum_x[2];           /* sum of M x_i, x the state each record starts from */
    double sum_x2[2];          /* sum of M x_i^2 */
    double sum_x4[2];          /* sum of M x_i^4 */
    double sum_pos[2];         /* sum of M [x_i > 0] */
    int64_t records;           /* jump-chain records (Metropolis: steps) */
    int64_t moves;
    int64_t budget_left;       /* Unbiased: L after the run */
    int64_t period_start;      /* Unbiased: record at which the current set was drawn */
    float x[2];                /* state after the run */
    int32_t pad[2];
} pns_donuts_stats;

/* Runs `chains` independent chains for `steps` records each from x0 (chains x 2
 * floats, host or device; NULL: every chain starts at (sqrt(mu0), 0)) and
 * writes one pns_donuts_stats per chain to `stats` (host or device).  Works in
 * device memory it allocates and frees itself; synchronises `stream`.
 * Fails with PNS_ERR_INVALID_ARG on a bad configuration. */
pns_status pns_donuts_run(const pns_donuts_config *cfg, int64_t chains, int64_t steps, const float *x0,
                          pns_donuts_stats *stats, void *stream);

/* Read bandwidth (GB/s, written to *gbs) that the current device sustains
 * from a buffer of `bytes` (>= 1 MiB, a multiple of 16; pick one well inside
 * L2, e.g. 64 MiB on GB300) read `passes` times by every SM after a warm-up
 * read, timed with CUDA events on `stream`.  A measurement aid for roofline
 * denominators (the L2 side of a kernel whose working set stays in L2); the
 * paper has no counterpart.  Allocates and frees its own buffer and
 * synchronises `stream`. */
pns_status pns_l2_read_probe(size_t bytes, int32_t passes, double *gbs, void *stream);

/* Size of the fixed device array that pns_sample_static works in.  Every GPU
 * that loads this library holds it until the process exits. */
#define PNS_STATIC_SCRATCH_BYTES (16u << 20)

/* pns_sample_static -- the paper has no counterpart; this is a convenience for
 * callers that cannot call cudaMalloc: code running while a framework's
 * caching allocator owns the device memory, services that allocate only at
 * start-up, library callbacks where an allocation and its implicit
 * synchronisation are not allowed.  One call creates, runs `steps` records of
 * every chain and reads back, for ONE dense instance, allocating nothing: all
 * working memory (chain states, fields, descriptors, validation words) lives
 * in one file-scope device array of PNS_STATIC_SCRATCH_BYTES.
 *   - prob: dense, n a positive multiple of 32; q (16-byte aligned), b and
 *     betas in device memory.  cfg: as for pns_create, without exchange
 *     (swap_interval = 0); cfg->x0, when given, in device memory; the
 *     producer warp is not used.
 *   - outputs: states (chains x n/32 words, host or device), multiplicities
 *     and flips (device, chains x steps, both or neither: one alone is
 *     PNS_ERR_INVALID_ARG), stats (host or device, chains entries); any may
 *     be NULL.
 *   - results equal pns_create + pns_run + pns_read on the same inputs, and
 *     inputs that pns_create rejects are rejected with the same status
 *     (configuration fields, symmetry, finiteness, field range, betas);
 *     track_best = 1 and tape = 2 return PNS_ERR_UNSUPPORTED.
 *   - sizes whose working memory exceeds the array return PNS_ERR_RANGE with
 *     the bytes needed; no partial work is done.
 *   - the first call on a device looks up the array's device address (with
 *     that device current), and so does the next call after a failed one.
 *   - it synchronises `stream`, so it cannot run while `stream` is being
 *     captured into a CUDA graph: such a call returns PNS_ERR_UNSUPPORTED and
 *     leaves the capture intact.
 *   - every call shares the array and leaves its contents behind; each call
 *     resets what it reads.  Calls that overlap on the GPU race on the array. */
pns_status pns_sample_static(const pns_problem *prob, const pns_config *cfg, int64_t steps, uint32_t *states,
                             double *multiplicities, int32_t *flips, pns_stats *stats, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PNS_H */
