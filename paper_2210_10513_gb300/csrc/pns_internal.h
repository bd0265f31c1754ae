// pns_internal.h -- descriptors shared by the host planner and the sm_103a
// kernels of libpns.  Not part of the public ABI (include/pns.h is).
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#define PNS_HD __host__ __device__ __forceinline__
#else
#define PNS_HD inline
#endif

namespace pnsk {

enum : int { VAR_BASIC = 0, VAR_UNBIASED = 1, VAR_RF = 2, VAR_METROPOLIS = 3 };
enum : int { SUB_SYSTEMATIC = 0, SUB_RANDOM = 1 };

// Philox stream tags (counter word 3, bits 24..31).
enum : uint32_t { TAG_RACE = 1, TAG_STEP = 2, TAG_SUBSET = 3, TAG_SWAP = 5 };

// Device status codes (mirror pns_status values).
enum : int { ST_OK = 0, ST_TIMEOUT = 6, ST_STATE = 7 };

// One QUBO instance as the kernels see it.
struct InstDesc {
    const void *q;          // dense: n rows of `ld` elements (zero padded); CSR: nnz values
    const int32_t *row_ptr; // CSR only
    const int32_t *col;     // CSR only
    const void *diag;       // n diagonal entries: int32 (integer QUBO) or float
    const void *b;          // n linear terms, same type as diag (zeros when absent)
    const float *betas;     // R inverse temperatures
    int32_t n, ld, k, R;
};

// One chain.
struct ChainDesc {
    int32_t inst;           // instance index
    int32_t slot;           // replica slot inside its exchange group
    int32_t group;          // global exchange group id
    int32_t smem_off;       // byte offset of the chain's area in its CTA's shared memory
};

// One CTA of the sampling launch.
struct CtaDesc {
    int32_t first;          // first entry in the CTA chain list
    int32_t count;          // chains (teams) in this CTA
    int32_t groups;         // exchange groups in this CTA (count / R when exchanging)
    int32_t pad;            // period-blocked kernel: warps per group in this CTA (0: the launch's)
};

// Persistent per-chain state in global memory (96 bytes).
struct ChainState {
    int64_t step;           // records emitted
    int64_t L;              // Unbiased budget left
    int64_t period_start;   // step at which the current random set was drawn
    int64_t flips, stays, saturated, swaps, tape_records;
    int32_t set_start;      // systematic set start bit
    int32_t beta_idx;       // temperature index held
    double E, sum_m, best_E;
};
static_assert(sizeof(ChainState) == 96, "ChainState layout");

// Kernel parameters (passed by value).
struct KParams {
    const InstDesc *inst;
    const ChainDesc *chain;
    const CtaDesc *cta;
    const int32_t *cta_chains;
    ChainState *state;
    uint32_t *xbits;        // chain c at c * W words
    void *fields;           // chain c at c * LD elements
    int32_t *tape_flip;     // chain c at c * tape_cap
    double *tape_m;
    uint32_t *tape_x;       // tape = 2: state bits at each record's start, W words per record
    double *tape_E;         // tape = 2: energy at each record's start
    uint32_t *xbest;        // NULL, or each chain's lowest-energy state (W words; X_max of Algorithms 8-10)
    int32_t *status;        // device status word (first error wins)
    int64_t tape_cap;
    int64_t steps;          // records (no exchange) or original samples (exchange)
    int64_t L0;
    int64_t swap_interval;
    uint64_t seed;
    int32_t variant, subset, W, LD;
    int32_t R;              // chains per exchange group (1 without exchange)
    int32_t pt;             // exchange on
    int32_t tape;
    int32_t prod;           // producer warps per chain (0: consumers draw their own numbers)
    uint32_t chain_base;    // global id of chain 0 (Philox stream id = chain_base + chain)
    uint32_t group_base;    // global id of exchange group 0
    int32_t prefetch;       // Unbiased: start the winner's row load before the budget test
    int32_t gw;             // period-blocked kernel: warps per exchange group
    const float4 *wtab;     // integer Q: weight tables e^{-beta d}, d = 0, 1, ... (w, its two quantised parts)
    const int2 *wtab_desc;  // per chain: (first entry, entries); entries 0 = no table
    uint32_t draw_cap;      // 0, or the most draws a random k-subset may take (host-set, for tests)
    float anneal_start;     // cooling schedule (Algorithms 8-10): s0, used when anneal_steps > 0
    int64_t anneal_steps;   // K: record k < K runs at beta s0^(1 - k/K); 0 = constant temperature
};

PNS_HD int32_t round16(int32_t b) { return (b + 15) & ~15; }

// Byte layout of one chain's shared-memory area.  Both the planner and the
// kernel derive it from (ld, k, field bytes, whether a subset list is kept,
// whether a producer warp fills the two look-ahead slots).  A slot holds the
// state-independent draws of one record: 16 bytes of scalars (the
// multiplicity's Exp(1), the Metropolis index and log-uniform, a dead flag),
// the k race exponentials and, for Basic PNS, the record's k-subset.
struct ChainSmem {
    int32_t fields, xw, list, bitmap, slots, slot_bytes, scratch, total;
};

PNS_HD ChainSmem chain_smem(int32_t ld, int32_t k, int32_t hbytes, bool list, bool slots, bool slot_list) {
    ChainSmem s;
    s.fields = 0;
    s.xw = round16(ld * hbytes);
    s.list = s.xw + round16(ld / 8);
    s.bitmap = s.list + (list ? round16(k * 4) : 0);
    s.slots = s.bitmap + (list ? round16(ld / 8) : 0);
    s.slot_bytes = slots ? round16(16 + 4 * k + (slot_list ? 4 * k : 0)) : 0;
    s.scratch = s.slots + 2 * s.slot_bytes;
    s.total = s.scratch + 768;   // 5 partials x 32 warps x 4 B, then publish / control words
    return s;
}

// Period-blocked kernel (Unbiased PNS, systematic sets, exchange groups).
// A chain's fields stay in global memory; shared memory holds, per chain, the
// k fields of its current set, its bits, a log of the period's flips, its
// ChainState and a few control words, and, per group, the k x k sub-block
// Q[N_i, N_i], the set's b and diagonal, the group's work queue and one draw
// buffer per warp (W warps).  The host
// gives every chain of a group ceil(group_bytes / R) bytes.
constexpr int BLOCK_LOG = 128;  // flips logged before a chain applies them itself
// Each warp of a group keeps the random numbers of its chain's next records:
// DRAW_BUF race exponentials (records of kp entries) and DRAW_MAXB Exp(1).
constexpr int DRAW_BUF = 256;
constexpr int DRAW_MAXB = 16;

// Positions of the current set each lane of the period-blocked kernel holds:
// the fewest of 1, 2 and 4 that leave lane 31 free (k <= 31 PPL), and 4 up to
// k = 128.  Also the kernel's code path (record form) for the group.
PNS_HD int block_ppl(int k) { return k <= 31 ? 1 : (k <= 62 ? 2 : 4); }

struct BlockSmem {
    int32_t insf, xw, log, state, scratch, chain_bytes, sub, bd, ctrl, wbuf, group_bytes;
};

PNS_HD BlockSmem block_smem(int32_t ld, int32_t k, int32_t hbytes, int32_t qbytes, int32_t R, int32_t W) {
    BlockSmem s;
    s.insf = 0;
    s.xw = round16(((k + 3) & ~3) * hbytes);
    s.log = s.xw + round16(ld / 8);
    s.state = s.log + 4 * BLOCK_LOG;
    s.scratch = s.state + static_cast<int32_t>(sizeof(ChainState));
    s.chain_bytes = s.scratch + 32;  // log length, records, finalised flag, set start, first step
    const int32_t kp = (k + 3) & ~3;         // sub-block row stride: 16-byte rows of 4-byte entries
    s.sub = R * s.chain_bytes;
    s.bd = s.sub + round16(k * kp * qbytes);  // b, then diag, of the set: 4-byte entries, 16-byte aligned
    s.ctrl = s.bd + 2 * round16(4 * kp);      // queue order[16], next, running, pad[2], records and slot by temperature [16] each
    s.wbuf = s.ctrl + 208;                    // W draw buffers
    s.group_bytes = s.wbuf + W * 4 * (DRAW_BUF + DRAW_MAXB);
    return s;
}

PNS_HD bool needs_list(int variant, int subset) {
    return variant == VAR_BASIC || (variant == VAR_UNBIASED && subset == SUB_RANDOM);
}

}  // namespace pnsk
