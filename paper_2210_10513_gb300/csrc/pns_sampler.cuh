// pns_sampler.cuh -- the persistent batched sampling kernel.
//
// One team of warps owns one chain for the whole launch: TC consumer warps
// that carry the state-dependent chain of each record, and (optionally) a
// producer warp that draws the state-independent random numbers one record
// ahead into a double-buffered shared-memory slot.  The chain's local fields
// h = Qx + b and its packed bits live in shared memory; Q rows stream from
// HBM / L2 with 16-byte non-coherent loads.  A CTA holds several teams (or the
// replicas of exchange groups), packed by the host planner.  Per record:
//
//   a1  candidate set N_i: systematic window, drawn k-subset, all bits (RF)
//   a2  Delta_t = s_i (2 h_i - b_i) + Q_ii for each candidate (shared memory)
//   a3  anchor A = min_t max(Delta_t, 0)                  (team min-reduction)
//   a4  w_t = e^{-beta (Delta+_t - A)}, race key E_t / w_t (Proposition 5),
//       S = sum_t floor(w_t 2^32)                         (order-free reductions)
//   a5  p = (S 2^-32 / k) e^{-beta A}, M = 1 + Geom(p); Unbiased budget test
//   a6  move: h += s_j Q[j, :], x_j ^= 1, E += Delta_j
//   a7  record (j or -1, M) to the tape
//   a8  (exchange) at period ends all replicas of a group meet at a named
//       barrier and adjacent temperatures swap.
//
// Reductions are integer (min / add) or lexicographic (key, position), and
// every random number is a pure function of (seed, chain, step, position),
// so a chain's records do not depend on the team shape or on the packing.
#pragma once

#include <cstdint>
#include <type_traits>

#include "pns_device.cuh"
#include "pns_internal.h"

namespace pnsk {

// ---------------------------------------------------------------------------
// Type helpers: integer QUBOs compute deltas in int32, fp32 QUBOs in float.
// ---------------------------------------------------------------------------
template <typename HT> struct Arith;
template <> struct Arith<float> {
    using D = float;     // delta type
    using C = float;     // type of b and diag arrays
    static __device__ __forceinline__ float delta(float h, float b, float d, bool x) {
        float g = __fsub_rn(__fadd_rn(h, h), b);
        if (x) g = -g;
        return __fadd_rn(g, d);
    }
    static __device__ __forceinline__ float pos(float v) { return v > 0.0f ? v : 0.0f; }
    static __device__ __forceinline__ uint32_t key(float v) { return __float_as_uint(v); }  // v >= 0
    static __device__ __forceinline__ float unkey(uint32_t u) { return __uint_as_float(u); }
    static __device__ __forceinline__ float diff(float a, float m) { return __fsub_rn(a, m); }
    static __device__ __forceinline__ float tof(float v) { return v; }
    static __device__ __forceinline__ double tod(float v) { return static_cast<double>(v); }
};
template <typename HT> struct ArithInt {
    using D = int32_t;
    using C = int32_t;
    static __device__ __forceinline__ int32_t delta(HT h, int32_t b, int32_t d, bool x) {
        int32_t g = 2 * static_cast<int32_t>(h) - b;
        if (x) g = -g;
        return g + d;
    }
    static __device__ __forceinline__ int32_t pos(int32_t v) { return v > 0 ? v : 0; }
    static __device__ __forceinline__ uint32_t key(int32_t v) { return static_cast<uint32_t>(v); }  // v >= 0
    static __device__ __forceinline__ int32_t unkey(uint32_t u) { return static_cast<int32_t>(u); }
    static __device__ __forceinline__ float diff(int32_t a, int32_t m) { return __int2float_rn(a - m); }
    static __device__ __forceinline__ float tof(int32_t v) { return __int2float_rn(v); }
    static __device__ __forceinline__ double tod(int32_t v) { return static_cast<double>(v); }
};
template <> struct Arith<int32_t> : ArithInt<int32_t> {};
template <> struct Arith<int16_t> : ArithInt<int16_t> {};
template <> struct Arith<int8_t> : ArithInt<int8_t> {};

__device__ __forceinline__ void named_sync(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

__device__ __forceinline__ uint4 ld_nc_v4(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ void set_status(int32_t *status, int code) { atomicCAS(status, 0, code); }

// Add s * (one 16-byte chunk of a Q row) into fields.  QT elements -> HT.
template <typename QT, typename HT>
__device__ __forceinline__ void add_chunk(HT *h, const uint4 &v, bool up) {
    constexpr int VE = 16 / static_cast<int>(sizeof(QT));
    QT q[VE];
    *reinterpret_cast<uint4 *>(q) = v;
    if constexpr (std::is_same<HT, float>::value) {
        float4 *hp = reinterpret_cast<float4 *>(h);
        float4 a = hp[0];
        if (up) {
            a.x = __fadd_rn(a.x, q[0]); a.y = __fadd_rn(a.y, q[1]);
            a.z = __fadd_rn(a.z, q[2]); a.w = __fadd_rn(a.w, q[3]);
        } else {
            a.x = __fsub_rn(a.x, q[0]); a.y = __fsub_rn(a.y, q[1]);
            a.z = __fsub_rn(a.z, q[2]); a.w = __fsub_rn(a.w, q[3]);
        }
        hp[0] = a;
    } else {
        static_assert(std::is_same<HT, int32_t>::value, "dense integer fields are int32");
        int4 *hp = reinterpret_cast<int4 *>(h);
#pragma unroll
        for (int g = 0; g < VE / 4; ++g) {
            int4 a = hp[g];
            const int32_t s0 = q[4 * g + 0], s1 = q[4 * g + 1], s2 = q[4 * g + 2], s3 = q[4 * g + 3];
            if (up) { a.x += s0; a.y += s1; a.z += s2; a.w += s3; }
            else    { a.x -= s0; a.y -= s1; a.z -= s2; a.w -= s3; }
            hp[g] = a;
        }
    }
}

// The race exponential of position t: -ln(1 - V), V the fine uniform of
// Philox word t of (RACE, chain, step).
__device__ __forceinline__ float race_exp(uint32_t word) { return det_neg_log1m(u01_fine(word)); }

// Race key E / w (Proposition 5).  Exact for every normal w; for w = 0,
// subnormal w or a key past the fp32 range the result is +inf or NaN, whose
// bits exceed every finite key, as IEEE's +inf or huge quotient does there:
// the least key, the anchor's E <= 16.7, is unchanged.
__device__ __forceinline__ float race_key(float e, float w) { return div_rn_pos(e, w); }

// Scalars of one record that do not depend on the chain state.
struct RecordDraws {
    float e1;      // Exp(1) of the multiplicity, from STEP words 0 and 1
    int32_t mi;    // Metropolis proposal index (STEP word 2)
    float mlu;     // Metropolis log-uniform (STEP word 3)
};

__device__ __forceinline__ RecordDraws record_draws(uint64_t seed, uint32_t chain, uint64_t step, int n,
                                                    bool metropolis = true, bool race = true) {
    const uint4 w = rng_block(seed, TAG_STEP, chain, step, 0);
    RecordDraws d;
    d.e1 = race ? -det_logf(u01_fine64((static_cast<uint64_t>(w.y) << 32) | static_cast<uint64_t>(w.x))) : 0.0f;
    d.mi = static_cast<int32_t>(__umulhi(w.z, static_cast<uint32_t>(n)));
    d.mlu = metropolis ? det_logf(u01_grid(w.w)) : 0.0f;
    return d;
}

// Multiplicity from the reduced weight sum S, the anchor and a ready Exp(1).
// (e^{-beta 0} = 1 exactly, so the anchor exponential is skipped at A = 0.)
// M = floor(g) + 1 is returned twice: as an integer (exact while g < 2^24,
// which covers every budget test of Unbiased PNS with L0 < 2^24) for the
// critical path, and as the fp64 record value.  GB300's fp64 pipe has a
// 64-cycle latency, so nothing on the per-record chain waits for the double.
struct Mult {
    int64_t mi;    // M when M < 2^24 + 1 (else -1)
    float fgl;     // large M: floor(g) = M - 1 (an integer in fp32); +inf when saturated
    int sat;
};

// M as recorded (fp64), formed only where it is needed (tape, sums): the
// fp64 pipe is narrow on GB300, so the decision path avoids it.
__device__ __forceinline__ double mult_md(const Mult &mu) {
    if (mu.mi >= 0) return static_cast<double>(static_cast<int32_t>(mu.mi));
    if (mu.sat) return 9223372036854775808.0;
    return __dadd_rn(static_cast<double>(mu.fgl), 1.0);
}

// M <= L for a budget 0 <= L < 2^31, in 32-bit arithmetic: every M that can
// fit is then below 2^31 and exact in fp32's integer range used here, so the
// result equals the fp64 comparison of mult_fits.
__device__ __forceinline__ bool mult_fits_small(const Mult &mu, int32_t L) {
    if (mu.mi >= 0) return mu.mi <= L;
    return !mu.sat && mu.fgl < 2147483648.0f && __float2int_rz(mu.fgl) < L;
}

// M <= L for a budget L >= 0, compared as the fp64 record value (as the
// specification does); fp64 is touched only in the rare large-M branch.
__device__ __forceinline__ bool mult_fits(const Mult &mu, int64_t L) {
    if (mu.mi >= 0) return mu.mi <= L;
    return mult_md(mu) <= static_cast<double>(L);
}

// Round-to-nearest-even conversion of an unsigned 64-bit integer to fp32 with
// 32-bit integer operations only (GB300 runs 64-bit int<->float conversions on
// its slow fp64 pipe), branch-free: v is normalised so that its leading one
// sits at bit 63, the top 24 bits are kept and rounded by the 40 dropped ones
// (half way: to even), and the result is scaled back by an exact power of 2.
// Equal to __ull2float_rn for every input.
__device__ __forceinline__ float u64_to_f32_rn(uint64_t v) {
    const int z = __clzll(static_cast<long long>(v)) & 63;  // (v = 0 takes the select below)
    const uint64_t nv = v << z;
    const uint32_t top = static_cast<uint32_t>(nv >> 40);
    const uint64_t rest = nv << 24;  // the dropped bits, at the top
    const bool up = rest > 0x8000000000000000ull || (rest == 0x8000000000000000ull && (top & 1u));
    const uint32_t m = top + (up ? 1u : 0u);  // <= 2^24, exact in fp32
    const float r = __fmul_rn(__uint2float_rn(m), pow2f(40 - z));
    return v == 0ull ? 0.0f : r;
}

// The multiplicity splits into a part fixed by the state and the set (the
// move probability p = S 2^-32 / k * e^{-beta A}, and -ln(1 - p)) and a part
// drawn per record (the Exp(1) e1): M = 1 + floor(e1 / -ln(1 - p)), i.e.
// 1 + Geom(p).  anchor_f = e^{-beta A} (1 when A = 0).
__device__ __forceinline__ float mult_p(uint64_t S, int32_t k, float anchor_f) {
    float ps = __fmul_rn(u64_to_f32_rn(S), 0x1p-32f);
    ps = div_rn_pos(ps, __int2float_rn(k));  // (ps >= 1: the anchor's weight is 1)
    return __fmul_rn(ps, anchor_f);
}

// M from p, c = -ln(1 - p) (read only when 0 < p < 1) and e1: p >= 1 gives
// M = 1, p <= 0 saturates, else g = e1 / c saturates at 2^63 (NaN included)
// and M = floor(g) + 1.  Branch-free: every case is evaluated and selected.
// (c normal: g exact wherever g < 2^63; c subnormal or g past the fp32 range:
// a quotient at or above 2^63 or NaN, saturated, as IEEE's would be.)
__device__ __forceinline__ Mult mult_from(float p, float c, float e1) {
    const float g = div_rn_pos(e1, c);
    const float fg = floorf(g);
    const bool one = p >= 1.0f;
    const bool sat = !one && (p <= 0.0f || !(g < 0x1p63f));
    const bool small = fg < 16777216.0f;  // (false for NaN)
    Mult r;
    r.sat = sat ? 1 : 0;
    const int64_t mi_g = small ? static_cast<int64_t>(__float2int_rz(fg)) + 1 : -1;
    r.mi = one ? 1 : (sat ? -1 : mi_g);
    r.fgl = one ? 0.0f : (sat ? __int_as_float(0x7f800000) : (small ? 0.0f : fg));
    return r;
}

__device__ __forceinline__ Mult multiplicity_e1(uint64_t S, int32_t k, float anchor_f, float e1) {
    const float p = mult_p(S, k, anchor_f);
    const float c = det_neg_log1m(p);  // (a value for every p; used only when 0 < p < 1)
    return mult_from(p, c, e1);
}

// beta / T(k) for record k of the cooling schedule of Algorithms 8-10: beta
// s0^(1 - k/K) for k < K, in fp32 as det_exp(ln(s0) (1 - k/K)) with IEEE
// division and products; beta itself when K = 0 or k >= K.
__device__ __forceinline__ float anneal_beta(float beta, float ln_s0, int64_t K, int64_t k) {
    if (K <= 0 || k >= K) return beta;
    const float r = __fdiv_rn(__ll2float_rn(k), __ll2float_rn(K));
    return __fmul_rn(beta, det_expf(__fmul_rn(ln_s0, __fsub_rn(1.0f, r))));
}

// First k distinct values of v_m = floor(word_m n / 2^32), m = 0, 1, ...,
// drawn by one warp into `list`.  Returns false when the draw cap is hit:
// 64 n + 1024 draws, or `cap_limit` when that is smaller and nonzero (a
// host-set limit that lets tests make this bounded loop give up).
__device__ __forceinline__ bool draw_subset_warp(uint64_t seed, uint32_t chain, uint64_t sstep, int n, int k,
                                                 int ld, int32_t *list, uint32_t *bitmap, int lane,
                                                 uint32_t cap_limit = 0u) {
    for (int w = lane; w < ld / 32; w += 32) bitmap[w] = 0u;
    __syncwarp();
    uint32_t cap = 64u * static_cast<uint32_t>(n) + 1024u;
    if (cap_limit != 0u && cap_limit < cap) cap = cap_limit;
    int got = 0;
    uint32_t m0 = 0;
    while (got < k) {
        const uint32_t m = m0 + lane;
        const bool valid = m < cap;
        const uint32_t word = rng_word(seed, TAG_SUBSET, chain, sstep, m);
        const uint32_t v = __umulhi(word, static_cast<uint32_t>(n));
        const uint32_t eq = __match_any_sync(0xFFFFFFFFu, valid ? v : 0xFFFFFFFFu);
        const bool first = (__ffs(eq) - 1) == lane;
        const bool seen = (bitmap[v >> 5] >> (v & 31u)) & 1u;
        const bool acc = valid && first && !seen;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, acc);
        const int rank = got + __popc(bal & ((1u << lane) - 1u));
        if (acc && rank < k) list[rank] = static_cast<int32_t>(v);
        if (acc) atomicOr(&bitmap[v >> 5], 1u << (v & 31u));
        got += __popc(bal);
        m0 += 32;
        __syncwarp();
        if (got < k && m0 >= cap) {
            // give up, leaving every list entry a valid bit index (a kernel
            // that evaluates the record before it checks the status reads
            // only in-range fields)
            for (int t = got + lane; t < k; t += 32) list[t] = 0;
            __syncwarp();
            return false;
        }
    }
    return true;
}

constexpr int CPT = 4;  // candidates per consumer thread kept in registers
constexpr int PF = 8;   // row chunks per consumer thread loaded ahead of the move

// ---------------------------------------------------------------------------
// The kernel.  TC consumer warps per chain; P.prod producer warps (0 or 1).
// ---------------------------------------------------------------------------
template <typename QT, typename HT, int TC, bool CSR>
__global__ void __launch_bounds__(TC == 32 ? 1024 : 512) pns_sample_kernel(const KParams P) {
    using A = Arith<HT>;
    using D = typename A::D;
    using CT = typename A::C;
    constexpr int TCC = 32 * TC;  // consumer threads per team

    extern __shared__ __align__(16) unsigned char smem[];
    const CtaDesc cd = P.cta[blockIdx.x];
    const int prod = P.prod;
    const int TT = TCC + 32 * prod;  // team threads
    const int team = threadIdx.x / TT;
    if (team >= cd.count) return;  // idle warps take part in no barrier
    const int tid = threadIdx.x - team * TT;
    const int lane = threadIdx.x & 31;
    const int wit = tid >> 5;
    const bool consumer = wit < TC;
    const int cid = P.cta_chains[cd.first + team];
    const ChainDesc chd = P.chain[cid];
    const InstDesc in = P.inst[chd.inst];
    const int n = in.n;
    const int ld = in.ld;
    const int variant = P.variant;
    const bool use_list = needs_list(variant, P.subset);
    const bool slot_list = prod > 0 && variant == VAR_BASIC;
    const int k = (variant == VAR_RF) ? n : (variant == VAR_METROPOLIS ? 1 : in.k);

    const ChainSmem L = chain_smem(ld, k, static_cast<int32_t>(sizeof(HT)), use_list, prod > 0, slot_list);
    unsigned char *base = smem + chd.smem_off;
    HT *h = reinterpret_cast<HT *>(base + L.fields);
    uint32_t *xw = reinterpret_cast<uint32_t *>(base + L.xw);
    int32_t *list = reinterpret_cast<int32_t *>(base + L.list);
    uint32_t *bitmap = reinterpret_cast<uint32_t *>(base + L.bitmap);
    uint32_t *red = reinterpret_cast<uint32_t *>(base + L.scratch);  // [5][32]
    double *pub_E = reinterpret_cast<double *>(base + L.scratch + 640);
    int32_t *pub_b = reinterpret_cast<int32_t *>(base + L.scratch + 648);
    int32_t *swap_cnt = reinterpret_cast<int32_t *>(base + L.scratch + 652);
    int32_t *dead_slot = reinterpret_cast<int32_t *>(base + L.scratch + 656);
    // "another record follows", one word per record parity: the consumers
    // write record r's word before the barrier ending r; the producer reads it
    // after that barrier, and the same word is rewritten only after the
    // producer has reached the next barrier.
    int32_t *more_slot = reinterpret_cast<int32_t *>(base + L.scratch + 660);

    const CT *bvec = reinterpret_cast<const CT *>(in.b);
    const CT *dvec = reinterpret_cast<const CT *>(in.diag);

    // named barriers: 1 + 2 team (whole team), 2 + 2 team (consumers), then groups
    const int bar_all = 1 + 2 * team;
    const int bar_cons = 2 + 2 * team;
    auto sync_all = [&]() {
        if (TT == 32) __syncwarp();
        else named_sync(bar_all, TT);
    };
    auto sync_cons = [&]() {
        if constexpr (TC == 1) __syncwarp();
        else named_sync(bar_cons, TCC);
    };

    // ---- load the chain ----------------------------------------------------
    {
        const HT *gh = reinterpret_cast<const HT *>(P.fields) + static_cast<int64_t>(cid) * P.LD;
        const uint32_t *gx = P.xbits + static_cast<int64_t>(cid) * P.W;
        const int hchunks = ld * static_cast<int>(sizeof(HT)) / 16;
        for (int c = tid; c < hchunks; c += TT)
            reinterpret_cast<uint4 *>(h)[c] = reinterpret_cast<const uint4 *>(gh)[c];
        for (int w = tid; w < ld / 32; w += TT) xw[w] = gx[w];
    }
    if (tid == 0) {
        *swap_cnt = 0;
        *dead_slot = 0;
        more_slot[0] = 1;
        more_slot[1] = 1;
    }
    ChainState st = P.state[cid];
    const uint64_t seed = P.seed;
    const uint32_t chain_id = static_cast<uint32_t>(cid) + P.chain_base;
    sync_all();

    // ---- producer: state-independent draws for record `step` into slot `s` --
    // Race numbers go one per lane over the first max(1, prod - 1) producer
    // warps; the last producer warp draws the record scalars (and Basic's
    // subset), so the two kinds of work do not diverge inside one warp.
    auto produce = [&](int s, uint64_t step) {
        unsigned char *slot = base + L.slots + s * L.slot_bytes;
        float *ex = reinterpret_cast<float *>(slot + 16);
        const int ptid = tid - TCC;
        const int race_warps = prod > 1 ? prod - 1 : 1;
        if (ptid < 32 * race_warps) {
            for (int t = ptid; t < k; t += 32 * race_warps)
                ex[t] = race_exp(rng_word(seed, TAG_RACE, chain_id, step, static_cast<uint32_t>(t)));
        }
        if (wit == TC + prod - 1 && lane == 0) {
            const RecordDraws d = record_draws(seed, chain_id, step, n);
            reinterpret_cast<float *>(slot)[0] = d.e1;
            reinterpret_cast<int32_t *>(slot)[1] = d.mi;
            reinterpret_cast<float *>(slot)[2] = d.mlu;
        }
        if (slot_list && wit == TC + prod - 1) {
            int32_t *sl = reinterpret_cast<int32_t *>(slot + 16 + 4 * k);
            const bool ok = draw_subset_warp(seed, chain_id, step, n, k, ld, sl, bitmap, lane, P.draw_cap);
            if (lane == 0) reinterpret_cast<int32_t *>(slot)[3] = ok ? 0 : 1;
        }
    };

    if (!consumer) {
        // The producer runs one record ahead of the consumers; it leaves when
        // they report that no record follows.
        uint64_t step = static_cast<uint64_t>(st.step);
        int s = 0;
        produce(0, step);
        sync_all();
        while (true) {
            produce(s ^ 1, step + 1);
            sync_all();  // end of the consumers' record that used slot s
            if (!more_slot[s]) break;
            s ^= 1;
            step += 1;
        }
        return;
    }

    // ---- consumers ------------------------------------------------------------
    const int ctid = tid;
    float beta_chain = in.betas[st.beta_idx];
    const float anneal_ls0 = P.anneal_steps > 0 ? det_logf(P.anneal_start) : 0.0f;
    int dead = 0;
    bool list_valid = false;
    int64_t tape_pos = 0;
    int cur = 0;  // current slot
    if (prod > 0) sync_all();  // slot 0 ready

    auto cand = [&](int t, const int32_t *sl) -> int {
        if (variant == VAR_RF) return t;
        if (use_list) return sl[t];
        int c = st.set_start + t;
        return c >= n ? c - n : c;
    };

    auto delta_of = [&](int i) -> D {
        const bool xi = (xw[i >> 5] >> (i & 31)) & 1u;
        return A::delta(h[i], bvec[i], dvec[i], xi);
    };

    // Dense row j: chunks [0, PF * TCC) are loaded into registers first.
    constexpr int VE = 16 / static_cast<int>(sizeof(QT));
    uint4 pre[PF];
    auto prefetch_row = [&](int j) {
        if constexpr (!CSR) {
            const QT *row = reinterpret_cast<const QT *>(in.q) + static_cast<int64_t>(j) * ld;
            const int chunks = ld / VE;
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int c = ctid + u * TCC;
                if (c < chunks) pre[u] = ld_nc_v4(row + c * VE);
            }
        }
    };

    // Apply the move to bit j (all consumer threads), then flip x_j.
    auto apply_move = [&](int j, bool prefetched) {
        const bool up = ((xw[j >> 5] >> (j & 31)) & 1u) == 0u;
        if constexpr (CSR) {
            const int e0 = in.row_ptr[j], e1 = in.row_ptr[j + 1];
            const QT *vals = reinterpret_cast<const QT *>(in.q);
            for (int e = e0 + ctid; e < e1; e += TCC) {
                const int r = in.col[e];
                const QT qv = vals[e];
                if constexpr (std::is_same<HT, float>::value) {
                    h[r] = up ? __fadd_rn(h[r], qv) : __fsub_rn(h[r], qv);
                } else {
                    h[r] = static_cast<HT>(up ? static_cast<int32_t>(h[r]) + static_cast<int32_t>(qv)
                                              : static_cast<int32_t>(h[r]) - static_cast<int32_t>(qv));
                }
            }
            if (ctid == TCC - 1) {
                const CT dv = dvec[j];
                if constexpr (std::is_same<HT, float>::value) {
                    h[j] = up ? __fadd_rn(h[j], dv) : __fsub_rn(h[j], dv);
                } else {
                    h[j] = static_cast<HT>(up ? static_cast<int32_t>(h[j]) + dv : static_cast<int32_t>(h[j]) - dv);
                }
            }
        } else {
            const QT *row = reinterpret_cast<const QT *>(in.q) + static_cast<int64_t>(j) * ld;
            const int chunks = ld / VE;
            if (!prefetched) prefetch_row(j);
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int c = ctid + u * TCC;
                if (c < chunks) add_chunk<QT, HT>(h + c * VE, pre[u], up);
            }
            // the rest in batches of PF loads in flight per thread
            for (int c0 = ctid + PF * TCC; c0 < chunks; c0 += PF * TCC) {
#pragma unroll
                for (int u = 0; u < PF; ++u) {
                    const int c = c0 + u * TCC;
                    if (c < chunks) pre[u] = ld_nc_v4(row + c * VE);
                }
#pragma unroll
                for (int u = 0; u < PF; ++u) {
                    const int c = c0 + u * TCC;
                    if (c < chunks) add_chunk<QT, HT>(h + c * VE, pre[u], up);
                }
            }
        }
        sync_cons();  // every consumer has read x_j
        if (ctid == 0) xw[j >> 5] ^= 1u << (j & 31);
    };

    // Tape and fp64 accumulators are written one record late, so that the
    // store and the 64-cycle fp64 adds never stall the record that made them.
    int32_t pend_flip = 0;
    double pend_m = 0.0;
    bool pend = false;
    // Unbiased PNS without exchange: its multiplicities are integers <= L0,
    // so their sum is kept exactly in int64 and added to the fp64 sum once
    // at the end (equal to the record-by-record fp64 sum: every partial sum
    // is an integer below 2^53); the fp64 M is formed only for the tape
    const bool int_sum = variant == VAR_UNBIASED && !P.pt;
    int64_t sum_int = 0;
    auto flush_record = [&]() {
        if (pend) {
            if (ctid == 0 && P.tape >= 1 && tape_pos < P.tape_cap) {
                const int64_t o = static_cast<int64_t>(cid) * P.tape_cap + tape_pos;
                P.tape_flip[o] = pend_flip;
                P.tape_m[o] = pend_m;
            }
            tape_pos += 1;
            pend = false;
        }
    };
    auto write_record = [&](int32_t flip, double m) {
        flush_record();
        pend_flip = flip;
        pend_m = m;
        pend = true;
        st.sum_m = __dadd_rn(st.sum_m, m);
    };
    auto write_record_int = [&](int32_t flip, int64_t mi) {  // (int_sum)
        flush_record();
        pend_flip = flip;
        pend_m = P.tape >= 1 && ctid == 0 ? static_cast<double>(mi) : 0.0;  // (only the tape reads it)
        pend = true;
        sum_int += mi;
    };

    // Race exponential of position t in the current record.
    auto ex_of = [&](int t, uint64_t step) -> float {
        if (prod > 0) return reinterpret_cast<const float *>(base + L.slots + cur * L.slot_bytes + 16)[t];
        return race_exp(rng_word(seed, TAG_RACE, chain_id, step, static_cast<uint32_t>(t)));
    };

    // tape = 2: the state a record starts from (the jump-chain sample J that
    // its multiplicity weighs) and its energy
    int64_t rec_started = 0;
    // Without producer warps the record scalars (the multiplicity's Exp(1),
    // Metropolis' proposal and log-uniform) are drawn 32 records at a time,
    // lane l drawing record b + l, and each record takes its own from that
    // lane: the same values, one STEP block per lane per 32 records.
    float bat_e1 = 0.0f, bat_mlu = 0.0f;
    int32_t bat_mi = 0;
    int bat_i = 32;
    auto sample_record = [&]() {
        if (P.tape == 2 && rec_started < P.tape_cap) {
            const int64_t o = static_cast<int64_t>(cid) * P.tape_cap + rec_started;
            uint32_t *tx = P.tape_x + o * P.W;
            for (int q = ctid; q < P.W; q += TCC) tx[q] = q < ld / 32 ? xw[q] : 0u;
            if (ctid == 0) P.tape_E[o] = st.E;
        }
        rec_started += 1;
    };

    // One record.  Returns true when the record was an Unbiased period end.
    auto one_record = [&]() -> bool {
        sample_record();
        const uint64_t step = static_cast<uint64_t>(st.step);
        // the record's inverse temperature: beta / T(k) of the cooling schedule
        // (Algorithms 8-10) for record k = step + 1, else the chain's beta
        const float beta = anneal_beta(beta_chain, anneal_ls0, P.anneal_steps, static_cast<int64_t>(step) + 1);
        const unsigned char *slot = base + L.slots + cur * L.slot_bytes;
        RecordDraws rd;
        if (prod > 0) {
            rd.e1 = reinterpret_cast<const float *>(slot)[0];
            rd.mi = reinterpret_cast<const int32_t *>(slot)[1];
            rd.mlu = reinterpret_cast<const float *>(slot)[2];
        } else {
            if (bat_i == 32) {
                const RecordDraws d = record_draws(seed, chain_id, step + static_cast<uint64_t>(lane), n,
                                                   variant == VAR_METROPOLIS, variant != VAR_METROPOLIS);
                bat_e1 = d.e1;
                bat_mi = d.mi;
                bat_mlu = d.mlu;
                bat_i = 0;
            }
            rd.e1 = __shfl_sync(0xFFFFFFFFu, bat_e1, bat_i);
            rd.mi = __shfl_sync(0xFFFFFFFFu, bat_mi, bat_i);
            rd.mlu = __shfl_sync(0xFFFFFFFFu, bat_mlu, bat_i);
            bat_i += 1;
        }
        bool period_end = false;
        if (variant == VAR_METROPOLIS) {
            const int i = rd.mi;
            const D d = delta_of(i);
            const float y = -__fmul_rn(beta, A::tof(d));
            sync_cons();  // all reads of h / x done before the move
            if (rd.mlu < y) {
                apply_move(i, false);
                st.E = __dadd_rn(st.E, A::tod(d));
                st.flips += 1;
                write_record(i, 1.0);
            } else {
                st.stays += 1;
                write_record(-1, 1.0);
            }
        } else {
            const int32_t *sl = list;
            if (variant == VAR_BASIC) {
                if (prod > 0) {
                    sl = reinterpret_cast<const int32_t *>(slot + 16 + 4 * k);
                    if (reinterpret_cast<const int32_t *>(slot)[3]) {
                        if (ctid == 0) set_status(P.status, ST_TIMEOUT);
                        dead = 1;
                    }
                } else {
                    if (wit == 0 && !draw_subset_warp(seed, chain_id, step, n, k, ld, list, bitmap, lane, P.draw_cap)) {
                        if (lane == 0) {
                            set_status(P.status, ST_TIMEOUT);
                            *dead_slot = 1;
                        }
                    }
                    sync_cons();
                    dead = *dead_slot;
                }
            } else if (use_list && !list_valid) {
                if (wit == 0 &&
                    !draw_subset_warp(seed, chain_id, static_cast<uint64_t>(st.period_start), n, k, ld, list, bitmap,
                                      lane, P.draw_cap)) {
                    if (lane == 0) {
                        set_status(P.status, ST_TIMEOUT);
                        *dead_slot = 1;
                    }
                }
                sync_cons();
                dead = *dead_slot;
                list_valid = true;
            }
            if (dead) return true;
            const bool fast = k <= CPT * TCC;
            // a2 + a3: deltas and the anchor.  Fast path: NP positions per
            // thread, one (k <= TCC) or CPT contiguous ones (one Philox block
            // of race words), evaluated without branches (positions at or
            // past k read position k - 1 and are masked)
            // (one position per thread only for one-warp teams: wider teams
            // serve large k, and the second code path costs them registers)
            const bool one_pos = TC == 1 && k <= TCC;  // (the same for the whole team)
            D dl[CPT];
            uint32_t lmin = 0xFFFFFFFFu;
            auto pos_of = [&](auto np_c, int u) {
                constexpr int NP = decltype(np_c)::value;
                return NP == 1 ? ctid : CPT * ctid + u;
            };
            auto deltas = [&](auto np_c) {
                constexpr int NP = decltype(np_c)::value;
#pragma unroll
                for (int u = 0; u < NP; ++u) {
                    const int t = pos_of(np_c, u);
                    dl[u] = delta_of(cand(t < k ? t : k - 1, sl));
                    const uint32_t kd = A::key(A::pos(dl[u]));
                    lmin = t < k && kd < lmin ? kd : lmin;
                }
            };
            if (fast) {
                if (one_pos) deltas(std::integral_constant<int, 1>{});
                else deltas(std::integral_constant<int, CPT>{});
            } else {
                for (int t = ctid; t < k; t += TCC) {
                    const uint32_t kd = A::key(A::pos(delta_of(cand(t, sl))));
                    lmin = kd < lmin ? kd : lmin;
                }
            }
            uint32_t amin_k = __reduce_min_sync(0xFFFFFFFFu, lmin);
            if constexpr (TC > 1) {
                if (lane == 0) red[0 * 32 + wit] = amin_k;
                sync_cons();
                amin_k = red[0];
#pragma unroll 4
                for (int w = 1; w < TC; ++w) amin_k = red[w] < amin_k ? red[w] : amin_k;
            }
            const D amin = A::unkey(amin_k);
            // a4: weights, race, quantised sum
            uint32_t bkey = 0xFFFFFFFFu, bpos = 0xFFFFFFFFu, sa = 0u, sb = 0u;
            // e^{-beta A} for the multiplicity, independent of the visits below
            const float af = A::tof(amin);
            const float anchor_e = det_expf(-__fmul_rn(beta, af));
            const float anchor_f = af > 0.0f ? anchor_e : 1.0f;
            auto visit = [&](int t, D dv) {
                const float w = det_expf(-__fmul_rn(beta, A::diff(A::pos(dv), amin)));
                // floor(w 2^32) as (floor(w 2^16), next 16 bits), all exact in fp32
                const float ws = __fmul_rn(w, 65536.0f);
                const float wa = truncf(ws);
                sa += __float2uint_rz(wa);
                sb += __float2uint_rz(__fmul_rn(__fsub_rn(ws, wa), 65536.0f));
                const uint32_t kb = __float_as_uint(race_key(ex_of(t, step), w));
                if (kb < bkey) {  // t ascending per thread: the first minimum is kept
                    bkey = kb;
                    bpos = static_cast<uint32_t>(t);
                }
            };
            // race exponentials: from the producer's slot, or from the
            // thread's one Philox block (position ctid: block ctid / 4; CPT =
            // 4 positions from 4 ctid: block ctid)
            static_assert(CPT == 4, "one Philox block per thread");
            auto weigh = [&](auto np_c) {
                constexpr int NP = decltype(np_c)::value;
                float exv[NP];
                if (prod > 0) {
#pragma unroll
                    for (int u = 0; u < NP; ++u) {
                        const int t = pos_of(np_c, u);
                        exv[u] = ex_of(t < k ? t : k - 1, step);
                    }
                } else if constexpr (NP == 1) {
                    const uint4 blk = rng_block(seed, TAG_RACE, chain_id, step, static_cast<uint32_t>(ctid >> 2));
                    exv[0] = race_exp(pick_word(blk, static_cast<uint32_t>(ctid & 3)));
                } else {
                    const uint4 blk = rng_block(seed, TAG_RACE, chain_id, step, static_cast<uint32_t>(ctid));
                    exv[0] = race_exp(blk.x);
                    exv[1] = race_exp(blk.y);
                    exv[2] = race_exp(blk.z);
                    exv[3] = race_exp(blk.w);
                }
#pragma unroll
                for (int u = 0; u < NP; ++u) {
                    const int t = pos_of(np_c, u);
                    const float ex = exv[u];
                    const float w = det_expf(-__fmul_rn(beta, A::diff(A::pos(dl[u]), amin)));
                    const float ws = __fmul_rn(w, 65536.0f);
                    const float wa = truncf(ws);
                    const uint32_t qa = __float2uint_rz(wa);
                    const uint32_t qb = __float2uint_rz(__fmul_rn(__fsub_rn(ws, wa), 65536.0f));
                    sa += t < k ? qa : 0u;
                    sb += t < k ? qb : 0u;
                    const uint32_t kb = t < k ? __float_as_uint(race_key(ex, w)) : 0xFFFFFFFFu;
                    const bool better = kb < bkey;  // t ascending per thread: the first minimum is kept
                    bkey = better ? kb : bkey;
                    bpos = better ? static_cast<uint32_t>(t) : bpos;
                }
            };
            if (fast) {
                if (one_pos) weigh(std::integral_constant<int, 1>{});
                else weigh(std::integral_constant<int, CPT>{});
            } else {
                for (int t = ctid; t < k; t += TCC) visit(t, delta_of(cand(t, sl)));
            }
            uint32_t wkey = __reduce_min_sync(0xFFFFFFFFu, bkey);
            uint32_t wpos = __reduce_min_sync(0xFFFFFFFFu, bkey == wkey ? bpos : 0xFFFFFFFFu);
            const uint32_t SA = __reduce_add_sync(0xFFFFFFFFu, sa);
            const uint32_t SB = __reduce_add_sync(0xFFFFFFFFu, sb);
            uint64_t S;
            if constexpr (TC > 1) {
                if (lane == 0) {
                    red[1 * 32 + wit] = wkey;
                    red[2 * 32 + wit] = wpos;
                    red[3 * 32 + wit] = SA;
                    red[4 * 32 + wit] = SB;
                }
                sync_cons();
                wkey = red[32];
                wpos = red[64];
                uint64_t SA64 = red[96], SB64 = red[128];
                for (int w = 1; w < TC; ++w) {
                    const uint32_t kk = red[32 + w], pp = red[64 + w];
                    if (kk < wkey || (kk == wkey && pp < wpos)) {
                        wkey = kk;
                        wpos = pp;
                    }
                    SA64 += red[96 + w];
                    SB64 += red[128 + w];
                }
                S = (SA64 << 16) + SB64;
            } else {
                S = (static_cast<uint64_t>(SA) << 16) + static_cast<uint64_t>(SB);
            }
            const int j = cand(static_cast<int>(wpos), sl);
            // Basic and RF always move: start the row load before the multiplicity.
            // For Unbiased PNS the load is speculative when P.prefetch is set
            // (rows from HBM, where the latency matters more than the bytes).
            const bool always_move = variant != VAR_UNBIASED || P.prefetch;
            if (always_move) prefetch_row(j);
            // a5: multiplicity and budget
            const Mult mu = multiplicity_e1(S, k, anchor_f, rd.e1);
            const int sat = mu.sat;
            const D dj = delta_of(j);
            sync_cons();  // reads of h, x and the list are done
            bool move = true;
            if (int_sum) {
                // the budget test in integers (fp64 only for a huge M)
                const bool fits = mult_fits(mu, st.L);
                int64_t mrec;
                if (fits) {
                    mrec = mu.mi >= 0 ? mu.mi : static_cast<int64_t>(mult_md(mu));
                    st.L -= mrec;
                    if (sat) st.saturated += 1;
                    apply_move(j, always_move);
                    st.E = __dadd_rn(st.E, A::tod(dj));
                    st.flips += 1;
                    write_record_int(j, mrec);
                } else {
                    mrec = st.L;
                    st.L = P.L0;
                    st.stays += 1;
                    int ns = st.set_start + k;
                    while (ns >= n) ns -= n;
                    st.set_start = ns;
                    st.period_start = static_cast<int64_t>(step) + 1;
                    list_valid = false;
                    period_end = true;
                    write_record_int(-1, mrec);
                }
            } else {
                double m = mult_md(mu);
                if (variant == VAR_UNBIASED) {
                    const bool fits = mu.mi >= 0 ? mu.mi <= st.L : m <= static_cast<double>(st.L);
                    if (fits) {
                        st.L -= mu.mi >= 0 ? mu.mi : static_cast<int64_t>(m);
                    } else {
                        move = false;
                        m = static_cast<double>(st.L);
                        st.L = P.L0;
                        st.stays += 1;
                        int ns = st.set_start + k;
                        while (ns >= n) ns -= n;
                        st.set_start = ns;
                        st.period_start = static_cast<int64_t>(step) + 1;
                        list_valid = false;
                        period_end = true;
                    }
                }
                if (move) {
                    if (sat) st.saturated += 1;
                    apply_move(j, always_move);
                    st.E = __dadd_rn(st.E, A::tod(dj));
                    st.flips += 1;
                    write_record(j, m);
                } else {
                    write_record(-1, m);
                }
            }
        }
        const bool improved = st.E < st.best_E;  // (the same for every thread of the team)
        if (improved) st.best_E = st.E;
        st.step += 1;
        sync_cons();
        if (improved && P.xbest) {
            // X_max (Algorithms 8-10): the state after this record; the next
            // change of the bits comes after a team barrier
            uint32_t *xb = P.xbest + static_cast<int64_t>(cid) * P.W;
            for (int q = ctid; q < P.W; q += TCC) xb[q] = q < ld / 32 ? xw[q] : 0u;
        }
        return period_end;
    };

    // Ends a record: tell the producer whether another one follows.
    auto end_record = [&](bool more) {
        if (prod > 0) {
            if (ctid == 0) more_slot[cur] = more ? 1 : 0;
            sync_all();
            cur ^= 1;
        }
    };

    // ---- main loop -----------------------------------------------------------
    if (!P.pt) {
        if (P.steps <= 0) end_record(false);
        for (int64_t r = 0; r < P.steps; ++r) {
            one_record();
            const bool more = r + 1 < P.steps && !dead;
            end_record(more);
            if (!more) break;
        }
    } else {
        const int R = P.R;
        // named barrier of the exchange group, after the ids the teams use
        const int gbar = (TT > 32 ? 1 + 2 * cd.count : 1) + team / R;
        const int gthreads = R * TCC;
        const int64_t rounds = P.steps / P.swap_interval;
        const int64_t per_round = variant == VAR_UNBIASED ? P.swap_interval / P.L0 : P.swap_interval;
        if (rounds <= 0) end_record(false);
        for (int64_t rdi = 0; rdi < rounds; ++rdi) {
            int64_t done = 0;
            while (done < per_round) {
                const bool pend = dead ? true : one_record();
                if (variant != VAR_UNBIASED || pend) done += 1;
                if (done == per_round) {
                    // exchange round among the R replicas of this group
                    if (ctid == 0) {
                        *pub_E = st.E;
                        *pub_b = st.beta_idx;
                    }
                    named_sync(gbar, gthreads);
                    if (chd.slot == 0 && ctid == 0) {
                        const uint64_t ndone =
                            static_cast<uint64_t>(st.sum_m) / static_cast<uint64_t>(P.swap_interval);
                        const uint64_t rnd = ndone - 1;
                        int slot_of[32];
                        for (int s2 = 0; s2 < R; ++s2) {
                            const int oc = P.cta_chains[cd.first + team + s2];
                            const unsigned char *ob = smem + P.chain[oc].smem_off;
                            slot_of[*reinterpret_cast<const int32_t *>(ob + L.scratch + 648)] = s2;
                        }
                        int q = 0;
                        for (int a = static_cast<int>(rnd & 1u); a + 1 < R; a += 2, ++q) {
                            const int sa_ = slot_of[a], sb_ = slot_of[a + 1];
                            const int ca = P.cta_chains[cd.first + team + sa_];
                            const int cb = P.cta_chains[cd.first + team + sb_];
                            unsigned char *pa = smem + P.chain[ca].smem_off + L.scratch;
                            unsigned char *pb = smem + P.chain[cb].smem_off + L.scratch;
                            const double Ea = *reinterpret_cast<double *>(pa + 640);
                            const double Eb = *reinterpret_cast<double *>(pb + 640);
                            const float db = __fsub_rn(in.betas[a], in.betas[a + 1]);
                            const float de = __double2float_rn(__dsub_rn(Ea, Eb));
                            const float xr = __fmul_rn(db, de);
                            const uint32_t w = rng_word(seed, TAG_SWAP, static_cast<uint32_t>(chd.group) + P.group_base, rnd,
                                                        static_cast<uint32_t>(q));
                            if (det_logf(u01_grid(w)) < xr) {
                                *reinterpret_cast<int32_t *>(pa + 648) = a + 1;
                                *reinterpret_cast<int32_t *>(pb + 648) = a;
                                slot_of[a] = sb_;
                                slot_of[a + 1] = sa_;
                                atomicAdd(reinterpret_cast<int32_t *>(pa + 652), 1);
                                atomicAdd(reinterpret_cast<int32_t *>(pb + 652), 1);
                            }
                        }
                    }
                    named_sync(gbar, gthreads);
                    st.beta_idx = *pub_b;
                    st.swaps += *swap_cnt;
                    sync_cons();
                    if (ctid == 0) *swap_cnt = 0;
                    beta_chain = in.betas[st.beta_idx];
                }
                end_record(!(done == per_round && rdi + 1 == rounds));
            }
        }
    }

    // ---- write the chain back (consumers) --------------------------------------
    flush_record();
    sync_cons();
    {
        HT *gh = reinterpret_cast<HT *>(P.fields) + static_cast<int64_t>(cid) * P.LD;
        uint32_t *gx = P.xbits + static_cast<int64_t>(cid) * P.W;
        const int hchunks = ld * static_cast<int>(sizeof(HT)) / 16;
        for (int c = ctid; c < hchunks; c += TCC)
            reinterpret_cast<uint4 *>(gh)[c] = reinterpret_cast<const uint4 *>(h)[c];
        for (int w = ctid; w < ld / 32; w += TCC) gx[w] = xw[w];
    }
    if (ctid == 0) {
        st.sum_m = __dadd_rn(st.sum_m, static_cast<double>(sum_int));
        st.tape_records = tape_pos < P.tape_cap ? tape_pos : P.tape_cap;
        if (!P.tape) st.tape_records = 0;
        P.state[cid] = st;
    }
}

}  // namespace pnsk
