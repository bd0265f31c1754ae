// pns_block.cuh -- period-blocked Unbiased PNS with replica exchange.
//
// Within one period of Unbiased PNS (Algorithm 6) a chain proposes and flips
// only bits of its current systematic set N_i, so only the k fields of N_i are
// ever read.  This kernel keeps those k fields in shared memory, current from
// the k x k sub-block Q[N_i, N_i], and logs the period's flips; every other
// field (in global memory) receives the logged rows once the chain's period is
// over, when all rows are known and can be loaded together instead of one
// dependent row load per flip.  Each field still receives the same IEEE
// additions in the same order as with the per-flip update (h_r += s_j Q_rj
// over the flips j in time order), so fields, energies and records are
// bit-identical to the per-flip kernel for integer and fp32 QUBOs alike.
//
// The replicas of an exchange group move through the same systematic sets
// (each completes one period per L0 original samples and the group meets at
// every period end), so one sub-block serves the whole group.  A group of R
// chains is served by W <= R warps.  Per period:
//   records   the warps take the group's chains from a queue, hottest first
//             (ordered by the records each temperature took in the previous
//             period), and run each to its period end; a move updates the k
//             set fields from the sub-block, appends (j, direction) to the
//             chain's log and prefetches row j into L2
//   finalise  a warp that ends a chain while others still run applies that
//             chain's log to its fields outside N_i and gathers the next
//             set's fields; the chain that ends last is finalised by the
//             whole group
//   exchange  at round ends adjacent temperatures swap, as in the per-flip
//             kernel (same random numbers and arithmetic)
// while the next set's sub-block arrives by cp.async.
#pragma once

#include "pns_sampler.cuh"

namespace pnsk {

constexpr int APPLY_U = 4;  // logged rows in flight per thread

template <typename QT, typename HT>
__device__ __forceinline__ HT add_elem(HT h, QT q, bool up) {
    if constexpr (std::is_same<HT, float>::value) {
        return up ? __fadd_rn(h, q) : __fsub_rn(h, q);
    } else {
        return up ? h + static_cast<int32_t>(q) : h - static_cast<int32_t>(q);
    }
}

// Global loads and stores of the chains' fields at the L2 only (.cg): the
// fields are touched once per period, and keeping them out of L1 leaves L1 to
// the record loop's own data.
__device__ __forceinline__ uint4 ld_cg_v4(const void *p) {
    uint4 v;
    asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_cg_v4(void *p, const uint4 &v) {
    asm volatile("st.global.cg.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}

// h + s q for s in {+1, -1}: fp32 as fma(s, q, h), one rounding of the
// exact h +- q (signed zeros included), equal to add_elem; integers exact.
template <typename QT, typename HT>
__device__ __forceinline__ HT add_signed(HT h, QT q, int s) {
    if constexpr (std::is_same<HT, float>::value) {
        return __fmaf_rn(static_cast<float>(s), q, h);
    } else {
        return h + s * static_cast<int32_t>(q);
    }
}

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async4_s(uint32_t smem_dst, const void *gmem_src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_dst), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The 16-byte chunks q = q0, q0 + dq, ... of Q columns for one chain: each
// applies `len` logged flips, in log order, to the chain's global fields hg
// outside the window [s_prev, s_prev + k) (mod n), then, when insf is given,
// copies the fields of the window [s_next, s_next + k) into insf (the next
// set's fields).  A log entry is the flipped bit j, with the sign bit set for
// a 0 -> 1 flip.  Only chunks that touch a window or the end of the row need
// per-element masks.
template <typename QT, typename HT>
__device__ __noinline__ void apply_log(const QT *Q, int ld, HT *hg, const int32_t *log, int len, int q0, int dq,
                                       int s_prev, int s_next, int k, int n, HT *insf) {
    constexpr int VE = 16 / static_cast<int>(sizeof(QT));
    const int nch = ld / VE;
    for (int q = q0; q < nch; q += dq) {
        const int r0 = q * VE;
        int d0 = r0 - s_prev;
        if (d0 < 0) d0 += n;
        int e0 = r0 - s_next;
        if (e0 < 0) e0 += n;
        const bool inside = r0 + VE <= n;
        uint32_t mask, nmask;
        if (inside && d0 >= k && d0 + VE <= n) {
            mask = (1u << VE) - 1u;  // no element of the old window
        } else {
            mask = 0u;
#pragma unroll
            for (int e = 0; e < VE; ++e) {
                int d = d0 + e;
                if (d >= n) d -= n;
                if (r0 + e < n && d >= k) mask |= 1u << e;
            }
        }
        if (!insf || (inside && e0 >= k && e0 + VE <= n)) {
            nmask = 0u;  // no element of the next window
        } else {
            nmask = 0u;
#pragma unroll
            for (int e = 0; e < VE; ++e) {
                int d = e0 + e;
                if (d >= n) d -= n;
                if (r0 + e < n && d < k) nmask |= 1u << e;
            }
        }
        if (len == 0) mask = 0u;
        if (mask == 0u && nmask == 0u) continue;
        HT acc[VE];
#pragma unroll
        for (int g = 0; g < VE / 4; ++g) *reinterpret_cast<uint4 *>(acc + 4 * g) = ld_cg_v4(hg + r0 + 4 * g);
        if (mask) {
            // h_r + s q_r, s = +1 or -1, as one fma (s q is exact, so the
            // sum is rounded once, as the per-flip addition rounds it)
            HT nv[VE];
#pragma unroll
            for (int e = 0; e < VE; ++e) nv[e] = acc[e];
            for (int t0 = 0; t0 < len; t0 += APPLY_U) {
                uint4 v[APPLY_U];
                int sg[APPLY_U];
#pragma unroll
                for (int u = 0; u < APPLY_U; ++u) {
                    if (t0 + u < len) {
                        const int32_t ent = log[t0 + u];
                        sg[u] = ent < 0 ? 1 : -1;
                        v[u] = ld_nc_v4(Q + static_cast<int64_t>(ent & 0x7FFFFFFF) * ld + r0);
                    }
                }
#pragma unroll
                for (int u = 0; u < APPLY_U; ++u) {
                    if (t0 + u < len) {
                        QT qv[VE];
                        *reinterpret_cast<uint4 *>(qv) = v[u];
#pragma unroll
                        for (int e = 0; e < VE; ++e) nv[e] = add_signed<QT, HT>(nv[e], qv[e], sg[u]);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < VE; ++e) acc[e] = ((mask >> e) & 1u) ? nv[e] : acc[e];
#pragma unroll
            for (int g = 0; g < VE / 4; ++g) st_cg_v4(hg + r0 + 4 * g, *reinterpret_cast<const uint4 *>(acc + 4 * g));
        }
        if (nmask) {
#pragma unroll
            for (int e = 0; e < VE; ++e) {
                if ((nmask >> e) & 1u) {
                    int dn = e0 + e;
                    if (dn >= n) dn -= n;
                    insf[dn] = acc[e];
                }
            }
        }
    }
}

__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// PPL consecutive elements at p (aligned to their total size) into v.
template <int PPL, typename T>
__device__ __forceinline__ void ld_vec(const T *p, T (&v)[PPL]) {
    constexpr int B = PPL * static_cast<int>(sizeof(T));
    static_assert(B == 2 || B == 4 || B == 8 || B == 16, "vector width");
    if constexpr (B == 16) *reinterpret_cast<uint4 *>(v) = *reinterpret_cast<const uint4 *>(p);
    else if constexpr (B == 8) *reinterpret_cast<uint2 *>(v) = *reinterpret_cast<const uint2 *>(p);
    else if constexpr (B == 4) *reinterpret_cast<uint32_t *>(v) = *reinterpret_cast<const uint32_t *>(p);
    else *reinterpret_cast<uint16_t *>(v) = *reinterpret_cast<const uint16_t *>(p);
}

__device__ __forceinline__ float shfl_d(float v, int src) { return __shfl_sync(0xFFFFFFFFu, v, src); }
__device__ __forceinline__ int32_t shfl_d(int32_t v, int src) { return __shfl_sync(0xFFFFFFFFu, v, src); }

// The fine uniform of the 64-bit word hi:lo (u01_fine64), written with 32-bit
// operations: 23 bits under the leading one, half a unit added, scaled by
// 2^-z with z the leading zeros; `zero` for hi:lo = 0.  With lo = 0 it is the
// fine uniform of the 32-bit word hi (u01_fine) when zero = 2^-56.
__device__ __forceinline__ float u01_fine_hl(uint32_t hi, uint32_t lo, float zero) {
    const int z = hi != 0u ? __clz(static_cast<int>(hi)) : 32 + (__clz(static_cast<int>(lo)) & 31);
    const uint32_t lead = z < 32 ? __funnelshift_l(lo, hi, static_cast<uint32_t>(z)) : lo << ((z - 32) & 31);
    const uint32_t top = lead >> 9;
    const float v = __fmul_rn(__fmul_rn(__uint2float_rn(2u * top + 1u), 0x1p-24f), pow2f(-(z & 63)));
    return (hi | lo) == 0u ? zero : v;
}

// The series branch of det_neg_log1m: v (1 + v/2 + ... + v^6/7), same steps.
__device__ __forceinline__ float neg_log1m_series(float v) {
    float p = 0x1.24924ap-3f;                       // 1/7
    p = __fadd_rn(0x1.555556p-3f, __fmul_rn(v, p)); // 1/6
    p = __fadd_rn(0x1.99999ap-3f, __fmul_rn(v, p)); // 1/5
    p = __fadd_rn(0.25f, __fmul_rn(v, p));
    p = __fadd_rn(0x1.555556p-2f, __fmul_rn(v, p)); // 1/3
    p = __fadd_rn(0.5f, __fmul_rn(v, p));
    p = __fadd_rn(1.0f, __fmul_rn(v, p));
    return __fmul_rn(v, p);
}

// The state-independent draws of one record for the lane's PPL = 4
// positions t = 4 lane + u: the race exponentials -ln(1 - V_t), V_t the fine
// uniform of RACE word u of Philox block lane.  When lane 31 holds no
// position (`step_lane`, k <= 124) it draws the STEP block instead and
// returns the multiplicity's Exp(1), -ln U with U the fine uniform of STEP
// words 1:0, in x[0].  The same values as race_exp and record_draws.
__device__ __forceinline__ void lane_draws4(uint64_t seed, uint32_t chain, uint64_t step, int lane, bool step_lane,
                                            float (&x)[4]) {
    const uint4 w = rng_block(seed, step_lane ? TAG_STEP : TAG_RACE, chain, step,
                              step_lane ? 0u : static_cast<uint32_t>(lane));
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const bool e1u = step_lane && u == 0;
        const uint32_t hi = e1u ? w.y : pick_word(w, static_cast<uint32_t>(u));
        const uint32_t lo = e1u ? w.x : 0u;
        const float v = u01_fine_hl(hi, lo, e1u ? 0x1p-88f : 0x1p-56f);
        const float lg = -det_logf(e1u ? v : __fsub_rn(1.0f, v));
        x[u] = (!e1u && v < 0.0625f) ? neg_log1m_series(v) : lg;
    }
}

// p = (S 2^-32 / k) e^{-beta A} (mult_p) from the weight sum's two parts,
// S = SA 2^16 + SB with SA, SB < 2^24 (at most 128 positions of 16-bit
// parts): SA 2^16 and SB are exact in fp32, so their rounded sum is S
// rounded to nearest, as the 64-bit conversion gives it.
__device__ __forceinline__ float mult_p_parts(uint32_t SA, uint32_t SB, int32_t k, float anchor_f) {
    const float sf = __fadd_rn(__fmul_rn(__uint2float_rn(SA), 65536.0f), __uint2float_rn(SB));
    float ps = __fmul_rn(sf, 0x1p-32f);
    ps = div_rn_pos(ps, __int2float_rn(k));
    return __fmul_rn(ps, anchor_f);
}

// cp.async.bulk.prefetch.L2 issued by lane 0 alone, without a branch.
__device__ __forceinline__ void prefetch_l2_lane0(const void *p, uint32_t bytes, int lane) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %2, 0;\n\t@p cp.async.bulk.prefetch.L2.global [%0], %1;\n\t}"
                 ::"l"(p), "r"(bytes), "r"(lane) : "memory");
}

// The state-independent draws of records step .. step + B - 1 of one chain,
// into the warp's buffer: xbuf[r kp + t] = -ln(1 - V_t), V_t the fine uniform
// of RACE word t mod 4 of Philox block t / 4 of record step + r, and e1buf[r]
// = -ln U, U the fine uniform of STEP words 1:0 of that record (the
// multiplicity's Exp(1)).  The B (blk + 1) Philox blocks (blk race blocks and
// the STEP block of each record) are spread over the 32 lanes, one block per
// lane per pass, so that a record with few candidates does not leave most
// lanes idle.  The same values as race_exp and record_draws.
__device__ __forceinline__ void batch_draws(uint64_t seed, uint32_t chain, uint64_t step, int B, int kp, int per,
                                            int lane, float *xbuf, float *e1buf) {
    const int items = B * per;
    const int blk = per - 1;
    const int q32 = 32 / per, m32 = 32 - q32 * per;
    int r = lane / per;  // item lane + 32 pass: record r, block b
    int b = lane - r * per;
    for (int p0 = 0; p0 < items; p0 += 32) {
        const bool stb = b == blk;
        const uint4 w = rng_block(seed, stb ? TAG_STEP : TAG_RACE, chain, step + static_cast<uint64_t>(r),
                                  stb ? 0u : static_cast<uint32_t>(b));
        float x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool e1u = stb && u == 0;
            const uint32_t hi = e1u ? w.y : pick_word(w, static_cast<uint32_t>(u));
            const uint32_t lo = e1u ? w.x : 0u;
            const float v = u01_fine_hl(hi, lo, e1u ? 0x1p-88f : 0x1p-56f);
            const float lg = -det_logf(e1u ? v : __fsub_rn(1.0f, v));
            x[u] = (!e1u && v < 0.0625f) ? neg_log1m_series(v) : lg;
        }
        if (p0 + lane < items) {
            if (stb) e1buf[r] = x[0];
            else *reinterpret_cast<float4 *>(xbuf + r * kp + 4 * b) = make_float4(x[0], x[1], x[2], x[3]);
        }
        b += m32;
        r += q32;
        if (b >= per) {
            b -= per;
            r += 1;
        }
    }
}

// -ln(1 - p) for the multiplicity, p the same on every lane of the warp: the
// series below 1/16, else -ln of the rounded 1 - p (det_neg_log1m's two
// forms, one evaluated: the branch does not diverge).
__device__ __forceinline__ float neg_log1m_uniform(float p) {
    float c;
    if (p < 0.0625f) c = neg_log1m_series(p);
    else c = -det_logf(__fsub_rn(1.0f, p));
    return c;
}

// What one warp needs to run one chain's period (the kernel's pointers into
// the group's shared memory and the chain's global fields).
template <typename QT, typename HT>
struct BlockChain {
    const QT *Q;          // the instance's padded rows
    const QT *sub;        // the set's sub-block, rows of kp entries
    const typename Arith<HT>::C *sub_b, *sub_d;
    HT *hg;               // the chain's fields in global memory
    HT *insf;             // the set's fields (shared memory)
    uint32_t *xw;         // the chain's bits (shared memory)
    int32_t *log;         // the period's flips
    ChainState *cs;       // the chain's state (shared memory)
    int32_t *sc;          // scratch words: [0] log length, [1] records this period
    float *wbuf;          // the warp's draw buffer (DRAW_BUF + DRAW_MAXB floats)
    int64_t step0;        // records before this launch
    float beta;
    uint32_t chain_id, row_bytes;
    int cid, n, ld, k, kp, s0, lane;
};

// One chain's period of Algorithm 6 by one warp, on the systematic set that
// starts at bit s0.  Lane l holds positions t = PPL l + u (u < PPL) of the
// set: their fields, b, diagonal and bits stay in registers for the whole
// period, so a move is one sub-block row read and PPL additions, with no
// shared-memory round trip on the record chain.  Returns false, with the
// chain's state back in shared memory, when the log holds BLOCK_LOG flips
// before the period ends: the caller applies the log and calls again.
template <typename QT, typename HT, int PPL>
__device__ __forceinline__ bool block_period(const KParams &P, const BlockChain<QT, HT> &c) {
    using A = Arith<HT>;
    using D = typename A::D;
    using CT = typename A::C;
    constexpr int VE = 16 / static_cast<int>(sizeof(QT));
    const int cid = c.cid, n = c.n, ld = c.ld, k = c.k, kp = c.kp, s0 = c.s0, lane = c.lane;
    const uint32_t chain_id = c.chain_id;
    // (launch constants read once: the loop's stores could alias them)
    const uint64_t seed = P.seed;
    const int tape = P.tape;
    const int64_t tape_cap = P.tape_cap;
    const int32_t L0 = static_cast<int32_t>(P.L0);
    const uint32_t row_bytes = c.row_bytes;
    const QT *const Q = c.Q;
    const QT *const sub = c.sub;
    HT *const insf = c.insf;
    uint32_t *const xw = c.xw;
    int32_t *const log = c.log;
    HT *const hg = c.hg;
    // the scalars a record changes stay in registers; the rest of the
    // chain's state is updated in shared memory at the period end
    ChainState *const cs = c.cs;
    int64_t stp = cs->step;
    int32_t Lb = static_cast<int32_t>(cs->L);  // (L0 < 2^31 here)
    double E = cs->E, bestE = cs->best_E;
    int32_t nflip = 0, nsat = 0;
    const int64_t step0 = c.step0;
    const float beta = c.beta;
    const int t0 = PPL * lane;
    // (a lane past the set reads an aligned block inside the padded set
    // and masks every position)
    const int tb = t0 < kp - PPL ? t0 : kp - PPL;
    HT hv[PPL];
    ld_vec<PPL>(insf + tb, hv);
    const CT *const sbp = c.sub_b + tb;  // (b and the diagonal are re-read per record: fewer live registers)
    const CT *const sdp = c.sub_d + tb;
    uint32_t xb = 0u;  // bit u: x at position t0 + u
#pragma unroll
    for (int u = 0; u < PPL; ++u) {
        int i = s0 + (t0 + u < k ? t0 + u : 0);
        i = i >= n ? i - n : i;
        xb |= ((xw[i >> 5] >> (i & 31)) & 1u) << u;
    }
    // Draws.  PPL 1 and 2: in batches of B records (batch_draws), B (blk + 1)
    // Philox blocks in ceil(B (blk + 1) / 32) passes of the warp.  PPL 4
    // (every lane busy): one Philox block per lane for the next record,
    // evaluated beside the current record's dependent chain.
    constexpr bool BATCH = PPL < 4;
    const int per = (kp >> 2) + 1;
    const int B = 64 / per < 2 ? 2 : (64 / per > DRAW_MAXB ? DRAW_MAXB : 64 / per);
    float *const xbuf = c.wbuf;
    float *const e1buf = c.wbuf + DRAW_BUF;
    int bi = B;  // next record's index in the batch (B: the batch is used up)
    // With k <= 31 PPL lane 31 holds no position: it forms the anchor's
    // weight e^{-beta A} in place of a candidate's.
    const bool anchor_lane = k <= 31 * PPL && lane == 31;
    int len = 0, nrec = 0;
    const bool extra_step = k > 31 * PPL;  // (PPL 4, k > 124: no lane is free for the STEP block)
    // With extra_step the multiplicity's Exp(1) is drawn 32 records at a
    // time, lane l drawing record e1_base + l (the same values).
    float e1_bat = 0.0f;
    int64_t e1_base = -64;
    auto e1_of = [&](int64_t s) -> float {
        if (s - e1_base >= 32) {
            e1_base = s;
            e1_bat = record_draws(seed, chain_id, static_cast<uint64_t>(s) + static_cast<uint64_t>(lane), n, false, true).e1;
        }
        return __shfl_sync(0xFFFFFFFFu, e1_bat, static_cast<int>(s - e1_base));
    };
    float exq[4], e1q = 0.0f;  // (PPL 4) the current record's draws
    if (!BATCH) {
        lane_draws4(seed, chain_id, static_cast<uint64_t>(stp), lane, !extra_step && lane == 31, exq);
        e1q = extra_step ? e1_of(stp)
                         : __shfl_sync(0xFFFFFFFFu, exq[0], 31);
    }
    // deferred tape entry (written one record late).  The multiplicities
    // are integers <= L0: the period's sum is kept in int64 and added to
    // the fp64 sum at the period end (exact: every partial sum is an
    // integer below 2^53), and the fp64 M is formed only for the tape
    int32_t pend_flip = 0;
    int32_t pend_m = 0;
    int64_t pend_pos = -1;
    int64_t sum_i = 0;
    // (the running minimum of E is also taken one record late, when its
    // operand is long ready)
    auto flush_record = [&]() {
        if (pend_pos >= 0) {
            if (lane == 0 && tape >= 1 && pend_pos < tape_cap) {
                const int64_t o = static_cast<int64_t>(cid) * tape_cap + pend_pos;
                P.tape_flip[o] = pend_flip;
                P.tape_m[o] = static_cast<double>(pend_m);
            }
            sum_i += pend_m;
            bestE = fmin(bestE, E);
        }
        pend_pos = -1;
    };
    auto write_record = [&](int32_t flip, int32_t m) {  // flushed at the start of the next record
        pend_flip = flip;
        pend_m = m;
        pend_pos = stp - step0;
    };
    auto bit_of = [&](int t) {
        const int i = s0 + t;
        return i >= n ? i - n : i;
    };
    // One record on the set at s0; true at the period end.
    auto one_record = [&]() -> bool {
        flush_record();  // the previous record (its E is the state this record starts from)
        const uint64_t step = static_cast<uint64_t>(stp);
        if (tape == 2) {
            const int64_t pos = stp - step0;
            if (pos < tape_cap) {
                const int64_t o = static_cast<int64_t>(cid) * tape_cap + pos;
                uint32_t *tx = P.tape_x + o * P.W;
                for (int q = lane; q < P.W; q += 32) tx[q] = q < ld / 32 ? xw[q] : 0u;
                if (lane == 0) P.tape_E[o] = E;
            }
        }
        float ex[PPL], e1;
        if constexpr (BATCH) {
            if (bi == B) {
                __syncwarp();  // (every lane has read the previous batch)
                batch_draws(seed, chain_id, step, B, kp, per, lane, xbuf, e1buf);
                __syncwarp();
                bi = 0;
            }
            ld_vec<PPL>(xbuf + bi * kp + tb, ex);
            e1 = e1buf[bi];
            bi += 1;
        } else {
#pragma unroll
            for (int u = 0; u < PPL; ++u) ex[u] = exq[u];
            e1 = e1q;
        }
        CT bv[PPL], dv[PPL];
        ld_vec<PPL>(sbp, bv);
        ld_vec<PPL>(sdp, dv);
        D dl[PPL];
        uint32_t lmin = 0xFFFFFFFFu;
#pragma unroll
        for (int u = 0; u < PPL; ++u) {
            dl[u] = A::delta(hv[u], bv[u], dv[u], (xb >> u) & 1u);
            const uint32_t kd = A::key(A::pos(dl[u]));
            lmin = t0 + u < k && kd < lmin ? kd : lmin;
        }
        if constexpr (!BATCH) {  // the next record's draws
            float xn[4];
            lane_draws4(seed, chain_id, step + 1, lane, !extra_step && lane == 31, xn);
            e1q = extra_step ? e1_of(static_cast<int64_t>(step) + 1) : xn[0];
#pragma unroll
            for (int u = 0; u < 4; ++u) exq[u] = xn[u];
        }
        const D amin = A::unkey(__reduce_min_sync(0xFFFFFFFFu, lmin));
        const float af = A::tof(amin);
        float anchor_e;
        if (k > 31 * PPL) anchor_e = det_expf(-__fmul_rn(beta, af));
        uint32_t bkey = 0xFFFFFFFFu, bpos = 0xFFFFFFFFu, sa = 0u, sb = 0u;
        D dbest = dl[0];
#pragma unroll
        for (int u = 0; u < PPL; ++u) {
            const int t = t0 + u;
            const bool ins = t < k;
            const float dv_u = (u == 0 && anchor_lane) ? af : A::diff(A::pos(dl[u]), amin);
            const float w = det_expf(-__fmul_rn(beta, dv_u));
            if (u == 0 && k <= 31 * PPL) anchor_e = __shfl_sync(0xFFFFFFFFu, w, 31);
            const float ws = __fmul_rn(w, 65536.0f);
            const float wa = truncf(ws);
            const uint32_t qa = __float2uint_rz(wa);
            const uint32_t qb = __float2uint_rz(__fmul_rn(__fsub_rn(ws, wa), 65536.0f));
            sa += ins ? qa : 0u;
            sb += ins ? qb : 0u;
            const uint32_t kb = ins ? __float_as_uint(race_key(ex[u], w)) : 0xFFFFFFFFu;
            const bool better = kb < bkey;  // t ascending: the first minimum is kept
            bkey = better ? kb : bkey;
            bpos = better ? static_cast<uint32_t>(t) : bpos;
            dbest = better ? dl[u] : dbest;
        }
        const uint32_t wkey = __reduce_min_sync(0xFFFFFFFFu, bkey);
        const uint32_t wpos = __reduce_min_sync(0xFFFFFFFFu, bkey == wkey ? bpos : 0xFFFFFFFFu);
        const uint32_t SA = __reduce_add_sync(0xFFFFFFFFu, sa);
        const uint32_t SB = __reduce_add_sync(0xFFFFFFFFu, sb);
        const int a = static_cast<int>(wpos);
        const int owner = a / PPL;  // the lane holding the winner
        const int j = bit_of(a);
        const float anchor_f = af > 0.0f ? anchor_e : 1.0f;
        const float p = mult_p_parts(SA, SB, k, anchor_f);
        const Mult mu = mult_from(p, neg_log1m_uniform(p), e1);
        // the winner's delta and bit, from the lane that holds it (its
        // first minimum is the winner)
        const D dj = shfl_d(dbest, owner);
        if constexpr (!BATCH) {
            if (!extra_step) e1q = __shfl_sync(0xFFFFFFFFu, e1q, 31);
        }
        const bool xj = __ballot_sync(0xFFFFFFFFu, lane == owner && ((xb >> (a - t0)) & 1u)) != 0u;
        bool period_end = false;
        const bool fits = mult_fits_small(mu, Lb);
        if (fits) {
            // (a move's M fits the budget: below 2^31, exact)
            const int32_t m = mu.mi >= 0 ? static_cast<int32_t>(mu.mi) : __float2int_rz(mu.fgl) + 1;
            Lb -= m;
            nsat += mu.sat ? 1 : 0;
            const bool up = !xj;
            prefetch_l2_lane0(Q + static_cast<int64_t>(j) * ld, row_bytes, lane);
            QT qv[PPL];
            ld_vec<PPL>(sub + a * kp + tb, qv);
#pragma unroll
            for (int u = 0; u < PPL; ++u) hv[u] = add_elem<QT, HT>(hv[u], qv[u], up);
            xb ^= lane == owner ? 1u << (a - t0) : 0u;
            // (every lane stores the same values: no divergent branch)
            const uint32_t xword = xw[j >> 5] ^ (1u << (j & 31));
            xw[j >> 5] = xword;
            log[len] = j | (up ? static_cast<int32_t>(0x80000000u) : 0);
            len += 1;
            E = __dadd_rn(E, A::tod(dj));
            nflip += 1;
            write_record(j, m);
        } else {
            const int32_t m = Lb;
            Lb = L0;
            if (lane == 0) {
                int ns = cs->set_start + k;
                while (ns >= n) ns -= n;
                cs->stays += 1;
                cs->set_start = ns;
                cs->period_start = static_cast<int64_t>(step) + 1;
            }
            period_end = true;
            write_record(-1, m);
        }
        stp += 1;
        nrec += 1;
        if (tape == 2) __syncwarp();  // (lane 0's bit update before the next record's snapshot)
        return period_end;
    };
    bool period_end;
    do {
        period_end = one_record();
    } while (!period_end && len < BLOCK_LOG);  // (a full log returns to the caller, which applies it)
    flush_record();
    const double sum_m = __dadd_rn(cs->sum_m, static_cast<double>(sum_i));
    // the set fields back to shared memory for the finalise step
#pragma unroll
    for (int u = 0; u < PPL; ++u)
        if (t0 + u < k) insf[t0 + u] = hv[u];
    __syncwarp();
    if (lane == 0) {
        cs->step = stp;
        cs->L = Lb;
        cs->E = E;
        cs->best_E = bestE;
        cs->sum_m = sum_m;
        cs->flips += nflip;
        cs->saturated += nsat;
        c.sc[0] = len;
        c.sc[1] += nrec;
    }
    __syncwarp();
    return period_end;
}

// The narrow record forms (PPL 1 or 2: at most 62 positions, lane 31 free)
// with the record loop software-pipelined.  A record's race fixes its winner
// before its multiplicity is known; the chain applies the winner's move to a
// copy of its set state at once and evaluates the next record on that copy
// while the current record's multiplicity and budget test run (the two
// dependent chains interleave in one basic block).  If the test says move,
// the copy becomes the state and the next record is already evaluated; if it
// says stay, the period ends and the evaluation is dropped.  The records, and
// every value they produce, are those of block_period.
template <typename QT, typename HT, int PPL>
__device__ __forceinline__ bool block_period_pipe(const KParams &P, const BlockChain<QT, HT> &c) {
    static_assert(PPL == 1 || PPL == 2, "narrow forms");
    using A = Arith<HT>;
    using D = typename A::D;
    using CT = typename A::C;
    const int cid = c.cid, n = c.n, k = c.k, kp = c.kp, s0 = c.s0, lane = c.lane, ld = c.ld;
    const uint32_t chain_id = c.chain_id;
    const uint64_t seed = P.seed;
    const int tape = P.tape;
    const int64_t tape_cap = P.tape_cap;
    const int32_t L0 = static_cast<int32_t>(P.L0);
    const uint32_t row_bytes = c.row_bytes;
    const QT *const Q = c.Q;
    const QT *const sub = c.sub;
    HT *const insf = c.insf;
    uint32_t *const xw = c.xw;
    int32_t *const log = c.log;
    ChainState *const cs = c.cs;
    int64_t stp = cs->step;
    int32_t Lb = static_cast<int32_t>(cs->L);
    double E = cs->E, bestE = cs->best_E;
    int32_t nflip = 0, nsat = 0;
    const int64_t step0 = c.step0;
    const float beta = c.beta;
    const int t0 = PPL * lane;
    const int tb = t0 < kp - PPL ? t0 : kp - PPL;
    HT hv[PPL];
    ld_vec<PPL>(insf + tb, hv);
    const CT *const sbp = c.sub_b + tb;
    const CT *const sdp = c.sub_d + tb;
    uint32_t xb = 0u;
#pragma unroll
    for (int u = 0; u < PPL; ++u) {
        int i = s0 + (t0 + u < k ? t0 + u : 0);
        i = i >= n ? i - n : i;
        xb |= ((xw[i >> 5] >> (i & 31)) & 1u) << u;
    }
    const int per = (kp >> 2) + 1;
    const int B = 64 / per < 2 ? 2 : (64 / per > DRAW_MAXB ? DRAW_MAXB : 64 / per);
    float *const xbuf = c.wbuf;
    float *const e1buf = c.wbuf + DRAW_BUF;
    int bi = B;
    const bool anchor_lane = lane == 31;  // (k <= 31 PPL: lane 31 holds no position)
    int len = 0, nrec = 0;
    int32_t pend_flip = 0, pend_m = 0;
    int64_t pend_pos = -1;
    int64_t sum_i = 0;
    auto flush_record = [&]() {
        if (pend_pos >= 0) {
            if (lane == 0 && tape >= 1 && pend_pos < tape_cap) {
                const int64_t o = static_cast<int64_t>(cid) * tape_cap + pend_pos;
                P.tape_flip[o] = pend_flip;
                P.tape_m[o] = static_cast<double>(pend_m);
            }
            sum_i += pend_m;
            bestE = fmin(bestE, E);
        }
        pend_pos = -1;
    };
    auto write_record = [&](int32_t flip, int32_t m) {
        pend_flip = flip;
        pend_m = m;
        pend_pos = stp - step0;
    };
    // the draws of record step (batch index bi), refilled outside the
    // pipelined region
    auto ensure_draws = [&](uint64_t step) {
        if (bi == B) {
            __syncwarp();
            batch_draws(seed, chain_id, step, B, kp, per, lane, xbuf, e1buf);
            __syncwarp();
            bi = 0;
        }
    };
    // evaluation of one record on the set state (h, x): the race winner, its
    // delta and bit, the quantised weight sum and the anchor's weight
    struct Eval {
        uint32_t SA, SB;
        int a;
        D dj;
        bool xj;
        float af, anchor_e, e1;
    };
    auto evaluate = [&](const HT (&h)[PPL], uint32_t xbits, int bidx) -> Eval {
        float ex[PPL];
        ld_vec<PPL>(xbuf + bidx * kp + tb, ex);
        CT bv[PPL], dv[PPL];
        ld_vec<PPL>(sbp, bv);
        ld_vec<PPL>(sdp, dv);
        D dl[PPL];
        uint32_t lmin = 0xFFFFFFFFu;
#pragma unroll
        for (int u = 0; u < PPL; ++u) {
            dl[u] = A::delta(h[u], bv[u], dv[u], (xbits >> u) & 1u);
            const uint32_t kd = A::key(A::pos(dl[u]));
            lmin = t0 + u < k && kd < lmin ? kd : lmin;
        }
        Eval r;
        r.e1 = e1buf[bidx];
        const D amin = A::unkey(__reduce_min_sync(0xFFFFFFFFu, lmin));
        r.af = A::tof(amin);
        uint32_t bkey = 0xFFFFFFFFu, bpos = 0xFFFFFFFFu, sa = 0u, sb = 0u;
        D dbest = dl[0];
#pragma unroll
        for (int u = 0; u < PPL; ++u) {
            const int t = t0 + u;
            const bool ins = t < k;
            const float dv_u = (u == 0 && anchor_lane) ? r.af : A::diff(A::pos(dl[u]), amin);
            const float w = det_expf(-__fmul_rn(beta, dv_u));
            if (u == 0) r.anchor_e = __shfl_sync(0xFFFFFFFFu, w, 31);
            const float ws = __fmul_rn(w, 65536.0f);
            const float wa = truncf(ws);
            const uint32_t qa = __float2uint_rz(wa);
            const uint32_t qb = __float2uint_rz(__fmul_rn(__fsub_rn(ws, wa), 65536.0f));
            sa += ins ? qa : 0u;
            sb += ins ? qb : 0u;
            const uint32_t kb = ins ? __float_as_uint(race_key(ex[u], w)) : 0xFFFFFFFFu;
            const bool better = kb < bkey;
            bkey = better ? kb : bkey;
            bpos = better ? static_cast<uint32_t>(t) : bpos;
            dbest = better ? dl[u] : dbest;
        }
        const uint32_t wkey = __reduce_min_sync(0xFFFFFFFFu, bkey);
        const uint32_t wpos = __reduce_min_sync(0xFFFFFFFFu, bkey == wkey ? bpos : 0xFFFFFFFFu);
        r.SA = __reduce_add_sync(0xFFFFFFFFu, sa);
        r.SB = __reduce_add_sync(0xFFFFFFFFu, sb);
        r.a = static_cast<int>(wpos);
        const int owner = r.a / PPL;
        r.dj = shfl_d(dbest, owner);
        r.xj = __ballot_sync(0xFFFFFFFFu, lane == owner && ((xbits >> (r.a - t0)) & 1u)) != 0u;
        return r;
    };
    auto tape2 = [&]() {
        if (tape == 2) {
            const int64_t pos = stp - step0;
            if (pos < tape_cap) {
                const int64_t o = static_cast<int64_t>(cid) * tape_cap + pos;
                uint32_t *tx = P.tape_x + o * P.W;
                for (int q = lane; q < P.W; q += 32) tx[q] = q < ld / 32 ? xw[q] : 0u;
                if (lane == 0) P.tape_E[o] = E;
            }
        }
    };

    tape2();
    ensure_draws(static_cast<uint64_t>(stp));
    Eval ev = evaluate(hv, xb, bi);
    bi += 1;
    bool period_end = false;
    while (true) {
        // record stp is evaluated (ev); its successor's draws come next
        ensure_draws(static_cast<uint64_t>(stp) + 1);
        const int a = ev.a;
        const int owner = a / PPL;
        int j = s0 + a;
        j = j >= n ? j - n : j;
        const bool up = !ev.xj;
        // the move of record stp, tentatively
        QT qv[PPL];
        ld_vec<PPL>(sub + a * kp + tb, qv);
        HT hn[PPL];
#pragma unroll
        for (int u = 0; u < PPL; ++u) hn[u] = add_elem<QT, HT>(hv[u], qv[u], up);
        const uint32_t xn = xb ^ (lane == owner ? 1u << (a - t0) : 0u);
        // record stp's multiplicity and budget test (branch-free) beside the
        // evaluation of record stp + 1 on the moved state, written in stages
        // between the warp collectives so that the two chains interleave
        //   M1: the weight sum in fp32           E1: deltas of the moved state
        float ex[PPL];
        ld_vec<PPL>(xbuf + bi * kp + tb, ex);
        CT bv[PPL], dv[PPL];
        ld_vec<PPL>(sbp, bv);
        ld_vec<PPL>(sdp, dv);
        const float anchor_f = ev.af > 0.0f ? ev.anchor_e : 1.0f;
        const float sf = __fadd_rn(__fmul_rn(__uint2float_rn(ev.SA), 65536.0f), __uint2float_rn(ev.SB));
        D dl[PPL];
        uint32_t lmin = 0xFFFFFFFFu;
#pragma unroll
        for (int u = 0; u < PPL; ++u) {
            dl[u] = A::delta(hn[u], bv[u], dv[u], (xn >> u) & 1u);
            const uint32_t kd = A::key(A::pos(dl[u]));
            lmin = t0 + u < k && kd < lmin ? kd : lmin;
        }
        Eval nx;
        nx.e1 = e1buf[bi];
        //   M2: p                                  E2: the anchor
        const float p = __fmul_rn(div_rn_pos(__fmul_rn(sf, 0x1p-32f), __int2float_rn(k)), anchor_f);
        const D amin = A::unkey(__reduce_min_sync(0xFFFFFFFFu, lmin));
        nx.af = A::tof(amin);
        //   M3: -ln(1 - p)                         E3: weights, keys, parts of the sum
        const float cser = neg_log1m_series(p);
        const float clog = -det_logf(__fsub_rn(1.0f, p));
        uint32_t bkey = 0xFFFFFFFFu, bpos = 0xFFFFFFFFu, sa = 0u, sb = 0u;
        D dbest = dl[0];
#pragma unroll
        for (int u = 0; u < PPL; ++u) {
            const int t = t0 + u;
            const bool ins = t < k;
            const float dv_u = (u == 0 && anchor_lane) ? nx.af : A::diff(A::pos(dl[u]), amin);
            const float w = det_expf(-__fmul_rn(beta, dv_u));
            if (u == 0) nx.anchor_e = __shfl_sync(0xFFFFFFFFu, w, 31);
            const float ws = __fmul_rn(w, 65536.0f);
            const float wa = truncf(ws);
            const uint32_t qa = __float2uint_rz(wa);
            const uint32_t qb = __float2uint_rz(__fmul_rn(__fsub_rn(ws, wa), 65536.0f));
            sa += ins ? qa : 0u;
            sb += ins ? qb : 0u;
            const uint32_t kb = ins ? __float_as_uint(race_key(ex[u], w)) : 0xFFFFFFFFu;
            const bool better = kb < bkey;
            bkey = better ? kb : bkey;
            bpos = better ? static_cast<uint32_t>(t) : bpos;
            dbest = better ? dl[u] : dbest;
        }
        //   M4: the multiplicity                   E4: the race winner and the sum
        const Mult mu = mult_from(p, p < 0.0625f ? cser : clog, ev.e1);
        const uint32_t wkey = __reduce_min_sync(0xFFFFFFFFu, bkey);
        const uint32_t wpos = __reduce_min_sync(0xFFFFFFFFu, bkey == wkey ? bpos : 0xFFFFFFFFu);
        nx.SA = __reduce_add_sync(0xFFFFFFFFu, sa);
        nx.SB = __reduce_add_sync(0xFFFFFFFFu, sb);
        nx.a = static_cast<int>(wpos);
        const int nowner = nx.a / PPL;
        nx.dj = shfl_d(dbest, nowner);
        nx.xj = __ballot_sync(0xFFFFFFFFu, lane == nowner && ((xn >> (nx.a - t0)) & 1u)) != 0u;
        const bool fits = mult_fits_small(mu, Lb);
        flush_record();
        if (fits) {
            const int32_t m = mu.mi >= 0 ? static_cast<int32_t>(mu.mi) : __float2int_rz(mu.fgl) + 1;
            Lb -= m;
            nsat += mu.sat ? 1 : 0;
            prefetch_l2_lane0(Q + static_cast<int64_t>(j) * ld, row_bytes, lane);
            const uint32_t xword = xw[j >> 5] ^ (1u << (j & 31));
            xw[j >> 5] = xword;
            log[len] = j | (up ? static_cast<int32_t>(0x80000000u) : 0);
            len += 1;
            E = __dadd_rn(E, A::tod(ev.dj));
            nflip += 1;
            write_record(j, m);
#pragma unroll
            for (int u = 0; u < PPL; ++u) hv[u] = hn[u];
            xb = xn;
            ev = nx;
            bi += 1;
        } else {
            const int32_t m = Lb;
            Lb = L0;
            if (lane == 0) {
                int ns = cs->set_start + k;
                while (ns >= n) ns -= n;
                cs->stays += 1;
                cs->set_start = ns;
                cs->period_start = static_cast<int64_t>(stp) + 1;
            }
            period_end = true;
            write_record(-1, m);
        }
        stp += 1;
        nrec += 1;
        if (period_end || len == BLOCK_LOG) break;
        if (tape == 2) __syncwarp();
        tape2();
    }
    flush_record();
    const double sum_m = __dadd_rn(cs->sum_m, static_cast<double>(sum_i));
#pragma unroll
    for (int u = 0; u < PPL; ++u)
        if (t0 + u < k) insf[t0 + u] = hv[u];
    __syncwarp();
    if (lane == 0) {
        cs->step = stp;
        cs->L = Lb;
        cs->E = E;
        cs->best_E = bestE;
        cs->sum_m = sum_m;
        cs->flips += nflip;
        cs->saturated += nsat;
        c.sc[0] = len;
        c.sc[1] += nrec;
    }
    __syncwarp();
    return period_end;
}

template <typename QT, typename HT>
__global__ void __launch_bounds__(512) pns_block_kernel(const __grid_constant__ KParams P) {
    using A = Arith<HT>;
    using D = typename A::D;
    using CT = typename A::C;
    constexpr int VE = 16 / static_cast<int>(sizeof(QT));

    extern __shared__ __align__(16) unsigned char smem[];
    const CtaDesc cd = P.cta[blockIdx.x];
    const int W = cd.pad > 0 ? cd.pad : P.gw;  // warps per group (the layout keeps the launch's P.gw)
    const int R = P.R;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int g = warp / W;
    if (g >= cd.groups) return;  // idle warps take part in no barrier
    const int wg = warp - g * W;
    const int gtid = wg * 32 + lane;
    const int GT = 32 * W;
    const int c0 = cd.first + g * R;  // the group's chains: cta_chains[c0 .. c0 + R)
    const ChainDesc chd0 = P.chain[P.cta_chains[c0]];
    const InstDesc in = P.inst[chd0.inst];
    const int n = in.n;
    const int ld = in.ld;
    const int k = in.k;
    const int kp = (k + 3) & ~3;  // sub-block row stride and padded set length
    const QT *Q = reinterpret_cast<const QT *>(in.q);
    const BlockSmem L = block_smem(ld, k, static_cast<int32_t>(sizeof(HT)), static_cast<int32_t>(sizeof(QT)), R, P.gw);
    unsigned char *gbase = smem + chd0.smem_off;
    auto area = [&](int s) { return gbase + s * L.chain_bytes; };
    auto cst = [&](int s) { return reinterpret_cast<ChainState *>(area(s) + L.state); };
    auto sc32 = [&](int s, int off) { return reinterpret_cast<int32_t *>(area(s) + L.scratch + off); };
    auto step0_of = [&](int s) { return reinterpret_cast<int64_t *>(area(s) + L.scratch + 16); };
    auto cid_of = [&](int s) { return P.cta_chains[c0 + s]; };
    auto hg_of = [&](int s) { return reinterpret_cast<HT *>(P.fields) + static_cast<int64_t>(cid_of(s)) * P.LD; };
    // scratch words: 0 log length, 4 records this period, 8 finalised, 12 set start
    QT *sub = reinterpret_cast<QT *>(gbase + L.sub);
    CT *sub_b = reinterpret_cast<CT *>(gbase + L.bd);
    CT *sub_d = reinterpret_cast<CT *>(gbase + L.bd + round16(4 * kp));
    int32_t *q_order = reinterpret_cast<int32_t *>(gbase + L.ctrl);
    int32_t *q_next = q_order + 16;
    int32_t *q_running = q_order + 17;
    const CT *bvec = reinterpret_cast<const CT *>(in.b);
    const CT *dvec = reinterpret_cast<const CT *>(in.diag);
    const uint64_t seed = P.seed;
    const uint32_t row_bytes = static_cast<uint32_t>(ld) * static_cast<uint32_t>(sizeof(QT));

    // one named barrier per exchange group (id 0 is __syncthreads')
    const int gbar = 1 + g;
    auto gsync = [&]() { named_sync(gbar, GT); };

    // ---- load the group's chains ------------------------------------------------
    for (int s = wg; s < R; s += W) {
        const int cid = cid_of(s);
        const ChainState st = P.state[cid];
        const uint32_t *gx = P.xbits + static_cast<int64_t>(cid) * P.W;
        uint32_t *xw = reinterpret_cast<uint32_t *>(area(s) + L.xw);
        HT *insf = reinterpret_cast<HT *>(area(s) + L.insf);
        const HT *hg = hg_of(s);
        for (int w = lane; w < ld / 32; w += 32) xw[w] = gx[w];
        for (int t = lane; t < k; t += 32) {
            int r = st.set_start + t;
            if (r >= n) r -= n;
            insf[t] = hg[r];
        }
        if (lane == 0) {
            *cst(s) = st;
            *sc32(s, 12) = st.set_start;
            *step0_of(s) = st.step;
        }
    }
    gsync();
    // every replica of the group must stand at the same systematic set
    int s0 = *sc32(0, 12);
    bool bad = false;
    for (int s = 1; s < R; ++s) bad |= *sc32(s, 12) != s0;
    if (bad && gtid == 0) set_status(P.status, ST_STATE);
    if (gtid == 0) {
        // first queue: hottest temperature first
        for (int s = 0; s < R; ++s) q_order[s] = s;
        for (int a = 1; a < R; ++a)
            for (int b = a; b > 0 && cst(q_order[b])->beta_idx < cst(q_order[b - 1])->beta_idx; --b) {
                const int t = q_order[b];
                q_order[b] = q_order[b - 1];
                q_order[b - 1] = t;
            }
        *q_next = 0;
        *q_running = R;
    }

    // The set's sub-block, b and diagonal, by cp.async (4-byte entries) or
    // plain loads (2-byte entries).
    auto load_set = [&](int s) {
        // row a of the sub-block by warp, columns t = lane + 32 u (k <= 128)
        // by lane: the lane's columns and the shared address once per set
        int ct[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = s + lane + 32 * u;
            ct[u] = c >= n ? c - n : c;
        }
        const uint32_t sub_s = static_cast<uint32_t>(__cvta_generic_to_shared(sub)) + 4u * static_cast<uint32_t>(lane);
        for (int a = wg; a < k; a += W) {
            int ra = s + a;
            if (ra >= n) ra -= n;
            const QT *row = Q + static_cast<int64_t>(ra) * ld;
            if constexpr (sizeof(QT) == 4) {
                const uint32_t d0 = sub_s + 4u * static_cast<uint32_t>(a * kp);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (lane + 32 * u < k) cp_async4_s(d0 + 128u * u, row + ct[u]);
            } else {
                QT *dst = sub + a * kp;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (lane + 32 * u < k) dst[lane + 32 * u] = row[ct[u]];
            }
        }
        for (int t = gtid; t < k; t += GT) {
            int ct = s + t;
            if (ct >= n) ct -= n;
            cp_async4(sub_b + t, bvec + ct);
            cp_async4(sub_d + t, dvec + ct);
        }
    };

    // positions per lane (block_ppl; the group's k is the same for every chain)
    auto run_chain_period = [&](int s) {
        BlockChain<QT, HT> bc;
        bc.Q = Q;
        bc.sub = sub;
        bc.sub_b = sub_b;
        bc.sub_d = sub_d;
        bc.cid = cid_of(s);
        bc.hg = hg_of(s);
        bc.insf = reinterpret_cast<HT *>(area(s) + L.insf);
        bc.xw = reinterpret_cast<uint32_t *>(area(s) + L.xw);
        bc.log = reinterpret_cast<int32_t *>(area(s) + L.log);
        bc.cs = cst(s);
        bc.sc = sc32(s, 0);
        bc.wbuf = reinterpret_cast<float *>(gbase + L.wbuf) + wg * (DRAW_BUF + DRAW_MAXB);
        bc.step0 = *step0_of(s);
        bc.beta = in.betas[bc.cs->beta_idx];
        bc.chain_id = static_cast<uint32_t>(bc.cid) + P.chain_base;
        bc.row_bytes = row_bytes;
        bc.n = n;
        bc.ld = ld;
        bc.k = k;
        bc.kp = kp;
        bc.s0 = s0;
        bc.lane = lane;
        if (lane == 0) bc.sc[1] = 0;  // (records this period: each call adds its own)
        __syncwarp();
        while (true) {
            bool done;
            const int ppl = block_ppl(k);
            if (ppl == 1) done = block_period_pipe<QT, HT, 1>(P, bc);
            else if (ppl == 2) done = block_period_pipe<QT, HT, 2>(P, bc);
            else done = block_period<QT, HT, 4>(P, bc);
            if (done) break;
            // a full log (more than BLOCK_LOG moves in the period, L0 > BLOCK_LOG):
            // apply it to the fields outside the set and continue the period
            apply_log<QT, HT>(Q, ld, bc.hg, bc.log, BLOCK_LOG, lane, 32, s0, 0, k, n, nullptr);
            __syncwarp();
        }
    };

    // Chain s after its period, by one warp: its set fields back to global
    // memory, its log onto the other fields, the next set's fields gathered.
    auto finalise_warp = [&](int s, int sn, bool last) {
        HT *insf = reinterpret_cast<HT *>(area(s) + L.insf);
        HT *const hg = hg_of(s);
        for (int t = lane; t < k; t += 32) {
            int r = s0 + t;
            if (r >= n) r -= n;
            hg[r] = insf[t];
        }
        __syncwarp();
        const int len = *sc32(s, 0);
        const int32_t *log = reinterpret_cast<const int32_t *>(area(s) + L.log);
        apply_log<QT, HT>(Q, ld, hg, log, len, lane, 32, s0, sn, k, n, last ? nullptr : insf);
        __syncwarp();
    };

    // ---- periods, exchange rounds ------------------------------------------------
    const int64_t rounds = bad ? 0 : P.steps / P.swap_interval;
    const int64_t per_round = P.swap_interval / P.L0;
    if (rounds > 0) load_set(s0);
    cp_async_wait_all();
    gsync();
    for (int64_t rdi = 0; rdi < rounds; ++rdi) {
        for (int64_t pr = 0; pr < per_round; ++pr) {
            const bool last = rdi + 1 == rounds && pr + 1 == per_round;
            int sn = s0 + k;  // the next set (the same for every chain of the group)
            while (sn >= n) sn -= n;
            while (true) {
                int qi = 0;
                if (lane == 0) qi = atomicAdd(q_next, 1);
                qi = __shfl_sync(0xFFFFFFFFu, qi, 0);
                if (qi >= R) break;
                const int s = q_order[qi];
                run_chain_period(s);
                int rem = 0;
                if (lane == 0) rem = atomicSub(q_running, 1) - 1;
                rem = __shfl_sync(0xFFFFFFFFu, rem, 0);
                const bool mine = rem > 0;  // others still run: finalise this chain here
                if (mine) finalise_warp(s, sn, last);
                if (lane == 0) *sc32(s, 8) = mine ? 1 : 0;
                __syncwarp();
            }
            gsync();
            if (wg == 0) {
                // warp 0 of the group, one lane per chain / pair: records per
                // temperature in this period, the exchange, the next queue
                // (small arrays in shared memory: local arrays would live in
                // cold local memory)
                int32_t *rec_b = q_order + 20;   // [16] records of temperature b
                int32_t *slot_of = rec_b + 16;   // [16] chain holding temperature b
                if (lane < R) {
                    const int b = cst(lane)->beta_idx;
                    rec_b[b] = *sc32(lane, 4);
                    slot_of[b] = lane;
                }
                __syncwarp();
                if (pr + 1 == per_round) {
                    const uint64_t ndone = static_cast<uint64_t>(cst(0)->sum_m) / static_cast<uint64_t>(P.swap_interval);
                    const uint64_t rnd = ndone - 1;
                    // pairs (a, a + 1), a = rnd mod 2 + 2q, are disjoint: pair q on lane q
                    const int a = static_cast<int>(rnd & 1u) + 2 * lane;
                    if (a + 1 < R) {
                        const int sa_ = slot_of[a], sb_ = slot_of[a + 1];
                        ChainState *pa = cst(sa_);
                        ChainState *pb = cst(sb_);
                        const float db = __fsub_rn(in.betas[a], in.betas[a + 1]);
                        const float de = __double2float_rn(__dsub_rn(pa->E, pb->E));
                        const float xr = __fmul_rn(db, de);
                        const uint32_t w = rng_word(seed, TAG_SWAP, static_cast<uint32_t>(chd0.group) + P.group_base,
                                                    rnd, static_cast<uint32_t>(lane));
                        if (det_logf(u01_grid(w)) < xr) {
                            pa->beta_idx = a + 1;
                            pb->beta_idx = a;
                            pa->swaps += 1;
                            pb->swaps += 1;
                        }
                    }
                    __syncwarp();
                }
                // next queue: chains by the records their (new) temperature took,
                // most first, ties by chain: the rank of chain `lane`
                if (lane < R) {
                    const int key = rec_b[cst(lane)->beta_idx];
                    int rank = 0;
                    for (int s2 = 0; s2 < R; ++s2) {
                        const int k2 = rec_b[cst(s2)->beta_idx];
                        rank += (k2 > key || (k2 == key && s2 < lane)) ? 1 : 0;
                    }
                    q_order[rank] = lane;
                }
                if (lane == 0) {
                    *q_next = 0;
                    *q_running = R;
                }
            }
            if (!last) load_set(sn);  // the sub-block is not read until the next period
            // the chain(s) that ended last, by the whole group
            for (int s = 0; s < R; ++s) {
                if (*sc32(s, 8)) continue;
                HT *insf = reinterpret_cast<HT *>(area(s) + L.insf);
                HT *const hg = hg_of(s);
                for (int t = gtid; t < k; t += GT) {
                    int r = s0 + t;
                    if (r >= n) r -= n;
                    hg[r] = insf[t];
                }
            }
            gsync();
            {
                const int nch = ld / VE;
                for (int s = 0; s < R; ++s) {
                    if (*sc32(s, 8)) continue;
                    HT *insf = reinterpret_cast<HT *>(area(s) + L.insf);
                    const int len = *sc32(s, 0);
                    const int32_t *log = reinterpret_cast<const int32_t *>(area(s) + L.log);
                    HT *const hg = hg_of(s);
                    apply_log<QT, HT>(Q, ld, hg, log, len, gtid, GT, s0, sn, k, n, last ? nullptr : insf);
                }
            }
            cp_async_wait_all();
            gsync();
            s0 = sn;
        }
    }

    // ---- write the chains back ------------------------------------------------------
    // (the fields are complete in global memory after the last finalise step)
    for (int s = wg; s < R; s += W) {
        const int cid = cid_of(s);
        const uint32_t *xw = reinterpret_cast<const uint32_t *>(area(s) + L.xw);
        uint32_t *gx = P.xbits + static_cast<int64_t>(cid) * P.W;
        for (int w = lane; w < ld / 32; w += 32) gx[w] = xw[w];
        if (lane == 0) {
            ChainState st = *cst(s);
            const int64_t recs = st.step - *step0_of(s);
            st.tape_records = P.tape ? (recs < P.tape_cap ? recs : P.tape_cap) : 0;
            P.state[cid] = st;
        }
    }
}

}  // namespace pnsk
