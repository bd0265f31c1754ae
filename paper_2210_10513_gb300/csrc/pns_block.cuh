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

constexpr int APPLY_U = 8;  // logged rows in flight per thread

template <typename QT, typename HT>
__device__ __forceinline__ HT add_elem(HT h, QT q, bool up) {
    if constexpr (std::is_same<HT, float>::value) {
        return up ? __fadd_rn(h, q) : __fsub_rn(h, q);
    } else {
        return up ? h + static_cast<int32_t>(q) : h - static_cast<int32_t>(q);
    }
}

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One 16-byte chunk q of Q columns for one chain: applies `len` logged
// flips, in log order, to the chain's global fields hg outside the window
// [s_prev, s_prev + k) (mod n), then, when insf is given, copies the fields
// of the window [s_next, s_next + k) into insf (the next set's fields).  A
// log entry is the flipped bit j, with the sign bit set for a 0 -> 1 flip.
template <typename QT, typename HT>
__device__ __noinline__ void apply_item(const QT *Q, int ld, HT *hg, const int32_t *log, int len, int q,
                                           int s_prev, int s_next, int k, int n, HT *insf) {
    constexpr int VE = 16 / static_cast<int>(sizeof(QT));
    const int r0 = q * VE;
    uint32_t mask = 0u, nmask = 0u;
#pragma unroll
    for (int e = 0; e < VE; ++e) {
        const int r = r0 + e;
        int d = r - s_prev;
        if (d < 0) d += n;
        if (r < n && d >= k) mask |= 1u << e;
        if (insf) {
            int dn = r - s_next;
            if (dn < 0) dn += n;
            if (r < n && dn < k) nmask |= 1u << e;
        }
    }
    if (len == 0) mask = 0u;
    if (mask == 0u && nmask == 0u) return;
    HT acc[VE];
#pragma unroll
    for (int g = 0; g < VE / 4; ++g) *reinterpret_cast<uint4 *>(acc + 4 * g) = reinterpret_cast<const uint4 *>(hg + r0)[g];
    if (mask) {
        for (int t0 = 0; t0 < len; t0 += APPLY_U) {
            uint4 v[APPLY_U];
            uint32_t ups = 0u;
#pragma unroll
            for (int u = 0; u < APPLY_U; ++u) {
                if (t0 + u < len) {
                    const int32_t ent = log[t0 + u];
                    if (ent < 0) ups |= 1u << u;
                    const int j = ent & 0x7FFFFFFF;
                    v[u] = ld_nc_v4(Q + static_cast<int64_t>(j) * ld + r0);
                }
            }
#pragma unroll
            for (int u = 0; u < APPLY_U; ++u) {
                if (t0 + u < len) {
                    QT qv[VE];
                    *reinterpret_cast<uint4 *>(qv) = v[u];
                    const bool up = (ups >> u) & 1u;
#pragma unroll
                    for (int e = 0; e < VE; ++e)
                        if ((mask >> e) & 1u) acc[e] = add_elem<QT, HT>(acc[e], qv[e], up);
                }
            }
        }
#pragma unroll
        for (int g = 0; g < VE / 4; ++g) reinterpret_cast<uint4 *>(hg + r0)[g] = *reinterpret_cast<const uint4 *>(acc + 4 * g);
    }
    if (nmask) {
#pragma unroll
        for (int e = 0; e < VE; ++e) {
            if ((nmask >> e) & 1u) {
                int dn = r0 + e - s_next;
                if (dn < 0) dn += n;
                insf[dn] = acc[e];
            }
        }
    }
}

__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <typename QT, typename HT>
__global__ void __launch_bounds__(512) pns_block_kernel(const KParams P) {
    using A = Arith<HT>;
    using D = typename A::D;
    using CT = typename A::C;
    constexpr int VE = 16 / static_cast<int>(sizeof(QT));

    extern __shared__ __align__(16) unsigned char smem[];
    const CtaDesc cd = P.cta[blockIdx.x];
    const int W = P.gw;
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
    const QT *Q = reinterpret_cast<const QT *>(in.q);
    const BlockSmem L = block_smem(ld, k, static_cast<int32_t>(sizeof(HT)), static_cast<int32_t>(sizeof(QT)), R);
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
    CT *sub_d = reinterpret_cast<CT *>(gbase + L.bd + round16(4 * k));
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
        for (int a = wg; a < k; a += W) {  // row a of the sub-block by warp, columns by lane
            int ra = s + a;
            if (ra >= n) ra -= n;
            const QT *row = Q + static_cast<int64_t>(ra) * ld;
            QT *dst = sub + a * k;
            for (int t = lane; t < k; t += 32) {
                int ct = s + t;
                if (ct >= n) ct -= n;
                if constexpr (sizeof(QT) == 4) cp_async4(dst + t, row + ct);
                else dst[t] = row[ct];
            }
        }
        for (int t = gtid; t < k; t += GT) {
            int ct = s + t;
            if (ct >= n) ct -= n;
            cp_async4(sub_b + t, bvec + ct);
            cp_async4(sub_d + t, dvec + ct);
        }
    };

    // ---- one chain's period (one warp) -----------------------------------------
    auto run_period = [&](int s) {
        const int cid = cid_of(s);
        const uint32_t chain_id = static_cast<uint32_t>(cid) + P.chain_base;
        HT *insf = reinterpret_cast<HT *>(area(s) + L.insf);
        uint32_t *xw = reinterpret_cast<uint32_t *>(area(s) + L.xw);
        int32_t *log = reinterpret_cast<int32_t *>(area(s) + L.log);
        HT *const hg = hg_of(s);
        ChainState st = *cst(s);
        const int64_t step0 = *step0_of(s);
        const float beta = in.betas[st.beta_idx];
        int len = 0, nrec = 0;
        // The state-independent draws of a record (race exponentials of the
        // lane's four positions, the multiplicity's Exp(1)), computed one
        // record ahead so that they fill the stalls of the current record's
        // dependent chain.
        float ex[4], e1;
        auto draws = [&](uint64_t step, float *x, float &e) {
            // (every lane draws: a lane past the set discards its words, and
            // the draws stay free of branches)
            const uint4 rw = rng_block(seed, TAG_RACE, chain_id, step, static_cast<uint32_t>(lane));
            x[0] = race_exp(rw.x);
            x[1] = race_exp(rw.y);
            x[2] = race_exp(rw.z);
            x[3] = race_exp(rw.w);
            e = record_draws(seed, chain_id, step, n, false, true).e1;
        };
        draws(static_cast<uint64_t>(st.step), ex, e1);
        // deferred tape entry (written one record late).  The multiplicities
        // are integers <= L0: the period's sum is kept in int64 and added to
        // the fp64 sum at the period end (exact: every partial sum is an
        // integer below 2^53), and the fp64 M is formed only for the tape
        int32_t pend_flip = 0;
        int64_t pend_m = 0;
        int64_t pend_pos = -1;
        int64_t sum_i = 0;
        // (the running minimum of E is also taken one record late, when its
        // operand is long ready)
        auto flush_record = [&]() {
            if (pend_pos >= 0) {
                if (lane == 0 && P.tape >= 1 && pend_pos < P.tape_cap) {
                    const int64_t o = static_cast<int64_t>(cid) * P.tape_cap + pend_pos;
                    P.tape_flip[o] = pend_flip;
                    P.tape_m[o] = static_cast<double>(pend_m);
                }
                sum_i += pend_m;
                st.best_E = fmin(st.best_E, st.E);
            }
            pend_pos = -1;
        };
        auto write_record = [&](int32_t flip, int64_t m) {  // flushed at the start of the next record
            pend_flip = flip;
            pend_m = m;
            pend_pos = st.step - step0;
        };
        auto bit_of = [&](int t) {
            const int i = s0 + t;
            return i >= n ? i - n : i;
        };
        auto delta_t = [&](int t, int i) -> D {
            const bool xi = (xw[i >> 5] >> (i & 31)) & 1u;
            return A::delta(insf[t], sub_b[t], sub_d[t], xi);
        };
        // One record on the set at s0; true at the period end.  Lane l
        // evaluates positions 4l .. 4l + 3 (k <= 128), whose race words are
        // the four words of Philox block l.
        auto one_record = [&]() -> bool {
            flush_record();  // the previous record (its E is the state this record starts from)
            const uint64_t step = static_cast<uint64_t>(st.step);
            if (P.tape == 2) {
                const int64_t pos = st.step - step0;
                if (pos < P.tape_cap) {
                    const int64_t o = static_cast<int64_t>(cid) * P.tape_cap + pos;
                    uint32_t *tx = P.tape_x + o * P.W;
                    for (int q = lane; q < P.W; q += 32) tx[q] = q < ld / 32 ? xw[q] : 0u;
                    if (lane == 0) P.tape_E[o] = st.E;
                }
            }
            const int t0 = 4 * lane;
            // branch-free over the lane's four positions: positions at or
            // past k read position k - 1 (in bounds) and are masked out
            const int tb = t0 < k ? t0 : ((k - 1) & ~3);  // (a 16-byte aligned block inside the set)
            HT hv[4];
            CT bv[4], dv[4];
            *reinterpret_cast<uint4 *>(hv) = *reinterpret_cast<const uint4 *>(insf + tb);
            *reinterpret_cast<uint4 *>(bv) = *reinterpret_cast<const uint4 *>(sub_b + tb);
            *reinterpret_cast<uint4 *>(dv) = *reinterpret_cast<const uint4 *>(sub_d + tb);
            D dl[4];
            bool in_set[4];
            uint32_t lmin = 0xFFFFFFFFu;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = t0 + u;
                in_set[u] = t < k;
                int i = s0 + (in_set[u] ? t : 0);
                i = i >= n ? i - n : i;
                const bool xi = (xw[i >> 5] >> (i & 31)) & 1u;
                dl[u] = A::delta(hv[u], bv[u], dv[u], xi);
                const uint32_t kd = A::key(A::pos(dl[u]));
                lmin = in_set[u] && kd < lmin ? kd : lmin;
            }
            float exn[4], e1n;
            draws(step + 1, exn, e1n);
            const D amin = A::unkey(__reduce_min_sync(0xFFFFFFFFu, lmin));
            const float af = A::tof(amin);
            const float anchor_e = det_expf(-__fmul_rn(beta, af));
            const float anchor_f = af > 0.0f ? anchor_e : 1.0f;
            uint32_t bkey = 0xFFFFFFFFu, bpos = 0xFFFFFFFFu, sa = 0u, sb = 0u;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = t0 + u;
                const float w = det_expf(-__fmul_rn(beta, A::diff(A::pos(dl[u]), amin)));
                const float ws = __fmul_rn(w, 65536.0f);
                const float wa = truncf(ws);
                const uint32_t qa = __float2uint_rz(wa);
                const uint32_t qb = __float2uint_rz(__fmul_rn(__fsub_rn(ws, wa), 65536.0f));
                sa += in_set[u] ? qa : 0u;
                sb += in_set[u] ? qb : 0u;
                const uint32_t kb = in_set[u] ? __float_as_uint(race_key(ex[u], w)) : 0xFFFFFFFFu;
                const bool better = kb < bkey;  // t ascending: the first minimum is kept
                bkey = better ? kb : bkey;
                bpos = better ? static_cast<uint32_t>(t) : bpos;
            }
            const uint32_t wkey = __reduce_min_sync(0xFFFFFFFFu, bkey);
            const uint32_t wpos = __reduce_min_sync(0xFFFFFFFFu, bkey == wkey ? bpos : 0xFFFFFFFFu);
            const uint32_t SA = __reduce_add_sync(0xFFFFFFFFu, sa);
            const uint32_t SB = __reduce_add_sync(0xFFFFFFFFu, sb);
            const uint64_t S = (static_cast<uint64_t>(SA) << 16) + static_cast<uint64_t>(SB);
            const int a = static_cast<int>(wpos);
            const int j = bit_of(a);
            const Mult mu = multiplicity_e1(S, k, anchor_f, e1);
#pragma unroll
            for (int u = 0; u < 4; ++u) ex[u] = exn[u];
            e1 = e1n;
            const D dj = delta_t(a, j);
            __syncwarp();
            bool period_end = false;
            const bool fits = mult_fits_small(mu, static_cast<int32_t>(st.L));  // (L0 < 2^31 here)
            if (fits) {
                // (a move's M fits the budget: below 2^31, exact)
                const int64_t m = mu.mi >= 0 ? mu.mi : static_cast<int64_t>(__float2int_rz(mu.fgl)) + 1;
                st.L -= m;
                if (mu.sat) st.saturated += 1;
                const bool up = ((xw[j >> 5] >> (j & 31)) & 1u) == 0u;
                if (lane == 0) prefetch_l2(Q + static_cast<int64_t>(j) * ld, row_bytes);
                const QT *srow = sub + a * k;
                for (int t = lane; t < k; t += 32) insf[t] = add_elem<QT, HT>(insf[t], srow[t], up);
                __syncwarp();
                if (lane == 0) {
                    xw[j >> 5] ^= 1u << (j & 31);
                    log[len] = j | (up ? static_cast<int32_t>(0x80000000u) : 0);
                }
                len += 1;
                st.E = __dadd_rn(st.E, A::tod(dj));
                st.flips += 1;
                write_record(j, m);
                __syncwarp();
                if (len == BLOCK_LOG) {  // full log: apply it now with this warp
                    const int nch = ld / VE;
                    for (int q = lane; q < nch; q += 32)
                        apply_item<QT, HT>(Q, ld, hg, log, len, q, s0, 0, k, n, nullptr);
                    __syncwarp();
                    len = 0;
                }
            } else {
                const int64_t m = st.L;
                st.L = P.L0;
                st.stays += 1;
                int ns = st.set_start + k;
                while (ns >= n) ns -= n;
                st.set_start = ns;
                st.period_start = static_cast<int64_t>(step) + 1;
                period_end = true;
                write_record(-1, m);
            }
            st.step += 1;
            nrec += 1;
            return period_end;
        };
        while (!one_record()) {
        }
        flush_record();
        st.sum_m = __dadd_rn(st.sum_m, static_cast<double>(sum_i));
        __syncwarp();
        if (lane == 0) {
            *cst(s) = st;
            *sc32(s, 0) = len;
            *sc32(s, 4) = nrec;
        }
        __syncwarp();
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
        const int nch = ld / VE;
        for (int q = lane; q < nch; q += 32) apply_item<QT, HT>(Q, ld, hg, log, len, q, s0, sn, k, n, last ? nullptr : insf);
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
                run_period(s);
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
                    for (int q = gtid; q < nch; q += GT)
                        apply_item<QT, HT>(Q, ld, hg, log, len, q, s0, sn, k, n, last ? nullptr : insf);
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
