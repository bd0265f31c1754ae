// pns_spec.cuh -- speculative record evaluation for Unbiased PNS and
// Metropolis.
//
// A record that does not move leaves the chain state (x, h, E) unchanged, and
// the records after it are then fully determined: Unbiased PNS resets the
// budget to L0 and moves to the next partial neighbour set; Metropolis just
// proposes again.  So with D warps per chain, warp w evaluates record
// step + w under the assumption that records step .. step + w - 1 all stay.
// The first record that moves (or all D records, if none does) is exactly
// what the sequential chain would have produced; the records after it are
// discarded.  The committed records are bit-identical to one-at-a-time
// evaluation; at low temperature, where most records are stays, one round
// commits several records for the latency of one.
#pragma once

#include "pns_sampler.cuh"

namespace pnsk {

// Shared-memory layout of one chain in the speculative kernel: fields, bits,
// D subset lists and bitmaps (random sets only), D result slots, scratch.
struct SpecSmem {
    int32_t fields, xw, lists, list_bytes, bitmaps, bitmap_bytes, slots, scratch, total;
};

PNS_HD SpecSmem spec_smem(int32_t ld, int32_t k, int32_t hbytes, bool list, int32_t D) {
    SpecSmem s;
    s.fields = 0;
    s.xw = round16(ld * hbytes);
    s.lists = s.xw + round16(ld / 8);
    s.list_bytes = list ? round16(4 * k) : 0;
    s.bitmaps = s.lists + D * s.list_bytes;
    s.bitmap_bytes = list ? round16(ld / 8) : 0;
    s.slots = s.bitmaps + D * s.bitmap_bytes;
    s.scratch = s.slots + 32 * D;
    s.total = s.scratch + 64;
    return s;
}

// Result of one speculative record, written by lane 0 of its warp.
struct SpecSlot {
    int32_t move;    // 1: the record moves (its assumptions make it the first mover)
    int32_t j;       // bit to flip
    int32_t sat;     // multiplicity saturated
    int32_t dj;      // delta of bit j (int32 bits or float bits)
    int32_t mi;      // multiplicity of a move (<= L0 < 2^31, an exact integer)
    int32_t pad[3];
};
static_assert(sizeof(SpecSlot) == 32, "slot layout");

template <typename QT, typename HT, int D>
__global__ void __launch_bounds__(32 * D <= 512 ? 512 : 1024) pns_spec_kernel(const KParams P) {
    using A = Arith<HT>;
    using D_t = typename A::D;
    using CT = typename A::C;
    constexpr int TT = 32 * D;
    extern __shared__ __align__(16) unsigned char smem[];
    const CtaDesc cd = P.cta[blockIdx.x];
    const int team = threadIdx.x / TT;
    if (team >= cd.count) return;
    const int tid = threadIdx.x - team * TT;
    const int lane = threadIdx.x & 31;
    const int w = tid >> 5;  // speculative offset of this warp
    const int cid = P.cta_chains[cd.first + team];
    const ChainDesc chd = P.chain[cid];
    const InstDesc in = P.inst[chd.inst];
    const int n = in.n;
    const int ld = in.ld;
    const int variant = P.variant;
    const bool use_list = needs_list(variant, P.subset);
    const int k = variant == VAR_METROPOLIS ? 1 : in.k;
    const SpecSmem L = spec_smem(ld, k, static_cast<int32_t>(sizeof(HT)), use_list, D);
    unsigned char *base = smem + chd.smem_off;
    HT *h = reinterpret_cast<HT *>(base + L.fields);
    uint32_t *xw = reinterpret_cast<uint32_t *>(base + L.xw);
    SpecSlot *slots = reinterpret_cast<SpecSlot *>(base + L.slots);
    int32_t *ctl = reinterpret_cast<int32_t *>(base + L.scratch);
    const CT *bvec = reinterpret_cast<const CT *>(in.b);
    const CT *dvec = reinterpret_cast<const CT *>(in.diag);
    const int bar = 1 + team;
    auto sync_team = [&]() {
        if constexpr (D == 1) __syncwarp();
        else named_sync(bar, TT);
    };

    {
        const HT *gh = reinterpret_cast<const HT *>(P.fields) + static_cast<int64_t>(cid) * P.LD;
        const uint32_t *gx = P.xbits + static_cast<int64_t>(cid) * P.W;
        const int hchunks = ld * static_cast<int>(sizeof(HT)) / 16;
        for (int c = tid; c < hchunks; c += TT)
            reinterpret_cast<uint4 *>(h)[c] = reinterpret_cast<const uint4 *>(gh)[c];
        for (int q = tid; q < ld / 32; q += TT) xw[q] = gx[q];
    }
    if (tid == 0) {
        ctl[0] = 0;
        ctl[1] = 0;
    }
    ChainState st = P.state[cid];
    const float beta = in.betas[st.beta_idx];
    const uint64_t seed = P.seed;
    const uint32_t chain_id = static_cast<uint32_t>(cid) + P.chain_base;
    int cur_list = 0;          // list buffer holding the current period's set
    bool list_valid = false;
    int64_t tape_pos = 0;
    int64_t sum_int = 0;       // sum of this launch's multiplicities (exact integers)
    int dead = 0;
    sync_team();

    auto delta_of = [&](int i) -> D_t {
        const bool xi = (xw[i >> 5] >> (i & 31)) & 1u;
        return A::delta(h[i], bvec[i], dvec[i], xi);
    };

    int64_t done = 0;
    while (done < P.steps && !dead) {
        const int64_t left = P.steps - done;
        const int Dr = left < D ? static_cast<int>(left) : D;
        const uint64_t step0 = static_cast<uint64_t>(st.step);
        // ---- warp w: record step0 + w, assuming the earlier ones stayed ----
        if (w < Dr) {
            const uint64_t step = step0 + w;
            const int64_t Lw = w == 0 ? st.L : P.L0;
            SpecSlot res;
            res.move = 0;
            res.j = -1;
            res.sat = 0;
            res.dj = 0;
            res.mi = 0;
            res.pad[0] = res.pad[1] = res.pad[2] = 0;
            const bool met = variant == VAR_METROPOLIS;
            const RecordDraws rd = record_draws(seed, chain_id, step, n, met, !met);
            if (variant == VAR_METROPOLIS) {
                const D_t d = delta_of(rd.mi);
                const float y = -__fmul_rn(beta, A::tof(d));
                if (rd.mlu < y) {
                    res.move = 1;
                    res.j = rd.mi;
                    res.mi = 1;
                    if constexpr (std::is_same<D_t, float>::value) res.dj = __float_as_int(d);
                    else res.dj = d;
                }
            } else {
                // the set of this record
                int start = st.set_start;
                const int32_t *lst = nullptr;
                if (use_list) {
                    int buf = (cur_list + w) % D;
                    int32_t *lb = reinterpret_cast<int32_t *>(base + L.lists + buf * L.list_bytes);
                    uint32_t *bm = reinterpret_cast<uint32_t *>(base + L.bitmaps + buf * L.bitmap_bytes);
                    if (!(w == 0 && list_valid)) {
                        const uint64_t ps = w == 0 ? static_cast<uint64_t>(st.period_start) : step;
                        if (!draw_subset_warp(seed, chain_id, ps, n, k, ld, lb, bm, lane, P.draw_cap)) {
                            if (lane == 0) {
                                set_status(P.status, ST_TIMEOUT);
                                ctl[1] = 1;
                            }
                        }
                    }
                    lst = lb;
                } else {
                    // start advances by k per skipped period
                    // (32-bit: set_start < n, w < D <= 16, k <= 128)
                    start = static_cast<int>(static_cast<uint32_t>(st.set_start + w * k) % static_cast<uint32_t>(n));
                }
                auto cand = [&](int t) -> int {
                    if (lst) return lst[t];
                    int c = start + t;
                    return c >= n ? c - n : c;
                };
                uint32_t lmin = 0xFFFFFFFFu;
                D_t dl[CPT];
                const bool fast = k <= 32 * CPT;
                // fast path: lane handles cpl consecutive positions, so one
                // Philox block (four words) serves up to four of them
                const int cpl = (k + 31) >> 5;
                const int t0 = lane * cpl;
                if (fast) {
#pragma unroll
                    for (int u = 0; u < CPT; ++u) {
                        const int t = t0 + u;
                        if (u < cpl && t < k) {
                            dl[u] = delta_of(cand(t));
                            const uint32_t kd = A::key(A::pos(dl[u]));
                            lmin = kd < lmin ? kd : lmin;
                        }
                    }
                } else {
                    for (int t = lane; t < k; t += 32) {
                        const uint32_t kd = A::key(A::pos(delta_of(cand(t))));
                        lmin = kd < lmin ? kd : lmin;
                    }
                }
                const D_t amin = A::unkey(__reduce_min_sync(0xFFFFFFFFu, lmin));
                const float af = A::tof(amin);
                const float anchor_e = det_expf(-__fmul_rn(beta, af));
                const float anchor_f = af > 0.0f ? anchor_e : 1.0f;
                // Weights and their quantised sum first: the multiplicity
                // alone decides a stay, and a stay needs no race winner, so
                // the race (exponentials, divisions, argmin) runs only for a
                // record that moves.  Its random numbers are counter-based,
                // so the order of evaluation does not change them.
                uint32_t sa = 0u, sb = 0u;
                float wt[CPT];
                auto weight = [&](D_t dv) -> float {
                    const float wv = det_expf(-__fmul_rn(beta, A::diff(A::pos(dv), amin)));
                    const float ws = __fmul_rn(wv, 65536.0f);
                    const float wa = truncf(ws);
                    sa += __float2uint_rz(wa);
                    sb += __float2uint_rz(__fmul_rn(__fsub_rn(ws, wa), 65536.0f));
                    return wv;
                };
                if (fast) {
#pragma unroll
                    for (int u = 0; u < CPT; ++u) {
                        const int t = t0 + u;
                        if (u < cpl && t < k) wt[u] = weight(dl[u]);
                    }
                } else {
                    for (int t = lane; t < k; t += 32) weight(delta_of(cand(t)));
                }
                const uint32_t SA = __reduce_add_sync(0xFFFFFFFFu, sa);
                const uint32_t SB = __reduce_add_sync(0xFFFFFFFFu, sb);
                const uint64_t S = (static_cast<uint64_t>(SA) << 16) + static_cast<uint64_t>(SB);
                const Mult mu = multiplicity_e1(S, k, anchor_f, rd.e1);
                const bool fits = mult_fits_small(mu, static_cast<int32_t>(Lw));  // (L0 < 2^31 here)
                if (fits) {  // (uniform across the warp)
                    uint32_t bkey = 0xFFFFFFFFu, bpos = 0xFFFFFFFFu;
                    auto race = [&](int t, float wv, uint32_t word) {
                        const uint32_t kb = __float_as_uint(race_key(race_exp(word), wv));
                        if (kb < bkey) {  // t ascending per lane: the first minimum is kept
                            bkey = kb;
                            bpos = static_cast<uint32_t>(t);
                        }
                    };
                    if (fast) {
                        uint4 blk = rng_block(seed, TAG_RACE, chain_id, step, static_cast<uint32_t>(t0 >> 2));
                        uint32_t cur_b = static_cast<uint32_t>(t0 >> 2);
#pragma unroll
                        for (int u = 0; u < CPT; ++u) {
                            const int t = t0 + u;
                            if (u < cpl && t < k) {
                                const uint32_t bt = static_cast<uint32_t>(t) >> 2;
                                if (bt != cur_b) {
                                    blk = rng_block(seed, TAG_RACE, chain_id, step, bt);
                                    cur_b = bt;
                                }
                                race(t, wt[u], pick_word(blk, static_cast<uint32_t>(t) & 3u));
                            }
                        }
                    } else {
                        for (int t = lane; t < k; t += 32) {
                            const D_t dv = delta_of(cand(t));
                            const float wv = det_expf(-__fmul_rn(beta, A::diff(A::pos(dv), amin)));
                            race(t, wv, rng_word(seed, TAG_RACE, chain_id, step, static_cast<uint32_t>(t)));
                        }
                    }
                    const uint32_t wkey = __reduce_min_sync(0xFFFFFFFFu, bkey);
                    const uint32_t wpos = __reduce_min_sync(0xFFFFFFFFu, bkey == wkey ? bpos : 0xFFFFFFFFu);
                    const int j = cand(static_cast<int>(wpos));
                    const D_t dj = delta_of(j);
                    res.move = 1;
                    res.j = j;
                    res.sat = mu.sat;
                    res.mi = static_cast<int32_t>(mu.mi >= 0 ? mu.mi : static_cast<int64_t>(mu.fgl) + 1);
                    if constexpr (std::is_same<D_t, float>::value) res.dj = __float_as_int(dj);
                    else res.dj = dj;
                }
            }
            if (lane == 0) slots[w] = res;
        }
        sync_team();
        if (use_list && ctl[1]) dead = 1;
        // ---- commit: the records up to and including the first mover -------
        uint32_t movers = 0u;  // (independent shared loads, no dependent scan)
#pragma unroll
        for (int q = 0; q < D; ++q)
            if (q < Dr && slots[q].move) movers |= 1u << q;
        const int first = movers ? __ffs(static_cast<int>(movers)) - 1 : Dr;
        const int ncommit = first < Dr ? first + 1 : Dr;
        if (P.tape == 2) {
            // every committed record starts from the current state
            for (int idx = tid; idx < ncommit * P.W; idx += TT) {
                const int q = idx / P.W, wd = idx - q * P.W;
                if (tape_pos + q < P.tape_cap) {
                    const int64_t o = static_cast<int64_t>(cid) * P.tape_cap + tape_pos + q;
                    P.tape_x[o * P.W + wd] = wd < ld / 32 ? xw[wd] : 0u;
                }
            }
            if (tid == 0)  // (the energy is kept by thread 0)
                for (int q = 0; q < ncommit && tape_pos + q < P.tape_cap; ++q)
                    P.tape_E[static_cast<int64_t>(cid) * P.tape_cap + tape_pos + q] = st.E;
        }
        if (w < ncommit && lane == 0 && P.tape && tape_pos + w < P.tape_cap) {
            const int64_t o = static_cast<int64_t>(cid) * P.tape_cap + tape_pos + w;
            const bool mv = w == first;
            const int64_t Lq = w == 0 ? st.L : P.L0;
            P.tape_flip[o] = mv ? slots[w].j : -1;
            P.tape_m[o] = static_cast<double>(mv ? static_cast<int64_t>(slots[w].mi) : (variant == VAR_METROPOLIS ? 1 : Lq));
        }
        // budget / set bookkeeping of the committed records, in closed form:
        // records 0 .. nstay-1 stay (each a period end for Unbiased PNS:
        // record (stay, L), L <- L0, next set), then the mover if any
        const int nstay = first < Dr ? first : Dr;
        if (variant == VAR_UNBIASED) {
            if (nstay > 0) {
                sum_int += st.L + static_cast<int64_t>(nstay - 1) * P.L0;
                st.L = P.L0;
                // (set_start < n, nstay <= D <= 16, k <= 128: 32-bit arithmetic)
                st.set_start = static_cast<int>(static_cast<uint32_t>(st.set_start + nstay * k) %
                                                static_cast<uint32_t>(n));
                st.period_start = static_cast<int64_t>(step0) + nstay;
            }
            if (first < Dr) {
                const int64_t mi = slots[first].mi;
                st.L -= mi;
                sum_int += mi;
            }
        } else {
            sum_int += ncommit;
        }
        st.stays += nstay;
        if (use_list) {
            if (first < Dr) {
                // the mover's set is the current one from now on
                cur_list = (cur_list + first) % D;
                list_valid = true;
            } else {
                list_valid = false;
                cur_list = (cur_list + Dr) % D;
            }
        }
        if (first < Dr) {
            const SpecSlot mv = slots[first];
            if (mv.sat) st.saturated += 1;
            st.flips += 1;
            // all warps apply the row
            const int j = mv.j;
            const bool up = ((xw[j >> 5] >> (j & 31)) & 1u) == 0u;
            constexpr int VE = 16 / static_cast<int>(sizeof(QT));
            const QT *row = reinterpret_cast<const QT *>(in.q) + static_cast<int64_t>(j) * ld;
            const int chunks = ld / VE;
            int c = tid;
            for (; c + 3 * TT < chunks; c += 4 * TT) {
                const uint4 v0 = ld_nc_v4(row + (c + 0 * TT) * VE);
                const uint4 v1 = ld_nc_v4(row + (c + 1 * TT) * VE);
                const uint4 v2 = ld_nc_v4(row + (c + 2 * TT) * VE);
                const uint4 v3 = ld_nc_v4(row + (c + 3 * TT) * VE);
                add_chunk<QT, HT>(h + (c + 0 * TT) * VE, v0, up);
                add_chunk<QT, HT>(h + (c + 1 * TT) * VE, v1, up);
                add_chunk<QT, HT>(h + (c + 2 * TT) * VE, v2, up);
                add_chunk<QT, HT>(h + (c + 3 * TT) * VE, v3, up);
            }
            for (; c < chunks; c += TT) add_chunk<QT, HT>(h + c * VE, ld_nc_v4(row + c * VE), up);
            sync_team();
            if (tid == 0) {
                xw[j >> 5] ^= 1u << (j & 31);
                // the fp64 energy lives in thread 0 only (GB300's fp64 pipe is narrow)
                double dE;
                if constexpr (std::is_same<D_t, float>::value) dE = static_cast<double>(__int_as_float(mv.dj));
                else dE = static_cast<double>(mv.dj);
                st.E = __dadd_rn(st.E, dE);
                st.best_E = fmin(st.best_E, st.E);
            }
        }
        st.step += ncommit;
        tape_pos += ncommit;
        done += ncommit;
        sync_team();
    }

    // ---- write back ---------------------------------------------------------
    {
        HT *gh = reinterpret_cast<HT *>(P.fields) + static_cast<int64_t>(cid) * P.LD;
        uint32_t *gx = P.xbits + static_cast<int64_t>(cid) * P.W;
        const int hchunks = ld * static_cast<int>(sizeof(HT)) / 16;
        for (int c = tid; c < hchunks; c += TT)
            reinterpret_cast<uint4 *>(gh)[c] = reinterpret_cast<const uint4 *>(h)[c];
        for (int q = tid; q < ld / 32; q += TT) gx[q] = xw[q];
    }
    if (tid == 0) {
        // the multiplicities of Unbiased PNS are integers <= L0 < 2^31 and
        // Metropolis adds 1 per record, so the fp64 sum is exact and equals
        // the record-by-record accumulation
        st.sum_m = __dadd_rn(st.sum_m, static_cast<double>(sum_int));
        st.tape_records = P.tape ? (tape_pos < P.tape_cap ? tape_pos : P.tape_cap) : 0;
        P.state[cid] = st;
    }
}

}  // namespace pnsk
