// pns_sweep.cuh -- set-sweep evaluation of Unbiased PNS with systematic sets.
//
// With systematic sets the chain cycles through I = n / gcd(n, k) partial
// neighbour sets of k consecutive bits, each starting k bits after the last
// (Sec. 5, the wrap-around sets of size 14 for n = 16), and a record that
// stays ends its period without changing the state (x, h, E).  For a fixed
// state, everything a record computes except its own random numbers is
// therefore a function of the set alone: the deltas, the anchor, the weights,
// their quantised sum and the move probability p (Algorithm 6 with the
// uniform proposal over the set).  This kernel evaluates all I sets of the
// current state once -- the D warps of a chain own I / D sets each and leave
// the quantised weight sum S, the anchor A and the weights in shared memory
// -- and then one warp alone
// decides the records 32 at a time: record r lies on set (s0 + r k / g) mod I
// (g = gcd(n, k)), its budget is the current L for r = 0 and L0 after a stay,
// and it moves iff its multiplicity 1 + Geom(p) fits the budget (each lane
// forms e^{-beta A}, p and -ln(1 - p) of its record's set beside its Exp(1)).  Stays are committed in closed
// form without a barrier; the first mover's race (Proposition 5) reads its
// set's weights, and that warp applies the row before the team evaluates the
// new state.  The other warps wait at the barrier meanwhile, so the issue
// slots of the SM go to the chains that need them.  The records are
// bit-identical to one-at-a-time evaluation: every decision uses the same
// operations on the same values.
#pragma once

#include "pns_spec.cuh"

namespace pnsk {

struct SweepSmem {
    int32_t fields, xw, table, wts, kpad, ctl, total;
};

// Per chain: fields, bits, per set S and A, per set the k weights, a control
// word.
PNS_HD SweepSmem sweep_smem(int32_t ld, int32_t hbytes, int32_t k, int32_t nsets) {
    SweepSmem s;
    s.fields = 0;
    s.xw = round16(ld * hbytes);
    s.table = s.xw + round16(ld / 8);
    s.kpad = (k + 3) & ~3;
    s.wts = s.table + 16 * nsets;
    s.ctl = s.wts + 4 * s.kpad * nsets;
    s.total = s.ctl + 16;
    return s;
}

PNS_HD int32_t gcd32(int32_t a, int32_t b) {
    while (b != 0) {
        const int32_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// CPL: positions per lane, 1, 2 or 4 (k <= 32 CPL); a lane's positions lie in
// one Philox block of race words.  Positions at or past k are evaluated at
// position k - 1 and masked, so the loops carry no branches.
template <typename QT, typename HT, int D, int SPW, int CPL>
__global__ void __launch_bounds__(32 * D <= 512 ? 512 : 1024) pns_sweep_kernel(const KParams P) {
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
    const int w = tid >> 5;
    // the warp that decides the records: warp `team & 3`, so that the serial
    // warps of the chains sharing a CTA sit on different warp schedulers
    const int wser = team & 3;
    const int cid = P.cta_chains[cd.first + team];
    const ChainDesc chd = P.chain[cid];
    const InstDesc in = P.inst[chd.inst];
    const int n = in.n;
    const int ld = in.ld;
    const int k = in.k;
    const int g = gcd32(n, k);
    const int nsets = n / g;  // set starts are r0, r0 + g, ...; a period moves k / g of them on
    const int kstep = k / g;
    const SweepSmem L = sweep_smem(ld, static_cast<int32_t>(sizeof(HT)), k, nsets);
    unsigned char *base = smem + chd.smem_off;
    HT *h = reinterpret_cast<HT *>(base + L.fields);
    uint32_t *xw = reinterpret_cast<uint32_t *>(base + L.xw);
    uint4 *table = reinterpret_cast<uint4 *>(base + L.table);  // per set: S (lo, hi), A's key bits
    float *wts = reinterpret_cast<float *>(base + L.wts);
    volatile int32_t *ctl = reinterpret_cast<volatile int32_t *>(base + L.ctl);
    const CT *bvec = reinterpret_cast<const CT *>(in.b);
    const CT *dvec = reinterpret_cast<const CT *>(in.diag);
    const QT *Q = reinterpret_cast<const QT *>(in.q);
    const int bar = 1 + team;
    auto sync_team = [&]() { named_sync(bar, TT); };

    {
        const HT *gh = reinterpret_cast<const HT *>(P.fields) + static_cast<int64_t>(cid) * P.LD;
        const uint32_t *gx = P.xbits + static_cast<int64_t>(cid) * P.W;
        const int hchunks = ld * static_cast<int>(sizeof(HT)) / 16;
        for (int c = tid; c < hchunks; c += TT)
            reinterpret_cast<uint4 *>(h)[c] = reinterpret_cast<const uint4 *>(gh)[c];
        for (int q = tid; q < ld / 32; q += TT) xw[q] = gx[q];
    }
    ChainState st = P.state[cid];  // (kept by warp wser; the state of its lane 0 is written back)
    const float beta = in.betas[st.beta_idx];
    const uint64_t seed = P.seed;
    const uint32_t chain_id = static_cast<uint32_t>(cid) + P.chain_base;
    const int r0 = st.set_start % g;
    const int t0 = lane * CPL;
    int64_t tape_pos = 0;
    int64_t sum_int = 0;  // sum of this launch's multiplicities (exact integers <= L0)
    int64_t done = 0;
    // integer Q: the weights e^{-beta d} and their quantised parts come from
    // the chain's table (entry d for the integer d = delta+ - anchor; the last
    // entry and everything past it are zero)
    int32_t wt_n = 0;
    const float4 *wtab = nullptr;
    if constexpr (!std::is_same<HT, float>::value) {
        if (P.wtab_desc) {
            const int2 td = P.wtab_desc[cid];
            wt_n = td.y;
            wtab = P.wtab + td.x;
        }
    }
    sync_team();

    auto delta_of = [&](int i) -> D_t {
        const bool xi = (xw[i >> 5] >> (i & 31)) & 1u;
        return A::delta(h[i], bvec[i], dvec[i], xi);
    };

    while (done < P.steps) {
        // ---- every set of the current state: S, A, the weights ---------------
        {
            // the warp's sets in lockstep (a warp without an own set evaluates
            // a copy of another and stores nothing)
            int sg[SPW];
            bool own[SPW];
#pragma unroll
            for (int u = 0; u < SPW; ++u) {
                const int s_ = w + u * D;
                own[u] = s_ < nsets;
                sg[u] = own[u] ? s_ : s_ % nsets;
            }
            D_t dl[SPW][CPL];
            uint32_t lmin[SPW];
#pragma unroll
            for (int u = 0; u < SPW; ++u) {
                lmin[u] = 0xFFFFFFFFu;
#pragma unroll
                for (int v = 0; v < CPL; ++v) {
                    const int t = t0 + v;
                    int i = sg[u] * g + r0 + (t < k ? t : k - 1);
                    i = i >= n ? i - n : i;
                    dl[u][v] = delta_of(i);
                    const uint32_t kd = A::key(A::pos(dl[u][v]));
                    lmin[u] = t < k && kd < lmin[u] ? kd : lmin[u];
                }
            }
            D_t amin[SPW];
#pragma unroll
            for (int u = 0; u < SPW; ++u) amin[u] = A::unkey(__reduce_min_sync(0xFFFFFFFFu, lmin[u]));
            uint32_t sa[SPW], sb[SPW];
#pragma unroll
            for (int u = 0; u < SPW; ++u) {
                sa[u] = 0u;
                sb[u] = 0u;
            }
            bool tabled = false;
            if constexpr (!std::is_same<HT, float>::value) {
                if (wt_n > 0) {  // (the same for the whole chain)
                    tabled = true;
#pragma unroll
                    for (int u = 0; u < SPW; ++u) {
#pragma unroll
                        for (int v = 0; v < CPL; ++v) {
                            const int t = t0 + v;
                            const int32_t d = A::pos(dl[u][v]) - amin[u];
                            const float4 e = __ldg(wtab + (d < wt_n ? d : wt_n - 1));
                            sa[u] += t < k ? __float_as_uint(e.y) : 0u;
                            sb[u] += t < k ? __float_as_uint(e.z) : 0u;
                            if (own[u] && t < k) wts[sg[u] * L.kpad + t] = e.x;
                        }
                    }
                }
            }
            if (!tabled) {
#pragma unroll
                for (int u = 0; u < SPW; ++u) {
#pragma unroll
                    for (int v = 0; v < CPL; ++v) {
                        const int t = t0 + v;
                        const float wv = det_expf(-__fmul_rn(beta, A::diff(A::pos(dl[u][v]), amin[u])));
                        const float ws = __fmul_rn(wv, 65536.0f);
                        const float wa = truncf(ws);
                        sa[u] += t < k ? __float2uint_rz(wa) : 0u;
                        sb[u] += t < k ? __float2uint_rz(__fmul_rn(__fsub_rn(ws, wa), 65536.0f)) : 0u;
                        if (own[u] && t < k) wts[sg[u] * L.kpad + t] = wv;
                    }
                }
            }
            // the per-set scalars, lane u for set u: S and the anchor A
            uint32_t abits = 0u;
            uint64_t S = 0;
            int my_sg = 0;
            bool my_own = false;
#pragma unroll
            for (int u = 0; u < SPW; ++u) {
                const uint32_t SA = __reduce_add_sync(0xFFFFFFFFu, sa[u]);
                const uint32_t SB = __reduce_add_sync(0xFFFFFFFFu, sb[u]);
                if (lane == u) {
                    abits = A::key(amin[u]);
                    S = (static_cast<uint64_t>(SA) << 16) + static_cast<uint64_t>(SB);
                    my_sg = sg[u];
                    my_own = own[u];
                }
            }
            if (lane < SPW && my_own)
                table[my_sg] = make_uint4(static_cast<uint32_t>(S), static_cast<uint32_t>(S >> 32), abits, 0u);
        }
        sync_team();
        // ---- warp wser: records 32 at a time up to the first mover ----------
        if (w == wser) {
            bool moved = false;
            while (!moved && done < P.steps) {
                const int64_t left = P.steps - done;
                const int nb = left < 32 ? static_cast<int>(left) : 32;
                const uint64_t step0 = static_cast<uint64_t>(st.step);
                const int sig0 = st.set_start / g;
                int sg = sig0 + (lane * kstep) % nsets;  // set of record lane after lane stays
                sg = sg >= nsets ? sg - nsets : sg;
                // (every lane decides; lanes past the last record are masked)
                const uint4 te = table[sg];
                const float e1 = record_draws(seed, chain_id, step0 + lane, n, false, true).e1;
                // e^{-beta A}, p and -ln(1 - p) (used only when 0 < p < 1) of
                // the record's set, evaluated beside its Exp(1)
                const D_t amin = A::unkey(te.z);
                const float af = A::tof(amin);
                float anchor_e;
                if constexpr (!std::is_same<HT, float>::value) {
                    if (wt_n > 0) anchor_e = __ldg(wtab + (amin < wt_n ? amin : wt_n - 1)).x;  // (uniform)
                    else anchor_e = det_expf(-__fmul_rn(beta, af));
                } else {
                    anchor_e = det_expf(-__fmul_rn(beta, af));
                }
                const float anchor_f = af > 0.0f ? anchor_e : 1.0f;
                const float p = mult_p((static_cast<uint64_t>(te.y) << 32) | te.x, k, anchor_f);
                const Mult mu = mult_from(p, det_neg_log1m(p), e1);
                const bool fits =
                    lane < nb && mult_fits_small(mu, static_cast<int32_t>(lane == 0 ? st.L : P.L0));  // (L0 < 2^31)
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, fits);
                moved = bal != 0u;
                const int first = moved ? __ffs(static_cast<int>(bal)) - 1 : nb;
                const int ncommit = moved ? first + 1 : nb;
                const int nstay = first;
                int j = -1, mi = 0, sat = 0;
                D_t dj = 0;
                constexpr int VE = 16 / static_cast<int>(sizeof(QT));
                constexpr int PRE = 4;
                const int chunks = ld / VE;
                uint4 pre[PRE];  // the mover's row: its first chunks are loaded ahead of the bookkeeping
                if (moved) {
                    mi = __shfl_sync(0xFFFFFFFFu,
                                     static_cast<int32_t>(mu.mi >= 0 ? mu.mi : static_cast<int64_t>(mu.fgl) + 1), first);
                    sat = __shfl_sync(0xFFFFFFFFu, mu.sat, first);
                    const int sf = __shfl_sync(0xFFFFFFFFu, sg, first);
                    // the mover's race on its set's stored weights
                    const uint64_t step = step0 + first;
                    const float *wv = wts + sf * L.kpad;
                    uint32_t bkey = 0xFFFFFFFFu, bpos = 0xFFFFFFFFu;
                    const uint4 blk = rng_block(seed, TAG_RACE, chain_id, step, static_cast<uint32_t>(t0 >> 2));
#pragma unroll
                    for (int v = 0; v < CPL; ++v) {
                        const int t = t0 + v;
                        const float ex = race_exp(pick_word(blk, static_cast<uint32_t>(t) & 3u));
                        const uint32_t kb = t < k ? __float_as_uint(race_key(ex, wv[t < k ? t : k - 1])) : 0xFFFFFFFFu;
                        const bool better = kb < bkey;  // t ascending per lane: the first minimum is kept
                        bkey = better ? kb : bkey;
                        bpos = better ? static_cast<uint32_t>(t) : bpos;
                    }
                    const uint32_t wkey = __reduce_min_sync(0xFFFFFFFFu, bkey);
                    const uint32_t wpos = __reduce_min_sync(0xFFFFFFFFu, bkey == wkey ? bpos : 0xFFFFFFFFu);
                    j = sf * g + r0 + static_cast<int>(wpos);
                    j = j >= n ? j - n : j;
                    dj = delta_of(j);
                    const QT *row = Q + static_cast<int64_t>(j) * ld;
#pragma unroll
                    for (int u = 0; u < PRE; ++u)
                        if (lane + 32 * u < chunks) pre[u] = ld_nc_v4(row + (lane + 32 * u) * VE);
                }
                // tape: record r stays with M = its budget, or is the mover
                if (P.tape == 2) {
                    for (int idx = lane; idx < ncommit * P.W; idx += 32) {
                        const int q = idx / P.W, wd = idx - q * P.W;
                        if (tape_pos + q < P.tape_cap) {
                            const int64_t o = static_cast<int64_t>(cid) * P.tape_cap + tape_pos + q;
                            P.tape_x[o * P.W + wd] = wd < ld / 32 ? xw[wd] : 0u;
                        }
                    }
                    if (lane == 0)  // (the energy is kept by lane 0)
                        for (int q = 0; q < ncommit && tape_pos + q < P.tape_cap; ++q)
                            P.tape_E[static_cast<int64_t>(cid) * P.tape_cap + tape_pos + q] = st.E;
                }
                if (P.tape && lane < ncommit && tape_pos + lane < P.tape_cap) {
                    const int64_t o = static_cast<int64_t>(cid) * P.tape_cap + tape_pos + lane;
                    const bool mv = moved && lane == first;
                    const int64_t Lq = lane == 0 ? st.L : P.L0;
                    P.tape_flip[o] = mv ? j : -1;
                    P.tape_m[o] = static_cast<double>(mv ? static_cast<int64_t>(mi) : Lq);
                }
                // bookkeeping of the committed records, in closed form
                if (nstay > 0) {
                    sum_int += st.L + static_cast<int64_t>(nstay - 1) * P.L0;
                    st.L = P.L0;
                    // (set_start < n, nstay <= 32, k <= 128: 32-bit arithmetic)
                    st.set_start = static_cast<int>(static_cast<uint32_t>(st.set_start + nstay * k) %
                                                    static_cast<uint32_t>(n));
                    st.period_start = static_cast<int64_t>(step0) + nstay;
                }
                st.stays += nstay;
                if (moved) {
                    st.L -= mi;
                    sum_int += mi;
                    if (sat) st.saturated += 1;
                    st.flips += 1;
                    const bool up = ((xw[j >> 5] >> (j & 31)) & 1u) == 0u;
                    const QT *row = Q + static_cast<int64_t>(j) * ld;
#pragma unroll
                    for (int u = 0; u < PRE; ++u)
                        if (lane + 32 * u < chunks) add_chunk<QT, HT>(h + (lane + 32 * u) * VE, pre[u], up);
                    int c = lane + 32 * PRE;
                    for (; c + 3 * 32 < chunks; c += 4 * 32) {
                        const uint4 v0 = ld_nc_v4(row + (c + 0 * 32) * VE);
                        const uint4 v1 = ld_nc_v4(row + (c + 1 * 32) * VE);
                        const uint4 v2 = ld_nc_v4(row + (c + 2 * 32) * VE);
                        const uint4 v3 = ld_nc_v4(row + (c + 3 * 32) * VE);
                        add_chunk<QT, HT>(h + (c + 0 * 32) * VE, v0, up);
                        add_chunk<QT, HT>(h + (c + 1 * 32) * VE, v1, up);
                        add_chunk<QT, HT>(h + (c + 2 * 32) * VE, v2, up);
                        add_chunk<QT, HT>(h + (c + 3 * 32) * VE, v3, up);
                    }
                    for (; c < chunks; c += 32) add_chunk<QT, HT>(h + c * VE, ld_nc_v4(row + c * VE), up);
                    __syncwarp();  // (every lane has read x_j)
                    if (lane == 0) {
                        xw[j >> 5] ^= 1u << (j & 31);
                        st.E = __dadd_rn(st.E, A::tod(dj));
                        st.best_E = fmin(st.best_E, st.E);
                    }
                }
                st.step += ncommit;
                tape_pos += ncommit;
                done += ncommit;
            }
            if (lane == 0) ctl[0] = static_cast<int32_t>(done < P.steps);
        }
        sync_team();
        if (!ctl[0]) break;  // (ctl is written again only after the next evaluation's barrier)
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
    if (tid == 32 * wser) {
        st.sum_m = __dadd_rn(st.sum_m, static_cast<double>(sum_int));
        st.tape_records = P.tape ? (tape_pos < P.tape_cap ? tape_pos : P.tape_cap) : 0;
        P.state[cid] = st;
    }
}

}  // namespace pnsk
