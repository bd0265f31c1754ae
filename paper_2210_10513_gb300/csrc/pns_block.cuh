// pns_block.cuh -- period-blocked Unbiased PNS with replica exchange.
//
// Within one period of Unbiased PNS (Algorithm 6) a chain proposes and flips
// only bits of its current systematic set N_i, so only the k fields of N_i are
// ever read.  This kernel keeps those k fields in shared memory, current from
// the k x k sub-block Q[N_i, N_i], and logs the period's flips; every other
// field (in global memory) receives the logged rows at the period end, when
// all rows are known and can be loaded together instead of one dependent row
// load per flip.  Each field still receives the same IEEE additions in the
// same order as with the per-flip update (h_r += s_j Q_rj over the flips j in
// time order), so fields, energies and records are bit-identical to the
// per-flip kernel for integer and fp32 QUBOs alike.
//
// The replicas of an exchange group move through the same systematic sets
// (each completes one period per L0 original samples and the group meets at
// every period end), so one sub-block serves the whole group.  Per period:
//   records   each chain (one warp) runs its records to the period end; a
//             move updates the k set fields from the sub-block and appends
//             (j, direction) to the chain's log
//   exchange  at round ends adjacent temperatures swap, as in the per-flip
//             kernel (same random numbers and arithmetic)
//   apply     the group applies every chain's log to its fields outside N_i
//             (16-byte row chunks, APPLY_U rows in flight per thread) and
//             gathers the next set's fields, while the next sub-block arrives
//             by cp.async
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
__device__ __forceinline__ void apply_item(const QT *Q, int ld, HT *hg, const int32_t *log, int len, int q,
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

template <typename QT, typename HT>
__global__ void __launch_bounds__(512) pns_block_kernel(const KParams P) {
    using A = Arith<HT>;
    using D = typename A::D;
    using CT = typename A::C;
    constexpr int VE = 16 / static_cast<int>(sizeof(QT));

    extern __shared__ __align__(16) unsigned char smem[];
    const CtaDesc cd = P.cta[blockIdx.x];
    const int team = threadIdx.x >> 5;
    if (team >= cd.count) return;  // idle warps take part in no barrier
    const int lane = threadIdx.x & 31;
    const int R = P.R;
    const int pos = team % R;  // position inside the exchange group
    const int cid = P.cta_chains[cd.first + team];
    const ChainDesc chd = P.chain[cid];
    const InstDesc in = P.inst[chd.inst];
    const int n = in.n;
    const int ld = in.ld;
    const int k = in.k;
    const QT *Q = reinterpret_cast<const QT *>(in.q);
    const BlockSmem L = block_smem(ld, k, static_cast<int32_t>(sizeof(HT)), static_cast<int32_t>(sizeof(QT)), R);
    unsigned char *gbase = smem + P.chain[P.cta_chains[cd.first + team - pos]].smem_off;
    auto area = [&](int p) { return gbase + p * L.chain_bytes; };
    unsigned char *base = area(pos);
    HT *insf = reinterpret_cast<HT *>(base + L.insf);  // fields of the current set, position t
    HT *const hg = reinterpret_cast<HT *>(P.fields) + static_cast<int64_t>(cid) * P.LD;
    uint32_t *xw = reinterpret_cast<uint32_t *>(base + L.xw);
    int32_t *log = reinterpret_cast<int32_t *>(base + L.log);
    double *pub_E = reinterpret_cast<double *>(base + L.scratch);
    int32_t *pub_b = reinterpret_cast<int32_t *>(base + L.scratch + 8);
    int32_t *swap_cnt = reinterpret_cast<int32_t *>(base + L.scratch + 12);
    int32_t *pub_set = reinterpret_cast<int32_t *>(base + L.scratch + 16);
    int32_t *pub_len = reinterpret_cast<int32_t *>(base + L.scratch + 20);
    QT *sub = reinterpret_cast<QT *>(gbase + L.sub);
    CT *sub_b = reinterpret_cast<CT *>(gbase + L.bd);
    CT *sub_d = sub_b + k;
    const CT *bvec = reinterpret_cast<const CT *>(in.b);
    const CT *dvec = reinterpret_cast<const CT *>(in.diag);

    // one named barrier per exchange group (id 0 is __syncthreads')
    const int gbar = 1 + team / R;
    const int GT = 32 * R;
    const int gtid = pos * 32 + lane;
    auto gsync = [&]() { named_sync(gbar, GT); };

    // ---- load the chain ------------------------------------------------------
    ChainState st = P.state[cid];
    {
        const uint32_t *gx = P.xbits + static_cast<int64_t>(cid) * P.W;
        for (int w = lane; w < ld / 32; w += 32) xw[w] = gx[w];
        for (int t = lane; t < k; t += 32) {
            int r = st.set_start + t;
            if (r >= n) r -= n;
            insf[t] = hg[r];
        }
    }
    const uint64_t seed = P.seed;
    const uint32_t chain_id = static_cast<uint32_t>(cid) + P.chain_base;
    float beta = in.betas[st.beta_idx];
    if (lane == 0) {
        *swap_cnt = 0;
        *pub_set = st.set_start;
    }
    gsync();
    // every replica of the group must stand at the same systematic set
    bool bad = false;
    for (int p = 0; p < R; ++p) bad |= *reinterpret_cast<const int32_t *>(area(p) + L.scratch + 16) != st.set_start;
    bad = __any_sync(0xFFFFFFFFu, bad);
    // (the flag is the same for all warps of the group: they compare the same words)
    if (bad && gtid == 0) set_status(P.status, ST_STATE);
    int s0 = st.set_start;

    // The next set's sub-block, b and diagonal, by cp.async (4-byte entries)
    // or plain loads (2-byte entries).
    auto load_set = [&](int s) {
        const int kk = k * k;
        for (int idx = gtid; idx < kk; idx += GT) {
            const int a = idx / k, t = idx - a * k;
            int ra = s + a;
            if (ra >= n) ra -= n;
            int ct = s + t;
            if (ct >= n) ct -= n;
            const QT *src = Q + static_cast<int64_t>(ra) * ld + ct;
            if constexpr (sizeof(QT) == 4) cp_async4(sub + idx, src);
            else sub[idx] = *src;
        }
        for (int t = gtid; t < k; t += GT) {
            int ct = s + t;
            if (ct >= n) ct -= n;
            cp_async4(sub_b + t, bvec + ct);
            cp_async4(sub_d + t, dvec + ct);
        }
    };

    // Every chain's log of the period, applied to its fields outside
    // [s, s + k); then the fields of the next set [sn, sn + k) are gathered
    // into the chains' set buffers (unless this was the last period).
    auto apply_group = [&](int s, int sn, bool last) {
        const int nch = ld / VE;
        const int total = R * nch;
        for (int it = gtid; it < total; it += GT) {
            const int c = it / nch, q = it - c * nch;
            unsigned char *b = area(c);
            const int len = *reinterpret_cast<const int32_t *>(b + L.scratch + 20);
            const int cc = P.cta_chains[cd.first + team - pos + c];
            apply_item<QT, HT>(Q, ld, reinterpret_cast<HT *>(P.fields) + static_cast<int64_t>(cc) * P.LD,
                               reinterpret_cast<const int32_t *>(b + L.log), len, q, s, sn, k, n,
                               last ? nullptr : reinterpret_cast<HT *>(b + L.insf));
        }
    };

    // ---- records ---------------------------------------------------------------
    int64_t tape_pos = 0;
    int32_t pend_flip = 0;
    double pend_m = 0.0;
    bool pend = false;
    auto flush_record = [&]() {
        if (pend) {
            if (lane == 0 && P.tape >= 1 && tape_pos < P.tape_cap) {
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
    int64_t rec_started = 0;
    auto sample_record = [&]() {
        if (P.tape == 2 && rec_started < P.tape_cap) {
            const int64_t o = static_cast<int64_t>(cid) * P.tape_cap + rec_started;
            uint32_t *tx = P.tape_x + o * P.W;
            for (int q = lane; q < P.W; q += 32) tx[q] = q < ld / 32 ? xw[q] : 0u;
            if (lane == 0) P.tape_E[o] = st.E;
        }
        rec_started += 1;
    };

    int len = 0;  // entries in this chain's log
    // Set position t -> bit.
    auto bit_of = [&](int t) {
        const int i = s0 + t;
        return i >= n ? i - n : i;
    };
    auto delta_t = [&](int t, int i) -> D {
        const bool xi = (xw[i >> 5] >> (i & 31)) & 1u;
        return A::delta(insf[t], sub_b[t], sub_d[t], xi);
    };

    // One record of Unbiased PNS on the set at s0; true at the period end.
    // Lane l evaluates positions 4l .. 4l + 3 (k <= 128), whose race words
    // are the four words of Philox block l.
    auto one_record = [&]() -> bool {
        sample_record();
        const uint64_t step = static_cast<uint64_t>(st.step);
        const RecordDraws rd = record_draws(seed, chain_id, step, n, false, true);
        const int t0 = 4 * lane;
        D dl[4];
        uint32_t lmin = 0xFFFFFFFFu;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = t0 + u;
            if (t < k) {
                dl[u] = delta_t(t, bit_of(t));
                const uint32_t kd = A::key(A::pos(dl[u]));
                lmin = kd < lmin ? kd : lmin;
            }
        }
        const D amin = A::unkey(__reduce_min_sync(0xFFFFFFFFu, lmin));
        const float af = A::tof(amin);
        const float anchor_f = af > 0.0f ? det_expf(-__fmul_rn(beta, af)) : 1.0f;
        const uint4 rw = t0 < k ? rng_block(seed, TAG_RACE, chain_id, step, static_cast<uint32_t>(lane))
                                : make_uint4(0u, 0u, 0u, 0u);
        uint32_t bkey = 0xFFFFFFFFu, bpos = 0xFFFFFFFFu, sa = 0u, sb = 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = t0 + u;
            if (t < k) {
                const float w = det_expf(-__fmul_rn(beta, A::diff(A::pos(dl[u]), amin)));
                const float ws = __fmul_rn(w, 65536.0f);
                const float wa = truncf(ws);
                sa += __float2uint_rz(wa);
                sb += __float2uint_rz(__fmul_rn(__fsub_rn(ws, wa), 65536.0f));
                const uint32_t kb = __float_as_uint(__fdiv_rn(race_exp(pick_word(rw, static_cast<uint32_t>(u))), w));
                if (kb < bkey) {  // t ascending: the first minimum is kept
                    bkey = kb;
                    bpos = static_cast<uint32_t>(t);
                }
            }
        }
        const uint32_t wkey = __reduce_min_sync(0xFFFFFFFFu, bkey);
        const uint32_t wpos = __reduce_min_sync(0xFFFFFFFFu, bkey == wkey ? bpos : 0xFFFFFFFFu);
        const uint32_t SA = __reduce_add_sync(0xFFFFFFFFu, sa);
        const uint32_t SB = __reduce_add_sync(0xFFFFFFFFu, sb);
        const uint64_t S = (static_cast<uint64_t>(SA) << 16) + static_cast<uint64_t>(SB);
        const int a = static_cast<int>(wpos);
        const int j = bit_of(a);
        const Mult mu = multiplicity_e1(S, k, anchor_f, rd.e1);
        double m = mu.md;
        const D dj = delta_t(a, j);
        __syncwarp();
        bool period_end = false;
        const bool fits = mu.mi >= 0 ? mu.mi <= st.L : m <= static_cast<double>(st.L);
        if (fits) {
            st.L -= mu.mi >= 0 ? mu.mi : static_cast<int64_t>(m);
            if (mu.sat) st.saturated += 1;
            // the set's fields from the sub-block row of j
            const bool up = ((xw[j >> 5] >> (j & 31)) & 1u) == 0u;
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
                for (int q = lane; q < nch; q += 32) apply_item<QT, HT>(Q, ld, hg, log, len, q, s0, 0, k, n, nullptr);
                __syncwarp();
                len = 0;
            }
        } else {
            m = static_cast<double>(st.L);
            st.L = P.L0;
            st.stays += 1;
            int ns = st.set_start + k;
            while (ns >= n) ns -= n;
            st.set_start = ns;
            st.period_start = static_cast<int64_t>(step) + 1;
            period_end = true;
            write_record(-1, m);
        }
        st.best_E = fmin(st.best_E, st.E);
        st.step += 1;
        return period_end;
    };

    // ---- periods, exchange rounds ------------------------------------------------
    const int64_t rounds = bad ? 0 : P.steps / P.swap_interval;
    const int64_t per_round = P.swap_interval / P.L0;
    if (rounds > 0) load_set(s0);
    cp_async_wait_all();
    gsync();
    for (int64_t rdi = 0; rdi < rounds; ++rdi) {
        for (int64_t pr = 0; pr < per_round; ++pr) {
            len = 0;
            while (!one_record()) {
            }
            // the set's fields back to global memory, where the apply step
            // (other warps of the group) reads whole chunks
            for (int t = lane; t < k; t += 32) hg[bit_of(t)] = insf[t];
            if (lane == 0) {
                *pub_E = st.E;
                *pub_b = st.beta_idx;
                *pub_len = len;
            }
            gsync();
            if (pr + 1 == per_round) {
                if (pos == 0 && lane == 0) {
                    const uint64_t ndone = static_cast<uint64_t>(st.sum_m) / static_cast<uint64_t>(P.swap_interval);
                    const uint64_t rnd = ndone - 1;
                    int slot_of[32];
                    for (int s2 = 0; s2 < R; ++s2) slot_of[*reinterpret_cast<const int32_t *>(area(s2) + L.scratch + 8)] = s2;
                    int q = 0;
                    for (int a = static_cast<int>(rnd & 1u); a + 1 < R; a += 2, ++q) {
                        const int sa_ = slot_of[a], sb_ = slot_of[a + 1];
                        unsigned char *pa = area(sa_) + L.scratch;
                        unsigned char *pb = area(sb_) + L.scratch;
                        const double Ea = *reinterpret_cast<double *>(pa);
                        const double Eb = *reinterpret_cast<double *>(pb);
                        const float db = __fsub_rn(in.betas[a], in.betas[a + 1]);
                        const float de = __double2float_rn(__dsub_rn(Ea, Eb));
                        const float xr = __fmul_rn(db, de);
                        const uint32_t w = rng_word(seed, TAG_SWAP, static_cast<uint32_t>(chd.group) + P.group_base, rnd,
                                                    static_cast<uint32_t>(q));
                        if (det_logf(u01_grid(w)) < xr) {
                            *reinterpret_cast<int32_t *>(pa + 8) = a + 1;
                            *reinterpret_cast<int32_t *>(pb + 8) = a;
                            slot_of[a] = sb_;
                            slot_of[a + 1] = sa_;
                            atomicAdd(reinterpret_cast<int32_t *>(pa + 12), 1);
                            atomicAdd(reinterpret_cast<int32_t *>(pb + 12), 1);
                        }
                    }
                }
                gsync();
                st.beta_idx = *pub_b;
                st.swaps += *swap_cnt;
                __syncwarp();
                if (lane == 0) *swap_cnt = 0;
                beta = in.betas[st.beta_idx];
            }
            const bool last = rdi + 1 == rounds && pr + 1 == per_round;
            const int s_next = st.set_start;  // the same for the whole group
            if (!last) load_set(s_next);      // the sub-block is not read until the next period
            apply_group(s0, s_next, last);
            cp_async_wait_all();
            gsync();
            s0 = s_next;
        }
    }

    // ---- write the chain back ------------------------------------------------------
    flush_record();
    __syncwarp();
    {
        // (the fields are complete in global memory after the last apply step)
        uint32_t *gx = P.xbits + static_cast<int64_t>(cid) * P.W;
        for (int w = lane; w < ld / 32; w += 32) gx[w] = xw[w];
    }
    if (lane == 0) {
        st.tape_records = tape_pos < P.tape_cap ? tape_pos : P.tape_cap;
        if (!P.tape) st.tape_records = 0;
        P.state[cid] = st;
    }
}

}  // namespace pnsk
