// pns_half.cu -- the per-flip sampling kernel with two chains per warp.
//
// For Unbiased PNS on systematic sets of k <= 16 positions (dense Q, no
// replica exchange, no producer warps) a one-warp chain leaves half of its
// lanes without a position, and every lane executes the record's scalar work
// (the Philox draws, the multiplicity, the bookkeeping).  Here each half of a
// warp (16 lanes, one position per lane) runs its own chain, so one warp
// instruction advances two chains.  The records are those of
// pns_sample_kernel, step for step: the same positions, draws, deltas,
// anchor, quantised weights, race (lexicographic minimum of key and
// position), multiplicity, budget test and row update, with the collectives
// taken over the half's 16 lanes.
#include "pns_sampler.cuh"

namespace pnsk {
namespace {

template <typename QT, typename HT>
__global__ void __launch_bounds__(512, 2) pns_half_kernel(const KParams P) {
    using A = Arith<HT>;
    using D = typename A::D;
    using CT = typename A::C;
    constexpr int HL = 16;  // lanes per chain
    constexpr int VE = 16 / static_cast<int>(sizeof(QT));

    extern __shared__ __align__(16) unsigned char smem[];
    const CtaDesc cd = P.cta[blockIdx.x];
    const int team = threadIdx.x / HL;
    if (team >= cd.count) return;  // (an idle half takes part in no collective)
    const int hl = threadIdx.x & (HL - 1);
    const unsigned hm = 0xFFFFu << (threadIdx.x & 16);  // this half's lanes
    const int cid = P.cta_chains[cd.first + team];
    const ChainDesc chd = P.chain[cid];
    const InstDesc in = P.inst[chd.inst];
    const int n = in.n;
    const int ld = in.ld;
    const int k = in.k;

    const ChainSmem L = chain_smem(ld, k, static_cast<int32_t>(sizeof(HT)), false, false, false);
    unsigned char *base = smem + chd.smem_off;
    HT *h = reinterpret_cast<HT *>(base + L.fields);
    uint32_t *xw = reinterpret_cast<uint32_t *>(base + L.xw);
    const CT *bvec = reinterpret_cast<const CT *>(in.b);
    const CT *dvec = reinterpret_cast<const CT *>(in.diag);
    const QT *Q = reinterpret_cast<const QT *>(in.q);

    // ---- load the chain ----------------------------------------------------
    {
        const HT *gh = reinterpret_cast<const HT *>(P.fields) + static_cast<int64_t>(cid) * P.LD;
        const uint32_t *gx = P.xbits + static_cast<int64_t>(cid) * P.W;
        const int hchunks = ld * static_cast<int>(sizeof(HT)) / 16;
        for (int c = hl; c < hchunks; c += HL) reinterpret_cast<uint4 *>(h)[c] = reinterpret_cast<const uint4 *>(gh)[c];
        for (int w = hl; w < ld / 32; w += HL) xw[w] = gx[w];
    }
    ChainState st = P.state[cid];
    const uint64_t seed = P.seed;
    const uint32_t chain_id = static_cast<uint32_t>(cid) + P.chain_base;
    const float beta_chain = in.betas[st.beta_idx];
    const float anneal_ls0 = P.anneal_steps > 0 ? det_logf(P.anneal_start) : 0.0f;
    __syncwarp(hm);

    // tape and sums one record late (as the one-warp kernel)
    int64_t tape_pos = 0, rec_started = 0, sum_int = 0;
    int32_t pend_flip = 0;
    double pend_m = 0.0;
    bool pend = false;
    auto flush_record = [&]() {
        if (pend) {
            if (hl == 0 && P.tape >= 1 && tape_pos < P.tape_cap) {
                const int64_t o = static_cast<int64_t>(cid) * P.tape_cap + tape_pos;
                P.tape_flip[o] = pend_flip;
                P.tape_m[o] = pend_m;
            }
            tape_pos += 1;
            pend = false;
        }
    };
    auto write_record_int = [&](int32_t flip, int64_t mi) {
        flush_record();
        pend_flip = flip;
        pend_m = P.tape >= 1 && hl == 0 ? static_cast<double>(mi) : 0.0;
        pend = true;
        sum_int += mi;
    };

    // The state-independent draws in batches across the half's lanes: lane
    // hl draws the multiplicity's Exp(1) of record b16 + hl (16 records per
    // batch), and the RACE block hl / 4 of record b4 + hl mod 4 (4 records
    // per batch); a record takes its numbers from the lanes that drew them.
    // The values are those of drawing each record's own numbers.
    float e1_mine = 0.0f;
    uint4 blk_mine = make_uint4(0u, 0u, 0u, 0u);
    const int seg = threadIdx.x & 16;  // first lane of this half
    // the position's bit index, b and diagonal, kept for the set (re-read
    // when the set moves on)
    int ci = 0, ci_set = -1;
    CT b_ci = CT(0), d_ci = CT(0);
    for (int64_t r = 0; r < P.steps; ++r) {
        // tape = 2: the state this record starts from and its energy
        if (P.tape == 2 && rec_started < P.tape_cap) {
            const int64_t o = static_cast<int64_t>(cid) * P.tape_cap + rec_started;
            uint32_t *tx = P.tape_x + o * P.W;
            for (int q = hl; q < P.W; q += HL) tx[q] = q < ld / 32 ? xw[q] : 0u;
            if (hl == 0) P.tape_E[o] = st.E;
        }
        rec_started += 1;
        const uint64_t step = static_cast<uint64_t>(st.step);
        const float beta = anneal_beta(beta_chain, anneal_ls0, P.anneal_steps, static_cast<int64_t>(step) + 1);
        const int r16 = static_cast<int>(r & 15), r4 = static_cast<int>(r & 3);
        if (r16 == 0) e1_mine = record_draws(seed, chain_id, step + static_cast<uint64_t>(hl), n, false, true).e1;
        if (r4 == 0)
            blk_mine = rng_block(seed, TAG_RACE, chain_id, step + static_cast<uint64_t>(hl & 3),
                                 static_cast<uint32_t>(hl >> 2));
        const float e1 = __shfl_sync(hm, e1_mine, seg + r16);
        // deltas of the set (position hl), the anchor
        const int t = hl;
        if (st.set_start != ci_set) {
            ci_set = st.set_start;
            ci = st.set_start + (t < k ? t : k - 1);
            ci = ci >= n ? ci - n : ci;
            b_ci = bvec[ci];
            d_ci = dvec[ci];
        }
        const D dl = A::delta(h[ci], b_ci, d_ci, (xw[ci >> 5] >> (ci & 31)) & 1u);
        const uint32_t kd = A::key(A::pos(dl));
        const uint32_t amin_k = __reduce_min_sync(hm, t < k ? kd : 0xFFFFFFFFu);
        const D amin = A::unkey(amin_k);
        const float af = A::tof(amin);
        const float anchor_e = det_expf(-__fmul_rn(beta, af));
        const float anchor_f = af > 0.0f ? anchor_e : 1.0f;
        // weight, race key and quantised weight of the position: race word t
        // mod 4 of RACE block t / 4
        const int src = seg + (hl & ~3) + r4;  // the lane that drew block t / 4 of this record
        uint4 blk;
        blk.x = __shfl_sync(hm, blk_mine.x, src);
        blk.y = __shfl_sync(hm, blk_mine.y, src);
        blk.z = __shfl_sync(hm, blk_mine.z, src);
        blk.w = __shfl_sync(hm, blk_mine.w, src);
        const float ex = race_exp(pick_word(blk, static_cast<uint32_t>(t & 3)));
        const float w = det_expf(-__fmul_rn(beta, A::diff(A::pos(dl), amin)));
        const float ws = __fmul_rn(w, 65536.0f);
        const float wa = truncf(ws);
        const uint32_t qa = t < k ? __float2uint_rz(wa) : 0u;
        const uint32_t qb = t < k ? __float2uint_rz(__fmul_rn(__fsub_rn(ws, wa), 65536.0f)) : 0u;
        const uint32_t bkey = t < k ? __float_as_uint(race_key(ex, w)) : 0xFFFFFFFFu;
        const uint32_t wkey = __reduce_min_sync(hm, bkey);
        const uint32_t wpos = __reduce_min_sync(hm, t < k && bkey == wkey ? static_cast<uint32_t>(t) : 0xFFFFFFFFu);
        const uint32_t SA = __reduce_add_sync(hm, qa);
        const uint32_t SB = __reduce_add_sync(hm, qb);
        const uint64_t S = (static_cast<uint64_t>(SA) << 16) + static_cast<uint64_t>(SB);
        int j = st.set_start + static_cast<int>(wpos);
        j = j >= n ? j - n : j;
        const Mult mu = multiplicity_e1(S, k, anchor_f, e1);
        const D dj = __shfl_sync(hm, dl, seg + static_cast<int>(wpos));  // the winner's delta
        __syncwarp(hm);  // reads of h and x are done
        if (mult_fits(mu, st.L)) {
            const int64_t mrec = mu.mi >= 0 ? mu.mi : static_cast<int64_t>(mult_md(mu));
            st.L -= mrec;
            if (mu.sat) st.saturated += 1;
            const bool up = ((xw[j >> 5] >> (j & 31)) & 1u) == 0u;
            const QT *row = Q + static_cast<int64_t>(j) * ld;
            const int chunks = ld / VE;
            for (int c = hl; c < chunks; c += HL) add_chunk<QT, HT>(h + c * VE, ld_nc_v4(row + c * VE), up);
            __syncwarp(hm);  // every lane has read x_j
            if (hl == 0) xw[j >> 5] ^= 1u << (j & 31);
            st.E = __dadd_rn(st.E, A::tod(dj));
            st.flips += 1;
            write_record_int(j, mrec);
        } else {
            const int64_t mrec = st.L;
            st.L = P.L0;
            st.stays += 1;
            int ns = st.set_start + k;
            while (ns >= n) ns -= n;
            st.set_start = ns;
            st.period_start = static_cast<int64_t>(step) + 1;
            write_record_int(-1, mrec);
        }
        const bool improved = st.E < st.best_E;
        if (improved) st.best_E = st.E;
        st.step += 1;
        __syncwarp(hm);
        if (improved && P.xbest) {
            uint32_t *xb = P.xbest + static_cast<int64_t>(cid) * P.W;
            for (int q = hl; q < P.W; q += HL) xb[q] = q < ld / 32 ? xw[q] : 0u;
        }
    }

    // ---- write the chain back ----------------------------------------------------
    flush_record();
    __syncwarp(hm);
    {
        HT *gh = reinterpret_cast<HT *>(P.fields) + static_cast<int64_t>(cid) * P.LD;
        uint32_t *gx = P.xbits + static_cast<int64_t>(cid) * P.W;
        const int hchunks = ld * static_cast<int>(sizeof(HT)) / 16;
        for (int c = hl; c < hchunks; c += HL) reinterpret_cast<uint4 *>(gh)[c] = reinterpret_cast<const uint4 *>(h)[c];
        for (int w2 = hl; w2 < ld / 32; w2 += HL) gx[w2] = xw[w2];
    }
    if (hl == 0) {
        st.sum_m = __dadd_rn(st.sum_m, static_cast<double>(sum_int));
        st.tape_records = tape_pos < P.tape_cap ? tape_pos : P.tape_cap;
        if (!P.tape) st.tape_records = 0;
        P.state[cid] = st;
    }
}

template <typename QT, typename HT>
cudaError_t launch_half_t(const KParams &P, int grid, int block, size_t smem, cudaStream_t s) {
    auto kern = pns_half_kernel<QT, HT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, block, smem, s>>>(P);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_half(int qtype, const KParams &P, int grid, int block, size_t smem, cudaStream_t s) {
    switch (qtype) {
    case 0: return launch_half_t<int16_t, int32_t>(P, grid, block, smem, s);
    case 1: return launch_half_t<int32_t, int32_t>(P, grid, block, smem, s);
    case 2: return launch_half_t<float, float>(P, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pnsk
