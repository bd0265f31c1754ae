// pns_donuts.cu -- continuous Unbiased PNS (Algorithm 7) and Metropolis on
// the Donuts target of Sec. 7, one warp per chain.
//
// The state is two fp32 coordinates; there are no local fields.  A period's
// partial neighbour set is {x + d_j, x - d_j}: lane j holds d_j ~ N(0, I)
// (Box-Muller, drawn when the period starts), evaluates its two candidates,
// and the record's anchor, weights, exponential race, quantised weight sum,
// multiplicity and budget are those of the discrete Unbiased PNS kernels
// (same counter-based streams, same fp32 decisions), so each record equals
// the oracle's.  The multiplicity-weighted sums of x, x^2, x^4 and [x > 0]
// are accumulated in fp64 by lane 0 in record order.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "pns.h"
#include "pns_launch.h"
#include "pns_sampler.cuh"

namespace pnsk {
namespace {

// (cos 2 pi u, sin 2 pi u) for u in [0, 1): quadrant q = floor(4u), angle
// t = (4u - q) pi/2 in [0, pi/2), Taylor series of sin to t^11 and of cos to
// t^12 in Horner form over t^2, then the quadrant's rotation.
__device__ __forceinline__ void sincos_2pi(float u, float &co, float &si) {
    const float u4 = __fmul_rn(u, 4.0f);
    const float qf = floorf(u4);
    const float f = __fsub_rn(u4, qf);
    const int q = static_cast<int>(qf) & 3;
    const float t = __fmul_rn(f, 0x1.921fb6p+0f);
    const float t2 = __fmul_rn(t, t);
    float ps = -0x1.ae6456p-26f;
    ps = __fadd_rn(0x1.71de3ap-19f, __fmul_rn(t2, ps));
    ps = __fadd_rn(-0x1.a01a02p-13f, __fmul_rn(t2, ps));
    ps = __fadd_rn(0x1.111112p-7f, __fmul_rn(t2, ps));
    ps = __fadd_rn(-0x1.555556p-3f, __fmul_rn(t2, ps));
    const float sn = __fadd_rn(t, __fmul_rn(t, __fmul_rn(t2, ps)));
    float pc = 0x1.1eed8ep-29f;
    pc = __fadd_rn(-0x1.27e4fcp-22f, __fmul_rn(t2, pc));
    pc = __fadd_rn(0x1.a01a02p-16f, __fmul_rn(t2, pc));
    pc = __fadd_rn(-0x1.6c16c2p-10f, __fmul_rn(t2, pc));
    pc = __fadd_rn(0x1.555556p-5f, __fmul_rn(t2, pc));
    pc = __fadd_rn(-0.5f, __fmul_rn(t2, pc));
    const float cs = __fadd_rn(1.0f, __fmul_rn(t2, pc));
    co = q == 0 ? cs : (q == 1 ? -sn : (q == 2 ? -cs : sn));
    si = q == 0 ? sn : (q == 1 ? cs : (q == 2 ? -sn : -cs));
}

// Box-Muller pair: r = sqrt(-2 ln U1) (U1 the fine uniform of w0), angle
// 2 pi U2 (U2 the grid uniform of w1).
__device__ __forceinline__ void normal_pair(uint32_t w0, uint32_t w1, float &z1, float &z2) {
    const float lg = det_logf(u01_fine(w0));
    const float r = __fsqrt_rn(__fmul_rn(-2.0f, lg));
    float co, si;
    sincos_2pi(u01_grid(w1), co, si);
    z1 = __fmul_rn(r, co);
    z2 = __fmul_rn(r, si);
}

__device__ __forceinline__ float donut_energy(float mu0, float c, float x1, float x2) {
    const float s = __fadd_rn(__fmul_rn(x1, x1), __fmul_rn(x2, x2));
    const float u = __fsub_rn(s, mu0);
    return __fmul_rn(c, __fmul_rn(u, u));
}

__global__ void __launch_bounds__(256) donuts_kernel(const pns_donuts_config cfg, int64_t chains, int64_t steps,
                                                     const float *x0, pns_donuts_stats *out) {
    const int64_t chain = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (chain >= chains) return;
    const int lane = threadIdx.x & 31;
    const uint32_t cid = static_cast<uint32_t>(chain) + static_cast<uint32_t>(cfg.chain_base);
    const uint64_t seed = cfg.seed;
    const bool unbiased = cfg.variant == PNS_UNBIASED;
    const int np = cfg.npairs;
    const int k = 2 * np;
    float x1, x2;
    if (x0) {
        x1 = x0[2 * chain];
        x2 = x0[2 * chain + 1];
    } else {
        x1 = __fsqrt_rn(cfg.mu0);
        x2 = 0.0f;
    }
    int64_t L = cfg.L0, pstart = 0, moves = 0;
    bool need_set = true;
    float dx = 0.0f, dy = 0.0f;
    double W = 0.0, sx[2] = {0.0, 0.0}, sx2[2] = {0.0, 0.0}, sx4[2] = {0.0, 0.0}, spos[2] = {0.0, 0.0};
    // Unbiased: the multiplicity's Exp(1) drawn 32 records at a time, lane l
    // drawing record b + l, each record taking its own from that lane (the
    // same values)
    float e1_bat = 0.0f;
    // The per-record sums in batches of 32 records: lane l keeps record b + l
    // (its multiplicity and state); at the batch end every lane forms its
    // record's fp64 products at once and lane 0 adds them in record order
    // (the additions, the only order-dependent part, stay sequential).
    double my_m = 0.0;
    float my_x1 = 0.0f, my_x2 = 0.0f;
    auto flush_sums = [&](int cnt) {
        const float mx[2] = {my_x1, my_x2};
        double p1[2], p2[2], p4[2];
        bool pz[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const double xd = static_cast<double>(mx[i]);
            const double x2d = __dmul_rn(xd, xd);
            p1[i] = __dmul_rn(my_m, xd);
            p2[i] = __dmul_rn(my_m, x2d);
            p4[i] = __dmul_rn(my_m, __dmul_rn(x2d, x2d));
            pz[i] = xd > 0.0;
        }
        for (int l = 0; l < cnt; ++l) {
            const double ml = __shfl_sync(0xFFFFFFFFu, my_m, l);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const double a = __shfl_sync(0xFFFFFFFFu, p1[i], l);
                const double b = __shfl_sync(0xFFFFFFFFu, p2[i], l);
                const double c = __shfl_sync(0xFFFFFFFFu, p4[i], l);
                const bool pos = __shfl_sync(0xFFFFFFFFu, pz[i] ? 1 : 0, l) != 0;
                if (lane == 0) {
                    sx[i] = __dadd_rn(sx[i], a);
                    sx2[i] = __dadd_rn(sx2[i], b);
                    sx4[i] = __dadd_rn(sx4[i], c);
                    if (pos) spos[i] = __dadd_rn(spos[i], ml);
                }
            }
            if (lane == 0) W = __dadd_rn(W, ml);
        }
    };
    for (int64_t step = 0; step < steps; ++step) {
        const float e0 = donut_energy(cfg.mu0, cfg.c, x1, x2);
        double m;
        float nx1 = x1, nx2 = x2;
        bool moved = false;
        if (!unbiased) {
            const uint4 w = rng_block(seed, TAG_STEP, cid, static_cast<uint64_t>(step), 0);
            float d1, d2;
            normal_pair(w.x, w.y, d1, d2);
            const float y1 = __fadd_rn(x1, d1), y2 = __fadd_rn(x2, d2);
            const float dlt = __fsub_rn(donut_energy(cfg.mu0, cfg.c, y1, y2), e0);
            if (det_logf(u01_grid(w.w)) < -dlt) {
                nx1 = y1;
                nx2 = y2;
                moved = true;
            }
            m = 1.0;
        } else {
            if (need_set) {
                if (lane < np) {
                    const uint4 w = rng_block(seed, TAG_SUBSET, cid, static_cast<uint64_t>(pstart),
                                              static_cast<uint32_t>(lane));
                    normal_pair(w.x, w.y, dx, dy);
                }
                need_set = false;
            }
            // candidates 2 lane (x + d) and 2 lane + 1 (x - d)
            float dl0 = 0.0f, dl1 = 0.0f;
            uint32_t lmin = 0xFFFFFFFFu;
            if (lane < np) {
                dl0 = __fsub_rn(donut_energy(cfg.mu0, cfg.c, __fadd_rn(x1, dx), __fadd_rn(x2, dy)), e0);
                dl1 = __fsub_rn(donut_energy(cfg.mu0, cfg.c, __fsub_rn(x1, dx), __fsub_rn(x2, dy)), e0);
                const uint32_t k0 = __float_as_uint(dl0 > 0.0f ? dl0 : 0.0f);
                const uint32_t k1 = __float_as_uint(dl1 > 0.0f ? dl1 : 0.0f);
                lmin = k0 < k1 ? k0 : k1;
            }
            const float amin = __uint_as_float(__reduce_min_sync(0xFFFFFFFFu, lmin));
            const float anchor_e = det_expf(-amin);
            const float anchor_f = amin > 0.0f ? anchor_e : 1.0f;
            uint32_t sa = 0u, sb = 0u, bkey = 0xFFFFFFFFu, bpos = 0xFFFFFFFFu;
            if (lane < np) {
                const uint4 rw = rng_block(seed, TAG_RACE, cid, static_cast<uint64_t>(step), static_cast<uint32_t>(lane >> 1));
                const uint32_t wa = (lane & 1) ? rw.z : rw.x;  // positions 2 lane, 2 lane + 1
                const uint32_t wb = (lane & 1) ? rw.w : rw.y;
                const float dd[2] = {dl0, dl1};
                const uint32_t ww[2] = {wa, wb};
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const float dp = dd[u] > 0.0f ? dd[u] : 0.0f;
                    const float wv = det_expf(-__fsub_rn(dp, amin));
                    const float ws = __fmul_rn(wv, 65536.0f);
                    const float wt = truncf(ws);
                    sa += __float2uint_rz(wt);
                    sb += __float2uint_rz(__fmul_rn(__fsub_rn(ws, wt), 65536.0f));
                    const uint32_t kb = __float_as_uint(__fdiv_rn(race_exp(ww[u]), wv));
                    if (kb < bkey) {  // positions ascending per lane: the first minimum is kept
                        bkey = kb;
                        bpos = static_cast<uint32_t>(2 * lane + u);
                    }
                }
            }
            const uint32_t wkey = __reduce_min_sync(0xFFFFFFFFu, bkey);
            const uint32_t wpos = __reduce_min_sync(0xFFFFFFFFu, bkey == wkey ? bpos : 0xFFFFFFFFu);
            const uint32_t SA = __reduce_add_sync(0xFFFFFFFFu, sa);
            const uint32_t SB = __reduce_add_sync(0xFFFFFFFFu, sb);
            const uint64_t S = (static_cast<uint64_t>(SA) << 16) + static_cast<uint64_t>(SB);
            if ((step & 31) == 0) {
                const uint4 sw = rng_block(seed, TAG_STEP, cid, static_cast<uint64_t>(step + lane), 0);
                e1_bat = -det_logf(u01_fine64((static_cast<uint64_t>(sw.y) << 32) | static_cast<uint64_t>(sw.x)));
            }
            const float e1 = __shfl_sync(0xFFFFFFFFu, e1_bat, static_cast<int>(step & 31));
            const Mult mu = multiplicity_e1(S, k, anchor_f, e1);
            const int wl = static_cast<int>(wpos >> 1);
            const float wdx = __shfl_sync(0xFFFFFFFFu, dx, wl);
            const float wdy = __shfl_sync(0xFFFFFFFFu, dy, wl);
            if (mult_fits(mu, L)) {
                m = mult_md(mu);
                L -= mu.mi >= 0 ? mu.mi : static_cast<int64_t>(m);
                if (wpos & 1u) {
                    nx1 = __fsub_rn(x1, wdx);
                    nx2 = __fsub_rn(x2, wdy);
                } else {
                    nx1 = __fadd_rn(x1, wdx);
                    nx2 = __fadd_rn(x2, wdy);
                }
                moved = true;
            } else {
                m = static_cast<double>(L);
                L = cfg.L0;
                pstart = step + 1;
                need_set = true;
            }
        }
        // the record weighs the state it starts from
        if (lane == static_cast<int>(step & 31)) {
            my_m = m;
            my_x1 = x1;
            my_x2 = x2;
        }
        if ((step & 31) == 31) flush_sums(32);
        moves += moved ? 1 : 0;
        x1 = nx1;
        x2 = nx2;
    }
    if (steps & 31) flush_sums(static_cast<int>(steps & 31));
    if (lane == 0) {
        pns_donuts_stats st;
        memset(&st, 0, sizeof(st));
        st.weight = W;
        for (int i = 0; i < 2; ++i) {
            st.sum_x[i] = sx[i];
            st.sum_x2[i] = sx2[i];
            st.sum_x4[i] = sx4[i];
            st.sum_pos[i] = spos[i];
        }
        st.records = steps;
        st.moves = moves;
        st.budget_left = L;
        st.period_start = pstart;
        st.x[0] = x1;
        st.x[1] = x2;
        out[chain] = st;
    }
}

pns_status dfail(pns_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return st;
}

}  // namespace
}  // namespace pnsk

using namespace pnsk;

#define DCU(call)                                                                                          \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) {                                                                           \
            st = dfail(PNS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));                             \
            goto done;                                                                                     \
        }                                                                                                  \
    } while (0)

extern "C" pns_status pns_donuts_run(const pns_donuts_config *cfg, int64_t chains, int64_t steps, const float *x0,
                                     pns_donuts_stats *stats, void *stream) {
    if (!cfg || !stats) return dfail(PNS_ERR_INVALID_ARG, "cfg and stats are required");
    if (cfg->variant != PNS_UNBIASED && cfg->variant != PNS_METROPOLIS)
        return dfail(PNS_ERR_INVALID_ARG, "pns_donuts_run takes PNS_UNBIASED or PNS_METROPOLIS");
    if (cfg->variant == PNS_UNBIASED && (cfg->npairs < 1 || cfg->npairs > 32))
        return dfail(PNS_ERR_INVALID_ARG, "npairs = %d must be in 1..32", cfg->npairs);
    if (cfg->L0 < 1) return dfail(PNS_ERR_INVALID_ARG, "L0 must be >= 1");
    if (!(cfg->c > 0.0f) || !(cfg->c < 3.0e38f) || !(cfg->mu0 > -3.0e38f && cfg->mu0 < 3.0e38f))
        return dfail(PNS_ERR_INVALID_ARG, "c must be positive and finite, mu0 finite");
    if (chains < 1 || chains > (1ll << 31) || steps < 0) return dfail(PNS_ERR_INVALID_ARG, "bad chains or steps");
    if (cfg->chain_base < 0 || cfg->reserved != 0) return dfail(PNS_ERR_INVALID_ARG, "chain_base >= 0, reserved = 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    pns_status st = PNS_OK;
    float *d_x0 = nullptr;
    pns_donuts_stats *d_out = nullptr;
    {
        const size_t xb = sizeof(float) * 2 * static_cast<size_t>(chains);
        const size_t ob = sizeof(pns_donuts_stats) * static_cast<size_t>(chains);
        if (x0) {
            DCU(cudaMalloc(&d_x0, xb));
            DCU(cudaMemcpyAsync(d_x0, x0, xb, cudaMemcpyDefault, s));
        }
        DCU(cudaMalloc(&d_out, ob));
        const int per_block = 8;
        const int64_t grid = (chains + per_block - 1) / per_block;
        donuts_kernel<<<static_cast<unsigned>(grid), 32 * per_block, 0, s>>>(*cfg, chains, steps, d_x0, d_out);
        DCU(cudaGetLastError());
        DCU(cudaMemcpyAsync(stats, d_out, ob, cudaMemcpyDefault, s));
        DCU(cudaStreamSynchronize(s));
    }
done:
    if (d_x0) cudaFree(d_x0);
    if (d_out) cudaFree(d_out);
    return st;
}
