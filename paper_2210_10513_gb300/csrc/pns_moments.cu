// pns_moments.cu -- multiplicity-weighted moments of the jump-chain samples
// and the gradients of expectations built from them.
//
// The estimator of Theorem 3 (5) weighs each recorded state J by its
// multiplicity M.  The backward of an expectation needs the second moments
//     G0 = X^T diag(M) X,        G1 = X^T diag(M (E - c)) X
// over S samples x_s in {0,1}^n.  These are dense contractions over the
// sample axis, run on the 5th-generation tensor cores: tcgen05.mma with
// bf16 operands and fp32 accumulators in tensor memory.  Bits are exact in
// bf16; each weight is split into three bf16 parts (w = w1 + w2 + w3, 24
// significant bits), and the three parts of M and of M (E - c) form six
// weighted-bit planes of 64 rows, two per 128-row MMA.  The weighted planes
// (the A operand) are written straight into tensor memory by the threads
// that form them, so shared memory carries only the bit tile (the B operand).
// Multiplicities up to 255 are exact in the first part, and fp32
// accumulation runs over at most 16384 samples before it is added into an
// fp64 partial, so G0 is exact for them; the energy-weighted sums carry an
// fp32 accumulation error of about 2^-24 sqrt(16384) sum|w| / W relative to
// Cov.  The energy-weighted matrix is centred at c = <E> to avoid
// cancellation.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pns_launch.h"

namespace pnsk {
namespace {

constexpr int MOM_N = 64;                       // n <= 64: one 32-bit word of bits per row half
constexpr int ST_SAMPLES = 32;                  // samples per stage (two K = 16 slabs)
constexpr int SUB_STAGES = 512;                 // stages per fp32 accumulation run (16384 samples)
constexpr int NGRP = 4;                         // builder warpgroups; stage g is built by group g mod 4
constexpr int BUILD_THREADS = NGRP * 128;
constexpr int NISSUE = 3;                        // issuing warps, one per accumulator (weight part)
constexpr int MOM_THREADS = BUILD_THREADS + 32 * NISSUE;
constexpr int B_SLAB_BYTES = 64 * 16 * 2;        // 64 rows x 16 bf16
constexpr int B_STAGE_BYTES = 2 * B_SLAB_BYTES;
constexpr int WPL_OFF = NGRP * B_STAGE_BYTES;    // weight parts per builder warp: [16][3][32] bf16
constexpr int BAR_OFF = WPL_OFF + 16 * 3 * 32 * 2;
constexpr int MOM_SMEM = BAR_OFF + 128;
constexpr int TMEM_COLS = 512;
constexpr uint32_t A_COL0 = 192;                 // accumulators in columns 0..191; A stages after them
constexpr int MAX_MOM_CTAS = 160;
constexpr int PART_DOUBLES = 2 * 64 * 64;        // per-CTA fp64 partial of G0 and G1
constexpr int SUM_BLOCKS = 1216;                 // blocks of the fp64 scalar pass (8 per SM of 152)
constexpr uint32_t WAIT_LIMIT = 1u << 22;

// Shared-memory matrix descriptor (no swizzle, K-major core matrices of 8 rows
// x 16 bytes): start address, K-direction core-matrix stride (leading byte
// offset), M/N-direction stride (stride byte offset), version bits 46..48 =
// 0b001.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    return d;
}

// Instruction descriptor for kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N = 64, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t saddr_of(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bounded wait on an mbarrier phase; gives up early once another thread of
// the CTA has raised `fail`.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int32_t *fail) {
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255u) == 255u && fail && *fail) return false;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// w ~ w1 + w2 + w3, each a bf16
__device__ __forceinline__ void split3(float w, uint16_t *o) {
    const __nv_bfloat16 a = __float2bfloat16_rn(w);
    const float r1 = __fsub_rn(w, __bfloat162float(a));
    const __nv_bfloat16 b = __float2bfloat16_rn(r1);
    const float r2 = __fsub_rn(r1, __bfloat162float(b));
    const __nv_bfloat16 c = __float2bfloat16_rn(r2);
    o[0] = __bfloat16_as_ushort(a);
    o[1] = __bfloat16_as_ushort(b);
    o[2] = __bfloat16_as_ushort(c);
}

// Byte permute with the sign-replicating selector form: a selector nibble
// with bit 3 set gives 0xFF or 0x00 from the top bit of the chosen byte.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

struct SampleSrc {
    const uint32_t *tape_x;  // W words per record
    const double *tape_m;
    const double *tape_E;
    const int32_t *chain_ids;
    int64_t cap;             // records per chain in the tape
    int64_t recs;            // records used per chain
    int64_t samples;         // chains * recs
    int W;
};

// Walks the samples s, s + stride, s + 2 stride, ... of the chain-major
// sample order (sample s = record s mod recs of chain s / recs) without a
// division per step.
// Chain indices and record numbers fit 32 bits (the host checks recs).
struct SampleWalk {
    int64_t s, row_base;
    int32_t ci, q, adv_c, adv_q, row_ci;
    __device__ void init(const SampleSrc &src, int64_t s0, int64_t stride) {
        s = s0;
        const int64_t c0 = s0 / src.recs;
        ci = static_cast<int32_t>(c0);
        q = static_cast<int32_t>(s0 - c0 * src.recs);
        adv_c = static_cast<int32_t>(stride / src.recs);
        adv_q = static_cast<int32_t>(stride - static_cast<int64_t>(adv_c) * src.recs);
        row_ci = -1;
        row_base = 0;
    }
    __device__ __forceinline__ int64_t row(const SampleSrc &src) {
        if (ci != row_ci) {
            row_ci = ci;
            row_base = static_cast<int64_t>(src.chain_ids[ci]) * src.cap;
        }
        return row_base + q;
    }
    __device__ __forceinline__ void next(const SampleSrc &src, int64_t stride) {
        s += stride;
        q += adv_q;
        ci += adv_c;
        if (q >= src.recs) {
            q -= static_cast<int32_t>(src.recs);
            ++ci;
        }
    }
};

// ---------------------------------------------------------------------------
// fp64 sums over the samples: W = sum M and sum M E.  Fixed grid and block:
// the summation order, hence the result, is reproducible.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) scalar_sums_kernel(SampleSrc src, double *partials) {
    __shared__ double sh[2][256];
    double a = 0.0, b = 0.0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t s0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s0 < src.samples) {
        SampleWalk it;
        it.init(src, s0, stride);
        for (; it.s < src.samples; it.next(src, stride)) {
            const int64_t row = it.row(src);
            const double m = src.tape_m[row];
            a += m;
            b += m * src.tape_E[row];
        }
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + st];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = sh[0][0];
        partials[2 * blockIdx.x + 1] = sh[1][0];
    }
}

// out[0..1] = the sums of `count` partial pairs, in a fixed order (strided
// per thread, then a tree); with `centre_out` set, also c = out[1] / out[0].
__global__ void __launch_bounds__(256) scalar_final_kernel(const double *partials, int count, double *out,
                                                           double *centre_out) {
    __shared__ double sh[2][256];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + st];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0][0];
        out[1] = sh[1][0];
        if (centre_out) *centre_out = sh[0][0] > 0.0 ? sh[1][0] / sh[0][0] : 0.0;
    }
}

// The MMA issue loop of issuer m (one thread), kept out of line so that its
// registers are allocated apart from the builders'.
__device__ __noinline__ void issue_mmas(int m, unsigned char *sm, uint32_t tmem, int nst, int nsub, uint64_t *full,
                                        uint64_t *empty, uint64_t *accbar, uint64_t *accfree, uint64_t *drain,
                                        volatile int32_t *fail) {
    uint32_t ta[NGRP][2], idesc, td;
    uint64_t bd[NGRP][2];
#pragma unroll
    for (int u = 0; u < NGRP; ++u)
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            asm volatile("mov.b32 %0, %1;" : "=r"(ta[u][t]) : "r"(tmem + A_COL0 + static_cast<uint32_t>(48 * u + 16 * m + 8 * t)));
            asm volatile("mov.b64 %0, %1;" : "=l"(bd[u][t])
                         : "l"(smem_desc(saddr_of(sm + u * B_STAGE_BYTES + t * B_SLAB_BYTES), 128, 256)));
        }
    asm volatile("mov.b32 %0, %1;" : "=r"(idesc) : "n"(kIdesc));
    asm volatile("mov.b32 %0, %1;" : "=r"(td) : "r"(tmem + static_cast<uint32_t>(64 * m)));
    for (int sub = 0; sub < nsub && !*fail; ++sub) {
        const int g0 = sub * SUB_STAGES;
        const int g1 = min(nst, g0 + SUB_STAGES);
        if (sub > 0 && !mbar_wait(saddr_of(accfree), static_cast<uint32_t>((sub - 1) & 1), fail)) {
            *fail = 1;
            break;
        }
        bool bad = false;
        for (int g = g0; g < g1 && !bad; g += NGRP) {
#pragma unroll
            for (int u = 0; u < NGRP; ++u) {
                if (bad || g + u >= g1) continue;
                if (!mbar_wait(saddr_of(&full[u]), static_cast<uint32_t>(((g + u) >> 2) & 1), fail)) {
                    bad = true;
                    continue;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (g + u == g0)
                    asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, 0;" ::"r"(td),
                                 "r"(ta[u][0]), "l"(bd[u][0]), "r"(idesc)
                                 : "memory");
                else
                    asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, 1;" ::"r"(td),
                                 "r"(ta[u][0]), "l"(bd[u][0]), "r"(idesc)
                                 : "memory");
                asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, 1;" ::"r"(td),
                             "r"(ta[u][1]), "l"(bd[u][1]), "r"(idesc)
                             : "memory");
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        saddr_of(&empty[u]))
                    : "memory");
            }
        }
        if (bad) {
            *fail = 1;
            break;
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         saddr_of(accbar))
                     : "memory");
    }
    if (*fail) {
        // let this issuer's MMAs still in flight finish before the columns are freed
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         saddr_of(&drain[m]))
                     : "memory");
        mbar_wait(saddr_of(&drain[m]), 0u, nullptr);
    }
}

// ---------------------------------------------------------------------------
// The tensor-core contraction.  One CTA per SM, each over a contiguous range
// of samples, in stages of 32.  Warp w < 16 is a builder: warpgroup u = w / 4
// builds the stages g = u (mod 4), and its warp of lane quarter q = w mod 4
// owns TMEM lanes 32 q .. 32 q + 31, i.e. bit row i = 32 (q mod 2) + lane of
// the planes of half h = q / 2 (h = 0: the parts of M, h = 1: the parts of
// M (E - c)).  For its 32 samples a builder warp
//   * loads one sample per lane (two stages ahead) and splits its weight,
//   * transposes the 32 x 32 bit block so that lane i holds row i's bits,
//   * turns each pair of bits into a 32-bit mask and ANDs it with the bf16
//     pairs of the three weight parts, storing them into TMEM (tcgen05.st),
//   * (h = 0) stores the bits as bf16 1.0 / 0 into the shared-memory B tile.
// Warps 16, 17, 18 issue the MMAs: warp 16 + m, for accumulator m, waits for
// each stage in order and issues the two MMAs of weight part m (K = 16 slabs;
// A from TMEM, B from shared memory).  Two or more issuers keep the tensor
// pipe full with N = 64 MMAs, which one issuing thread does not.
// Every 512 stages the builders add the fp32 accumulators into the CTA's
// fp64 partial and the next run starts from zero.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(MOM_THREADS, 1)
    moments_tc_kernel(SampleSrc src, const double *centre, double *part, double *spart, int32_t *status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + BAR_OFF);  // [4]: a stage built (128 arrivals)
    uint64_t *empty = full + 4;                                   // [4]: its MMAs done (commit)
    uint64_t *accbar = full + 8;                                  // a run's MMAs done (commit)
    uint64_t *accfree = full + 9;                                 // the run's accumulators read out
    uint64_t *drain = full + 10;                                  // [3]: an issuer's MMAs done (failure path)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + BAR_OFF + 104);
    volatile int32_t *fail = reinterpret_cast<volatile int32_t *>(sm + BAR_OFF + 108);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int64_t S = src.samples;
    const int64_t beg = S * blockIdx.x / gridDim.x;
    const int64_t end = S * (blockIdx.x + 1) / gridDim.x;
    const int nst = static_cast<int>((end - beg + ST_SAMPLES - 1) / ST_SAMPLES);
    const int nsub = (nst + SUB_STAGES - 1) / SUB_STAGES;

    if (tid == 0) {
        for (int u = 0; u < NGRP; ++u) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr_of(&full[u])), "r"(128) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr_of(&empty[u])), "r"(NISSUE) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr_of(accbar)), "r"(NISSUE) : "memory");
        for (int m = 0; m < NISSUE; ++m)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr_of(&drain[m])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr_of(accfree)), "r"(BUILD_THREADS)
                     : "memory");
        *fail = 0;
    }
    if (warp == 16) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr_of(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp >= 16) {
        // Issuer m = warp - 16 owns accumulator m: for every stage in order it
        // issues the two MMAs (K = 16 slabs) of weight part m.  Its operands
        // sit in registers written once: a tcgen05.mma keeps reading its
        // register operands while it runs, so a register rewritten for the
        // next MMA would wait for the previous one to finish.
        if (lane == 0) issue_mmas(warp - 16, sm, tmem, nst, nsub, full, empty, accbar, accfree, drain, fail);
        __syncwarp();
    } else {
        const int u = warp >> 2;
        const int q = warp & 3;
        const int h = q >> 1;
        const int wi = q & 1;
        const int row = 32 * wi + lane;
        const double c = *centre;
        double *prow = part + (static_cast<int64_t>(blockIdx.x) * 2 + h) * 64 * 64 + row * 64 + 16 * u;
#pragma unroll
        for (int k = 0; k < 16; ++k) prow[k] = 0.0;
        uint16_t *wp = reinterpret_cast<uint16_t *>(sm + WPL_OFF) + warp * 96;
        const uint32_t tq = tmem + (static_cast<uint32_t>(32 * q) << 16);
        double sa = 0.0, sb = 0.0;  // q == 2: sum M (E - c); q == 3: sum M (E - c)^2

        // this lane's sample of stage g = u + 4 j is beg + 32 g + lane
        constexpr int64_t STRIDE = NGRP * ST_SAMPLES;
        SampleWalk it;
        it.init(src, beg + ST_SAMPLES * u + lane, STRIDE);
        auto fetch = [&](double &fm, double &fe, uint32_t &fx) {
            if (it.s < end) {
                const int64_t r = it.row(src);
                fm = src.tape_m[r];
                fe = src.tape_E[r];
                fx = wi < src.W ? src.tape_x[r * src.W + wi] : 0u;
            } else {
                fm = 0.0;
                fe = 0.0;
                fx = 0u;
            }
            it.next(src, STRIDE);
        };
        // two stages in flight, in two register sets used alternately, so
        // that no register copy waits for a load
        double mA, eA, mB, eB;
        uint32_t xA, xB;
        fetch(mA, eA, xA);
        fetch(mB, eB, xB);
        // one stage of this group: consumes the set (pm, pe, px), refills it
        // with the stage two ahead, builds the A parts and the B tile
        auto build_stage = [&](int j, double &pm, double &pe, uint32_t &px) -> bool {
            float wv;
            if (h == 0) {
                wv = static_cast<float>(pm);
            } else {
                const double d = pe - c;
                const double md = pm * d;
                wv = static_cast<float>(md);
                // the fp64 pipe is narrow: the two scalar sums go to the two
                // warps of this half, which sit on different schedulers
                if (q == 2)
                    sa += md;
                else
                    sb = fma(md, d, sb);
            }
            const uint32_t x = px;
            fetch(pm, pe, px);  // stage j + 2
            uint16_t p3[3];
            split3(wv, p3);
            __syncwarp();
            wp[lane] = p3[0];
            wp[32 + lane] = p3[1];
            wp[64 + lane] = p3[2];
            // transpose: lane i gets row i's bits (bit s = sample s)
            uint32_t xr = x;
#pragma unroll
            for (int jj = 16; jj >= 1; jj >>= 1) {
                const uint32_t mk = jj == 16 ? 0x0000FFFFu
                                    : jj == 8 ? 0x00FF00FFu
                                    : jj == 4 ? 0x0F0F0F0Fu
                                    : jj == 2 ? 0x33333333u
                                              : 0x55555555u;
                const uint32_t p = __shfl_xor_sync(0xFFFFFFFFu, xr, jj);
                xr = (lane & jj) == 0 ? ((xr & mk) | ((p & mk) << jj)) : ((xr & ~mk) | ((p & ~mk) >> jj));
            }
            // masks: word e covers samples 2e (low half) and 2e + 1.  Each
            // nibble of bits is spread to the top bits of four bytes
            // (multiplying by 0x10204081 places bit k at bit 8 k + 7,
            // without overlapping terms), which the sign-replicating
            // byte permute widens to 16-bit masks.
            uint32_t mw[16];
            const uint32_t xe = xr & 0x0F0F0F0Fu;
            const uint32_t xo = (xr >> 4) & 0x0F0F0F0Fu;
#pragma unroll
            for (int nb = 0; nb < 8; ++nb) {
                const uint32_t nib = prmt((nb & 1) ? xo : xe, 0u, 0x4440u | static_cast<uint32_t>(nb >> 1));
                const uint32_t sp = nib * 0x10204081u;
                mw[2 * nb] = prmt(sp, 0u, 0x9988u);
                mw[2 * nb + 1] = prmt(sp, 0u, 0xBBAAu);
            }
            __syncwarp();
            // the MMAs of this group's previous stage read the buffers
            if (j > 0) {
                const bool w_ok = mbar_wait(saddr_of(&empty[u]), static_cast<uint32_t>((j - 1) & 1), fail);
                if (!__all_sync(0xFFFFFFFFu, w_ok)) {
                    *fail = 1;
                    return false;
                }
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int k = 0; k < 3; ++k) {
#pragma unroll
                for (int t = 0; t < 2; ++t) {  // slab t: words 8 t .. 8 t + 7
                    const uint4 *wk = reinterpret_cast<const uint4 *>(wp + 32 * k + 16 * t);
                    const uint4 wa = wk[0], wb = wk[1];
                    const uint32_t *mt = mw + 8 * t;
                    const uint32_t ta = tq + A_COL0 + static_cast<uint32_t>(48 * u + 16 * k + 8 * t);
                    asm volatile(
                        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(ta),
                        "r"(wa.x & mt[0]), "r"(wa.y & mt[1]), "r"(wa.z & mt[2]), "r"(wa.w & mt[3]),
                        "r"(wb.x & mt[4]), "r"(wb.y & mt[5]), "r"(wb.z & mt[6]), "r"(wb.w & mt[7])
                        : "memory");
                }
            }
            if (h == 0) {
                unsigned char *bb = sm + u * B_STAGE_BYTES + (row >> 3) * 256 + (row & 7) * 16;
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const uint32_t one = 0x3F803F80u;  // bf16 1.0 in both halves
                    *reinterpret_cast<uint4 *>(bb + (o >> 1) * B_SLAB_BYTES + (o & 1) * 128) =
                        make_uint4(mw[4 * o] & one, mw[4 * o + 1] & one, mw[4 * o + 2] & one,
                                   mw[4 * o + 3] & one);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(saddr_of(&full[u]));
            return true;
        };
        int j = 0;  // this group's stage count
        bool ok = true;
        for (int sub = 0; sub < nsub && ok; ++sub) {
            const int g0 = sub * SUB_STAGES;
            const int g1 = min(nst, g0 + SUB_STAGES);
            for (int g = g0 + u; g < g1; g += NGRP, ++j) {
                const bool r = (j & 1) == 0 ? build_stage(j, mA, eA, xA) : build_stage(j, mB, eB, xB);
                if (!r) {
                    ok = false;
                    break;
                }
            }
            if (!ok) break;
            // the run's accumulators: this warp's lanes, columns 16 u .. 16 u + 15 of each part
            const bool w_ok = mbar_wait(saddr_of(accbar), static_cast<uint32_t>(sub & 1), fail);
            if (!__all_sync(0xFFFFFFFFu, w_ok)) {
                *fail = 1;
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int hc = 0; hc < 2; ++hc) {  // columns 16 u + 8 hc .. + 7
                uint32_t d[3][8];
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const uint32_t ta = tq + static_cast<uint32_t>(64 * m + 16 * u + 8 * hc);
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                                 : "=r"(d[m][0]), "=r"(d[m][1]), "=r"(d[m][2]), "=r"(d[m][3]), "=r"(d[m][4]),
                                   "=r"(d[m][5]), "=r"(d[m][6]), "=r"(d[m][7])
                                 : "r"(ta)
                                 : "memory");
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    prow[8 * hc + k] += (static_cast<double>(__uint_as_float(d[0][k])) +
                                         static_cast<double>(__uint_as_float(d[1][k]))) +
                                        static_cast<double>(__uint_as_float(d[2][k]));
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(saddr_of(accfree));
        }
        if (h == 1) {
            double v = q == 2 ? sa : sb;
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
            if (lane == 0) spart[2 * (blockIdx.x * NGRP + u) + (q - 2)] = v;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && *fail) atomicCAS(status, 0, ST_TIMEOUT);
    if (warp == 16) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// G_h[i][j] = sum over CTAs (in order) of the fp64 partials.
__global__ void reduce_parts_kernel(const double *part, int ctas, int n, double *G0, double *G1) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * n * n) return;
    const int g = idx / (n * n);
    const int rem = idx - g * n * n;
    const int i = rem / n, j = rem - (rem / n) * n;
    double acc = 0.0;
    for (int b = 0; b < ctas; ++b) acc += part[(static_cast<int64_t>(b) * 2 + g) * 64 * 64 + i * 64 + j];
    (g == 0 ? G0 : G1)[i * n + j] = acc;
}

// Moments from the sums: <x x^T>, <x>, Cov(E, x x^T), Cov(E, x); scalars
// {W, <E>, Var(E), samples}.
__global__ void assemble_kernel(int n, const double *G0, const double *G1, const double *s0, const double *s1,
                                const double *centre, double samples, double *scalars, double *mean_x,
                                double *mean_xx, double *cov_ex, double *cov_exx) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const double W = s0[0];
    const double c = *centre;
    const double se = s1[0] / W;   // <E - c>
    const double se2 = s1[1] / W;  // <(E - c)^2>
    if (idx == 0 && scalars) {
        scalars[0] = W;
        scalars[1] = c + se;
        scalars[2] = se2 - se * se;
        scalars[3] = samples;
    }
    if (idx < n * n) {
        const int i = idx / n, j = idx - (idx / n) * n;
        const double mxx = G0[idx] / W;
        if (mean_xx) mean_xx[idx] = mxx;
        if (cov_exx) cov_exx[idx] = G1[idx] / W - se * mxx;
        if (i == j) {
            if (mean_x) mean_x[i] = mxx;
            if (cov_ex) cov_ex[i] = G1[idx] / W - se * mxx;
        }
    }
}

// Gradients.  Mean energy <E>:  dQ = <x x^T> - beta Cov(E, x x^T),
// db = <x> - beta Cov(E, x), dbeta = -Var(E).  Boltzmann log-likelihood of
// data D (when data_xx is given): dQ = -beta (<x x^T>_D - <x x^T>),
// db = -beta (<x>_D - <x>), dbeta = -<E>_D + <E>.
__global__ void grads_kernel(int n, float beta, const double *scalars, const double *mean_x, const double *mean_xx,
                             const double *cov_ex, const double *cov_exx, const double *data_x, const double *data_xx,
                             double data_E, double *dQ, double *db, double *dbeta) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const double b = static_cast<double>(beta);
    if (idx < n * n) {
        dQ[idx] = data_xx ? -b * (data_xx[idx] - mean_xx[idx]) : mean_xx[idx] - b * cov_exx[idx];
    }
    if (idx < n) {
        db[idx] = data_xx ? -b * (data_x[idx] - mean_x[idx]) : mean_x[idx] - b * cov_ex[idx];
    }
    if (idx == 0) *dbeta = data_xx ? -data_E + scalars[1] : -scalars[2];
}

}  // namespace

// ---------------------------------------------------------------------------
// Host entry points (internal; the C ABI wrappers live in pns_host.cu).
// ---------------------------------------------------------------------------
size_t moments_scratch_bytes(int64_t samples, int n) {
    (void)samples;
    return static_cast<size_t>(MAX_MOM_CTAS) * PART_DOUBLES * 8 + 2 * static_cast<size_t>(n) * n * 8 +
           (2 * SUM_BLOCKS + 2 * NGRP * MAX_MOM_CTAS + 8) * 8;
}

cudaError_t launch_moments(const uint32_t *tape_x, const double *tape_m, const double *tape_E,
                           const int32_t *chain_ids, int64_t chains, int64_t cap, int64_t recs, int W, int n,
                           void *scratch, int32_t *status, double *scalars, double *mean_x, double *mean_xx,
                           double *cov_ex, double *cov_exx, cudaStream_t s) {
    if (n < 1 || n > MOM_N || W < 1 || recs < 0 || recs > INT32_MAX || chains > INT32_MAX) return cudaErrorInvalidValue;
    SampleSrc src;
    src.tape_x = tape_x;
    src.tape_m = tape_m;
    src.tape_E = tape_E;
    src.chain_ids = chain_ids;
    src.cap = cap;
    src.recs = recs;
    src.samples = recs > 0 ? chains * recs : 0;
    src.W = W;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // one CTA per SM, each over at least 2048 samples
    int64_t ctas = (src.samples + 2047) / 2048;
    if (ctas > sms) ctas = sms;
    if (ctas > MAX_MOM_CTAS) ctas = MAX_MOM_CTAS;
    char *p = static_cast<char *>(scratch);
    double *part = reinterpret_cast<double *>(p);
    p += static_cast<size_t>(MAX_MOM_CTAS) * PART_DOUBLES * 8;
    double *G0 = reinterpret_cast<double *>(p);
    double *G1 = G0 + n * n;
    double *sp0 = G1 + n * n;              // [SUM_BLOCKS][2]
    double *sp1 = sp0 + 2 * SUM_BLOCKS;    // [ctas][NGRP][2]
    double *s0 = sp1 + 2 * NGRP * MAX_MOM_CTAS;  // [2]
    double *s1 = s0 + 2;                   // [2]
    double *centre = s1 + 2;               // [1]
    if (src.samples > 0) {
        scalar_sums_kernel<<<SUM_BLOCKS, 256, 0, s>>>(src, sp0);
        scalar_final_kernel<<<1, 256, 0, s>>>(sp0, SUM_BLOCKS, s0, centre);
        // one CTA per SM: ask for more shared memory than two CTAs could share
        const int smem = MOM_SMEM > (116 << 10) ? MOM_SMEM : (116 << 10);
        e = cudaFuncSetAttribute(moments_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        moments_tc_kernel<<<static_cast<unsigned>(ctas), MOM_THREADS, smem, s>>>(src, centre, part, sp1, status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        scalar_final_kernel<<<1, 256, 0, s>>>(sp1, static_cast<int>(ctas) * NGRP, s1, nullptr);
    } else {
        ctas = 0;
        e = cudaMemsetAsync(s0, 0, 5 * sizeof(double), s);
        if (e != cudaSuccess) return e;
    }
    reduce_parts_kernel<<<(2 * n * n + 127) / 128, 128, 0, s>>>(part, static_cast<int>(ctas), n, G0, G1);
    assemble_kernel<<<(n * n + 127) / 128, 128, 0, s>>>(n, G0, G1, s0, s1, centre, static_cast<double>(src.samples),
                                                        scalars, mean_x, mean_xx, cov_ex, cov_exx);
    return cudaGetLastError();
}

// Mean energy of data with moments data_x, data_xx under (Q, b):
// sum_ij data_xx_ij Q_ij + sum_i data_x_i b_i in fp64, one block, a fixed
// reduction order (deterministic).
__global__ void __launch_bounds__(256) data_energy_kernel(int n, const float *q, const float *b, const double *data_x,
                                                          const double *data_xx, double *out) {
    __shared__ double part[256];
    double acc = 0.0;
    const int64_t nn = static_cast<int64_t>(n) * n;
    for (int64_t i = threadIdx.x; i < nn; i += blockDim.x) acc = fma(data_xx[i], static_cast<double>(q[i]), acc);
    if (b)
        for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fma(data_x[i], static_cast<double>(b[i]), acc);
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

cudaError_t launch_data_energy(int n, const float *q, const float *b, const double *data_x, const double *data_xx,
                               double *out, cudaStream_t s) {
    data_energy_kernel<<<1, 256, 0, s>>>(n, q, b, data_x, data_xx, out);
    return cudaGetLastError();
}

cudaError_t launch_grads(int n, float beta, const double *scalars, const double *mean_x, const double *mean_xx,
                         const double *cov_ex, const double *cov_exx, const double *data_x, const double *data_xx,
                         double data_E, double *dQ, double *db, double *dbeta, cudaStream_t s) {
    grads_kernel<<<(n * n + 127) / 128, 128, 0, s>>>(n, beta, scalars, mean_x, mean_xx, cov_ex, cov_exx, data_x,
                                                     data_xx, data_E, dQ, db, dbeta);
    return cudaGetLastError();
}

}  // namespace pnsk
