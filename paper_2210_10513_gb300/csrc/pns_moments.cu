// pns_moments.cu -- multiplicity-weighted moments of the jump-chain samples
// and the gradients of expectations built from them.
//
// The estimator of Theorem 3 (5) weighs each recorded state J by its
// multiplicity M.  The backward of an expectation needs the second moments
//     G0 = X^T diag(M) X,        G1 = X^T diag(M (E - c)) X
// over S samples x_s in {0,1}^n.  These are dense contractions over the
// sample axis, run on the 5th-generation tensor cores: tcgen05.mma with
// bf16 operands in shared memory and fp32 accumulators in tensor memory.
// Bits are exact in bf16; each weight is split into three bf16 parts
// (w = w1 + w2 + w3, 24 significant bits), and the three parts of M and of
// M (E - c) form six A-operand planes, two per 128-row MMA.  Multiplicities up
// to 255 are exact in the first part, and each CTA accumulates at most 16384
// samples in fp32 before its partial result is summed in fp64, so G0 is exact
// for them; the energy-weighted sums carry an fp32 accumulation error of about
// 2^-24 sqrt(16384) sum|w| / W relative to Cov.  The energy-weighted matrix is centred at c = <E> to avoid
// cancellation.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pns_launch.h"

namespace pnsk {
namespace {

constexpr int MOM_N = 64;             // n <= 64 (rows of one plane)
constexpr int STAGE_K = 64;           // samples per pipeline stage (four K = 16 slabs)
constexpr int SAMPLES_PER_CTA = 16384;
constexpr int A_SLAB_BYTES = 128 * 16 * 2;  // 128 rows x 16 bf16
constexpr int B_SLAB_BYTES = 64 * 16 * 2;   // 64 rows x 16 bf16
constexpr int STAGE_BYTES = 3 * 4 * A_SLAB_BYTES + 4 * B_SLAB_BYTES;  // 56 KiB
constexpr int NBUF = 1;               // stage buffers per CTA (two CTAs share an SM and overlap)
constexpr int MOM_SMEM = NBUF * STAGE_BYTES + 2048;
constexpr int TMEM_COLS = 256;        // three 64-column fp32 accumulators
constexpr uint32_t WAIT_LIMIT = 1u << 22;
constexpr int MOM_THREADS = 512;      // 16 warps build the operand tiles

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

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ uint16_t bf16_bits(float f) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
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

__device__ __forceinline__ int64_t sample_row(const SampleSrc &src, int64_t s) {
    const int64_t ci = s / src.recs;
    const int64_t q = s - ci * src.recs;
    return static_cast<int64_t>(src.chain_ids[ci]) * src.cap + q;
}

// ---------------------------------------------------------------------------
// fp64 sums over the samples: W = sum M, sum M E (pass 0); with the centre c:
// sum M (E - c), sum M (E - c)^2 (pass 1).  Fixed grid and block: the
// summation order, hence the result, is reproducible.
// ---------------------------------------------------------------------------
__global__ void scalar_sums_kernel(SampleSrc src, const double *centre, double *partials) {
    __shared__ double sh[2][256];
    double a = 0.0, b = 0.0;
    const double c = centre ? *centre : 0.0;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < src.samples;
         s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t row = sample_row(src, s);
        const double m = src.tape_m[row];
        const double e = src.tape_E[row];
        if (centre) {
            const double d = e - c;
            a += m * d;
            b += m * d * d;
        } else {
            a += m;
            b += m * e;
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

// out[0..1] = sums of the partials in block order; with `centre_out` set,
// also c = out[1] / out[0].
__global__ void scalar_final_kernel(const double *partials, int blocks, double *out, double *centre_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int i = 0; i < blocks; ++i) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
    }
    out[0] = a;
    out[1] = b;
    if (centre_out) *centre_out = a > 0.0 ? b / a : 0.0;
}

// ---------------------------------------------------------------------------
// The tensor-core contraction.  512 threads; each CTA takes up to 16384
// samples in stages of 64.  All 16 warps build a stage's operand tiles (the
// build, not the MMA, sets the pace); with NBUF = 1 stage buffer a CTA needs
// 58 KiB, so two CTAs share an SM and one builds while the other's MMAs run.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(MOM_THREADS, 3 - NBUF) moments_tc_kernel(SampleSrc src, const double *centre, float *partials,
                                                            int32_t *status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *const stage_base = sm;
    uint16_t *planes = reinterpret_cast<uint16_t *>(sm + NBUF * STAGE_BYTES);       // [6][64]
    uint32_t *bits_t = reinterpret_cast<uint32_t *>(sm + NBUF * STAGE_BYTES + 1024);  // [64 rows][2]: bit s = sample s
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + NBUF * STAGE_BYTES + 1536);  // [NBUF]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + NBUF * STAGE_BYTES + 1552);
    int32_t *fail = reinterpret_cast<int32_t *>(sm + NBUF * STAGE_BYTES + 1556);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int64_t s_begin = static_cast<int64_t>(blockIdx.x) * SAMPLES_PER_CTA;
    int64_t s_end = s_begin + SAMPLES_PER_CTA;
    if (s_end > src.samples) s_end = src.samples;
    const int stages = static_cast<int>((s_end - s_begin + STAGE_K - 1) / STAGE_K);
    const double c = *centre;

    if (tid == 0) {
        for (int b = 0; b < NBUF; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr_of(&mbar[b])) : "memory");
        *fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr_of(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // One sample per thread of the first 64, held in registers one stage
    // ahead so that its global loads overlap the build of the current stage.
    double nx_m = 0.0, nx_e = 0.0;
    uint32_t nx_x0 = 0u, nx_x1 = 0u;
    bool nx_valid = false;
    auto load_sample = [&](int g) {
        const int64_t s = s_begin + static_cast<int64_t>(g) * STAGE_K + tid;
        nx_valid = g < stages && s < s_end;
        if (nx_valid) {
            const int64_t row = sample_row(src, s);
            nx_m = src.tape_m[row];
            nx_e = src.tape_E[row];
            nx_x0 = src.tape_x[row * src.W];
            nx_x1 = src.W > 1 ? src.tape_x[row * src.W + 1] : 0u;
        }
    };
    if (tid < STAGE_K) load_sample(0);
    int committed = 0;  // stages whose MMAs were issued
    for (int g = 0; g < stages; ++g) {
        const int buf = g % NBUF;
        unsigned char *sb = stage_base + buf * STAGE_BYTES;
        if (g >= NBUF) {
            // the MMAs of stage g - NBUF read this buffer
            if (!mbar_wait(saddr_of(&mbar[buf]), static_cast<uint32_t>(((g - NBUF) / NBUF) & 1))) {
                if (tid == 0) *fail = 1;
            }
        }
        __syncthreads();
        if (*fail) break;
        // stage the 64 samples (loaded during the previous stage): six weight
        // planes and the bits; then start the loads of the next stage
        if (tid < STAGE_K) {
            uint16_t pw[6] = {0, 0, 0, 0, 0, 0};
            if (nx_valid) {
                split3(static_cast<float>(nx_m), pw);
                split3(static_cast<float>(nx_m * (nx_e - c)), pw + 3);
            }
            for (int p = 0; p < 6; ++p) planes[p * STAGE_K + tid] = pw[p];
            // the bits transposed: row i's word w holds bit i of samples
            // 32 w .. 32 w + 31.  Each warp transposes its two 32 x 32 bit
            // blocks (lane = sample, bit = row) by the recursive block swap:
            // at size j, a lane with bit j clear keeps its columns with bit j
            // clear and takes its partner's (lane + j) same columns moved up
            // by j; the partner keeps the others and takes the rest moved
            // down.  Afterwards lane l holds rows l and l + 32.
            uint32_t r0 = nx_valid ? nx_x0 : 0u, r1 = nx_valid ? nx_x1 : 0u;
            const int ln = tid & 31;
#pragma unroll
            for (int j = 16; j >= 1; j >>= 1) {
                const uint32_t m = j == 16 ? 0x0000FFFFu
                                   : j == 8 ? 0x00FF00FFu
                                   : j == 4 ? 0x0F0F0F0Fu
                                   : j == 2 ? 0x33333333u
                                            : 0x55555555u;
                const uint32_t p0 = __shfl_xor_sync(0xFFFFFFFFu, r0, j);
                const uint32_t p1 = __shfl_xor_sync(0xFFFFFFFFu, r1, j);
                const bool low = (ln & j) == 0;
                r0 = low ? ((r0 & m) | ((p0 & m) << j)) : ((r0 & ~m) | ((p0 & ~m) >> j));
                r1 = low ? ((r1 & m) | ((p1 & m) << j)) : ((r1 & ~m) | ((p1 & ~m) >> j));
            }
            bits_t[2 * ln + (tid >> 5)] = r0;
            bits_t[2 * (ln + 32) + (tid >> 5)] = r1;
            load_sample(g + 1);
        }
        __syncthreads();
        // A chunks: (mma m, row r, octet o) -> 8 bf16 along the sample axis
        for (int cidx = tid; cidx < 3 * 128 * 8; cidx += MOM_THREADS) {
            const int m = cidx / (128 * 8);
            const int rem = cidx - m * 128 * 8;
            const int r = rem >> 3;
            const int o = rem & 7;
            const int i = r & 63;
            const int p = 2 * m + (r >> 6);
            // samples 8 o .. 8 o + 7: their bits of row i (one byte) mask the
            // plane's eight weights (one 16-byte read)
            const uint32_t byte = (bits_t[2 * i + (o >> 2)] >> (8 * (o & 3))) & 0xFFu;
            const uint4 w8 = *reinterpret_cast<const uint4 *>(planes + p * STAGE_K + 8 * o);
            const uint32_t wv[4] = {w8.x, w8.y, w8.z, w8.w};
            uint32_t packed[4];
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) {
                const uint32_t two = byte >> (2 * e2);
                const uint32_t mask = ((two & 1u) * 0x0000FFFFu) | (((two >> 1) & 1u) * 0xFFFF0000u);
                packed[e2] = wv[e2] & mask;
            }
            const int slab = o >> 1;
            const int off = m * 4 * A_SLAB_BYTES + slab * A_SLAB_BYTES + (r >> 3) * 256 + (o & 1) * 128 + (r & 7) * 16;
            *reinterpret_cast<uint4 *>(sb + off) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        }
        // B chunks: (row j, octet o) -> bits as bf16 1.0 / 0
        for (int cidx = tid; cidx < 64 * 8; cidx += MOM_THREADS) {
            const int j = cidx >> 3;
            const int o = cidx & 7;
            const uint32_t byte = (bits_t[2 * j + (o >> 2)] >> (8 * (o & 3))) & 0xFFu;
            uint32_t packed[4];
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) {
                const uint32_t two = byte >> (2 * e2);
                const uint32_t mask = ((two & 1u) * 0x0000FFFFu) | (((two >> 1) & 1u) * 0xFFFF0000u);
                packed[e2] = 0x3F803F80u & mask;  // bf16 1.0 where the bit is set
            }
            const int slab = o >> 1;
            const int off = 3 * 4 * A_SLAB_BYTES + slab * B_SLAB_BYTES + (j >> 3) * 256 + (o & 1) * 128 + (j & 7) * 16;
            *reinterpret_cast<uint4 *>(sb + off) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        }
        // make the generic-proxy writes visible to the tensor cores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = saddr_of(sb);
            for (int slab = 0; slab < 4; ++slab) {
                const uint64_t bdesc = smem_desc(base + 3 * 4 * A_SLAB_BYTES + slab * B_SLAB_BYTES, 128, 256);
                for (int m = 0; m < 3; ++m) {
                    const uint64_t adesc = smem_desc(base + m * 4 * A_SLAB_BYTES + slab * A_SLAB_BYTES, 128, 256);
                    const uint32_t acc = (g > 0 || slab > 0) ? 1u : 0u;
                    const uint32_t dt = tmem + static_cast<uint32_t>(m * 64);
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             saddr_of(&mbar[buf]))
                         : "memory");
        }
        committed = g + 1;
    }
    // wait for the MMAs of the last (up to two) committed stages
    for (int g = committed - NBUF; g < committed; ++g) {
        if (g < 0) continue;
        if (!mbar_wait(saddr_of(&mbar[g % NBUF]), static_cast<uint32_t>((g / NBUF) & 1))) {
            if (tid == 0) *fail = 1;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool ok = *fail == 0 && committed == stages;
    if (ok) {
        // warp w reads TMEM lanes 32 (w mod 4) .. + 31 (rows of the
        // accumulators); the four warps of a lane quarter split the columns
        const int quarter = warp & 3;
        const int lane_row = 32 * quarter + (tid & 31);
        float *dst = partials + static_cast<int64_t>(blockIdx.x) * 3 * 128 * 64;
        for (int blk = warp >> 2; blk < 12; blk += MOM_THREADS / 128) {
            const int m = blk >> 2;
            const int c0 = (blk & 3) * 16;
            {
                uint32_t v[16];
                const uint32_t ta = tmem + (static_cast<uint32_t>(32 * quarter) << 16) + static_cast<uint32_t>(m * 64 + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(ta)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float *row = dst + (static_cast<int64_t>(m) * 128 + lane_row) * 64 + c0;
                for (int q = 0; q < 16; ++q) row[q] = __uint_as_float(v[q]);
            }
        }
    } else if (tid == 0) {
        atomicCAS(status, 0, ST_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// G_g[i][j] = sum over CTAs (in order) of the three planes of group g, fp64.
// Planes 0..5 = (mma, row half) (0,0) (0,1) (1,0) | (1,1) (2,0) (2,1).
__global__ void reduce_planes_kernel(const float *partials, int ctas, int n, double *G0, double *G1) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * n * n) return;
    const int g = idx / (n * n);
    const int rem = idx - g * n * n;
    const int i = rem / n, j = rem - (rem / n) * n;
    double acc = 0.0;
    for (int b = 0; b < ctas; ++b) {
        const float *pb = partials + static_cast<int64_t>(b) * 3 * 128 * 64;
        for (int q = 0; q < 3; ++q) {
            const int plane = 3 * g + q;
            const int m = plane >> 1, half = plane & 1;
            acc += static_cast<double>(pb[(static_cast<int64_t>(m) * 128 + half * 64 + i) * 64 + j]);
        }
    }
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
    const int64_t ctas = (samples + SAMPLES_PER_CTA - 1) / SAMPLES_PER_CTA;
    return static_cast<size_t>(ctas) * 3 * 128 * 64 * 4 + 2 * static_cast<size_t>(n) * n * 8 + 4096 * 8 + 64 * 8;
}

cudaError_t launch_moments(const uint32_t *tape_x, const double *tape_m, const double *tape_E,
                           const int32_t *chain_ids, int64_t chains, int64_t cap, int64_t recs, int W, int n,
                           void *scratch, int32_t *status, double *scalars, double *mean_x, double *mean_xx,
                           double *cov_ex, double *cov_exx, cudaStream_t s) {
    if (n < 1 || n > MOM_N || W < 1) return cudaErrorInvalidValue;
    SampleSrc src;
    src.tape_x = tape_x;
    src.tape_m = tape_m;
    src.tape_E = tape_E;
    src.chain_ids = chain_ids;
    src.cap = cap;
    src.recs = recs;
    src.samples = chains * recs;
    src.W = W;
    const int64_t ctas = (src.samples + SAMPLES_PER_CTA - 1) / SAMPLES_PER_CTA;
    char *p = static_cast<char *>(scratch);
    float *partials = reinterpret_cast<float *>(p);
    p += static_cast<size_t>(ctas) * 3 * 128 * 64 * 4;
    double *G0 = reinterpret_cast<double *>(p);
    double *G1 = G0 + n * n;
    double *sp = G1 + n * n;   // 4096 doubles of scalar partials
    double *s0 = sp + 4096;    // [2]
    double *s1 = s0 + 2;       // [2]
    double *centre = s1 + 2;   // [1]
    const int sb = 512;
    scalar_sums_kernel<<<sb, 256, 0, s>>>(src, nullptr, sp);
    scalar_final_kernel<<<1, 32, 0, s>>>(sp, sb, s0, centre);
    scalar_sums_kernel<<<sb, 256, 0, s>>>(src, centre, sp);
    scalar_final_kernel<<<1, 32, 0, s>>>(sp, sb, s1, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (src.samples > 0) {
        const int smem = MOM_SMEM;
        e = cudaFuncSetAttribute(moments_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        moments_tc_kernel<<<static_cast<unsigned>(ctas), MOM_THREADS, smem, s>>>(src, centre, partials, status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    reduce_planes_kernel<<<(2 * n * n + 127) / 128, 128, 0, s>>>(partials, static_cast<int>(ctas), n, G0, G1);
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
