// pns_aux.cu -- instance validation, type conversion and field initialisation.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "pns_launch.h"

namespace pnsk {
namespace {

template <typename QT> struct Mirror;
template <> struct Mirror<int16_t> { using C = int32_t; using Acc = long long; };
template <> struct Mirror<int32_t> { using C = int32_t; using Acc = long long; };
template <> struct Mirror<float> { using C = float; using Acc = double; };

template <typename T> __device__ __forceinline__ bool finite_v(T v) {
    if constexpr (std::is_same<T, float>::value) return isfinite(v);
    else return true;
}

template <typename T> __device__ __forceinline__ uint32_t bits_of(T v) {
    if constexpr (std::is_same<T, float>::value) return __float_as_uint(v);
    else return static_cast<uint32_t>(static_cast<int32_t>(v));
}

__device__ __forceinline__ void atomic_max_bound(unsigned long long *bound, long long v) {
    atomicMax(bound, static_cast<unsigned long long>(v));
}
__device__ __forceinline__ void atomic_max_bound(unsigned long long *bound, double v) {
    atomicMax(bound, static_cast<unsigned long long>(__double_as_longlong(v)));  // v >= 0: order preserved
}

// One block per row: symmetry, finiteness, row bound, diag / b extraction.
template <typename QT>
__global__ void prepare_dense_kernel(const QT *q, int n, int ld, const QT *b_raw, typename Mirror<QT>::C *diag_out,
                                     typename Mirror<QT>::C *b_out, int32_t *flags, unsigned long long *bound) {
    using C = typename Mirror<QT>::C;
    using Acc = typename Mirror<QT>::Acc;
    const int i = blockIdx.x;
    if (i >= n) return;
    __shared__ Acc part[256];
    Acc acc = 0;
    int32_t f = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const QT a = q[static_cast<int64_t>(i) * ld + j];
        const QT t = q[static_cast<int64_t>(j) * ld + i];
        if (bits_of(a) != bits_of(t)) f |= FLAG_ASYM;
        if (!finite_v(a)) f |= FLAG_NONFINITE;
        acc += a < QT(0) ? -static_cast<Acc>(a) : static_cast<Acc>(a);
    }
    if (f) atomicOr(flags, f);
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        Acc tot = part[0];
        const QT bi = b_raw ? b_raw[i] : QT(0);
        if (!finite_v(bi)) atomicOr(flags, FLAG_NONFINITE);
        tot += bi < QT(0) ? -static_cast<Acc>(bi) : static_cast<Acc>(bi);
        if constexpr (std::is_same<QT, float>::value) {
            if (!isfinite(tot)) atomicOr(flags, FLAG_NONFINITE);
        }
        atomic_max_bound(bound, tot);
        diag_out[i] = static_cast<C>(q[static_cast<int64_t>(i) * ld + i]);
        b_out[i] = static_cast<C>(bi);
    }
}

__device__ __forceinline__ void acc_add(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ double ld_cg_acc(const double *p) { return __ldcg(p); }
__device__ __forceinline__ long long ld_cg_acc(const long long *p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg_q(const float *p) { return __ldcg(p); }
__device__ __forceinline__ int32_t ld_cg_q(const int32_t *p) { return __ldcg(p); }
__device__ __forceinline__ int16_t ld_cg_q(const int16_t *p) { return __ldcg(p); }
__device__ __forceinline__ void acc_add(long long *p, long long v) {  // v >= 0
    atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}

// Tiled form for pns_create: block (I, J), J >= I, compares the 32 x 32 tile
// (I, J) with the transpose of tile (J, I), both read row-wise through
// shared memory from src (row pitch sld); adds each row's |q| into rowsum
// (the tile's rows of I and, off the diagonal, of J); when src is a packed
// copy (src != q), writes both tiles into q (row pitch ld); zeroes q's
// padding columns n .. ld - 1 (last column tile).  Every element is read
// twice, coalesced.  The last block to finish (a counter in `done`) forms
// the row bounds, their finiteness and diag / b.  fp32 rows are summed over
// a tile in fp32 (an overflow reads as a non-finite bound, which is rejected
// like a bound over the limit) and across tiles in fp64.
template <typename QT>
__global__ void __launch_bounds__(256)
    prepare_tiles_kernel(const QT *src, int sld, QT *q, int ld, int n, const QT *b_raw,
                         typename Mirror<QT>::Acc *rowsum, unsigned int *done, typename Mirror<QT>::C *diag_out,
                         typename Mirror<QT>::C *b_out, int32_t *flags, unsigned long long *bound) {
    using C = typename Mirror<QT>::C;
    using Acc = typename Mirror<QT>::Acc;
    using Red = typename std::conditional<std::is_same<QT, float>::value, float, long long>::type;
    const int I = blockIdx.y, J = blockIdx.x;
    if (J < I) return;
    __shared__ QT A[32][33], B[32][33];
    __shared__ bool last;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int ca = J * 32 + tx, cb = I * 32 + tx;
    for (int r = ty; r < 32; r += 8) {
        const int ra = I * 32 + r, rb = J * 32 + r;
        A[r][tx] = ra < n && ca < n ? src[static_cast<int64_t>(ra) * sld + ca] : QT(0);
        B[r][tx] = rb < n && cb < n ? src[static_cast<int64_t>(rb) * sld + cb] : QT(0);
    }
    __syncthreads();
    int32_t f = 0;
    for (int r = ty; r < 32; r += 8) {
        const QT a = A[r][tx], t = B[tx][r], b = B[r][tx];
        if (bits_of(a) != bits_of(t)) f |= FLAG_ASYM;
        if (!finite_v(a) || !finite_v(b)) f |= FLAG_NONFINITE;
        // row sums: warp ty adds row r's |A| and |B| over its lanes
        Red sa = a < QT(0) ? -static_cast<Red>(a) : static_cast<Red>(a);
        Red sb = b < QT(0) ? -static_cast<Red>(b) : static_cast<Red>(b);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            sa += __shfl_xor_sync(0xFFFFFFFFu, sa, o);
            sb += __shfl_xor_sync(0xFFFFFFFFu, sb, o);
        }
        if (tx == 0) {
            if (I * 32 + r < n) acc_add(&rowsum[I * 32 + r], static_cast<Acc>(sa));
            if (I != J && J * 32 + r < n) acc_add(&rowsum[J * 32 + r], static_cast<Acc>(sb));
        }
    }
    if (f) atomicOr(flags, f);
    if (src != q) {  // a packed copy: both tiles into the pitched matrix
        for (int r = ty; r < 32; r += 8) {
            const int ra = I * 32 + r, rb = J * 32 + r;
            if (ra < n && ca < n) q[static_cast<int64_t>(ra) * ld + ca] = A[r][tx];
            if (I != J && rb < n && cb < n) q[static_cast<int64_t>(rb) * ld + cb] = B[r][tx];
        }
    }
    if (J == static_cast<int>(gridDim.x) - 1) {
        for (int r = ty; r < 32; r += 8) {
            const int ra = I * 32 + r;
            if (ra < n && ca >= n && ca < ld) q[static_cast<int64_t>(ra) * ld + ca] = QT(0);
        }
    }
    // the last block to finish: every tile's sums and writes are in
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int T = gridDim.x;
        last = atomicAdd(done, 1u) == T * (T + 1) / 2 - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const QT bi = b_raw ? b_raw[i] : QT(0);
        Acc tot = ld_cg_acc(&rowsum[i]);
        if (!finite_v(bi)) atomicOr(flags, FLAG_NONFINITE);
        tot += bi < QT(0) ? -static_cast<Acc>(bi) : static_cast<Acc>(bi);
        if constexpr (std::is_same<QT, float>::value) {
            if (!isfinite(tot)) atomicOr(flags, FLAG_NONFINITE);
        }
        atomic_max_bound(bound, tot);
        diag_out[i] = static_cast<C>(ld_cg_q(&q[static_cast<int64_t>(i) * ld + i]));
        b_out[i] = static_cast<C>(bi);
    }
}

// One thread per row of a CSR matrix (values already int32 or float).
template <typename VT>
__global__ void prepare_csr_kernel(const int32_t *row_ptr, const int32_t *col, const VT *val, const VT *diag_raw,
                                   const VT *b_raw, int n, int64_t nnz, VT *diag_out, VT *b_out, int32_t *flags,
                                   unsigned long long *bound) {
    using Acc = typename std::conditional<std::is_same<VT, float>::value, double, long long>::type;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t f = 0;
    const int32_t e0 = row_ptr[i], e1 = row_ptr[i + 1];
    if (e0 < 0 || e1 < e0 || e1 > nnz) {
        atomicOr(flags, FLAG_BAD_CSR);
        return;
    }
    Acc acc = 0;
    for (int32_t e = e0; e < e1; ++e) {
        const int32_t c = col[e];
        if (c < 0 || c >= n || c == i) {
            f |= FLAG_BAD_CSR;
            continue;
        }
        for (int32_t e2 = e0; e2 < e; ++e2)
            if (col[e2] == c) f |= FLAG_BAD_CSR;
        const VT v = val[e];
        if (!finite_v(v)) f |= FLAG_NONFINITE;
        acc += v < VT(0) ? -static_cast<Acc>(v) : static_cast<Acc>(v);
        // mirror entry (c, i) with the same value
        const int32_t m0 = row_ptr[c], m1 = row_ptr[c + 1];
        bool found = false;
        if (m0 >= 0 && m1 >= m0 && m1 <= nnz) {
            for (int32_t e2 = m0; e2 < m1; ++e2)
                if (col[e2] == i) {
                    found = bits_of(val[e2]) == bits_of(v);
                    break;
                }
        }
        if (!found) f |= FLAG_ASYM;
    }
    const VT d = diag_raw ? diag_raw[i] : VT(0);
    const VT bi = b_raw ? b_raw[i] : VT(0);
    if (!finite_v(d) || !finite_v(bi)) f |= FLAG_NONFINITE;
    acc += d < VT(0) ? -static_cast<Acc>(d) : static_cast<Acc>(d);
    acc += bi < VT(0) ? -static_cast<Acc>(bi) : static_cast<Acc>(bi);
    if (f) atomicOr(flags, f);
    atomic_max_bound(bound, acc);
    diag_out[i] = d;
    b_out[i] = bi;
}

template <typename S, typename D>
__global__ void convert_kernel(const S *src, D *dst, int64_t count) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = static_cast<D>(src[i]);
}

// h_i = b_i + sum over set bits j ascending of Q[j][i] (Q symmetric, so this
// is row i read down column i; coalesced across i).
template <typename QT, typename HT>
__global__ void init_fields_dense_kernel(const InstDesc *inst, const ChainDesc *chain, const uint32_t *xbits,
                                         HT *fields, int W, int LD) {
    const int64_t c = blockIdx.x;
    const InstDesc in = inst[chain[c].inst];
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= in.ld) return;
    HT *hc = fields + c * LD;
    if (i >= in.n) {
        hc[i] = HT(0);
        return;
    }
    const QT *q = reinterpret_cast<const QT *>(in.q);
    const uint32_t *x = xbits + c * W;
    if constexpr (std::is_same<HT, float>::value) {
        float acc = reinterpret_cast<const float *>(in.b)[i];
        for (int w = 0; w < in.ld / 32; ++w) {
            uint32_t bits = x[w];
            while (bits) {
                const int j = w * 32 + __ffs(bits) - 1;
                bits &= bits - 1u;
                acc = __fadd_rn(acc, q[static_cast<int64_t>(j) * in.ld + i]);
            }
        }
        hc[i] = acc;
    } else {
        long long acc = reinterpret_cast<const int32_t *>(in.b)[i];
        for (int w = 0; w < in.ld / 32; ++w) {
            uint32_t bits = x[w];
            while (bits) {
                const int j = w * 32 + __ffs(bits) - 1;
                bits &= bits - 1u;
                acc += static_cast<long long>(q[static_cast<int64_t>(j) * in.ld + i]);
            }
        }
        hc[i] = static_cast<HT>(acc);
    }
}

// CSR: h_i = b_i, then the diagonal if x_i, then row i in stored order.
template <typename VT, typename HT>
__global__ void init_fields_csr_kernel(const InstDesc *inst, const ChainDesc *chain, const uint32_t *xbits,
                                       HT *fields, int W, int LD) {
    const int64_t c = blockIdx.x;
    const InstDesc in = inst[chain[c].inst];
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= in.ld) return;
    HT *hc = fields + c * LD;
    if (i >= in.n) {
        hc[i] = HT(0);
        return;
    }
    const uint32_t *x = xbits + c * W;
    const VT *val = reinterpret_cast<const VT *>(in.q);
    const VT *dg = reinterpret_cast<const VT *>(in.diag);
    const VT *bb = reinterpret_cast<const VT *>(in.b);
    auto bit = [&](int j) { return (x[j >> 5] >> (j & 31)) & 1u; };
    if constexpr (std::is_same<VT, float>::value) {
        float acc = bb[i];
        if (bit(i)) acc = __fadd_rn(acc, dg[i]);
        for (int e = in.row_ptr[i]; e < in.row_ptr[i + 1]; ++e)
            if (bit(in.col[e])) acc = __fadd_rn(acc, val[e]);
        hc[i] = acc;
    } else {
        long long acc = bb[i];
        if (bit(i)) acc += dg[i];
        for (int e = in.row_ptr[i]; e < in.row_ptr[i + 1]; ++e)
            if (bit(in.col[e])) acc += val[e];
        hc[i] = static_cast<HT>(acc);
    }
}

// E = sum over set bits i ascending of h_i, in double (= x^T Q x + b^T x).
template <typename HT>
__global__ void init_energy_kernel(const InstDesc *inst, const ChainDesc *chain, const uint32_t *xbits,
                                   const HT *fields, ChainState *state, int64_t chains, int W, int LD) {
    const int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= chains) return;
    const InstDesc in = inst[chain[c].inst];
    const uint32_t *x = xbits + c * W;
    const HT *hc = fields + c * LD;
    double e = 0.0;
    for (int w = 0; w < in.ld / 32; ++w) {
        uint32_t bits = x[w];
        while (bits) {
            const int i = w * 32 + __ffs(bits) - 1;
            bits &= bits - 1u;
            e = __dadd_rn(e, static_cast<double>(hc[i]));
        }
    }
    state[c].E = e;
    state[c].best_E = e;
}

template <typename QT>
cudaError_t prepare_dense_t(const void *q, int n, int ld, const void *b_raw, void *diag_out, void *b_out,
                            int32_t *flags, unsigned long long *bound, cudaStream_t s) {
    using C = typename Mirror<QT>::C;
    prepare_dense_kernel<QT><<<n, 256, 0, s>>>(static_cast<const QT *>(q), n, ld, static_cast<const QT *>(b_raw),
                                               static_cast<C *>(diag_out), static_cast<C *>(b_out), flags, bound);
    return cudaGetLastError();
}

template <typename QT, typename HT>
cudaError_t init_dense_t(const InstDesc *inst, const ChainDesc *chain, const uint32_t *xbits, void *fields,
                         ChainState *state, int64_t chains, int W, int LD, int max_ld, cudaStream_t s) {
    dim3 grid(static_cast<unsigned>(chains), (max_ld + 127) / 128);
    init_fields_dense_kernel<QT, HT><<<grid, 128, 0, s>>>(inst, chain, xbits, static_cast<HT *>(fields), W, LD);
    init_energy_kernel<HT><<<static_cast<unsigned>((chains + 127) / 128), 128, 0, s>>>(
        inst, chain, xbits, static_cast<const HT *>(fields), state, chains, W, LD);
    return cudaGetLastError();
}

template <typename VT, typename HT>
cudaError_t init_csr_t(const InstDesc *inst, const ChainDesc *chain, const uint32_t *xbits, void *fields,
                       ChainState *state, int64_t chains, int W, int LD, int max_ld, cudaStream_t s) {
    dim3 grid(static_cast<unsigned>(chains), (max_ld + 127) / 128);
    init_fields_csr_kernel<VT, HT><<<grid, 128, 0, s>>>(inst, chain, xbits, static_cast<HT *>(fields), W, LD);
    init_energy_kernel<HT><<<static_cast<unsigned>((chains + 127) / 128), 128, 0, s>>>(
        inst, chain, xbits, static_cast<const HT *>(fields), state, chains, W, LD);
    return cudaGetLastError();
}

}  // namespace

namespace {
template <typename QT>
cudaError_t prepare_tiled_t(const void *src, int sld, void *q, int n, int ld, const void *b_raw, void *diag_out,
                            void *b_out, void *rowsum, int32_t *flags, unsigned long long *bound, cudaStream_t s) {
    using C = typename Mirror<QT>::C;
    using Acc = typename Mirror<QT>::Acc;
    const int T = (n + 31) / 32;
    prepare_tiles_kernel<QT><<<dim3(T, T), 256, 0, s>>>(
        static_cast<const QT *>(src), sld, static_cast<QT *>(q), ld, n, static_cast<const QT *>(b_raw),
        static_cast<Acc *>(rowsum), reinterpret_cast<unsigned int *>(static_cast<Acc *>(rowsum) + n),
        static_cast<C *>(diag_out), static_cast<C *>(b_out), flags, bound);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_prepare_dense_tiled(int qtype, const void *src, int sld, void *q, int n, int ld, const void *b_raw,
                                       void *diag_out, void *b_out, void *rowsum, int32_t *flags,
                                       unsigned long long *bound, cudaStream_t s) {
    switch (qtype) {
    case 0: return prepare_tiled_t<int16_t>(src, sld, q, n, ld, b_raw, diag_out, b_out, rowsum, flags, bound, s);
    case 1: return prepare_tiled_t<int32_t>(src, sld, q, n, ld, b_raw, diag_out, b_out, rowsum, flags, bound, s);
    case 2: return prepare_tiled_t<float>(src, sld, q, n, ld, b_raw, diag_out, b_out, rowsum, flags, bound, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_prepare_dense(int qtype, const void *q, int n, int ld, const void *b_raw, void *diag_out,
                                 void *b_out, int32_t *flags, unsigned long long *bound, cudaStream_t s) {
    switch (qtype) {
    case 0: return prepare_dense_t<int16_t>(q, n, ld, b_raw, diag_out, b_out, flags, bound, s);
    case 1: return prepare_dense_t<int32_t>(q, n, ld, b_raw, diag_out, b_out, flags, bound, s);
    case 2: return prepare_dense_t<float>(q, n, ld, b_raw, diag_out, b_out, flags, bound, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_prepare_csr(int is_float, const int32_t *row_ptr, const int32_t *col, const void *val,
                               const void *diag_raw, const void *b_raw, int n, int64_t nnz, void *diag_out,
                               void *b_out, int32_t *flags, unsigned long long *bound, cudaStream_t s) {
    const int blocks = (n + 127) / 128;
    if (is_float) {
        prepare_csr_kernel<float><<<blocks, 128, 0, s>>>(
            row_ptr, col, static_cast<const float *>(val), static_cast<const float *>(diag_raw),
            static_cast<const float *>(b_raw), n, nnz, static_cast<float *>(diag_out), static_cast<float *>(b_out),
            flags, bound);
    } else {
        prepare_csr_kernel<int32_t><<<blocks, 128, 0, s>>>(
            row_ptr, col, static_cast<const int32_t *>(val), static_cast<const int32_t *>(diag_raw),
            static_cast<const int32_t *>(b_raw), n, nnz, static_cast<int32_t *>(diag_out),
            static_cast<int32_t *>(b_out), flags, bound);
    }
    return cudaGetLastError();
}

cudaError_t launch_convert(int qtype, const void *src, void *dst, int64_t count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const unsigned blocks = static_cast<unsigned>((count + 255) / 256);
    switch (qtype) {
    case 0:
        convert_kernel<int16_t, int32_t><<<blocks, 256, 0, s>>>(static_cast<const int16_t *>(src),
                                                                static_cast<int32_t *>(dst), count);
        break;
    case 1:
        convert_kernel<int32_t, int32_t><<<blocks, 256, 0, s>>>(static_cast<const int32_t *>(src),
                                                                static_cast<int32_t *>(dst), count);
        break;
    case 2:
        convert_kernel<float, float><<<blocks, 256, 0, s>>>(static_cast<const float *>(src),
                                                            static_cast<float *>(dst), count);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_init_fields(int fmt, int qtype, int hbytes, const InstDesc *inst, const ChainDesc *chain,
                               const uint32_t *xbits, void *fields, ChainState *state, int64_t chains, int W,
                               int LD, int max_ld, cudaStream_t s) {
    if (chains <= 0) return cudaSuccess;
    if (fmt == 0) {
        if (qtype == 0) return init_dense_t<int16_t, int32_t>(inst, chain, xbits, fields, state, chains, W, LD, max_ld, s);
        if (qtype == 1) return init_dense_t<int32_t, int32_t>(inst, chain, xbits, fields, state, chains, W, LD, max_ld, s);
        return init_dense_t<float, float>(inst, chain, xbits, fields, state, chains, W, LD, max_ld, s);
    }
    if (qtype == 2) return init_csr_t<float, float>(inst, chain, xbits, fields, state, chains, W, LD, max_ld, s);
    if (hbytes == 1) return init_csr_t<int32_t, int8_t>(inst, chain, xbits, fields, state, chains, W, LD, max_ld, s);
    if (hbytes == 2) return init_csr_t<int32_t, int16_t>(inst, chain, xbits, fields, state, chains, W, LD, max_ld, s);
    return init_csr_t<int32_t, int32_t>(inst, chain, xbits, fields, state, chains, W, LD, max_ld, s);
}

}  // namespace pnsk
