// pns_sweep_dense.cu -- instantiations of the set-sweep kernel (dense Q):
// 8 warps per chain, 1, 2 or 4 sets per warp.
#include "pns_launch.h"
#include "pns_sweep.cuh"

namespace pnsk {

constexpr int SWEEP_WARPS = 8;

template <typename QT, typename HT, int SPW, int CPL>
static cudaError_t launch_sweep_t(const KParams &P, int grid, int block, size_t smem, cudaStream_t s) {
    auto kern = pns_sweep_kernel<QT, HT, SWEEP_WARPS, SPW, CPL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, block, smem, s>>>(P);
    return cudaGetLastError();
}

template <typename QT, typename HT, int CPL>
static cudaError_t sweep_by_spw(int spw, const KParams &P, int grid, int block, size_t smem, cudaStream_t s) {
    switch (spw) {
    case 1: return launch_sweep_t<QT, HT, 1, CPL>(P, grid, block, smem, s);
    case 2: return launch_sweep_t<QT, HT, 2, CPL>(P, grid, block, smem, s);
    case 4: return launch_sweep_t<QT, HT, 4, CPL>(P, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename QT, typename HT>
static cudaError_t sweep_by_cpl(int spw, int cpl, const KParams &P, int grid, int block, size_t smem,
                                cudaStream_t s) {
    switch (cpl) {
    case 1: return sweep_by_spw<QT, HT, 1>(spw, P, grid, block, smem, s);
    case 2: return sweep_by_spw<QT, HT, 2>(spw, P, grid, block, smem, s);
    case 4: return sweep_by_spw<QT, HT, 4>(spw, P, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

int sweep_sets(int n, int k) { return n / gcd32(n, k); }

bool sweep_supported(int qtype, int D, int n, int k) {
    if (!((qtype == 0 || qtype == 1 || qtype == 2) && D == SWEEP_WARPS)) return false;
    if (k < 1 || k > 128 || k > n) return false;
    return sweep_sets(n, k) <= 4 * SWEEP_WARPS;
}

cudaError_t launch_sweep(int qtype, int max_sets, int max_k, const KParams &P, int grid, int block, size_t smem,
                         cudaStream_t s) {
    const int spw = max_sets <= SWEEP_WARPS ? 1 : max_sets <= 2 * SWEEP_WARPS ? 2 : 4;
    const int cpl = max_k <= 32 ? 1 : max_k <= 64 ? 2 : 4;
    switch (qtype) {
    case 0: return sweep_by_cpl<int16_t, int32_t>(spw, cpl, P, grid, block, smem, s);
    case 1: return sweep_by_cpl<int32_t, int32_t>(spw, cpl, P, grid, block, smem, s);
    case 2: return sweep_by_cpl<float, float>(spw, cpl, P, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

// Entries of the table: up to the first d with beta d > 87 in fp32 (where the
// deterministic exponential returns 0 for every larger d as well), plus two
// zero entries; 0 (no table) past 8192 entries.
int32_t wtab_entries(float beta) {
    if (!(beta > 0.0f)) return 0;
    for (int32_t d = 0; d <= 8190; ++d) {
        const float prod = beta * static_cast<float>(d);  // (IEEE fp32 product, as on the device)
        if (!(-prod >= -87.0f)) return d + 2;
    }
    return 0;
}

__global__ void build_wtab_kernel(float4 *tab, float beta, int32_t entries) {
    for (int32_t d = blockIdx.x * blockDim.x + threadIdx.x; d < entries; d += gridDim.x * blockDim.x) {
        const float w = det_expf(-__fmul_rn(beta, __int2float_rn(d)));
        const float ws = __fmul_rn(w, 65536.0f);
        const float wa = truncf(ws);
        const uint32_t a = __float2uint_rz(wa);
        const uint32_t b = __float2uint_rz(__fmul_rn(__fsub_rn(ws, wa), 65536.0f));
        tab[d] = make_float4(w, __uint_as_float(a), __uint_as_float(b), 0.0f);
    }
}

cudaError_t launch_build_wtab(float4 *tab, float beta, int32_t entries, cudaStream_t s) {
    if (entries <= 0) return cudaSuccess;
    build_wtab_kernel<<<(entries + 255) / 256, 256, 0, s>>>(tab, beta, entries);
    return cudaGetLastError();
}

int32_t sweep_chain_bytes(int32_t ld, int32_t n, int32_t k, int32_t hbytes, int32_t D) {
    (void)D;
    return sweep_smem(ld, hbytes, k, sweep_sets(n, k)).total;
}

}  // namespace pnsk
