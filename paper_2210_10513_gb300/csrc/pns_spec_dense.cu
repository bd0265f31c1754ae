// pns_spec_dense.cu -- instantiations of the speculative kernel (dense Q).
#include "pns_launch.h"
#include "pns_spec.cuh"

namespace pnsk {

template <typename QT, typename HT, int D>
static cudaError_t launch_spec_t(const KParams &P, int grid, int block, size_t smem, cudaStream_t s) {
    auto kern = pns_spec_kernel<QT, HT, D>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, block, smem, s>>>(P);
    return cudaGetLastError();
}

template <typename QT, typename HT>
static cudaError_t spec_by_D(int D, const KParams &P, int grid, int block, size_t smem, cudaStream_t s) {
    switch (D) {
    case 2: return launch_spec_t<QT, HT, 2>(P, grid, block, smem, s);
    case 4: return launch_spec_t<QT, HT, 4>(P, grid, block, smem, s);
    case 8: return launch_spec_t<QT, HT, 8>(P, grid, block, smem, s);
    case 16: return launch_spec_t<QT, HT, 16>(P, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

bool spec_supported(int qtype, int D) {
    return (qtype == 0 || qtype == 1 || qtype == 2) && (D == 2 || D == 4 || D == 8 || D == 16);
}

cudaError_t launch_spec(int qtype, int D, const KParams &P, int grid, int block, size_t smem, cudaStream_t s) {
    switch (qtype) {
    case 0: return spec_by_D<int16_t, int32_t>(D, P, grid, block, smem, s);
    case 1: return spec_by_D<int32_t, int32_t>(D, P, grid, block, smem, s);
    case 2: return spec_by_D<float, float>(D, P, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

int32_t spec_chain_bytes(int32_t ld, int32_t k, int32_t hbytes, bool list, int32_t D) {
    return spec_smem(ld, k, hbytes, list, D).total;
}

}  // namespace pnsk
