// pns_sampler_dense.cu -- dense-Q instantiations of the sampling kernel.
#include "pns_sampler.cuh"

namespace pnsk {

template <typename QT, typename HT, int T>
static cudaError_t launch_dense_t(const KParams &P, int grid, int block, size_t smem, cudaStream_t s) {
    auto kern = pns_sample_kernel<QT, HT, T, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, block, smem, s>>>(P);
    return cudaGetLastError();
}

template <typename QT, typename HT>
static cudaError_t dense_by_T(int T, const KParams &P, int grid, int block, size_t smem, cudaStream_t s) {
    switch (T) {
    case 1: return launch_dense_t<QT, HT, 1>(P, grid, block, smem, s);
    case 2: return launch_dense_t<QT, HT, 2>(P, grid, block, smem, s);
    case 4: return launch_dense_t<QT, HT, 4>(P, grid, block, smem, s);
    case 8: return launch_dense_t<QT, HT, 8>(P, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

bool dense_supported(int qtype, int hbytes, int T) {
    if (!(T == 1 || T == 2 || T == 4 || T == 8)) return false;
    return (qtype == 0 || qtype == 1 || qtype == 2) && hbytes == 4;
}

cudaError_t launch_sampler_dense(int qtype, int T, const KParams &P, int grid, int block, size_t smem,
                                 cudaStream_t s) {
    switch (qtype) {
    case 0: return dense_by_T<int16_t, int32_t>(T, P, grid, block, smem, s);
    case 1: return dense_by_T<int32_t, int32_t>(T, P, grid, block, smem, s);
    case 2: return dense_by_T<float, float>(T, P, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pnsk
