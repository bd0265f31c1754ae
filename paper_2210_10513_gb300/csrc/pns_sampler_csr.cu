// pns_sampler_csr.cu -- CSR-Q instantiations of the sampling kernel.
#include "pns_sampler.cuh"

namespace pnsk {

template <typename VT, typename HT, int T>
static cudaError_t launch_csr_t(const KParams &P, int grid, int block, size_t smem, cudaStream_t s) {
    auto kern = pns_sample_kernel<VT, HT, T, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, block, smem, s>>>(P);
    return cudaGetLastError();
}

template <typename VT, typename HT>
static cudaError_t csr_by_T(int T, const KParams &P, int grid, int block, size_t smem, cudaStream_t s) {
    switch (T) {
    case 1: return launch_csr_t<VT, HT, 1>(P, grid, block, smem, s);
    case 4: return launch_csr_t<VT, HT, 4>(P, grid, block, smem, s);
    case 8: return launch_csr_t<VT, HT, 8>(P, grid, block, smem, s);
    case 16: return launch_csr_t<VT, HT, 16>(P, grid, block, smem, s);
    case 32: return launch_csr_t<VT, HT, 32>(P, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

bool csr_supported(int qtype, int hbytes, int T) {
    if (!(T == 1 || T == 4 || T == 8 || T == 16 || T == 32)) return false;
    if (qtype == 2) return hbytes == 4;
    return qtype == 1 && (hbytes == 1 || hbytes == 2 || hbytes == 4);
}

// CSR values are stored as int32 (integer QUBOs) or float.
cudaError_t launch_sampler_csr(int qtype, int hbytes, int T, const KParams &P, int grid, int block, size_t smem,
                               cudaStream_t s) {
    if (qtype == 2) return csr_by_T<float, float>(T, P, grid, block, smem, s);
    switch (hbytes) {
    case 1: return csr_by_T<int32_t, int8_t>(T, P, grid, block, smem, s);
    case 2: return csr_by_T<int32_t, int16_t>(T, P, grid, block, smem, s);
    case 4: return csr_by_T<int32_t, int32_t>(T, P, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pnsk
