// pns_block_dense.cu -- instantiations of the period-blocked kernel (dense Q).
#include "pns_block.cuh"
#include "pns_launch.h"

namespace pnsk {

template <typename QT, typename HT>
static cudaError_t launch_block_t(const KParams &P, int grid, int block, size_t smem, cudaStream_t s) {
    auto kern = pns_block_kernel<QT, HT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, block, smem, s>>>(P);
    return cudaGetLastError();
}

bool block_supported(int qtype, int k) { return (qtype == 0 || qtype == 1 || qtype == 2) && k >= 1 && k <= 128; }

cudaError_t launch_block(int qtype, const KParams &P, int grid, int block, size_t smem, cudaStream_t s) {
    switch (qtype) {
    case 0: return launch_block_t<int16_t, int32_t>(P, grid, block, smem, s);
    case 1: return launch_block_t<int32_t, int32_t>(P, grid, block, smem, s);
    case 2: return launch_block_t<float, float>(P, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

int block_occupancy(int qtype, int threads, size_t smem) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    auto query = [&](auto kern) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem);
    };
    switch (qtype) {
    case 0: query(pns_block_kernel<int16_t, int32_t>); break;
    case 1: query(pns_block_kernel<int32_t, int32_t>); break;
    case 2: query(pns_block_kernel<float, float>); break;
    default: break;
    }
    return e == cudaSuccess ? nb : 0;
}

int32_t block_chain_bytes(int32_t ld, int32_t k, int32_t hbytes, int32_t qbytes, int32_t R, int32_t W) {
    const BlockSmem L = block_smem(ld, k, hbytes, qbytes, R, W);
    return round16((L.group_bytes + R - 1) / R);
}

}  // namespace pnsk
