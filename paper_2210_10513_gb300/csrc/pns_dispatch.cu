// pns_dispatch.cu -- routes a sampling launch to its instantiation.
#include "pns_launch.h"

namespace pnsk {

bool dense_supported(int qtype, int hbytes, int T);
bool csr_supported(int qtype, int hbytes, int T);
cudaError_t launch_sampler_dense(int qtype, int T, const KParams &P, int grid, int block, size_t smem,
                                 cudaStream_t s);
cudaError_t launch_sampler_csr(int qtype, int hbytes, int T, const KParams &P, int grid, int block, size_t smem,
                               cudaStream_t s);

bool sampler_supported(int fmt, int qtype, int hbytes, int T) {
    return fmt == 0 ? dense_supported(qtype, hbytes, T) : csr_supported(qtype, hbytes, T);
}

cudaError_t launch_sampler(int fmt, int qtype, int hbytes, int T, const KParams &P, int grid, int block,
                           size_t smem, cudaStream_t s) {
    if (!sampler_supported(fmt, qtype, hbytes, T)) return cudaErrorInvalidValue;
    if (fmt == 0) return launch_sampler_dense(qtype, T, P, grid, block, smem, s);
    return launch_sampler_csr(qtype, hbytes, T, P, grid, block, smem, s);
}

}  // namespace pnsk
