// pns_launch.h -- host-side entry points of the kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pns_internal.h"

namespace pnsk {

// Validation flags written by the check kernels.
enum : int32_t { FLAG_ASYM = 1, FLAG_NONFINITE = 2, FLAG_BAD_CSR = 4 };

// Sampling launch.  fmt: 0 dense, 1 CSR.  qtype: 0 int16, 1 int32, 2 fp32.
// hbytes: field element bytes (dense integer: 4; CSR integer: 1, 2 or 4; fp32: 4).
// T: warps per chain.
cudaError_t launch_sampler(int fmt, int qtype, int hbytes, int T, const KParams &P, int grid, int block,
                           size_t smem, cudaStream_t s);
bool sampler_supported(int fmt, int qtype, int hbytes, int T);

// Dense instance set-up: validates the padded copy `q` (n rows of ld
// elements of qtype) and the raw linear term `b_raw` (qtype, may be null);
// writes diag / b as int32 (integer) or float, the row bound
// max_i (sum_j |Q_ij| + |b_i|) (integer: exact; fp32: as double bits) and
// flags.
cudaError_t launch_prepare_dense(int qtype, const void *q, int n, int ld, const void *b_raw, void *diag_out,
                                 void *b_out, int32_t *flags, unsigned long long *bound, cudaStream_t s);
// The same checks in 32 x 32 tiles (coalesced), for a matrix the library
// owns (q, row pitch ld), read from src (row pitch sld): src == q checks in
// place; otherwise src is a packed copy that is written into q.  Also
// zeroes q's padding columns n .. ld - 1.  rowsum: scratch of n 8-byte
// accumulators and one 4-byte counter after them, zeroed by the caller.
cudaError_t launch_prepare_dense_tiled(int qtype, const void *src, int sld, void *q, int n, int ld, const void *b_raw,
                                       void *diag_out, void *b_out, void *rowsum, int32_t *flags,
                                       unsigned long long *bound, cudaStream_t s);
// CSR instance set-up: values are stored as int32 or float already.
cudaError_t launch_prepare_csr(int is_float, const int32_t *row_ptr, const int32_t *col, const void *val,
                               const void *diag_raw, const void *b_raw, int n, int64_t nnz, void *diag_out,
                               void *b_out, int32_t *flags, unsigned long long *bound, cudaStream_t s);
// Convert raw values of qtype into int32 / float.
cudaError_t launch_convert(int qtype, const void *src, void *dst, int64_t count, cudaStream_t s);

// Fields h = Qx + b and energies for chains [0, chains).
cudaError_t launch_init_fields(int fmt, int qtype, int hbytes, const InstDesc *inst, const ChainDesc *chain,
                               const uint32_t *xbits, void *fields, ChainState *state, int64_t chains, int W,
                               int LD, int max_ld, cudaStream_t s);

// Speculative kernel for Unbiased PNS / Metropolis on dense Q: D warps per
// chain, warp w evaluates record step + w assuming the earlier ones stay.
bool spec_supported(int qtype, int D);
cudaError_t launch_spec(int qtype, int D, const KParams &P, int grid, int block, size_t smem, cudaStream_t s);
int32_t spec_chain_bytes(int32_t ld, int32_t k, int32_t hbytes, bool list, int32_t D);

// Set-sweep kernel for Unbiased PNS with systematic sets on dense Q: 8 warps
// per chain evaluate all n / gcd(n, k) sets of the current state (at most
// 32), then decide up to 256 records at once.
int sweep_sets(int n, int k);
bool sweep_supported(int qtype, int D, int n, int k);
cudaError_t launch_sweep(int qtype, int max_sets, int max_k, const KParams &P, int grid, int block, size_t smem,
                         cudaStream_t s);
int32_t sweep_chain_bytes(int32_t ld, int32_t n, int32_t k, int32_t hbytes, int32_t D);
// Weight table of an integer QUBO at inverse temperature beta: entry d holds
// w = e^{-beta d} as the samplers compute it and w's two 16-bit quantised
// parts; entries at and past `entries` are all zero.
int32_t wtab_entries(float beta);
cudaError_t launch_build_wtab(float4 *tab, float beta, int32_t entries, cudaStream_t s);

// Period-blocked kernel for Unbiased PNS with systematic sets and replica
// exchange on dense Q (k <= 128): one warp per chain, the group's set
// sub-block in shared memory, logged rows applied at period ends.
bool block_supported(int qtype, int k);
cudaError_t launch_block(int qtype, const KParams &P, int grid, int block, size_t smem, cudaStream_t s);
// pns_half.cu: Unbiased PNS, systematic sets of k <= 16, dense Q (hbytes 4), no
// exchange, no producer warps: two chains per warp, 16 threads per chain.
cudaError_t launch_half(int qtype, const KParams &P, int grid, int block, size_t smem, cudaStream_t s);
int32_t block_chain_bytes(int32_t ld, int32_t k, int32_t hbytes, int32_t qbytes, int32_t R, int32_t W);
// CTAs of the blocked kernel resident per SM at this shape (0 on error).
int block_occupancy(int qtype, int threads, size_t smem);

// Multiplicity-weighted moments of tape = 2 samples (n <= 64) on tcgen05
// tensor cores, and gradients assembled from them.
size_t moments_scratch_bytes(int64_t samples, int n);
cudaError_t launch_moments(const uint32_t *tape_x, const double *tape_m, const double *tape_E,
                           const int32_t *chain_ids, int64_t chains, int64_t cap, int64_t recs, int W, int n,
                           void *scratch, int32_t *status, double *scalars, double *mean_x, double *mean_xx,
                           double *cov_ex, double *cov_exx, cudaStream_t s);
cudaError_t launch_grads(int n, float beta, const double *scalars, const double *mean_x, const double *mean_xx,
                         const double *cov_ex, const double *cov_exx, const double *data_x, const double *data_xx,
                         double data_E, double *dQ, double *db, double *dbeta, cudaStream_t s);

// Mean energy of data moments under (Q, b), fp64, deterministic.
cudaError_t launch_data_energy(int n, const float *q, const float *b, const double *data_x, const double *data_xx,
                               double *out, cudaStream_t s);

// Sets the message pns_last_error() returns on this thread.
void set_last_error(const char *msg);

}  // namespace pnsk
