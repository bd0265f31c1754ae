// pns_static.cu -- pns_sample_static: the sampler for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a framework's
// caching allocator owns the device memory budget, real-time or embedded
// services that allocate only at start-up, and code inside library callbacks
// where an allocation (and its implicit synchronisation) is forbidden.  For
// them this entry point runs one dense instance end to end -- set-up, the
// sampling kernel, read-back -- with every piece of working memory (chain
// states, fields, descriptors, validation words) carved from one file-scope
// __device__ array of fixed size.  The caller passes the inputs and receives
// the outputs; nothing else is allocated.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call rewrites every word it reads.  Calls that overlap on
// the GPU (different streams or threads at once) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "pns.h"
#include "pns_launch.h"

using namespace pnsk;

namespace {

constexpr size_t kScratchBytes = PNS_STATIC_SCRATCH_BYTES;
static_assert(kScratchBytes == (16u << 20), "scratch size is part of the ABI");

__device__ __align__(256) unsigned char g_pns_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};

pns_status sfail(pns_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);  // read back through pns_last_error()
    return st;
}

#define SCU(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return sfail(PNS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

size_t up256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

// The device address of the scratch array on the current device, resolved
// once per device with that device current (and again after a call on that
// device failed, so that an address from a torn-down context is not reused).
pns_status scratch_address(int *dev_out, void **out) {
    int dev = -1;
    SCU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return sfail(PNS_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        SCU(cudaGetSymbolAddress(&p, g_pns_static_scratch));
        g_scratch_addr[dev] = p;
    }
    *dev_out = dev;
    *out = g_scratch_addr[dev];
    return PNS_OK;
}

// Forgets the device's cached address unless the call completed.
struct ForgetOnFailure {
    int dev = -1;
    bool done = false;
    ~ForgetOnFailure() {
        if (done || dev < 0) return;
        std::lock_guard<std::mutex> lock(g_mutex);
        g_scratch_addr[dev] = nullptr;
    }
};

// Fills the chain / CTA descriptors and the initial chain states for one
// instance: chains_per_cta consecutive chains per CTA, slot = c mod R.
__global__ void static_setup_kernel(InstDesc inst_val, InstDesc *inst, ChainDesc *chain, CtaDesc *cta,
                                    int32_t *cta_chains, ChainState *state, uint32_t *x, const uint32_t *x0,
                                    int64_t chains, int R, int per_cta, int chain_bytes, int W, int64_t L0,
                                    int32_t *status) {
    const int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c == 0) {
        *inst = inst_val;
        *status = 0;
    }
    if (c >= chains) return;
    ChainDesc d;
    d.inst = 0;
    d.slot = static_cast<int32_t>(c % R);
    d.group = static_cast<int32_t>(c / R);
    d.smem_off = static_cast<int32_t>(c % per_cta) * chain_bytes;
    chain[c] = d;
    cta_chains[c] = static_cast<int32_t>(c);
    if (c % per_cta == 0) {
        CtaDesc cd;
        cd.first = static_cast<int32_t>(c);
        const int64_t left = chains - c;
        cd.count = static_cast<int32_t>(left < per_cta ? left : per_cta);
        cd.groups = 0;
        cd.pad = 0;
        cta[c / per_cta] = cd;
    }
    ChainState s;
    memset(&s, 0, sizeof(s));
    s.L = L0;
    s.beta_idx = d.slot;
    state[c] = s;
    for (int w = 0; w < W; ++w) x[c * W + w] = x0 ? x0[c * W + w] : 0u;
}

__global__ void static_stats_kernel(const ChainState *state, pns_stats *out, int64_t chains) {
    const int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= chains) return;
    const ChainState z = state[c];
    pns_stats o;
    o.steps = z.step;
    o.flips = z.flips;
    o.stays = z.stays;
    o.saturated = z.saturated;
    o.swaps_accepted = z.swaps;
    o.budget_left = z.L;
    o.tape_records = z.tape_records;
    o.set_start = z.set_start;
    o.beta_idx = z.beta_idx;
    o.energy = z.E;
    o.sum_m = z.sum_m;
    o.best_energy = z.best_E;
    out[c] = o;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

pns_status pns_sample_static(const pns_problem *prob, const pns_config *cfg, int64_t steps, uint32_t *states,
                             double *multiplicities, int32_t *flips, pns_stats *stats, void *stream) {
    if (!prob || !cfg) return sfail(PNS_ERR_INVALID_ARG, "prob and cfg are required");
    // the configuration fields pns_create checks, with its messages
    const int wpc = cfg->warps_per_chain;
    if (!(wpc == 0 || wpc == 1 || wpc == 2 || wpc == 4 || wpc == 8 || wpc == 16 || wpc == 32))
        return sfail(PNS_ERR_INVALID_ARG, "warps_per_chain must be 0, 1, 2, 4, 8, 16 or 32");
    if (cfg->tape < 0 || cfg->tape > 2) return sfail(PNS_ERR_INVALID_ARG, "tape must be 0, 1 or 2");
    if (cfg->graph != 0 && cfg->graph != 1) return sfail(PNS_ERR_INVALID_ARG, "graph must be 0 or 1");
    if (cfg->autotune != 0 && cfg->autotune != 1) return sfail(PNS_ERR_INVALID_ARG, "autotune must be 0 or 1");
    if (cfg->track_best != 0 && cfg->track_best != 1) return sfail(PNS_ERR_INVALID_ARG, "track_best must be 0 or 1");
    if (cfg->chains_per_cta < 0 || cfg->reserved != 0 || cfg->chain_base < 0 || cfg->group_base < 0)
        return sfail(PNS_ERR_INVALID_ARG, "chains_per_cta, chain_base, group_base must be >= 0 and reserved 0");
    if (prob->k < 0 || prob->reserved != 0) return sfail(PNS_ERR_INVALID_ARG, "problem: k < 0 or reserved != 0");
    if (cfg->reserved2 != 0 || cfg->anneal_steps < 0)
        return sfail(PNS_ERR_INVALID_ARG, "anneal_steps must be >= 0 and reserved2 0");
    if (cfg->anneal_steps > 0 && (!(cfg->anneal_start > 0.0f) || !(cfg->anneal_start <= 1.0f)))
        return sfail(PNS_ERR_INVALID_ARG, "anneal_start must be in (0, 1]");
    // what this entry point does not do
    if (cfg->track_best) return sfail(PNS_ERR_UNSUPPORTED, "pns_sample_static keeps no best states (track_best)");
    if (cfg->tape == 2) return sfail(PNS_ERR_UNSUPPORTED, "pns_sample_static writes no sample tape (tape = 2)");
    if ((multiplicities != nullptr) != (flips != nullptr))
        return sfail(PNS_ERR_INVALID_ARG, "pass both tape outputs (multiplicities and flips) or neither");
    if (cfg->tape == 1 && !multiplicities)
        return sfail(PNS_ERR_INVALID_ARG, "tape = 1 needs the multiplicities and flips outputs");
    {
        // it synchronises `stream`, which a stream capture does not allow
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        SCU(cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs));
        if (cs != cudaStreamCaptureStatusNone)
            return sfail(PNS_ERR_UNSUPPORTED, "pns_sample_static synchronises its stream: not under stream capture");
    }
    const int n = prob->n;
    if (prob->fmt != PNS_DENSE) return sfail(PNS_ERR_UNSUPPORTED, "pns_sample_static takes a dense instance");
    if (n < 32 || n % 32 != 0) return sfail(PNS_ERR_INVALID_ARG, "n = %d must be a positive multiple of 32", n);
    if (prob->qtype < PNS_Q_I16 || prob->qtype > PNS_Q_F32) return sfail(PNS_ERR_INVALID_ARG, "unknown qtype");
    if (!prob->q || !is_device_ptr(prob->q)) return sfail(PNS_ERR_INVALID_ARG, "q must be device memory");
    if (reinterpret_cast<uintptr_t>(prob->q) % 16 != 0) return sfail(PNS_ERR_INVALID_ARG, "q must be 16-byte aligned");
    if (prob->b && !is_device_ptr(prob->b)) return sfail(PNS_ERR_INVALID_ARG, "b must be device memory");
    if (!prob->betas || !is_device_ptr(prob->betas)) return sfail(PNS_ERR_INVALID_ARG, "betas must be device memory");
    if (cfg->x0 && !is_device_ptr(cfg->x0)) return sfail(PNS_ERR_INVALID_ARG, "x0 must be device memory");
    if ((multiplicities && !is_device_ptr(multiplicities)) || (flips && !is_device_ptr(flips)))
        return sfail(PNS_ERR_INVALID_ARG, "tape outputs must be device memory");
    if (cfg->variant < PNS_BASIC || cfg->variant > PNS_METROPOLIS) return sfail(PNS_ERR_INVALID_ARG, "bad variant");
    if (cfg->swap_interval != 0) return sfail(PNS_ERR_UNSUPPORTED, "pns_sample_static has no replica exchange");
    if (cfg->L0 < 1 || cfg->chains_per_replica < 1 || prob->n_replicas < 1 || steps < 0)
        return sfail(PNS_ERR_INVALID_ARG, "L0, chains_per_replica, n_replicas must be >= 1 and steps >= 0");
    if (cfg->subset != PNS_SUBSET_SYSTEMATIC && cfg->subset != PNS_SUBSET_RANDOM)
        return sfail(PNS_ERR_INVALID_ARG, "bad subset mode");
    int k = cfg->variant == PNS_RF ? n : (cfg->variant == PNS_METROPOLIS ? 1 : (prob->k > 0 ? prob->k : cfg->k));
    if (k < 1 || k > n) return sfail(PNS_ERR_INVALID_ARG, "k = %d must be in [1, n]", k);
    const int T = cfg->warps_per_chain > 0 ? cfg->warps_per_chain : 1;
    const int qt = prob->qtype;
    if (!sampler_supported(PNS_DENSE, qt, 4, T)) return sfail(PNS_ERR_UNSUPPORTED, "warps_per_chain %d", T);
    const int R = prob->n_replicas;
    const int64_t chains = static_cast<int64_t>(R) * cfg->chains_per_replica;
    const int W = n / 32;
    const bool list = needs_list(cfg->variant, cfg->subset);
    const int chain_bytes = chain_smem(n, k, 4, list, false, false).total;
    int per_cta = cfg->chains_per_cta > 0 ? cfg->chains_per_cta : 1;
    const int max_teams = T == 32 ? 1 : (T > 1 ? std::min(512 / (32 * T), 7) : 16);
    if (per_cta > max_teams) per_cta = max_teams;
    while (per_cta > 1 && static_cast<size_t>(per_cta) * chain_bytes > 200 * 1024) --per_cta;
    if (chain_bytes > 227 * 1024) return sfail(PNS_ERR_UNSUPPORTED, "n too large for shared memory");
    const int64_t ctas = (chains + per_cta - 1) / per_cta;

    // carve the scratch array
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = up256(off + bytes);
        return o;
    };
    const size_t o_status = take(64);
    const size_t o_flags = take(64);
    const size_t o_inst = take(sizeof(InstDesc));
    const size_t o_diag = take(static_cast<size_t>(n) * 4);
    const size_t o_b = take(static_cast<size_t>(n) * 4);
    const size_t o_cta = take(sizeof(CtaDesc) * ctas);
    const size_t o_ctach = take(sizeof(int32_t) * chains);
    const size_t o_chain = take(sizeof(ChainDesc) * chains);
    const size_t o_state = take(sizeof(ChainState) * chains);
    const size_t o_x = take(sizeof(uint32_t) * W * chains);
    const size_t o_fields = take(static_cast<size_t>(4) * n * chains);
    const size_t o_stats = take(sizeof(pns_stats) * chains);
    if (off > kScratchBytes)
        return sfail(PNS_ERR_RANGE, "needs %zu bytes of scratch, over the fixed %zu (fewer chains or smaller n)", off,
                     kScratchBytes);

    void *base_v = nullptr;
    ForgetOnFailure forget;
    pns_status st = scratch_address(&forget.dev, &base_v);
    if (st != PNS_OK) return st;
    unsigned char *base = static_cast<unsigned char *>(base_v);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t *d_status = reinterpret_cast<int32_t *>(base + o_status);
    int32_t *d_flags = reinterpret_cast<int32_t *>(base + o_flags);
    unsigned long long *d_bound = reinterpret_cast<unsigned long long *>(base + o_flags + 8);

    // validate and extract diag / b (the scratch keeps old contents: clear first)
    SCU(cudaMemsetAsync(base + o_flags, 0, 64, s));
    SCU(launch_prepare_dense(qt, prob->q, n, n, prob->b, base + o_diag, base + o_b, d_flags, d_bound, s));
    struct {
        int32_t flags;
        int32_t pad;
        unsigned long long bound;
    } chk;
    SCU(cudaMemcpyAsync(&chk, base + o_flags, sizeof(chk), cudaMemcpyDeviceToHost, s));
    SCU(cudaStreamSynchronize(s));
    if (chk.flags & FLAG_NONFINITE) return sfail(PNS_ERR_RANGE, "non-finite entry");
    if (chk.flags & FLAG_ASYM) return sfail(PNS_ERR_NOT_SYMMETRIC, "Q is not symmetric");
    if (qt == PNS_Q_F32) {
        double v;
        memcpy(&v, &chk.bound, sizeof(double));
        if (!(v < 1e30)) return sfail(PNS_ERR_RANGE, "field bound %g too large for fp32 fields", v);
    } else if (static_cast<long long>(chk.bound) > 715827882LL) {
        return sfail(PNS_ERR_RANGE, "3 * field bound reaches 2^31");
    }
    // the temperatures, as pns_create checks them (copied through a small host buffer)
    for (int r0 = 0; r0 < R; r0 += 64) {
        float bh[64];
        const int m = std::min(64, R - r0);
        SCU(cudaMemcpyAsync(bh, prob->betas + r0, sizeof(float) * m, cudaMemcpyDeviceToHost, s));
        SCU(cudaStreamSynchronize(s));
        for (int i = 0; i < m; ++i)
            if (!(bh[i] >= 0.0f) || !(bh[i] < 3.0e38f)) return sfail(PNS_ERR_INVALID_ARG, "betas must be finite and >= 0");
    }

    InstDesc in;
    in.q = prob->q;
    in.row_ptr = nullptr;
    in.col = nullptr;
    in.diag = base + o_diag;
    in.b = base + o_b;
    in.betas = prob->betas;
    in.n = n;
    in.ld = n;
    in.k = k;
    in.R = R;
    InstDesc *d_inst = reinterpret_cast<InstDesc *>(base + o_inst);
    ChainDesc *d_chain = reinterpret_cast<ChainDesc *>(base + o_chain);
    CtaDesc *d_cta = reinterpret_cast<CtaDesc *>(base + o_cta);
    int32_t *d_ctach = reinterpret_cast<int32_t *>(base + o_ctach);
    ChainState *d_state = reinterpret_cast<ChainState *>(base + o_state);
    uint32_t *d_x = reinterpret_cast<uint32_t *>(base + o_x);
    void *d_fields = base + o_fields;
    static_setup_kernel<<<static_cast<unsigned>((chains + 127) / 128), 128, 0, s>>>(
        in, d_inst, d_chain, d_cta, d_ctach, d_state, d_x, cfg->x0, chains, R, per_cta, chain_bytes, W, cfg->L0,
        d_status);
    SCU(cudaGetLastError());
    SCU(launch_init_fields(PNS_DENSE, qt, 4, d_inst, d_chain, d_x, d_fields, d_state, chains, W, n, n, s));

    KParams P;
    memset(&P, 0, sizeof(P));
    P.inst = d_inst;
    P.chain = d_chain;
    P.cta = d_cta;
    P.cta_chains = d_ctach;
    P.state = d_state;
    P.xbits = d_x;
    P.fields = d_fields;
    P.tape_flip = flips;
    P.tape_m = multiplicities;
    P.status = d_status;
    P.tape_cap = (flips && multiplicities) ? steps : 0;
    P.steps = steps;
    P.L0 = cfg->L0;
    P.seed = cfg->seed;
    P.variant = cfg->variant;
    P.subset = cfg->subset;
    P.W = W;
    P.LD = n;
    P.R = 1;
    P.pt = 0;
    P.tape = (flips && multiplicities) ? 1 : 0;
    P.prod = 0;
    P.chain_base = static_cast<uint32_t>(cfg->chain_base);
    P.anneal_start = cfg->anneal_start;
    P.anneal_steps = cfg->anneal_steps;
    if (steps > 0)
        SCU(launch_sampler(PNS_DENSE, qt, 4, T, P, static_cast<int>(ctas), per_cta * 32 * T,
                           static_cast<size_t>(per_cta) * chain_bytes, s));
    int32_t code = 0;
    SCU(cudaMemcpyAsync(&code, d_status, sizeof(code), cudaMemcpyDeviceToHost, s));
    if (states)
        SCU(cudaMemcpyAsync(states, d_x, sizeof(uint32_t) * W * chains, cudaMemcpyDefault, s));
    if (stats) {
        pns_stats *d_stats = reinterpret_cast<pns_stats *>(base + o_stats);
        static_stats_kernel<<<static_cast<unsigned>((chains + 127) / 128), 128, 0, s>>>(d_state, d_stats, chains);
        SCU(cudaGetLastError());
        SCU(cudaMemcpyAsync(stats, d_stats, sizeof(pns_stats) * chains, cudaMemcpyDefault, s));
    }
    SCU(cudaStreamSynchronize(s));
    forget.done = true;
    if (code != 0) return sfail(static_cast<pns_status>(code), "device reported error %d", code);
    return PNS_OK;
}

}  // extern "C"
