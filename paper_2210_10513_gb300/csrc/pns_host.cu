// pns_host.cu -- the C ABI of include/pns.h: instance upload and validation,
// chain-to-CTA planning, launches, read-back and checkpoints.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pns.h"
#include "pns_launch.h"

using namespace pnsk;

namespace {

thread_local std::string g_err;

pns_status fail(pns_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CU(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            if (e_ == cudaErrorMemoryAllocation)                                                   \
                return fail(PNS_ERR_OOM, "%s: %s", #call, cudaGetErrorString(e_));                 \
            return fail(PNS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));                    \
        }                                                                                          \
    } while (0)

// Host-side fault injection for failure-path tests (environment variable
// PNS_FAULT, read at each call): "alloc" makes every device allocation of the
// library fail with PNS_ERR_OOM, "alloc_after=N" every allocation after the
// first N made since PNS_FAULT took its current value, and "launch" makes
// pns_run / pns_run_plain fail with PNS_ERR_CUDA before launching.  Nothing
// reaches the GPU; the call returns as the real failure would.
bool fault_injected(const char *what) {
    const char *e = getenv("PNS_FAULT");
    return e && strstr(e, what);
}

bool alloc_fault() {
    static std::mutex mu;
    static std::string seen;
    static long long allocs = 0;
    const char *e = getenv("PNS_FAULT");
    std::lock_guard<std::mutex> lock(mu);
    const std::string now = e ? e : "";
    if (now != seen) {  // a new setting: count from zero
        seen = now;
        allocs = 0;
    }
    const long long done = allocs++;
    if (!e) return false;
    if (const char *a = strstr(e, "alloc_after=")) return done >= atoll(a + 12);
    return strstr(e, "alloc") != nullptr;
}

#define CU_MALLOC(ptr, bytes)                                                                      \
    do {                                                                                           \
        if (alloc_fault()) return fail(PNS_ERR_OOM, "injected allocation failure (PNS_FAULT)");    \
        CU(cudaMalloc(ptr, bytes));                                                                \
    } while (0)

int qtype_bytes(int qtype) { return qtype == PNS_Q_I16 ? 2 : 4; }

int32_t round_up(int32_t v, int32_t m) { return (v + m - 1) / m * m; }

struct InstHost {
    int32_t n, ld, k, R;
    int64_t q_off;       // elements (dense) / values (CSR) into the Q buffer
    int64_t nnz;
    int64_t rp_off;      // CSR row_ptr offset
    int64_t vec_off;     // offset of diag / b (elements)
    int64_t beta_off;
};

constexpr uint64_t kCkptMagic = 0x31504b4353504e50ull;  // "PNSCKP1"

}  // namespace

void pnsk::set_last_error(const char *msg) { g_err = msg; }

struct pns_ctx {
    int device = 0;
    pns_config cfg{};
    int fmt = 0, qtype = 0, is_float = 0, hbytes = 4, T = 1, prod = 0;
    int spec = 0;  // > 0: speculative kernel with this many warps (records) per chain
    bool blocked = false;  // period-blocked kernel
    bool sweep = false;    // with spec > 0: the set-sweep kernel (spec warps per chain)
    bool half = false;     // two chains per warp (pns_half.cu)
    int gw = 1;            // blocked kernel: warps per exchange group
    std::vector<InstHost> inst;
    int32_t max_ld = 32, LD = 32, W = 1;
    int64_t chains = 0;
    int R = 1;  // exchange group size
    // device memory
    void *d_q = nullptr;
    size_t q_bytes = 0;
    int32_t *d_rowptr = nullptr, *d_col = nullptr;
    void *d_diag = nullptr, *d_b = nullptr;
    float *d_betas = nullptr;
    InstDesc *d_inst = nullptr;
    ChainDesc *d_chain = nullptr;
    ChainState *d_state = nullptr;
    uint32_t *d_x = nullptr;
    void *d_fields = nullptr;
    CtaDesc *d_cta = nullptr;
    int32_t *d_cta_chains = nullptr;
    int32_t *d_status = nullptr;
    int32_t *d_tape_flip = nullptr;
    double *d_tape_m = nullptr;
    uint32_t *d_tape_x = nullptr;   // tape = 2
    double *d_tape_E = nullptr;
    uint32_t *d_xbest = nullptr;    // track_best: X_max per chain (W words)
    float4 *d_wtab = nullptr;       // integer Q without exchange: weight tables per distinct beta
    int2 *d_wtab_desc = nullptr;
    int64_t tape_alloc = 0;  // records per chain allocated
    int64_t tape_cap = 0;    // records per chain of the last run
    // plan
    int n_cta = 0, n_threads = 32;
    size_t smem = 0;
    int latched = 0;
    std::vector<ChainDesc> h_chains;  // host copy of the chain descriptors (smem offsets per mapping)
    int num_sms = 0, smem_optin = 0;
    int per_cta = 0;
    // CUDA graph of the last pns_run launch
    cudaGraphExec_t gexec = nullptr;
    int64_t g_steps = -1;
    cudaStream_t g_stream = nullptr;
    bool tape_off = false;  // autotuner probes run without the tape
    // pns_moments working memory, kept between calls (grow only)
    void *d_mom = nullptr;
    size_t mom_bytes = 0;
};

namespace {

void free_ctx(pns_ctx *c) {
    if (!c) return;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    void *ptrs[] = {c->d_q, c->d_rowptr, c->d_col, c->d_diag, c->d_b, c->d_betas, c->d_inst, c->d_chain,
                    c->d_state, c->d_x, c->d_fields, c->d_cta, c->d_cta_chains, c->d_status, c->d_tape_flip,
                    c->d_tape_m,  c->d_tape_x, c->d_tape_E, c->d_xbest, c->d_wtab, c->d_wtab_desc, c->d_mom};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete c;
}

pns_status check_args(const pns_problem *probs, int32_t n_probs, const pns_config *cfg) {
    if (!probs || n_probs < 1) return fail(PNS_ERR_INVALID_ARG, "need at least one problem");
    if (!cfg) return fail(PNS_ERR_INVALID_ARG, "cfg is NULL");
    if (cfg->variant < PNS_BASIC || cfg->variant > PNS_METROPOLIS)
        return fail(PNS_ERR_INVALID_ARG, "unknown variant %d", cfg->variant);
    if (cfg->subset != PNS_SUBSET_SYSTEMATIC && cfg->subset != PNS_SUBSET_RANDOM)
        return fail(PNS_ERR_INVALID_ARG, "unknown subset mode %d", cfg->subset);
    if (cfg->chains_per_replica < 1) return fail(PNS_ERR_INVALID_ARG, "chains_per_replica must be >= 1");
    if (cfg->L0 < 1) return fail(PNS_ERR_INVALID_ARG, "L0 must be >= 1");
    if (cfg->tape < 0 || cfg->tape > 2) return fail(PNS_ERR_INVALID_ARG, "tape must be 0, 1 or 2");
    const int w = cfg->warps_per_chain;
    if (!(w == 0 || w == 1 || w == 2 || w == 4 || w == 8 || w == 16 || w == 32))
        return fail(PNS_ERR_INVALID_ARG, "warps_per_chain must be 0, 1, 2, 4, 8, 16 or 32");
    if (cfg->swap_interval < 0) return fail(PNS_ERR_INVALID_ARG, "swap_interval must be >= 0");
    if (cfg->graph != 0 && cfg->graph != 1) return fail(PNS_ERR_INVALID_ARG, "graph must be 0 or 1");
    if (cfg->autotune != 0 && cfg->autotune != 1) return fail(PNS_ERR_INVALID_ARG, "autotune must be 0 or 1");
    if (cfg->track_best != 0 && cfg->track_best != 1) return fail(PNS_ERR_INVALID_ARG, "track_best must be 0 or 1");
    if (cfg->chains_per_cta < 0 || cfg->reserved != 0 || cfg->chain_base < 0 || cfg->group_base < 0)
        return fail(PNS_ERR_INVALID_ARG, "chains_per_cta, chain_base, group_base must be >= 0 and reserved 0");
    if (cfg->reserved2 != 0 || cfg->anneal_steps < 0)
        return fail(PNS_ERR_INVALID_ARG, "anneal_steps must be >= 0 and reserved2 0");
    if (cfg->anneal_steps > 0) {
        if (!(cfg->anneal_start > 0.0f) || !(cfg->anneal_start <= 1.0f))
            return fail(PNS_ERR_INVALID_ARG, "anneal_start must be in (0, 1]");
        if (cfg->swap_interval > 0)
            return fail(PNS_ERR_UNSUPPORTED, "a cooling schedule with replica exchange is not supported");
    }
    if (cfg->swap_interval > 0) {
        if (cfg->variant != PNS_UNBIASED && cfg->variant != PNS_METROPOLIS)
            return fail(PNS_ERR_INVALID_ARG, "replica exchange needs PNS_UNBIASED or PNS_METROPOLIS");
        if (cfg->variant == PNS_UNBIASED && cfg->swap_interval % cfg->L0 != 0)
            return fail(PNS_ERR_INVALID_ARG, "swap_interval must be a multiple of L0");
    }
    const int fmt = probs[0].fmt, qt = probs[0].qtype;
    if (fmt != PNS_DENSE && fmt != PNS_CSR) return fail(PNS_ERR_INVALID_ARG, "unknown format %d", fmt);
    if (qt < PNS_Q_I16 || qt > PNS_Q_F32) return fail(PNS_ERR_INVALID_ARG, "unknown qtype %d", qt);
    const int R0 = probs[0].n_replicas;
    for (int p = 0; p < n_probs; ++p) {
        const pns_problem &pr = probs[p];
        if (pr.fmt != fmt || pr.qtype != qt)
            return fail(PNS_ERR_INVALID_ARG, "problem %d: all problems must share fmt and qtype", p);
        if (pr.n < 1 || pr.n > (1 << 24)) return fail(PNS_ERR_INVALID_ARG, "problem %d: n = %d out of range", p, pr.n);
        if (pr.n_replicas < 1 || !pr.betas)
            return fail(PNS_ERR_INVALID_ARG, "problem %d: need n_replicas >= 1 and betas", p);
        if (!pr.q && !(fmt == PNS_CSR && pr.nnz == 0)) return fail(PNS_ERR_INVALID_ARG, "problem %d: q is NULL", p);
        if (fmt == PNS_CSR && (!pr.row_ptr || pr.nnz < 0 || (pr.nnz > 0 && !pr.col)))
            return fail(PNS_ERR_INVALID_ARG, "problem %d: CSR needs row_ptr, col and nnz >= 0", p);
        if (pr.k < 0 || pr.reserved != 0) return fail(PNS_ERR_INVALID_ARG, "problem %d: k < 0 or reserved != 0", p);
        if (cfg->variant == PNS_BASIC || cfg->variant == PNS_UNBIASED) {
            const int k = pr.k > 0 ? pr.k : cfg->k;
            if (k < 1 || k > pr.n)
                return fail(PNS_ERR_INVALID_ARG, "problem %d: k = %d must be in [1, n = %d]", p, k, pr.n);
        }
        if (cfg->swap_interval > 0 && pr.n_replicas != R0)
            return fail(PNS_ERR_INVALID_ARG, "replica exchange needs the same n_replicas for every problem");
        if (cfg->swap_interval > 0 && pr.n_replicas > 32)
            return fail(PNS_ERR_UNSUPPORTED, "replica exchange supports at most 32 replicas");
    }
    return PNS_OK;
}

}  // namespace

// Per-instance subset size: RF uses all n bits, Metropolis one; Basic and
// Unbiased take the instance's k, or cfg.k when it is 0.
static int32_t inst_k(const pns_config &cfg, const pns_problem &pr) {
    if (cfg.variant == PNS_RF) return pr.n;
    if (cfg.variant == PNS_METROPOLIS) return 1;
    return pr.k > 0 ? pr.k : cfg.k;
}

struct PlanOut {
    std::vector<CtaDesc> cta;
    std::vector<int32_t> cta_chains;
    std::vector<int32_t> smem_off;  // per chain
    int block = 32;
    size_t smem = 0;
    bool resident = true;  // every CTA fits on the GPU at once (blocked kernel: checked)
};

// Placement of exchange-group CTAs when the grid has more CTAs than SMs but
// fewer than two per SM.  The block scheduler gives CTAs 0 .. S-1 one SM each
// (S SMs) and CTAs S .. C-1 to SMs 0 .. C-S-1 again, so the CTAs at positions
// C-S .. S-1 run alone on their SM.  The pack places groups largest first and
// pairs the largest instances with the smallest in its first CTAs: those hold
// the slowest groups (the longest rows and widest sets, or the most records
// per period for the hottest replica), and they move to the positions that
// run alone.  Placement changes no result: a group's draws and arithmetic do
// not depend on its CTA.  PNS_PLACE_ALONE=0 keeps the packed order.
static void place_heavy_alone(PlanOut &o, int num_sms) {
    const int C = static_cast<int>(o.cta.size());
    if (C <= num_sms || C >= 2 * num_sms) return;
    if (const char *e = getenv("PNS_PLACE_ALONE"))
        if (!atoi(e)) return;
    const int alone = 2 * num_sms - C;  // SMs that hold one CTA
    std::vector<CtaDesc> v;
    v.reserve(C);
    v.insert(v.end(), o.cta.begin() + alone, o.cta.begin() + num_sms);
    v.insert(v.end(), o.cta.begin(), o.cta.begin() + alone);
    v.insert(v.end(), o.cta.begin() + num_sms, o.cta.end());
    o.cta.swap(v);
}

// Packs chains (or whole exchange groups) into CTAs.  Units are placed in
// decreasing order of shared-memory need; a CTA takes units until it reaches
// the team limit, the shared-memory limit or its share of the work.
static pns_status plan(const pns_ctx &c, const std::vector<ChainDesc> &chains, int num_sms, size_t smem_cap,
                       int per_cta_override, PlanOut &out) {
    const int T = c.T;
    const bool list = needs_list(c.cfg.variant, c.cfg.subset);
    const bool slot_list = c.prod > 0 && c.cfg.variant == PNS_BASIC;
    const bool pt = c.cfg.swap_interval > 0;
    const int TT = c.half ? 16 : 32 * (T + c.prod);  // threads per chain
    // named barriers per CTA (ids 1..15): two per team when a team has more
    // than one warp, then one per exchange group
    const bool team_bars = TT > 32;
    int teams_cap = T == 32 ? 1 : std::min(512 / TT, team_bars ? 7 : (c.half ? 32 : 16));
    if (c.spec > 0) teams_cap = std::max(1, std::min(512 / (32 * c.spec), 15));
    if (c.blocked) teams_cap = 16;
    struct Unit {
        int32_t first, count, bytes;
    };
    std::vector<Unit> units;
    const int R = pt ? c.R : 1;
    for (int64_t i = 0; i < c.chains; i += R) {
        const InstHost &ih = c.inst[chains[i].inst];
        const int32_t per = c.blocked   ? block_chain_bytes(ih.ld, ih.k, c.hbytes, c.qtype == PNS_Q_I16 ? 2 : 4, R, c.gw)
                            : c.spec > 0 && c.sweep ? sweep_chain_bytes(ih.ld, ih.n, ih.k, c.hbytes, c.spec)
                            : c.spec > 0 ? spec_chain_bytes(ih.ld, ih.k, c.hbytes, list, c.spec)
                                         : chain_smem(ih.ld, ih.k, c.hbytes, list, c.prod > 0, slot_list).total;
        units.push_back({static_cast<int32_t>(i), R, per * R});
    }
    if (R > teams_cap) return fail(PNS_ERR_UNSUPPORTED, "exchange group of %d chains exceeds %d teams per CTA", R, teams_cap);
    std::stable_sort(units.begin(), units.end(), [](const Unit &a, const Unit &b) { return a.bytes > b.bytes; });
    if (pt && per_cta_override <= 0) {
        // Exchange groups: up to cap_u groups per CTA, each group (largest
        // first) to the CTA with the least shared memory so far.  Balanced
        // CTAs keep the launch's dynamic shared memory (the maximum over
        // CTAs) near the mean, so that the CTAs can be resident together.
        const int wpg = c.blocked ? c.gw : R * (T + c.prod);  // warps per group
        int cap_units = 0;
        const int max_warps = (!c.blocked && T == 32) ? 32 : 16;
        for (int u = 1; u * wpg <= max_warps; ++u) {
            const int ids = c.blocked ? u : (team_bars ? 2 * u * R : 0) + u;
            if (ids <= 15) cap_units = u;
        }
        if (cap_units == 0) return fail(PNS_ERR_UNSUPPORTED, "an exchange group of %d chains needs too many warps or barriers", R);
        for (const Unit &u : units)
            if (static_cast<size_t>(u.bytes) > smem_cap)
                return fail(PNS_ERR_UNSUPPORTED, "an exchange group needs %d bytes of shared memory, over %zu", u.bytes,
                            smem_cap);
        auto pack = [&](int cap_u, PlanOut &o) {
            const int64_t n_cta = (static_cast<int64_t>(units.size()) + cap_u - 1) / cap_u;
            std::vector<std::vector<int>> members(n_cta);
            std::vector<size_t> load(n_cta, 0);
            for (size_t ui = 0; ui < units.size(); ++ui) {
                const Unit &u = units[ui];
                int64_t best = -1;
                for (int64_t b = 0; b < static_cast<int64_t>(members.size()); ++b) {
                    if (static_cast<int>(members[b].size()) >= cap_u || load[b] + u.bytes > smem_cap) continue;
                    if (best < 0 || load[b] < load[best]) best = b;
                }
                if (best < 0) {
                    members.emplace_back();
                    load.push_back(0);
                    best = static_cast<int64_t>(members.size()) - 1;
                }
                members[best].push_back(static_cast<int>(ui));
                load[best] += u.bytes;
            }
            o = PlanOut();
            o.smem_off.assign(c.chains, 0);
            int max_groups = 0;
            for (size_t b = 0; b < members.size(); ++b) {
                if (members[b].empty()) continue;
                CtaDesc d;
                d.first = static_cast<int32_t>(o.cta_chains.size());
                d.count = 0;
                d.groups = static_cast<int32_t>(members[b].size());
                d.pad = 0;
                size_t off = 0;
                for (int ui : members[b]) {
                    const Unit &u = units[ui];
                    const int32_t per = u.bytes / u.count;
                    for (int s2 = 0; s2 < u.count; ++s2) {
                        o.smem_off[u.first + s2] = static_cast<int32_t>(off) + s2 * per;
                        o.cta_chains.push_back(u.first + s2);
                    }
                    off += u.bytes;
                    d.count += u.count;
                }
                o.cta.push_back(d);
                o.smem = std::max(o.smem, off);
                max_groups = std::max(max_groups, static_cast<int>(d.groups));
            }
            o.block = max_groups * 32 * wpg;
        };
        if (!c.blocked) {
            pack(cap_units, out);
            return PNS_OK;
        }
        // Blocked kernel, first choice: one CTA per SM, each holding the
        // exchange groups of one record form (positions per lane,
        // block_ppl), so that every SM runs a single code path: groups of
        // different forms on one SM thrash the instruction cache.  CTAs are
        // shared out over the forms in proportion to their groups.
        if (const char *e = getenv("PNS_FORM_PER_SM"); !e || atoi(e)) {
            const int S = num_sms;
            const char *ew = getenv("PNS_WIDE_GROUPS");
            const bool wide_groups = !ew || atoi(ew);
            std::vector<int> ucls(units.size());
            int64_t ncls[3] = {0, 0, 0};
            for (size_t i = 0; i < units.size(); ++i) {
                const int ppl = block_ppl(c.inst[chains[units[i].first].inst].k);
                ucls[i] = ppl == 1 ? 0 : (ppl == 2 ? 1 : 2);
                ncls[ucls[i]] += 1;
            }
            int64_t m[3];
            int64_t msum = 0;
            for (int f = 0; f < 3; ++f) {
                m[f] = (ncls[f] + cap_units - 1) / cap_units;
                msum += m[f];
            }
            if (msum <= S) {
                // the remaining SMs in proportion to each form's groups times
                // a per-group weight (largest remainder), never more CTAs than
                // groups.  The weights follow the measured time of a group's
                // period: the wide-set form (4 positions per lane, k > 62)
                // takes about three times as long per record as one position
                // per lane, and runs fewer records per period.
                double wf[3] = {1.0, 1.5, 3.0};
                if (const char *e = getenv("PNS_FORM_WEIGHTS"))
                    if (sscanf(e, "%lf,%lf,%lf", &wf[0], &wf[1], &wf[2]) != 3) wf[0] = 1.0, wf[1] = 1.5, wf[2] = 3.0;
                double wsum = 0.0;
                for (int f = 0; f < 3; ++f) wsum += wf[f] * static_cast<double>(ncls[f]);
                const int64_t spare = S - msum;
                int64_t give[3] = {0, 0, 0}, given = 0;
                double rem[3];
                for (int f = 0; f < 3; ++f) {
                    const double want = static_cast<double>(S) * wf[f] * ncls[f] / wsum - m[f];
                    give[f] = want > 0 ? std::min<int64_t>(static_cast<int64_t>(want), ncls[f] - m[f]) : 0;
                    rem[f] = want > 0 ? want - give[f] : 0.0;
                    given += give[f];
                }
                while (given > spare) {  // (rounding cannot overshoot, but stay safe)
                    for (int f = 0; f < 3 && given > spare; ++f)
                        if (give[f] > 0) give[f] -= 1, given -= 1;
                }
                while (given < spare) {
                    int fb = -1;
                    for (int f = 0; f < 3; ++f)
                        if (m[f] + give[f] < ncls[f] && (fb < 0 || rem[f] > rem[fb])) fb = f;
                    if (fb < 0) break;
                    give[fb] += 1;
                    rem[fb] -= 1.0;
                    given += 1;
                }
                for (int f = 0; f < 3; ++f) m[f] += give[f];
                // pack each form: largest group first to the least-filled CTA with room
                std::vector<std::vector<int>> members;
                std::vector<size_t> load;
                bool ok = true;
                for (int f = 0; f < 3 && ok; ++f) {
                    const size_t b0 = members.size();
                    for (int64_t i = 0; i < m[f]; ++i) {
                        members.emplace_back();
                        load.push_back(0);
                    }
                    for (size_t ui = 0; ui < units.size(); ++ui) {
                        if (ucls[ui] != f) continue;
                        const Unit &u = units[ui];
                        int64_t best = -1;
                        for (size_t b2 = b0; b2 < members.size(); ++b2) {
                            if (static_cast<int>(members[b2].size()) >= cap_units || load[b2] + u.bytes > smem_cap) continue;
                            if (best < 0 || load[b2] < load[best]) best = static_cast<int64_t>(b2);
                        }
                        if (best < 0) {
                            if (static_cast<int>(members.size()) >= S) {
                                ok = false;
                                break;
                            }
                            members.emplace_back();
                            load.push_back(0);
                            best = static_cast<int64_t>(members.size()) - 1;
                        }
                        members[best].push_back(static_cast<int>(ui));
                        load[best] += u.bytes;
                    }
                }
                if (ok) {
                    PlanOut o;
                    o.smem_off.assign(c.chains, 0);
                    int max_groups = 0;
                    for (size_t b2 = 0; b2 < members.size(); ++b2) {
                        if (members[b2].empty()) continue;
                        CtaDesc d;
                        d.first = static_cast<int32_t>(o.cta_chains.size());
                        d.count = 0;
                        d.groups = static_cast<int32_t>(members[b2].size());
                        // wide-set CTAs (4 positions per lane, no draw
                        // buffers) give each group the CTA's spare warps, up
                        // to one warp per chain
                        d.pad = 0;
                        if (wide_groups && ucls[members[b2][0]] == 2) {
                            const int wcta = std::min(R, (cap_units * wpg) / d.groups);
                            if (wcta > wpg) d.pad = wcta;
                        }
                        size_t off = 0;
                        for (int ui : members[b2]) {
                            const Unit &u = units[ui];
                            const int32_t per = u.bytes / u.count;
                            for (int s2 = 0; s2 < u.count; ++s2) {
                                o.smem_off[u.first + s2] = static_cast<int32_t>(off) + s2 * per;
                                o.cta_chains.push_back(u.first + s2);
                            }
                            off += u.bytes;
                            d.count += u.count;
                        }
                        o.cta.push_back(d);
                        o.smem = std::max(o.smem, off);
                        max_groups = std::max(max_groups, static_cast<int>(d.groups));
                    }
                    // a full SM's registers per CTA keeps every CTA alone on its SM
                    o.block = cap_units * 32 * wpg;
                    const int occ = block_occupancy(c.qtype, o.block, o.smem);
                    o.resident = occ >= 1 && static_cast<int>(o.cta.size()) <= S;
                    (void)max_groups;
                    if (o.resident) {
                        out = o;
                        return PNS_OK;
                    }
                }
            }
        }
        // otherwise: the fewest groups per CTA at which every CTA is resident
        // at once (else the shape with the most resident share)
        double best_share = -1.0;
        for (int u = 1; u <= cap_units; ++u) {
            PlanOut o;
            pack(u, o);
            const int occ = block_occupancy(c.qtype, o.block, o.smem);
            const double share = static_cast<double>(occ) * num_sms / static_cast<double>(o.cta.size());
            o.resident = share >= 1.0;
            if (share > best_share) {
                best_share = share;
                out = o;
            }
            if (o.resident) {
                out = o;
                break;
            }
        }
        if (out.resident) place_heavy_alone(out, num_sms);
        return PNS_OK;
    }
    int64_t target = (static_cast<int64_t>(units.size()) + num_sms - 1) / num_sms;
    if (per_cta_override > 0) target = per_cta_override;
    if (target < 1) target = 1;
    out.smem_off.assign(c.chains, 0);
    size_t cur_bytes = 0;
    int cur_teams = 0, cur_units = 0, cur_groups = 0;
    auto close = [&]() {
        if (cur_teams == 0) return;
        CtaDesc d;
        d.first = static_cast<int32_t>(out.cta_chains.size()) - cur_teams;
        d.count = cur_teams;
        d.groups = pt ? cur_groups : 0;
        d.pad = 0;
        out.cta.push_back(d);
        out.smem = std::max(out.smem, cur_bytes);
        cur_bytes = 0;
        cur_teams = cur_units = cur_groups = 0;
    };
    for (const Unit &u : units) {
        if (static_cast<size_t>(u.bytes) > smem_cap)
            return fail(PNS_ERR_UNSUPPORTED, "a chain (or exchange group) needs %d bytes of shared memory, over %zu",
                        u.bytes, smem_cap);
        // named barriers: ids 1..teams for T > 1 teams, then one per exchange group; 15 at most
        const bool bars_ok = !pt || (team_bars ? 2 * (cur_teams + u.count) + cur_groups + 1 <= 15 : cur_groups + 1 <= 15);
        const bool fits = cur_teams + u.count <= teams_cap && cur_bytes + u.bytes <= smem_cap && cur_units < target &&
                          bars_ok;
        if (!fits) close();
        const int32_t per = u.bytes / u.count;
        for (int s = 0; s < u.count; ++s) {
            out.smem_off[u.first + s] = static_cast<int32_t>(cur_bytes) + s * per;
            out.cta_chains.push_back(u.first + s);
        }
        cur_bytes += u.bytes;
        cur_teams += u.count;
        cur_units += 1;
        cur_groups += 1;
    }
    close();
    int max_teams = 0;
    for (const CtaDesc &d : out.cta) max_teams = std::max(max_teams, static_cast<int>(d.count));
    out.block = max_teams * (c.spec > 0 ? 32 * c.spec : (c.blocked ? 32 : TT));
    for (const CtaDesc &d : out.cta) {
        const int ids = c.spec > 0 ? d.count : c.blocked ? d.groups : (team_bars ? 2 * d.count : 0) + (pt ? d.groups : 0);
        if (ids > 15) return fail(PNS_ERR_UNSUPPORTED, "a CTA needs %d named barriers (15 available)", ids);
    }
    return PNS_OK;
}

static int auto_warps(const pns_ctx &c) {
    int kmax = 1;
    for (const InstHost &ih : c.inst) kmax = std::max(kmax, ih.k);
    int T = 1;
    if (c.fmt == PNS_DENSE) {
        if (kmax > 1024) T = 8;
        else if (kmax > 512) T = 4;
        else if (kmax > 256) T = 2;
    } else {
        if (kmax >= 4096) T = 32;
        else if (kmax >= 2048) T = 16;
        else if (kmax >= 512) T = 8;
        else if (kmax >= 128) T = 4;
    }
    return T;
}

// A chain-to-CTA mapping: warps per chain, producer warps, speculation depth.
struct Mapping {
    int T = 1, prod = 0, spec = 0, per_cta = 0, block = 0, gw = 0;  // gw 0: chosen by the planner
    int sweep = 0;  // with spec: the set-sweep kernel
    int half = 0;   // two chains per warp
};

// The period-blocked kernel: Unbiased PNS, systematic sets, exchange, dense Q, k <= 128.
static bool block_allowed(const pns_ctx &c) {
    int kmax = 1;
    for (const InstHost &ih : c.inst) kmax = std::max(kmax, ih.k);
    return c.fmt == PNS_DENSE && c.cfg.swap_interval > 0 && c.cfg.variant == PNS_UNBIASED && c.R <= 16 &&
           c.cfg.L0 < (1ll << 31) && c.cfg.subset == PNS_SUBSET_SYSTEMATIC && block_supported(c.qtype, kmax);
}

// Two chains per warp: Unbiased PNS on systematic sets of k <= 16, dense Q
// with 4-byte fields, no exchange.
static bool half_allowed(const pns_ctx &c) {
    int kmax = 1;
    for (const InstHost &ih : c.inst) kmax = std::max(kmax, ih.k);
    return c.fmt == PNS_DENSE && c.hbytes == 4 && c.cfg.swap_interval == 0 && c.cfg.variant == PNS_UNBIASED &&
           c.cfg.subset == PNS_SUBSET_SYSTEMATIC && kmax <= 16 && c.cfg.warps_per_chain <= 1;
}

static bool spec_allowed(const pns_ctx &c) {
    int kmax = 1;
    for (const InstHost &ih : c.inst) kmax = std::max(kmax, ih.k);
    return c.fmt == PNS_DENSE && c.cfg.swap_interval == 0 && c.cfg.L0 < (1ll << 31) && kmax <= 128 &&
           (c.cfg.variant == PNS_UNBIASED || c.cfg.variant == PNS_METROPOLIS);
}

// The set-sweep kernel with D warps per chain: Unbiased PNS, systematic sets,
// every instance with at most 4 D sets.
static bool sweep_allowed(const pns_ctx &c, int D) {
    if (!spec_allowed(c) || c.cfg.variant != PNS_UNBIASED || c.cfg.subset != PNS_SUBSET_SYSTEMATIC) return false;
    for (const InstHost &ih : c.inst)
        if (!sweep_supported(c.qtype, D, ih.n, ih.k)) return false;
    return true;
}

// The heuristic mapping (and the environment overrides used by the tests).
static pns_status default_mapping(const pns_ctx &c, Mapping &m) {
    const pns_config *cfg = &c.cfg;
    m.per_cta = c.per_cta;
    m.T = cfg->warps_per_chain > 0 ? cfg->warps_per_chain : auto_warps(c);
    if (!sampler_supported(c.fmt, c.qtype, c.hbytes, m.T)) {
        if (cfg->warps_per_chain > 0)
            return fail(PNS_ERR_UNSUPPORTED, "warps_per_chain = %d is not built for this format", m.T);
        m.T = 1;
    }
    // A producer warp per chain pays off when the GPU is latency-bound (few
    // warps per SM); with many chains every warp already has work.
    // Producer warps: one per 32 race numbers, plus one for the record scalars.
    int kmax = 1;
    for (const InstHost &ih : c.inst) kmax = std::max(kmax, ih.k);
    const int prod_want = cfg->variant == PNS_METROPOLIS ? 1 : std::min(3, 1 + (kmax + 31) / 32);
    m.prod = 0;
    if (m.T < 32 && c.chains * m.T <= 8ll * c.num_sms) m.prod = prod_want;
    if (const char *e = getenv("PNS_PRODUCER_WARPS")) m.prod = std::max(0, std::min(3, atoi(e)));
    if (m.T + m.prod > 16 || (m.T == 32 && m.prod > 0)) m.prod = 0;
    // Speculative evaluation (Unbiased / Metropolis, dense, no exchange): a
    // stay leaves the state unchanged, so D warps evaluate D future records at
    // once.  Used when the GPU would otherwise be latency-bound.
    m.spec = 0;
    if (spec_allowed(c) && cfg->warps_per_chain == 0) {
        if (c.chains * 8 <= 16ll * c.num_sms) m.spec = 8;
        else if (c.chains * 4 <= 16ll * c.num_sms) m.spec = 4;
    }
    if (const char *e = getenv("PNS_SPEC_DEPTH")) {
        const int d = atoi(e);
        m.spec = (d == 0 || spec_supported(c.qtype, d)) ? d : 0;
    }
    if (m.spec > 0 && !spec_allowed(c)) m.spec = 0;
    if (cfg->track_best || cfg->anneal_steps > 0) m.spec = 0;  // X_max and the schedule: the per-flip kernel
    if (m.spec > 0) m.prod = 0;
    // The set sweep (systematic sets) evaluates each set once per state
    // instead of once per record.
    m.sweep = m.spec == 8 ? 1 : 0;
    if (const char *e = getenv("PNS_SWEEP")) m.sweep = atoi(e) ? 1 : 0;
    if (m.sweep && !(m.spec > 0 && sweep_allowed(c, m.spec))) m.sweep = 0;
    // one chain per CTA when two CTAs per SM hold them all: the deciding
    // warps of different chains then rarely share an SM
    if (m.sweep && m.per_cta == 0 && c.chains <= 2ll * c.num_sms) m.per_cta = 1;
    // Period blocking takes the dependent row loads off the record chain of
    // every exchange group (whose hottest replica sets the pace).
    m.block = block_allowed(c) && cfg->warps_per_chain <= 1 && !cfg->track_best ? 1 : 0;
    if (const char *e = getenv("PNS_BLOCKED")) m.block = atoi(e) && block_allowed(c) && !cfg->track_best ? 1 : 0;
    if (cfg->anneal_steps > 0) m.sweep = 0;
    if (m.block) {
        m.T = 1;
        m.prod = 0;
        m.spec = 0;
    }
    // Two chains per warp where many one-warp chains make the launch
    // throughput-bound (more chains than 16 warps on every SM hold).
    m.half = half_allowed(c) && m.T == 1 && m.prod == 0 && m.spec == 0 && !m.block &&
                     c.chains > 16ll * c.num_sms
                 ? 1
                 : 0;
    if (const char *e = getenv("PNS_HALF")) m.half = atoi(e) && half_allowed(c) && !m.block ? 1 : 0;
    if (m.half) {
        m.T = 1;
        m.prod = 0;
        m.spec = 0;
        m.sweep = 0;
    }
    return PNS_OK;
}

// Plans the CTAs for a mapping and installs the descriptors on the device
// (fewer producer warps when an exchange group or the barrier budget does not
// fit with them).
static pns_status apply_mapping(pns_ctx *c, Mapping m, cudaStream_t s) {
    pns_status st;
    PlanOut pl;
    while (true) {
        c->T = m.T;
        c->prod = m.prod;
        c->spec = m.spec;
        c->sweep = m.spec > 0 && m.sweep != 0;
        c->blocked = m.block != 0;
        c->half = m.half != 0;
        pl = PlanOut();
        if (c->blocked) {
            // warps per group: the most (up to R) at which every CTA is resident
            int gw = m.gw;
            if (gw == 0)
                if (const char *e = getenv("PNS_GROUP_WARPS")) gw = atoi(e);
            if (gw > 0) {
                c->gw = std::min(gw, c->R);
                st = plan(*c, c->h_chains, c->num_sms, static_cast<size_t>(c->smem_optin), m.per_cta, pl);
            } else {
                st = PNS_ERR_UNSUPPORTED;
                for (int w = c->R; w >= 1; w = w > 1 ? (w + 1) / 2 : 0) {
                    c->gw = w;
                    PlanOut o;
                    const pns_status s2 = plan(*c, c->h_chains, c->num_sms, static_cast<size_t>(c->smem_optin), m.per_cta, o);
                    if (s2 != PNS_OK) continue;
                    st = s2;
                    pl = o;
                    if (o.resident) break;
                    if (w == 1) break;
                }
            }
            break;
        }
        st = plan(*c, c->h_chains, c->num_sms, static_cast<size_t>(c->smem_optin), m.per_cta, pl);
        if (st == PNS_OK || m.prod == 0) break;
        m.prod -= 1;
    }
    if (st != PNS_OK) return st;
    std::vector<ChainDesc> chains = c->h_chains;
    for (int64_t i = 0; i < c->chains; ++i) chains[i].smem_off = pl.smem_off[i];
    if (c->d_chain) cudaFree(c->d_chain);
    if (c->d_cta) cudaFree(c->d_cta);
    if (c->d_cta_chains) cudaFree(c->d_cta_chains);
    c->d_chain = nullptr;
    c->d_cta = nullptr;
    c->d_cta_chains = nullptr;
    c->n_cta = static_cast<int>(pl.cta.size());
    c->n_threads = pl.block;
    c->smem = pl.smem;
    CU_MALLOC(&c->d_chain, sizeof(ChainDesc) * chains.size());
    CU(cudaMemcpyAsync(c->d_chain, chains.data(), sizeof(ChainDesc) * chains.size(), cudaMemcpyHostToDevice, s));
    CU_MALLOC(&c->d_cta, sizeof(CtaDesc) * pl.cta.size());
    CU(cudaMemcpyAsync(c->d_cta, pl.cta.data(), sizeof(CtaDesc) * pl.cta.size(), cudaMemcpyHostToDevice, s));
    CU_MALLOC(&c->d_cta_chains, sizeof(int32_t) * pl.cta_chains.size());
    CU(cudaMemcpyAsync(c->d_cta_chains, pl.cta_chains.data(), sizeof(int32_t) * pl.cta_chains.size(),
                       cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
        c->g_steps = -1;
    }
    return PNS_OK;
}

static pns_status run_impl(pns_ctx *c, int64_t steps, void *stream, bool plain);

// Key of a problem shape for the autotuner cache.
static std::string tune_key(const pns_ctx &c) {
    int64_t n_sum = 0, n_max = 0, k_max = 0;
    for (const InstHost &ih : c.inst) {
        n_sum += ih.n;
        n_max = std::max<int64_t>(n_max, ih.n);
        k_max = std::max<int64_t>(k_max, ih.k);
    }
    char buf[256];
    snprintf(buf, sizeof(buf), "v%d f%d q%d h%d sub%d pt%lld inst%zu nsum%lld nmax%lld kmax%lld chains%lld sms%d",
             c.cfg.variant, c.fmt, c.qtype, c.hbytes, c.cfg.subset, (long long)c.cfg.swap_interval, c.inst.size(),
             (long long)n_sum, (long long)n_max, (long long)k_max, (long long)c.chains, c.num_sms);
    return buf;
}

// Times candidate mappings on short probe runs from a snapshot of the chain
// state (restored after each probe, so the chains are untouched) and keeps
// the fastest.  The records a chain produces do not depend on the mapping.
static pns_status autotune(pns_ctx *c, cudaStream_t s) {
    const std::string key = tune_key(*c);
    const char *path = getenv("PNS_AUTOTUNE_CACHE");
    if (path) {
        if (FILE *f = fopen(path, "r")) {
            char line[512];
            while (fgets(line, sizeof(line), f)) {
                const char *bar = strchr(line, '|');
                if (!bar) continue;
                if (std::string(line, bar - line) == key) {
                    Mapping m;
                    const int got = sscanf(bar + 1, "%d %d %d %d %d %d %d %d", &m.T, &m.prod, &m.spec, &m.per_cta,
                                           &m.block, &m.gw, &m.sweep, &m.half);
                    if (got == 7 || got == 8) {
                        if (got == 7 || !half_allowed(*c)) m.half = 0;
                        fclose(f);
                        return apply_mapping(c, m, s);
                    }
                }
            }
            fclose(f);
        }
    }
    std::vector<Mapping> cands;
    Mapping base;
    pns_status st = default_mapping(*c, base);
    if (st != PNS_OK) return st;
    cands.push_back(base);
    const int Ts_dense[] = {1, 2, 4};
    const int Ts_csr[] = {1, 4, 8, 16, 32};
    const int T_fixed = c->cfg.warps_per_chain;  // an explicit choice is kept
    auto add = [&](Mapping m) {
        if (T_fixed > 0 && (m.T != T_fixed || m.spec > 0)) return;
        if (!sampler_supported(c->fmt, c->qtype, c->hbytes, m.T)) return;
        if (m.spec > 0 && (!spec_allowed(*c) || !spec_supported(c->qtype, m.spec))) return;
        if (m.sweep && (m.spec <= 0 || !sweep_allowed(*c, m.spec))) return;
        if (m.block && (!block_allowed(*c) || m.T != 1)) return;
        if ((c->cfg.track_best || c->cfg.anneal_steps > 0) && (m.block || m.spec > 0)) return;
        if (m.half && (!half_allowed(*c) || m.T != 1 || m.prod || m.spec || m.block)) return;
        for (const Mapping &o : cands)
            if (o.T == m.T && o.prod == m.prod && o.spec == m.spec && o.per_cta == m.per_cta && o.block == m.block &&
                o.gw == m.gw && o.sweep == m.sweep && o.half == m.half)
                return;
        cands.push_back(m);
    };
    if (c->fmt == PNS_DENSE) {
        for (int T : Ts_dense)
            for (int prod = 0; prod <= 3; ++prod) add(Mapping{T, prod, 0, c->per_cta});
        add(Mapping{8, 0, 0, c->per_cta});
        for (int d : {4, 8, 16}) add(Mapping{1, 0, d, c->per_cta});
        add(Mapping{1, 0, 8, c->per_cta, 0, 0, 1});
        if (c->per_cta == 0) add(Mapping{1, 0, 8, 1, 0, 0, 1});  // one chain per CTA: two CTAs share an SM
        for (int gw : {0, c->R, (c->R + 1) / 2, (c->R + 3) / 4}) add(Mapping{1, 0, 0, c->per_cta, 1, gw});
        Mapping hm{1, 0, 0, c->per_cta};
        hm.half = 1;
        add(hm);
    } else {
        for (int T : Ts_csr) add(Mapping{T, 0, 0, c->per_cta});
    }
    // Snapshots: the chains as created (restored at the end) and after a
    // burn-in with the heuristic mapping, from which every candidate is timed
    // (a chain started from its initial state moves far more often than in
    // equilibrium, which would favour the wrong mapping).
    const size_t b_state = sizeof(ChainState) * c->chains, b_x = sizeof(uint32_t) * c->W * c->chains,
                 b_f = static_cast<size_t>(c->hbytes) * c->LD * c->chains, b_all = b_state + b_x + b_f;
    void *snap = nullptr;
    CU_MALLOC(&snap, 2 * b_all);
    struct FreeSnap {
        void *p;
        ~FreeSnap() { cudaFree(p); }
    } fs{snap};
    char *orig = static_cast<char *>(snap), *burned = orig + b_all;
    auto save = [&](char *dst) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(dst, c->d_state, b_state, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst + b_state, c->d_x, b_x, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst + b_state + b_x, c->d_fields, b_f, cudaMemcpyDeviceToDevice, s);
        return e;
    };
    auto load = [&](const char *src) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(c->d_state, src, b_state, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_x, src + b_state, b_x, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_fields, src + b_state + b_x, b_f, cudaMemcpyDeviceToDevice, s);
        return e;
    };
    int64_t n_max = 1;
    for (const InstHost &ih : c->inst) n_max = std::max<int64_t>(n_max, ih.n);
    const int64_t swap = c->cfg.swap_interval;
    auto round_up = [&](int64_t v) { return swap > 0 ? (v + swap - 1) / swap * swap : v; };
    const int64_t burn = round_up(std::min<int64_t>(16 * n_max, 65536));
    const int64_t warm = round_up(64), probe = round_up(1024);
    CU(save(orig));
    c->tape_off = true;
    struct TapeOn {
        pns_ctx *c;
        ~TapeOn() { c->tape_off = false; }
    } tape_on{c};
    pns_status st_b = run_impl(c, burn, s, false);
    if (st_b != PNS_OK) return st_b;
    CU(save(burned));
    struct Events {  // (destroyed on every return path)
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~Events() {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        }
    } ev;
    CU(cudaEventCreate(&ev.e0));
    CU(cudaEventCreate(&ev.e1));
    float best_ms = 1e30f;
    Mapping best = base;
    for (const Mapping &m : cands) {
        if (apply_mapping(c, m, s) != PNS_OK) continue;
        if (run_impl(c, warm, s, false) != PNS_OK) continue;  // first launch of this kernel
        CU(load(burned));
        CU(cudaEventRecord(ev.e0, s));
        pns_status rs = run_impl(c, probe, s, false);
        CU(cudaEventRecord(ev.e1, s));
        CU(cudaEventSynchronize(ev.e1));
        float ms = 0.0f;
        CU(cudaEventElapsedTime(&ms, ev.e0, ev.e1));
        if (rs == PNS_OK && ms < best_ms) {
            best_ms = ms;
            best = m;
        }
        CU(load(burned));
    }
    CU(load(orig));
    CU(cudaStreamSynchronize(s));
    int32_t code = 0;
    CU(cudaMemcpy(&code, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (code != 0) return fail(static_cast<pns_status>(code), "device error while autotuning");
    if (path) {
        if (FILE *f = fopen(path, "a")) {
            fprintf(f, "%s|%d %d %d %d %d %d %d %d\n", key.c_str(), best.T, best.prod, best.spec, best.per_cta,
                    best.block, best.gw, best.sweep, best.half);
            fclose(f);
        }
    }
    return apply_mapping(c, best, s);
}

extern "C" {

const char *pns_last_error(void) { return g_err.c_str(); }

void pns_destroy(pns_ctx *ctx) { free_ctx(ctx); }

pns_status pns_get_info(const pns_ctx *ctx, pns_info *info) {
    if (!ctx || !info) return fail(PNS_ERR_INVALID_ARG, "NULL argument");
    info->chains = ctx->chains;
    info->words_per_chain = ctx->W;
    info->field_stride = ctx->LD;
    info->field_bytes = ctx->hbytes;
    info->field_is_float = ctx->is_float;
    info->tape_capacity = ctx->tape_cap;
    info->warps_per_chain = ctx->spec > 0 ? ctx->spec : ctx->T + ctx->prod;
    info->ctas = ctx->n_cta;
    info->team_warps = ctx->blocked ? ctx->gw : (ctx->spec > 0 ? 0 : ctx->T);
    info->producer_warps = ctx->spec > 0 ? 0 : ctx->prod;
    info->spec_depth = ctx->spec;
    info->set_sweep = ctx->sweep ? 1 : 0;
    info->period_blocked = ctx->blocked ? 1 : 0;
    info->chains_per_warp = ctx->half ? 2 : 1;
    info->reserved_info = 0;
    return PNS_OK;
}

pns_status pns_create(const pns_problem *probs, int32_t n_probs, const pns_config *cfg, void *stream,
                      pns_ctx **out) {
    if (!out) return fail(PNS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    pns_status st = check_args(probs, n_probs, cfg);
    if (st != PNS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    pns_ctx *c = new pns_ctx();
    struct Guard {
        pns_ctx *c;
        bool keep = false;
        ~Guard() {
            if (!keep) free_ctx(c);
        }
    } guard{c};

    c->cfg = *cfg;
    c->cfg.x0 = nullptr;
    c->fmt = probs[0].fmt;
    c->qtype = probs[0].qtype;
    c->is_float = c->qtype == PNS_Q_F32;
    CU(cudaGetDevice(&c->device));
    int num_sms = 0, smem_optin = 0;
    CU(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, c->device));
    CU(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));

    // ---- instance layout ----------------------------------------------------
    const int qb = qtype_bytes(c->qtype);
    const int vb = 4;  // CSR values, diag and b are stored as int32 or float
    int64_t q_elems = 0, rp_elems = 0, vec_elems = 0, beta_elems = 0;
    c->inst.resize(n_probs);
    for (int p = 0; p < n_probs; ++p) {
        InstHost &ih = c->inst[p];
        ih.n = probs[p].n;
        ih.ld = round_up(ih.n, 32);
        ih.k = inst_k(*cfg, probs[p]);
        ih.R = probs[p].n_replicas;
        ih.nnz = probs[p].nnz;
        ih.q_off = q_elems;
        q_elems += c->fmt == PNS_DENSE ? static_cast<int64_t>(ih.n) * ih.ld : ih.nnz;
        ih.rp_off = rp_elems;
        rp_elems += c->fmt == PNS_CSR ? ih.n + 1 : 0;
        ih.vec_off = vec_elems;
        vec_elems += ih.ld;
        ih.beta_off = beta_elems;
        beta_elems += ih.R;
        c->max_ld = std::max(c->max_ld, ih.ld);
    }
    c->LD = c->max_ld;
    c->W = c->max_ld / 32;
    c->R = probs[0].n_replicas;

    // ---- upload ---------------------------------------------------------------
    const size_t q_bytes = static_cast<size_t>(std::max<int64_t>(q_elems, 1)) * (c->fmt == PNS_DENSE ? qb : vb);
    CU_MALLOC(&c->d_q, q_bytes);
    c->q_bytes = q_bytes;
    // (dense: the tiled check zeroes the padding columns; nothing else is unwritten)
    if (c->fmt != PNS_DENSE) CU(cudaMemsetAsync(c->d_q, 0, q_bytes, s));
    // Dense instances arrive packed (row pitch n) through a transient staging
    // copy of them all: one plain copy per instance, then the tiled check
    // writes them into the pitched layout.  Without room for it, each is
    // copied pitched (a 2D copy) and checked in place.
    void *d_stage = nullptr;
    struct StageFree {
        void **p;
        ~StageFree() {
            if (*p) cudaFree(*p);
        }
    } stagefree{&d_stage};
    if (c->fmt == PNS_DENSE) {
        int64_t st_elems = 0;
        for (const InstHost &ih : c->inst) st_elems += static_cast<int64_t>(ih.n) * ih.n;
        if (cudaMalloc(&d_stage, static_cast<size_t>(std::max<int64_t>(st_elems, 1)) * qb) != cudaSuccess) {
            (void)cudaGetLastError();
            d_stage = nullptr;
        }
    }
    int64_t st_off = 0;
    CU_MALLOC(&c->d_diag, static_cast<size_t>(vec_elems) * vb);
    CU_MALLOC(&c->d_b, static_cast<size_t>(vec_elems) * vb);
    CU(cudaMemsetAsync(c->d_diag, 0, static_cast<size_t>(vec_elems) * vb, s));
    CU(cudaMemsetAsync(c->d_b, 0, static_cast<size_t>(vec_elems) * vb, s));
    CU_MALLOC(&c->d_betas, static_cast<size_t>(beta_elems) * sizeof(float));
    if (c->fmt == PNS_CSR) {
        CU_MALLOC(&c->d_rowptr, static_cast<size_t>(rp_elems) * sizeof(int32_t));
        CU_MALLOC(&c->d_col, static_cast<size_t>(std::max<int64_t>(q_elems, 1)) * sizeof(int32_t));
    }
    int32_t *d_flags = nullptr;
    unsigned long long *d_bound = nullptr;
    void *d_tmp = nullptr;
    struct TmpFree {
        void **a, **b, **t;
        ~TmpFree() {
            if (*a) cudaFree(*a);
            if (*b) cudaFree(*b);
            if (*t) cudaFree(*t);
        }
    } tmpfree{reinterpret_cast<void **>(&d_flags), reinterpret_cast<void **>(&d_bound), &d_tmp};
    CU_MALLOC(&d_flags, sizeof(int32_t) * n_probs);
    CU_MALLOC(&d_bound, sizeof(unsigned long long) * n_probs);
    CU(cudaMemsetAsync(d_flags, 0, sizeof(int32_t) * n_probs, s));
    CU(cudaMemsetAsync(d_bound, 0, sizeof(unsigned long long) * n_probs, s));
    int64_t max_n = 0, max_nnz = 0;
    for (const InstHost &ih : c->inst) {
        max_n = std::max<int64_t>(max_n, ih.n);
        max_nnz = std::max<int64_t>(max_nnz, ih.nnz);
    }
    // scratch: dense, every instance's raw b and row sums side by side (no
    // reuse, so no wait between instances); CSR, raw b / diag / values of
    // one instance at a time
    const size_t tmp_bytes = c->fmt == PNS_DENSE ? static_cast<size_t>(vec_elems) * (4 + 8) + 8 * n_probs + 64
                                                 : static_cast<size_t>(std::max<int64_t>({2 * max_n, max_nnz, 1})) * 4 + 64;
    CU_MALLOC(&d_tmp, tmp_bytes);
    char *tmp = static_cast<char *>(d_tmp);
    // the ladders: device ones copied each, host ones gathered and copied in
    // runs of consecutive instances
    {
        std::vector<char> on_dev(n_probs, 0);
        std::vector<float> hb(static_cast<size_t>(beta_elems), 0.0f);
        for (int p = 0; p < n_probs; ++p) {
            const InstHost &ih = c->inst[p];
            cudaPointerAttributes pa{};
            on_dev[p] = cudaPointerGetAttributes(&pa, probs[p].betas) == cudaSuccess &&
                        (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
            (void)cudaGetLastError();
            if (on_dev[p])
                CU(cudaMemcpyAsync(c->d_betas + ih.beta_off, probs[p].betas, sizeof(float) * ih.R, cudaMemcpyDefault,
                                   s));
            else
                memcpy(hb.data() + ih.beta_off, probs[p].betas, sizeof(float) * ih.R);
        }
        for (int p = 0; p < n_probs;) {
            if (on_dev[p]) {
                ++p;
                continue;
            }
            int q = p;
            while (q + 1 < n_probs && !on_dev[q + 1]) ++q;
            const int64_t o = c->inst[p].beta_off, e = c->inst[q].beta_off + c->inst[q].R;
            CU(cudaMemcpy(c->d_betas + o, hb.data() + o, sizeof(float) * (e - o), cudaMemcpyHostToDevice));
            p = q + 1;
        }
    }
    if (c->fmt == PNS_DENSE)
        CU(cudaMemsetAsync(tmp + static_cast<size_t>(vec_elems) * 4, 0,
                           static_cast<size_t>(vec_elems) * 8 + 8 * n_probs, s));
    // dense: the copies on a copy stream, back to back, in 8 batches of
    // instances; each batch's checks (on s) wait only for its own copies
    std::vector<int64_t> st_at(n_probs, 0);
    constexpr int NB = 8;
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev[NB] = {};
    struct CopyStreamFree {
        cudaStream_t *cs;
        cudaEvent_t *ev;
        ~CopyStreamFree() {
            for (int i = 0; i < NB; ++i)
                if (ev[i]) cudaEventDestroy(ev[i]);
            if (*cs) cudaStreamDestroy(*cs);
        }
    } csfree{&cstream, ev};
    auto batch_of = [&](int p) { return static_cast<int>(static_cast<int64_t>(p) * NB / n_probs); };
    if (c->fmt == PNS_DENSE) {
        CU(cudaStreamCreateWithFlags(&cstream, cudaStreamNonBlocking));
        for (int i = 0; i < NB; ++i) CU(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
        CU(cudaEventRecord(ev[0], s));  // (the copies follow the memsets above)
        CU(cudaStreamWaitEvent(cstream, ev[0], 0));
        for (int p = 0; p < n_probs; ++p) {
            const pns_problem &pr = probs[p];
            const InstHost &ih = c->inst[p];
            char *qd = static_cast<char *>(c->d_q) + ih.q_off * qb;
            if (d_stage) {
                st_at[p] = st_off;
                st_off += static_cast<int64_t>(ih.n) * ih.n;
                CU(cudaMemcpyAsync(static_cast<char *>(d_stage) + st_at[p] * qb, pr.q,
                                   static_cast<size_t>(ih.n) * ih.n * qb, cudaMemcpyDefault, cstream));
            } else {
                CU(cudaMemcpy2DAsync(qd, static_cast<size_t>(ih.ld) * qb, pr.q, static_cast<size_t>(ih.n) * qb,
                                     static_cast<size_t>(ih.n) * qb, ih.n, cudaMemcpyDefault, cstream));
            }
            if (pr.b)
                CU(cudaMemcpyAsync(tmp + static_cast<size_t>(ih.vec_off) * 4, pr.b, static_cast<size_t>(ih.n) * qb,
                                   cudaMemcpyDefault, cstream));
            if (p + 1 == n_probs || batch_of(p + 1) != batch_of(p)) CU(cudaEventRecord(ev[batch_of(p)], cstream));
        }
    }
    for (int p = 0; p < n_probs; ++p) {
        const pns_problem &pr = probs[p];
        const InstHost &ih = c->inst[p];
        char *diag_out = static_cast<char *>(c->d_diag) + ih.vec_off * vb;
        char *b_out = static_cast<char *>(c->d_b) + ih.vec_off * vb;
        if (c->fmt == PNS_DENSE) {
            if (p == 0 || batch_of(p) != batch_of(p - 1)) CU(cudaStreamWaitEvent(s, ev[batch_of(p)], 0));
            char *qd = static_cast<char *>(c->d_q) + ih.q_off * qb;
            const void *src = d_stage ? static_cast<const void *>(static_cast<char *>(d_stage) + st_at[p] * qb) : qd;
            const int sld = d_stage ? ih.n : ih.ld;
            const void *braw = pr.b ? tmp + static_cast<size_t>(ih.vec_off) * 4 : nullptr;
            // instance p's row sums, then its block counter (8 bytes per instance apart)
            void *rowsum = tmp + static_cast<size_t>(vec_elems) * 4 + static_cast<size_t>(ih.vec_off) * 8 + 8 * p;
            CU(launch_prepare_dense_tiled(c->qtype, src, sld, qd, ih.n, ih.ld, braw, diag_out, b_out, rowsum,
                                          d_flags + p, d_bound + p, s));
        } else {
            CU(cudaMemcpyAsync(c->d_rowptr + ih.rp_off, pr.row_ptr, sizeof(int32_t) * (ih.n + 1), cudaMemcpyDefault, s));
            char *vals = static_cast<char *>(c->d_q) + ih.q_off * vb;
            if (ih.nnz > 0) {
                CU(cudaMemcpyAsync(c->d_col + ih.q_off, pr.col, sizeof(int32_t) * ih.nnz, cudaMemcpyDefault, s));
                CU(cudaMemcpyAsync(tmp, pr.q, static_cast<size_t>(ih.nnz) * qb, cudaMemcpyDefault, s));
                CU(launch_convert(c->qtype, tmp, vals, ih.nnz, s));
            }
            // raw diag / b converted into the output arrays, then checked in place
            if (pr.diag) {
                CU(cudaMemcpyAsync(tmp, pr.diag, static_cast<size_t>(ih.n) * qb, cudaMemcpyDefault, s));
                CU(launch_convert(c->qtype, tmp, diag_out, ih.n, s));
            }
            if (pr.b) {
                CU(cudaMemcpyAsync(tmp, pr.b, static_cast<size_t>(ih.n) * qb, cudaMemcpyDefault, s));
                CU(launch_convert(c->qtype, tmp, b_out, ih.n, s));
            }
            CU(launch_prepare_csr(c->is_float, c->d_rowptr + ih.rp_off, c->d_col + ih.q_off, vals, diag_out, b_out,
                                  ih.n, ih.nnz, diag_out, b_out, d_flags + p, d_bound + p, s));
        }
        // (CSR: the scratch buffer is reused by the next instance)
        if (c->fmt != PNS_DENSE) CU(cudaStreamSynchronize(s));
    }
    std::vector<int32_t> flags(n_probs);
    std::vector<unsigned long long> bound(n_probs);
    CU(cudaMemcpyAsync(flags.data(), d_flags, sizeof(int32_t) * n_probs, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(bound.data(), d_bound, sizeof(unsigned long long) * n_probs, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (d_stage) {
        CU(cudaFree(d_stage));
        d_stage = nullptr;
    }
    long long ibound = 0;
    for (int p = 0; p < n_probs; ++p) {
        if (flags[p] & FLAG_BAD_CSR) return fail(PNS_ERR_INVALID_ARG, "problem %d: malformed CSR structure", p);
        if (flags[p] & FLAG_NONFINITE) return fail(PNS_ERR_RANGE, "problem %d: non-finite entry", p);
        if (flags[p] & FLAG_ASYM) return fail(PNS_ERR_NOT_SYMMETRIC, "problem %d: Q is not symmetric", p);
        if (c->is_float) {
            double v;
            memcpy(&v, &bound[p], sizeof(double));
            if (!(v < 1e30)) return fail(PNS_ERR_RANGE, "problem %d: field bound %g too large for fp32 fields", p, v);
        } else {
            const long long v = static_cast<long long>(bound[p]);
            if (v > 715827882LL)
                return fail(PNS_ERR_RANGE, "problem %d: 3 * field bound %lld reaches 2^31 (int32 deltas)", p, v);
            ibound = std::max(ibound, v);
        }
    }
    {
        std::vector<float> b(static_cast<size_t>(beta_elems));
        CU(cudaMemcpy(b.data(), c->d_betas, sizeof(float) * b.size(), cudaMemcpyDeviceToHost));
        for (float v : b)
            if (!(v >= 0.0f) || !(v < 3.0e38f)) return fail(PNS_ERR_INVALID_ARG, "betas must be finite and >= 0");
    }
    // field storage width
    if (c->is_float) c->hbytes = 4;
    else if (c->fmt == PNS_DENSE) c->hbytes = 4;
    else c->hbytes = ibound <= 127 ? 1 : (ibound <= 32767 ? 2 : 4);

    // ---- instance descriptors ---------------------------------------------------
    std::vector<InstDesc> idesc(n_probs);
    for (int p = 0; p < n_probs; ++p) {
        const InstHost &ih = c->inst[p];
        InstDesc &d = idesc[p];
        d.q = static_cast<char *>(c->d_q) + ih.q_off * (c->fmt == PNS_DENSE ? qb : vb);
        d.row_ptr = c->fmt == PNS_CSR ? c->d_rowptr + ih.rp_off : nullptr;
        d.col = c->fmt == PNS_CSR ? c->d_col + ih.q_off : nullptr;
        d.diag = static_cast<char *>(c->d_diag) + ih.vec_off * vb;
        d.b = static_cast<char *>(c->d_b) + ih.vec_off * vb;
        d.betas = c->d_betas + ih.beta_off;
        d.n = ih.n;
        d.ld = ih.ld;
        d.k = ih.k;
        d.R = ih.R;
    }
    CU_MALLOC(&c->d_inst, sizeof(InstDesc) * n_probs);
    CU(cudaMemcpyAsync(c->d_inst, idesc.data(), sizeof(InstDesc) * n_probs, cudaMemcpyHostToDevice, s));

    // ---- chains -------------------------------------------------------------------
    std::vector<ChainDesc> chains;
    int32_t group = 0;
    for (int p = 0; p < n_probs; ++p) {
        for (int r = 0; r < cfg->chains_per_replica; ++r, ++group) {
            for (int sl = 0; sl < c->inst[p].R; ++sl) {
                ChainDesc d;
                d.inst = p;
                d.slot = sl;
                d.group = group;
                d.smem_off = 0;
                chains.push_back(d);
            }
        }
    }
    c->chains = static_cast<int64_t>(chains.size());
    if (c->chains > (1ll << 31) - 1) return fail(PNS_ERR_INVALID_ARG, "too many chains");

    // ---- mapping ------------------------------------------------------------------
    c->h_chains = chains;
    c->num_sms = num_sms;
    c->smem_optin = smem_optin;
    c->per_cta = cfg->chains_per_cta;
    if (c->per_cta == 0)
        if (const char *e = getenv("PNS_CHAINS_PER_CTA")) c->per_cta = atoi(e);
    Mapping mp;
    st = default_mapping(*c, mp);
    if (st != PNS_OK) return st;
    st = apply_mapping(c, mp, s);
    if (st != PNS_OK) return st;

    // ---- chain state ------------------------------------------------------------------
    CU_MALLOC(&c->d_state, sizeof(ChainState) * c->chains);
    CU_MALLOC(&c->d_x, sizeof(uint32_t) * c->W * c->chains);
    CU_MALLOC(&c->d_fields, static_cast<size_t>(c->hbytes) * c->LD * c->chains);
    CU_MALLOC(&c->d_status, sizeof(int32_t));
    CU(cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), s));
    std::vector<uint32_t> x(static_cast<size_t>(c->W) * c->chains, 0u);
    if (cfg->x0) {
        CU(cudaMemcpyAsync(x.data(), cfg->x0, sizeof(uint32_t) * x.size(), cudaMemcpyDefault, s));
        CU(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < c->chains; ++i) {
            const int n = c->inst[chains[i].inst].n;
            for (int w = 0; w < c->W; ++w) {
                const int lo = w * 32;
                uint32_t valid = lo >= n ? 0u : (n - lo >= 32 ? 0xFFFFFFFFu : ((1u << (n - lo)) - 1u));
                if (x[i * c->W + w] & ~valid)
                    return fail(PNS_ERR_INVALID_ARG, "x0 of chain %lld has bits set at or beyond n", (long long)i);
            }
        }
    }
    CU(cudaMemcpyAsync(c->d_x, x.data(), sizeof(uint32_t) * x.size(), cudaMemcpyHostToDevice, s));
    std::vector<ChainState> cs(c->chains);
    for (int64_t i = 0; i < c->chains; ++i) {
        ChainState &z = cs[i];
        memset(&z, 0, sizeof(z));
        z.L = cfg->L0;
        z.beta_idx = chains[i].slot;
    }
    CU(cudaMemcpyAsync(c->d_state, cs.data(), sizeof(ChainState) * cs.size(), cudaMemcpyHostToDevice, s));
    CU(launch_init_fields(c->fmt, c->qtype, c->hbytes, c->d_inst, c->d_chain, c->d_x, c->d_fields, c->d_state,
                          c->chains, c->W, c->LD, c->max_ld, s));
    // ---- weight tables: integer dense Q, Unbiased PNS, fixed temperatures --------
    if (!c->is_float && c->fmt == PNS_DENSE && cfg->variant == PNS_UNBIASED && cfg->swap_interval == 0) {
        std::vector<std::pair<uint32_t, int2>> seen;  // beta bits -> (first entry, entries)
        std::vector<int2> desc(c->chains);
        int64_t total = 0;
        std::vector<std::vector<float>> betas(n_probs);
        for (int p = 0; p < n_probs; ++p) {
            betas[p].resize(c->inst[p].R);
            CU(cudaMemcpy(betas[p].data(), c->d_betas + c->inst[p].beta_off, sizeof(float) * c->inst[p].R,
                          cudaMemcpyDeviceToHost));
        }
        for (int64_t i = 0; i < c->chains; ++i) {
            const float beta = betas[chains[i].inst][chains[i].slot];
            uint32_t bits;
            memcpy(&bits, &beta, sizeof(bits));
            int2 d = make_int2(0, 0);
            bool found = false;
            for (const auto &e : seen)
                if (e.first == bits) {
                    d = e.second;
                    found = true;
                    break;
                }
            if (!found) {
                const int32_t ent = wtab_entries(beta);
                if (ent > 0 && total + ent < (1ll << 30)) {
                    d = make_int2(static_cast<int32_t>(total), ent);
                    total += ent;
                }
                seen.push_back({bits, d});
            }
            desc[i] = d;
        }
        if (total > 0) {
            CU_MALLOC(&c->d_wtab, sizeof(float4) * total);
            CU_MALLOC(&c->d_wtab_desc, sizeof(int2) * c->chains);
            CU(cudaMemcpyAsync(c->d_wtab_desc, desc.data(), sizeof(int2) * c->chains, cudaMemcpyHostToDevice, s));
            for (const auto &e : seen)
                if (e.second.y > 0) {
                    float beta;
                    memcpy(&beta, &e.first, sizeof(beta));
                    CU(launch_build_wtab(c->d_wtab + e.second.x, beta, e.second.y, s));
                }
            CU(cudaStreamSynchronize(s));  // (desc is a host vector)
        }
    }
    if (cfg->track_best) {
        // X_max starts as the initial state (Algorithms 8-10)
        CU_MALLOC(&c->d_xbest, sizeof(uint32_t) * c->W * c->chains);
        CU(cudaMemcpyAsync(c->d_xbest, c->d_x, sizeof(uint32_t) * c->W * c->chains, cudaMemcpyDeviceToDevice, s));
    }
    CU(cudaStreamSynchronize(s));
    if (cfg->autotune) {
        st = autotune(c, s);
        if (st != PNS_OK) return st;
    }
    guard.keep = true;
    *out = c;
    return PNS_OK;
}

}  // extern "C"

static pns_status run_impl(pns_ctx *c, int64_t steps, void *stream, bool plain) {
    if (!c) return fail(PNS_ERR_INVALID_ARG, "ctx is NULL");
    if (c->latched) return fail(PNS_ERR_STATE, "context holds a device error (%d); restore or destroy", c->latched);
    if (steps < 0) return fail(PNS_ERR_INVALID_ARG, "steps must be >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool pt = c->cfg.swap_interval > 0;
    int64_t cap = steps;
    if (pt) {
        if (steps % c->cfg.swap_interval != 0)
            return fail(PNS_ERR_INVALID_ARG, "with exchange, steps must be a multiple of swap_interval");
        if (c->cfg.variant == PNS_UNBIASED) cap = steps / c->cfg.L0 * (c->cfg.L0 + 1);
    }
    if (steps == 0) return PNS_OK;
    if (c->cfg.tape && !c->tape_off) {
        if (cap > c->tape_alloc) {
            if (c->d_tape_flip) cudaFree(c->d_tape_flip);
            if (c->d_tape_m) cudaFree(c->d_tape_m);
            if (c->d_tape_x) cudaFree(c->d_tape_x);
            if (c->d_tape_E) cudaFree(c->d_tape_E);
            c->d_tape_flip = nullptr;
            c->d_tape_m = nullptr;
            c->d_tape_x = nullptr;
            c->d_tape_E = nullptr;
            c->tape_alloc = 0;
            CU_MALLOC(&c->d_tape_flip, sizeof(int32_t) * cap * c->chains);
            CU_MALLOC(&c->d_tape_m, sizeof(double) * cap * c->chains);
            if (c->cfg.tape == 2) {
                CU_MALLOC(&c->d_tape_x, sizeof(uint32_t) * c->W * cap * c->chains);
                CU_MALLOC(&c->d_tape_E, sizeof(double) * cap * c->chains);
            }
            c->tape_alloc = cap;
            if (c->gexec) {
                cudaGraphExecDestroy(c->gexec);
                c->gexec = nullptr;
            }
        }
        c->tape_cap = cap;
    } else {
        c->tape_cap = 0;
    }
    KParams P;
    memset(&P, 0, sizeof(P));
    P.inst = c->d_inst;
    P.chain = c->d_chain;
    P.cta = c->d_cta;
    P.cta_chains = c->d_cta_chains;
    P.state = c->d_state;
    P.xbits = c->d_x;
    P.fields = c->d_fields;
    P.tape_flip = c->d_tape_flip;
    P.tape_m = c->d_tape_m;
    P.tape_x = c->d_tape_x;
    P.tape_E = c->d_tape_E;
    P.xbest = c->tape_off ? nullptr : c->d_xbest;  // (autotuner probes leave X_max alone)
    P.status = c->d_status;
    P.tape_cap = c->tape_cap;
    P.steps = steps;
    P.L0 = c->cfg.L0;
    P.swap_interval = c->cfg.swap_interval;
    P.seed = c->cfg.seed;
    P.variant = c->cfg.variant;
    P.subset = c->cfg.subset;
    P.W = c->W;
    P.LD = c->LD;
    P.R = pt ? c->R : 1;
    P.pt = pt ? 1 : 0;
    P.tape = c->tape_off ? 0 : c->cfg.tape;
    P.prod = c->prod;
    // speculative row loads for Unbiased PNS when Q does not stay in L2
    P.gw = c->gw;
    P.wtab = c->d_wtab;
    P.wtab_desc = c->d_wtab_desc;
    P.prefetch = (c->cfg.variant == PNS_UNBIASED && c->q_bytes > (64ull << 20)) ? 1 : 0;
    if (const char *e = getenv("PNS_PREFETCH")) P.prefetch = atoi(e) ? 1 : 0;
    // a host-set cap on the draws of a random k-subset (tests make the bounded
    // loop give up with it); read at each run, baked into a graph when captured
    if (const char *e = getenv("PNS_DRAW_CAP")) P.draw_cap = static_cast<uint32_t>(strtoul(e, nullptr, 10));
    P.anneal_start = c->cfg.anneal_start;
    P.anneal_steps = c->cfg.anneal_steps;
    if (fault_injected("launch")) return fail(PNS_ERR_CUDA, "injected launch failure (PNS_FAULT)");
    P.chain_base = static_cast<uint32_t>(c->cfg.chain_base);
    P.group_base = static_cast<uint32_t>(c->cfg.group_base);
    auto launch = [&](const KParams &Pl, int grid) -> cudaError_t {
        if (c->blocked) return launch_block(c->qtype, Pl, grid, c->n_threads, c->smem, s);
        if (c->half) return launch_half(c->qtype, Pl, grid, c->n_threads, c->smem, s);
        if (c->spec > 0 && c->sweep) {
            int max_sets = 1, max_k = 1;
            for (const InstHost &ih : c->inst) {
                max_sets = std::max(max_sets, sweep_sets(ih.n, ih.k));
                max_k = std::max(max_k, ih.k);
            }
            return launch_sweep(c->qtype, max_sets, max_k, Pl, grid, c->n_threads, c->smem, s);
        }
        if (c->spec > 0) return launch_spec(c->qtype, c->spec, Pl, grid, c->n_threads, c->smem, s);
        return launch_sampler(c->fmt, c->qtype, c->hbytes, c->T, Pl, grid, c->n_threads, c->smem, s);
    };
    if (P.tape && pt) {
        // with exchange a run is counted in original samples, so chains make
        // different numbers of records: the tape past a chain's records reads
        // as zeros, not as an earlier run's entries
        const size_t recs = static_cast<size_t>(c->tape_cap) * static_cast<size_t>(c->chains);
        CU(cudaMemsetAsync(c->d_tape_flip, 0, sizeof(int32_t) * recs, s));
        CU(cudaMemsetAsync(c->d_tape_m, 0, sizeof(double) * recs, s));
        if (c->d_tape_x) CU(cudaMemsetAsync(c->d_tape_x, 0, sizeof(uint32_t) * c->W * recs, s));
        if (c->d_tape_E) CU(cudaMemsetAsync(c->d_tape_E, 0, sizeof(double) * recs, s));
    }
    if (!plain && c->cfg.graph && s != nullptr && !c->tape_off) {
        // one captured launch per step count; the chain state lives in device
        // memory, so replaying the same graph continues the chains
        if (!c->gexec || c->g_steps != steps || c->g_stream != s) {
            if (c->gexec) {
                cudaGraphExecDestroy(c->gexec);
                c->gexec = nullptr;
            }
            cudaGraph_t g = nullptr;
            CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
            const cudaError_t le = launch(P, c->n_cta);
            const cudaError_t ce = cudaStreamEndCapture(s, &g);
            if (g && (le != cudaSuccess || ce != cudaSuccess)) cudaGraphDestroy(g);
            if (le != cudaSuccess) return fail(PNS_ERR_CUDA, "capture: %s", cudaGetErrorString(le));
            if (ce != cudaSuccess) return fail(PNS_ERR_CUDA, "capture: %s", cudaGetErrorString(ce));
            const cudaError_t ie = cudaGraphInstantiate(&c->gexec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                c->gexec = nullptr;
                return fail(PNS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ie));
            }
            c->g_steps = steps;
            c->g_stream = s;
        }
        CU(cudaGraphLaunch(c->gexec, s));
    } else if (!plain) {
        CU(launch(P, c->n_cta));
    } else {
        for (int b = 0; b < c->n_cta; ++b) {
            P.cta = c->d_cta + b;
            CU(launch(P, 1));
        }
    }
    return PNS_OK;
}

extern "C" {

pns_status pns_run(pns_ctx *c, int64_t steps, void *stream) { return run_impl(c, steps, stream, false); }

pns_status pns_run_plain(pns_ctx *c, int64_t steps, void *stream) { return run_impl(c, steps, stream, true); }

static pns_status sync_and_check(pns_ctx *c, cudaStream_t s) {
    CU(cudaStreamSynchronize(s));
    int32_t code = 0;
    CU(cudaMemcpy(&code, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (code != 0) {
        c->latched = code;
        return fail(static_cast<pns_status>(code), "device reported error %d (a bounded loop gave up)", code);
    }
    return PNS_OK;
}

pns_status pns_read(pns_ctx *c, uint32_t *states, double *mult, int32_t *flips, pns_stats *stats, void *stream) {
    if (!c) return fail(PNS_ERR_INVALID_ARG, "ctx is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    pns_status st = sync_and_check(c, s);
    if (st != PNS_OK) return st;
    if (c->latched) return fail(PNS_ERR_STATE, "context holds a device error");
    if (states) CU(cudaMemcpyAsync(states, c->d_x, sizeof(uint32_t) * c->W * c->chains, cudaMemcpyDefault, s));
    if ((mult || flips) && c->tape_cap > 0) {
        if (mult) CU(cudaMemcpyAsync(mult, c->d_tape_m, sizeof(double) * c->tape_cap * c->chains, cudaMemcpyDefault, s));
        if (flips)
            CU(cudaMemcpyAsync(flips, c->d_tape_flip, sizeof(int32_t) * c->tape_cap * c->chains, cudaMemcpyDefault, s));
    }
    if (stats) {
        std::vector<ChainState> cs(c->chains);
        CU(cudaMemcpyAsync(cs.data(), c->d_state, sizeof(ChainState) * c->chains, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < c->chains; ++i) {
            const ChainState &z = cs[i];
            pns_stats &o = stats[i];
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
        }
    }
    CU(cudaStreamSynchronize(s));
    return PNS_OK;
}

pns_status pns_read_samples(pns_ctx *c, uint32_t *states, double *energies, void *stream) {
    if (!c) return fail(PNS_ERR_INVALID_ARG, "ctx is NULL");
    if (c->cfg.tape != 2 || !c->d_tape_x) return fail(PNS_ERR_STATE, "no sample tape (needs tape = 2 and a run)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    pns_status st = sync_and_check(c, s);
    if (st != PNS_OK) return st;
    if (states)
        CU(cudaMemcpyAsync(states, c->d_tape_x, sizeof(uint32_t) * c->W * c->tape_cap * c->chains,
                           cudaMemcpyDefault, s));
    if (energies)
        CU(cudaMemcpyAsync(energies, c->d_tape_E, sizeof(double) * c->tape_cap * c->chains, cudaMemcpyDefault, s));
    CU(cudaStreamSynchronize(s));
    return PNS_OK;
}

pns_status pns_read_best(pns_ctx *c, uint32_t *states, void *stream) {
    if (!c || !states) return fail(PNS_ERR_INVALID_ARG, "NULL argument");
    if (!c->d_xbest) return fail(PNS_ERR_STATE, "the context keeps no best states (needs track_best = 1)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    pns_status st = sync_and_check(c, s);
    if (st != PNS_OK) return st;
    CU(cudaMemcpyAsync(states, c->d_xbest, sizeof(uint32_t) * c->W * c->chains, cudaMemcpyDefault, s));
    CU(cudaStreamSynchronize(s));
    return PNS_OK;
}

pns_status pns_moments(pns_ctx *c, int32_t instance, int32_t beta_idx, pns_moment_scalars *scalars, double *mean_x,
                       double *mean_xx, double *cov_ex, double *cov_exx, void *stream) {
    if (!c) return fail(PNS_ERR_INVALID_ARG, "ctx is NULL");
    if (c->cfg.tape != 2 || !c->d_tape_x) return fail(PNS_ERR_STATE, "no sample tape (needs tape = 2 and a run)");
    if (c->cfg.swap_interval != 0) return fail(PNS_ERR_UNSUPPORTED, "moments need a run without replica exchange");
    if (instance < 0 || instance >= static_cast<int32_t>(c->inst.size()))
        return fail(PNS_ERR_INVALID_ARG, "instance out of range");
    const InstHost &ih = c->inst[instance];
    if (beta_idx < 0 || beta_idx >= ih.R) return fail(PNS_ERR_INVALID_ARG, "beta_idx out of range");
    if (ih.n > 64) return fail(PNS_ERR_UNSUPPORTED, "moments support n <= 64");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    pns_status st = sync_and_check(c, s);
    if (st != PNS_OK) return st;
    // chains of (instance, slot = beta_idx); without exchange slot == temperature
    std::vector<int32_t> ids;
    int64_t base = 0;
    for (int p = 0; p < instance; ++p) base += static_cast<int64_t>(c->cfg.chains_per_replica) * c->inst[p].R;
    for (int r = 0; r < c->cfg.chains_per_replica; ++r) ids.push_back(static_cast<int32_t>(base + r * ih.R + beta_idx));
    const int64_t recs = c->tape_cap;
    const int n = ih.n;
    const size_t scratch_bytes = moments_scratch_bytes(recs * static_cast<int64_t>(ids.size()), n);
    const size_t out_elems = 4 + 2 * static_cast<size_t>(n) + 2 * static_cast<size_t>(n) * n;
    const size_t ids_bytes = (sizeof(int32_t) * ids.size() + 255) & ~static_cast<size_t>(255);
    const size_t need = ids_bytes + ((scratch_bytes + 255) & ~static_cast<size_t>(255)) + sizeof(double) * out_elems;
    if (c->mom_bytes < need) {
        if (c->d_mom) CU(cudaFree(c->d_mom));
        c->d_mom = nullptr;
        c->mom_bytes = 0;
        CU_MALLOC(&c->d_mom, need);
        c->mom_bytes = need;
    }
    int32_t *d_ids = static_cast<int32_t *>(c->d_mom);
    void *d_scratch = static_cast<char *>(c->d_mom) + ids_bytes;
    double *d_out = reinterpret_cast<double *>(static_cast<char *>(d_scratch) +
                                               ((scratch_bytes + 255) & ~static_cast<size_t>(255)));
    CU(cudaMemcpyAsync(d_ids, ids.data(), sizeof(int32_t) * ids.size(), cudaMemcpyHostToDevice, s));
    double *o_sc = d_out, *o_x = d_out + 4, *o_xx = o_x + n, *o_ex = o_xx + n * n, *o_exx = o_ex + n;
    CU(launch_moments(c->d_tape_x, c->d_tape_m, c->d_tape_E, d_ids, static_cast<int64_t>(ids.size()), c->tape_cap,
                      recs, c->W, n, d_scratch, c->d_status, o_sc, o_x, o_xx, o_ex, o_exx, s));
    st = sync_and_check(c, s);
    if (st != PNS_OK) return st;
    if (scalars) CU(cudaMemcpyAsync(scalars, o_sc, sizeof(double) * 4, cudaMemcpyDefault, s));
    if (mean_x) CU(cudaMemcpyAsync(mean_x, o_x, sizeof(double) * n, cudaMemcpyDefault, s));
    if (mean_xx) CU(cudaMemcpyAsync(mean_xx, o_xx, sizeof(double) * n * n, cudaMemcpyDefault, s));
    if (cov_ex) CU(cudaMemcpyAsync(cov_ex, o_ex, sizeof(double) * n, cudaMemcpyDefault, s));
    if (cov_exx) CU(cudaMemcpyAsync(cov_exx, o_exx, sizeof(double) * n * n, cudaMemcpyDefault, s));
    CU(cudaStreamSynchronize(s));
    return PNS_OK;
}

pns_status pns_energy_grads(int32_t n, float beta, const pns_moment_scalars *scalars, const double *mean_x,
                            const double *mean_xx, const double *cov_ex, const double *cov_exx, const double *data_x,
                            const double *data_xx, double data_mean_energy, double *dQ, double *db, double *dbeta,
                            void *stream) {
    if (n < 1 || !scalars || !mean_x || !mean_xx || !dQ || !db || !dbeta)
        return fail(PNS_ERR_INVALID_ARG, "missing argument");
    if (!data_xx && (!cov_ex || !cov_exx)) return fail(PNS_ERR_INVALID_ARG, "mean-energy gradients need covariances");
    if (data_xx && !data_x) return fail(PNS_ERR_INVALID_ARG, "data_x is required with data_xx");
    CU(launch_grads(n, beta, reinterpret_cast<const double *>(scalars), mean_x, mean_xx, cov_ex, cov_exx, data_x,
                    data_xx, data_mean_energy, dQ, db, dbeta, static_cast<cudaStream_t>(stream)));
    return PNS_OK;
}

pns_status pns_data_energy(int32_t n, const float *q, const float *b, const double *data_x, const double *data_xx,
                           double *out, void *stream) {
    if (n < 1 || !q || !data_xx || !out || (b && !data_x)) return fail(PNS_ERR_INVALID_ARG, "missing argument");
    CU(launch_data_energy(n, q, b, data_x, data_xx, out, static_cast<cudaStream_t>(stream)));
    return PNS_OK;
}

pns_status pns_fields(pns_ctx *c, void *out, void *stream) {
    if (!c || !out) return fail(PNS_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    pns_status st = sync_and_check(c, s);
    if (st != PNS_OK) return st;
    CU(cudaMemcpyAsync(out, c->d_fields, static_cast<size_t>(c->hbytes) * c->LD * c->chains, cudaMemcpyDefault, s));
    CU(cudaStreamSynchronize(s));
    return PNS_OK;
}

struct CkptHeader {
    uint64_t magic;
    int64_t chains;
    int32_t W, LD, hbytes, fmt;
};

pns_status pns_checkpoint(pns_ctx *c, void *buf, size_t *bytes) {
    if (!c || !bytes) return fail(PNS_ERR_INVALID_ARG, "NULL argument");
    const size_t xb_bytes = c->d_xbest ? sizeof(uint32_t) * c->W * c->chains : 0;
    const size_t nbytes = sizeof(CkptHeader) + sizeof(ChainState) * c->chains + sizeof(uint32_t) * c->W * c->chains +
                          static_cast<size_t>(c->hbytes) * c->LD * c->chains + xb_bytes;
    if (!buf) {
        *bytes = nbytes;
        return PNS_OK;
    }
    if (*bytes < nbytes) return fail(PNS_ERR_INVALID_ARG, "checkpoint buffer too small (%zu < %zu)", *bytes, nbytes);
    pns_status st = sync_and_check(c, nullptr);
    if (st != PNS_OK) return st;
    CU(cudaDeviceSynchronize());
    char *p = static_cast<char *>(buf);
    CkptHeader h{kCkptMagic, c->chains, c->W, c->LD, c->hbytes, c->fmt};
    memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    CU(cudaMemcpy(p, c->d_state, sizeof(ChainState) * c->chains, cudaMemcpyDefault));
    p += sizeof(ChainState) * c->chains;
    CU(cudaMemcpy(p, c->d_x, sizeof(uint32_t) * c->W * c->chains, cudaMemcpyDefault));
    p += sizeof(uint32_t) * c->W * c->chains;
    CU(cudaMemcpy(p, c->d_fields, static_cast<size_t>(c->hbytes) * c->LD * c->chains, cudaMemcpyDefault));
    p += static_cast<size_t>(c->hbytes) * c->LD * c->chains;
    if (xb_bytes) CU(cudaMemcpy(p, c->d_xbest, xb_bytes, cudaMemcpyDefault));
    *bytes = nbytes;
    return PNS_OK;
}

pns_status pns_restore(pns_ctx *c, const void *buf, size_t bytes) {
    if (!c || !buf) return fail(PNS_ERR_INVALID_ARG, "NULL argument");
    CkptHeader h;
    if (bytes < sizeof(h)) return fail(PNS_ERR_INVALID_ARG, "checkpoint too short");
    memcpy(&h, buf, sizeof(h));
    const size_t xb_bytes = c->d_xbest ? sizeof(uint32_t) * c->W * c->chains : 0;
    const size_t nbytes = sizeof(CkptHeader) + sizeof(ChainState) * c->chains + sizeof(uint32_t) * c->W * c->chains +
                          static_cast<size_t>(c->hbytes) * c->LD * c->chains + xb_bytes;
    if (h.magic != kCkptMagic || h.chains != c->chains || h.W != c->W || h.LD != c->LD || h.hbytes != c->hbytes ||
        h.fmt != c->fmt || bytes != nbytes)
        return fail(PNS_ERR_INVALID_ARG, "checkpoint does not match this context");
    CU(cudaDeviceSynchronize());
    const char *p = static_cast<const char *>(buf) + sizeof(h);
    CU(cudaMemcpy(c->d_state, p, sizeof(ChainState) * c->chains, cudaMemcpyDefault));
    p += sizeof(ChainState) * c->chains;
    CU(cudaMemcpy(c->d_x, p, sizeof(uint32_t) * c->W * c->chains, cudaMemcpyDefault));
    p += sizeof(uint32_t) * c->W * c->chains;
    CU(cudaMemcpy(c->d_fields, p, static_cast<size_t>(c->hbytes) * c->LD * c->chains, cudaMemcpyDefault));
    p += static_cast<size_t>(c->hbytes) * c->LD * c->chains;
    if (xb_bytes) CU(cudaMemcpy(c->d_xbest, p, xb_bytes, cudaMemcpyDefault));
    CU(cudaMemset(c->d_status, 0, sizeof(int32_t)));
    c->latched = 0;
    return PNS_OK;
}

}  // extern "C"
