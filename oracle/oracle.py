"""ctypes front end of the C oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
leg may import this module.  It drives oracle/pns_oracle.c one chain at a
time, in plain loops, and lays chains out with the same global chain ids the
library uses: instance p, chain c of each replica, replica slot r ->
id = base_p + c * R_p + r, base_p = sum over earlier instances of C * R.
Parallel-tempering groups are the R replicas of one (p, c), numbered in the
same order.
"""
import ctypes as C
import os

import numpy as np

from .build_oracle import build

VARIANTS = {"basic": 0, "unbiased": 1, "rf": 2, "metropolis": 3}
SUBSETS = {"systematic": 0, "random": 1}
TAGS = {"race": 1, "step": 2, "subset": 3, "swap": 5, "alg11": 7}


class _Problem(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("is_float", C.c_int32), ("is_csr", C.c_int32), ("pad", C.c_int32),
        ("q_i", C.c_void_p), ("q_f", C.c_void_p), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
        ("diag_i", C.c_void_p), ("diag_f", C.c_void_p), ("b_i", C.c_void_p), ("b_f", C.c_void_p),
    ]


class _Config(C.Structure):
    _fields_ = [("variant", C.c_int32), ("k", C.c_int32), ("subset", C.c_int32), ("pad", C.c_int32),
                ("L0", C.c_int64), ("seed", C.c_uint64), ("anneal_start", C.c_float), ("pad2", C.c_int32),
                ("anneal_steps", C.c_int64)]


class _Chain(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("L", C.c_int64), ("period_start", C.c_int64), ("flips", C.c_int64),
        ("stays", C.c_int64), ("saturated", C.c_int64), ("swaps_accepted", C.c_int64),
        ("set_start", C.c_int32), ("beta_idx", C.c_int32),
        ("E", C.c_double), ("sum_m", C.c_double), ("best_E", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        vp, i32, i64, u32, u64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_float
        L.oq_init_fields.argtypes = [vp, vp, vp, vp, vp]
        L.oq_decide.argtypes = [i32, vp, vp, i32, f32, u64, u32, u64, vp, vp, vp, vp, vp]
        L.oq_decide.restype = i32
        L.oq_random_subset.argtypes = [i32, i32, u64, u32, u64, vp]
        L.oq_random_subset.restype = i32
        L.oq_run_chain.argtypes = [vp, vp, f32, u32, vp, vp, vp, vp, i64, i64, vp, vp, vp, vp]
        L.oq_run_chain.restype = i32
        L.oq_swap_round.argtypes = [i32, vp, vp, vp, u64, u32, u64, vp]
        L.oq_swap_round.restype = i32
        L.oq_run_alg11.argtypes = [vp, i32, i64, f32, u64, u32, vp, vp, vp, i64, vp]
        L.oq_run_alg11.restype = i32
        L.oq_philox.argtypes = [vp, u32, u32, vp]
        L.oq_donuts_chain.argtypes = [vp, u32, i64, f32, f32, vp]
        L.oq_donuts_chain.restype = i32
        L.oq_sincos2pi_vec.argtypes = [vp, vp, vp, i64]
        L.oq_normal_pair_vec.argtypes = [vp, vp, vp, vp, i64]
        L.oq_donut_energy.argtypes = [f32, f32, f32, f32]
        L.oq_donut_energy.restype = f32
        L.oq_rng_word.argtypes = [u64, u32, u32, u64, u32]
        L.oq_rng_word.restype = u32
        for name in ("oq_logf_vec", "oq_expf_vec", "oq_neg_log1m_vec", "oq_uniform_fine32_vec",
                     "oq_uniform_fine64_vec"):
            getattr(L, name).argtypes = [vp, vp, i64]
        for name in ("oq_logf", "oq_expf", "oq_neg_log1m"):
            getattr(L, name).argtypes = [f32]
            getattr(L, name).restype = f32
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class Problem:
    """One QUBO instance for the oracle.  Integer QUBOs (int16/int32 entries)
    use exact int64 arithmetic; fp32 QUBOs use fp32 fields."""

    def __init__(self, q=None, b=None, csr=None):
        self._keep = []
        st = _Problem()
        if csr is not None:
            row_ptr, col, val, diag = csr
            n = len(row_ptr) - 1
            is_float = np.asarray(val).dtype.kind == "f"
            st.is_csr = 1
            self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
            self.col = np.ascontiguousarray(col, dtype=np.int32)
            st.row_ptr, st.col = _ptr(self.row_ptr), _ptr(self.col)
            if is_float:
                self.val = np.ascontiguousarray(val, dtype=np.float32)
                self.diag = np.ascontiguousarray(diag, dtype=np.float32)
                st.q_f, st.diag_f = _ptr(self.val), _ptr(self.diag)
            else:
                self.val = np.ascontiguousarray(val, dtype=np.int32)
                self.diag = np.ascontiguousarray(diag, dtype=np.int32)
                st.q_i, st.diag_i = _ptr(self.val), _ptr(self.diag)
        else:
            q = np.asarray(q)
            n = q.shape[0]
            is_float = q.dtype.kind == "f"
            if is_float:
                self.q = np.ascontiguousarray(q, dtype=np.float32)
                st.q_f = _ptr(self.q)
            else:
                self.q = np.ascontiguousarray(q, dtype=np.int32)
                st.q_i = _ptr(self.q)
        st.n = n
        st.is_float = int(is_float)
        if b is not None:
            if is_float:
                self.b = np.ascontiguousarray(b, dtype=np.float32)
                st.b_f = _ptr(self.b)
            else:
                self.b = np.ascontiguousarray(b, dtype=np.int32)
                st.b_i = _ptr(self.b)
        self.n = n
        self.is_float = bool(is_float)
        self.struct = st

    def init_fields(self, x):
        x = np.ascontiguousarray(x, dtype=np.uint8)
        h = np.zeros(self.n, dtype=np.float32 if self.is_float else np.int64)
        E = C.c_double(0.0)
        if self.is_float:
            lib().oq_init_fields(C.byref(self.struct), _ptr(x), None, _ptr(h), C.byref(E))
        else:
            lib().oq_init_fields(C.byref(self.struct), _ptr(x), _ptr(h), None, C.byref(E))
        return h, E.value


class ChainState:
    """Mutable state of one oracle chain."""

    def __init__(self, problem, x0, L0, beta_idx=0):
        self.x = np.ascontiguousarray(x0, dtype=np.uint8).copy()
        self.h, E = problem.init_fields(self.x)
        self.st = _Chain()
        self.st.L = L0
        self.st.E = E
        self.st.best_E = E
        self.st.beta_idx = beta_idx
        self.x_best = self.x.copy()  # X_max of Algorithms 8-10


def make_config(variant, k=0, subset="systematic", L0=100, seed=0, anneal_start=1.0, anneal_steps=0):
    """anneal_start s0 and anneal_steps K: the cooling schedule of
    Algorithms 8-10, record k at inverse temperature beta s0^(1 - k/K) for
    k < K (K = 0: constant temperature)."""
    c = _Config()
    c.variant = VARIANTS[variant]
    c.k = int(k)
    c.subset = SUBSETS[subset]
    c.L0 = int(L0)
    c.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    c.anneal_start = float(anneal_start)
    c.anneal_steps = int(anneal_steps)
    return c


def run_chain(problem, cfg, beta, chain_id, state, n_records, stop_after_periods=0, tape=True):
    """Run one chain for n_records records (or until stop_after_periods
    Unbiased periods end).  Returns (flips, M) tapes truncated to the records
    emitted."""
    flips = np.empty(n_records, dtype=np.int32) if tape else None
    ms = np.empty(n_records, dtype=np.float64) if tape else None
    got = C.c_int64(0)
    hi = state.h if not problem.is_float else None
    hf = state.h if problem.is_float else None
    rc = lib().oq_run_chain(C.byref(problem.struct), C.byref(cfg), C.c_float(beta), chain_id,
                            _ptr(state.x), _ptr(hi), _ptr(hf), C.byref(state.st), int(n_records),
                            int(stop_after_periods), _ptr(flips), _ptr(ms), C.byref(got), _ptr(state.x_best))
    if rc != 0:
        raise RuntimeError("oracle run_chain failed with code %d" % rc)
    r = got.value
    if tape:
        return flips[:r], ms[:r]
    return None, None


def decide(deltas, k, beta, seed, chain, step):
    """One race + multiplicity decision over given flip deltas."""
    d = np.asarray(deltas)
    is_float = d.dtype.kind == "f"
    di = np.ascontiguousarray(d, dtype=np.int64) if not is_float else None
    df = np.ascontiguousarray(d, dtype=np.float32) if is_float else None
    win, sq, p, m, sat = C.c_int32(), C.c_uint64(), C.c_float(), C.c_double(), C.c_int32()
    rc = lib().oq_decide(int(is_float), _ptr(di), _ptr(df), int(k), C.c_float(beta), int(seed) & (2**64 - 1),
                         chain, step, C.byref(win), C.byref(sq), C.byref(p), C.byref(m), C.byref(sat))
    if rc:
        raise RuntimeError("oq_decide failed")
    return win.value, sq.value, p.value, m.value, sat.value


def random_subset(n, k, seed, chain, step):
    out = np.empty(k, dtype=np.int32)
    rc = lib().oq_random_subset(n, k, int(seed) & (2**64 - 1), chain, step, _ptr(out))
    if rc:
        raise RuntimeError("oq_random_subset failed")
    return out


def swap_round(betas, E, beta_idx, seed, group, rnd):
    betas = np.ascontiguousarray(betas, dtype=np.float32)
    E = np.ascontiguousarray(E, dtype=np.float64)
    bi = np.ascontiguousarray(beta_idx, dtype=np.int32).copy()
    acc = np.zeros(len(bi), dtype=np.int64)
    lib().oq_swap_round(len(bi), _ptr(betas), _ptr(E), _ptr(bi), int(seed) & (2**64 - 1), group, rnd, _ptr(acc))
    return bi, acc


def run_alg11(problem, k, L0, beta, seed, chain, x0, n_steps):
    x = np.ascontiguousarray(x0, dtype=np.uint8).copy()
    h, _ = problem.init_fields(x)
    codes = np.empty(n_steps, dtype=np.uint32)
    hi = h if not problem.is_float else None
    hf = h if problem.is_float else None
    rc = lib().oq_run_alg11(C.byref(problem.struct), k, L0, C.c_float(beta), int(seed) & (2**64 - 1), chain,
                            _ptr(x), _ptr(hi), _ptr(hf), n_steps, _ptr(codes))
    if rc:
        raise RuntimeError("oq_run_alg11 failed")
    return codes


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    lib().oq_philox(_ptr(c), int(key[0]), int(key[1]), _ptr(out))
    return out


def rng_word(seed, tag, ident, step, index):
    return lib().oq_rng_word(int(seed) & (2**64 - 1), TAGS[tag] if isinstance(tag, str) else tag, ident, step, index)


def _vec(name, x, out_dtype=np.float32):
    x = np.ascontiguousarray(x)
    y = np.empty(x.shape, dtype=out_dtype)
    getattr(lib(), name)(_ptr(x), _ptr(y), x.size)
    return y


def logf(x):
    return _vec("oq_logf_vec", np.asarray(x, dtype=np.float32))


def expf(x):
    return _vec("oq_expf_vec", np.asarray(x, dtype=np.float32))


def neg_log1m(x):
    return _vec("oq_neg_log1m_vec", np.asarray(x, dtype=np.float32))


def uniform_fine32(w):
    return _vec("oq_uniform_fine32_vec", np.asarray(w, dtype=np.uint32))


def uniform_fine64(w):
    return _vec("oq_uniform_fine64_vec", np.asarray(w, dtype=np.uint64))


# ---------------------------------------------------------------------------
# Multi-chain drivers with the library's chain / group numbering.
# ---------------------------------------------------------------------------

def chain_layout(n_replicas, chains_per_replica):
    """Yields (instance, chain_rep, slot, chain_id, group_id) in id order."""
    cid = 0
    gid = 0
    for p, R in enumerate(n_replicas):
        for c in range(chains_per_replica):
            for r in range(R):
                yield p, c, r, cid, gid
                cid += 1
            gid += 1


def run_independent(problems, betas, cfg_kwargs, chains_per_replica, x0, n_records, chain_ids=None, tape=True,
                    id_base=0):
    """Run every chain (or the listed chain ids) independently for n_records
    records.  x0: dict chain_id -> bits (uint8[n]) or None for all-zero.
    Chain ids start at `id_base` (a shard of a larger job).
    Returns dict chain_id -> result dict."""
    cfg = make_config(**cfg_kwargs)
    out = {}
    layout = [(p, c, r, cid + id_base, gid) for p, c, r, cid, gid in
              chain_layout([len(b) for b in betas], chains_per_replica)]
    want = None if chain_ids is None else set(int(c) for c in chain_ids)
    for p, c, r, cid, gid in layout:
        if want is not None and cid not in want:
            continue
        prob = problems[p]
        bits = np.zeros(prob.n, np.uint8) if (x0 is None or cid not in x0) else x0[cid]
        stt = ChainState(prob, bits, cfg.L0, beta_idx=r)
        beta = float(np.float32(betas[p][r]))
        fl, ms = run_chain(prob, cfg, beta, cid, stt, n_records, tape=tape)
        out[cid] = dict(flips=fl, m=ms, x=stt.x.copy(), h=stt.h.copy(), state=stt.st, instance=p, group=gid,
                        x_best=stt.x_best.copy())
    return out


def run_tempering(problem, betas, cfg_kwargs, group_id, chain_id0, x0s, rounds, periods_per_round, tape=True,
                  max_records_per_period=None):
    """Parallel tempering for one group of R replicas: each round every
    replica runs `periods_per_round` units, then one swap round.  Unbiased PNS
    (Algorithm 6): a unit is one complete period of L0 original samples.
    Metropolis (Algorithm 1): a unit is one record, i.e. one original sample.
    Returns per-slot tapes and states."""
    cfg = make_config(**cfg_kwargs)
    metropolis = cfg_kwargs.get("variant") == "metropolis"
    R = len(betas)
    states = [ChainState(problem, x0s[s], cfg.L0, beta_idx=s) for s in range(R)]
    tapes = [([], []) for _ in range(R)]
    cap = max_records_per_period or (cfg.L0 + 1)
    betas32 = np.asarray(betas, dtype=np.float32)
    for rnd in range(rounds):
        for s in range(R):
            st = states[s]
            beta = float(betas32[st.st.beta_idx])
            if metropolis:
                fl, ms = run_chain(problem, cfg, beta, chain_id0 + s, st, periods_per_round, tape=True)
            else:
                fl, ms = run_chain(problem, cfg, beta, chain_id0 + s, st, cap * periods_per_round,
                                   stop_after_periods=periods_per_round, tape=True)
            if tape:
                tapes[s][0].append(fl)
                tapes[s][1].append(ms)
        E = np.array([st.st.E for st in states])
        bidx = np.array([st.st.beta_idx for st in states], dtype=np.int32)
        new_idx, acc = swap_round(betas32, E, bidx, cfg.seed, group_id, rnd)
        for s in range(R):
            states[s].st.beta_idx = int(new_idx[s])
            states[s].st.swaps_accepted += int(acc[s])
    res = []
    for s in range(R):
        fl = np.concatenate(tapes[s][0]) if tape else None
        ms = np.concatenate(tapes[s][1]) if tape else None
        res.append(dict(flips=fl, m=ms, x=states[s].x.copy(), h=states[s].h.copy(), state=states[s].st))
    return res


# ---------------------------------------------------------------------------
# Continuous Unbiased PNS (Algorithm 7) and Metropolis on the Donuts target
# (Sec. 7).
# ---------------------------------------------------------------------------
class _DonutsCfg(C.Structure):
    _fields_ = [("mu0", C.c_float), ("c", C.c_float), ("L0", C.c_int64), ("seed", C.c_uint64),
                ("variant", C.c_int32), ("npairs", C.c_int32)]


class _DonutsStats(C.Structure):
    _fields_ = [("weight", C.c_double), ("sum_x", C.c_double * 2), ("sum_x2", C.c_double * 2),
                ("sum_x4", C.c_double * 2), ("sum_pos", C.c_double * 2), ("records", C.c_int64),
                ("moves", C.c_int64), ("budget_left", C.c_int64), ("period_start", C.c_int64),
                ("x", C.c_float * 2)]


def donuts_chain(variant, chain, steps, x0, mu0=9.0, c=50.0, L0=1000, seed=0, npairs=25):
    """One oracle chain on the Donuts target; returns its statistics as a dict
    (weight, sum_x, sum_x2, sum_x4, sum_pos as 2-arrays, records, moves,
    budget_left, period_start, x)."""
    cfg = _DonutsCfg(np.float32(mu0), np.float32(c), int(L0), int(seed) & (2**64 - 1), VARIANTS[variant], int(npairs))
    st = _DonutsStats()
    rc = lib().oq_donuts_chain(C.byref(cfg), int(chain), int(steps), C.c_float(x0[0]), C.c_float(x0[1]), C.byref(st))
    if rc:
        raise RuntimeError("oq_donuts_chain failed with code %d" % rc)
    return dict(weight=st.weight, sum_x=np.array(st.sum_x[:]), sum_x2=np.array(st.sum_x2[:]),
                sum_x4=np.array(st.sum_x4[:]), sum_pos=np.array(st.sum_pos[:]), records=st.records, moves=st.moves,
                budget_left=st.budget_left, period_start=st.period_start, x=np.array(st.x[:], dtype=np.float32))


def sincos2pi(u):
    u = np.ascontiguousarray(u, dtype=np.float32)
    c = np.empty_like(u)
    s = np.empty_like(u)
    lib().oq_sincos2pi_vec(_ptr(u), _ptr(c), _ptr(s), u.size)
    return c, s


def normal_pairs(w0, w1):
    w0 = np.ascontiguousarray(w0, dtype=np.uint32)
    w1 = np.ascontiguousarray(w1, dtype=np.uint32)
    z1 = np.empty(w0.shape, np.float32)
    z2 = np.empty(w0.shape, np.float32)
    lib().oq_normal_pair_vec(_ptr(w0), _ptr(w1), _ptr(z1), _ptr(z2), w0.size)
    return z1, z2


def donut_energy(x1, x2, mu0=9.0, c=50.0):
    return lib().oq_donut_energy(np.float32(mu0), np.float32(c), np.float32(x1), np.float32(x2))
