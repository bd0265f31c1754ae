"""Thin ctypes binding of libpns (include/pns.h).

Argument marshalling only: every step of the sampler runs in the CUDA
library.  The functions keep the C names (pns_create, pns_run, pns_read,
pns_fields, pns_get_info, pns_checkpoint, pns_restore, pns_destroy,
pns_last_error).  Arrays may be numpy arrays (host memory) or torch tensors
(host or device); streams are torch streams or raw cudaStream_t integers.
If the library is missing this module raises: there is no CPU fallback.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpns.so")

BASIC, UNBIASED, RF, METROPOLIS = 0, 1, 2, 3
VARIANTS = {"basic": BASIC, "unbiased": UNBIASED, "rf": RF, "metropolis": METROPOLIS}
Q_I16, Q_I32, Q_F32 = 0, 1, 2
DENSE, CSR = 0, 1
SYSTEMATIC, RANDOM = 0, 1

STATUS = {0: "PNS_OK", 1: "PNS_ERR_INVALID_ARG", 2: "PNS_ERR_NOT_SYMMETRIC", 3: "PNS_ERR_RANGE", 4: "PNS_ERR_OOM",
          5: "PNS_ERR_CUDA", 6: "PNS_ERR_TIMEOUT", 7: "PNS_ERR_STATE", 8: "PNS_ERR_UNSUPPORTED"}


class PnsError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


class pns_problem(C.Structure):
    _fields_ = [("n", C.c_int32), ("fmt", C.c_int32), ("qtype", C.c_int32), ("n_replicas", C.c_int32),
                ("k", C.c_int32), ("reserved", C.c_int32), ("q", C.c_void_p), ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("nnz", C.c_int64),
                ("diag", C.c_void_p), ("b", C.c_void_p), ("betas", C.c_void_p)]


class pns_config(C.Structure):
    _fields_ = [("variant", C.c_int32), ("k", C.c_int32), ("subset", C.c_int32), ("chains_per_replica", C.c_int32),
                ("L0", C.c_int64), ("swap_interval", C.c_int64), ("seed", C.c_uint64), ("tape", C.c_int32),
                ("warps_per_chain", C.c_int32), ("chains_per_cta", C.c_int32), ("chain_base", C.c_int32),
                ("x0", C.c_void_p), ("group_base", C.c_int32), ("graph", C.c_int32), ("autotune", C.c_int32),
                ("track_best", C.c_int32), ("reserved", C.c_int32), ("anneal_start", C.c_float),
                ("reserved2", C.c_int32), ("anneal_steps", C.c_int64)]


class pns_info(C.Structure):
    _fields_ = [("chains", C.c_int64), ("words_per_chain", C.c_int32), ("field_stride", C.c_int32),
                ("field_bytes", C.c_int32), ("field_is_float", C.c_int32), ("tape_capacity", C.c_int64),
                ("warps_per_chain", C.c_int32), ("ctas", C.c_int32), ("team_warps", C.c_int32),
                ("producer_warps", C.c_int32), ("spec_depth", C.c_int32), ("period_blocked", C.c_int32),
                ("set_sweep", C.c_int32), ("chains_per_warp", C.c_int32), ("reserved_info", C.c_int32)]


class pns_moment_scalars(C.Structure):
    _fields_ = [("weight", C.c_double), ("mean_energy", C.c_double), ("var_energy", C.c_double),
                ("samples", C.c_double)]


class pns_stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("flips", C.c_int64), ("stays", C.c_int64), ("saturated", C.c_int64),
                ("swaps_accepted", C.c_int64), ("budget_left", C.c_int64), ("tape_records", C.c_int64),
                ("set_start", C.c_int32), ("beta_idx", C.c_int32), ("energy", C.c_double), ("sum_m", C.c_double),
                ("best_energy", C.c_double)]


STATS_DTYPE = np.dtype([("steps", np.int64), ("flips", np.int64), ("stays", np.int64), ("saturated", np.int64),
                        ("swaps_accepted", np.int64), ("budget_left", np.int64), ("tape_records", np.int64),
                        ("set_start", np.int32), ("beta_idx", np.int32), ("energy", np.float64),
                        ("sum_m", np.float64), ("best_energy", np.float64)])
assert STATS_DTYPE.itemsize == C.sizeof(pns_stats)

EXPORTS = ("pns_create", "pns_run", "pns_run_plain", "pns_read", "pns_read_samples", "pns_moments",
           "pns_energy_grads", "pns_fields", "pns_get_info", "pns_checkpoint", "pns_restore", "pns_destroy",
           "pns_last_error", "pns_sample_static", "pns_read_best", "pns_donuts_run", "pns_l2_read_probe",
           "pns_data_energy")
STATIC_SCRATCH_BYTES = 16 << 20

_lib = None


def lib():
    """Load libpns.so (built by paper_2210_10513_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpns.so is not built (run paper_2210_10513_gb300.build.build()); "
                               "the sampler has no CPU fallback")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.pns_create.argtypes = [vp, C.c_int32, vp, vp, C.POINTER(vp)]
        L.pns_run.argtypes = [vp, C.c_int64, vp]
        L.pns_run_plain.argtypes = [vp, C.c_int64, vp]
        L.pns_read.argtypes = [vp, vp, vp, vp, vp, vp]
        L.pns_fields.argtypes = [vp, vp, vp]
        L.pns_get_info.argtypes = [vp, vp]
        L.pns_checkpoint.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
        L.pns_restore.argtypes = [vp, vp, C.c_size_t]
        L.pns_read_samples.argtypes = [vp, vp, vp, vp]
        L.pns_read_samples.restype = C.c_int
        L.pns_moments.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp, vp, vp, vp]
        L.pns_moments.restype = C.c_int
        L.pns_energy_grads.argtypes = [C.c_int32, C.c_float, vp, vp, vp, vp, vp, vp, vp, C.c_double, vp, vp, vp, vp]
        L.pns_energy_grads.restype = C.c_int
        L.pns_sample_static.argtypes = [vp, vp, C.c_int64, vp, vp, vp, vp, vp]
        L.pns_sample_static.restype = C.c_int
        L.pns_read_best.argtypes = [vp, vp, vp]
        L.pns_read_best.restype = C.c_int
        L.pns_donuts_run.argtypes = [vp, C.c_int64, C.c_int64, vp, vp, vp]
        L.pns_donuts_run.restype = C.c_int
        L.pns_l2_read_probe.argtypes = [C.c_size_t, C.c_int32, C.POINTER(C.c_double), vp]
        L.pns_l2_read_probe.restype = C.c_int
        L.pns_data_energy.argtypes = [C.c_int32, vp, vp, vp, vp, vp, vp]
        L.pns_data_energy.restype = C.c_int
        L.pns_destroy.argtypes = [vp]
        L.pns_destroy.restype = None
        L.pns_last_error.argtypes = []
        L.pns_last_error.restype = C.c_char_p
        for name in ("pns_create", "pns_run", "pns_run_plain", "pns_read", "pns_fields", "pns_get_info", "pns_checkpoint",
                     "pns_restore"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def pns_last_error():
    return lib().pns_last_error().decode()


def _check(status):
    if status != 0:
        raise PnsError(status, pns_last_error())


def _addr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError("unsupported array type %r" % type(a))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _qtype_of(dtype):
    dt = np.dtype(str(dtype).replace("torch.", ""))
    if dt == np.int16:
        return Q_I16
    if dt == np.int32:
        return Q_I32
    if dt == np.float32:
        return Q_F32
    raise TypeError("Q must be int16, int32 or float32, got %s" % dt)


def make_problem(n, q=None, b=None, betas=(1.0,), csr=None, k=0, keep=None):
    """Fill a pns_problem.  `keep` collects the arrays that must stay alive
    until pns_create returns."""
    keep = keep if keep is not None else []
    p = pns_problem()
    p.n = int(n)
    p.k = int(k)
    betas = np.ascontiguousarray(np.asarray(betas, dtype=np.float32).reshape(-1))
    keep.append(betas)
    p.betas = _addr(betas)
    p.n_replicas = len(betas)
    if csr is not None:
        row_ptr, col, val, diag = csr
        p.fmt = CSR
        p.qtype = _qtype_of(val.dtype)
        for a in (row_ptr, col, val, diag):
            if a is not None:
                keep.append(a)
        p.row_ptr, p.col, p.q, p.diag = _addr(row_ptr), _addr(col), _addr(val), _addr(diag)
        p.nnz = int(len(col))
    else:
        p.fmt = DENSE
        p.qtype = _qtype_of(q.dtype)
        keep.append(q)
        p.q = _addr(q)
    if b is not None:
        keep.append(b)
        p.b = _addr(b)
    return p


def make_config(variant="unbiased", k=1, subset="systematic", chains_per_replica=1, L0=100, swap_interval=0, seed=0,
                tape=False, warps_per_chain=0, x0=None, chains_per_cta=0, chain_base=0, group_base=0, graph=False,
                autotune=False, track_best=False, anneal_start=1.0, anneal_steps=0):
    c = pns_config()
    c.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    c.k = int(k)
    c.subset = {"systematic": SYSTEMATIC, "random": RANDOM}[subset] if isinstance(subset, str) else int(subset)
    c.chains_per_replica = int(chains_per_replica)
    c.L0 = int(L0)
    c.swap_interval = int(swap_interval)
    c.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    c.tape = int(tape)
    c.warps_per_chain = int(warps_per_chain)
    c.chains_per_cta = int(chains_per_cta)
    c.chain_base = int(chain_base)
    c.group_base = int(group_base)
    c.graph = int(bool(graph))
    c.autotune = int(bool(autotune))
    c.track_best = int(bool(track_best))
    c.anneal_start = float(anneal_start)
    c.anneal_steps = int(anneal_steps)
    c.x0 = _addr(x0)
    return c


def pns_create(problems, config, stream=None):
    arr = (pns_problem * len(problems))(*problems)
    ctx = C.c_void_p()
    _check(lib().pns_create(C.cast(arr, C.c_void_p), len(problems), C.byref(config), _stream(stream), C.byref(ctx)))
    return ctx


def pns_run(ctx, steps, stream=None):
    _check(lib().pns_run(ctx, int(steps), _stream(stream)))


def pns_run_plain(ctx, steps, stream=None):
    _check(lib().pns_run_plain(ctx, int(steps), _stream(stream)))


def pns_get_info(ctx):
    info = pns_info()
    _check(lib().pns_get_info(ctx, C.byref(info)))
    return info


def pns_read(ctx, states=None, multiplicities=None, flips=None, stats=None, stream=None):
    _check(lib().pns_read(ctx, _addr(states), _addr(multiplicities), _addr(flips), _addr(stats), _stream(stream)))


def pns_read_samples(ctx, states=None, energies=None, stream=None):
    _check(lib().pns_read_samples(ctx, _addr(states), _addr(energies), _stream(stream)))


def pns_read_best(ctx, states, stream=None):
    _check(lib().pns_read_best(ctx, _addr(states), _stream(stream)))


def pns_moments(ctx, instance, beta_idx, scalars=None, mean_x=None, mean_xx=None, cov_ex=None, cov_exx=None,
                stream=None):
    _check(lib().pns_moments(ctx, int(instance), int(beta_idx), _addr(scalars), _addr(mean_x), _addr(mean_xx),
                             _addr(cov_ex), _addr(cov_exx), _stream(stream)))


def pns_energy_grads(n, beta, scalars, mean_x, mean_xx, cov_ex, cov_exx, data_x, data_xx, data_mean_energy, dQ, db,
                     dbeta, stream=None):
    _check(lib().pns_energy_grads(int(n), C.c_float(beta), _addr(scalars), _addr(mean_x), _addr(mean_xx),
                                  _addr(cov_ex), _addr(cov_exx), _addr(data_x), _addr(data_xx),
                                  float(data_mean_energy), _addr(dQ), _addr(db), _addr(dbeta), _stream(stream)))


def pns_data_energy(n, q, b, data_x, data_xx, out, stream=None):
    """out[0] = sum data_xx * Q + sum data_x * b (fp64, device), pns_data_energy."""
    _check(lib().pns_data_energy(int(n), _addr(q), _addr(b), _addr(data_x), _addr(data_xx), _addr(out),
                                 _stream(stream)))


def pns_fields(ctx, out, stream=None):
    _check(lib().pns_fields(ctx, _addr(out), _stream(stream)))


def pns_checkpoint(ctx):
    n = C.c_size_t(0)
    _check(lib().pns_checkpoint(ctx, None, C.byref(n)))
    buf = np.empty(n.value, dtype=np.uint8)
    _check(lib().pns_checkpoint(ctx, _addr(buf), C.byref(n)))
    return buf


def pns_restore(ctx, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib().pns_restore(ctx, _addr(buf), buf.nbytes))


def pns_l2_read_probe(nbytes=64 << 20, passes=50, stream=None):
    """GB/s read from a buffer resident in L2 (pns_l2_read_probe)."""
    out = C.c_double(0.0)
    _check(lib().pns_l2_read_probe(nbytes, passes, C.byref(out), _stream(stream)))
    return out.value


def pns_destroy(ctx):
    if ctx:
        lib().pns_destroy(ctx)


def pns_sample_static(problem, config, steps, states=None, multiplicities=None, flips=None, stats=None,
                      stream=None):
    """One dense instance, create + run + read, with no device allocation
    (working memory is the library's fixed device array)."""
    _check(lib().pns_sample_static(C.byref(problem), C.byref(config), int(steps), _addr(states),
                                   _addr(multiplicities), _addr(flips), _addr(stats), _stream(stream)))


class Sampler:
    """Owns one pns context.  Marshals numpy / torch inputs into the C calls
    and returns numpy results."""

    def __init__(self, problems, variant="unbiased", k=1, subset="systematic", chains_per_replica=1, L0=100,
                 swap_interval=0, seed=0, tape=False, warps_per_chain=0, x0=None, stream=None, chains_per_cta=0,
                 chain_base=0, group_base=0, graph=False, autotune=False, track_best=False, anneal_start=1.0,
                 anneal_steps=0):
        keep = []
        probs = []
        for pr in problems:
            probs.append(make_problem(keep=keep, **pr))
        if x0 is not None:
            keep.append(x0)
        cfg = make_config(variant, k, subset, chains_per_replica, L0, swap_interval, seed, tape, warps_per_chain, x0,
                          chains_per_cta, chain_base, group_base, graph, autotune, track_best, anneal_start,
                          anneal_steps)
        self.ctx = pns_create(probs, cfg, stream)
        self.info = pns_get_info(self.ctx)
        self.tape = bool(tape)

    def run(self, steps, stream=None):
        pns_run(self.ctx, steps, stream)

    def run_plain(self, steps, stream=None):
        pns_run_plain(self.ctx, steps, stream)

    def read(self, stream=None, tape=True):
        info = pns_get_info(self.ctx)
        C_ = info.chains
        states = np.empty((C_, info.words_per_chain), dtype=np.uint32)
        stats = np.empty(C_, dtype=STATS_DTYPE)
        m = f = None
        if tape and self.tape and info.tape_capacity > 0:
            m = np.empty((C_, info.tape_capacity), dtype=np.float64)
            f = np.empty((C_, info.tape_capacity), dtype=np.int32)
        pns_read(self.ctx, states, m, f, stats, stream)
        return dict(states=states, stats=stats, m=m, flips=f)

    def samples(self, stream=None):
        """State bits (chains x capacity x W) and energies at each record's start (tape = 2)."""
        info = pns_get_info(self.ctx)
        x = np.empty((info.chains, info.tape_capacity, info.words_per_chain), dtype=np.uint32)
        e = np.empty((info.chains, info.tape_capacity), dtype=np.float64)
        pns_read_samples(self.ctx, x, e, stream)
        return x, e

    def best(self, stream=None):
        """X_max of every chain (chains x W words, track_best = 1)."""
        info = pns_get_info(self.ctx)
        out = np.empty((info.chains, info.words_per_chain), dtype=np.uint32)
        pns_read_best(self.ctx, out, stream)
        return out

    def moments(self, n, instance=0, beta_idx=0, stream=None, device=None):
        """Multiplicity-weighted moments (fp64): scalars [W, <E>, Var E, samples],
        <x>, <x x^T>, Cov(E, x), Cov(E, x x^T).  numpy on the host, or torch
        tensors on `device`."""
        if device is None:
            out = dict(scalars=np.empty(4), mean_x=np.empty(n), mean_xx=np.empty((n, n)), cov_ex=np.empty(n),
                       cov_exx=np.empty((n, n)))
        else:
            import torch
            f = lambda *shape: torch.empty(shape, dtype=torch.float64, device=device)  # noqa: E731
            out = dict(scalars=f(4), mean_x=f(n), mean_xx=f(n, n), cov_ex=f(n), cov_exx=f(n, n))
        pns_moments(self.ctx, instance, beta_idx, out["scalars"], out["mean_x"], out["mean_xx"], out["cov_ex"],
                    out["cov_exx"], stream)
        return out

    def fields(self, stream=None):
        info = pns_get_info(self.ctx)
        dt = np.float32 if info.field_is_float else {1: np.int8, 2: np.int16, 4: np.int32}[info.field_bytes]
        out = np.empty((info.chains, info.field_stride), dtype=dt)
        pns_fields(self.ctx, out, stream)
        return out

    def checkpoint(self):
        return pns_checkpoint(self.ctx)

    def restore(self, buf):
        pns_restore(self.ctx, buf)

    def close(self):
        if getattr(self, "ctx", None):
            pns_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Continuous targets: Unbiased PNS (Algorithm 7) and Metropolis on the Donuts
# example (Sec. 7).
# ---------------------------------------------------------------------------
class pns_donuts_config(C.Structure):
    _fields_ = [("mu0", C.c_float), ("c", C.c_float), ("L0", C.c_int64), ("seed", C.c_uint64),
                ("variant", C.c_int32), ("npairs", C.c_int32), ("chain_base", C.c_int32), ("reserved", C.c_int32)]


DONUTS_STATS_DTYPE = np.dtype([("weight", np.float64), ("sum_x", np.float64, 2), ("sum_x2", np.float64, 2),
                               ("sum_x4", np.float64, 2), ("sum_pos", np.float64, 2), ("records", np.int64),
                               ("moves", np.int64), ("budget_left", np.int64), ("period_start", np.int64),
                               ("x", np.float32, 2), ("pad", np.int32, 2)])


def pns_donuts_run(variant, chains, steps, x0=None, mu0=9.0, c=50.0, L0=1000, seed=0, npairs=25, chain_base=0,
                   stats=None, stream=None):
    """Runs the Donuts chains; returns per-chain statistics (a numpy record
    array of DONUTS_STATS_DTYPE, or fills `stats`, a device buffer of
    chains * DONUTS_STATS_DTYPE.itemsize bytes)."""
    cfg = pns_donuts_config(float(np.float32(mu0)), float(np.float32(c)), int(L0), int(seed) & 0xFFFFFFFFFFFFFFFF,
                            VARIANTS[variant] if isinstance(variant, str) else int(variant), int(npairs),
                            int(chain_base), 0)
    out = np.zeros(int(chains), dtype=DONUTS_STATS_DTYPE) if stats is None else stats
    if x0 is not None and isinstance(x0, np.ndarray):
        x0 = np.ascontiguousarray(x0, dtype=np.float32)
    _check(lib().pns_donuts_run(C.byref(cfg), int(chains), int(steps), _addr(x0), _addr(out), _stream(stream)))
    return out
