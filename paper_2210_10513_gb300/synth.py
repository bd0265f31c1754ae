"""Seeded synthetic QUBO inputs shaped like the paper's workloads.

This module only draws inputs (matrices, linear terms, temperature ladders,
initial states); it holds none of the sampler's arithmetic, and both the CUDA
path and the CPU oracle are fed from it.  All draws use numpy's PCG64 with an
explicit seed.

Workloads (the paper runs random QUBOs, Sec. 4 and Sec. 8.2, and the 4-cube of
Example 2; the shapes below follow the benchmark configurations):
  dense_int      symmetric integer Q, entries i.i.d. uniform in [lo, hi] on and
                 above the diagonal, mirrored below (int16 or int32 storage)
  dense_normal   Q = (A + A^T)/2, A i.i.d. N(0, sigma^2) in fp32
  lattice_csr    L x L periodic nearest-neighbour lattice, couplings +-1 by a
                 fair coin, integer diagonal uniform in [-2, 2], as CSR
  geometric ladder  beta_r = beta_lo (beta_hi/beta_lo)^(r/(R-1))
"""
import numpy as np


def _rng(seed, stream=0):
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def dense_int(n, lo, hi, seed, dtype=np.int16, stream=0):
    g = _rng(seed, stream)
    a = g.integers(lo, hi + 1, size=(n, n), dtype=np.int64)
    up = np.triu(a)
    q = up + np.triu(up, 1).T
    return q.astype(dtype)


def vector_int(n, lo, hi, seed, dtype=np.int16, stream=1):
    g = _rng(seed, stream)
    return g.integers(lo, hi + 1, size=n, dtype=np.int64).astype(dtype)


def dense_normal(n, sigma, seed, stream=0):
    g = _rng(seed, stream)
    a = (g.standard_normal(size=(n, n)) * sigma).astype(np.float32)
    return ((a + a.T) * np.float32(0.5)).astype(np.float32)


def upper_triangular_qubo(n, sigma, seed, stream=2):
    """The paper's random QUBO instance (Sec. 4): U_ij ~ N(0, sigma^2) for
    i <= j, target exp(x^T U x).  Returned in this library's convention,
    E(x) = x^T Q x with pi ~ exp(-beta E): Q = -(U + U^T) / 2 (fp32; halving
    and negating are exact)."""
    g = _rng(seed, stream)
    u = np.triu(g.standard_normal(size=(n, n)) * sigma).astype(np.float32)
    return (-(u + u.T) * np.float32(0.5)).astype(np.float32)


def vector_normal(n, sigma, seed, stream=1):
    g = _rng(seed, stream)
    return (g.standard_normal(size=n) * sigma).astype(np.float32)


def lattice_csr(side, seed, stream=0):
    """Periodic side x side lattice; returns (row_ptr, col, val, diag) with the
    four neighbours of each site in the order left, right, up, down."""
    g = _rng(seed, stream)
    n = side * side
    # one coupling per undirected edge: horizontal (i, right(i)), vertical (i, down(i))
    jh = g.integers(0, 2, size=n, dtype=np.int64) * 2 - 1
    jv = g.integers(0, 2, size=n, dtype=np.int64) * 2 - 1
    diag = g.integers(-2, 3, size=n, dtype=np.int64).astype(np.int32)
    idx = np.arange(n)
    r, c = idx // side, idx % side
    left = r * side + (c - 1) % side
    right = r * side + (c + 1) % side
    up = ((r - 1) % side) * side + c
    down = ((r + 1) % side) * side + c
    col = np.stack([left, right, up, down], axis=1).astype(np.int32)
    val = np.stack([jh[left], jh[idx], jv[up], jv[idx]], axis=1).astype(np.int32)
    row_ptr = (np.arange(n + 1) * 4).astype(np.int32)
    return row_ptr, col.reshape(-1), val.reshape(-1), diag


def csr_to_dense(row_ptr, col, val, diag):
    n = len(row_ptr) - 1
    q = np.zeros((n, n), dtype=np.asarray(val).dtype)
    for i in range(n):
        for e in range(row_ptr[i], row_ptr[i + 1]):
            q[i, col[e]] += val[e]
        q[i, i] += diag[i]
    return q


def geometric_ladder(beta_lo, beta_hi, R):
    if R == 1:
        return np.array([beta_lo], dtype=np.float32)
    r = np.arange(R, dtype=np.float64)
    return (beta_lo * (beta_hi / beta_lo) ** (r / (R - 1))).astype(np.float32)


def random_bits(n_chains, n, seed, stream=7):
    g = _rng(seed, stream)
    return g.integers(0, 2, size=(n_chains, n), dtype=np.int64).astype(np.uint8)


def pack_bits(bits):
    """(C, n) 0/1 -> (C, ceil(n/32)) uint32, bit i of chain c in word i//32,
    position i%32."""
    bits = np.asarray(bits, dtype=np.uint8)
    C, n = bits.shape
    W = (n + 31) // 32
    pad = np.zeros((C, W * 32), dtype=np.uint64)
    pad[:, :n] = bits
    sh = np.arange(32, dtype=np.uint64)
    return (pad.reshape(C, W, 32) << sh).sum(axis=2).astype(np.uint32)


def unpack_bits(words, n):
    words = np.asarray(words, dtype=np.uint32)
    C, W = words.shape
    sh = np.arange(32, dtype=np.uint32)
    bits = (words[:, :, None] >> sh) & 1
    return bits.reshape(C, W * 32)[:, :n].astype(np.uint8)


# ---------------------------------------------------------------------------
# Benchmark-shaped workloads
# ---------------------------------------------------------------------------

def workload_small_dense(seed=0):
    """n=16 dense symmetric int QUBO, entries uniform in [-8, 8], b = 0,
    beta = 1 (and 0.2 for a flatter target)."""
    return dict(q=dense_int(16, -8, 8, seed, np.int32), b=None, n=16)


def workload_dense_int1024(seed=0, n=1024):
    """n=1024 dense symmetric int16 QUBO, entries and b uniform in [-100, 100],
    beta = 0.05, 256 chains, k = 64."""
    return dict(q=dense_int(n, -100, 100, seed, np.int16), b=vector_int(n, -100, 100, seed, np.int16), n=n,
                beta=0.05, chains=256, k=64)


def tempering_sizes(n_instances=512, seed=0, n_lo=128, n_hi=2048):
    """n of each instance of the tempering workload: uniform in [n_lo, n_hi]."""
    g = _rng(seed, 99)
    return [int(n) for n in g.integers(n_lo, n_hi + 1, size=n_instances)]


def tempering_q(p, n, seed=0):
    """Q of instance p of the tempering workload: (A + A^T)/2, A N(0, 1) fp32
    (drawn on its own stream, so that any subset of instances can be made)."""
    return dense_normal(int(n), 1.0, seed, stream=1000 + p)


def workload_tempering(n_instances=512, seed=0, n_lo=128, n_hi=2048, replicas=8):
    """Instances with n uniform in [n_lo, n_hi], Q = (A + A^T)/2 with A
    N(0, 1) fp32, b = 0, geometric beta ladder 0.1 .. 10 with `replicas`
    rungs, k = max(1, n // 16)."""
    ns = tempering_sizes(n_instances, seed, n_lo, n_hi)
    probs = [dict(q=tempering_q(p, n, seed), b=None, n=n) for p, n in enumerate(ns)]
    return probs, geometric_ladder(0.1, 10.0, replicas)


def workload_lattice(side=256, seed=0):
    """side x side periodic lattice (n = side^2) as CSR, b = 0, k = 1024,
    beta in {0.2, 0.44, 1.0}, 64 chains per beta."""
    return dict(csr=lattice_csr(side, seed), b=None, n=side * side, betas=np.array([0.2, 0.44, 1.0], np.float32))


def workload_fit(n=64, seed=0):
    """n=64 fp32 QUBO, Q = (A + A^T)/2 with A N(0, 0.1^2), b N(0, 0.1^2)."""
    return dict(q=dense_normal(n, 0.1, seed), b=vector_normal(n, 0.1, seed), n=n)
