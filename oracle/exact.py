"""Exact enumeration for small QUBOs and small graphs (TEST INFRASTRUCTURE ONLY).

Plain numpy, fp64.  Each function states the definition it writes out:
  - target pi(x) ~ exp(-beta E(x)), E(x) = x^T Q x + b^T x    (Sec. 4, sign of
    the exponent read as exp(-beta E); the paper's exp(x^T Q x) is Q -> -Q)
  - total variation distance, Eq. (5) (Sec. 2.2)
  - multiplicity-weighted histogram of a jump chain (Sec. 2.2, Theorem 3 (5))
  - exact long-run weighted distribution of Basic PNS (Algorithm 3) on any
    finite graph: jump chain transition matrix averaged over the uniformly
    drawn subsets, times E[M | state]
  - per-set Metropolis kernels of Alg. 11 (Appendix A, Prop. 1)
  - moments and gradients of multiplicity-weighted expectations.
"""
import itertools

import numpy as np


def state_bits(n):
    """(2^n, n) uint8 matrix; row c holds the bits of code c (bit i = x_i)."""
    codes = np.arange(1 << n, dtype=np.int64)
    return ((codes[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)


def energies(Q, b=None):
    Q = np.asarray(Q, dtype=np.float64)
    n = Q.shape[0]
    X = state_bits(n).astype(np.float64)
    E = np.einsum("si,ij,sj->s", X, Q, X)
    if b is not None:
        E = E + X @ np.asarray(b, dtype=np.float64)
    return E


def boltzmann(E, beta):
    a = -beta * (np.asarray(E, dtype=np.float64))
    a = a - a.max()
    w = np.exp(a)
    return w / w.sum()


def target(Q, b, beta):
    return boltzmann(energies(Q, b), beta)


def tvd(p, q):
    return 0.5 * float(np.abs(np.asarray(p, np.float64) - np.asarray(q, np.float64)).sum())


def replay_codes(x0_code, flips):
    """State code at the start of each record (J_{k-1} of record k) given the
    flip tape (-1 = stay); n <= 62."""
    flips = np.asarray(flips)
    masks = np.where(flips >= 0, np.left_shift(np.int64(1), np.maximum(flips, 0).astype(np.int64)), 0)
    after = np.bitwise_xor.accumulate(masks) ^ np.int64(x0_code)
    before = np.empty_like(after)
    before[0] = x0_code
    before[1:] = after[:-1]
    return before, (after[-1] if len(after) else np.int64(x0_code))


def weighted_hist(codes, weights, n):
    h = np.bincount(np.asarray(codes, np.int64), weights=np.asarray(weights, np.float64), minlength=1 << n)
    s = h.sum()
    return h / s if s > 0 else h


def code_of(bits):
    bits = np.asarray(bits).astype(np.int64)
    return int((bits << np.arange(len(bits))).sum())


# ---------------------------------------------------------------------------
# Basic PNS (Algorithm 3), exact long-run behaviour on a finite graph.
# ---------------------------------------------------------------------------

def basic_exact_graph(neighbors, pi, k):
    """neighbors[x]: list of neighbour states of x (all of equal size N is not
    required); pi: target weights (unnormalised ok); a uniformly drawn
    k-subset S of the neighbours is used per step with proposal 1/k on S.

    From x with subset S: w_y = (1/k) min(1, pi(y)/pi(x)), p_S = sum w,
    jump to y w.p. w_y / p_S, and M = 1 + Geom(p_S) so E[M | x, S] = 1/p_S.
    Returns (weighted long-run distribution, jump-chain stationary, E[M|x]).
    """
    pi = np.asarray(pi, dtype=np.float64)
    S_n = len(pi)
    P = np.zeros((S_n, S_n))
    mbar = np.zeros(S_n)
    for x in range(S_n):
        nb = list(neighbors[x])
        subsets = list(itertools.combinations(nb, k))
        ps = 1.0 / len(subsets)
        for S in subsets:
            w = np.array([min(1.0, pi[y] / pi[x]) / k for y in S])
            pS = w.sum()
            for y, wy in zip(S, w):
                P[x, y] += ps * wy / pS
            mbar[x] += ps / pS
    # stationary distribution of the jump chain: left eigenvector for 1
    vals, vecs = np.linalg.eig(P.T)
    i = int(np.argmin(np.abs(vals - 1.0)))
    st = np.real(vecs[:, i])
    st = st / st.sum()
    wt = st * mbar
    return wt / wt.sum(), st, mbar


def hypercube_neighbors(n):
    return [[c ^ (1 << i) for i in range(n)] for c in range(1 << n)]


def basic_exact_qubo(Q, b, beta, k):
    n = np.asarray(Q).shape[0]
    pi = target(Q, b, beta)
    wt, _, _ = basic_exact_graph(hypercube_neighbors(n), pi, k)
    return wt, pi


# ---------------------------------------------------------------------------
# Alg. 11 per-set kernels (Appendix A, Proposition 1).
# ---------------------------------------------------------------------------

def systematic_sets(n, k):
    """Sets of the systematic scheme: start advances by k (mod n) per period,
    I = n / gcd(n, k) distinct sets (Sec. 5's wrap-around for k not dividing n)."""
    from math import gcd
    count = n // gcd(n, k)
    return [[(s * k + t) % n for t in range(k)] for s in range(count)]


def alg11_kernel(Q, b, beta, bits_subset):
    """Metropolis kernel restricted to flipping bits in `bits_subset`, proposal
    uniform (1/k) on the subset: P(x, x^e_i) = (1/k) min(1, pi(y)/pi(x))."""
    pi = target(Q, b, beta)
    n = np.asarray(Q).shape[0]
    k = len(bits_subset)
    S_n = 1 << n
    P = np.zeros((S_n, S_n))
    for x in range(S_n):
        for i in bits_subset:
            y = x ^ (1 << i)
            P[x, y] += min(1.0, pi[y] / pi[x]) / k
        P[x, x] = 1.0 - P[x].sum()
    return P, pi


# ---------------------------------------------------------------------------
# Moments and gradients (exact, fp64).
# ---------------------------------------------------------------------------

def exact_moments(Q, b, beta):
    """<E>, Var(E), <x>, <x x^T>, Cov(E, x), Cov(E, x x^T) under pi."""
    n = np.asarray(Q).shape[0]
    X = state_bits(n).astype(np.float64)
    E = energies(Q, b)
    pi = boltzmann(E, beta)
    mE = pi @ E
    vE = pi @ (E - mE) ** 2
    mx = pi @ X
    mxx = (X * pi[:, None]).T @ X
    cEx = (pi * (E - mE)) @ X
    cExx = (X * (pi * (E - mE))[:, None]).T @ X
    return dict(E=mE, varE=vE, x=mx, xx=mxx, covEx=cEx, covExx=cExx)


def log_partition(Q, b, beta):
    E = energies(Q, b)
    a = -beta * E
    m = a.max()
    return float(m + np.log(np.exp(a - m).sum()))


def mean_energy_grads(Q, b, beta):
    """Gradients of <E>_pi.  With E = sum_ij Q_ij x_i x_j + b.x and Q symmetric
    treated entrywise:  d<E>/dQ_ij = <x_i x_j> - beta Cov(E, x_i x_j),
    d<E>/db_i = <x_i> - beta Cov(E, x_i), d<E>/dbeta = -Var(E)."""
    m = exact_moments(Q, b, beta)
    gQ = m["xx"] - beta * m["covExx"]
    gb = m["x"] - beta * m["covEx"]
    gbeta = -m["varE"]
    return gQ, gb, gbeta, m["E"]


def log_likelihood_grads(Q, b, beta, data_xx, data_x, data_E_mean):
    """Boltzmann log-likelihood l = -beta <E>_D - log Z per sample:
    dl/dQ_ij = -beta (<x_i x_j>_D - <x_i x_j>_pi), dl/db = -beta(<x>_D - <x>_pi),
    dl/dbeta = -<E>_D + <E>_pi."""
    m = exact_moments(Q, b, beta)
    gQ = -beta * (data_xx - m["xx"])
    gb = -beta * (data_x - m["x"])
    gbeta = -data_E_mean + m["E"]
    return gQ, gb, gbeta
