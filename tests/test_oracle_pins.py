"""Pins for the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  Statistical bars are stated with the
sample counts they hold at; exact checks are exact.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact as X
from oracle import oracle as O
from paper_2210_10513_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _frac(s):
    return float(Fraction(s))


# ---------------------------------------------------------------------------
# Example 1 (Sec. 2.1): closed form of Basic PNS on the triangle.
# ---------------------------------------------------------------------------

def test_example1_triangle_closed_form():
    g = json.load(open(os.path.join(GOLDEN, "example1_triangle.json")))
    pi = np.array(g["pi_unnormalised"], dtype=np.float64)
    nb = [[1, 2], [0, 2], [0, 1]]
    wt, jump_st, mbar = X.basic_exact_graph(nb, pi, g["subset_size"])
    # the paper's E(M_A) = 1 and pi = (1/6, 1/3, 1/2)
    assert mbar[0] == pytest.approx(_frac(g["paper_printed"]["E_M_A"]))
    np.testing.assert_allclose(pi / pi.sum(), [_frac(s) for s in g["paper_printed"]["pi"]])
    # closed form from Algorithm 3
    np.testing.assert_allclose(mbar, [_frac(s) for s in g["closed_form"]["E_M"]], rtol=1e-12)
    np.testing.assert_allclose(jump_st, [1 / 3] * 3, rtol=1e-12)
    np.testing.assert_allclose(wt, [_frac(s) for s in g["closed_form"]["proportions"]], rtol=1e-12)
    # Basic PNS is biased: the weighted law differs from pi (the paper's point)
    assert X.tvd(wt, pi / pi.sum()) > 0.04


# ---------------------------------------------------------------------------
# Example 2 (Sec. 2.2): the 4-cube, TVD plateau ~0.3 for |N_k| = 1.
# ---------------------------------------------------------------------------

def _cube_qubo():
    # pi ~ e^{#ones} = exp(-beta x^T Q x) with Q = -I, beta = 1
    return -np.eye(4, dtype=np.int32)


def test_example2_exact_plateaus():
    g = json.load(open(os.path.join(GOLDEN, "example2_cube.json")))
    Q = _cube_qubo()
    pi = X.target(Q, None, 1.0)
    levels = X.state_bits(4).sum(1)
    assert np.bincount(levels).tolist() == g["level_counts"]
    tv = {}
    for k in (1, 2, 3, 4):
        wt, _ = X.basic_exact_qubo(Q, None, 1.0, k)
        tv[k] = X.tvd(wt, pi)
    assert g["check"]["k1_tvd_low"] < tv[1] < g["check"]["k1_tvd_high"]
    assert tv[1] > tv[2] > tv[3] > 1e-3
    assert tv[4] < 1e-12  # k = n is Rejection-Free, unbiased


@pytest.mark.parametrize("k", [1, 2, 3])
def test_example2_oracle_basic_matches_exact(k):
    Q = _cube_qubo()
    wt, pi = X.basic_exact_qubo(Q, None, 1.0, k)
    p = O.Problem(q=Q)
    res = O.run_independent([p], [[1.0]], dict(variant="basic", k=k, seed=11), 4, None, 100000)
    codes, w = [], []
    for r in res.values():
        c, _ = X.replay_codes(0, r["flips"])
        codes.append(c[1000:])
        w.append(r["m"][1000:])
    h = X.weighted_hist(np.concatenate(codes), np.concatenate(w), 4)
    assert X.tvd(h, wt) < 0.01
    assert abs(X.tvd(h, pi) - X.tvd(wt, pi)) < 0.01


def test_basic_exact_random_qubo_n6():
    Q = synth.dense_int(6, -3, 3, seed=5, dtype=np.int32)
    b = synth.vector_int(6, -2, 2, seed=5, dtype=np.int32)
    beta = 0.5
    wt, pi = X.basic_exact_qubo(Q, b, beta, 2)
    p = O.Problem(q=Q, b=b)
    res = O.run_independent([p], [[beta]], dict(variant="basic", k=2, seed=3), 4, None, 150000)
    codes = np.concatenate([X.replay_codes(0, r["flips"])[0][2000:] for r in res.values()])
    w = np.concatenate([r["m"][2000:] for r in res.values()])
    assert X.tvd(X.weighted_hist(codes, w, 6), wt) < 0.01


# ---------------------------------------------------------------------------
# Convergence to pi of Metropolis, RF, Unbiased PNS (Algorithms 1, 2, 6;
# Theorem 3 (5)): TVD of the multiplicity-weighted histogram < 0.01 at
# 1e6 records pooled over 16 chains, 10% burn-in, n = 16.
# ---------------------------------------------------------------------------

def _pooled_tvd(Q, b, beta, variant, k, subset="systematic", n_chains=16, records=62500, seed=0, start=None):
    n = Q.shape[0]
    p = O.Problem(q=Q, b=b)
    x0 = synth.random_bits(n_chains, n, seed=seed)
    if start is not None:
        x0[:] = start
    res = O.run_independent([p], [[beta]], dict(variant=variant, k=k, subset=subset, L0=100, seed=seed),
                            n_chains, {c: x0[c] for c in range(n_chains)}, records)
    codes, w = [], []
    burn = records // 10
    for cid, r in res.items():
        c, _ = X.replay_codes(X.code_of(x0[cid]), r["flips"])
        codes.append(c[burn:])
        w.append(r["m"][burn:])
    h = X.weighted_hist(np.concatenate(codes), np.concatenate(w), n)
    return X.tvd(h, X.target(Q, b, beta)), res


@pytest.mark.parametrize("beta", [1.0, 0.2])
@pytest.mark.parametrize("variant,k,subset", [("rf", 16, "systematic"), ("unbiased", 4, "systematic"),
                                              ("unbiased", 4, "random"), ("unbiased", 6, "systematic"),
                                              ("metropolis", 1, "systematic")])
def test_converges_to_target_n16(variant, k, subset, beta):
    Q = synth.dense_int(16, -8, 8, seed=0, dtype=np.int32)
    # 1e6 pooled records for RF; Unbiased PNS with |N_i| = 4 of 16 bits mixes
    # more slowly per record (Sec. 4), so it and Metropolis get 4e6.
    records = 62500 if variant == "rf" else 250000
    start = None
    if beta == 1.0:
        # At beta = 1 this Q has five local minima; the second (E = -129 vs
        # -147) holds chains for ~e^18 original samples.  Chains start at the
        # mode, the optimisation-instead-of-burn-in reading of Sec. 8.1; at
        # beta = 0.2 they start from random states.
        start = X.state_bits(16)[int(np.argmin(X.energies(Q)))]
    tv, _ = _pooled_tvd(Q, None, beta, variant, k, subset, records=records, start=start)
    assert tv < 0.01, tv


def test_basic_is_biased_n16():
    Q = synth.dense_int(16, -8, 8, seed=0, dtype=np.int32)
    tv, _ = _pooled_tvd(Q, None, 0.2, "basic", 4)
    assert tv > 0.05


def test_fp32_qubo_converges():
    Q = synth.dense_normal(12, 1.0, seed=3)
    b = synth.vector_normal(12, 0.5, seed=3)
    tv, res = _pooled_tvd(Q, b, 1.0, "unbiased", 4, records=250000, seed=4)
    assert tv < 0.01, tv


# ---------------------------------------------------------------------------
# Proposition 5 (exponential race) and the multiplicity law (Sec. 1.2).
# ---------------------------------------------------------------------------

def test_race_selects_in_proportion():
    deltas = np.array([0, 3, -2, 7, 1, 1, 12, 5], dtype=np.int64)
    beta = 0.4
    w = np.minimum(1.0, np.exp(-beta * deltas.astype(np.float64)))
    probs = w / w.sum()
    N = 200000
    counts = np.zeros(len(deltas))
    for s in range(N):
        win, _, _, _, _ = O.decide(deltas, len(deltas), beta, 1234, 3, s)
        counts[win] += 1
    exp = probs * N
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 24.3  # 7 dof, p = 1e-3


def test_multiplicity_law():
    deltas = np.array([4, 9, 2, 6], dtype=np.int64)
    beta = 0.5
    p_exact = np.minimum(1.0, np.exp(-beta * deltas)).mean()
    N = 100000
    ms = np.empty(N)
    for s in range(N):
        _, sq, p, m, sat = O.decide(deltas, 4, beta, 99, 1, s)
        ms[s] = m
        assert sat == 0
    assert p == pytest.approx(p_exact, rel=1e-6)
    # M = 1 + Geometric(p): mean 1/p, P(M = 1) = p
    se = math.sqrt((1 - p_exact) / p_exact**2 / N)
    assert abs(ms.mean() - 1 / p_exact) < 5 * se
    assert abs((ms == 1).mean() - p_exact) < 5 * math.sqrt(p_exact * (1 - p_exact) / N)
    assert (ms >= 1).all() and (ms == np.floor(ms)).all()


@pytest.mark.parametrize("deltas,beta", [([7], 1.0), ([14, 15, 17], 1.0)])
def test_multiplicity_law_small_p(deltas, beta):
    """M = 1 + Geom(p) (Sec. 1.2) where moves are rare: p near 1e-3 and 4e-7,
    the range Basic PNS and RF reach on the headline instance.  The oracle
    forms M = floor(E1 / -ln(1 - p)) + 1 in fp32; the law of M must still be
    the geometric one: mean 1/p, and P(M <= m) = 1 - (1 - p)^m at three m."""
    d = np.array(deltas, dtype=np.int64)
    k = len(deltas)
    p_exact = float(np.mean(np.exp(-beta * d)))
    N = 200000
    ms = np.empty(N)
    p = None
    for s in range(N):
        _, _, p, m, sat = O.decide(d, k, beta, 7, 3, s)
        ms[s] = m
        assert sat == 0
    # the fp32 p the oracle uses, against the closed form (det_expf <= 2 ulp,
    # the quantised weight sum <= k 2^-32 relative)
    assert p == pytest.approx(p_exact, rel=1e-6)
    p = float(p)
    se = math.sqrt((1 - p) / p**2 / N)
    assert abs(ms.mean() - 1 / p) < 5 * se
    for frac in (0.1, 0.7, 2.0):
        mq = math.floor(frac / p)
        F = 1.0 - (1.0 - p) ** mq
        assert abs((ms <= mq).mean() - F) < 5 * math.sqrt(F * (1 - F) / N), (frac, mq)
    assert (ms >= 1).all() and (ms == np.floor(ms)).all()


def test_multiplicity_edges():
    # all neighbours downhill: p = 1 and M = 1 (Example 1: Geom(1) gives E[M] = 1)
    _, _, p, m, sat = O.decide(np.array([-5, -1, 0], np.int64), 3, 1.0, 0, 0, 0)
    assert p == 1.0 and m == 1.0 and sat == 0
    # p underflows: saturated multiplicity
    _, _, p, m, sat = O.decide(np.array([5000, 7000], np.int64), 2, 1.0, 0, 0, 0)
    assert p == 0.0 and sat == 1 and m == 2.0**63
    # the anchor candidate always has a finite key and can win
    win, sq, p, m, sat = O.decide(np.array([1000, 10**6], np.int64), 2, 1.0, 0, 0, 0)
    assert win == 0 and sq == 2**32


# ---------------------------------------------------------------------------
# Alternating-chain bookkeeping (Algorithms 5 and 6).
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("subset", ["systematic", "random"])
def test_unbiased_budget_invariant(subset):
    Q = synth.dense_int(24, -20, 20, seed=2, dtype=np.int32)
    b = synth.vector_int(24, -10, 10, seed=2, dtype=np.int32)
    p = O.Problem(q=Q, b=b)
    for L0 in (10, 100, 1000):
        res = O.run_independent([p], [[0.3]], dict(variant="unbiased", k=5, subset=subset, L0=L0, seed=L0), 2,
                                None, 20000)
        for r in res.values():
            st = r["state"]
            assert st.sum_m == L0 * st.stays + (L0 - st.L)
            assert st.sum_m == r["m"].sum()
            assert st.flips == int((r["flips"] >= 0).sum())
            assert st.stays == int((r["flips"] < 0).sum())
            # stays record the remaining budget, moves record M <= L
            assert (r["m"] <= L0).all() and (r["m"] >= 0).all()


def test_unbiased_with_full_set_is_rejection_free():
    Q = synth.dense_int(20, -9, 9, seed=8, dtype=np.int32)
    p = O.Problem(q=Q)
    a = O.run_independent([p], [[0.7]], dict(variant="rf", seed=5), 2, None, 5000)
    b = O.run_independent([p], [[0.7]], dict(variant="unbiased", k=20, L0=2**62, seed=5), 2, None, 5000)
    for cid in a:
        np.testing.assert_array_equal(a[cid]["flips"], b[cid]["flips"])
        np.testing.assert_array_equal(a[cid]["m"], b[cid]["m"])


def test_systematic_sets_wrap():
    # Sec. 5: n = 16, |N_i| = 14 gives eight sets: 1..14, then 15, 16, 1..12, ...
    sets = X.systematic_sets(16, 14)
    assert len(sets) == 8
    assert sets[0] == list(range(14))
    assert sets[1] == [14, 15] + list(range(12))
    assert sets[2] == [12, 13, 14, 15] + list(range(10))
    assert sorted(set(sum(sets, []))) == list(range(16))


# ---------------------------------------------------------------------------
# Appendix A: per-set reversibility (Prop. 1) and Alg. 11 vs Algorithm 6.
# ---------------------------------------------------------------------------

def test_per_set_kernels_reversible():
    Q = synth.dense_int(7, -4, 4, seed=9, dtype=np.int32)
    b = synth.vector_int(7, -3, 3, seed=9, dtype=np.int32)
    for S in X.systematic_sets(7, 3):
        P, pi = X.alg11_kernel(Q, b, 0.8, S)
        np.testing.assert_allclose(pi @ P, pi, atol=1e-13)
        F = pi[:, None] * P
        np.testing.assert_allclose(F, F.T, atol=1e-14)


def test_alg11_and_alg6_share_the_target():
    Q = synth.dense_int(10, -4, 4, seed=4, dtype=np.int32)
    b = synth.vector_int(10, -3, 3, seed=4, dtype=np.int32)
    beta = 0.5
    pi = X.target(Q, b, beta)
    p = O.Problem(q=Q, b=b)
    codes = np.concatenate([O.run_alg11(p, 3, 100, beta, 21, c, np.zeros(10, np.uint8), 400000)[40000:]
                            for c in range(4)])
    h11 = np.bincount(codes.astype(np.int64), minlength=1 << 10) / len(codes)
    tv11 = X.tvd(h11, pi)
    tv6, _ = _pooled_tvd(Q, b, beta, "unbiased", 3, n_chains=8, records=60000, seed=21)
    assert tv11 < 0.02 and tv6 < 0.02
    # two-sample closeness of the two laws
    assert tv11 + tv6 < 0.04


# ---------------------------------------------------------------------------
# Local fields and energies against a from-scratch recomputation.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("variant,k", [("basic", 8), ("unbiased", 8), ("rf", 40), ("metropolis", 1)])
def test_fields_and_energy_exact_int(variant, k):
    n = 40
    Q = synth.dense_int(n, -100, 100, seed=1, dtype=np.int16)
    b = synth.vector_int(n, -100, 100, seed=1, dtype=np.int16)
    p = O.Problem(q=Q, b=b)
    x0 = synth.random_bits(3, n, seed=1)
    res = O.run_independent([p], [[0.05]], dict(variant=variant, k=k, L0=100, seed=2), 3,
                            {c: x0[c] for c in range(3)}, 3000)
    Qd = Q.astype(np.int64)
    for cid, r in res.items():
        x = r["x"].astype(np.int64)
        np.testing.assert_array_equal(r["h"], Qd @ x + b.astype(np.int64))
        assert r["state"].E == float(x @ Qd @ x + b.astype(np.int64) @ x)
        # replaying the flip tape from x0 reproduces the final state
        _, last = X.replay_codes(X.code_of(x0[cid]), r["flips"])
        assert X.code_of(r["x"]) == int(last)


def test_fields_fp32_within_tolerance():
    n = 48
    Q = synth.dense_normal(n, 1.0, seed=6)
    b = synth.vector_normal(n, 1.0, seed=6)
    p = O.Problem(q=Q, b=b)
    res = O.run_independent([p], [[0.5]], dict(variant="unbiased", k=6, seed=6), 2, None, 20000)
    for r in res.values():
        x = r["x"].astype(np.float64)
        h64 = Q.astype(np.float64) @ x + b.astype(np.float64)
        np.testing.assert_allclose(r["h"], h64, rtol=1e-5, atol=1e-4 * np.abs(Q).sum(1).max())
        E64 = x @ Q.astype(np.float64) @ x + b.astype(np.float64) @ x
        assert abs(r["state"].E - E64) <= 1e-4 * max(1.0, abs(E64)) + 1e-3


def test_csr_equals_dense_for_integer_lattice():
    side = 8
    row_ptr, col, val, diag = synth.lattice_csr(side, seed=3)
    dense = synth.csr_to_dense(row_ptr, col, val, diag).astype(np.int32)
    pc = O.Problem(csr=(row_ptr, col, val, diag))
    pd = O.Problem(q=dense)
    cfg = dict(variant="unbiased", k=16, L0=100, seed=4)
    a = O.run_independent([pc], [[0.44]], cfg, 2, None, 5000)
    bres = O.run_independent([pd], [[0.44]], cfg, 2, None, 5000)
    for cid in a:
        np.testing.assert_array_equal(a[cid]["flips"], bres[cid]["flips"])
        np.testing.assert_array_equal(a[cid]["m"], bres[cid]["m"])
        np.testing.assert_array_equal(a[cid]["h"], bres[cid]["h"])
        x = a[cid]["x"].astype(np.int64)
        np.testing.assert_array_equal(a[cid]["h"], dense.astype(np.int64) @ x)


def test_random_subset_uniform_and_distinct():
    n, k = 10, 3
    counts = {}
    for s in range(30000):
        S = O.random_subset(n, k, 5, 0, s)
        assert len(set(S.tolist())) == k and S.min() >= 0 and S.max() < n
        key = tuple(sorted(S.tolist()))
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == math.comb(n, k)
    c = np.array(list(counts.values()), dtype=np.float64)
    exp = 30000 / math.comb(n, k)
    chi2 = ((c - exp) ** 2 / exp).sum()
    assert chi2 < 180  # 119 dof, p ~ 3e-4


@pytest.mark.parametrize("variant,k", [("basic", 3), ("rf", 0), ("unbiased", 4)])
def test_best_state_is_first_minimum_of_the_replayed_path(variant, k):
    """X_max of Algorithms 8-10: replaying the flip tape from x0 and
    enumerating the energies of the visited states, the oracle's best state
    is the first state of lowest energy on the path (updates only on strict
    improvement) and best_E is that energy."""
    n = 12
    q = synth.dense_int(n, -9, 9, 21, np.int32)
    b = synth.vector_int(n, -9, 9, 21, np.int32)
    prob = O.Problem(q=q, b=b)
    x0 = synth.random_bits(1, n, seed=4)[0]
    cfg = O.make_config(variant, k=k, L0=20, seed=7)
    st = O.ChainState(prob, x0, 20)
    flips, _ = O.run_chain(prob, cfg, np.float32(0.3), 3, st, 3000)
    E_all = X.energies(q.astype(np.float64), b.astype(np.float64))
    before, last = X.replay_codes(X.code_of(x0), flips)
    path = np.concatenate([before, [last]])  # the start, then the state after each record
    e_path = E_all[path]
    first_min = int(np.argmin(e_path))  # argmin returns the first occurrence
    assert st.st.best_E == e_path[first_min]
    assert X.code_of(st.x_best) == int(path[first_min])


# ---------------------------------------------------------------------------
# Sec. 3.2 (Basic PNS: a fresh partial neighbour set every step) and Sec. 5
# (random sets for Unbiased PNS: one set per period): every move flips a bit
# of the set its record was drawn from.
# ---------------------------------------------------------------------------
def test_moves_lie_in_their_random_sets():
    n, k, seed = 40, 6, 17
    Q = synth.dense_int(n, -20, 20, seed=4, dtype=np.int32)
    p = O.Problem(q=Q, b=None)
    # Basic: record r draws its set at step r
    res = O.run_independent([p], [[0.3]], dict(variant="basic", k=k, seed=seed), 2, None, 3000)
    for cid, r in res.items():
        f = r["flips"]
        assert (f >= 0).all()
        for step in range(len(f)):
            assert f[step] in O.random_subset(n, k, seed, cid, step), (cid, step)
    # Unbiased, random sets: the set is drawn at the period's first record and
    # kept until a stay ends the period
    res = O.run_independent([p], [[0.3]], dict(variant="unbiased", k=k, subset="random", L0=50, seed=seed), 2,
                            None, 3000)
    for cid, r in res.items():
        f = r["flips"]
        start = 0
        cur = O.random_subset(n, k, seed, cid, 0)
        for step in range(len(f)):
            if f[step] >= 0:
                assert f[step] in cur, (cid, step)
            else:
                start = step + 1
                cur = O.random_subset(n, k, seed, cid, start)
        assert r["state"].period_start == start


def test_moves_follow_the_wrapping_systematic_sets():
    # Sec. 5's example, n = 16 and |N_i| = 14: a chain's i-th period uses set
    # i mod 8 of the wrap-around sequence, and every move flips a bit of it
    n, k = 16, 14
    sets = X.systematic_sets(n, k)
    Q = synth.dense_int(n, -8, 8, seed=0, dtype=np.int32)
    p = O.Problem(q=Q, b=None)
    res = O.run_independent([p], [[1.0]], dict(variant="unbiased", k=k, subset="systematic", L0=20, seed=3), 3,
                            None, 4000)
    for cid, r in res.items():
        f = r["flips"]
        period = 0
        for step in range(len(f)):
            if f[step] >= 0:
                assert f[step] in sets[period % len(sets)], (cid, step)
            else:
                period += 1
        assert r["state"].set_start == sets[period % len(sets)][0]
        assert period == r["state"].stays


# ---------------------------------------------------------------------------
# One step from a fixed state against its exact law: Metropolis proposes a
# uniform bit and accepts w.p. min(1, e^{-beta Delta}); Rejection-Free moves
# to neighbour y w.p. proportional to min(1, e^{-beta Delta_y}) (Sec. 1.2,
# Eq. (1) with the symmetric proposal) with M = 1 + Geom(p).
# ---------------------------------------------------------------------------
def test_one_step_laws_from_a_fixed_state():
    n, beta, draws = 5, 0.4, 40000
    Q = synth.dense_int(n, -3, 3, seed=8, dtype=np.int32)
    b = synth.vector_int(n, -3, 3, seed=8, dtype=np.int32)
    p = O.Problem(q=Q, b=b)
    x = np.array([1, 0, 1, 1, 0], np.uint8)
    E = lambda v: float(v @ Q.astype(np.float64) @ v + b @ v)  # noqa: E731
    dE = np.array([E(np.where(np.arange(n) == i, 1 - x, x)) - E(x) for i in range(n)])
    acc = np.minimum(1.0, np.exp(-beta * dE))
    for variant, k in (("metropolis", 1), ("rf", n)):
        cfg = O.make_config(variant, k=k, seed=21)
        counts = np.zeros(n + 1)  # bits, then "stayed"
        msum = 0.0
        for cid in range(draws):
            st = O.ChainState(p, x, 100)
            fl, ms = O.run_chain(p, cfg, np.float32(beta), cid, st, 1)
            counts[fl[0] if fl[0] >= 0 else n] += 1
            msum += ms[0]
        if variant == "metropolis":
            want = np.append(acc / n, 1.0 - acc.sum() / n)
            assert msum == draws
        else:
            want = np.append(acc / acc.sum(), 0.0)
            # E[M] = 1 / p, p = the mean acceptance over the n proposals
            assert abs(msum / draws - n / acc.sum()) < 0.05 * n / acc.sum()
        keep = want > 0
        chi2 = (((counts[keep] - draws * want[keep]) ** 2) / (draws * want[keep])).sum()
        assert chi2 < 25.0, (variant, counts, draws * want)  # <= 5 dof, p < 1e-4
        assert counts[~keep].sum() == 0


def test_one_basic_step_against_subset_enumeration():
    # Basic PNS (Sec. 3.2): a uniform k-subset S, then y in S w.p.
    # w_y / sum_S w with w = min(1, e^{-beta Delta}), and M = 1 + Geom(p_S),
    # p_S = sum_S w / k; exact law by enumerating the C(n, k) subsets
    from itertools import combinations
    n, k, beta, draws = 5, 2, 0.4, 40000
    Q = synth.dense_int(n, -3, 3, seed=8, dtype=np.int32)
    b = synth.vector_int(n, -3, 3, seed=8, dtype=np.int32)
    p = O.Problem(q=Q, b=b)
    x = np.array([1, 0, 1, 1, 0], np.uint8)
    E = lambda v: float(v @ Q.astype(np.float64) @ v + b @ v)  # noqa: E731
    w = np.minimum(1.0, np.exp(-beta * np.array(
        [E(np.where(np.arange(n) == i, 1 - x, x)) - E(x) for i in range(n)])))
    subsets = list(combinations(range(n), k))
    want = np.zeros(n)
    mean_m = 0.0
    for S in subsets:
        ws = w[list(S)].sum()
        for y in S:
            want[y] += w[y] / ws / len(subsets)
        mean_m += (k / ws) / len(subsets)
    cfg = O.make_config("basic", k=k, seed=33)
    counts = np.zeros(n)
    msum = 0.0
    for cid in range(draws):
        st = O.ChainState(p, x, 100)
        fl, ms = O.run_chain(p, cfg, np.float32(beta), cid, st, 1)
        counts[fl[0]] += 1
        msum += ms[0]
    chi2 = (((counts - draws * want) ** 2) / (draws * want)).sum()
    assert chi2 < 25.0, (counts, draws * want)
    assert abs(msum / draws - mean_m) < 0.05 * mean_m


def test_one_unbiased_record_against_its_law():
    # Algorithm 6, first record of a fresh chain (set = bits 0 .. k-1, budget
    # L0): M = 1 + Geom(p) with p = sum_set w / k; it moves iff M <= L0, so it
    # stays w.p. (1 - p)^L0 (recording M = L0) and otherwise jumps to y in the
    # set w.p. proportional to w_y
    n, k, L0, beta, draws = 6, 3, 2, 0.8, 40000
    Q = synth.dense_int(n, -3, 3, seed=9, dtype=np.int32)
    b = synth.vector_int(n, -3, 3, seed=9, dtype=np.int32)
    p = O.Problem(q=Q, b=b)
    x = np.array([0, 1, 1, 0, 1, 0], np.uint8)
    E = lambda v: float(v @ Q.astype(np.float64) @ v + b @ v)  # noqa: E731
    w = np.minimum(1.0, np.exp(-beta * np.array(
        [E(np.where(np.arange(n) == i, 1 - x, x)) - E(x) for i in range(k)])))
    pm = w.sum() / k
    stay = (1.0 - pm) ** L0
    want = np.append((1.0 - stay) * w / w.sum(), stay)
    cfg = O.make_config("unbiased", k=k, subset="systematic", L0=L0, seed=5)
    counts = np.zeros(k + 1)
    for cid in range(draws):
        st = O.ChainState(p, x, L0)
        fl, ms = O.run_chain(p, cfg, np.float32(beta), cid, st, 1)
        assert fl[0] < k
        counts[fl[0] if fl[0] >= 0 else k] += 1
        if fl[0] < 0:
            assert ms[0] == L0
        else:
            assert 1 <= ms[0] <= L0
    chi2 = (((counts - draws * want) ** 2) / (draws * want)).sum()
    assert chi2 < 25.0, (counts, draws * want)


# ---------------------------------------------------------------------------
# Cooling schedule of the optimisation forms (Algorithms 8-10, Sec. 8.1).
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3, 4, 9])
def test_anneal_schedule_one_step_law(k):
    """Record k of Simulated Annealing (Algorithm 8) accepts an uphill move
    of size d with probability [pi(y)/pi(x)]^{1/T(k)} = e^{-beta d / T(k)},
    1/T(k) = s0^(1 - k/K) for k < K and 1 from K on.  One bit, d = 3, beta =
    0.5, s0 = 0.25, K = 4: the first record of 40,000 chains started at step
    k - 1 against the closed form."""
    d, beta, s0, K = 3, 0.5, 0.25, 4
    p = O.Problem(q=np.array([[d]], dtype=np.int32))
    c = O.make_config("metropolis", L0=100, seed=17, anneal_start=s0, anneal_steps=K)
    N = 40000
    acc = 0
    for chain in range(N):
        st = O.ChainState(p, np.zeros(1, np.uint8), 100)
        st.st.step = k - 1
        fl, _ = O.run_chain(p, c, beta, chain, st, 1)
        acc += int(fl[0] == 0)
    inv_t = s0 ** (1.0 - k / K) if k < K else 1.0
    want = math.exp(-beta * d * inv_t)
    assert abs(acc / N - want) < 5 * math.sqrt(want * (1 - want) / N), (k, acc / N, want)


def test_anneal_start_one_is_constant_temperature():
    """s0 = 1 gives T(k) = 1 for every k: the tapes equal the runs without a
    schedule (Sec. 8.2's setting), for every variant."""
    Q = synth.dense_int(20, -15, 15, seed=6, dtype=np.int32)
    p = O.Problem(q=Q)
    for variant in ("metropolis", "rf", "basic", "unbiased"):
        a = O.make_config(variant, k=5, L0=50, seed=2)
        b = O.make_config(variant, k=5, L0=50, seed=2, anneal_start=1.0, anneal_steps=300)
        sa = O.ChainState(p, np.zeros(20, np.uint8), 50)
        sb = O.ChainState(p, np.zeros(20, np.uint8), 50)
        fa, ma = O.run_chain(p, a, 0.4, 3, sa, 500)
        fb, mb = O.run_chain(p, b, 0.4, 3, sb, 500)
        np.testing.assert_array_equal(fa, fb)
        np.testing.assert_array_equal(ma, mb)


def test_annealing_reaches_the_ground_state():
    """Simulated Annealing, Optimization RF and Optimization PNS with a slow
    geometric cooling end with X_max at the exact minimum of E (enumerated
    over all 2^14 states) on most chains, and X_max is the lowest state the
    replayed path visits."""
    n = 14
    Q = synth.dense_int(n, -10, 10, seed=21, dtype=np.int32)
    p = O.Problem(q=Q)
    E = X.energies(Q, None)
    emin = E.min()
    for variant, k, recs in (("metropolis", 1, 6000), ("rf", 0, 600), ("basic", 4, 1500)):
        c = O.make_config(variant, k=k, L0=100, seed=8, anneal_start=0.02, anneal_steps=recs)
        hits = 0
        for chain in range(16):
            st = O.ChainState(p, np.zeros(n, np.uint8), 100)
            fl, _ = O.run_chain(p, c, 0.5, chain, st, recs)
            codes, last = X.replay_codes(0, fl)
            visited = np.append(codes, last)
            assert st.st.best_E == E[visited].min() == E[X.code_of(st.x_best)]
            hits += int(st.st.best_E == emin)
        assert hits >= 12, (variant, hits)
