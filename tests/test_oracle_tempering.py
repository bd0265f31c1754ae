"""Replica exchange on top of Unbiased PNS in the oracle.

Swaps act on the original (Algorithm 6) process at period ends, where every
replica has consumed exactly L0 original samples per period, so each
temperature's multiplicity-weighted histogram must still converge to its own
pi_beta (Sec. 4's parallel tempering, Theorem 3 (5) per temperature).
"""
import numpy as np

from oracle import exact as X
from oracle import oracle as O
from paper_2210_10513_gb300 import synth


def test_tempering_per_temperature_histograms():
    n = 8
    Q = synth.dense_int(n, -6, 6, seed=12, dtype=np.int32)
    b = synth.vector_int(n, -4, 4, seed=12, dtype=np.int32)
    betas = np.array([0.1, 0.25, 0.5, 1.0], dtype=np.float32)
    p = O.Problem(q=Q, b=b)
    R = len(betas)
    cfg = dict(variant="unbiased", k=3, L0=100, seed=31)
    rounds = 20000
    x0s = synth.random_bits(R, n, seed=12)
    # run round by round to know which temperature each slot held
    c = O.make_config(**cfg)
    states = [O.ChainState(p, x0s[s], c.L0, beta_idx=s) for s in range(R)]
    hist = np.zeros((R, 1 << n))
    accepted = 0
    for rnd in range(rounds):
        for s in range(R):
            st = states[s]
            code0 = X.code_of(st.x)
            bi = st.st.beta_idx
            fl, ms = O.run_chain(p, c, float(betas[bi]), s, st, c.L0 + 1, stop_after_periods=1)
            codes, last = X.replay_codes(code0, fl)
            assert int(last) == X.code_of(st.x)
            assert ms.sum() == c.L0  # exactly one period of original samples
            if rnd >= rounds // 10:
                hist[bi] += np.bincount(codes, weights=ms, minlength=1 << n)
        E = np.array([st.st.E for st in states])
        bidx = np.array([st.st.beta_idx for st in states], dtype=np.int32)
        new_idx, acc = O.swap_round(betas, E, bidx, c.seed, 0, rnd)
        assert sorted(new_idx.tolist()) == list(range(R))
        accepted += int(acc.sum()) // 2
        for s in range(R):
            states[s].st.beta_idx = int(new_idx[s])
    assert accepted > rounds // 10  # swaps do happen
    for r in range(R):
        pi = X.target(Q, b, float(betas[r]))
        h = hist[r] / hist[r].sum()
        assert X.tvd(h, pi) < 0.03, (r, X.tvd(h, pi))


def test_swap_rule_exact_acceptance():
    # a pair with (beta_a - beta_b)(E_a - E_b) = ln(0.25): accepted w.p. 1/4
    betas = np.array([0.5, 1.0], dtype=np.float32)
    dE = np.log(0.25) / (0.5 - 1.0)
    N = 40000
    hits = 0
    for rnd in range(0, 2 * N, 2):  # even rounds pair (0, 1)
        new, _ = O.swap_round(betas, np.array([dE, 0.0]), np.array([0, 1], np.int32), 3, 0, rnd)
        hits += int(new[0] == 1)
    assert abs(hits / N - 0.25) < 5 * np.sqrt(0.25 * 0.75 / N)
    # downhill in the swap ratio always accepts
    new, _ = O.swap_round(betas, np.array([-5.0, 0.0]), np.array([0, 1], np.int32), 3, 0, 0)
    assert new.tolist() == [1, 0]
    # odd rounds have no pair when R = 2
    new, _ = O.swap_round(betas, np.array([-5.0, 0.0]), np.array([0, 1], np.int32), 3, 0, 1)
    assert new.tolist() == [0, 1]


def test_metropolis_tempering_per_temperature_histograms():
    """Replica exchange on Metropolis chains (Algorithm 1, every record one
    original sample): with swaps every 10 records each temperature's record
    histogram still converges to its own pi_beta, and a chain's temperatures
    stay a permutation of the ladder."""
    n = 8
    Q = synth.dense_int(n, -6, 6, seed=14, dtype=np.int32)
    b = synth.vector_int(n, -4, 4, seed=14, dtype=np.int32)
    betas = np.array([0.1, 0.3, 0.6, 1.0], dtype=np.float32)
    p = O.Problem(q=Q, b=b)
    R = len(betas)
    c = O.make_config("metropolis", L0=100, seed=5)
    per_round, rounds = 10, 25000
    states = [O.ChainState(p, synth.random_bits(R, n, seed=14)[s], c.L0, beta_idx=s) for s in range(R)]
    hist = np.zeros((R, 1 << n))
    accepted = 0
    for rnd in range(rounds):
        for s in range(R):
            st = states[s]
            code0 = X.code_of(st.x)
            bi = st.st.beta_idx
            fl, ms = O.run_chain(p, c, float(betas[bi]), s, st, per_round)
            assert len(fl) == per_round and (ms == 1).all()
            codes, last = X.replay_codes(code0, fl)
            assert int(last) == X.code_of(st.x)
            if rnd >= rounds // 10:
                hist[bi] += np.bincount(codes, minlength=1 << n)
        E = np.array([st.st.E for st in states])
        bidx = np.array([st.st.beta_idx for st in states], dtype=np.int32)
        new_idx, acc = O.swap_round(betas, E, bidx, c.seed, 0, rnd)
        assert sorted(new_idx.tolist()) == list(range(R))
        accepted += int(acc.sum()) // 2
        for s in range(R):
            states[s].st.beta_idx = int(new_idx[s])
    assert accepted > rounds // 10
    for r in range(R):
        pi = X.target(Q, b, float(betas[r]))
        h = hist[r] / hist[r].sum()
        assert X.tvd(h, pi) < 0.03, (r, X.tvd(h, pi))


def test_run_tempering_metropolis_rounds_of_records():
    """run_tempering's Metropolis arm: `periods_per_round` records per slot per
    round, the same records as running the slots and swap rounds by hand."""
    n = 10
    Q = synth.dense_int(n, -9, 9, seed=3, dtype=np.int32)
    p = O.Problem(q=Q)
    betas = synth.geometric_ladder(0.2, 2.0, 3)
    res = O.run_tempering(p, betas, dict(variant="metropolis", L0=100, seed=9), group_id=4, chain_id0=12,
                          x0s=[np.zeros(n, np.uint8)] * 3, rounds=30, periods_per_round=7)
    c = O.make_config("metropolis", L0=100, seed=9)
    states = [O.ChainState(p, np.zeros(n, np.uint8), c.L0, beta_idx=s) for s in range(3)]
    tapes = [[] for _ in range(3)]
    for rnd in range(30):
        for s in range(3):
            fl, _ = O.run_chain(p, c, float(betas[states[s].st.beta_idx]), 12 + s, states[s], 7)
            tapes[s].append(fl)
        E = np.array([st.st.E for st in states])
        bidx = np.array([st.st.beta_idx for st in states], dtype=np.int32)
        new_idx, _ = O.swap_round(np.asarray(betas, np.float32), E, bidx, c.seed, 4, rnd)
        for s in range(3):
            states[s].st.beta_idx = int(new_idx[s])
    for s in range(3):
        np.testing.assert_array_equal(res[s]["flips"], np.concatenate(tapes[s]))
        assert res[s]["state"].beta_idx == states[s].st.beta_idx
        assert len(res[s]["flips"]) == 30 * 7
