"""The benchmark workloads at their full sizes, in the launch configuration the
bench times (CUDA graph, default mapping): sampled chains (always including
the one with the most moves, which sets the launch time) against the oracle
record by record, and every chain against properties that hold at any size:

* the jump chain's bookkeeping of Unbiased PNS (Algorithm 6): each period's
  multiplicities sum to L0, so sum M = L0 * stays + (L0 - L) from a fresh
  chain, and the systematic set moves on by k bits at every stay;
* every move flips a bit of the set its record lies on;
* the final state is the initial state (all zeros) with the tape's flips
  applied, and its energy x^T Q x + b^T x and fields Q x + b are the ones the
  chain carries: exactly for integer Q; for fp32 each field is within the
  rounding its F fp32 additions can accumulate (F 2^-24 max|h|, max|h| at most
  the largest row sum of |Q| plus max|b|), and the energy within
  1e-5 (F + 1) of that scale.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2210_10513_gb300 import synth
from tests.gpu_helpers import gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def _concat(g, key):
    """Per-chain records of every run of gpu_run(..., runs=R), in order."""
    rows = []
    for cid in range(len(g["stats"])):
        rows.append(np.concatenate([r[key][cid, :int(r["stats"]["tape_records"][cid])] for r in g["all"]]))
    return rows


def _check_unbiased_bookkeeping(g, ns, ks, L0, flips, ms):
    """Algorithm 6's budget and set sequence for chains started fresh
    (L = L0, set start 0, all-zero state)."""
    st = g["stats"]
    for cid in range(len(st)):
        n, k = int(ns[cid]), int(ks[cid])
        f, m = flips[cid], ms[cid]
        assert len(f) == st["steps"][cid]
        stay = f < 0
        assert int(stay.sum()) == st["stays"][cid] and int((~stay).sum()) == st["flips"][cid]
        # (a move spends M >= 1 of the budget; a stay records the budget
        # left, 0 after a move that spent it exactly)
        assert (m[~stay] >= 1).all() and (m >= 0).all() and (m <= L0).all(), cid
        assert st["sum_m"][cid] == float(m.sum())
        assert st["sum_m"][cid] == L0 * st["stays"][cid] + (L0 - st["budget_left"][cid]), cid
        assert st["set_start"][cid] == (int(st["stays"][cid]) * k) % n
        # the set of each record: k bits from (stays before it) * k mod n
        before = np.concatenate([[0], np.cumsum(stay)[:-1]]).astype(np.int64)
        start = (before * k) % n
        off = (f[~stay].astype(np.int64) - start[~stay]) % n
        assert (off < k).all(), cid


def _replayed_bits(flips, n):
    x = np.zeros(n, np.int64)
    moved = flips[flips >= 0]
    np.add.at(x, moved, 1)
    return x & 1


def test_headline_dense_int16_n1024_full_size():
    """Dense int16 n = 1024, 256 chains, Unbiased k = 64, beta = 0.05,
    L0 = 100, two launches of 10,000 records per chain (the set-sweep kernel,
    one chain per CTA)."""
    wl = synth.workload_dense_int1024(0)
    n, L0, k, recs = 1024, 100, 64, 10000
    p = dict(n=n, q=wl["q"], b=wl["b"], betas=[wl["beta"]])
    cfg = dict(variant="unbiased", k=k, chains_per_replica=256, L0=L0, seed=0, graph=True)
    g = gpu_run([p], recs, runs=2, tape=True, **cfg)
    assert g["info"].set_sweep == 1 and g["info"].ctas == 256
    flips, ms = _concat(g, "flips"), _concat(g, "m")
    _check_unbiased_bookkeeping(g, np.full(256, n), np.full(256, k), L0, flips, ms)
    st = g["stats"]
    q64 = wl["q"].astype(np.float64)
    b64 = wl["b"].astype(np.float64)
    bits = synth.unpack_bits(g["states"], n).astype(np.float64)
    for cid in range(256):
        np.testing.assert_array_equal(bits[cid], _replayed_bits(flips[cid], n), err_msg="chain %d" % cid)
    # (integer sums below 2^53: exact in fp64)
    E = np.einsum("ci,ci->c", bits @ q64, bits) + bits @ b64
    np.testing.assert_array_equal(st["energy"], E)
    np.testing.assert_array_equal(g["fields"][:, :n].astype(np.float64), bits @ q64 + b64)
    assert st["best_energy"].max() <= 0.0
    # sampled chains against the oracle, the busiest among them
    busiest = int(np.argmax(st["flips"]))
    ids = sorted({0, 1, 97, 128, 255, busiest})
    ref = oracle_run([p], 2 * recs, ids, **cfg)
    for cid in ids:
        np.testing.assert_array_equal(flips[cid], ref[cid]["flips"], err_msg="flip tape, chain %d" % cid)
        np.testing.assert_array_equal(ms[cid], ref[cid]["m"], err_msg="multiplicities, chain %d" % cid)
        rs = ref[cid]["state"]
        assert st["energy"][cid] == rs.E and st["sum_m"][cid] == rs.sum_m and st["best_energy"][cid] == rs.best_E
        np.testing.assert_array_equal(g["fields"][cid, :n].astype(np.int64), ref[cid]["h"].astype(np.int64))


def test_tempering_512_instances_full_size():
    """512 fp32 instances, n uniform in [128, 2048], 8 replicas each on the
    geometric ladder 0.1 .. 10, Unbiased k = n / 16, exchange every L0 = 100
    original samples; two launches of 1000 original samples per chain (the
    period-blocked kernel).  Three whole exchange groups (the smallest, the
    median and the largest instance) against the oracle."""
    probs, ladder = synth.workload_tempering(512, seed=0)
    R, L0 = len(ladder), 100
    plist = [dict(n=pr["n"], q=pr["q"], b=None, betas=ladder, k=max(1, pr["n"] // 16)) for pr in probs]
    g = gpu_run(plist, 1000, runs=2, tape=True, variant="unbiased", k=1, chains_per_replica=1, L0=L0,
                swap_interval=100, seed=0, graph=True)
    assert g["info"].period_blocked == 1
    st = g["stats"]
    ns = np.repeat([pr["n"] for pr in plist], R)
    ks = np.repeat([pr["k"] for pr in plist], R)
    flips, ms = _concat(g, "flips"), _concat(g, "m")
    # every chain: exactly 2000 original samples, whole periods only
    assert (st["sum_m"] == 2000.0).all() and (st["budget_left"] == L0).all()
    for cid in range(len(st)):
        n, k = int(ns[cid]), int(ks[cid])
        f = flips[cid]
        stay = f < 0
        before = np.concatenate([[0], np.cumsum(stay)[:-1]]).astype(np.int64)
        off = (f[~stay].astype(np.int64) - (before[~stay] * k) % n) % n
        assert (off < k).all(), cid
        assert st["set_start"][cid] == (int(stay.sum()) * k) % n
    # each group holds every temperature once
    bidx = st["beta_idx"].reshape(len(plist), R)
    assert (np.sort(bidx, axis=1) == np.arange(R)).all()
    assert st["swaps_accepted"].sum() > 0
    # fields and energies against fp64 recomputations from the final states
    for p, pr in enumerate(plist):
        n = pr["n"]
        q64 = pr["q"].astype(np.float64)
        sl = slice(p * R, (p + 1) * R)
        bits = synth.unpack_bits(g["states"][sl], n).astype(np.float64)
        for s in range(R):
            np.testing.assert_array_equal(bits[s], _replayed_bits(flips[p * R + s], n))
        h64 = bits @ q64
        scale = np.abs(q64).sum(1).max()
        F = st["flips"][sl].astype(np.float64) + 1
        err = np.abs(g["fields"][sl, :n] - h64).max(axis=1)
        assert (err <= F * 2.0 ** -24 * scale).all(), p
        E64 = np.einsum("ci,ci->c", h64, bits)
        assert (np.abs(st["energy"][sl] - E64) <= 1e-5 * scale * F).all(), p
    # whole groups against the oracle
    order = np.argsort([pr["n"] for pr in plist], kind="stable")
    for p in sorted({int(order[0]), int(order[len(order) // 2]), int(order[-1])}):
        pr = plist[p]
        res = O.run_tempering(O.Problem(q=pr["q"]), ladder, dict(variant="unbiased", k=pr["k"], L0=L0, seed=0),
                              group_id=p, chain_id0=p * R, x0s=[np.zeros(pr["n"], np.uint8)] * R, rounds=20,
                              periods_per_round=1)
        for s in range(R):
            cid = p * R + s
            np.testing.assert_array_equal(flips[cid], res[s]["flips"], err_msg="group %d slot %d" % (p, s))
            np.testing.assert_array_equal(ms[cid], res[s]["m"])
            assert st["beta_idx"][cid] == res[s]["state"].beta_idx
            assert st["swaps_accepted"][cid] == res[s]["state"].swaps_accepted
            assert st["energy"][cid] == res[s]["state"].E
            np.testing.assert_array_equal(g["fields"][cid, :pr["n"]].view(np.uint32),
                                          res[s]["h"].astype(np.float32).view(np.uint32))


def test_lattice_csr_n65536_full_size():
    """256 x 256 periodic lattice (n = 65536) as CSR, 64 chains for each beta
    in {0.2, 0.44, 1.0}, Unbiased k = 1024, one launch of 10,000 records per
    chain."""
    sp = pytest.importorskip("scipy.sparse")
    side, L0, k, recs = 256, 100, 1024, 10000
    n = side * side
    csr = synth.lattice_csr(side, seed=0)
    p = dict(n=n, csr=csr, b=None, betas=[0.2, 0.44, 1.0])
    cfg = dict(variant="unbiased", k=k, chains_per_replica=64, L0=L0, seed=0, graph=True)
    g = gpu_run([p], recs, tape=True, **cfg)
    st = g["stats"]
    C_ = len(st)
    assert C_ == 192
    flips, ms = _concat(g, "flips"), _concat(g, "m")
    _check_unbiased_bookkeeping(g, np.full(C_, n), np.full(C_, k), L0, flips, ms)
    row_ptr, col, val, diag = csr
    Q = sp.csr_matrix((val.astype(np.float64), col, row_ptr), shape=(n, n)) + sp.diags(diag.astype(np.float64))
    bits = synth.unpack_bits(g["states"], n).astype(np.float64)
    for cid in range(C_):
        np.testing.assert_array_equal(bits[cid], _replayed_bits(flips[cid], n), err_msg="chain %d" % cid)
    h = np.asarray((Q @ bits.T).T)
    np.testing.assert_array_equal(g["fields"][:, :n].astype(np.float64), h)
    np.testing.assert_array_equal(st["energy"], np.einsum("ci,ci->c", h, bits))
    busiest = int(np.argmax(st["flips"]))
    ids = sorted({0, 100, C_ - 1, busiest})
    ref = oracle_run([p], recs, ids, **cfg)
    for cid in ids:
        np.testing.assert_array_equal(flips[cid], ref[cid]["flips"], err_msg="flip tape, chain %d" % cid)
        np.testing.assert_array_equal(ms[cid], ref[cid]["m"], err_msg="multiplicities, chain %d" % cid)
        assert st["energy"][cid] == ref[cid]["state"].E


def test_fit_n64_8192_chains_full_size():
    """n = 64 fp32 QUBO, 8192 chains, Unbiased k = 16, beta = 1, one launch of
    10,000 records per chain with the sample tape (the forward of the
    differentiation workload)."""
    wl = synth.workload_fit(64, seed=0)
    n, L0, k, recs, C_ = 64, 100, 16, 10000, 8192
    p = dict(n=n, q=wl["q"], b=wl["b"], betas=[1.0])
    cfg = dict(variant="unbiased", k=k, chains_per_replica=C_, L0=L0, seed=0)
    g = gpu_run([p], recs, tape=2, **cfg)
    st = g["stats"]
    flips, ms = _concat(g, "flips"), _concat(g, "m")
    _check_unbiased_bookkeeping(g, np.full(C_, n), np.full(C_, k), L0, flips, ms)
    q64 = wl["q"].astype(np.float64)
    b64 = wl["b"].astype(np.float64)
    bits = synth.unpack_bits(g["states"], n).astype(np.float64)
    parity = np.zeros((C_, n), np.int64)
    for cid in range(C_):
        parity[cid] = _replayed_bits(flips[cid], n)
    np.testing.assert_array_equal(bits, parity)
    h64 = bits @ q64 + b64
    scale = np.abs(q64).sum(1).max() + np.abs(b64).max()
    F = st["flips"].astype(np.float64) + 1
    assert (np.abs(g["fields"][:, :n] - h64).max(axis=1) <= F * 2.0 ** -24 * scale).all()
    E64 = np.einsum("ci,ci->c", h64 - b64, bits) + bits @ b64
    assert (np.abs(st["energy"] - E64) <= 1e-5 * scale * F).all()
    busiest = int(np.argmax(st["flips"]))
    ids = sorted({0, 4095, C_ - 1, busiest})
    ref = oracle_run([p], recs, ids, **cfg)
    for cid in ids:
        np.testing.assert_array_equal(flips[cid], ref[cid]["flips"], err_msg="flip tape, chain %d" % cid)
        np.testing.assert_array_equal(ms[cid], ref[cid]["m"], err_msg="multiplicities, chain %d" % cid)
        assert st["energy"][cid] == ref[cid]["state"].E
        np.testing.assert_array_equal(g["fields"][cid, :n].view(np.uint32),
                                      ref[cid]["h"].astype(np.float32).view(np.uint32))


def test_headline_basic_full_size():
    """The headline instance with Basic PNS (a fresh random 64-subset every
    record, every record a move), 256 chains, one launch of 10,000 records."""
    wl = synth.workload_dense_int1024(0)
    n, k, recs = 1024, 64, 10000
    p = dict(n=n, q=wl["q"], b=wl["b"], betas=[wl["beta"]])
    cfg = dict(variant="basic", k=k, chains_per_replica=256, seed=0, graph=True)
    g = gpu_run([p], recs, tape=True, **cfg)
    st = g["stats"]
    flips, ms = _concat(g, "flips"), _concat(g, "m")
    q64 = wl["q"].astype(np.float64)
    b64 = wl["b"].astype(np.float64)
    bits = synth.unpack_bits(g["states"], n).astype(np.float64)
    for cid in range(256):
        assert len(flips[cid]) == recs and (flips[cid] >= 0).all() and (flips[cid] < n).all()
        # (M reaches 1e20 here: the chain's fp64 sum is taken in record order)
        assert (ms[cid] >= 1).all() and st["sum_m"][cid] == np.cumsum(ms[cid])[-1]
        np.testing.assert_array_equal(bits[cid], _replayed_bits(flips[cid], n), err_msg="chain %d" % cid)
    assert (st["flips"] == recs).all()
    E = np.einsum("ci,ci->c", bits @ q64, bits) + bits @ b64
    np.testing.assert_array_equal(st["energy"], E)
    np.testing.assert_array_equal(g["fields"][:, :n].astype(np.float64), bits @ q64 + b64)
    ids = [0, 129, 255]
    ref = oracle_run([p], recs, ids, **cfg)
    for cid in ids:
        np.testing.assert_array_equal(flips[cid], ref[cid]["flips"], err_msg="flip tape, chain %d" % cid)
        np.testing.assert_array_equal(ms[cid], ref[cid]["m"], err_msg="multiplicities, chain %d" % cid)
        assert st["energy"][cid] == ref[cid]["state"].E


def test_donuts_65536_chains_full_size():
    """Continuous Unbiased PNS (Algorithm 7) on the Donuts target: 65,536
    chains from the circle of radius 3, 50 neighbours, L0 = 1000, 4000 records
    per chain.  Every chain: sum M = L0 * stays + (L0 - L); sampled chains
    (with the one that moved most) equal the oracle bit for bit."""
    from paper_2210_10513_gb300 import pns
    chains, steps, L0 = 65536, 4000, 1000
    mu0, sigma = 9.0, 0.1
    c = 1.0 / (2 * sigma * sigma)
    rng = np.random.default_rng(0)
    ang = rng.uniform(0, 2 * np.pi, chains)
    x0 = np.stack([3 * np.cos(ang), 3 * np.sin(ang)], 1).astype(np.float32)
    st = pns.pns_donuts_run("unbiased", chains, steps, x0=x0, mu0=mu0, c=c, L0=L0, seed=100)
    assert (st["records"] == steps).all()
    stays = st["records"] - st["moves"]
    np.testing.assert_array_equal(st["weight"], L0 * stays + (L0 - st["budget_left"]).astype(np.float64))
    assert np.isfinite(st["sum_x4"]).all() and (st["sum_x2"] >= 0).all()
    busiest = int(np.argmax(st["moves"]))
    for ch in sorted({0, 12345, chains - 1, busiest}):
        r = O.donuts_chain("unbiased", ch, steps, tuple(x0[ch]), mu0=mu0, c=c, L0=L0, seed=100, npairs=25)
        for key in ("sum_x", "sum_x2", "sum_x4", "sum_pos", "x"):
            np.testing.assert_array_equal(st[ch][key], r[key], err_msg="%s chain %d" % (key, ch))
        for key in ("weight", "records", "moves", "budget_left", "period_start"):
            assert st[ch][key] == r[key], (key, ch)
