"""The set-sweep kernel (every systematic set of the current state evaluated
once, up to 32 D records decided at once) against the oracle and against the
speculative kernel: committed records must be bit-identical."""
import numpy as np
import pytest

from paper_2210_10513_gb300 import synth
from tests.gpu_helpers import assert_chain_equal, gpu_run, oracle_run, to_dev

pytestmark = pytest.mark.gpu


def _problem(n, lo, hi, seed, dtype, beta):
    return dict(n=n, q=synth.dense_int(n, lo, hi, seed, dtype), b=synth.vector_int(n, lo, hi, seed, dtype),
                betas=[beta])


def _sweep(monkeypatch):
    monkeypatch.setenv("PNS_SPEC_DEPTH", "8")
    monkeypatch.setenv("PNS_SWEEP", "1")


@pytest.mark.parametrize("k", [128, 64, 32])
@pytest.mark.parametrize("beta", [0.05, 0.5, 0.005])
def test_sweep_matches_oracle_int16(monkeypatch, k, beta):
    # n = 1024: 8, 16 or 32 sets, so 1, 2 or 4 per warp; the weights come
    # from the tabled e^{-beta d} at beta 0.05 and 0.5 (1742 and 176 entries)
    # and from the exponential itself at beta 0.005 (over 8192 entries)
    _sweep(monkeypatch)
    p = _problem(1024, -100, 100, 7, np.int16, beta)
    cfg = dict(variant="unbiased", k=k, chains_per_replica=4, seed=13, L0=100)
    g = gpu_run([p], 3000, tape=True, **cfg)
    assert g["info"].set_sweep == 1 and g["info"].spec_depth == 8
    ref = oracle_run([p], 3000, list(range(4)), **cfg)
    for cid in range(4):
        assert_chain_equal(g, ref[cid], cid, 1024, 3000)


@pytest.mark.parametrize("n", [2048, 4096])
def test_sweep_four_positions_per_lane(monkeypatch, n):
    # k = 128: 16 or 32 sets (2 or 4 per warp), four positions per lane
    _sweep(monkeypatch)
    p = _problem(n, -30, 30, 9, np.int16, 0.05)
    cfg = dict(variant="unbiased", k=128, chains_per_replica=2, seed=17, L0=100)
    g = gpu_run([p], 1500, tape=True, **cfg)
    assert g["info"].set_sweep == 1
    ref = oracle_run([p], 1500, [0, 1], **cfg)
    for cid in range(2):
        assert_chain_equal(g, ref[cid], cid, n, 1500)


def test_sweep_sets_not_dividing_n(monkeypatch):
    # n = 96, k = 36: gcd 12, so 8 sets visited 3 apart; odd run lengths end
    # inside a batch of records
    _sweep(monkeypatch)
    p = _problem(96, -20, 20, 3, np.int32, 0.2)
    cfg = dict(variant="unbiased", k=36, chains_per_replica=3, seed=5, L0=30)
    g = gpu_run([p], 37, runs=3, tape=True, **cfg)
    assert g["info"].set_sweep == 1
    ref = oracle_run([p], 111, list(range(3)), **cfg)
    for cid in range(3):
        got = np.concatenate([r["flips"][cid] for r in g["all"]])
        np.testing.assert_array_equal(got, ref[cid]["flips"])
        gm = np.concatenate([r["m"][cid] for r in g["all"]])
        np.testing.assert_array_equal(gm, ref[cid]["m"])
    st = g["stats"]
    for cid in range(3):
        assert st["sum_m"][cid] == ref[cid]["state"].sum_m
        assert st["energy"][cid] == ref[cid]["state"].E
        assert st["set_start"][cid] == ref[cid]["state"].set_start


def test_sweep_uneven_instances(monkeypatch):
    # instances with 4, 8 and 32 sets in one launch (up to 4 sets per warp)
    _sweep(monkeypatch)
    probs = [_problem(64, -50, 50, 21, np.int32, 0.1), _problem(96, -50, 50, 22, np.int32, 0.3),
             _problem(256, -50, 50, 23, np.int32, 0.05)]
    ks = [16, 12, 8]
    for p, k in zip(probs, ks):
        p["k"] = k
    cfg = dict(variant="unbiased", k=1, chains_per_replica=2, seed=4, L0=100)
    g = gpu_run(probs, 2000, tape=True, **cfg)
    assert g["info"].set_sweep == 1
    refs = _oracle_multi(probs, ks, 2000, cfg)
    for cid, ref in refs.items():
        assert_chain_equal(g, ref, cid, probs[cid // 2]["n"], 2000)


def _oracle_multi(probs, ks, steps, cfg):
    from oracle import oracle as O
    oprobs = [O.Problem(q=p["q"], b=p["b"]) for p in probs]
    betas = [list(np.asarray(p["betas"], dtype=np.float32)) for p in probs]
    out = {}
    for i, k in enumerate(ks):
        okw = dict(variant="unbiased", k=k, subset="systematic", L0=cfg["L0"], seed=cfg["seed"])
        ids = [2 * i, 2 * i + 1]
        r = O.run_independent(oprobs, betas, okw, cfg["chains_per_replica"], None, steps, chain_ids=ids)
        out.update(r)
    return out


@pytest.mark.parametrize("beta", [0.02, 0.3, 3.0])
def test_sweep_equals_spec_kernel_fp32(monkeypatch, beta):
    # n = 208, k = 13: 16 sets; fp32 fields follow the same operation order
    p = dict(n=208, q=synth.dense_normal(208, 1.0, 4), b=synth.vector_normal(208, 1.0, 4), betas=[beta, 2 * beta])
    cfg = dict(variant="unbiased", k=13, chains_per_replica=5, seed=2, L0=50)
    monkeypatch.setenv("PNS_SPEC_DEPTH", "8")
    monkeypatch.setenv("PNS_SWEEP", "0")
    a = gpu_run([p], 2500, runs=2, tape=True, **cfg)
    assert a["info"].set_sweep == 0
    monkeypatch.setenv("PNS_SWEEP", "1")
    b = gpu_run([p], 2500, runs=2, tape=True, **cfg)
    assert b["info"].set_sweep == 1
    for x, y in zip(a["all"], b["all"]):
        np.testing.assert_array_equal(x["flips"], y["flips"])
        np.testing.assert_array_equal(x["m"], y["m"])
        np.testing.assert_array_equal(x["states"], y["states"])
        np.testing.assert_array_equal(x["stats"], y["stats"])
    np.testing.assert_array_equal(a["fields"], b["fields"])


def test_sweep_not_used_with_too_many_sets(monkeypatch):
    # n = 1000, k = 64: 125 sets, more than 4 per warp: the speculative kernel runs
    _sweep(monkeypatch)
    p = _problem(1000, -10, 10, 5, np.int32, 0.1)
    g = gpu_run([p], 200, tape=True, variant="unbiased", k=64, chains_per_replica=2, seed=1, L0=100)
    assert g["info"].set_sweep == 0 and g["info"].spec_depth == 8


@pytest.mark.parametrize("sweep", ["1", "0"])
def test_sweep_sample_tape(monkeypatch, sweep):
    # tape = 2: the state and energy each record starts from.  The bits are
    # the initial state (all zeros) with the earlier records' flips applied;
    # the energy is x^T Q x + b^T x of those bits, exact for integer Q.
    from paper_2210_10513_gb300 import pns
    monkeypatch.setenv("PNS_SPEC_DEPTH", "8" if sweep == "1" else "0")
    monkeypatch.setenv("PNS_SWEEP", sweep)
    n, recs = 256, 1500
    p = _problem(n, -40, 40, 12, np.int32, 0.1)
    s = pns.Sampler([dict(n=n, q=to_dev(p["q"]), b=to_dev(p["b"]), betas=p["betas"])], variant="unbiased", k=16,
                    chains_per_replica=3, L0=100, seed=21, tape=2)
    assert s.info.set_sweep == int(sweep)
    s.run(recs)
    out = s.read()
    xb, E = s.samples()
    s.close()
    q = p["q"].astype(np.int64)
    bvec = p["b"].astype(np.int64)
    for cid in range(3):
        x = np.zeros(n, dtype=np.int64)
        bits = synth.unpack_bits(xb[cid, :recs], n)
        for r in range(recs):
            np.testing.assert_array_equal(bits[r], x, err_msg="state at record %d, chain %d" % (r, cid))
            assert E[cid, r] == float(x @ q @ x + bvec @ x), (cid, r)
            j = out["flips"][cid, r]
            if j >= 0:
                x[j] ^= 1


@pytest.mark.parametrize("n,k,L0", [(64, 64, 100), (32, 1, 100), (40, 5, 1), (40, 5, 7)])
def test_sweep_edge_shapes(monkeypatch, n, k, L0):
    # one set (k = n), 32 one-bit sets (k = 1), and budgets of 1 and 7 original
    # samples (many records end a period on an exact budget)
    _sweep(monkeypatch)
    p = _problem(n, -20, 20, 31, np.int32, 0.3)
    cfg = dict(variant="unbiased", k=k, chains_per_replica=3, seed=8, L0=L0)
    g = gpu_run([p], 1200, tape=True, **cfg)
    assert g["info"].set_sweep == 1
    ref = oracle_run([p], 1200, list(range(3)), **cfg)
    for cid in range(3):
        assert_chain_equal(g, ref[cid], cid, n, 1200)


def test_sweep_weight_table_per_temperature(monkeypatch):
    # one integer instance at four temperatures without exchange: every chain
    # takes the weight table of its own beta (beta = 0.005 has none and uses
    # the exponential itself)
    _sweep(monkeypatch)
    p = _problem(256, -60, 60, 41, np.int32, 0.05)
    p["betas"] = [0.05, 0.1, 0.5, 0.005]
    cfg = dict(variant="unbiased", k=16, chains_per_replica=2, seed=6, L0=100)
    g = gpu_run([p], 1500, tape=True, **cfg)
    assert g["info"].set_sweep == 1
    ref = oracle_run([p], 1500, list(range(8)), **cfg)
    for cid in range(8):
        assert_chain_equal(g, ref[cid], cid, 256, 1500)
