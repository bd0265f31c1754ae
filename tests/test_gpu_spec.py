"""The speculative kernel (D warps evaluate D future records under the
assumption that the earlier ones stay) against the oracle and against the
one-record-at-a-time kernel: committed records must be bit-identical."""
import numpy as np
import pytest

from paper_2210_10513_gb300 import synth
from tests.gpu_helpers import assert_chain_equal, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def _problem(n, lo, hi, seed, dtype, beta):
    return dict(n=n, q=synth.dense_int(n, lo, hi, seed, dtype), b=synth.vector_int(n, lo, hi, seed, dtype),
                betas=[beta])


@pytest.mark.parametrize("depth", ["2", "4", "8", "16"])
@pytest.mark.parametrize("variant,k,subset", [("unbiased", 64, "systematic"), ("unbiased", 48, "random"),
                                              ("metropolis", 1, "systematic")])
def test_spec_matches_oracle(monkeypatch, depth, variant, k, subset):
    monkeypatch.setenv("PNS_SPEC_DEPTH", depth)
    monkeypatch.setenv("PNS_SWEEP", "0")  # (the set sweep has its own tests)
    p = _problem(1024, -100, 100, 7, np.int16, 0.05)
    cfg = dict(variant=variant, k=k, subset=subset, chains_per_replica=4, seed=13, L0=100)
    g = gpu_run([p], 3000, tape=True, **cfg)
    assert g["info"].warps_per_chain == int(depth)
    ref = oracle_run([p], 3000, list(range(4)), **cfg)
    for cid in range(4):
        assert_chain_equal(g, ref[cid], cid, 1024, 3000)


@pytest.mark.parametrize("beta", [0.02, 0.3, 3.0])
def test_spec_equals_sequential_kernel(monkeypatch, beta):
    p = dict(n=200, q=synth.dense_normal(200, 1.0, 4), b=synth.vector_normal(200, 1.0, 4), betas=[beta, 2 * beta])
    cfg = dict(variant="unbiased", k=13, chains_per_replica=5, seed=2, L0=50)
    monkeypatch.setenv("PNS_SPEC_DEPTH", "0")
    monkeypatch.setenv("PNS_SWEEP", "0")
    a = gpu_run([p], 2500, runs=2, tape=True, **cfg)
    monkeypatch.setenv("PNS_SPEC_DEPTH", "8")
    b = gpu_run([p], 2500, runs=2, tape=True, **cfg)
    assert b["info"].warps_per_chain == 8
    for x, y in zip(a["all"], b["all"]):
        np.testing.assert_array_equal(x["flips"], y["flips"])
        np.testing.assert_array_equal(x["m"], y["m"])
        np.testing.assert_array_equal(x["states"], y["states"])
        np.testing.assert_array_equal(x["stats"], y["stats"])
    np.testing.assert_array_equal(a["fields"], b["fields"])


def test_spec_odd_run_lengths(monkeypatch):
    # run lengths that are not multiples of the depth end mid-round
    monkeypatch.setenv("PNS_SPEC_DEPTH", "16")
    p = _problem(96, -20, 20, 3, np.int32, 0.2)
    cfg = dict(variant="unbiased", k=7, chains_per_replica=3, seed=5, L0=30)
    g = gpu_run([p], 37, runs=3, tape=True, **cfg)
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
