"""Replica exchange on the GPU vs the oracle: per-slot tapes, states,
temperatures and exchange counts agree exactly (uneven n, per-instance k)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2210_10513_gb300 import synth
from tests.gpu_helpers import gpu_run

pytestmark = pytest.mark.gpu


def _problems(ns, seed=0, integer=False):
    probs = []
    for i, n in enumerate(ns):
        if integer:
            q = synth.dense_int(n, -20, 20, seed + i, np.int32)
        else:
            q = synth.dense_normal(n, 1.0, seed + i)
        probs.append(dict(n=n, q=q, b=None, k=max(1, n // 16)))
    return probs


@pytest.mark.parametrize("integer,prefetch,blocked", [(False, "0", "1"), (True, "0", "1"), (False, "0", "0"),
                                                      (True, "0", "0"), (False, "1", "0")])
def test_unbiased_tempering_matches_oracle(monkeypatch, integer, prefetch, blocked):
    monkeypatch.setenv("PNS_PREFETCH", prefetch)
    monkeypatch.setenv("PNS_BLOCKED", blocked)
    ns = [130, 257, 96]
    betas = synth.geometric_ladder(0.1, 10.0, 4)
    probs = _problems(ns, seed=3, integer=integer)
    for p in probs:
        p["betas"] = betas
    L0, swap, steps = 100, 200, 3000
    g = gpu_run(probs, steps, tape=True, variant="unbiased", k=1, L0=L0, swap_interval=swap, chains_per_replica=1,
                seed=21)
    R = len(betas)
    for p, pr in enumerate(probs):
        op = O.Problem(q=pr["q"])
        res = O.run_tempering(op, betas, dict(variant="unbiased", k=pr["k"], L0=L0, seed=21), group_id=p,
                              chain_id0=p * R, x0s=[np.zeros(pr["n"], np.uint8)] * R, rounds=steps // swap,
                              periods_per_round=swap // L0)
        for s in range(R):
            cid = p * R + s
            r = res[s]
            rec = int(g["stats"]["tape_records"][cid])
            assert rec == len(r["flips"]), (cid, rec, len(r["flips"]))
            np.testing.assert_array_equal(g["flips"][cid, :rec], r["flips"])
            np.testing.assert_array_equal(g["m"][cid, :rec], r["m"])
            st = g["stats"][cid]
            assert st["beta_idx"] == r["state"].beta_idx
            assert st["swaps_accepted"] == r["state"].swaps_accepted
            assert st["energy"] == r["state"].E
            assert st["sum_m"] == steps
            bits = synth.unpack_bits(g["states"][cid:cid + 1], pr["n"])[0]
            np.testing.assert_array_equal(bits, r["x"])
    assert g["stats"]["swaps_accepted"].sum() > 0


@pytest.mark.parametrize("integer", [True, False])
def test_metropolis_tempering_matches_oracle(integer):
    """Metropolis (Algorithm 1) with replica exchange every swap_interval
    records: per-slot tapes, temperatures, exchange counts, energies and
    states equal the oracle's (two chains per temperature, uneven n)."""
    probs = _problems([64, 96], seed=5, integer=integer)
    betas = synth.geometric_ladder(0.05, 2.0, 6)
    for p in probs:
        p["betas"] = betas
    cpr, swap, steps = 2, 50, 1000
    g = gpu_run(probs, steps, tape=True, variant="metropolis", L0=100, swap_interval=swap, chains_per_replica=cpr,
                seed=2)
    R = len(betas)
    for p, pr in enumerate(probs):
        op = O.Problem(q=pr["q"])
        for r in range(cpr):
            grp = p * cpr + r
            res = O.run_tempering(op, betas, dict(variant="metropolis", L0=100, seed=2), group_id=grp,
                                  chain_id0=grp * R, x0s=[np.zeros(pr["n"], np.uint8)] * R, rounds=steps // swap,
                                  periods_per_round=swap)
            for s in range(R):
                cid = grp * R + s
                o = res[s]
                rec = int(g["stats"]["tape_records"][cid])
                assert rec == len(o["flips"]) == steps
                np.testing.assert_array_equal(g["flips"][cid, :rec], o["flips"])
                assert (g["m"][cid, :rec] == 1.0).all()
                st = g["stats"][cid]
                assert st["beta_idx"] == o["state"].beta_idx
                assert st["swaps_accepted"] == o["state"].swaps_accepted
                assert st["energy"] == o["state"].E
                bits = synth.unpack_bits(g["states"][cid:cid + 1], pr["n"])[0]
                np.testing.assert_array_equal(bits, o["x"])
    bidx = g["stats"]["beta_idx"].reshape(-1, R)
    for row in bidx:
        assert sorted(row.tolist()) == list(range(R))
    assert g["stats"]["swaps_accepted"].sum() > 0
