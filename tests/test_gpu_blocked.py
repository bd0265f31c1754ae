"""Period-blocked Unbiased PNS with replica exchange: the set fields follow the
k x k sub-block during a period and the other fields take the logged rows at
the period end.  Every field receives the same additions in the same order as
with the per-flip update, so tapes, states, fields and statistics are
bit-identical to the per-flip kernel (fp32 and integer Q) and to the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2210_10513_gb300 import synth
from tests.gpu_helpers import gpu_run

pytestmark = pytest.mark.gpu


def _probs(ns, qkind, betas, seed=0, kdiv=16, kmin=1):
    out = []
    for i, n in enumerate(ns):
        if qkind == "f32":
            q = synth.dense_normal(n, 1.0, seed + i)
        elif qkind == "i16":
            q = synth.dense_int(n, -100, 100, seed + i, np.int16)
        else:
            q = synth.dense_int(n, -20, 20, seed + i, np.int32)
        out.append(dict(n=n, q=q, b=None, betas=betas, k=max(kmin, n // kdiv)))
    return out


def _pair(monkeypatch, probs, steps, **cfg):
    monkeypatch.setenv("PNS_BLOCKED", "1")
    a = gpu_run(probs, steps, tape=True, **cfg)
    monkeypatch.setenv("PNS_BLOCKED", "0")
    b = gpu_run(probs, steps, tape=True, **cfg)
    monkeypatch.delenv("PNS_BLOCKED")
    assert a["info"].period_blocked == 1 and b["info"].period_blocked == 0
    np.testing.assert_array_equal(a["stats"], b["stats"])
    np.testing.assert_array_equal(a["states"], b["states"])
    np.testing.assert_array_equal(a["fields"], b["fields"])
    for cid, rec in enumerate(a["stats"]["tape_records"]):
        np.testing.assert_array_equal(a["flips"][cid, :rec], b["flips"][cid, :rec])
        np.testing.assert_array_equal(a["m"][cid, :rec], b["m"][cid, :rec])
    return a


@pytest.mark.parametrize("qkind,gw", [("f32", "0"), ("i16", "0"), ("i32", "0"), ("f32", "1"), ("f32", "3"),
                                     ("f32", "8")])
def test_blocked_equals_per_flip(monkeypatch, qkind, gw):
    """gw: warps per exchange group (0: the planner's choice); 3 does not
    divide the 8 replicas."""
    monkeypatch.setenv("PNS_GROUP_WARPS", gw)
    betas = synth.geometric_ladder(0.1, 10.0, 8)
    probs = _probs([130, 257, 96, 2048], qkind, betas, seed=4)
    g = _pair(monkeypatch, probs, 2000, variant="unbiased", k=1, L0=100, swap_interval=100, seed=8)
    assert g["stats"]["swaps_accepted"].sum() > 0


def test_blocked_long_periods_flush_the_log(monkeypatch):
    """L0 = 1000 at hot temperatures: more than 128 moves in a period, so the
    chain applies its full log itself in the middle of the period."""
    betas = synth.geometric_ladder(0.01, 0.05, 4)
    probs = _probs([200, 333], "f32", betas, seed=6)
    g = _pair(monkeypatch, probs, 4000, variant="unbiased", k=1, L0=1000, swap_interval=2000, seed=3)
    m = g["m"]
    assert (g["stats"]["flips"] > 300).all()
    assert g["stats"]["tape_records"].max() > 2 * 128
    assert np.isfinite(m).all()


@pytest.mark.parametrize("n,k", [(128, 128), (100, 1), (97, 13), (64, 40)])
def test_blocked_set_shapes(monkeypatch, n, k):
    """Whole-set windows, single-bit sets and windows that wrap around n."""
    betas = synth.geometric_ladder(0.2, 3.0, 3)
    q = synth.dense_int(n, -30, 30, n, np.int32)
    probs = [dict(n=n, q=q, b=synth.vector_int(n, -30, 30, n, np.int32), betas=betas, k=k)]
    _pair(monkeypatch, probs, 1500, variant="unbiased", k=1, L0=50, swap_interval=150, seed=n,
          chains_per_replica=2)


def test_blocked_placement_changes_nothing(monkeypatch):
    """200 exchange groups, one CTA each: more CTAs than SMs, fewer than two
    per SM, so the planner moves the first CTAs of its pack (the largest and
    smallest instances) to the SMs that hold one CTA.  The records do not
    depend on where a group runs."""
    monkeypatch.setenv("PNS_BLOCKED", "1")
    monkeypatch.setenv("PNS_GROUP_WARPS", "4")
    betas = synth.geometric_ladder(0.1, 5.0, 4)
    rng = np.random.default_rng(11)
    probs = _probs([int(v) for v in rng.integers(32, 160, 200)], "i32", betas, seed=100, kdiv=8)
    cfg = dict(variant="unbiased", k=1, L0=50, swap_interval=100, seed=5)
    out = {}
    for place in ("1", "0"):
        monkeypatch.setenv("PNS_PLACE_ALONE", place)
        out[place] = gpu_run(probs, 600, tape=True, **cfg)
        assert out[place]["info"].period_blocked == 1
    a, b = out["1"], out["0"]
    assert a["info"].ctas == b["info"].ctas
    np.testing.assert_array_equal(a["stats"], b["stats"])
    np.testing.assert_array_equal(a["states"], b["states"])
    np.testing.assert_array_equal(a["fields"], b["fields"])
    np.testing.assert_array_equal(a["flips"], b["flips"])
    np.testing.assert_array_equal(a["m"], b["m"])
    assert a["stats"]["swaps_accepted"].sum() > 0


def test_blocked_matches_oracle(monkeypatch):
    monkeypatch.setenv("PNS_BLOCKED", "1")
    ns = [130, 97]
    betas = synth.geometric_ladder(0.1, 10.0, 4)
    probs = _probs(ns, "f32", betas, seed=9, kdiv=8)
    L0, swap, steps = 100, 200, 2000
    g = gpu_run(probs, steps, tape=True, variant="unbiased", k=1, L0=L0, swap_interval=swap, seed=17)
    assert g["info"].period_blocked == 1
    R = len(betas)
    for p, pr in enumerate(probs):
        res = O.run_tempering(O.Problem(q=pr["q"]), betas, dict(variant="unbiased", k=pr["k"], L0=L0, seed=17),
                              group_id=p, chain_id0=p * R, x0s=[np.zeros(pr["n"], np.uint8)] * R,
                              rounds=steps // swap, periods_per_round=swap // L0)
        for s in range(R):
            cid = p * R + s
            rec = int(g["stats"]["tape_records"][cid])
            assert rec == len(res[s]["flips"])
            np.testing.assert_array_equal(g["flips"][cid, :rec], res[s]["flips"])
            np.testing.assert_array_equal(g["m"][cid, :rec], res[s]["m"])
            assert g["stats"][cid]["energy"] == res[s]["state"].E
            bits = synth.unpack_bits(g["states"][cid:cid + 1], pr["n"])[0]
            np.testing.assert_array_equal(bits, res[s]["x"])


@pytest.mark.parametrize("L0,swap", [(100, 100), (1000, 2000)])
def test_blocked_sample_tape_equals_per_flip(monkeypatch, L0, swap):
    """tape = 2: the bits and energy each record starts from.  The blocked
    kernel sums a period's energies when it settles the period's log (and in
    the middle of a period whose log fills up); the per-flip kernel record by
    record: the same values."""
    from paper_2210_10513_gb300 import pns
    from tests.gpu_helpers import to_dev
    betas = synth.geometric_ladder(0.01, 1.0, 4)
    probs = _probs([200, 333], "f32", betas, seed=9)
    out = {}
    for blocked in ("1", "0"):
        monkeypatch.setenv("PNS_BLOCKED", blocked)
        s = pns.Sampler([dict(p, q=to_dev(p["q"])) for p in probs], variant="unbiased", k=1, L0=L0,
                        swap_interval=swap, seed=12, tape=2)
        assert s.info.period_blocked == int(blocked)
        s.run(4000)
        r = s.read()
        x, e = s.samples()
        s.close()
        out[blocked] = (r, x, e)
    (ra, xa, ea), (rb, xb, eb) = out["1"], out["0"]
    np.testing.assert_array_equal(ra["stats"], rb["stats"])
    for cid, rec in enumerate(ra["stats"]["tape_records"]):
        np.testing.assert_array_equal(xa[cid, :rec], xb[cid, :rec])
        np.testing.assert_array_equal(ea[cid, :rec], eb[cid, :rec])
