"""The per-flip kernel with two chains per warp (Unbiased PNS on systematic
sets of k <= 16): records equal to the oracle's and to the one-warp kernel's,
bit for bit, on ragged sizes, several instances, odd chain counts (a warp
with one idle half), every Q type, the sample tape, X_max and the cooling
schedule."""
import numpy as np
import pytest

from paper_2210_10513_gb300 import synth
from tests.gpu_helpers import assert_chain_equal, gpu_run, oracle_run, to_dev

pytestmark = pytest.mark.gpu


def _problems(dtype):
    if dtype == np.float32:
        return [dict(n=77, q=synth.dense_normal(77, 0.5, 3), b=synth.vector_normal(77, 0.5, 3), betas=[0.7, 1.3]),
                dict(n=40, q=synth.dense_normal(40, 0.5, 4), b=None, betas=[1.0])]
    return [dict(n=77, q=synth.dense_int(77, -20, 20, 3, dtype), b=synth.vector_int(77, -20, 20, 3, dtype),
                 betas=[0.05, 0.1]),
            dict(n=40, q=synth.dense_int(40, -20, 20, 4, dtype), b=None, betas=[0.2])]


@pytest.mark.parametrize("dtype", [np.int16, np.int32, np.float32])
@pytest.mark.parametrize("k", [16, 5])
def test_half_warp_chains_equal_oracle(monkeypatch, dtype, k):
    monkeypatch.setenv("PNS_HALF", "1")
    probs = _problems(dtype)
    cfg = dict(variant="unbiased", k=k, chains_per_replica=3, L0=50, seed=7)  # 9 chains: an odd count
    g = gpu_run(probs, 700, tape=True, **cfg)
    assert g["info"].chains_per_warp == 2
    ids = list(range(9))
    ref = oracle_run(probs, 700, ids, **cfg)
    for cid in ids:
        assert_chain_equal(g, ref[cid], cid, probs[ref[cid]["instance"]]["n"], 700)


@pytest.mark.parametrize("extra", [dict(tape=2), dict(track_best=True), dict(anneal_start=0.3, anneal_steps=400)])
def test_half_warp_equals_one_warp_kernel(monkeypatch, extra):
    """The same records, tape, fields and best states as the one-warp form."""
    from paper_2210_10513_gb300 import pns
    probs = _problems(np.float32)
    cfg = dict(variant="unbiased", k=12, chains_per_replica=7, L0=100, seed=11, **extra)
    if "tape" not in extra:
        cfg["tape"] = True
    out = {}
    for half in ("0", "1"):
        monkeypatch.setenv("PNS_HALF", half)
        s = pns.Sampler([dict(p, q=to_dev(p["q"]), b=to_dev(p.get("b"))) for p in probs], **cfg)
        assert s.info.chains_per_warp == (2 if half == "1" else 1)
        s.run(600)
        s.run(300)  # a second launch continues the chains
        r = s.read()
        r["fields"] = s.fields()
        if extra.get("tape") == 2:
            r["samples"] = s.samples()
        if extra.get("track_best"):
            r["best"] = s.best()
        s.close()
        out[half] = r
    a, b = out["0"], out["1"]
    for key in ("states", "flips", "m", "fields"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)
    for key in a["stats"].dtype.names:
        np.testing.assert_array_equal(a["stats"][key], b["stats"][key], err_msg=key)
    if "samples" in a:
        for x, y in zip(a["samples"], b["samples"]):
            np.testing.assert_array_equal(x, y)
    if "best" in a:
        np.testing.assert_array_equal(a["best"], b["best"])


def test_half_warp_is_the_default_for_many_chains():
    from paper_2210_10513_gb300 import pns
    n = 64
    wl = synth.workload_fit(n, seed=0)
    s = pns.Sampler([dict(n=n, q=to_dev(wl["q"]), b=to_dev(wl["b"]), betas=[1.0])], variant="unbiased", k=16,
                    chains_per_replica=8192, L0=100, seed=0)
    assert s.info.chains_per_warp == 2
    s.close()
