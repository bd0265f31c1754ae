"""CUDA-graph replay and the autotuned chain-to-CTA mapping leave every record
unchanged: tapes, states and fields equal those of plain launches with the
heuristic mapping."""
import numpy as np
import pytest

from paper_2210_10513_gb300 import synth
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


def _sampler(graph=False, autotune=False, **kw):
    from paper_2210_10513_gb300 import pns
    n = 200
    q = synth.dense_int(n, -50, 50, 7, np.int16)
    b = synth.vector_int(n, -50, 50, 7, np.int16)
    cfg = dict(variant="unbiased", k=24, chains_per_replica=40, L0=100, seed=13, tape=True)
    cfg.update(kw)
    return pns.Sampler([dict(n=n, q=to_dev(q), b=to_dev(b), betas=[0.1])], graph=graph, autotune=autotune, **cfg)


def _runs(s, steps_list, stream=None):
    outs = []
    for st in steps_list:
        s.run(st, stream)
        o = s.read(stream)
        o["fields"] = s.fields(stream)
        outs.append(o)
    s.close()
    return outs


def _equal(a, b):
    np.testing.assert_array_equal(a["stats"], b["stats"])
    for key in ("states", "fields"):
        np.testing.assert_array_equal(a[key], b[key])
    # tape entries past a chain's tape_records are undefined
    for cid, rec in enumerate(a["stats"]["tape_records"]):
        for key in ("flips", "m"):
            np.testing.assert_array_equal(a[key][cid, :rec], b[key][cid, :rec])


@pytest.mark.parametrize("variant", ["unbiased", "basic", "metropolis"])
def test_graph_replay_equals_launches(variant):
    import torch
    steps = [300, 300, 500, 300]
    ref = _runs(_sampler(variant=variant), steps)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        got = _runs(_sampler(graph=True, variant=variant), steps, st)
    for a, b in zip(got, ref):
        _equal(a, b)


def test_graph_replay_tempering():
    import torch

    from paper_2210_10513_gb300 import pns
    n = 96
    q = synth.dense_int(n, -20, 20, 3, np.int32)
    betas = synth.geometric_ladder(0.1, 2.0, 4)

    def make(graph, autotune=False):
        return pns.Sampler([dict(n=n, q=to_dev(q), betas=betas)], variant="unbiased", k=6, L0=50, swap_interval=100,
                           seed=4, tape=True, graph=graph, autotune=autotune)
    ref = _runs(make(False), [400, 400])
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        got = _runs(make(True), [400, 400], st)
        tuned = _runs(make(True, True), [400, 400], st)
    for a, b, c in zip(got, ref, tuned):
        _equal(a, b)
        _equal(c, b)


@pytest.mark.parametrize("variant", ["unbiased", "metropolis"])
def test_autotuned_mapping_equals_heuristic(tmp_path, monkeypatch, variant):
    ref = _runs(_sampler(variant=variant), [700])[0]
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("PNS_AUTOTUNE_CACHE", str(cache))
    s = _sampler(autotune=True, variant=variant)
    info = s.info
    got = _runs(s, [700])[0]
    _equal(got, ref)
    assert cache.exists() and len(cache.read_text().strip().splitlines()) == 1
    # a second context takes the cached choice
    s2 = _sampler(autotune=True, variant=variant)
    for key in ("team_warps", "producer_warps", "spec_depth", "set_sweep", "ctas"):
        assert getattr(s2.info, key) == getattr(info, key)
    got2 = _runs(s2, [700])[0]
    _equal(got2, ref)
    assert len(cache.read_text().strip().splitlines()) == 1


def test_autotune_csr_lattice():
    from paper_2210_10513_gb300 import pns
    side = 16
    csr = synth.lattice_csr(side, seed=3)

    def make(autotune):
        return pns.Sampler([dict(n=side * side, csr=tuple(to_dev(a) for a in csr), betas=[0.44])], variant="unbiased",
                           k=64, chains_per_replica=8, seed=4, tape=True, autotune=autotune)
    ref = _runs(make(False), [600])[0]
    got = _runs(make(True), [600])[0]
    _equal(got, ref)
