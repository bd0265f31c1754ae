"""pns_sample_static, the entry point for callers that cannot allocate device
memory (working memory comes from the library's fixed device array), must
give the same records as the allocating path pns_create + pns_run + pns_read.

Collected last on purpose: it also checks that the shared array carries no
state from earlier calls into later ones.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2210_10513_gb300 import synth

pytestmark = pytest.mark.gpu


def _static_run(problem, steps, **cfg):
    import torch

    from paper_2210_10513_gb300 import pns
    keep = []
    qd = torch.from_numpy(problem["q"]).cuda()
    bd = torch.from_numpy(problem["b"]).cuda() if problem.get("b") is not None else None
    betas = torch.tensor(np.asarray(problem["betas"], np.float32)).cuda()
    p = pns.make_problem(problem["n"], q=qd, b=bd, betas=[0.0] * len(problem["betas"]), keep=keep)
    p.betas = betas.data_ptr()
    c = pns.make_config(**cfg)
    chains = len(problem["betas"]) * c.chains_per_replica
    W = problem["n"] // 32
    states = np.zeros((chains, W), np.uint32)
    stats = np.zeros(chains, pns.STATS_DTYPE)
    m = torch.zeros((chains, steps), dtype=torch.float64, device="cuda")
    f = torch.zeros((chains, steps), dtype=torch.int32, device="cuda")
    pns.pns_sample_static(p, c, steps, states, m, f, stats)
    return dict(states=states, stats=stats, m=m.cpu().numpy(), flips=f.cpu().numpy())


def _alloc_run(problem, steps, **cfg):
    from paper_2210_10513_gb300 import pns
    s = pns.Sampler([dict(n=problem["n"], q=problem["q"], b=problem.get("b"), betas=problem["betas"])], tape=True,
                    **cfg)
    s.run(steps)
    out = s.read()
    s.close()
    return out


def _compare(a, b, steps):
    np.testing.assert_array_equal(a["states"], b["states"])
    np.testing.assert_array_equal(a["flips"], b["flips"][:, :steps])
    np.testing.assert_array_equal(a["m"], b["m"][:, :steps])
    for key in ("steps", "flips", "stays", "saturated", "budget_left", "set_start", "beta_idx", "energy", "sum_m",
                "best_energy"):
        np.testing.assert_array_equal(a["stats"][key], b["stats"][key], err_msg=key)


def test_static_equals_allocating_path_two_calls_in_a_row():
    # call 1: larger instance, Unbiased, integer QUBO
    p1 = dict(n=256, q=synth.dense_int(256, -100, 100, 4, np.int16), b=synth.vector_int(256, -100, 100, 4, np.int16),
              betas=[0.05, 0.1])
    cfg1 = dict(variant="unbiased", k=32, chains_per_replica=3, seed=11)
    a1 = _static_run(p1, 1500, **cfg1)
    b1 = _alloc_run(p1, 1500, **cfg1)
    _compare(a1, b1, 1500)
    # call 2: smaller instance and another variant; nothing of call 1 may leak
    p2 = dict(n=64, q=synth.dense_normal(64, 1.0, 5), b=synth.vector_normal(64, 0.5, 5), betas=[0.7])
    cfg2 = dict(variant="basic", k=8, chains_per_replica=5, seed=3)
    a2 = _static_run(p2, 1000, **cfg2)
    b2 = _alloc_run(p2, 1000, **cfg2)
    _compare(a2, b2, 1000)
    # call 3: the first problem again gives the first answer again
    a3 = _static_run(p1, 1500, **cfg1)
    _compare(a3, b1, 1500)


def test_static_rejects_sizes_beyond_the_array():
    import torch

    from paper_2210_10513_gb300 import pns
    n = 2048
    q = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    betas = torch.ones(1, dtype=torch.float32, device="cuda")
    keep = []
    p = pns.make_problem(n, q=q, betas=[1.0], keep=keep)
    p.betas = betas.data_ptr()
    c = pns.make_config("unbiased", k=16, chains_per_replica=4096)  # 4096 x 8 KiB of fields = 32 MiB
    with pytest.raises(pns.PnsError) as ei:
        pns.pns_sample_static(p, c, 10)
    assert ei.value.status == 3 and "scratch" in str(ei.value)
    assert C.sizeof(C.c_char * pns.STATIC_SCRATCH_BYTES) == 16 << 20


def _static_problem(n=64, q=None, betas=(0.5,)):
    import torch

    from paper_2210_10513_gb300 import pns
    q = q if q is not None else synth.dense_int(n, -20, 20, 1, np.int32)
    qd = torch.from_numpy(q).cuda()
    bt = torch.tensor(np.asarray(betas, np.float32)).cuda()
    keep = [qd, bt]
    p = pns.make_problem(n, q=qd, betas=[0.0] * len(betas), keep=keep)
    p.betas = bt.data_ptr()
    return p, keep


def test_static_rejects_what_create_rejects():
    """The inputs pns_create turns away get the same status here: a negative
    or non-finite beta, an fp32 entry whose field bound overflows fp32
    fields, one tape output without the other, and options this entry point
    does not carry out."""
    import torch

    from paper_2210_10513_gb300 import pns
    for betas in ([-0.5], [float("inf")], [0.3, float("nan")]):
        p, keep = _static_problem(betas=betas)
        with pytest.raises(pns.PnsError) as ei:
            pns.pns_sample_static(p, pns.make_config("unbiased", k=4), 10)
        assert ei.value.status == 1 and "betas" in str(ei.value)
    big = np.zeros((64, 64), np.float32)
    big[3, 5] = big[5, 3] = 3.0e38  # finite, but a row sum past 1e30
    p, keep = _static_problem(q=big)
    with pytest.raises(pns.PnsError) as ei:
        pns.pns_sample_static(p, pns.make_config("unbiased", k=4), 10)
    assert ei.value.status == 3
    p, keep = _static_problem()
    m = torch.zeros((1, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(pns.PnsError) as ei:
        pns.pns_sample_static(p, pns.make_config("unbiased", k=4), 10, multiplicities=m)
    assert ei.value.status == 1
    for kw, status in ((dict(track_best=True), 8), (dict(tape=2), 8), (dict(chain_base=-1), 1)):
        with pytest.raises(pns.PnsError) as ei:
            pns.pns_sample_static(p, pns.make_config("unbiased", k=4, **kw), 10)
        assert ei.value.status == status, kw
    # the same problem with valid options still runs
    stats = np.zeros(1, pns.STATS_DTYPE)
    pns.pns_sample_static(p, pns.make_config("unbiased", k=4, seed=2), 50, stats=stats)
    assert stats["steps"][0] == 50


def test_static_refuses_a_capturing_stream():
    """It synchronises its stream, so under stream capture it must return
    PNS_ERR_UNSUPPORTED and leave the caller's capture valid."""
    import torch

    from paper_2210_10513_gb300 import pns
    p, keep = _static_problem()
    s = torch.cuda.Stream()
    x = torch.zeros(4, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            pns.pns_sample_static(p, pns.make_config("unbiased", k=4), 10, stream=s)
        except pns.PnsError as e:
            err = e
        x.add_(1.0)
        g.capture_end()
    assert err is not None and err.status == 8
    g.replay()
    torch.cuda.synchronize()
    assert float(x.sum()) == 4.0
