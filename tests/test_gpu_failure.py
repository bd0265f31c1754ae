"""Failure detection and recovery without faulting the GPU.

A bounded device loop (the draw of a random k-subset) is made to give up with
a host-set cap: the kernel latches PNS_ERR_TIMEOUT in the context's status
word and the chain stops, the next pns_run answers PNS_ERR_STATE, and
pns_restore from an earlier checkpoint continues the chains with the records
of an uninterrupted run.  Host-side injection (PNS_FAULT) fails allocations
and launches before anything reaches the GPU; the calls return the status of
the real failure and leave the process able to carry on."""
import numpy as np
import pytest

from paper_2210_10513_gb300 import synth

pytestmark = pytest.mark.gpu


def _problem():
    n = 64
    return dict(n=n, q=synth.dense_int(n, -30, 30, 8, np.int32), b=synth.vector_int(n, -10, 10, 8, np.int32),
                betas=[0.2, 0.5])


def _sampler(variant, **kw):
    from paper_2210_10513_gb300 import pns
    opts = dict(variant=variant, k=8, chains_per_replica=3, L0=50, seed=5, tape=True, graph=False)
    opts.update(kw)
    return pns.Sampler([_problem()], **opts)


@pytest.mark.parametrize("variant,subset,prod", [("basic", "systematic", None), ("basic", "systematic", "0"),
                                                 ("unbiased", "random", None)])
def test_subset_draw_gives_up_and_restore_recovers(monkeypatch, variant, subset, prod):
    from paper_2210_10513_gb300 import pns
    if prod is not None:
        monkeypatch.setenv("PNS_PRODUCER_WARPS", prod)
    ref = _sampler(variant, subset=subset)
    ref.run(100)
    ref.run(300)
    want = ref.read()
    ref.close()

    s = _sampler(variant, subset=subset)
    s.run(100)
    ck = s.checkpoint()
    monkeypatch.setenv("PNS_DRAW_CAP", "1")  # fewer draws than k distinct values need
    s.run(300)
    with pytest.raises(pns.PnsError) as ei:
        s.read()
    assert ei.value.status == 6  # PNS_ERR_TIMEOUT, latched by the kernel
    with pytest.raises(pns.PnsError) as ei:
        s.run(10)
    assert ei.value.status == 7  # PNS_ERR_STATE until restored
    monkeypatch.delenv("PNS_DRAW_CAP")
    s.restore(ck)
    s.run(300)
    got = s.read()
    s.close()
    np.testing.assert_array_equal(got["states"], want["states"])
    np.testing.assert_array_equal(got["stats"], want["stats"])
    np.testing.assert_array_equal(got["flips"], want["flips"])
    np.testing.assert_array_equal(got["m"], want["m"])


@pytest.mark.parametrize("fault", ["alloc", "alloc_after=3", "alloc_after=9"])
def test_injected_allocation_failure(monkeypatch, fault):
    """The first, fourth or tenth device allocation of pns_create fails: the
    call returns PNS_ERR_OOM, frees what it had allocated, and a create after
    the fault is gone works."""
    import torch

    from paper_2210_10513_gb300 import pns
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("PNS_FAULT", fault)
    with pytest.raises(pns.PnsError) as ei:
        _sampler("unbiased")
    assert ei.value.status == 4 and "injected" in str(ei.value)
    monkeypatch.delenv("PNS_FAULT")
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= (4 << 20)
    s = _sampler("unbiased")
    s.run(50)
    assert s.read()["stats"]["steps"].min() == 50
    s.close()


def test_injected_launch_failure_changes_nothing(monkeypatch):
    from paper_2210_10513_gb300 import pns
    ref = _sampler("unbiased", subset="random")
    ref.run(200)
    want = ref.read()
    ref.close()
    s = _sampler("unbiased", subset="random")
    s.run(100)
    monkeypatch.setenv("PNS_FAULT", "launch")
    with pytest.raises(pns.PnsError) as ei:
        s.run(100)
    assert ei.value.status == 5 and "injected" in str(ei.value)
    monkeypatch.delenv("PNS_FAULT")
    s.run(100)  # the failed call launched nothing: the chains continue where they were
    got = s.read()
    s.close()
    np.testing.assert_array_equal(got["states"], want["states"])
    np.testing.assert_array_equal(got["stats"]["sum_m"], want["stats"]["sum_m"])
    np.testing.assert_array_equal(got["stats"]["energy"], want["stats"]["energy"])
