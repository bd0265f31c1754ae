"""The subset-size / L0 / subset-kind study of Sec. 5, run on the GPU with
1000 independent chains per setting (the paper averages the TVD of 1000
simulation runs): the paper's 16-bit QUBO with upper-triangular N(0, 10^2)
entries, beta = 1, each chain's multiplicity-weighted histogram cut at K
original samples and compared with exact pi.

Checked (the paper's findings, read from the discussion of its figures):
  * every setting converges: the mean TVD falls as K grows;
  * at equal original samples, larger partial neighbour sets are less
    biased (|N_i| = 14 best, 2 worst);
  * at equal original samples, L0 = 10 is the least biased, L0 = 1000 the
    most;
  * random and systematic sets perform close to each other.
"""
import numpy as np
import pytest

from oracle import exact as X
from paper_2210_10513_gb300 import synth

pytestmark = pytest.mark.gpu

N = 16
CHAINS = 1000
KS = (6000, 24000, 96000)


def _mean_tvd(q, pi, k, L0, subset, seed):
    import torch

    from paper_2210_10513_gb300 import pns
    dev = torch.device("cuda")
    s = pns.Sampler([dict(n=N, q=torch.from_numpy(q).to(dev), betas=[1.0])], variant="unbiased", k=k, subset=subset,
                    chains_per_replica=CHAINS, L0=L0, seed=seed, tape=2)
    hists = {K: torch.zeros((CHAINS, 1 << N), dtype=torch.float64, device=dev) for K in KS}
    cum = torch.zeros(CHAINS, dtype=torch.float64, device=dev)
    for _ in range(200):
        s.run(2000)
        info = pns.pns_get_info(s.ctx)
        xs = torch.empty((CHAINS, info.tape_capacity, info.words_per_chain), dtype=torch.int32, device=dev)
        ms = torch.empty((CHAINS, info.tape_capacity), dtype=torch.float64, device=dev)
        pns.pns_read(s.ctx, None, ms, None, None)
        pns.pns_read_samples(s.ctx, xs, None)
        codes = (xs[:, :, 0] & 0xFFFF).long()  # bit i of the code is x_i, as in oracle.exact.state_bits
        csum = torch.cumsum(ms, dim=1) + cum[:, None]
        before = csum - ms
        for K in KS:  # each chain's weights cut at K original samples
            hists[K].scatter_add_(1, codes, torch.clamp(torch.minimum(ms, K - before), min=0.0))
        cum = csum[:, -1].clone()
        if bool((cum >= KS[-1]).all()):
            break
    s.close()
    assert bool((cum >= KS[-1]).all())
    pit = torch.tensor(pi, device=dev)
    return {K: float((0.5 * (hists[K] / K - pit[None, :]).abs().sum(dim=1)).mean()) for K in KS}


@pytest.mark.parametrize("inst", [0, 1])
def test_subset_size_and_L0_study(inst):
    q = synth.upper_triangular_qubo(N, 10.0, inst)
    pi = X.target(q.astype(np.float64), None, 1.0)
    settings = {"k2": (2, 100, "systematic"), "k8": (8, 100, "systematic"), "k14": (14, 100, "systematic"),
                "rand8": (8, 100, "random"), "L10": (8, 10, "systematic"), "L1000": (8, 1000, "systematic")}
    res = {}
    for i, (name, (k, L0, sub)) in enumerate(settings.items()):
        res[name] = _mean_tvd(q, pi, k, L0, sub, seed=100 * inst + i)
        print(inst, name, {K: round(v, 4) for K, v in res[name].items()})
    big, small = KS[-1], KS[0]
    for name, r in res.items():
        assert r[big] < 0.5 * r[small], name  # converges
    assert res["k14"][big] < res["k8"][big] < res["k2"][big]
    assert res["L10"][big] < res["k8"][big] < res["L1000"][big]
    ratio = res["rand8"][big] / res["k8"][big]
    assert 1 / 3 < ratio < 3
