"""Continuous Unbiased PNS (Algorithm 7) and Metropolis on the Donuts target
(Sec. 7) on the GPU: every chain's weighted sums, counters and final state
equal the oracle's bit for bit; at scale, the multiplicity-weighted moments
approach the target's closed forms and the paper's bias measures fall with
the number of samples."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

MU0, SIGMA = 9.0, 0.1
C = 1.0 / (2.0 * SIGMA * SIGMA)


@pytest.mark.parametrize("variant,steps,L0,npairs", [("unbiased", 3000, 1000, 25), ("unbiased", 2000, 50, 7),
                                                     ("metropolis", 20000, 1000, 25)])
def test_donuts_match_oracle(variant, steps, L0, npairs):
    from paper_2210_10513_gb300 import pns
    chains = 40
    ang = np.arange(chains) * 0.37
    x0 = np.stack([3.0 * np.cos(ang), 3.0 * np.sin(ang)], axis=1).astype(np.float32)
    g = pns.pns_donuts_run(variant, chains, steps, x0=x0, mu0=MU0, c=C, L0=L0, seed=13, npairs=npairs, chain_base=5)
    for ch in range(0, chains, 3):
        r = O.donuts_chain(variant, 5 + ch, steps, tuple(x0[ch]), mu0=MU0, c=C, L0=L0, seed=13, npairs=npairs)
        st = g[ch]
        for key in ("sum_x", "sum_x2", "sum_x4", "sum_pos", "x"):
            np.testing.assert_array_equal(st[key], r[key], err_msg="%s chain %d" % (key, ch))
        for key in ("weight", "records", "moves", "budget_left", "period_start"):
            assert st[key] == r[key], (key, ch)


def _moments(stats):
    W = stats["weight"][:, None]
    return dict(x=stats["sum_x"] / W, x2=stats["sum_x2"] / W, x4=stats["sum_x4"] / W, pos=stats["sum_pos"] / W)


def test_donuts_moments_at_scale():
    """16,384 chains: the Unbiased chains' weighted moments (2000 records,
    L0 = 1000, 50 neighbours) and Metropolis' (40,000 steps) against
    E[x_i] = 0, E[x_i^2] = mu0/2, E[x_i^4] = 3/8 (mu0^2 + sigma^2),
    P(x_i > 0) = 1/2; the paper's first-degree bias falls as the chains run
    longer."""
    from paper_2210_10513_gb300 import pns
    chains = 16384
    rng = np.random.default_rng(0)
    ang = rng.uniform(0, 2 * np.pi, chains)
    x0 = np.stack([3.0 * np.cos(ang), 3.0 * np.sin(ang)], axis=1).astype(np.float32)
    want = dict(x=0.0, x2=MU0 / 2, x4=3 / 8 * (MU0 ** 2 + SIGMA ** 2), pos=0.5)
    for variant, steps in (("unbiased", 2000), ("metropolis", 40000)):
        st = pns.pns_donuts_run(variant, chains, steps, x0=x0, mu0=MU0, c=C, L0=1000, seed=1)
        mo = _moments(st)
        for key, val in want.items():
            est = mo[key]
            mean = est.mean(axis=0)
            se = est.std(axis=0, ddof=1) / np.sqrt(chains)
            assert np.all(np.abs(mean - val) < 6 * se + 1e-3 * max(1.0, abs(val))), (variant, key, mean, val, se)
        r2 = (st["sum_x2"][:, 0] + st["sum_x2"][:, 1]) / st["weight"]
        assert abs(r2.mean() - MU0) < 0.01
    # the paper's bias of the first-degree terms, |mean x1| + |mean x2| per chain, averaged over chains
    bias = []
    for steps in (500, 2000, 8000):
        st = pns.pns_donuts_run("unbiased", 4096, steps, x0=x0[:4096], mu0=MU0, c=C, L0=1000, seed=2)
        mo = _moments(st)
        bias.append(float(np.abs(mo["x"]).sum(axis=1).mean()))
    print("unbiased first-degree bias at 500/2000/8000 records:", bias)
    assert bias[2] < bias[1] < bias[0]
