"""The optimisation forms (Algorithms 8-10) on the GPU: with track_best the
per-flip kernel keeps each chain's X_max.  Basic PNS is then Optimization
PNS and RF Optimization Rejection-Free (constant temperature).  Checked
against the oracle bit for bit, records unchanged by the tracking, and the
burn-in use of Sec. 8.2: Optimization PNS before Unbiased PNS brings the
distribution of the chains' states closer to pi sooner."""
import numpy as np
import pytest

from oracle import exact as X
from paper_2210_10513_gb300 import synth
from tests.gpu_helpers import gpu_run, oracle_run, to_dev

pytestmark = pytest.mark.gpu


def _prob(n=64, seed=0):
    return dict(n=n, q=synth.dense_int(n, -50, 50, seed, np.int32), b=synth.vector_int(n, -50, 50, seed, np.int32),
                betas=[0.2])


def _best_gpu(probs, steps, x0=None, **cfg):
    from paper_2210_10513_gb300 import pns
    ps = []
    for p in probs:
        d = dict(p)
        d["q"] = to_dev(d["q"])
        d["b"] = to_dev(d["b"])
        ps.append(d)
    s = pns.Sampler(ps, track_best=True, tape=True, x0=x0, **cfg)
    s.run(steps)
    out = s.read()
    out["best"] = s.best()
    s.close()
    return out


@pytest.mark.parametrize("variant,k", [("basic", 8), ("rf", 0), ("unbiased", 8), ("metropolis", 1)])
def test_best_states_match_oracle(variant, k):
    p = _prob(64, seed=3)
    chains = 6
    x0 = synth.pack_bits(synth.random_bits(chains, 64, seed=5))
    cfg = dict(variant=variant, k=k, chains_per_replica=chains, seed=11, L0=50)
    g = _best_gpu([p], 1500, x0=x0, **cfg)
    ref = oracle_run([p], 1500, list(range(chains)), x0=x0, **cfg)
    plain = gpu_run([p], 1500, tape=True, x0=x0, **cfg)  # the default mapping, no tracking
    for cid in range(chains):
        r = ref[cid]
        bits = synth.unpack_bits(g["best"][cid:cid + 1], 64)[0]
        np.testing.assert_array_equal(bits, r["x_best"])
        assert g["stats"][cid]["best_energy"] == r["state"].best_E
        np.testing.assert_array_equal(g["flips"][cid], plain["flips"][cid])
        np.testing.assert_array_equal(g["m"][cid], plain["m"][cid])


@pytest.mark.parametrize("variant,k,subset", [("metropolis", 1, "systematic"), ("rf", 0, "systematic"),
                                              ("basic", 8, "systematic"), ("unbiased", 8, "random")])
def test_cooling_schedule_matches_oracle(variant, k, subset):
    """Algorithms 8-10 with the cooling schedule T(k) (geometric from
    T = 1/0.05 to 1 over the first 1000 records, then constant): Simulated
    Annealing (Metropolis), Optimization RF and Optimization PNS (Basic), and
    Unbiased PNS on the same schedule.  Tapes, X_max, best energies and
    states equal the oracle's; a run split in two launches gives the same
    records (the schedule counts the chain's records, not the launch's)."""
    p = _prob(64, seed=4)
    chains = 5
    cfg = dict(variant=variant, k=k, subset=subset, chains_per_replica=chains, seed=7, L0=50, anneal_start=0.05,
               anneal_steps=1000)
    g = _best_gpu([p], 1500, **cfg)
    ref = oracle_run([p], 1500, list(range(chains)), **cfg)
    for cid in range(chains):
        r = ref[cid]
        np.testing.assert_array_equal(g["flips"][cid], r["flips"])
        np.testing.assert_array_equal(g["m"][cid], r["m"])
        bits = synth.unpack_bits(g["best"][cid:cid + 1], 64)[0]
        np.testing.assert_array_equal(bits, r["x_best"])
        assert g["stats"][cid]["best_energy"] == r["state"].best_E
        assert g["stats"][cid]["energy"] == r["state"].E
    from paper_2210_10513_gb300 import pns
    d = dict(p)
    d["q"], d["b"] = to_dev(d["q"]), to_dev(d["b"])
    s = pns.Sampler([d], tape=False, **cfg)
    s.run(700)
    s.run(800)
    st = s.read(tape=False)["stats"]
    s.close()
    np.testing.assert_array_equal(st["energy"], g["stats"]["energy"])
    np.testing.assert_array_equal(st["flips"], g["stats"]["flips"])


def test_cooling_schedule_argument_checks():
    from paper_2210_10513_gb300 import pns
    p = _prob(32, seed=1)
    for kw, status in ((dict(anneal_start=0.0, anneal_steps=10), 1), (dict(anneal_start=1.5, anneal_steps=10), 1),
                       (dict(anneal_steps=-1), 1), (dict(anneal_start=0.5, anneal_steps=10, swap_interval=100), 8)):
        with pytest.raises(pns.PnsError) as ei:
            pns.Sampler([dict(p)], variant="unbiased", k=4, **kw)
        assert ei.value.status == status, kw


def test_best_state_survives_checkpoint():
    from paper_2210_10513_gb300 import pns
    p = _prob(40, seed=8)
    d = dict(n=40, q=to_dev(p["q"]), b=to_dev(p["b"]), betas=[0.5])
    s = pns.Sampler([d], variant="basic", k=6, chains_per_replica=4, seed=2, track_best=True)
    s.run(300)
    ck = s.checkpoint()
    s.run(700)
    a, sa = s.best(), s.read(tape=False)["stats"]
    s.restore(ck)
    s.run(700)
    b, sb = s.best(), s.read(tape=False)["stats"]
    s.close()
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(sa["best_energy"], sb["best_energy"])


def _state_at(s, chains, K, n):
    """Each chain's state at original sample K (the record whose multiplicity
    covers sample K), from the sample tape of the last run."""
    import torch

    from paper_2210_10513_gb300 import pns
    dev = torch.device("cuda")
    info = pns.pns_get_info(s.ctx)
    xs = torch.empty((chains, info.tape_capacity, info.words_per_chain), dtype=torch.int32, device=dev)
    ms = torch.empty((chains, info.tape_capacity), dtype=torch.float64, device=dev)
    pns.pns_read(s.ctx, None, ms, None, None)
    pns.pns_read_samples(s.ctx, xs, None)
    csum = torch.cumsum(ms, dim=1)
    assert bool((csum[:, -1] >= K).all())
    idx = torch.searchsorted(csum, torch.full((chains, 1), float(K), dtype=torch.float64, device=dev))
    codes = (xs[:, :, 0] & ((1 << n) - 1)).long()
    return torch.gather(codes, 1, idx).squeeze(1)


def test_optimization_pns_burn_in():
    """Sec. 8.2 and its convergence figure: 100,000 chains on the 16-bit QUBO
    with upper-triangular N(0, 1) entries; the distribution of the chains'
    states after K1 original samples of Unbiased PNS, with and without
    K0 = K1 / 40 steps of Optimization PNS first (sampling starts from
    X_max)."""
    import torch

    from paper_2210_10513_gb300 import pns
    n, chains = 16, 100_000
    q = synth.upper_triangular_qubo(n, 1.0, 3)
    pi = torch.tensor(X.target(q.astype(np.float64), None, 1.0), device="cuda")
    qd = torch.from_numpy(q).cuda()
    x0 = synth.pack_bits(synth.random_bits(chains, n, seed=9))

    def unbiased_from(xs, K1, seed):
        s = pns.Sampler([dict(n=n, q=qd, betas=[1.0])], variant="unbiased", k=8, L0=100, chains_per_replica=chains,
                        seed=seed, tape=2, x0=xs)
        s.run(2 * K1 + 16)  # M >= 1 except for the rare (stay, 0) records: enough to cover sample K1
        codes = _state_at(s, chains, K1, n)
        s.close()
        hist = torch.bincount(codes, minlength=1 << n).double() / chains
        return 0.5 * float((hist - pi).abs().sum())

    opt = pns.Sampler([dict(n=n, q=qd, betas=[1.0])], variant="basic", k=8, chains_per_replica=chains, seed=5,
                      track_best=True, x0=x0)
    start_ck = opt.checkpoint()
    plain_tvd, hybrid_tvd = {}, {}
    for K1 in (40, 80, 160, 320):
        opt.restore(start_ck)  # every K1 starts Optimization PNS afresh
        opt.run(K1 // 40)
        hybrid_tvd[K1] = unbiased_from(opt.best(), K1, seed=100 + K1)
        plain_tvd[K1] = unbiased_from(x0, K1, seed=200 + K1)
        print(K1, round(plain_tvd[K1], 4), round(hybrid_tvd[K1], 4))
    opt.close()
    for K1 in plain_tvd:
        assert hybrid_tvd[K1] < plain_tvd[K1], K1
    assert plain_tvd[320] < plain_tvd[40]
