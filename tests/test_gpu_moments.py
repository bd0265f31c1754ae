"""Tensor-core moments and the backward: against an fp64 reduction of the
same sample tape (arithmetic error only), against exact enumeration
(statistical), and through torch.autograd."""
import numpy as np
import pytest

from oracle import exact as X
from paper_2210_10513_gb300 import synth
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


def _sampler(n, q, b, beta, chains, steps, seed=0, variant="unbiased", k=None, burn=0):
    from paper_2210_10513_gb300 import pns
    s = pns.Sampler([dict(n=n, q=to_dev(q), b=to_dev(b), betas=[beta])], variant=variant, k=k or max(1, n // 4),
                    chains_per_replica=chains, L0=100, seed=seed, tape=2)
    if burn:
        s.run(burn)  # burn-in; the tape keeps the last run only
    s.run(steps)
    return s


def _fp64_moments(xbits, E, M, n):
    """Plain fp64 reduction of the tape (the same-tape reference)."""
    C, R = M.shape
    bits = ((xbits[:, :, 0:1].astype(np.uint64) | (xbits[:, :, 1:2].astype(np.uint64) << 32 if xbits.shape[2] > 1
                                                   else 0)) >> np.arange(n, dtype=np.uint64)) & 1
    x = bits.reshape(C * R, n).astype(np.float64)
    w = M.reshape(-1)
    e = E.reshape(-1)
    W = w.sum()
    mE = (w * e).sum() / W
    d = e - mE
    mxx = (x * w[:, None]).T @ x / W
    mx = (w @ x) / W
    cexx = (x * (w * d)[:, None]).T @ x / W
    cex = ((w * d) @ x) / W
    var = (w * d * d).sum() / W
    return dict(W=W, mE=mE, var=var, mx=mx, mxx=mxx, cex=cex, cexx=cexx, x=x, w=w)


@pytest.mark.parametrize("n,integer", [(16, False), (64, False), (40, True)])
def test_moments_match_fp64_same_tape(n, integer):
    if integer:
        q = synth.dense_int(n, -5, 5, 3, np.int32)
        b = synth.vector_int(n, -5, 5, 3, np.int32)
        beta = 0.2
    else:
        q = synth.dense_normal(n, 0.3, 3)
        b = synth.vector_normal(n, 0.3, 3)
        beta = 1.0
    s = _sampler(n, q, b, beta, chains=64, steps=3000)
    out = s.read()
    xb, E = s.samples()
    mom = s.moments(n)
    s.close()
    ref = _fp64_moments(xb, E, out["m"], n)
    sc = mom["scalars"]
    assert sc[0] == ref["W"]
    assert sc[3] == out["m"].size
    assert abs(sc[1] - ref["mE"]) <= 1e-12 * max(1.0, abs(ref["mE"]))
    assert abs(sc[2] - ref["var"]) <= 1e-9 * max(1.0, ref["var"])
    # multiplicities <= 100: X^T diag(M) X is exact on the tensor cores
    np.testing.assert_array_equal(mom["mean_xx"] * ref["W"], ref["mxx"] * ref["W"])
    np.testing.assert_array_equal(mom["mean_x"] * ref["W"], ref["mx"] * ref["W"])
    # fp32 accumulation of mixed-sign weights per 16384 samples:
    # error ~ 2^-24 sqrt(16384) <|E - <E>|> ~ 1e-5 of the scale
    scale = np.abs(ref["cexx"]).max()
    assert np.abs(mom["cov_exx"] - ref["cexx"]).max() <= 3e-5 * scale
    assert np.abs(mom["cov_ex"] - ref["cex"]).max() <= 3e-5 * scale


def test_grads_within_1e4_of_fp64_same_tape():
    import torch

    from paper_2210_10513_gb300 import pns
    n = 64
    wl = synth.workload_fit(n, seed=0)
    s = _sampler(n, wl["q"], wl["b"], 1.0, chains=256, steps=2000, k=16)
    out = s.read()
    xb, E = s.samples()
    mom = s.moments(n, device="cuda")
    s.close()
    ref = _fp64_moments(xb, E, out["m"], n)
    dQ = torch.empty((n, n), dtype=torch.float64, device="cuda")
    db = torch.empty(n, dtype=torch.float64, device="cuda")
    dbeta = torch.empty(1, dtype=torch.float64, device="cuda")
    pns.pns_energy_grads(n, 1.0, mom["scalars"], mom["mean_x"], mom["mean_xx"], mom["cov_ex"], mom["cov_exx"], None,
                         None, 0.0, dQ, db, dbeta)
    gQ = ref["mxx"] - ref["cexx"]
    gb = ref["mx"] - ref["cex"]
    for got, want in ((dQ.cpu().numpy(), gQ), (db.cpu().numpy(), gb)):
        assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max()
    assert abs(dbeta.item() + ref["var"]) <= 1e-4 * ref["var"]


def test_grads_match_exact_enumeration_n12():
    """Statistical: batch means over independent chain groups."""
    n = 12
    q = synth.dense_normal(n, 0.5, 9)
    b = synth.vector_normal(n, 0.5, 9)
    beta = 1.0
    gQ_ex, gb_ex, gbeta_ex, E_ex = X.mean_energy_grads(q.astype(np.float64), b.astype(np.float64), beta)
    ests = []
    for rep in range(8):
        s = _sampler(n, q, b, beta, chains=128, steps=4000, seed=100 + rep, k=4, burn=2000)
        mom = s.moments(n)
        s.close()
        ests.append((mom["scalars"][1], mom["mean_xx"] - beta * mom["cov_exx"], -mom["scalars"][2]))
    Es = np.array([e[0] for e in ests])
    gQs = np.stack([e[1] for e in ests])
    gbetas = np.array([e[2] for e in ests])
    se = lambda a: a.std(axis=0, ddof=1) / np.sqrt(len(a))  # noqa: E731
    assert abs(Es.mean() - E_ex) <= 5 * se(Es) + 1e-3
    assert abs(gbetas.mean() - gbeta_ex) <= 5 * se(gbetas) + 1e-3
    z = np.abs(gQs.mean(0) - gQ_ex) / (se(gQs) + 1e-4)
    assert z.max() < 6.0


def test_autograd_functions():
    import torch

    from paper_2210_10513_gb300 import autograd as AG
    n = 16
    q = torch.tensor(synth.dense_normal(n, 0.4, 5), device="cuda", requires_grad=True)
    b = torch.tensor(synth.vector_normal(n, 0.4, 5), device="cuda", requires_grad=True)
    beta = torch.tensor(1.0, device="cuda", requires_grad=True)
    E = AG.mean_energy(q, b, beta, steps=2000, chains_per_replica=256, k=4, seed=3)
    E.backward()
    gQ_ex, gb_ex, gbeta_ex, E_ex = X.mean_energy_grads(q.detach().cpu().double().numpy(),
                                                       b.detach().cpu().double().numpy(), 1.0)
    assert abs(E.item() - E_ex) < 0.05 * max(1.0, abs(E_ex))
    assert np.abs(q.grad.cpu().numpy() - gQ_ex).max() < 0.1
    assert abs(beta.grad.item() - gbeta_ex) < 0.1 * max(1.0, abs(gbeta_ex))
    # Boltzmann fit: data drawn from the model itself has zero expected gradient
    m = X.exact_moments(q.detach().cpu().double().numpy(), b.detach().cpu().double().numpy(), 1.0)
    q.grad = None
    b.grad = None
    beta.grad = None
    ll = AG.boltzmann_fit(q, b, beta, torch.tensor(m["x"], device="cuda"), torch.tensor(m["xx"], device="cuda"),
                          steps=2000, chains_per_replica=256, k=4, seed=4)
    ll.backward()
    assert np.abs(q.grad.cpu().numpy()).max() < 0.05
    assert abs(beta.grad.item()) < 0.05 * max(1.0, abs(m["E"]))


def test_data_energy_kernel_equals_fp64_sum():
    """pns_data_energy: sum_ij data_xx_ij Q_ij + sum_i data_x_i b_i in fp64
    equals the plain fp64 sum (rounding order only), with and without b."""
    import torch

    from paper_2210_10513_gb300 import pns
    rng = np.random.default_rng(5)
    for n in (1, 16, 64, 300):
        q = synth.dense_normal(n, 0.1, n)
        b = synth.vector_normal(n, 0.1, n)
        x = rng.uniform(0, 1, n)
        xx = rng.uniform(0, 1, (n, n))
        xx = (xx + xx.T) / 2
        want = float((xx * q.astype(np.float64)).sum() + (x * b.astype(np.float64)).sum())
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
        pns.pns_data_energy(n, dev(q), dev(b), dev(x), dev(xx), out)
        assert float(out.item()) == pytest.approx(want, rel=1e-12, abs=1e-12)
        pns.pns_data_energy(n, dev(q), None, None, dev(xx), out)
        assert float(out.item()) == pytest.approx(float((xx * q.astype(np.float64)).sum()), rel=1e-12, abs=1e-12)
