"""torch.autograd functions over the PNS sampler.

The forward passes run the CUDA sampler (Unbiased PNS by default) with the
sample tape on and reduce the tape to multiplicity-weighted moments on the
tensor cores (pns_moments); the data energy of the fit (pns_data_energy) and
the gradients (pns_energy_grads) are CUDA kernels too.  This module only
marshals tensors.

MeanEnergy(Q, b, beta) -> <E>, the multiplicity-weighted mean of
    E(x) = x^T Q x + b^T x under pi(x) ~ exp(-beta E(x)).  Its gradients are
    d<E>/dQ_ij = <x_i x_j> - beta Cov(E, x_i x_j),
    d<E>/db_i  = <x_i> - beta Cov(E, x_i),      d<E>/dbeta = -Var(E).
BoltzmannFit(Q, b, beta, data_x, data_xx) -> -beta <E>_D, the data part of the
    per-sample log-likelihood l = -beta <E>_D - log Z; backward returns the
    gradient of l itself:  dl/dQ = -beta (<x x^T>_D - <x x^T>),
    dl/db = -beta (<x>_D - <x>),  dl/dbeta = -<E>_D + <E>.
"""
import numpy as np
import torch

from . import pns


def _run_moments(Q, b, beta, sampler_kw, steps, burn=None):
    n = Q.shape[0]
    q = Q.detach().to(torch.float32).contiguous()
    bb = b.detach().to(torch.float32).contiguous() if b is not None else None
    kw = dict(variant="unbiased", k=max(1, n // 4), chains_per_replica=1024, L0=100, seed=0)
    kw.update(sampler_kw or {})
    s = pns.Sampler([dict(n=n, q=q, b=bb, betas=[float(beta)])], tape=2, **kw)
    burn = steps // 2 if burn is None else burn
    if burn:
        s.run(burn)  # burn-in records are not part of the moments
    s.run(steps)
    mom = s.moments(n, device=Q.device)
    s.close()
    return mom


def _grads(n, beta, mom, data_x=None, data_xx=None, data_E=0.0):
    dev = mom["mean_xx"].device
    dQ = torch.empty((n, n), dtype=torch.float64, device=dev)
    db = torch.empty(n, dtype=torch.float64, device=dev)
    dbeta = torch.empty(1, dtype=torch.float64, device=dev)
    dx = data_x.to(torch.float64).contiguous() if data_x is not None else None
    dxx = data_xx.to(torch.float64).contiguous() if data_xx is not None else None
    pns.pns_energy_grads(n, float(beta), mom["scalars"], mom["mean_x"], mom["mean_xx"], mom["cov_ex"],
                         mom["cov_exx"], dx, dxx, float(data_E), dQ, db, dbeta)
    return dQ, db, dbeta


class MeanEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q, b, beta, steps=2000, sampler_kw=None):
        mom = _run_moments(Q, b, float(beta), sampler_kw, steps)
        ctx.n = Q.shape[0]
        ctx.beta = float(beta)
        ctx.mom = mom
        ctx.dtypes = (Q.dtype, b.dtype, beta.dtype if torch.is_tensor(beta) else torch.float32)
        return mom["scalars"][1].to(Q.dtype)

    @staticmethod
    def backward(ctx, gE):
        dQ, db, dbeta = _grads(ctx.n, ctx.beta, ctx.mom)
        g = gE.to(torch.float64)
        return (g * dQ).to(ctx.dtypes[0]), (g * db).to(ctx.dtypes[1]), (g * dbeta[0]).to(ctx.dtypes[2]), None, None


class BoltzmannFit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q, b, beta, data_x, data_xx, steps=2000, sampler_kw=None):
        mom = _run_moments(Q, b, float(beta), sampler_kw, steps)
        out = torch.empty(1, dtype=torch.float64, device=Q.device)
        q32 = Q.detach().to(torch.float32).contiguous()
        b32 = b.detach().to(torch.float32).contiguous() if b is not None else None
        dx = data_x.detach().to(torch.float64).contiguous()
        pns.pns_data_energy(Q.shape[0], q32, b32, dx, data_xx.detach().to(torch.float64).contiguous(), out)
        data_E = float(out.item())
        ctx.n = Q.shape[0]
        ctx.beta = float(beta)
        ctx.mom = mom
        ctx.data = (data_x.detach(), data_xx.detach(), data_E)
        ctx.dtypes = (Q.dtype, b.dtype, beta.dtype if torch.is_tensor(beta) else torch.float32)
        return torch.tensor(-float(beta) * data_E, dtype=Q.dtype, device=Q.device)

    @staticmethod
    def backward(ctx, gl):
        dx, dxx, dE = ctx.data
        dQ, db, dbeta = _grads(ctx.n, ctx.beta, ctx.mom, dx, dxx, dE)
        g = gl.to(torch.float64)
        return ((g * dQ).to(ctx.dtypes[0]), (g * db).to(ctx.dtypes[1]), (g * dbeta[0]).to(ctx.dtypes[2]), None,
                None, None, None)


def mean_energy(Q, b, beta, steps=2000, **sampler_kw):
    return MeanEnergy.apply(Q, b, beta, steps, sampler_kw)


def boltzmann_fit(Q, b, beta, data_x, data_xx, steps=2000, **sampler_kw):
    return BoltzmannFit.apply(Q, b, beta, data_x, data_xx, steps, sampler_kw)


__all__ = ["MeanEnergy", "BoltzmannFit", "mean_energy", "boltzmann_fit", "np"]
