"""Oracle of continuous Unbiased PNS (Algorithm 7) and Metropolis on the
Donuts target (Sec. 7), pinned to closed forms and library routines:

  * the deterministic (cos 2 pi u, sin 2 pi u) against numpy in fp64;
  * the Box-Muller pairs against N(0, 1) (moments, Kolmogorov-Smirnov);
  * the Unbiased budget bookkeeping, sum M = L0 * stays + (L0 - L);
  * the multiplicity-weighted moments against the target's closed forms:
    x1^2 + x2^2 = mu ~ N(mu0, sigma^2) (truncation negligible at mu0/sigma =
    90) and the angle is uniform, so E[x_i] = 0, E[x_i^2] = mu0 / 2,
    E[x_i^4] = 3/8 (mu0^2 + sigma^2), P(x_i > 0) = 1/2.
"""
import numpy as np
import pytest

from oracle import oracle as O

MU0 = 9.0
SIGMA = 0.1
C = 1.0 / (2.0 * SIGMA * SIGMA)


def test_sincos2pi_against_numpy():
    u = (np.arange(1 << 20, dtype=np.float64) / (1 << 20)).astype(np.float32)
    c, s = O.sincos2pi(u)
    ang = 2.0 * np.pi * u.astype(np.float64)
    assert np.abs(c - np.cos(ang)).max() < 4e-7
    assert np.abs(s - np.sin(ang)).max() < 4e-7
    c4, s4 = O.sincos2pi(np.array([0.0, 0.25, 0.5, 0.75], np.float32))
    np.testing.assert_array_equal(c4, [1.0, 0.0, -1.0, 0.0])
    np.testing.assert_array_equal(s4, [0.0, 1.0, 0.0, -1.0])


def test_box_muller_pairs_are_standard_normal():
    from scipy import stats
    n = 200_000
    w0 = np.array([O.rng_word(5, 3, 7, i, 0) for i in range(n)], dtype=np.uint32)
    w1 = np.array([O.rng_word(5, 3, 7, i, 1) for i in range(n)], dtype=np.uint32)
    z1, z2 = O.normal_pairs(w0, w1)
    for z in (z1, z2):
        z = z.astype(np.float64)
        assert abs(z.mean()) < 5 / np.sqrt(n)
        assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
        assert stats.kstest(z, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(z1, z2)[0, 1]) < 5 / np.sqrt(n)


@pytest.mark.parametrize("L0", [100, 1000])
def test_unbiased_budget_bookkeeping(L0):
    r = O.donuts_chain("unbiased", 3, 5000, (3.0, 0.0), mu0=MU0, c=C, L0=L0, seed=2)
    stays = r["records"] - r["moves"]
    assert r["weight"] == L0 * stays + (L0 - r["budget_left"])


@pytest.mark.parametrize("variant,steps", [("unbiased", 20_000), ("metropolis", 400_000)])
def test_weighted_moments_match_closed_forms(variant, steps):
    chains = 16
    est = []
    for ch in range(chains):
        x0 = (3.0 * np.cos(ch), 3.0 * np.sin(ch))
        r = O.donuts_chain(variant, ch, steps, x0, mu0=MU0, c=C, L0=1000, seed=11)
        W = r["weight"]
        est.append(np.concatenate([r["sum_x"] / W, r["sum_x2"] / W, r["sum_x4"] / W, r["sum_pos"] / W,
                                   [(r["sum_x2"][0] + r["sum_x2"][1]) / W]]))
    est = np.array(est)
    mean = est.mean(0)
    se = est.std(0, ddof=1) / np.sqrt(chains)
    want = np.array([0.0, 0.0, MU0 / 2, MU0 / 2, 3 / 8 * (MU0 ** 2 + SIGMA ** 2), 3 / 8 * (MU0 ** 2 + SIGMA ** 2),
                     0.5, 0.5, MU0])
    z = np.abs(mean - want) / (se + 1e-3)
    assert z.max() < 6.0, (mean, want, se)
    assert abs(mean[-1] - MU0) < 0.02  # the ring radius is pinned far more tightly than the angle
