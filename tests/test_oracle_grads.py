"""Pins for the exact-enumeration gradients used to check the backward:
central finite differences of the exact <E> and log Z (fp64, step h, error
O(h^2) ~ 1e-8 here)."""
import numpy as np

from oracle import exact as X
from paper_2210_10513_gb300 import synth


def _mean_energy(Q, b, beta):
    E = X.energies(Q, b)
    return float(X.boltzmann(E, beta) @ E)


def test_mean_energy_gradients_match_finite_differences():
    n = 8
    Q = synth.dense_normal(n, 0.6, 2).astype(np.float64)
    b = synth.vector_normal(n, 0.6, 2).astype(np.float64)
    beta = 0.9
    gQ, gb, gbeta, mE = X.mean_energy_grads(Q, b, beta)
    assert abs(mE - _mean_energy(Q, b, beta)) < 1e-12
    h = 1e-5
    for (i, j) in [(0, 0), (1, 3), (3, 1), (7, 2), (5, 5)]:
        Qp = Q.copy()
        Qp[i, j] += h
        Qm = Q.copy()
        Qm[i, j] -= h
        fd = (_mean_energy(Qp, b, beta) - _mean_energy(Qm, b, beta)) / (2 * h)
        assert abs(fd - gQ[i, j]) < 1e-7, (i, j, fd, gQ[i, j])
    for i in [0, 4, 7]:
        bp = b.copy()
        bp[i] += h
        bm = b.copy()
        bm[i] -= h
        fd = (_mean_energy(Q, bp, beta) - _mean_energy(Q, bm, beta)) / (2 * h)
        assert abs(fd - gb[i]) < 1e-7
    fd = (_mean_energy(Q, b, beta + h) - _mean_energy(Q, b, beta - h)) / (2 * h)
    assert abs(fd - gbeta) < 1e-7


def test_log_partition_derivatives_are_model_moments():
    n = 8
    Q = synth.dense_normal(n, 0.6, 4).astype(np.float64)
    b = synth.vector_normal(n, 0.6, 4).astype(np.float64)
    beta = 1.3
    m = X.exact_moments(Q, b, beta)
    h = 1e-5
    # d log Z / dQ_ij = -beta <x_i x_j>,  d log Z / dbeta = -<E>
    Qp = Q.copy()
    Qp[2, 5] += h
    Qm = Q.copy()
    Qm[2, 5] -= h
    fd = (X.log_partition(Qp, b, beta) - X.log_partition(Qm, b, beta)) / (2 * h)
    assert abs(fd + beta * m["xx"][2, 5]) < 1e-7
    fd = (X.log_partition(Q, b, beta + h) - X.log_partition(Q, b, beta - h)) / (2 * h)
    assert abs(fd + m["E"]) < 1e-7
    # the log-likelihood gradient vanishes when the data moments are the model's
    gQ, gb, gbeta = X.log_likelihood_grads(Q, b, beta, m["xx"], m["x"], m["E"])
    assert np.abs(gQ).max() < 1e-12 and np.abs(gb).max() < 1e-12 and abs(gbeta) < 1e-12
