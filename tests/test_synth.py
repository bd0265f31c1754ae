"""The seeded input generators follow the recipe the workloads are stated in:
symmetric matrices with the stated entry laws, the periodic lattice's
neighbourhoods, the temperature ladder, the bit packing the C ABI uses, and
determinism per seed (CPU only)."""
import numpy as np
import pytest

from paper_2210_10513_gb300 import synth


def test_dense_int_symmetric_in_range_and_seeded():
    q = synth.dense_int(300, -100, 100, 5, np.int16)
    assert q.dtype == np.int16 and q.shape == (300, 300)
    np.testing.assert_array_equal(q, q.T)
    assert q.min() >= -100 and q.max() <= 100
    # the upper triangle is i.i.d. uniform on the 201 integers: every value occurs
    up = q[np.triu_indices(300)]
    assert len(np.unique(up)) == 201
    assert abs(float(up.mean())) < 3 * 58.0 / np.sqrt(up.size)  # sd of U{-100..100} is 58.0
    np.testing.assert_array_equal(q, synth.dense_int(300, -100, 100, 5, np.int16))
    assert not np.array_equal(q, synth.dense_int(300, -100, 100, 6, np.int16))
    b = synth.vector_int(300, -100, 100, 5, np.int16)
    assert b.dtype == np.int16 and b.min() >= -100 and b.max() <= 100


def test_dense_normal_is_symmetrised_gaussian():
    n, sigma = 400, 1.0
    q = synth.dense_normal(n, sigma, 3)
    assert q.dtype == np.float32
    np.testing.assert_array_equal(q, q.T)
    # (A + A^T)/2: off-diagonal variance sigma^2/2, diagonal variance sigma^2
    off = q[np.triu_indices(n, 1)].astype(np.float64)
    dia = np.diag(q).astype(np.float64)
    assert abs(off.var() - sigma ** 2 / 2) < 0.02
    assert abs(dia.var() - sigma ** 2) < 0.25
    assert abs(off.mean()) < 0.01


def test_upper_triangular_qubo_convention():
    # E = x^T Q x with Q = -(U + U^T)/2 equals -x^T U x for every x
    n = 10
    q = synth.upper_triangular_qubo(n, 10.0, 1)
    np.testing.assert_array_equal(q, q.T)
    g = np.random.Generator(np.random.PCG64([1, 2]))
    u = np.triu(g.standard_normal(size=(n, n)) * 10.0).astype(np.float32)
    x = synth.random_bits(50, n, 3).astype(np.float64)
    e_ours = np.einsum("ci,ij,cj->c", x, q.astype(np.float64), x)
    e_paper = np.einsum("ci,ij,cj->c", x, u.astype(np.float64), x)
    np.testing.assert_allclose(e_ours, -e_paper, rtol=1e-6, atol=1e-4)


def test_lattice_csr_neighbourhoods():
    side = 12
    row_ptr, col, val, diag = synth.lattice_csr(side, 4)
    n = side * side
    assert len(row_ptr) == n + 1 and (np.diff(row_ptr) == 4).all()
    assert set(np.unique(val)) <= {-1, 1} and diag.min() >= -2 and diag.max() <= 2
    q = synth.csr_to_dense(row_ptr, col, val, diag)
    np.testing.assert_array_equal(q, q.T)
    for i in range(n):
        r, c = divmod(i, side)
        nb = {r * side + (c - 1) % side, r * side + (c + 1) % side, ((r - 1) % side) * side + c,
              ((r + 1) % side) * side + c}
        assert set(col[row_ptr[i]:row_ptr[i + 1]].tolist()) == nb
        assert np.count_nonzero(q[i]) - (1 if q[i, i] != 0 else 0) == 4
    # couplings are fair coins: both signs occur in about equal numbers
    assert abs(float(val.mean())) < 0.2


def test_geometric_ladder():
    b = synth.geometric_ladder(0.1, 10.0, 8)
    assert b.dtype == np.float32 and len(b) == 8
    assert b[0] == np.float32(0.1) and abs(b[-1] - 10.0) < 1e-5
    ratios = b[1:].astype(np.float64) / b[:-1]
    np.testing.assert_allclose(ratios, (100.0) ** (1 / 7), rtol=1e-6)
    assert synth.geometric_ladder(0.3, 5.0, 1).tolist() == [np.float32(0.3)]


@pytest.mark.parametrize("n", [1, 31, 32, 33, 100])
def test_pack_unpack_round_trip(n):
    bits = synth.random_bits(5, n, n)
    words = synth.pack_bits(bits)
    assert words.shape == (5, (n + 31) // 32) and words.dtype == np.uint32
    np.testing.assert_array_equal(synth.unpack_bits(words, n), bits)
    # bit i of a chain is bit i % 32 of word i // 32
    for c in range(5):
        for i in range(n):
            assert (int(words[c, i // 32]) >> (i % 32)) & 1 == bits[c, i]


def test_benchmark_workload_shapes():
    probs, ladder = synth.workload_tempering(64, seed=0)
    ns = np.array([p["n"] for p in probs])
    assert len(probs) == 64 and ns.min() >= 128 and ns.max() <= 2048
    assert all(p["q"].shape == (p["n"], p["n"]) and p["q"].dtype == np.float32 for p in probs)
    assert len(ladder) == 8
    wl = synth.workload_dense_int1024(0)
    assert wl["q"].dtype == np.int16 and wl["q"].shape == (1024, 1024) and wl["b"].shape == (1024,)
    assert (wl["beta"], wl["chains"], wl["k"]) == (0.05, 256, 64)
    fit = synth.workload_fit(64, 0)
    assert fit["q"].shape == (64, 64) and fit["b"].dtype == np.float32
