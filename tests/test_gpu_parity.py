"""CUDA sampler vs the CPU oracle, record by record, through the C ABI.

Integer QUBOs: bit-exact flip tapes, multiplicities, states, fields, energies
and statistics.  fp32 QUBOs: the same, because both sides take every
decision in fp32 with one operation order (the fields are then bit-equal
too); the fp64-recomputed fields are within 1e-5 relative.
"""
import numpy as np
import pytest

from paper_2210_10513_gb300 import synth
from tests.gpu_helpers import assert_chain_equal, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def _int_problem(n, lo=-100, hi=100, seed=0, dtype=np.int16, b=True, betas=(0.05,)):
    return dict(n=n, q=synth.dense_int(n, lo, hi, seed, dtype),
                b=synth.vector_int(n, lo, hi, seed, dtype) if b else None, betas=list(betas))


def _check_all(problems, steps, chains, **cfg):
    g = gpu_run(problems, steps, tape=True, **cfg)
    ids = list(range(chains))
    ref = oracle_run(problems, steps, ids, **cfg)
    for cid in ids:
        n = problems[ref[cid]["instance"]]["n"]
        assert_chain_equal(g, ref[cid], cid, n, steps)
    return g


@pytest.mark.parametrize("variant,k,subset", [("rf", 16, "systematic"), ("basic", 4, "systematic"),
                                              ("unbiased", 4, "systematic"), ("unbiased", 4, "random"),
                                              ("metropolis", 1, "systematic")])
def test_small_dense_n16(variant, k, subset):
    p = dict(n=16, q=synth.dense_int(16, -8, 8, 0, np.int32), b=None, betas=[1.0])
    _check_all([p], 3000, 8, variant=variant, k=k, subset=subset, chains_per_replica=8, seed=3)


@pytest.mark.parametrize("variant", ["basic", "unbiased"])
def test_dense_int16_n1024(variant):
    p = _int_problem(1024)
    _check_all([p], 1500, 6, variant=variant, k=64, chains_per_replica=6, seed=11)


@pytest.mark.parametrize("n,k,subset", [(200, 13, "systematic"), (200, 13, "random"), (37, 37, "systematic"),
                                        (33, 1, "systematic"), (1, 1, "systematic")])
def test_ragged_sizes(n, k, subset):
    p = _int_problem(n, lo=-30, hi=30, seed=n, dtype=np.int32, betas=(0.3,))
    _check_all([p], 2000, 4, variant="unbiased", k=k, subset=subset, chains_per_replica=4, seed=5, L0=50)


@pytest.mark.parametrize("variant,k", [("unbiased", 17), ("basic", 9), ("rf", 300), ("metropolis", 1)])
def test_fp32_dense(variant, k):
    n = 300
    p = dict(n=n, q=synth.dense_normal(n, 1.0, 2), b=synth.vector_normal(n, 0.5, 2), betas=[0.7])
    g = _check_all([p], 1500, 4, variant=variant, k=k, chains_per_replica=4, seed=2)
    # fields against an fp64 recomputation from the final states
    bits = synth.unpack_bits(g["states"][:4], n).astype(np.float64)
    h64 = bits @ p["q"].astype(np.float64) + p["b"].astype(np.float64)
    scale = np.abs(p["q"]).sum(1).max()
    assert np.abs(g["fields"][:4, :n] - h64).max() <= 1e-5 * scale


def test_random_initial_states_and_multiple_instances():
    probs = [_int_problem(96, seed=1, dtype=np.int32, betas=(0.05, 0.2)),
             _int_problem(160, seed=2, dtype=np.int32, betas=(0.1,))]
    chains = 2 * 3 + 1 * 3
    W = 160 // 32
    bits = np.zeros((chains, 160), np.uint8)
    rb = synth.random_bits(chains, 160, seed=4)
    ns = [96] * 6 + [160] * 3
    for c in range(chains):
        bits[c, :ns[c]] = rb[c, :ns[c]]
    x0 = synth.pack_bits(bits)
    assert x0.shape == (chains, W)
    g = gpu_run(probs, 1000, tape=True, variant="unbiased", k=8, chains_per_replica=3, seed=9, x0=x0)
    ref = oracle_run(probs, 1000, list(range(chains)), x0=x0, variant="unbiased", k=8, chains_per_replica=3, seed=9)
    for cid in range(chains):
        assert_chain_equal(g, ref[cid], cid, ns[cid], 1000)


@pytest.mark.parametrize("T", [1, 4, 8])
def test_csr_lattice(T):
    side = 16
    csr = synth.lattice_csr(side, seed=3)
    p = dict(n=side * side, csr=csr, b=None, betas=[0.44])
    g = _check_all([p], 2000, 3, variant="unbiased", k=64, chains_per_replica=3, seed=4, warps_per_chain=T)
    assert g["info"].field_bytes == 1  # |h| <= 6 fits int8


def test_mapping_does_not_change_results(monkeypatch):
    p = _int_problem(256, dtype=np.int32)
    base = gpu_run([p], 800, tape=True, variant="unbiased", k=40, chains_per_replica=12, seed=1, warps_per_chain=1)
    for T in (2, 4):
        o = gpu_run([p], 800, tape=True, variant="unbiased", k=40, chains_per_replica=12, seed=1, warps_per_chain=T)
        np.testing.assert_array_equal(o["flips"], base["flips"])
        np.testing.assert_array_equal(o["m"], base["m"])
        np.testing.assert_array_equal(o["fields"], base["fields"])
    monkeypatch.setenv("PNS_CHAINS_PER_CTA", "5")
    o = gpu_run([p], 800, tape=True, variant="unbiased", k=40, chains_per_replica=12, seed=1, warps_per_chain=1)
    np.testing.assert_array_equal(o["flips"], base["flips"])
    np.testing.assert_array_equal(o["m"], base["m"])


def test_host_inputs_equal_device_inputs():
    p = _int_problem(128, dtype=np.int16)
    a = gpu_run([p], 500, tape=True, device_inputs=True, variant="basic", k=16, chains_per_replica=4, seed=2)
    b = gpu_run([p], 500, tape=True, device_inputs=False, variant="basic", k=16, chains_per_replica=4, seed=2)
    np.testing.assert_array_equal(a["flips"], b["flips"])
    np.testing.assert_array_equal(a["m"], b["m"])


def test_consecutive_runs_continue_the_chain():
    p = _int_problem(64, dtype=np.int32)
    two = gpu_run([p], 700, runs=2, tape=True, variant="unbiased", k=8, chains_per_replica=3, seed=6)
    one = gpu_run([p], 1400, tape=True, variant="unbiased", k=8, chains_per_replica=3, seed=6)
    first, second = two["all"]
    np.testing.assert_array_equal(np.concatenate([first["flips"], second["flips"]], axis=1), one["flips"])
    np.testing.assert_array_equal(np.concatenate([first["m"], second["m"]], axis=1), one["m"])
    np.testing.assert_array_equal(two["states"], one["states"])


@pytest.mark.parametrize("subset", ["random", "systematic"])
def test_checkpoint_restore_bit_identical(subset):
    # (random sets: the speculative kernel; systematic: the set sweep)
    from paper_2210_10513_gb300 import pns
    from tests.gpu_helpers import to_dev
    p = dict(n=100, q=synth.dense_normal(100, 1.0, 8), b=synth.vector_normal(100, 1.0, 8), betas=[0.5])
    s = pns.Sampler([dict(n=100, q=to_dev(p["q"]), b=to_dev(p["b"]), betas=[0.5])], variant="unbiased", k=10,
                    subset=subset, chains_per_replica=4, seed=3, tape=True)
    assert s.info.set_sweep == (1 if subset == "systematic" else 0)
    s.run(500)
    ck = s.checkpoint()
    s.run(600)
    a = s.read()
    fa = s.fields()
    s.restore(ck)
    s.run(600)
    b = s.read()
    fb = s.fields()
    s.close()
    np.testing.assert_array_equal(a["flips"], b["flips"])
    np.testing.assert_array_equal(a["m"], b["m"])
    np.testing.assert_array_equal(a["states"], b["states"])
    np.testing.assert_array_equal(fa, fb)
    np.testing.assert_array_equal(a["stats"], b["stats"])


def test_rf_equals_unbiased_full_set():
    p = _int_problem(48, dtype=np.int32, betas=(0.2,))
    a = gpu_run([p], 1000, tape=True, variant="rf", chains_per_replica=2, seed=5)
    b = gpu_run([p], 1000, tape=True, variant="unbiased", k=48, L0=2**62, chains_per_replica=2, seed=5)
    np.testing.assert_array_equal(a["flips"], b["flips"])
    np.testing.assert_array_equal(a["m"], b["m"])


def test_beta_zero_and_budget_one():
    p = _int_problem(40, dtype=np.int32, betas=(0.0,))
    _check_all([p], 500, 2, variant="unbiased", k=5, L0=1, chains_per_replica=2, seed=8)
    _check_all([p], 500, 2, variant="basic", k=40, chains_per_replica=2, seed=8)


@pytest.mark.parametrize("bad", ["asym", "nan", "range", "k", "csr_mirror"])
def test_invalid_inputs_rejected(bad):
    from paper_2210_10513_gb300 import pns
    n = 8
    q = synth.dense_int(n, -3, 3, 0, np.int32)
    kw = dict(variant="unbiased", k=2)
    prob = dict(n=n, q=q, betas=[1.0])
    expect = pns.PnsError
    if bad == "asym":
        q = q.copy()
        q[0, 1] += 1
        prob["q"] = q
        status = 2
    elif bad == "nan":
        qf = synth.dense_normal(n, 1.0, 0)
        qf[2, 2] = np.nan
        prob["q"] = qf
        status = 3
    elif bad == "range":
        q = np.full((n, n), 2**28, dtype=np.int32)
        prob["q"] = q
        status = 3
    elif bad == "k":
        kw["k"] = n + 1
        status = 1
    else:
        row_ptr, col, val, diag = synth.lattice_csr(4, seed=1)
        val = val.copy()
        val[0] = -val[0] if val[0] != 0 else 1
        prob = dict(n=16, csr=(row_ptr, col, val, diag), betas=[1.0])
        status = 2
    with pytest.raises(expect) as ei:
        pns.Sampler([prob], **kw)
    assert ei.value.status == status


def test_sharded_contexts_equal_one_context():
    """Instances split over two contexts (as over two GPUs) with chain_base /
    group_base give the records of the single context."""
    probs = [_int_problem(64, seed=3, dtype=np.int32, betas=(0.1, 0.2)),
             _int_problem(96, seed=4, dtype=np.int32, betas=(0.3, 0.4))]
    cfg = dict(variant="unbiased", k=8, chains_per_replica=3, seed=5)
    whole = gpu_run(probs, 600, tape=True, **cfg)
    a = gpu_run(probs[:1], 600, tape=True, **cfg)
    b = gpu_run(probs[1:], 600, tape=True, chain_base=6, group_base=3, **cfg)
    np.testing.assert_array_equal(np.concatenate([a["flips"], b["flips"]]), whole["flips"])
    np.testing.assert_array_equal(np.concatenate([a["m"], b["m"]]), whole["m"])


@pytest.mark.parametrize("form", ["per_flip_basic", "sweep", "spec_random", "blocked"])
def test_zero_steps_change_nothing(form):
    """A run of 0 records (0 original samples with exchange) changes nothing:
    states, fields and statistics stay as created, and the next run's records
    are those of a context that never made the empty run."""
    from paper_2210_10513_gb300 import pns
    from tests.gpu_helpers import to_dev
    if form == "blocked":
        betas = synth.geometric_ladder(0.1, 5.0, 4)
        probs = [dict(n=96, q=synth.dense_normal(96, 1.0, 1), b=None, betas=betas, k=6)]
        cfg = dict(variant="unbiased", k=1, L0=50, swap_interval=100, seed=3, chains_per_replica=1)
        steps = 400
    else:
        probs = [_int_problem(256, lo=-40, hi=40, seed=2, dtype=np.int32, betas=(0.1,))]
        cfg = dict(variant="basic" if form == "per_flip_basic" else "unbiased", k=16,
                   subset="random" if form == "spec_random" else "systematic", L0=100, seed=3,
                   chains_per_replica=4)
        steps = 500

    def make():
        return pns.Sampler([dict(d, q=to_dev(d["q"]), b=to_dev(d.get("b"))) for d in probs], tape=True, **cfg)

    a, b = make(), make()
    info = a.info
    want = dict(per_flip_basic=(0, 0, 0), sweep=(8, 1, 0), spec_random=(8, 0, 0), blocked=(0, 0, 1))[form]
    assert (info.spec_depth, info.set_sweep, info.period_blocked) == want
    before, f0 = a.read(), a.fields()
    a.run(0)
    after, f1 = a.read(), a.fields()
    np.testing.assert_array_equal(before["states"], after["states"])
    np.testing.assert_array_equal(before["stats"], after["stats"])
    np.testing.assert_array_equal(f0, f1)
    a.run(steps)
    b.run(steps)
    ra, rb = a.read(), b.read()
    for key in ("states", "stats", "flips", "m"):
        np.testing.assert_array_equal(ra[key], rb[key], err_msg=key)
    np.testing.assert_array_equal(a.fields(), b.fields())
    a.close()
    b.close()


def test_donuts_zero_steps():
    from paper_2210_10513_gb300 import pns
    x0 = np.array([[3.0, 0.5], [-1.0, 2.0], [0.0, -3.0]], np.float32)
    st = pns.pns_donuts_run("unbiased", 3, 0, x0=x0, L0=1000, seed=1)
    assert (st["records"] == 0).all() and (st["moves"] == 0).all() and (st["weight"] == 0).all()
    assert (st["budget_left"] == 1000).all() and (st["period_start"] == 0).all()
    np.testing.assert_array_equal(st["x"], x0)


@pytest.mark.parametrize("variant,k", [("basic", 16), ("rf", 64), ("unbiased", 16)])
def test_saturated_multiplicity(variant, k):
    """Q = 1000 I at beta = 1: from the all-zero state every flip costs 1000,
    the weights underflow, p = 0 and M saturates at 2^63 (counted) for Basic
    and RF, which move anyway; a flip back has weight 1.  Unbiased PNS cannot
    fit a saturated M in its budget, so those records stay with M = L."""
    n = 64
    q = np.zeros((n, n), np.int32)
    np.fill_diagonal(q, 1000)
    p = dict(n=n, q=q, b=None, betas=[1.0])
    g = _check_all([p], 400, 4, variant=variant, k=k, chains_per_replica=4, seed=9, L0=100)
    m = g["m"][:4, :400]
    if variant == "unbiased":
        assert (g["stats"]["saturated"][:4] == 0).all()
        assert (g["stats"]["stays"][:4] == 400).all() and (m == 100.0).all()
    else:
        assert (g["stats"]["saturated"][:4] > 0).all()
        np.testing.assert_array_equal((m == 2.0 ** 63).sum(axis=1), g["stats"]["saturated"][:4])


@pytest.mark.parametrize("subset", ["systematic", "random"])
def test_largest_budget_of_the_fast_kernels(subset):
    """L0 = 2^31 - 1, the largest budget the set-sweep and speculative kernels
    take (their budget test runs in 32-bit integers)."""
    p = _int_problem(128, lo=-30, hi=30, seed=6, dtype=np.int32, betas=(0.2,))
    g = _check_all([p], 2000, 4, variant="unbiased", k=16, subset=subset, chains_per_replica=4, seed=12,
                   L0=2 ** 31 - 1)
    assert g["info"].spec_depth == 8 and g["info"].set_sweep == (1 if subset == "systematic" else 0)


@pytest.mark.parametrize("src,dst", [("sweep", "per_flip"), ("per_flip", "sweep"), ("per_flip", "spec")])
def test_checkpoint_moves_between_kernel_forms(monkeypatch, src, dst):
    """A checkpoint holds the chains, not the kernel: restored into a context
    that runs another kernel form, the chains continue with the same records."""
    from paper_2210_10513_gb300 import pns
    from tests.gpu_helpers import to_dev
    env = dict(sweep=("8", "1"), spec=("8", "0"), per_flip=("0", "0"))
    p = _int_problem(256, lo=-40, hi=40, seed=4, dtype=np.int32, betas=(0.1,))

    def make(form):
        monkeypatch.setenv("PNS_SPEC_DEPTH", env[form][0])
        monkeypatch.setenv("PNS_SWEEP", env[form][1])
        s = pns.Sampler([dict(n=256, q=to_dev(p["q"]), b=to_dev(p["b"]), betas=p["betas"])], variant="unbiased",
                        k=16, chains_per_replica=3, seed=7, L0=100, tape=True)
        assert (s.info.spec_depth, s.info.set_sweep) == (int(env[form][0]), int(env[form][1]))
        return s

    a = make(src)
    a.run(700)
    ck = a.checkpoint()
    a.run(700)
    ra, fa = a.read(), a.fields()
    b = make(dst)
    b.restore(ck)
    b.run(700)
    rb, fb = b.read(), b.fields()
    a.close()
    b.close()
    for key in ("states", "stats", "flips", "m"):
        np.testing.assert_array_equal(ra[key], rb[key], err_msg=key)
    np.testing.assert_array_equal(fa, fb)


@pytest.mark.parametrize("case", ["asym_lower", "asym_upper", "asym_int16", "nan_lower", "b_inf", "range_int32",
                                  "range_fp32", "valid"])
def test_create_checks_span_tiles(case):
    """pns_create's checks run in 32 x 32 tiles: n = 77 spans three tile rows
    with a ragged last one.  A broken symmetry or a non-finite entry in any
    tile, or a field bound reached only by summing a row over several tiles,
    is rejected with the status of Sec. 4's input rules; a valid instance
    passes."""
    from paper_2210_10513_gb300 import pns
    n = 77
    q = synth.dense_int(n, -3, 3, 4, np.int32)
    b = None
    status = None
    if case == "asym_lower":
        q = q.copy()
        q[70, 3] += 1
        status = 2
    elif case == "asym_upper":
        q = q.copy()
        q[3, 70] += 1
        status = 2
    elif case == "asym_int16":
        q = q.astype(np.int16)
        q[40, 66] += 1
        status = 2
    elif case == "nan_lower":
        q = synth.dense_normal(n, 1.0, 4)
        q[75, 40] = np.nan
        status = 3
    elif case == "b_inf":
        q = synth.dense_normal(n, 1.0, 4)
        b = synth.vector_normal(n, 1.0, 4)
        b[76] = np.inf
        status = 3
    elif case == "range_int32":
        # row 50: 77 entries of 1e7, each tile's part (32 e7) below the
        # 715,827,882 limit, the whole row above it
        q = q.copy()
        q[50, :] = 10 ** 7
        q[:, 50] = 10 ** 7
        status = 3
    elif case == "range_fp32":
        q = synth.dense_normal(n, 1.0, 4)
        q[40, :] = 2e28
        q[:, 40] = 2e28
        status = 3
    prob = dict(n=n, q=q, b=b, betas=[1.0])
    if status is None:
        s = pns.Sampler([prob], variant="unbiased", k=7)
        s.run(100)
        assert s.read()["stats"]["steps"].min() == 100
        s.close()
        return
    with pytest.raises(pns.PnsError) as ei:
        pns.Sampler([prob], variant="unbiased", k=7)
    assert ei.value.status == status, (case, ei.value.status)
