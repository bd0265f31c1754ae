"""Pins for the oracle's counter-based generator and deterministic fp32 math.

Philox4x32-10 is checked against an independent implementation (Triton's
`philox_impl`, run by the Triton CPU interpreter); the fp32 log / exp /
-log1m routines against numpy's fp64 libm within stated ulp bounds.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _ulps(got, ref):
    ref32 = ref.astype(np.float32)
    sp = np.spacing(np.abs(ref32)).astype(np.float64)
    return np.abs(got.astype(np.float64) - ref) / sp


def _triton_philox(ctrs, key):
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    # A fresh interpreter, so that Triton starts in CPU-interpreter mode.
    req = json.dumps({"ctrs": np.asarray(ctrs, np.uint64).tolist(), "key": [int(key[0]), int(key[1])]})
    env = dict(os.environ, TRITON_INTERPRET="1")
    out = subprocess.run([sys.executable, "-m", "tests._triton_philox_ref"], input=req, capture_output=True,
                         text=True, cwd=ROOT, env=env, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    return np.array(json.loads(out.stdout), dtype=np.uint64).astype(np.uint32)


def test_philox_matches_independent_implementation():
    rng = np.random.default_rng(7)
    N = 64
    ctrs = rng.integers(0, 2**32, size=(N, 4), dtype=np.uint64).astype(np.uint32)
    ctrs[0] = 0
    ctrs[1] = 0xFFFFFFFF
    for key in [(0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (0x01234567, 0x89ABCDEF)]:
        ref = _triton_philox(ctrs, key)
        got = np.stack([O.philox(c, key) for c in ctrs])
        np.testing.assert_array_equal(got, ref)


def test_rng_word_counter_layout():
    seed = 0x0123456789ABCDEF
    for tag, ident, step, index in [(1, 5, 7, 0), (1, 5, 7, 6), (2, 0, 2**33 + 9, 3), (3, 99, 0, 1029)]:
        ctr = np.array([index >> 2, ident, step & 0xFFFFFFFF, (tag << 24) | ((step >> 32) & 0xFFFFFF)], np.uint32)
        ref = O.philox(ctr, (seed & 0xFFFFFFFF, seed >> 32))[index & 3]
        assert O.rng_word(seed, tag, ident, step, index) == ref


def test_philox_words_uniform():
    words = np.array([O.rng_word(1, 1, c, s, i) for c in range(8) for s in range(64) for i in range(16)],
                     dtype=np.uint32)
    counts = np.bincount(words >> 28, minlength=16)
    exp = len(words) / 16
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 45.0  # 15 dof, p ~ 1e-4


def test_logf_ulp_bound():
    rng = np.random.default_rng(1)
    grid = ((2 * np.arange(2**23, dtype=np.float64) + 1) * 2.0**-24).astype(np.float32)
    assert _ulps(O.logf(grid), np.log(grid.astype(np.float64))).max() <= 2.0
    assert O.logf(grid).max() < 0.0
    x = rng.random(2 * 10**6).astype(np.float32)
    x = x[x > 0]
    assert _ulps(O.logf(x), np.log(x.astype(np.float64))).max() <= 2.0
    t = (rng.random(10**5) * 2.0**-60).astype(np.float32)
    t = t[t > 2.0**-126]
    assert _ulps(O.logf(t), np.log(t.astype(np.float64))).max() <= 2.0
    assert O.logf(np.array([1.0], np.float32))[0] == 0.0


def test_expf_ulp_bound_and_edges():
    y = np.linspace(-87.0, 0.0, 2 * 10**6).astype(np.float32)
    assert _ulps(O.expf(y), np.exp(y.astype(np.float64))).max() <= 2.0
    e = O.expf(np.array([0.0, -0.0, -87.5, -1000.0, -np.inf], np.float32))
    assert e[0] == 1.0 and e[1] == 1.0 and e[2] == 0.0 and e[3] == 0.0 and e[4] == 0.0


def test_neg_log1m_bound():
    rng = np.random.default_rng(2)
    v = rng.random(2 * 10**6).astype(np.float32)
    v = v[(v > 0) & (v < 1)]
    ref = -np.log1p(-v.astype(np.float64))
    assert _ulps(O.neg_log1m(v), ref).max() <= 6.0
    s = (rng.random(10**5) * 2.0**-30).astype(np.float32)
    s = s[s > 0]
    assert _ulps(O.neg_log1m(s), -np.log1p(-s.astype(np.float64))).max() <= 2.0
    assert (O.neg_log1m(v) > 0).all()


def test_fine_uniforms():
    rng = np.random.default_rng(3)
    w = rng.integers(1, 2**32, size=10**6, dtype=np.uint64).astype(np.uint32)
    w[:1000] = rng.integers(1, 2**23, size=1000, dtype=np.uint64).astype(np.uint32)
    v = O.uniform_fine32(w).astype(np.float64)
    assert (v > 0).all() and (v < 1).all()
    wf = w.astype(np.float64)
    # below 2^23 every bit is kept and v lies in the cell [w, w+1) 2^-32;
    # above, 23 bits below the leading one are kept: within 2^-22 relative
    big = w >= 2**23
    small = ~big
    assert (v[small] >= wf[small] * 2.0**-32).all() and (v[small] <= (wf[small] + 1) * 2.0**-32).all()
    ideal = (wf[big] + 0.5) * 2.0**-32
    assert (np.abs(v[big] - ideal) <= 2.0**-22 * ideal).all()
    w64 = rng.integers(1, 2**63, size=10**5, dtype=np.uint64) * np.uint64(2)
    v64 = O.uniform_fine64(w64).astype(np.float64)
    ideal64 = w64.astype(np.float64) * 2.0**-64
    assert (v64 > 0).all() and (v64 < 1).all()
    assert (np.abs(v64 - ideal64) <= 2.0**-22 * ideal64).all()
    edge = O.uniform_fine32(np.array([0, 1, 0xFFFFFFFF], np.uint32))
    assert 0 < edge[0] < edge[1] < 1e-9 and edge[2] < 1.0
