"""The C ABI without a GPU: the library builds, loads, exports every entry
point include/pns.h declares, its structs have the sizes the binding uses,
and argument validation fails cleanly before any device work."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2210_10513_gb300 import build as B
from paper_2210_10513_gb300 import pns

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pns.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return pns.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(pns_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert set(names) == set(pns.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", pns.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(pns_\w+)", out))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)


def test_struct_sizes_match_header():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "pns.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(pns_problem), sizeof(pns_config), sizeof(pns_info),
         sizeof(pns_stats), offsetof(pns_config, x0), offsetof(pns_stats, energy), sizeof(pns_donuts_config),
         sizeof(pns_donuts_stats), offsetof(pns_donuts_stats, x));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        exe = os.path.join(d, "s")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    want = [C.sizeof(pns.pns_problem), C.sizeof(pns.pns_config), C.sizeof(pns.pns_info), C.sizeof(pns.pns_stats),
            pns.pns_config.x0.offset, pns.pns_stats.energy.offset, C.sizeof(pns.pns_donuts_config),
            pns.DONUTS_STATS_DTYPE.itemsize, pns.DONUTS_STATS_DTYPE.fields["x"][1]]
    assert got == want


def _status_of(probs, cfg):
    arr = (pns.pns_problem * max(1, len(probs)))(*probs)
    ctx = C.c_void_p()
    return pns.lib().pns_create(C.cast(arr, C.c_void_p), len(probs), C.byref(cfg), None, C.byref(ctx)), ctx


def test_argument_validation_without_device(lib):
    q = np.zeros((8, 8), np.int32)
    keep = []
    good = pns.make_problem(8, q=q, betas=[1.0], keep=keep)
    cases = [
        (pns.make_config("unbiased", k=9), 1),           # k > n
        (pns.make_config("unbiased", k=0), 1),           # k < 1
        (pns.make_config("unbiased", k=2, L0=0), 1),     # L0 < 1
        (pns.make_config("basic", k=2, swap_interval=100), 1),  # exchange needs Unbiased / Metropolis
        (pns.make_config("unbiased", k=2, swap_interval=150, L0=100), 1),  # not a multiple of L0
        (pns.make_config("unbiased", k=2, warps_per_chain=3), 1),
        (pns.make_config("unbiased", k=2, chains_per_replica=0), 1),
    ]
    for cfg, want in cases:
        st, ctx = _status_of([good], cfg)
        assert st == want, (st, pns.pns_last_error())
        assert not ctx.value
        assert pns.pns_last_error()
    bad_q = pns.make_problem(8, q=np.zeros((8, 8), np.int64).astype(np.int32), betas=[1.0], keep=keep)
    bad_q.qtype = 7
    st, _ = _status_of([bad_q], pns.make_config("unbiased", k=2))
    assert st == 1
    # NULL context and NULL outputs
    assert lib.pns_run(None, 10, None) == 1
    assert lib.pns_read(None, None, None, None, None, None) == 1
    assert lib.pns_get_info(None, None) == 1
    lib.pns_destroy(None)


def test_device_work_fails_loudly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    q = np.zeros((8, 8), np.int32)
    keep = []
    st, ctx = _status_of([pns.make_problem(8, q=q, betas=[1.0], keep=keep)], pns.make_config("unbiased", k=2))
    assert st == 5  # PNS_ERR_CUDA, never a silent CPU path
    assert "cuda" in pns.pns_last_error().lower() or "device" in pns.pns_last_error().lower()


def test_binding_refuses_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(pns, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pns, "_lib", None)
    with pytest.raises(RuntimeError):
        pns.lib()
