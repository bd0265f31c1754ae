"""Independent Philox4x32-10: Triton's `philox_impl`, executed by the Triton
CPU interpreter.  Imported lazily by the RNG pin test only."""
import os

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402
from triton.language.random import philox_impl  # noqa: E402


@triton.jit
def _kern(c0p, c1p, c2p, c3p, k0p, k1p, o0, o1, o2, o3, N: tl.constexpr):
    i = tl.arange(0, N)
    a, b, c, d = philox_impl(tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i),
                             tl.load(k0p + i), tl.load(k1p + i), 10)
    tl.store(o0 + i, a)
    tl.store(o1 + i, b)
    tl.store(o2 + i, c)
    tl.store(o3 + i, d)


def philox_rows(ctrs, key):
    ctrs = np.ascontiguousarray(ctrs, dtype=np.uint32)
    N = ctrs.shape[0]
    cols = [torch.from_numpy(np.ascontiguousarray(ctrs[:, j]).view(np.int32)).view(torch.uint32) for j in range(4)]
    ks = [torch.from_numpy(np.full(N, key[j], np.uint32).view(np.int32)).view(torch.uint32) for j in range(2)]
    outs = [torch.zeros(N, dtype=torch.uint32) for _ in range(4)]
    _kern[(1,)](*cols, *ks, *outs, N=N)
    return np.stack([o.view(torch.int32).numpy().view(np.uint32) for o in outs], axis=1)


if __name__ == "__main__":
    import json
    import sys

    req = json.load(sys.stdin)
    out = philox_rows(np.array(req["ctrs"], dtype=np.uint64).astype(np.uint32), req["key"])
    json.dump(out.astype(np.uint64).tolist(), sys.stdout)
