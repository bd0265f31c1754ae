"""Shared helpers of the GPU parity tests: run the CUDA sampler through the
C ABI and the CPU oracle on the same seeded inputs."""
import numpy as np

from oracle import oracle as O
from paper_2210_10513_gb300 import synth


def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def to_dev(a):
    if a is None:
        return None
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_run(problems, steps, device_inputs=True, runs=1, **cfg):
    """problems: list of dicts (n, q | csr, b, betas) with numpy arrays."""
    from paper_2210_10513_gb300 import pns
    probs = []
    for p in problems:
        d = dict(p)
        if device_inputs:
            if d.get("q") is not None:
                d["q"] = to_dev(d["q"])
            if d.get("b") is not None:
                d["b"] = to_dev(d["b"])
            if d.get("csr") is not None:
                d["csr"] = tuple(to_dev(a) for a in d["csr"])
        probs.append(d)
    s = pns.Sampler(probs, **cfg)
    outs = []
    for _ in range(runs):
        s.run(steps)
        outs.append(s.read())
    out = outs[-1]
    out["fields"] = s.fields()
    out["info"] = s.info
    out["all"] = outs
    s.close()
    return out


def oracle_problem(p):
    if p.get("csr") is not None:
        return O.Problem(csr=p["csr"], b=p.get("b"))
    return O.Problem(q=p["q"], b=p.get("b"))


def oracle_run(problems, steps, chain_ids, x0=None, **cfg):
    okw = dict(variant=cfg.get("variant", "unbiased"), k=cfg.get("k", 1), subset=cfg.get("subset", "systematic"),
               L0=cfg.get("L0", 100), seed=cfg.get("seed", 0), anneal_start=cfg.get("anneal_start", 1.0),
               anneal_steps=cfg.get("anneal_steps", 0))
    oprobs = [oracle_problem(p) for p in problems]
    betas = [list(np.asarray(p["betas"], dtype=np.float32)) for p in problems]
    x0d = None
    if x0 is not None:
        x0d = {}
        for cid in chain_ids:
            inst = _instance_of(problems, cfg.get("chains_per_replica", 1), cid)
            x0d[cid] = synth.unpack_bits(x0[cid:cid + 1], problems[inst]["n"])[0]
    return O.run_independent(oprobs, betas, okw, cfg.get("chains_per_replica", 1), x0d, steps, chain_ids=chain_ids)


def _instance_of(problems, cpr, cid):
    for p, _, _, c, _ in O.chain_layout([len(np.atleast_1d(pr["betas"])) for pr in problems], cpr):
        if c == cid:
            return p
    raise KeyError(cid)


def assert_chain_equal(gpu, ref, cid, n, steps, check_fields=True):
    rec = int(gpu["stats"]["tape_records"][cid])
    assert rec == len(ref["flips"])
    if steps is not None:
        assert rec == steps
    np.testing.assert_array_equal(gpu["flips"][cid, :rec], ref["flips"], err_msg="flip tape, chain %d" % cid)
    np.testing.assert_array_equal(gpu["m"][cid, :rec], ref["m"], err_msg="multiplicities, chain %d" % cid)
    bits = synth.unpack_bits(gpu["states"][cid:cid + 1], n)[0]
    np.testing.assert_array_equal(bits, ref["x"], err_msg="final state, chain %d" % cid)
    st = gpu["stats"][cid]
    rs = ref["state"]
    assert st["energy"] == rs.E, (cid, st["energy"], rs.E)
    assert st["sum_m"] == rs.sum_m
    assert st["flips"] == rs.flips and st["stays"] == rs.stays and st["saturated"] == rs.saturated
    assert st["budget_left"] == rs.L and st["set_start"] == rs.set_start and st["steps"] == rs.step
    assert st["best_energy"] == rs.best_E
    if check_fields:
        f = gpu["fields"][cid, :n]
        if f.dtype.kind == "f":
            np.testing.assert_array_equal(f.view(np.uint32), ref["h"].astype(np.float32).view(np.uint32),
                                          err_msg="fields, chain %d" % cid)
        else:
            np.testing.assert_array_equal(f.astype(np.int64), ref["h"].astype(np.int64), err_msg="fields %d" % cid)
