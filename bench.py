"""Benchmark of the batched PNS sampler on one GB300 (or N, one process each).

Default workload (the headline line): batched uneven parallel tempering.
512 fp32 QUBO instances with n uniform in [128, 2048] and Q = (A + A^T)/2,
A i.i.d. N(0, 1), b = 0; 8 replicas per instance on the geometric beta ladder
0.1 .. 10 (4096 chains); Unbiased PNS on systematic sets of k = max(1, n // 16)
with L0 = 100; adjacent temperatures exchange every 100 original samples.
One bench step = one pns_run of `--samples` (default 10,000) original samples
for every chain, i.e. 100 exchange rounds.  The metric is jump samples
(records) per second over all chains; flips/s and original (Metropolis-
equivalent) samples/s are reported beside it, and the roofline counts one
fp32 row of Q (4 n bytes) per flip against the measured HBM copy bandwidth.

The line also carries the end-to-end rate through the public API (instances
copied in from pinned host memory, create + run + read per step), the CPU
oracle timed on the host cores (`cpu_baseline`), the one-group-per-launch
form (`batched_over_plain`) and, unless `--quick`, the dense int16 n = 1024
workload's figures with its L2-side roofline (`dense1024`).

With torchrun (N > 1) the workload grows with N (`--instances` per GPU) and
all N x 512 instances are sharded across ranks by n^2 (whole exchange groups,
no data-path collective): weak scaling; the value is the records of all ranks
over the slowest rank's time.

`--impl reference` times the CPU oracle instead (a bounded sample of the same
workload on the host cores).  `--workload dense1024|lattice|fit|donuts` prints
the other benchmark shapes.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2210_10513_gb300 import synth  # noqa: E402

# ---- tempering workload ---------------------------------------------------------
T_INST = 512
T_REPLICAS = 8
T_L0 = 100
T_SWAP = 100

# ---- dense int16 workload -----------------------------------------------------------
N = 1024
K = 64
CHAINS = 256
BETA = 0.05
L0 = 100
ROW_BYTES = N * 2  # one int16 row of Q per flip


def workload(seed):
    q = synth.dense_int(N, -100, 100, seed, np.int16)
    b = synth.vector_int(N, -100, 100, seed, np.int16)
    return q, b


def tempering_ladder():
    return synth.geometric_ladder(0.1, 10.0, T_REPLICAS)


def tempering_desc(n_inst, samples):
    return ("parallel tempering: %d fp32 QUBO instances n~U[128,2048], Q=(A+A^T)/2 A~N(0,1), b=0, %d replicas on "
            "beta 0.1..10 (%d chains), Unbiased PNS k=n//16 L0=100, exchange every 100 original samples; %d original "
            "samples per chain per step" % (n_inst, T_REPLICAS, n_inst * T_REPLICAS, samples))


def tempering_config(n_inst, samples, world=1):
    return {"workload": tempering_desc(n_inst, samples), "instances": n_inst, "replicas": T_REPLICAS,
            "chains": n_inst * T_REPLICAS, "L0": T_L0, "swap_interval": T_SWAP, "samples_per_step": samples,
            "l2": "Q (3 GB) exceeds L2; a 256 MiB buffer is also written between timed steps",
            "parallelism": "%d instances per GPU: %d instances sharded by n^2 over %d rank(s), no data-path "
                           "collective" % (n_inst // world, n_inst, world)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(p)) if os.path.exists(p) else {}


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def _oracle_tempering_worker(args):
    seed, inst_ids, n_inst, warm, samples = args
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    ns = synth.tempering_sizes(n_inst, seed)
    ladder = tempering_ladder()
    recs = flips = 0
    summ = 0.0
    busy = 0.0
    for p in inst_ids:
        n = ns[p]
        prob = O.Problem(q=synth.tempering_q(p, n, seed))
        cfg = dict(variant="unbiased", k=max(1, n // 16), L0=T_L0, seed=seed)
        x0s = [np.zeros(n, np.uint8)] * T_REPLICAS
        # warm-up rounds, then the timed rounds continue the same chains
        res = O.run_tempering(prob, ladder, cfg, p, p * T_REPLICAS, x0s, warm // T_SWAP, 1, tape=False) if warm else None
        if res is not None:
            x0s = [r["x"] for r in res]
        t0 = time.perf_counter()
        res = O.run_tempering(prob, ladder, cfg, p, p * T_REPLICAS, x0s, samples // T_SWAP, 1, tape=False)
        busy += time.perf_counter() - t0
        recs += sum(int(r["state"].step) for r in res)
        flips += sum(int(r["state"].flips) for r in res)
        summ += sum(float(r["state"].sum_m) for r in res)
    return recs, flips, summ, busy


def oracle_tempering_rate(n_inst, every, warm, samples, seed=0):
    """The oracle as it stands on all host cores (spawned workers), on every
    `every`-th exchange group of the workload: `warm` original samples of
    warm-up (untimed), then `samples` timed.  The rate is the sample's
    records over the summed busy time divided by the workers."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ids = list(range(0, n_inst, every))
    workers = min(cores, len(ids))
    parts = [ids[i::workers] for i in range(workers)]
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as pool:
        list(pool.map(_oracle_tempering_worker, [(seed, [0], n_inst, 0, T_SWAP)] * workers, timeout=600))
        t0 = time.perf_counter()
        res = list(pool.map(_oracle_tempering_worker, [(seed, p, n_inst, warm, samples) for p in parts], timeout=3000))
        wall = time.perf_counter() - t0
    recs = sum(r[0] for r in res)
    flips = sum(r[1] for r in res)
    summ = sum(r[2] for r in res)
    busy = max(r[3] for r in res)  # the slowest worker's timed part
    single = float(np.mean([r[0] / r[3] for r in res if r[3] > 0]))
    return dict(rate=recs / busy, flips_rate=flips / busy, orig_rate=summ / busy, wall=wall, busy=busy, cores=workers,
                single_core_rate=single,
                sample="%d of the %d exchange groups (every %d-th instance, 8 replicas each): %d original samples of "
                       "warm-up, then %d timed" % (len(ids), n_inst, every, warm, samples))


def _oracle_dense_worker(args):
    seed, chain_ids, records, variant = args
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    q, b = workload(seed)
    prob = O.Problem(q=q, b=b)
    cfg = O.make_config(variant, k=K, L0=L0, seed=seed)
    t0 = time.perf_counter()
    tot = 0
    for cid in chain_ids:
        st = O.ChainState(prob, np.zeros(N, np.uint8), L0)
        O.run_chain(prob, cfg, np.float32(BETA), cid, st, records, tape=False)
        tot += records
    return tot, time.perf_counter() - t0


def oracle_dense_rate(records, chains_sample, seed=0, variant="unbiased"):
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    workers = min(cores, chains_sample)
    ids = list(range(chains_sample))
    parts = [ids[i::workers] for i in range(workers)]
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as pool:
        list(pool.map(_oracle_dense_worker, [(seed, [0], 10, variant)] * workers, timeout=600))
        t0 = time.perf_counter()
        res = list(pool.map(_oracle_dense_worker, [(seed, p, records, variant) for p in parts], timeout=1200))
        wall = time.perf_counter() - t0
    tot = sum(r[0] for r in res)
    return dict(rate=tot / wall, cores=workers, single_core_rate=float(np.mean([r[0] / r[1] for r in res])),
                sample="%d chains x %d records of the dense int16 n=1024 workload" % (chains_sample, records))


def reference_arm(args):
    """The CPU oracle, as it stands, on the tempering workload (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import build_oracle
    build_oracle.build()
    every, warm, samples = 4, 1000, 5000
    for _ in range(args.warmup):
        oracle_tempering_rate(args.instances, 64, 0, T_SWAP)
    rates, times = [], []
    last = None
    for _ in range(args.steps):
        r = oracle_tempering_rate(args.instances, every, warm, samples)
        rates.append(r["rate"])
        times.append(r["busy"])
        last = r
    value = float(np.mean(rates))
    line = {"impl": "reference", "metric": "PNS jump samples/s (records/s)", "value": value, "unit": "samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(times) * 1e3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": tempering_config(args.instances * max(1, int(os.environ.get("WORLD_SIZE", "1"))), args.samples,
                                       max(1, int(os.environ.get("WORLD_SIZE", "1")))),
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"], "single_core_value": last["single_core_rate"]},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Clock sampling
# ---------------------------------------------------------------------------

class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, path, index):
        self.path = path
        self.index = index
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q, "--format=csv",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path).read().splitlines()[1:]:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1].split()[0]), float(parts[2].split()[0]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        mx = max(r[1] for r in rows)
        load = [r for r in rows if r[0] > 0.5 * mx] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i, v in enumerate(r[2]) if "Active" in v and "Not" not in v})
        return {"sm_mhz": float(np.median([r[0] for r in load])), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def _dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local, dist


def _allreduce(dist, vals, op="sum"):
    if dist is None:
        return vals
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return [float(v) for v in t.tolist()]


def tempering_arm(args):
    """The headline: the tempering workload, sharded by instance over ranks."""
    import torch

    from paper_2210_10513_gb300 import pns, shard

    world, rank, local, dist = _dist_setup()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)  # non-default stream: pns_run replays a captured CUDA graph
    torch.cuda.set_stream(stream)
    # weak scaling: `--instances` instances per GPU, all of them sharded over
    # the ranks by n^2 (at N = 1 the 512 of the single-GPU workload)
    n_inst = args.instances * world
    samples = args.samples
    ns_all = synth.tempering_sizes(n_inst, args.seed)
    lo, hi = shard.shard_instances([n * n * T_REPLICAS for n in ns_all], world, rank)
    ladder = tempering_ladder()
    cb = shard.chain_base([T_REPLICAS] * n_inst, 1, lo)
    gb = shard.group_base(1, lo)
    qs = [synth.tempering_q(p, ns_all[p], args.seed) for p in range(lo, hi)]
    ns = ns_all[lo:hi]

    def make(q_list, **kw):
        plist = [dict(n=n, q=q, betas=ladder, k=max(1, n // 16)) for n, q in zip(ns, q_list)]
        opts = dict(variant="unbiased", k=1, chains_per_replica=1, L0=T_L0, swap_interval=T_SWAP, seed=args.seed,
                    tape=False, chain_base=cb, group_base=gb)
        opts.update(kw)
        return pns.Sampler(plist, **opts)

    qd = [torch.from_numpy(q).to(dev) for q in qs]
    s = make(qd, graph=True, autotune=not args.no_autotune)
    row_bytes = np.repeat(4 * np.asarray(ns, dtype=np.float64), T_REPLICAS)  # one fp32 row per flip, per chain
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2 (Q itself is 3 GB)
    for _ in range(args.warmup):
        s.run(samples)
    torch.cuda.synchronize()
    before = s.read(tape=False)["stats"]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    os.makedirs(os.path.join(ROOT, "gpurun_out"), exist_ok=True)
    clk = Clocks(os.path.join(ROOT, "gpurun_out", "bench_clocks_rank%d.csv" % rank), local)
    ms = []
    with clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.run(samples)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if dist is not None:
        dist.barrier()
    after = s.read(tape=False)["stats"]
    info = s.info
    d = {k: (after[k] - before[k]).astype(np.float64) for k in ("steps", "flips", "sum_m", "saturated", "swaps_accepted")}
    kernel_s = sum(ms) / 1e3
    byts = float((d["flips"] * row_bytes).sum())
    tot = _allreduce(dist, [d["steps"].sum(), d["flips"].sum(), d["sum_m"].sum(), d["saturated"].sum(), byts,
                            d["swaps_accepted"].sum()])
    kmax = _allreduce(dist, [kernel_s], "max")[0]
    records, flips, summ, sat, byts_all, swaps = tot
    value = records / kmax

    extra = {}
    if rank == 0 and not args.quick and world == 1:
        # one exchange group per launch, launches back to back: the form
        # that runs one group at a time (records are the same)
        sp = make(qd, chains_per_cta=1)
        p_samples = 10 * T_SWAP
        sp.run_plain(p_samples)
        torch.cuda.synchronize()
        b0 = sp.read(tape=False)["stats"]["steps"].sum()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sp.run_plain(p_samples)
        e1.record(stream)
        e1.synchronize()
        p_recs = float(sp.read(tape=False)["stats"]["steps"].sum() - b0)
        extra["plain_samples_per_s"] = p_recs / (e0.elapsed_time(e1) / 1e3)
        extra["batched_over_plain"] = value / extra["plain_samples_per_s"]
        extra["plain_form"] = "one exchange group per launch, %d launches back to back, %d original samples" % (
            sp.info.ctas, p_samples)
        sp.close()
    s.close()
    del qd

    # e2e: the instances from pinned host memory through the public API;
    # create + run + read (states and statistics) per step
    q_host = [torch.from_numpy(q).pin_memory() for q in qs]
    h2d = int(sum(q.nbytes for q in qs) + 4 * T_REPLICAS * len(qs))
    e_steps = max(2, min(args.steps, 6))
    t_e, recs_e, d2h = [], 0.0, 0
    parts = np.zeros(4)  # create, run, read, destroy (host clock, summed over the timed steps)
    for i in range(e_steps + 1):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        se = make(q_host, seed=args.seed + 1000 + i)
        ta = time.perf_counter()
        se.run(samples)
        torch.cuda.current_stream().synchronize()
        tb = time.perf_counter()
        out = se.read(tape=False)
        tc = time.perf_counter()
        se.close()
        t2 = time.perf_counter()
        if i > 0:  # the first one warms the allocator and the module
            t_e.append(t2 - t1)
            parts += [ta - t1, tb - ta, tc - tb, t2 - tc]
            recs_e += float(out["stats"]["steps"].sum())
            d2h = int(out["states"].nbytes + out["stats"].nbytes)
    e_tot = _allreduce(dist, [recs_e])[0]
    e_time = _allreduce(dist, [sum(t_e)], "max")[0]
    e2e = {"value": e_tot / e_time, "unit": "samples/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": e_time / len(t_e) * 1e3,
           "split_ms": {k: float(v) / len(t_e) * 1e3 for k, v in zip(("create", "run", "read", "destroy"), parts)},
           "steps": len(t_e)}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    peak_note = "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    if hbm is None:
        hbm, peak_note = 6800.0, "fallback"
    avg_launch = kernel_s / max(1, args.steps)
    achieved = byts / max(1, args.steps) / avg_launch / 1e9  # rank 0's kernel
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic_tempering.json")
    if os.path.exists(tr_path):
        tr = json.load(open(tr_path))
        if tr.get("kernel", "").startswith("pns_block_kernel") and tr.get("samples") == samples and \
                tr.get("instances") == n_inst and tr.get("source_sha") == _kernel_sha():
            traffic = tr.get("dram_bytes_per_launch")
    cpu = None
    if world == 1 and not args.no_cpu:
        from oracle import build_oracle
        build_oracle.build()
        r = oracle_tempering_rate(n_inst, 4, 1000, 5000, args.seed)
        cpu = {"value": r["rate"], "unit": "samples/s", "cores": r["cores"], "kind": "oracle", "sample": r["sample"],
               "single_core_value": r["single_core_rate"]}
    line = {
        "metric": "PNS jump samples/s (records/s)",
        "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": kmax * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": tempering_config(n_inst, samples, world),
        "flips_per_s": flips / kmax, "original_samples_per_s": summ / kmax, "saturated_moves": int(sat),
        "swaps_accepted": int(swaps),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic, "peak_kind": peak_note,
                     "algorithmic_bytes": "4 n bytes (one fp32 row of Q) per flip, summed over the launch's flips"},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
        "clocks": clk.summary(), "wall_s": wall,
        "mapping": {"period_blocked": info.period_blocked, "team_warps": info.team_warps, "ctas": info.ctas,
                    "autotune": not args.no_autotune, "cuda_graph": True},
    }
    line.update(extra)
    if not args.quick and world == 1:
        line["dense1024"] = dense1024_figures(args, stream)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _kernel_sha():
    """Hash of the sources of the period-blocked kernel: a stored ncu traffic
    figure is used only for the kernel it was taken on."""
    import hashlib
    h = hashlib.sha256()
    for f in ("pns_block.cuh", "pns_block_dense.cu", "pns_sampler.cuh", "pns_device.cuh", "pns_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2210_10513_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def dense1024_figures(args, stream, records=10000, steps=10, warmup=3):
    """The dense int16 n = 1024 workload (256 chains, Unbiased k = 64, beta =
    0.05): records/s and its roofline on the L2 side (Q, 2 MiB, stays in L2)
    against the library's measured L2 read bandwidth."""
    import torch

    from paper_2210_10513_gb300 import pns
    dev = torch.device("cuda", torch.cuda.current_device())
    q, b = workload(args.seed)
    qd, bd = torch.from_numpy(q).to(dev), torch.from_numpy(b).to(dev)
    s = pns.Sampler([dict(n=N, q=qd, b=bd, betas=[BETA])], variant="unbiased", k=K, chains_per_replica=CHAINS, L0=L0,
                    seed=args.seed, tape=False, graph=True, autotune=not args.no_autotune)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for _ in range(warmup):
        s.run(records)
    torch.cuda.synchronize()
    before = s.read(tape=False)["stats"]
    ms = []
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.run(records)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    after = s.read(tape=False)["stats"]
    info = s.info
    s.close()
    secs = sum(ms) / 1e3
    recs = float(after["steps"].sum() - before["steps"].sum())
    flips = float(after["flips"].sum() - before["flips"].sum())
    l2 = pns.pns_l2_read_probe(64 << 20, 50, stream.cuda_stream)
    achieved = flips / steps * ROW_BYTES / (secs / steps) / 1e9
    hbm = peaks().get("hbm_gbs", 6800.0)
    return {"workload": "dense int16 QUBO n=1024, 256 chains, Unbiased PNS k=64 L0=100, beta=0.05, %d records per "
                        "chain per step" % records,
            "value": recs / secs, "unit": "samples/s", "flips_per_s": flips / secs, "ms_per_step": secs * 1e3 / steps,
            "roofline_l2": {"bound": "l2", "achieved": achieved, "peak": l2, "unit": "GB/s", "frac": achieved / l2,
                            "peak_kind": "measured (pns_l2_read_probe: 64 MiB resident buffer read by every SM)",
                            "algorithmic_bytes": "2048 B (one int16 row of Q) per flip"},
            "roofline_hbm_frac": achieved / hbm,
            "mapping": {"set_sweep": info.set_sweep, "spec_depth": info.spec_depth, "ctas": info.ctas}}


def dense1024_arm(args):
    """`--workload dense1024`: the dense int16 workload's own line."""
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    fig = dense1024_figures(args, stream, records=args.records, steps=args.steps, warmup=args.warmup)
    fig.update({"metric": "PNS jump samples/s (records/s)", "workload": "dense1024", "steps": args.steps,
                "warmup": args.warmup})
    print(json.dumps(fig), flush=True)


def fit_workload(args):
    """Differentiation: n = 64 fp32 QUBO, Q = (A + A^T)/2 with A N(0, 0.1^2),
    b N(0, 0.1^2), beta = 1, 8192 chains, Unbiased k = 16, L0 = 100.  One step
    = one forward (the sampler for `--records` records per chain with the
    sample tape) + the tensor-core moments + the gradient kernel."""
    import torch

    from paper_2210_10513_gb300 import pns
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    wl = synth.workload_fit(64, seed=args.seed)
    n = 64
    chains = 8192
    recs = args.records
    s = pns.Sampler([dict(n=n, q=torch.from_numpy(wl["q"]).to(dev), b=torch.from_numpy(wl["b"]).to(dev),
                          betas=[1.0])], variant="unbiased", k=16, chains_per_replica=chains, L0=100, seed=args.seed,
                    tape=2)
    s.run(recs)  # burn-in
    f64 = lambda *shape: torch.empty(shape, dtype=torch.float64, device=dev)  # noqa: E731
    mom = dict(scalars=f64(4), mean_x=f64(n), mean_xx=f64(n, n), cov_ex=f64(n), cov_exx=f64(n, n))
    dQ, db, dbeta = f64(n, n), f64(n), f64(1)
    t_samp, t_mom = [], []
    for it in range(args.warmup + args.steps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        s.run(recs)
        e1.record(stream)
        pns.pns_moments(s.ctx, 0, 0, mom["scalars"], mom["mean_x"], mom["mean_xx"], mom["cov_ex"], mom["cov_exx"])
        pns.pns_energy_grads(n, 1.0, mom["scalars"], mom["mean_x"], mom["mean_xx"], mom["cov_ex"], mom["cov_exx"],
                             None, None, 0.0, dQ, db, dbeta)
        e2.record(stream)
        e2.synchronize()
        if it >= args.warmup:
            t_samp.append(e0.elapsed_time(e1))
            t_mom.append(e1.elapsed_time(e2))
    samples = float(chains) * recs
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16 = peaks.get("bf16_tflops", 1900.0)
    mma_flops = samples * 2 * 128 * 64 * 3  # three M = 128, N = 64 MMAs per sample (padded planes)
    tape_bytes = samples * (8 + 8 + 8)  # bits (2 words), M, E read by the moments kernels
    ms_s = float(np.mean(t_samp))
    ms_m = float(np.mean(t_mom))
    line = {"metric": "forward+backward samples/s", "workload": "fit", "value": samples / ((ms_s + ms_m) / 1e3),
            "unit": "samples/s", "forward_ms": ms_s, "moments_and_grads_ms": ms_m,
            "forward_records_per_s": samples / (ms_s / 1e3),
            "moments_mma_tflops": mma_flops / (ms_m / 1e3) / 1e12, "bf16_peak_tflops": bf16,
            "moments_tape_GBs": tape_bytes / (ms_m / 1e3) / 1e9, "mean_energy": float(mom["scalars"][1].item()),
            "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": "fit: n=64 fp32, 8192 chains, Unbiased k=16, beta=1, %d records per chain per step, "
                                   "moments on tcgen05 + gradients" % recs}}
    s.close()
    print(json.dumps(line), flush=True)


def donuts_workload(args):
    """Continuous Unbiased PNS (Algorithm 7) on the Donuts target of Sec. 7
    (mu0 = 9, sigma = 0.1, 50 neighbours, L0 = 1000) against Metropolis with
    the same N(0, I) proposal: 65,536 chains each; one step = one
    pns_donuts_run of `--records` records (Unbiased), and Metropolis runs for
    as many steps as fit in the same GPU time (calibrated on a short run), as
    the paper compares them at equal time.  Reports records/s, original
    samples/s and the paper's first-degree bias |mean x1| + |mean x2| per
    chain, averaged over chains."""
    import torch

    from paper_2210_10513_gb300 import pns
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    chains = 65536
    mu0, sigma = 9.0, 0.1
    c = 1.0 / (2 * sigma * sigma)
    rng = np.random.default_rng(args.seed)
    ang = rng.uniform(0, 2 * np.pi, chains)
    x0 = torch.from_numpy(np.stack([3 * np.cos(ang), 3 * np.sin(ang)], 1).astype(np.float32)).to(dev)
    out = torch.empty((chains, pns.DONUTS_STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    res = {}

    def per_step_ms(variant, steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pns.pns_donuts_run(variant, chains, steps, x0=x0, mu0=mu0, c=c, L0=1000, seed=7, stats=out)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps

    per_step_ms("metropolis", 200)  # first launch
    ratio = per_step_ms("unbiased", 500) / per_step_ms("metropolis", 2000)
    metro_steps = max(1, int(round(args.records * ratio)))
    for variant, steps in (("unbiased", args.records), ("metropolis", metro_steps)):
        for w in range(args.warmup):
            pns.pns_donuts_run(variant, chains, steps, x0=x0, mu0=mu0, c=c, L0=1000, seed=w, stats=out)
        ms = []
        for i in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pns.pns_donuts_run(variant, chains, steps, x0=x0, mu0=mu0, c=c, L0=1000, seed=100 + i, stats=out)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = np.frombuffer(out.cpu().numpy().tobytes(), dtype=pns.DONUTS_STATS_DTYPE)
        W = st["weight"]
        bias1 = float((np.abs(st["sum_x"][:, 0] / W) + np.abs(st["sum_x"][:, 1] / W)).mean())
        secs = float(np.median(ms)) / 1e3
        res[variant] = {"records_per_s": chains * steps / secs, "original_samples_per_s": float(W.sum()) / secs,
                        "ms_per_step": secs * 1e3, "moves_per_record": float(st["moves"].sum()) / (chains * steps),
                        "first_degree_bias": bias1}
    line = {"metric": "PNS jump samples/s (records/s)", "workload": "donuts", "value": res["unbiased"]["records_per_s"],
            "unit": "samples/s", "steps": args.steps, "warmup": args.warmup, "unbiased": res["unbiased"],
            "metropolis": res["metropolis"],
            "config": {"workload": "donuts: mu0=9 sigma=0.1, 65536 chains, Unbiased |N|=50 L0=1000 (%d records) vs "
                                   "Metropolis in the same GPU time (%d steps)" % (args.records, metro_steps)}}
    print(json.dumps(line), flush=True)


def side_workload(args):
    """Other benchmark shapes, one JSON line each (not the headline):
    lattice   -- 256 x 256 periodic +-1 lattice (n = 65536) as CSR, 64 chains
                 for each beta in {0.2, 0.44, 1.0}, Unbiased k = 1024; one step
                 = `--records` records for every chain."""
    import torch

    from paper_2210_10513_gb300 import pns
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    tune = dict(graph=True, autotune=not args.no_autotune)
    if args.workload == "donuts":
        return donuts_workload(args)
    elif args.workload == "fit":
        return fit_workload(args)
    else:
        side = 256
        csr = synth.lattice_csr(side, seed=args.seed)
        csr_d = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in csr)
        s = pns.Sampler([dict(n=side * side, csr=csr_d, betas=[0.2, 0.44, 1.0])], variant="unbiased", k=1024,
                        chains_per_replica=64, L0=100, seed=args.seed, tape=False, **tune)
        per_step = args.records
        row_bytes = np.full(s.info.chains, 5 * 4 + 4, dtype=np.int64)
        desc = ("lattice: 256x256 periodic +-1 couplings, CSR, 64 chains x beta {0.2,0.44,1.0}, Unbiased k=1024, "
                "%d records per chain per step" % per_step)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        s.run(per_step)
    torch.cuda.synchronize()
    before = s.read(tape=False)["stats"]
    ms = []
    clk = Clocks(os.path.join(ROOT, "gpurun_out", "bench_clocks_%s.csv" % args.workload), 0)
    with clk:
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.run(per_step)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    after = s.read(tape=False)["stats"]
    secs = sum(ms) / 1e3
    flips = (after["flips"] - before["flips"]).astype(np.float64)
    recs = float((after["steps"] - before["steps"]).sum())
    byts = float((flips * row_bytes).sum())
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    line = {"metric": "PNS jump samples/s (records/s)", "workload": args.workload, "value": recs / secs,
            "unit": "samples/s", "flips_per_s": float(flips.sum()) / secs,
            "original_samples_per_s": float((after["sum_m"] - before["sum_m"]).sum()) / secs,
            "ms_per_step": secs * 1e3 / args.steps, "steps": args.steps, "warmup": args.warmup,
            "row_bytes_per_s_GBs": byts / secs / 1e9, "hbm_peak_GBs": hbm, "frac_of_hbm": byts / secs / 1e9 / hbm,
            "chains": int(s.info.chains), "ctas": int(s.info.ctas), "warps_per_chain": int(s.info.warps_per_chain),
            "mapping": {"team_warps": s.info.team_warps, "producer_warps": s.info.producer_warps,
                        "spec_depth": s.info.spec_depth, "period_blocked": s.info.period_blocked,
                        "autotune": not args.no_autotune, "cuda_graph": True},
            "swaps_accepted": int((after["swaps_accepted"] - before["swaps_accepted"]).sum()),
            "config": {"workload": desc}, "clocks": clk.summary()}
    s.close()
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--samples", type=int, default=10000, help="tempering: original samples per chain per step")
    ap.add_argument("--records", type=int, default=10000, help="dense1024 / lattice / fit / donuts: records per step")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="heuristic chain-to-CTA mapping")
    ap.add_argument("--quick", action="store_true", help="skip the plain-form and dense1024 side measurements")
    ap.add_argument("--workload", default="tempering", choices=["tempering", "dense1024", "lattice", "fit", "donuts"])
    ap.add_argument("--instances", type=int, default=T_INST)
    args = ap.parse_args()
    if args.samples % T_SWAP != 0:
        ap.error("--samples must be a multiple of %d" % T_SWAP)
    if args.impl == "reference":
        reference_arm(args)
        return
    from paper_2210_10513_gb300 import build as B
    B.build()
    if args.workload == "tempering":
        tempering_arm(args)
    elif args.workload == "dense1024":
        dense1024_arm(args)
    else:
        side_workload(args)


if __name__ == "__main__":
    main()
