"""Benchmark of the batched PNS sampler on one GB300 (or N, one process each).

Workload (default): dense symmetric int16 QUBO, n = 1024, entries and b
uniform in [-100, 100], beta = 0.05, 256 independent chains, Unbiased PNS with
systematic sets of k = 64 and L0 = 100.  One bench step = one pns_run of
`--records` jump steps (records) for every chain.  The metric is jump samples
(records) per second over all chains; flips/s, original (Metropolis-
equivalent) samples/s, the Basic-PNS rate and the plain one-chain-per-launch
rate are reported beside it.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on
the host cores instead (bounded sample of the same workload).
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


def config_desc(records, l2):
    return {"workload": "dense int16 QUBO n=1024, 256 chains, Unbiased PNS k=64 L0=100, beta=0.05, "
                        "%d records per chain per step" % records,
            "n": N, "k": K, "chains": CHAINS, "beta": BETA, "L0": L0, "variant": "unbiased-systematic",
            "records_per_step": records, "l2": l2, "parallelism": "independent chains"}


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def _oracle_worker(args):
    seed, chain_ids, records, variant = args
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    q, b = workload(seed)
    prob = O.Problem(q=q, b=b)
    cfg = O.make_config(variant, k=K, L0=L0, seed=seed)
    t0 = time.perf_counter()
    tot = 0
    flips = 0
    summ = 0.0
    for cid in chain_ids:
        st = O.ChainState(prob, np.zeros(N, np.uint8), L0)
        O.run_chain(prob, cfg, np.float32(BETA), cid, st, records, tape=False)
        tot += records
        flips += st.st.flips
        summ += st.st.sum_m
    return tot, flips, summ, time.perf_counter() - t0


def oracle_rate(records, chains_sample, seed=0, variant="unbiased"):
    """Time the oracle as it stands on all host cores (spawned workers)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    workers = min(cores, chains_sample)
    ids = list(range(chains_sample))
    parts = [ids[i::workers] for i in range(workers)]
    # spawned workers (never forked after CUDA initialisation); a dead worker
    # raises BrokenProcessPool instead of hanging
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as pool:
        list(pool.map(_oracle_worker, [(seed, [0], 10, variant)] * workers, timeout=600))  # load the library
        t0 = time.perf_counter()
        res = list(pool.map(_oracle_worker, [(seed, p, records, variant) for p in parts], timeout=1200))
        wall = time.perf_counter() - t0
    tot = sum(r[0] for r in res)
    flips = sum(r[1] for r in res)
    summ = sum(r[2] for r in res)
    # one core's rate: each worker runs its chains serially on one core
    single = float(np.mean([r[0] / r[3] for r in res]))
    return dict(rate=tot / wall, flips_rate=flips / wall, orig_rate=summ / wall, wall=wall, cores=workers,
                single_core_rate=single,
                sample="%d chains x %d records of the same workload (chains 0..%d)" % (chains_sample, records,
                                                                                      chains_sample - 1))


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import build_oracle
    build_oracle.build()
    cores = os.cpu_count() or 1
    chains_sample = min(CHAINS, cores)
    records = 100000
    for _ in range(args.warmup):
        oracle_rate(2000, chains_sample)
    times = []
    rates = []
    last = None
    for _ in range(args.steps):
        r = oracle_rate(records, chains_sample)
        times.append(r["wall"])
        rates.append(r["rate"])
        last = r
    value = float(np.mean(rates))
    line = {"impl": "reference", "metric": "PNS jump samples/s (records/s)", "value": value, "unit": "samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(times) * 1e3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": config_desc(args.records, "flushed between timed steps (256 MiB write)"),
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"], "single_core_value": last["single_core_rate"]},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
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


def gpu_arm(args):
    import torch

    from paper_2210_10513_gb300 import pns

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)  # non-default stream: pns_run replays a captured CUDA graph
    torch.cuda.set_stream(stream)
    seed = args.seed + rank  # weak scaling: each rank samples its own independent chains
    q, b = workload(args.seed)
    qd = torch.from_numpy(q).to(dev)
    bd = torch.from_numpy(b).to(dev)
    records = args.records

    def make(variant, **kw):
        opts = dict(graph=True, autotune=not args.no_autotune)
        opts.update(kw)
        return pns.Sampler([dict(n=N, q=qd, b=bd, betas=[BETA])], variant=variant, k=K, chains_per_replica=CHAINS,
                           L0=L0, seed=seed, tape=False, **opts)

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def timed(sampler, steps, warmup, plain=False, recs=None):
        recs = recs or records
        for _ in range(warmup):
            (sampler.run_plain if plain else sampler.run)(recs)
        torch.cuda.synchronize()
        before = sampler.read(tape=False)["stats"]
        ms = []
        for _ in range(steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            (sampler.run_plain if plain else sampler.run)(recs)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        after = sampler.read(tape=False)["stats"]
        d = {k: float(after[k].sum() - before[k].sum()) for k in ("steps", "flips", "sum_m", "saturated")}
        return ms, d

    s_unb = make("unbiased")
    # main timed region, barrier + sync on both sides, clocks sampled during it
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(os.path.join(ROOT, "gpurun_out", "bench_clocks_rank%d.csv" % rank), local)
    os.makedirs(os.path.join(ROOT, "gpurun_out"), exist_ok=True)
    with clk:
        t0 = time.perf_counter()
        ms, d = timed(s_unb, args.steps, args.warmup)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if dist is not None:
        dist.barrier()
    kernel_s = sum(ms) / 1e3
    if dist is not None:
        t = torch.tensor([kernel_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        kernel_s = float(t.item())
        tot = torch.tensor([d["steps"], d["flips"], d["sum_m"], d["saturated"]], dtype=torch.float64, device=dev)
        dist.all_reduce(tot)
        d = dict(steps=float(tot[0]), flips=float(tot[1]), sum_m=float(tot[2]), saturated=float(tot[3]))
    value = d["steps"] / kernel_s
    extra = {}
    if rank == 0 and not args.quick:
        # Basic PNS (fresh random 64-subset every step), same workload
        s_basic = make("basic")
        ms_b, d_b = timed(s_basic, max(3, args.steps // 2), 2)
        extra["basic_samples_per_s"] = d_b["steps"] / (sum(ms_b) / 1e3)
        s_basic.close()
        # plain form: one chain per launch, launches back to back
        s_plain = make("unbiased", chains_per_cta=1, graph=False, autotune=False)
        plain_records = max(100, records // 10)
        ms_p, d_p = timed(s_plain, 1, 1, plain=True, recs=plain_records)
        extra["plain_samples_per_s"] = d_p["steps"] / (sum(ms_p) / 1e3)
        extra["batched_over_plain"] = value / extra["plain_samples_per_s"]
        extra["plain_records_per_chain"] = plain_records
        s_plain.close()
    info = s_unb.info
    s_unb.close()

    # e2e: pinned host buffers through the public API, copies inside the timed region
    e2e = None
    if rank == 0:
        q_host = torch.from_numpy(q.copy()).pin_memory()
        b_host = torch.from_numpy(b.copy()).pin_memory()
        e_steps = max(2, min(args.steps, 5))
        h2d = q.nbytes + b.nbytes + 4
        t_e = []
        recs = 0
        d2h = 0
        for i in range(e_steps + 1):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            s = pns.Sampler([dict(n=N, q=q_host, b=b_host, betas=[BETA])], variant="unbiased", k=K,
                            chains_per_replica=CHAINS, L0=L0, seed=seed + 1000 + i, tape=False)
            s.run(records)
            out = s.read(tape=False)
            s.close()
            t2 = time.perf_counter()
            if i > 0:  # first one warms the allocator
                t_e.append(t2 - t1)
                recs += int(out["stats"]["steps"].sum())
                d2h = out["states"].nbytes + out["stats"].nbytes
        e2e = {"value": recs / sum(t_e), "unit": "samples/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm = peaks.get("hbm_gbs")
    peak_note = "measured"
    if hbm is None:
        hbm = 6800.0
        peak_note = "fallback"
    flips_per_launch = d["flips"] / max(1, args.steps) / max(1, world)
    avg_launch_s = kernel_s / max(1, args.steps)
    achieved = flips_per_launch * ROW_BYTES / avg_launch_s / 1e9
    # DRAM bytes per launch from one ncu capture of the kernel this mapping
    # runs (null when the capture was of another kernel)
    traffic = None
    kernel = "pns_sweep_kernel" if info.set_sweep else ("pns_spec_kernel" if info.spec_depth else "pns_sample_kernel")
    tr_path = os.path.join(ROOT, "profiles", "traffic_dense_int16_n1024.json")
    if os.path.exists(tr_path):
        tr = json.load(open(tr_path))
        if tr.get("kernel", "").startswith(kernel):
            traffic = tr.get("dram_bytes_per_launch")
    cpu = None
    if world == 1 and not args.no_cpu:
        from oracle import build_oracle
        build_oracle.build()
        cores = os.cpu_count() or 1
        r = oracle_rate(100000, min(CHAINS, cores))
        cpu = {"value": r["rate"], "unit": "samples/s", "cores": r["cores"], "kind": "oracle", "sample": r["sample"],
               "single_core_value": r["single_core_rate"]}
    line = {
        "metric": "PNS jump samples/s (records/s)",
        "value": value * 1.0, "unit": "samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": kernel_s * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": config_desc(records, "flushed between timed steps (256 MiB write)"),
        "flips_per_s": d["flips"] / kernel_s, "original_samples_per_s": d["sum_m"] / kernel_s,
        "saturated_moves": int(d["saturated"]),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic, "peak_kind": peak_note,
                     "algorithmic_bytes": "2048 B (one int16 row of Q) per flip"},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
        "clocks": clk.summary(), "wall_s": wall,
        "mapping": {"warps_per_chain": info.warps_per_chain, "team_warps": info.team_warps,
                    "producer_warps": info.producer_warps, "spec_depth": info.spec_depth,
                    "set_sweep": info.set_sweep, "ctas": info.ctas,
                    "autotune": not args.no_autotune,
                    "cuda_graph": True},
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


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
    tempering -- 512 fp32 instances, n uniform in [128, 2048], 8 replicas on a
                 geometric beta ladder 0.1..10, Unbiased PNS k = n // 16,
                 exchange every L0 = 100 original samples; one step = 1000
                 original samples (10 exchange rounds) for every chain.
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
    if args.workload == "tempering":
        n_inst = args.instances
        probs, ladder = synth.workload_tempering(n_inst, seed=args.seed)
        plist = []
        for pr in probs:
            plist.append(dict(n=pr["n"], q=torch.from_numpy(pr["q"]).to(dev), betas=ladder, k=max(1, pr["n"] // 16)))
        s = pns.Sampler(plist, variant="unbiased", k=1, chains_per_replica=1, L0=100, swap_interval=100,
                        seed=args.seed, tape=False, **tune)
        per_step = 1000
        ns = np.repeat(np.array([pr["n"] for pr in probs]), len(ladder))
        row_bytes = 4 * ns
        desc = ("tempering: %d fp32 instances n~U[128,2048], 8 replicas (beta 0.1..10), Unbiased k=n/16, "
                "swap every 100 original samples, 1000 original samples per chain per step" % n_inst)
    elif args.workload == "donuts":
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
    ap.add_argument("--records", type=int, default=10000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="heuristic chain-to-CTA mapping")
    ap.add_argument("--quick", action="store_true", help="skip the Basic / plain side measurements")
    ap.add_argument("--workload", default="dense1024", choices=["dense1024", "tempering", "lattice", "fit", "donuts"])
    ap.add_argument("--instances", type=int, default=512)
    args = ap.parse_args()
    if args.workload != "dense1024":
        from paper_2210_10513_gb300 import build as B
        B.build()
        side_workload(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        from paper_2210_10513_gb300 import build as B
        B.build()
        gpu_arm(args)


if __name__ == "__main__":
    main()
