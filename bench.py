"""Benchmark: exact dense assignments per second on one GB300.

Headline workload: ``geometric-n8192`` (n = 8192 optical-flow-like
instances: points in the unit square, targets a jittered permutation of
them, cost round(10^4 |a_i - b_j|^2)), plain cold-start cost scaling (costs
scaled by n + 1, prices from 0). One step = one complete solve of one
instance already resident in HBM (min/max pass, every refine phase, arc
fixing between phases, finalisation). Eight seeded instances (2 GiB, many
times the 129 MB L2) rotate, so no step starts with its matrix in L2. Every
timed cost is compared with the optimum stored for its seed by the oracle's
Hungarian method (``tests/golden/optimal_costs.json``); a mismatch fails the
run.

Two more single-GPU workloads get full lines of their own under
``extra.lines`` (the same keys, timing rules and exactness gate):
``uniform-n4096-c2^20`` (i.i.d. costs in [0, 2^20), ten instances, alpha
tuned on two untimed ones) and ``uniform-n256-c1000`` (costs in [0, 1000],
alpha = 10, one solve of each of 100 instances).

Prints ONE JSON line. ``value`` is solves/s over all ranks; ``roofline`` is
the dominant refine-phase kernel's algorithmic arc-scan bandwidth (4 n bytes
per full row scan, the list bytes per candidate-list scan, counted on the
device) over its CUDA-event time (``roofline_by_kernel`` has each kernel);
``e2e`` repeats the solve through the public Python API from pinned host
memory with the host<->device copies inside the timed region;
``cpu_baseline`` times the oracle's sequential cost scaling on the host.
``--impl reference`` times that oracle alone as the reference arm.

Multi-GPU (torchrun): replicas only. Each rank solves its own instances; the
time is the max over ranks and ``value`` counts every rank's solves.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "assignments/sec and refine arc-scan GB/s (vs GB300 roofline), exact cost; warm vs plain"
UNIT = "assignments/s"
HEADLINE = "geometric-n8192"

# Each single-solve line: instances (seeds 0..count-1, whose optima are
# stored), alpha (0: tuned on two untimed instances) and further la_options.
LINES = {
    "geometric-n8192": dict(count=8, alpha=10, options={"price_updates": 4, "tail_threshold": 128}),
    "uniform-n4096-c2^20": dict(count=10, alpha=48, options={"alpha_fine": 4}),
    "uniform-n256-c1000": dict(count=100, alpha=10, options={}, steps=100),
}
GOLDEN = os.path.join(ROOT, "tests", "golden", "optimal_costs.json")


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seeds(rank, count):
    """Seeds of the instances a replica solves: disjoint across ranks."""
    return [10_000 * rank + i for i in range(count)]


def max_over_ranks(value, device=None):
    """The slowest rank's time (every rank gets it); identity without a
    process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(steps, world, elapsed):
    """Whole-job solves per second: every rank's steps over the slowest rank's time."""
    return steps * world / elapsed


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def stored_optima(workload):
    """{seed: optimal cost} stored for the workload at its own size."""
    from paper_1110_6231_gb300 import synth
    n = synth.WORKLOADS[workload]["n"]
    try:
        cases = json.load(open(GOLDEN))["cases"]
    except Exception:
        return {}
    return {c["seed"]: c["cost"] for c in cases if c["workload"] == workload and c["n"] == n}


# The sources the single-solve kernels (k_refine, k_tail, k_fix and their
# helpers) are compiled from; the DRAM traffic recorded for them stays valid
# while these are unchanged.
SINGLE_SOLVE_SOURCES = ("la_solve.cu", "la_device.cuh", "la_lists.cuh")


def code_tokens(text: str) -> str:
    """C/CUDA source without its comments and with whitespace runs collapsed,
    so that an edit to a comment leaves the kernel hash unchanged (none of
    the hashed sources has a comment marker inside a string literal)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_hash():
    """Hash of the code (not the comments) of the single-solve kernels."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1110_6231_gb300", "csrc")
    for name in SINGLE_SOLVE_SOURCES:
        h.update(code_tokens(open(os.path.join(csrc, name)).read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload, alpha, kernel, options=None):
    """DRAM bytes (read + write) per launch of ``kernel`` from the committed
    ncu record, if one was taken on this workload at this alpha with these
    solver options and on the kernel source that is built now; None
    otherwise."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    h = kernel_hash()
    for e in rec.get("entries", []):
        if (e.get("kernel_hash") == h and e.get("workload") == workload and e.get("alpha") == alpha
                and (e.get("options") or {}) == (options or {})):
            return e.get("dram_bytes_per_launch", {}).get(kernel)
    return None


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, out_dir=None, tag=""):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        self.index = ids[index] if index < len(ids) else str(index)
        self.proc = None
        self.path = os.path.join(out_dir or tempfile.gettempdir(), f"clocks_rank{index}{tag}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, flag in zip(names, parts[5:9]):
                    if flag.lower().startswith("active"):
                        reasons.add(name)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_oracle_baseline(workload, alpha, budget_s, rank_seed=0):
    """The oracle's sequential cost scaling, as it stands, on one host core,
    at the line's alpha, on instances of the same workload (seeds 1000 on)."""
    import oracle
    from paper_1110_6231_gb300 import synth
    done, t_solve, seeds = 0, 0.0, []
    s = 1000 + rank_seed
    while t_solve < budget_s or done == 0:
        C = synth.instance(workload, s)
        t0 = time.perf_counter()
        oracle.cost_scaling(C, alpha=alpha)
        t_solve += time.perf_counter() - t0
        done += 1
        seeds.append(s)
        s += 1
    return {"value": done / t_solve, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} instance(s) of {workload} (seeds {seeds[0]}..{seeds[-1]}), "
                      f"oracle.cost_scaling at alpha = {alpha}, single-threaded, {t_solve:.1f} s of CPU time"}


def run_reference(args):
    """The reference arm: the oracle's cost scaling on the headline workload,
    at the headline's alpha, one solve per step (eight instances rotate)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1110_6231_gb300 import synth
    spec = LINES[HEADLINE]
    alpha = args.alpha or spec["alpha"] or 10
    count = min(spec["count"], args.steps + args.warmup)
    insts = [synth.instance(HEADLINE, 1000 + i) for i in range(count)]
    for i in range(args.warmup):
        oracle.cost_scaling(insts[i % count], alpha=alpha)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.cost_scaling(insts[(args.warmup + i) % count], alpha=alpha)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    n = synth.WORKLOADS[HEADLINE]["n"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": HEADLINE, "n": n, "alpha": alpha, "start_prices": "zero (cold)",
                   "solver": "oracle.cost_scaling"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} timed solves of {HEADLINE} (seeds 1000..{999 + count} "
                                   f"rotating) after {args.warmup} warm-up, single-threaded"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- single solves

def kernel_rooflines(workload, alpha, n, stats, peak, peak_src, l2_gbps=None, options=None):
    """Roofline entries of the refine-phase kernels from the per-solve
    counters: algorithmic bytes (4 n per full row scan, the list's bytes per
    candidate-list scan) over each kernel's own CUDA-event time (events on
    the solve's stream around every phase's grid refine and its one-CTA tail
    kernel)."""
    full = sum(s["full_scans"] for s in stats)
    listed = sum(s["list_scans"] for s in stats)
    tail_scans = sum(s["tail_scans"] for s in stats)
    tail_full = sum(s["tail_full_scans"] for s in stats)
    sweep_scans = sum(s["sweep_scans"] for s in stats)
    sweep_full = sum(s["sweep_full_scans"] for s in stats)
    list_bytes = stats[0]["list_entries"] * 8 + 8 if stats else 0
    phase_ms = sum(s["refine_ms"] for s in stats)
    tail_ms = sum(s["tail_ms"] for s in stats)
    sweep_ms = sum(s["sweep_ms"] for s in stats)
    phases_run = sum(s["phases"] for s in stats)
    tail_launches = sum(s["tail_phases"] for s in stats)
    per_kernel = {}
    if stats and all(st.get("small_kernel") for st in stats):
        # small instances: the whole solve is one launch of the shared-memory kernel
        roles = (("k_small", full, 0, phase_ms, len(stats)),)
    else:
        roles = (
            # the bulk sweep: the k_refine launch that opens each phase (each row's first bid)
            ("k_refine_sweep", sweep_full, sweep_scans - sweep_full, sweep_ms, phases_run),
            # the grid refine launches that carry the displacement chains
            ("k_refine", full - tail_full - sweep_full, listed - (tail_scans - tail_full) - (sweep_scans - sweep_full),
             phase_ms - tail_ms - sweep_ms, phases_run),
            ("k_tail", tail_full, tail_scans - tail_full, tail_ms, max(1, tail_launches)))
    for kname, kfull, klist, kms, launches in roles:
        kbytes = 4.0 * n * kfull + list_bytes * klist
        ach = kbytes / (kms * 1e-3) / 1e9 if kms > 0 else 0.0
        r = {"bound": "hbm", "kernel": kname, "achieved": ach, "peak": peak, "peak_source": peak_src,
             "unit": "GB/s", "frac": ach / peak, "traffic": recorded_traffic(workload, alpha, kname, options),
             "algorithmic_bytes_per_launch": kbytes / max(1, launches),
             "avg_launch_ms": kms / max(1, launches), "launches": launches,
             "share_of_refine_time": kms / phase_ms if phase_ms > 0 else None,
             "regime": ("latency: the chains of bids on one CTA, rows read from shared memory after one load"
                        if kname == "k_small" else
                        "latency: dependent displacement chains, few warps busy at once")}
        if l2_gbps:
            r["l2"] = {"peak": l2_gbps, "frac": ach / l2_gbps, "unit": "GB/s"}
        per_kernel[kname] = r
    # the dominant kernel: the one that takes most of the refine time
    dominant = max(per_kernel, key=lambda k: per_kernel[k]["share_of_refine_time"] or 0.0)
    return per_kernel, dominant


def measure_line(args, la, synth, dev, stream, workload, spec, steps, warmup, rank, world, clocks_tag,
                 cpu_seconds, probe_l2=False):
    """One full bench line for a single-solve workload: the device-timed
    throughput over ``steps`` solves (instances resident, rotating), the
    exactness gate, per-kernel rooflines, e2e through the public API, the
    oracle's CPU baseline."""
    import torch
    n = synth.WORKLOADS[workload]["n"]
    count = spec["count"]
    seeds = rank_seeds(rank, count)
    optima = stored_optima(workload)
    host = [synth.instance(workload, s) for s in seeds]
    dmats = [torch.from_numpy(h).to(dev) for h in host]
    match = torch.empty(n, dtype=torch.int32, device=dev)
    costs = torch.zeros(max(1, steps), dtype=torch.int64, device=dev)
    scratch_cost = torch.zeros(1, dtype=torch.int64, device=dev)
    extra_opts = dict(spec.get("options", {}))

    tuning = None
    alpha = args.alpha or spec["alpha"]
    if alpha == 0:
        from paper_1110_6231_gb300 import tune
        samples = [torch.from_numpy(synth.instance(workload, 500 + s)).to(dev) for s in rank_seeds(rank, 2)]
        tuning = tune.autotune_alpha(samples)
        alpha = tuning["alpha"]
        del samples

    def step(i, out, stats_acc=None, a=None):
        opt = la.la_options()
        opt.profile = 1
        opt.alpha = alpha if a is None else a
        for k, v in extra_opts.items():
            setattr(opt, k, v)
        st = la.la_stats()
        rc = la.la_solve_ex(dmats[i % count], n, opt, stream, match, out, st)
        if rc != la.LA_OK:
            raise la.LaError(rc, "la_solve_ex")
        if stats_acc is not None:
            stats_acc.append(st.as_dict())

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    for i in range(warmup):
        step(i, scratch_cost)
    stats = []
    barrier()
    with Clocks(dev.index or 0, args.clocks_dir, clocks_tag) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        ev0.record(stream)
        step_ms = []
        for i in range(steps):
            ts = time.perf_counter()
            step(warmup + i, costs[i:i + 1], stats)   # returns once the solve is done
            step_ms.append(1e3 * (time.perf_counter() - ts))
        ev1.record(stream)
        barrier()
        wall = time.perf_counter() - t0
    dev_ms = ev0.elapsed_time(ev1)
    elapsed = max_over_ranks(max(wall, dev_ms / 1e3), dev)
    value = replica_throughput(steps, world, elapsed)

    # exactness gate: every timed cost against the optimum stored for its seed
    got = costs.cpu().tolist()
    checked, wrong = 0, []
    for i in range(steps):
        seed = seeds[(warmup + i) % count]
        if seed in optima:
            checked += 1
            if got[i] != optima[seed]:
                wrong.append({"seed": seed, "cost": got[i], "optimum": optima[seed]})

    peak, peak_src = peaks()
    l2_gbps = None
    if probe_l2:
        la.probe_read_gbps(dmats[0], 1, stream=stream)
        l2_gbps = max(la.probe_read_gbps(dmats[0], 20, stream=stream) for _ in range(3))
    per_kernel, dominant = kernel_rooflines(workload, alpha, n, stats, peak, peak_src, l2_gbps, extra_opts)

    # e2e through the public API: pinned host matrices, copies and the
    # readback of the matching and cost inside the timed region; the next
    # step's matrix is copied on a second stream while the current one solves
    pinned = [torch.from_numpy(h).pin_memory() for h in host]
    bufs = [torch.empty((n, n), dtype=torch.int32, device=dev) for _ in range(2)]
    ready = [torch.cuda.Event() for _ in range(2)]
    copy_stream = torch.cuda.Stream(dev)
    e2e_opts = dict(alpha=alpha, **{k: v for k, v in extra_opts.items()})

    def e2e_copy(i):
        with torch.cuda.stream(copy_stream):
            bufs[i % 2].copy_(pinned[i % count], non_blocking=True)
            ready[i % 2].record(copy_stream)

    def e2e_loop(k, first):
        e2e_copy(first)
        out = []
        for i in range(k):
            if i + 1 < k:
                e2e_copy(first + i + 1)
            stream.wait_event(ready[(first + i) % 2])
            sol = la.solve(bufs[(first + i) % 2], stream=stream, **e2e_opts)
            sol.match.cpu()
            out.append(sol.cost)
        return out

    e2e_loop(2, 0)
    barrier()
    copy_stream.synchronize()
    t0 = time.perf_counter()
    e2e_costs = e2e_loop(steps, warmup)
    barrier()
    e2e_t = max_over_ranks(time.perf_counter() - t0, dev)
    for i, c in enumerate(e2e_costs):
        seed = seeds[(warmup + i) % count]
        if seed in optima and c != optima[seed]:
            wrong.append({"seed": seed, "cost": c, "optimum": optima[seed], "e2e": True})

    # where an e2e step's time goes: one step at a time, no overlap
    h2d, solve, d2h = [], [], []
    for i in range(min(3, count)):
        e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e_a.record(stream)
        bufs[0].copy_(pinned[i], non_blocking=True)
        e_b.record(stream)
        torch.cuda.synchronize(dev)
        h2d.append(e_a.elapsed_time(e_b))
        t1 = time.perf_counter()
        sol = la.solve(bufs[0], stream=stream, **e2e_opts)
        t2 = time.perf_counter()
        sol.match.cpu()
        t3 = time.perf_counter()
        solve.append(1e3 * (t2 - t1))
        d2h.append(1e3 * (t3 - t2))

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warmup,
        "ms_per_step": 1e3 * elapsed / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "u64" if stats and stats[0]["wide"] else "u32", "data": "synthetic",
        "config": {"workload": workload, "n": n, "alpha": alpha,
                   "alpha_tuning": None if tuning is None else
                   {"over": "2 instances of the workload (seeds 500, 501), not timed",
                    "mean_ms": {str(a): round(v, 2) for a, v in tuning["mean_ms"].items()}},
                   "options": extra_opts or None,
                   "start_prices": "zero (cold)", "instances": f"seeds {seeds[0]}..{seeds[-1]}",
                   "l2": f"{count} rotating instances ({count * 4 * n * n >> 20} MiB) "
                         + ("> 129 MB L2" if count * 4 * n * n > 129e6 else "fit in L2"),
                   "parallelism": f"replicas x{world}"},
        "exact": {"checked": checked + len([c for c in e2e_costs]), "device_timed_checked": checked,
                  "wrong": wrong, "source": "tests/golden/optimal_costs.json (oracle.hungarian, duals checked)"},
        "roofline": per_kernel[dominant],
        "roofline_by_kernel": per_kernel,
        "median_ms_per_solve": statistics.median(step_ms),
        "ms_per_solve_range": [min(step_ms), max(step_ms)],
        "arc_scans_per_solve": sum(s["scans"] for s in stats) / max(1, len(stats)),
        # every phase starts with all n rows free, so n scans per phase is
        # the least a solve can make; this is that bound over the scans made
        "scan_efficiency": (sum(s["phases"] for s in stats) * n) / max(1, sum(s["scans"] for s in stats)),
        "full_row_scans_per_solve": sum(s["full_scans"] for s in stats) / max(1, len(stats)),
        "list_scans_per_solve": sum(s["list_scans"] for s in stats) / max(1, len(stats)),
        "fixed_rows_per_solve": sum(s["fixed_rows"] for s in stats) / max(1, len(stats)),
        "phases": stats[0]["phases"] if stats else None,
        "max_chain": max(s["max_chain"] for s in stats) if stats else None,
        "e2e": {"value": steps * world / e2e_t, "unit": UNIT,
                "h2d_bytes_per_step": 4 * n * n, "d2h_bytes_per_step": 4 * n + 8,
                "breakdown_ms": {"h2d_copy": statistics.median(h2d), "la_solve_call": statistics.median(solve),
                                 "match_readback": statistics.median(d2h),
                                 "note": "one step at a time, no overlap; medians of 3"}},
        "gpu_launches": sum(s["launches"] for s in stats),
        "clocks": clk.summary(),
        "cpu_baseline": None,
    }
    if rank == 0 and world == 1 and cpu_seconds > 0:
        line["cpu_baseline"] = cpu_oracle_baseline(workload, alpha, cpu_seconds, rank)
    del dmats, bufs, pinned
    return line, alpha


# ---------------------------------------------------------------- extra lines

def bench_batched(args, la, synth, dev, stream, l2_gbps=None):
    """10,000 instances, n log-uniform in [16, 1024] (half uniform [0, 10^4],
    half geometric): one persistent launch replayed from a CUDA graph, versus
    one la_solve call per instance on a sample."""
    import torch
    t0 = time.perf_counter()
    flat, off, ns = synth.batch(args.batch, 0)
    gen_s = time.perf_counter() - t0
    dc, do, dn = (torch.from_numpy(a).to(dev) for a in (flat, off, ns))
    from paper_1110_6231_gb300 import tune
    t_tune = time.perf_counter()
    if args.no_tune:   # library defaults (for profiling runs: no tuning launches first)
        table = {"block_threads": 0, "slots": 0, "max_n": int(ns.max()), "alpha": [0] * 16}
    else:
        table = tune.autotune_batched(dc, do, dn, reps=1)   # CTA shape and alpha per size bucket
    t_tune = time.perf_counter() - t_tune
    opt = tune.options_from_table(table, profile=True)
    la.solve_batched(dc, do, dn, options=opt)           # capture the graph
    times, stats = [], None
    for _ in range(3):
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        sol = la.solve_batched(dc, do, dn, options=opt)
        torch.cuda.synchronize(dev)
        times.append(time.perf_counter() - t1)
        stats = sol.stats
    best = min(times)
    idx = list(range(0, args.batch, max(1, args.batch // 100)))
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    for i in idx:
        n = int(ns[i])
        la.solve(dc[int(off[i]):int(off[i]) + n * n].view(n, n))
    torch.cuda.synchronize(dev)
    per = len(idx) / (time.perf_counter() - t2)
    scan_gbps = stats["scan_bytes"] / (stats["device_ms"] * 1e-3) / 1e9
    return {"workload": f"{args.batch} instances, n log-uniform [16,1024], half uniform [0,1e4], half geometric",
            "solves_per_s": args.batch / best, "ms": 1e3 * best, "device_ms": stats["device_ms"],
            "graph": stats["graph"], "scan_GBps": scan_gbps,
            "scan_GBps_note": "algorithmic arc-scan bytes (4 n per row scan); rows are staged through shared "
                              "memory and mostly served by L2 (DRAM reads about 17x the compulsory bytes, "
                              "profiles/batched_mixed_1500.md); compare with l2_frac, not with HBM",
            "l2_frac": scan_gbps / l2_gbps if l2_gbps else None,
            "scans": stats["scans"], "cost_bytes": int(flat.size) * 4,
            "per_instance_la_solve_per_s": per, "per_instance_sample": len(idx),
            "speedup_vs_per_instance": (args.batch / best) / per, "generate_s": gen_s,
            "autotuned": {"block_threads": table["block_threads"], "slots": table["slots"], "max_n": table["max_n"],
                          "alpha_by_log2n": table["alpha"], "tune_s": t_tune}}


def bench_concurrent(args, la, synth, dev, stream, alpha):
    """Many n = 4096 instances of the uniform workload solved at once by the
    batched kernel with candidate lists (256 threads per CTA, two instances
    resident per CTA, two CTAs per SM): throughput when the caller has many
    instances, beside the single-solve latency. The distinct matrices (seeds
    2000, 2001, ...) are drawn on the GPU by the torch twin of the generator.
    Unless --alpha fixes it, alpha is tuned first on as many other instances
    (seeds 3000, 3001, ...), which are not timed."""
    import torch
    n, B = 4096, args.concurrent
    dc = torch.empty(B * n * n, dtype=torch.int32, device=dev)

    def fill(seed0):
        for i in range(B):
            dc[i * n * n:(i + 1) * n * n] = synth.uniform_costs_torch(n, 0, (1 << 20) - 1, seed0 + i,
                                                                      device=dev).view(-1)

    off = torch.arange(B, dtype=torch.int64, device=dev) * (n * n)
    ns = torch.full((B,), n, dtype=torch.int32, device=dev)
    shape = dict(block_threads=256, slots=2, max_n=n, lists=1)
    tuning = None
    if args.alpha == 0:
        from paper_1110_6231_gb300 import tune
        fill(3000)
        tuning = tune.autotune_batch_alpha(dc, off, ns, **shape)
        alpha = tuning["alpha"]
    fill(2000)
    opt = la.batch_options(alpha=[alpha] * la.LA_ALPHA_BUCKETS, profile=True, **shape)
    la.solve_batched(dc, off, ns, options=opt)           # capture the graph
    best, stats = None, None
    for _ in range(2):
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        sol = la.solve_batched(dc, off, ns, options=opt)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t1
        if best is None or dt < best:
            best, stats = dt, sol.stats
    failed = int((sol.status != 0).sum().item())
    del dc
    return {"workload": f"{B} distinct uniform-n4096-c2^20 instances (seeds 2000..{2000 + B - 1})",
            "solves_per_s": B / best, "ms": 1e3 * best, "device_ms": stats["device_ms"], "failed": failed,
            "scans_per_instance": stats["scans"] / B,
            "scan_GBps": stats["scan_bytes"] / (stats["device_ms"] * 1e-3) / 1e9,
            "full_scan_fraction": stats["full_scans"] / max(1, stats["scans"]),
            "shape": {"block_threads": 256, "slots": 2, "grid": stats["grid"], "alpha": alpha, "lists": stats["lists"]},
            "alpha_tuning": None if tuning is None else
            {"over": f"{B} other instances (seeds 3000..{3000 + B - 1}), not timed, one launch per alpha",
             "device_ms": {str(a): round(v, 2) for a, v in tuning["device_ms"].items()}}}


def bench_warm(args, la, synth, dev):
    """Learned warm start versus plain cold start on fresh geometric
    instances (seeds never used in training), identical exact costs."""
    import numpy as np
    import torch
    from paper_1110_6231_gb300 import learn
    if not os.path.exists(learn.DEFAULT_WEIGHTS):
        return {"unavailable": "no trained weights"}
    P = torch.from_numpy(np.fromfile(learn.DEFAULT_WEIGHTS, dtype=np.float32)).to(dev)
    out = {}
    for n, cnt in ((1024, args.warm_n1024), (8192, args.warm_n8192)):
        if cnt <= 0:
            continue
        tc = tw = tp = 0.0
        sc = sw = 0
        stream = torch.cuda.current_stream(dev)
        for s in range(cnt):
            C = torch.from_numpy(synth.geometric_costs(n, 2_000_000 + s)).to(dev)
            if s == 0:
                la.solve(C)
                la.solve_warm(C, P)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            cold = la.solve(C)
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            warm = la.solve_warm(C, P)
            torch.cuda.synchronize(dev)
            t2 = time.perf_counter()
            if warm.cost != cold.cost:
                raise RuntimeError("warm and cold costs differ")
            # the predictor alone (features, BF16 weights, the fused network
            # launch), timed by CUDA events on the stream it runs on
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            la.predict_prices(C, P)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            tp += e0.elapsed_time(e1)
            tc += t1 - t0
            tw += t2 - t1
            sc += cold.stats["scans"]
            sw += warm.stats["scans"]
        out[f"n{n}"] = {"instances": cnt, "cold_ms": 1e3 * tc / cnt, "warm_ms": 1e3 * tw / cnt,
                        "speedup": tc / tw, "cold_scans": sc / cnt, "warm_scans": sw / cnt,
                        "predictor_ms": tp / cnt, "predictor_share_of_warm": (tp / cnt) / (1e3 * tw / cnt),
                        "identical_cost": True, "warm_includes": "features + set encoder + solve"}
    return out


def bench_sparse(la, synth, dev, reps=2):
    """The sparse-graph solver on the two n = 65536 workloads (planted perfect
    matching; uniform arcs of degree 32, and the geometric neighbourhood
    graph): best of ``reps`` solves, exact cost certified in the tests."""
    import torch
    out = {}
    for name in sorted(synth.SPARSE_WORKLOADS):
        rp, cols, costs = synth.sparse_instance(name, 0)
        t = [torch.from_numpy(a).to(dev) for a in (rp, cols, costs)]
        la.solve_sparse(*t)
        best, st = None, None
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            sol = la.solve_sparse(*t, profile=True)
            torch.cuda.synchronize(dev)
            dt = time.perf_counter() - t0
            if best is None or dt < best:
                best, st = dt, sol.stats
        out[name] = {"ms": 1e3 * best, "arcs": int(cols.size), "scans": st["scans"], "phases": st["phases"],
                     "max_chain": st["max_chain"], "solves_per_s": 1.0 / best}
    return out


def bench_maxflow(la, synth, dev, reps=3):
    """Grid max-flow (the paper's Sect. 4 problem): the 1024 x 1024
    graph-cut instance and the 512 x 512 grid whose flow crosses from the
    left column to the right; best of ``reps`` solves. Push work in units of
    node visits is not counted on the device, so the line reports time."""
    import torch
    out = {}
    for name in ("gridcut-1024x1024", "gridcross-512x512"):
        cap, src, snk = synth.grid_instance(name, 0)
        t = [torch.from_numpy(a).to(dev) for a in (cap, src, snk)]
        la.maxflow_grid(*t)
        best, st = None, None
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            r = la.maxflow_grid(*t)
            torch.cuda.synchronize(dev)
            dt = time.perf_counter() - t0
            if best is None or dt < best:
                best, st = dt, r.stats
        out[name] = {"ms": 1e3 * best, "nodes": int(src.size), "flow": st["flow"], "rounds": st["rounds"],
                     "global_relabels": st["global_relabels"], "relabel_passes": st["relabel_sweeps"]}
    return out


def run_gpu(args):
    import torch

    import paper_1110_6231_gb300 as la
    from paper_1110_6231_gb300 import synth

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    la.lib()
    stream = torch.cuda.current_stream(dev)
    cpu_s = 0 if args.no_cpu_baseline else args.cpu_seconds

    spec = dict(LINES[args.headline])
    if args.instances:   # profiling runs: fewer instances resident
        spec["count"] = args.instances
    head, head_alpha = measure_line(args, la, synth, dev, stream, args.headline, spec, args.steps,
                                    args.warmup, rank, world, "", cpu_s)

    # the HBM read rate beside the headline's arc-scan rate (its 2 GiB of
    # matrices do not fit in L2), and the L2 read rate on a 64 MiB matrix
    big = torch.empty(1 << 30, dtype=torch.int32, device=dev)
    la.probe_read_gbps(big, 1, stream=stream)
    hbm_read_gbps = max(la.probe_read_gbps(big, 2, stream=stream) for _ in range(2))
    del big
    small = torch.empty(1 << 24, dtype=torch.int32, device=dev)
    la.probe_read_gbps(small, 1, stream=stream)
    l2_gbps = max(la.probe_read_gbps(small, 20, stream=stream) for _ in range(3))
    del small

    wanted = set() if args.no_extra else set(args.extras.split(","))
    extra = {}

    def guarded(fn, *a, **k):
        # an extra line that fails is reported in its own entry; the headline
        # line is still printed (extras make no collective calls, so ranks
        # cannot fall out of step)
        try:
            return fn(*a, **k)
        except Exception as ex:
            return {"error": f"{type(ex).__name__}: {ex}"[:400]}

    lines = {}
    u4096_alpha = 10
    if "lines" in wanted:
        for w in [w for w in LINES if w != args.headline]:
            spec = LINES[w]

            def one(w=w, spec=spec):
                line, a = measure_line(args, la, synth, dev, stream, w, spec,
                                       spec.get("steps", args.steps), args.warmup, rank, world, "_" + w[:12],
                                       cpu_s, probe_l2=(w == "uniform-n4096-c2^20"))
                return line, a
            r = guarded(one)
            if isinstance(r, dict):
                lines[w] = r
            else:
                lines[w] = r[0]
                if w == "uniform-n4096-c2^20":
                    u4096_alpha = r[1]
        extra["lines"] = lines
    if "batched" in wanted:
        extra["batched"] = guarded(bench_batched, args, la, synth, dev, stream, l2_gbps)
    if "concurrent" in wanted:
        extra["concurrent_n4096"] = guarded(bench_concurrent, args, la, synth, dev, stream, u4096_alpha)
    if "warm" in wanted:
        extra["warm_start"] = guarded(bench_warm, args, la, synth, dev)
    if "sparse" in wanted:
        extra["sparse"] = guarded(bench_sparse, la, synth, dev)
    if "maxflow" in wanted:
        extra["maxflow"] = guarded(bench_maxflow, la, synth, dev)

    wrong = list(head["exact"]["wrong"])
    for w, l in lines.items():
        wrong += [dict(x, workload=w) for x in l.get("exact", {}).get("wrong", [])]
    if rank == 0:
        line = dict(head)
        line["read_probe"] = {"hbm_read_GBps": hbm_read_gbps, "hbm_buffer": "4 GiB, 2 passes per launch",
                              "l2_GBps": l2_gbps, "l2_buffer": "64 MiB, 20 passes per launch",
                              "kernel": "la_probe_read (128-bit ld.global.cg, 4 CTAs x 512 threads per SM)"}
        line["extra"] = extra
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if wrong:
        print(f"exactness gate failed: {wrong[:5]}", file=sys.stderr)
        return 1
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--alpha", type=int, default=0,
                    help="eps divisor of every line's timed solves (0: each line's own; 10: the paper's)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip every extra line")
    ap.add_argument("--extras", default="lines,batched,concurrent,warm,sparse,maxflow",
                    help="comma-separated extra lines: lines, batched, concurrent, warm, sparse, maxflow")
    ap.add_argument("--batch", type=int, default=10_000)
    ap.add_argument("--concurrent", type=int, default=608, help="n=4096 instances solved at once (extra line)")
    ap.add_argument("--no-tune", action="store_true", help="batched line with the library defaults, no autotuner")
    ap.add_argument("--warm-n1024", type=int, default=1000)
    ap.add_argument("--warm-n8192", type=int, default=16)
    ap.add_argument("--headline", default=HEADLINE, choices=sorted(LINES),
                    help="workload of the headline line (the others become extra lines)")
    ap.add_argument("--instances", type=int, default=0,
                    help="instances of the headline workload held on the device (0: the line's own count)")
    ap.add_argument("--clocks-dir", default=None,
                    help="folder for the raw nvidia-smi samples (default: the temp folder)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
