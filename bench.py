"""Benchmark: PCF Learned Sort on GB300 (one JSON line on rank 0).

Workload (one step): sort four arrays of n = 10^8 float64 keys, one per
distribution (Normal(0,1), LogNormal(0,1), Exponential(1), a 5-Gaussian
mixture), keys only, through pcf_sort_keys (pristine device input ->
device output; inputs are 800 MB each, larger than the 129 MB L2).  The
four independent sorts are issued by --sort-threads host threads (default
4, one per array), each with its own context and stream, so one
array's on-chip finish (instruction-bound) overlaps another's global
passes (memory-bound); every sort is the whole algorithm on its array.

  value        sorted Gkeys/s over the K timed steps (device-resident inputs)
  sequential   the same steps from one thread on one stream, for comparison
  e2e          the same through pcf_sort_keys_host_batch: the step's four
               arrays from pinned host buffers -> device -> sort -> host,
               every copy inside the timed region (the library overlaps
               one array's copies with its neighbours' sorts)
  roofline     the dominant stage's algorithmic bytes per launch / its mean
               launch time (CUDA events on the sort's stream, in two extra
               untimed steps), vs the measured copy bandwidth; traffic from
               the ncu capture in profiles/traffic.json when it matches the
               current sources
  roofline_job the whole sort's bytes (the library's pass model, and the
               48 B/key one-level minimum) per second vs the copy bandwidth
  cpu_baseline the CPU oracle, single-threaded, on a bounded sample

`--impl reference` times the CPU oracle instead (the reference arm).
Multi-GPU (torchrun): the sort does not shard; each rank sorts its own
replica of the workload ("weak" scaling, no collective on the data path).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
from concurrent.futures import ThreadPoolExecutor
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2405_07122_gb300 import workloads as W  # noqa: E402

N = 10**8
DISTS = [("normal", 1), ("lognormal", 2), ("exponential", 3), ("mixture", 4)]
METRIC = "sorted Gkeys/s"
WORKLOAD = "plain PCF sort, 4 arrays x 10^8 float64 keys (Normal, LogNormal, Exponential, 5-Gaussian mixture), keys only"
CPU_SAMPLE_N = 25 * 10**6

# algorithmic bytes per key of each kernel (keys only)
KERNEL_BYTES = {
    "range": 8,        # read the key
    "hist1_scan": 12,  # read the key, write its bucket id (the table hits L2)
    "scatter1": 22,    # read key + bucket id, write the key and its 2-byte low digit
    "hist2_scan": 2,   # read the low digit
    "scatter2": 18,    # read key + digit, write the key
    "leaf": 16,        # read and write each key finished on chip
}


def stage_traffic(stage, n):
    """DRAM bytes (read + write) of one launch of `stage` at n keys, scaled
    from the ncu capture summarised in profiles/traffic.json, or None when
    that capture was taken on sources that have changed since."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[stage]
        h = hashlib.sha256()
        for rel in rec["sources"]:
            with open(os.path.join(ROOT, rel), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != rec["sha256"]:
            return None
        return rec["dram_bytes_per_key"] * n
    except Exception:
        return None


def max_over_ranks(ms, dist, device=None):
    """The job's time is the slowest rank's (each rank sorts its own replica)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(keys_per_rank_step, world, steps, ms):
    """Whole-job throughput (Gkeys/s): every rank's keys over the slowest time."""
    return keys_per_rank_step * world * steps / (ms / 1e3) / 1e9


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 3 + k and r[3 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_gkeys(keys_list, model="pcf", range_mode="array"):
    """Single-threaded oracle on the first CPU_SAMPLE_N keys of each array."""
    import oracle
    pol = oracle.paper_policy(
        model=oracle.MODEL_SPLINE if model == "spline" else oracle.MODEL_PCF,
        range_mode=oracle.RANGE_SAMPLE if range_mode == "sample" else oracle.RANGE_ARRAY)
    total, secs = 0, 0.0
    for x in keys_list:
        s = np.ascontiguousarray(x[:CPU_SAMPLE_N])
        t0 = time.perf_counter()
        oracle.sort(s, policy=pol)
        secs += time.perf_counter() - t0
        total += s.size
    return total / secs / 1e9, total, secs


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    keys = [W.f64_keys(d, CPU_SAMPLE_N, seed) for d, seed in DISTS]
    import oracle
    oracle.lib()
    times = []
    for step in range(args.warmup + args.steps):
        total, secs = 0, 0.0
        for x in keys:
            t0 = time.perf_counter()
            oracle.sort(x)
            secs += time.perf_counter() - t0
            total += x.size
        if step >= args.warmup:
            times.append(secs)
    v = total / (sum(times) / len(times)) / 1e9
    sample = "first %d keys of each of the 4 distributions (n=%d per array, seeds as the GPU arm)" % (
        CPU_SAMPLE_N, CPU_SAMPLE_N)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gkeys/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (CPU oracle on a bounded sample)",
                       "n_per_array": CPU_SAMPLE_N, "arrays_per_step": 4},
            "cpu_baseline": {"value": v, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "Gkeys/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=N, help="keys per array (default 10^8)")
    ap.add_argument("--model", default="pcf", choices=["pcf", "spline"],
                    help="CDF model of the plain workload: the PCF of Sec. 3.3 (default) "
                         "or the spline of App. A.5 (Spline Learned Sort)")
    ap.add_argument("--range", default="array", choices=["array", "sample"],
                    help="range the bins span in the plain workload: the (sub)array's "
                         "(Sec. 3.3, default) or the alpha samples' (one pass fewer per level)")
    ap.add_argument("--workload", default="plain",
                    choices=["plain", "small", "zipf", "batched", "serve", "dupinject",
                             "failsweep"],
                    help="plain: the default 4 x 10^8 f64 line; the others are the "
                         "secondary configurations")
    ap.add_argument("--duration", type=float, default=10.0, help="serve: seconds of arrivals")
    ap.add_argument("--sort-threads", type=int, default=4, choices=[1, 2, 4],
                    help="plain workload: host threads issuing the step's four sorts, "
                         "one context and stream each (1: one thread, one stream)")
    ap.add_argument("--leaf-mode", type=int, default=0, choices=[0, 1, 2],
                    help="on-chip finish of keys-only sorts: 1 block-local sort, 2 Learned-Sort "
                         "steps in shared memory, 0 the library default (1)")
    args = ap.parse_args()
    n = args.n
    if args.workload != "plain" and args.impl == "ours":
        return run_secondary(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_07122_gb300 import pcfsort

    host_keys = [W.f64_keys(d, n, seed) for d, seed in DISTS]
    ins = [torch.from_numpy(x).to(dev) for x in host_keys]
    outs = [torch.empty_like(t) for t in ins]
    T = args.sort_threads
    ctxs = [pcfsort.Context(local) for _ in range(T)]
    for c in ctxs:
        if args.model != "pcf" or args.range != "array":
            c.set_policy(model=args.model, range_mode=args.range)
        if args.leaf_mode:
            c.set_tuning(leaf_mode=args.leaf_mode)
        c.reserve(n)
    ctx = ctxs[0]
    # the sorts' own streams (created non-blocking by torch): on the legacy
    # default stream every launch would also order against other streams
    streams = [torch.cuda.Stream(dev) for _ in range(T)]
    stream = streams[0]

    def sort_some(t, timing):
        # thread t: arrays t, t + T, ... on context t and stream t; a sort
        # call returns when its sort is complete on the device
        torch.cuda.set_device(local)
        st = {k: 0.0 for k in pcfsort.STAGES}
        launches, moved = 0, 0
        for i in range(t, 4, T):
            ctxs[t].sort_keys(ins[i], outs[i], key_type="f64", seed=0, stream=streams[t])
            s = ctxs[t].last_stats()
            launches += s["kernel_launches"]
            moved += s["bytes_moved"]
            if timing:
                for k, v in ctxs[t].stage_ms().items():
                    st[k] += v
        return st, launches, moved

    pool = ThreadPoolExecutor(max_workers=T) if T > 1 else None

    def step(timing=False, concurrent=True):
        if not concurrent or pool is None:
            # one thread, one stream: context 0 sorts all four arrays
            st = {k: 0.0 for k in pcfsort.STAGES}
            launches, moved = 0, 0
            for i in range(4):
                ctx.sort_keys(ins[i], outs[i], key_type="f64", seed=0, stream=stream)
                s = ctx.last_stats()
                launches += s["kernel_launches"]
                moved += s["bytes_moved"]
                if timing:
                    for k, v in ctx.stage_ms().items():
                        st[k] += v
            return st, launches, moved
        parts = list(pool.map(lambda t: sort_some(t, timing), range(T)))
        st = {k: sum(p[0][k] for p in parts) for k in pcfsort.STAGES}
        return st, sum(p[1] for p in parts), sum(p[2] for p in parts)

    def timed_steps(k, concurrent):
        # device time from an event on stream 0 (which the other streams wait
        # on) to one recorded there after the other streams' last work
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s2 in streams[1:]:
            s2.wait_event(e0)
        launches, moved = 0, 0
        for _ in range(k):
            _, nl, mv = step(concurrent=concurrent)
            launches += nl
            moved += mv
        for s2 in streams[1:]:
            ev = torch.cuda.Event()
            ev.record(s2)
            stream.wait_event(ev)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1), launches, moved

    for _ in range(args.warmup):
        if T > 1:
            step(concurrent=False)
        step()
    # correctness guard on the timed configuration (full check is in tests):
    # the outputs of the last warm-up step, taken in the timed form
    for o in outs:
        b = o.view(torch.int64)
        low63 = torch.tensor(2**63 - 1, dtype=torch.int64, device=dev)
        ok = torch.where(b < 0, b ^ low63, b)
        assert bool((ok[1:] >= ok[:-1]).all()), "output not sorted"

    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        ms_dev, launches, moved = timed_steps(args.steps, concurrent=True)
    ms = max_over_ranks(ms_dev, dist, dev)
    if dist:
        dist.barrier()
    keys_per_step = 4 * n * world
    value = job_value(4 * n, world, args.steps, ms)
    # the one-thread, one-stream form of the same steps (untimed by the
    # contract, reported beside the value)
    if T > 1:
        if dist:
            dist.barrier()
        ms_seq = max_over_ranks(timed_steps(args.steps, concurrent=False)[0], dist, dev)
        sequential = {"value": job_value(4 * n, world, args.steps, ms_seq), "unit": "Gkeys/s",
                      "ms_per_step": ms_seq / args.steps,
                      "how": "the same steps from one host thread on one stream"}
    else:
        sequential = None
    # stage breakdown (CUDA events on the sort's stream), untimed steps
    ctx.enable_timing(True)
    t_steps = 2
    stages = {k: 0.0 for k in pcfsort.STAGES}
    for _ in range(t_steps):
        st, _, _ = step(timing=True, concurrent=False)
        for k in stages:
            stages[k] += st[k]
    ctx.enable_timing(False)

    # end to end: the step's arrays from pinned host buffers -> device ->
    # sort -> host, one public call per step (each array back on the host,
    # sorted, when it returns); the inputs are restored between steps,
    # outside the timed region
    pinned = [torch.from_numpy(x.copy()).pin_memory() for x in host_keys]
    ctx.sort_keys_host_batch(pinned, key_type="f64", stream=stream)
    torch.cuda.synchronize(dev)
    e_steps = max(1, min(args.steps, 3))
    e2e_s = 0.0
    for _ in range(e_steps):
        for p, x in zip(pinned, host_keys):
            p.copy_(torch.from_numpy(x))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx.sort_keys_host_batch(pinned, key_type="f64", stream=stream)
        torch.cuda.synchronize(dev)
        e2e_s += time.perf_counter() - t0
    e2e = keys_per_step * e_steps / e2e_s / 1e9
    assert all(bool((p[1:] >= p[:-1]).all()) for p in pinned), "e2e output not sorted"

    peak, peak_kind = peaks()
    # the library's own 16-byte copy over two 800 MB arrays: the passes'
    # access pattern at full speed, a reference beside the measured peak
    copy_gbs = ctx.copy_bandwidth(ins[0], outs[0], reps=10, stream=stream)
    per_launch = {}
    for k, b in KERNEL_BYTES.items():
        ms_k = stages[k] / (t_steps * 4)
        if ms_k > 0:
            per_launch[k] = (ms_k, b)
    dom = max(per_launch, key=lambda k: per_launch[k][0])
    dom_ms, dom_b = per_launch[dom]
    # keys processed by one launch of the dominant stage: all n (every key of
    # this workload passes through the global passes and the on-chip finish)
    achieved = dom_b * n / (dom_ms / 1e3) / 1e9
    step_s = ms / args.steps / 1e3
    # the whole sort against the copy peak first (the target is defined on
    # it): the bytes the passes it ran must move (the library's pass model),
    # and the 48 B/key minimum of one bucketing level (range 8, predict 8,
    # move 16, finish 16)
    roofline_job = {"frac_measured_passes": moved / args.steps / step_s / 1e9 / peak,
                    "bytes_measured_passes": moved / args.steps,
                    "frac_algorithmic": 48 * 4 * n / step_s / 1e9 / peak,
                    "bytes_algorithmic": 48 * 4 * n, "peak": peak, "peak_kind": peak_kind}
    line = {
        "metric": METRIC, "value": value, "unit": "Gkeys/s", "roofline_job": roofline_job,
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": (WORKLOAD if n == N else WORKLOAD.replace("10^8", str(n)))
                   .replace("plain PCF sort", "plain PCF sort" if args.model == "pcf"
                            else "Spline Learned Sort (App. A.5)")
                   + ("" if args.range == "array" else ", bins over the samples' range"),
                   "n_per_array": n, "arrays_per_step": 4,
                   "l2": "inputs larger than L2 (800 MB per array, L2 129 MB)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "e2e": {"value": e2e, "unit": "Gkeys/s", "h2d_bytes_per_step": 8 * 4 * n,
                "d2h_bytes_per_step": 8 * 4 * n},
        "gpu_launches": int(launches),
        # every stage against the same peak: its algorithmic bytes per key x
        # n over its time per array (all levels of the array included)
        "stage_rooflines": {k: {"bytes_per_key": b_k, "ms_per_array": ms_k,
                                "achieved_gbs": b_k * n / (ms_k / 1e3) / 1e9,
                                "frac": b_k * n / (ms_k / 1e3) / 1e9 / peak}
                            for k, (ms_k, b_k) in per_launch.items()},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": stage_traffic(dom, n), "bytes_per_key": dom_b,
                     "copy_kernel_gbs": copy_gbs},
        "stage_ms_per_array": {k: v / (t_steps * 4) for k, v in stages.items()},
        "clocks": clk.summary(),
    }
    line["config"]["sort_threads"] = T
    line["config"]["streams"] = ("%d host threads, one context and stream each, arrays "
                                 "round-robin; stage times from one-stream steps" % T
                                 if T > 1 else "one host thread, one stream")
    if sequential:
        line["sequential"] = sequential
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, total, secs = cpu_oracle_gkeys(host_keys, args.model, args.range)
        line["cpu_baseline"] = {"value": v, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
                                "sample": "first %d keys of each of the 4 arrays (%d keys, %.1f s)"
                                          % (CPU_SAMPLE_N, total, secs)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pool is not None:
        pool.shutdown()
    for c in ctxs:
        c.close()
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# secondary configurations (not the default line)
# ---------------------------------------------------------------------------
def secondary_roofline(torch, ctx, run, n_global, n_total, peak, peak_kind):
    """Stage times of one more run (CUDA events on the sort's stream) and the
    dominant stage's roofline.  Algorithmic bytes: the global passes move
    every key of the arrays they bucket (n_global, level 0 counted once: a
    lower bound where keys take further levels), the on-chip finish reads
    and writes every key not sent to the standard sort, the standard sort at
    least one read and write of its keys."""
    ctx.enable_timing(True)
    run()
    torch.cuda.synchronize()
    st = ctx.stage_ms()
    stats = ctx.last_stats()
    ctx.enable_timing(False)
    fb = stats["fallback_keys"]
    algo = {k: KERNEL_BYTES[k] * n_global for k in
            ("range", "hist1_scan", "scatter1", "hist2_scan", "scatter2")}
    algo["leaf"] = KERNEL_BYTES["leaf"] * (n_total - fb)
    algo["fallback"] = 16 * fb
    cand = {k: v for k, v in st.items() if k in algo and v > 0 and algo[k] > 0}
    dom = max(cand, key=cand.get)
    achieved = algo[dom] / (cand[dom] / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
            "bytes": algo[dom]}
    return roof, st, stats


def oracle_sample(arrays, vals=None, threads=1):
    """The CPU oracle, as it stands, on host arrays: (Gkeys/s, keys, seconds,
    threads used).  threads > 1: one array per host thread (its C calls
    release the GIL)."""
    import concurrent.futures as cf
    import oracle
    oracle.lib()
    total = sum(int(a.size) for a in arrays)

    def one(i):
        oracle.sort(arrays[i], None if vals is None else vals[i])

    t0 = time.perf_counter()
    if threads > 1:
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(one, range(len(arrays))))
    else:
        for i in range(len(arrays)):
            one(i)
    secs = time.perf_counter() - t0
    return total / secs / 1e9, total, secs, threads


def _cpu_line(v, total, secs, cores, what):
    return {"value": v, "unit": "Gkeys/s", "cores": cores, "kind": "oracle",
            "sample": "%s (%d keys, %.1f s)" % (what, total, secs)}


def _device_sort_timer(torch):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    return timed


def run_secondary(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_07122_gb300 import pcfsort
    timed = _device_sort_timer(torch)
    ctx = pcfsort.Context(0)
    peak, peak_kind = peaks()
    cpu = not args.no_cpu_baseline
    line = {"impl": "ours", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "unit": "Gkeys/s"}
    if args.workload == "small":
        xh = W.f64_keys("uniform", 10**6, 0)
        x = torch.from_numpy(xh).cuda()
        o = torch.empty_like(x)
        run = lambda: ctx.sort_keys(x, o, key_type="f64")  # noqa: E731
        ms = timed(run, max(args.steps, 10))
        roof, st, stats = secondary_roofline(torch, ctx, run, 10**6, 10**6, peak, peak_kind)
        line.update(metric=METRIC, value=1e6 / ms / 1e6, ms_per_sort=ms, dtype="f64",
                    roofline=roof, stage_ms=st,
                    plain_form="this line is the plain per-array form",
                    config={"workload": "plain PCF sort, n = 10^6 float64 Uniform[0,1), keys only"})
        if cpu:
            line["cpu_baseline"] = _cpu_line(*oracle_sample([xh]), "the same 10^6 keys")
    elif args.workload == "zipf":
        n = 2**28
        k = W.zipf_u64(n, seed=5)
        v = np.arange(n, dtype=np.uint32)
        tk = torch.from_numpy(k.view(np.int64)).cuda()
        tv = torch.from_numpy(v.view(np.int32)).cuda()
        ko, vo = torch.empty_like(tk), torch.empty_like(tv)
        run = lambda: ctx.sort_pairs(tk, tv, ko, vo, key_type="u64")  # noqa: E731
        ms = timed(run, max(1, args.steps))
        st = ctx.last_stats()
        # sorted as unsigned keys, equal keys in input order (payload = index),
        # and every payload still with its key
        flip = torch.tensor(-2**63, dtype=torch.int64, device="cuda")
        a, b = ko[:-1] ^ flip, ko[1:] ^ flip
        assert bool(((a < b) | ((a == b) & (vo[:-1] < vo[1:]))).all()), "pairs not stably sorted"
        assert bool((tk[vo.long()] == ko).all()), "a payload left its key"
        assert bool((torch.sort(vo).values == tv).all()), "payloads not a permutation"
        roof, stages, _ = secondary_roofline(torch, ctx, run, n, n, peak, peak_kind)
        line.update(metric=METRIC, value=n / ms / 1e6, ms_per_sort=ms, dtype="u64",
                    stats=st, roofline=roof, stage_ms=stages,
                    plain_form="this line is the plain per-array form",
                    config={"workload": "PCF sort, n = 2^28 uint64 keys, Zipf(1.2) over 10^7 "
                                        "hashed values, uint32 payload = index (stable pairs)"})
        if cpu:
            m = 1 << 24
            line["cpu_baseline"] = _cpu_line(*oracle_sample([k[:m]], [v[:m]]),
                                             "the first 2^24 key-value pairs")
    elif args.workload == "dupinject":
        # the appendix's adversarial input at GPU scale: 5x10^7 Normal(0,1)
        # keys plus as many copies of one value drawn in [min, max], shuffled
        x = W.inject_duplicates(W.f64_keys("normal", 5 * 10**7, 9), seed=9)
        n = x.size
        t = torch.from_numpy(x).cuda()
        o = torch.empty_like(t)
        run = lambda: ctx.sort_keys(t, o, key_type="f64")  # noqa: E731
        ms = timed(run, max(3, args.steps))
        st = ctx.last_stats()
        b = o.view(torch.int64)
        flip = torch.tensor(2**63 - 1, dtype=torch.int64, device="cuda")
        ok = torch.where(b < 0, b ^ flip, b)
        assert bool((ok[1:] >= ok[:-1]).all()), "output not sorted"
        roof, stages, _ = secondary_roofline(torch, ctx, run, n, n, peak, peak_kind)
        line.update(metric=METRIC, value=n / ms / 1e6, ms_per_sort=ms, dtype="f64", stats=st,
                    roofline=roof, stage_ms=stages,
                    plain_form="this line is the plain per-array form",
                    config={"workload": "duplicate injection (appendix): 5x10^7 Normal(0,1) "
                                        "float64 keys + 5x10^7 copies of one value in [min, max], "
                                        "shuffled, keys only", "n": n})
        if cpu:
            sub = W.inject_duplicates(W.f64_keys("normal", 5 * 10**6, 9), seed=9)
            line["cpu_baseline"] = _cpu_line(*oracle_sample([sub]),
                                             "the same recipe at 5x10^6 + 5x10^6 keys")
    elif args.workload == "failsweep":
        # Sec. 4.2: level-0 bucketing of R = 100 uniform arrays of 10^6 keys
        # at every grid setting of the six heat maps (two of a, b, c, d
        # varied over 0.05..0.95, the others 0.75), failure = a bucket of
        # more than delta keys
        from paper_2405_07122_gb300 import failsweep as F
        n, R = 10**6, 100
        x = np.concatenate([W.f64_keys("uniform", n, 1000 + r) for r in range(R)])
        keys = torch.from_numpy(x).cuda()
        offs = np.arange(R + 1, dtype=np.uint64) * n
        F.heat_map(ctx, keys, offs, n, ("a", "b"), grid=[0.75])  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        maps = {ax: F.heat_map(ctx, keys, offs, n, ax) for ax in F.MAPS}
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        settings = len(F.MAPS) * len(F.GRID) ** 2
        summary = {}
        for ax, pts in maps.items():
            inside, viol = F.agreement(pts)
            # one row per value of the second axis (0.95 first), one digit per
            # value of the first: failure frequency x 10 (X = every array)
            rows = ["".join("X" if pts[(xv, yv)][0] >= 1.0 else str(int(pts[(xv, yv)][0] * 10))
                            for xv in F.GRID) for yv in reversed(F.GRID)]
            summary["".join(ax)] = {"bound_le_half": inside, "of_those_failing_often": viol,
                                    "freq_x10_rows_y_desc": rows}
        line.update(metric="bucketed Gkeys/s (failure sweep)",
                    value=settings * R * n / secs / 1e9, ms_per_setting=secs * 1e3 / settings,
                    dtype="f64", maps=summary,
                    config={"workload": "Sec. 4.2 bucketing-failure sweep: 6 heat maps x 19 x 19 "
                                        "settings, each bucketing 100 Uniform[0,1) arrays of "
                                        "10^6 float64 keys (level 0 of Algorithm 1)",
                            "settings": settings, "arrays_per_setting": R})
    elif args.workload == "batched":
        keys, offs, _dists = W.batched_f64(2048, seed=6)
        total = int(offs[-1])
        t = torch.from_numpy(keys).cuda()
        o = torch.empty_like(t)
        # the knobs (digit width, count-tile size, on-chip capacity) chosen by
        # the autotuner on a sample of the batch: its first 512 arrays (not timed)
        from paper_2405_07122_gb300 import autotune
        s_offs = offs[:513]
        s_in, s_out = t[:int(s_offs[-1])], torch.empty(int(s_offs[-1]), dtype=t.dtype,
                                                        device=t.device)
        tctx = autotune.tuned_context(
            autotune.workload_key("segmented", total),
            sample_runner=lambda c: c.sort_segmented(s_in, s_offs, keys_out=s_out,
                                                     key_type="f64"))
        tuning = tctx.tuning()
        del s_out
        # the batched form: one CUDA graph replay of the whole segmented sort
        # (creating the graph sorts once and captures; not timed)
        graph = pcfsort.SortGraph(tctx, t, offs, o, key_type="f64")
        batched_out = o.clone()
        replayed = []
        ms_g = timed(lambda: replayed.append(graph.launch()), max(1, args.steps))
        ginfo = graph.info()
        assert bool((o == batched_out).all()), "graph replay output differs"
        ms_b = timed(lambda: ctx.sort_segmented(t, offs, keys_out=o, key_type="f64"),
                     max(1, args.steps))
        assert bool((o == batched_out).all()), "segmented call and graph outputs differ"

        def plain():
            for s in range(2048):
                a, b = int(offs[s]), int(offs[s + 1])
                ctx.sort_keys(t[a:b], o[a:b], key_type="f64", seed=s)
        ms_p = timed(plain, 1)
        assert bool((o == batched_out).all()), "batched and plain outputs differ"
        roof, stages, _ = secondary_roofline(
            torch, ctx, lambda: ctx.sort_segmented(t, offs, keys_out=o, key_type="f64"),
            int(sum(b - a for a, b in zip(offs[:-1], offs[1:]) if b - a > 8192)), total, peak,
            peak_kind)
        # fresh data every launch: new keys for every array (same lengths and
        # distributions, new seeds, drawn on the device); the graph replays
        # when the sort takes its recorded plan, else sorts without it and
        # records again
        gen = torch.Generator(device="cuda")
        bounds = torch.zeros(total, dtype=torch.bool, device="cuda")
        bounds[torch.from_numpy(offs[1:-1].astype(np.int64)).cuda()] = True
        fresh = []
        for r in range(5):
            gen.manual_seed(1000 + r)
            for i, d in enumerate(_dists):
                a, b = int(offs[i]), int(offs[i + 1])
                t[a:b] = _torch_dist(torch, d, b - a, gen)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = graph.launch()
            torch.cuda.synchronize()
            fresh.append((rep, (time.perf_counter() - t0) * 1e3))
            ob = o.view(torch.int64)
            low63 = torch.tensor(2**63 - 1, dtype=torch.int64, device="cuda")
            ordk = torch.where(ob < 0, ob ^ low63, ob)
            assert bool(((ordk[1:] >= ordk[:-1]) | bounds[1:]).all()), "fresh batch not sorted"
        fresh_ms = sorted(ms for _, ms in fresh)
        line["fresh_data"] = {"launches": len(fresh),
                              "replayed": sum(1 for rep, _ in fresh if rep),
                              "ms_per_launch": [round(ms, 3) for _, ms in fresh],
                              "value": total / fresh_ms[len(fresh_ms) // 2] / 1e6,
                              "unit": "Gkeys/s",
                              "how": "new keys in every array before each pcf_graph_launch "
                                     "(drawn on the device, same lengths and distributions, "
                                     "new seeds); host wall time of the call (the replay and "
                                     "its status read; a miss sorts without the graph and "
                                     "records again); value = keys / median time"}
        graph.close()
        tctx.close()
        if cpu:
            # the oracle on the first 256 arrays: one array per host core, and
            # single-threaded
            sample = [keys[int(offs[i]):int(offs[i + 1])] for i in range(256)]
            ncores = os.cpu_count() or 1
            line["cpu_baseline"] = _cpu_line(*oracle_sample(sample, threads=ncores),
                                             "the first 256 arrays, one array per core")
            line["cpu_baseline_1core"] = _cpu_line(*oracle_sample(sample[:64]),
                                                   "the first 64 arrays, one core")
        line.update(roofline=roof, stage_ms=stages)
        line.update(metric=METRIC, value=total / ms_g / 1e6, ms_per_batch=ms_g,
                    graph={"captured": ginfo["captured"], "every_launch_replayed": all(replayed),
                           "launches": len(replayed)},
                    segmented_call_value=total / ms_b / 1e6, segmented_call_ms=ms_b,
                    plain_value=total / ms_p / 1e6, plain_ms=ms_p, dtype="f64",
                    config={"workload": "batched segmented sort: 2048 float64 arrays, lengths "
                                        "floor(2^U(10,22)), distributions drawn from 5",
                            "total_keys": total, "tuning": tuning,
                            "tuned_by": "autotune.tuned_context on the first 512 arrays",
                            "form": "one CUDA graph replay of the segmented sort "
                                    "(pcf_graph_launch) vs one pcf_sort_segmented call vs "
                                    "2048 pcf_sort_keys calls"})
    elif args.workload == "serve":
        from paper_2405_07122_gb300 import serve
        stream = W.request_stream(2000.0, args.duration, seed=7)
        # device pools per (key type, distribution): requests take slices
        pool_n = 1 << 26
        pools = {}
        g = torch.Generator(device="cuda")
        g.manual_seed(7)
        for d in W.DISTRIBUTIONS:
            f = _torch_dist(torch, d, pool_n, g)
            pools[("f64", d)] = f
            pools[("u64", d)] = (torch.round(f * 4294967296.0).to(torch.int64) +
                                 torch.tensor(-2**63, dtype=torch.int64, device="cuda"))
        torch.cuda.synchronize()
        rng = np.random.Generator(np.random.PCG64(8))
        reqs = [(ta, pools[(kt, dist)][off:off + n], kt)
                for (ta, n, kt, dist, _s), off in
                ((r, int(rng.integers(0, pool_n - r[1] + 1))) for r in stream)]

        def serve_run(items, paced):
            """Submits items (arrival time, keys, type); paced: at their
            arrival times, else all at once (the server's capacity).  The
            client takes each result as it completes and releases it."""
            srv = serve.SortServer(device=0, workers=4, mem_budget=64 << 30,
                                   batch_keys=1 << 27)
            handles, pending = [], []

            def consume(block=False):
                keep = []
                for h in pending:
                    if block:
                        h.done.wait()
                    if h.done.is_set():
                        h.release()
                    else:
                        keep.append(h)
                pending[:] = keep

            t0 = time.perf_counter()
            for ta, keys, kt in items:
                if paced:
                    now = time.perf_counter() - t0
                    if ta > now:
                        time.sleep(ta - now)
                h = srv.submit(keys, kt)
                handles.append(h)
                pending.append(h)
                consume()
            consume(block=True)
            t1 = time.perf_counter()
            srv.close()
            errors = [h.error for h in handles if h.error is not None]
            if errors:
                raise RuntimeError("%d of %d requests failed, first: %r"
                                   % (len(errors), len(handles), errors[0]))
            keys_done = sum(h.n for h in handles)
            return keys_done / (t1 - t0) / 1e9, serve.latency_summary(handles), keys_done

        value, lat, keys_done = serve_run(reqs, True)
        # capacity: the first 4000 requests submitted at once (the queue
        # never runs dry), and the same requests sorted one by one with
        # pcf_sort_keys on one stream (the plain per-request form)
        head = reqs[:4000]
        cap, cap_lat, cap_keys = serve_run(head, False)
        obuf = torch.empty(max(k.numel() for _, k, _ in head), dtype=torch.int64,
                           device="cuda")

        def plain():
            for _, k, kt in head:
                o = obuf[:k.numel()]
                ctx.sort_keys(k, o if k.dtype == torch.int64 else o.view(torch.float64),
                              key_type=kt)
        ms_plain = timed(plain, 1)
        line.update(metric="served sorted Gkeys/s (sustained)",
                    value=value, latency=lat, requests=len(reqs),
                    offered_gkeys_per_s=keys_done / args.duration / 1e9, dtype="f64|u64",
                    capacity={"value": cap, "unit": "Gkeys/s", "latency": cap_lat,
                              "requests": len(head),
                              "how": "the first 4000 requests submitted at once"},
                    plain_form={"value": cap_keys / (ms_plain / 1e3) / 1e9, "unit": "Gkeys/s",
                                "how": "the same 4000 requests, one pcf_sort_keys call each, "
                                       "one stream"},
                    config={"workload": "serving loop: Poisson arrivals 2000/s, sizes "
                                        "floor(2^U(12,26)), f64 or u64, 5 distributions, "
                                        "64 GB admission budget (resident result pool), "
                                        "4 streams",
                            "duration_s": args.duration})
        if cpu:
            smp = [k.cpu().numpy() for _, k, _ in head[:20]]
            smp = [a if a.dtype == np.float64 else a.view(np.uint64) for a in smp]
            line["cpu_baseline"] = _cpu_line(*oracle_sample(smp),
                                             "the first 20 requests, one core")
    ctx.close()
    print(json.dumps(line), flush=True)
    return 0


def _torch_dist(torch, dist, n, g):
    if dist == "uniform":
        return torch.rand(n, dtype=torch.float64, device="cuda", generator=g)
    if dist == "normal":
        return torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    if dist == "lognormal":
        return torch.exp(torch.randn(n, dtype=torch.float64, device="cuda", generator=g))
    if dist == "exponential":
        return -torch.log1p(-torch.rand(n, dtype=torch.float64, device="cuda", generator=g))
    means = torch.rand(5, dtype=torch.float64, device="cuda", generator=g) * 200 - 100
    sds = torch.rand(5, dtype=torch.float64, device="cuda", generator=g) * 9.9 + 0.1
    comp = torch.randint(0, 5, (n,), device="cuda", generator=g)
    return means[comp] + sds[comp] * torch.randn(n, dtype=torch.float64, device="cuda",
                                                  generator=g)


if __name__ == "__main__":
    sys.exit(main())
