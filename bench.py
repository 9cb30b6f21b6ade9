#!/usr/bin/env python3
"""Items packed per second on the batched VSBPP workload, on GB300.

Workload (config 3): 4096 independent instances in one batch, m per instance
log-uniform in [100, 10^4], n in {3,5,7}, capacities distinct integers in
[20, 1000] sorted descending, weights uniform in [1, B_1] (seeded synthetic
data standing in for the paper's benchmark files).

One step = one pass of the whole hot path over the batch: the first
heuristic (Section 6.3) with FF, BF and WF, and the second heuristic
(Section 6.4, 5-item sublists, BF), each a CUDA-graph replay of the batched
persistent launch; the four passes run at once, each on a stream of its
own (the step is timed from the fork to the join).  items_per_step =
4 * sum(m).  L2 is flushed (a 256 MiB
write) before every timed step, outside the timed region.  The same passes
back to back on one stream are reported as serial_ms_per_step.

Also reported: the same step through the plain path (one kernel launch per
instance), end-to-end throughput with host buffers (copies timed), the
fit-test (integer ALU) roofline of the dominant kernel, timed with CUDA events
through the library's kernel-timing hook, SM clocks sampled during the timed
region, and the CPU oracle on a bounded sample on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PASSES = [("H1-FF", 1, 0, 0), ("H1-BF", 1, 1, 0), ("H1-WF", 1, 2, 0), ("H2-BF", 2, 1, 5)]
# kernels one step launches: three first-heuristic passes x (validate, order,
# scatter, large/small/wide packing kernels, full-size rerun) + second
# heuristic (validate, sublist scan, permutation kernel, compose)
LAUNCHES_PER_STEP = 3 * 7 + 4
WORKLOAD = "config3: 4096 VSBPP instances, m log-uniform [100,1e4], n in {3,5,7}, B in [20,1000], w~U[1,B1]"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--instances", type=int, default=4096)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=1024, help="instances in the oracle sample")
    ap.add_argument("--no-side", action="store_true", help="skip configs 1, 2, 4 and 5 side numbers")
    ap.add_argument("--no-autotune", action="store_true", help="use the library's default launch config")
    ap.add_argument("--config4-instances", type=int, default=64)
    ap.add_argument("--config4-m", type=int, default=1_000_000)
    ap.add_argument("--only", choices=["all", "config4"], default="all",
                    help="config4: run only the config-4 pass (a small case for profiling)")
    ap.add_argument("--profile-once", action="store_true",
                    help="run each pass of one step once, untimed, and exit (for ncu captures)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="config 5 arrivals per second")
    ap.add_argument("--serve-requests", type=int, default=400)
    return ap.parse_args()


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ clocks
CLOCK_FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"vsbpp_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
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
        try:
            self.f.close()
        except Exception:
            pass

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
            os.remove(self.path)
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for k, nm in enumerate(names):
                    if r[4 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if sm:
            out.update(sm_mhz=float(np.median(sm)), sm_max_mhz=float(max(mx)), samples=len(sm),
                       reasons=sorted(reasons))
        return out


# ----------------------------------------------------------- side numbers
def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def single_instance_latency(native, I, dev, stream):
    """Configs 1 and 2: one instance per call, device-resident, per pass."""
    import torch
    out = {}
    for name, batch in (("config1", I.config1()), ("config2u", I.config2("u")), ("config2m", I.config2("m"))):
        db = native.DeviceBatch.from_host(batch, device=dev)
        res = native.DeviceResult.empty(db.N, db.total_items, device=dev)
        row = {}
        for (pname, h, c, s_) in PASSES:
            plan = native.Plan(db.N, db.total_items, db.max_m, h, c, s_)
            for _ in range(3):
                plan.run(db, res, stream)
            e0, e1 = _events(torch)
            reps = 5
            e0.record(stream)
            for _ in range(reps):
                plan.run(db, res, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            row[pname] = {"ms": ms, "items_per_s": db.total_items / (ms / 1e3)}
            plan.close()
        out[name] = row
    return out


def config4_pass(native, I, dev, stream, N, m=1_000_000):
    """Config 4: N instances of 10^6 items (the two-CTA cluster kernel, the
    global-memory kernel past it), one first-heuristic pass per criterion."""
    import torch
    batch = I.config4(N=N, m=m)
    db = native.DeviceBatch.from_host(batch, device=dev)
    res = native.DeviceResult.empty(db.N, db.total_items, device=dev)
    out = {"instances": db.N, "items": db.total_items}
    for name, crit in (("H1-BF", 1), ("H1-FF", 0), ("H1-WF", 2)):
        plan = native.Plan(db.N, db.total_items, db.max_m, 1, crit, 0)
        plan.run(db, res, stream)                   # warm-up (records the graph)
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record(stream)
        plan.run(db, res, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ok = int((res.status[:db.N] == 0).sum().item())
        plan.close()
        out[name] = {"ms": ms, "items_per_s": db.total_items / (ms / 1e3),
                     "us_per_item_per_system": ms * 1e3 / max(m, 1), "instances_ok": ok}
    return out


def exhaustive_search(native, I, dev, stream):
    """The exhaustive second heuristic (Section 7's comparison): one list of
    10 and one of 12 items, every permutation packed (BF)."""
    import torch
    rng = np.random.default_rng(12)
    res = {}
    for m in (10, 12):
        b = I.from_instances([I.random_instance(rng, m, 5, 150)])
        db = native.DeviceBatch.from_host(b, device=dev)
        out = native.DeviceResult.empty(db.N, db.total_items, device=dev)
        assert native.pack_batch(db, out, 2, 1, m, stream=stream) == 0
        e0, e1 = _events(torch)
        torch.cuda.synchronize()
        e0.record(stream)
        assert native.pack_batch(db, out, 2, 1, m, stream=stream) == 0
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        perms = math.factorial(m)
        res[f"m{m}"] = {"ms": ms, "permutations": perms, "permutations_per_s": perms / (ms / 1e3),
                        "total": int(out.total[0].item())}
    return res


def latency_roof(native, batch, dev, stream, flush, name, kernel_ms, sm_mhz, reps):
    """The bound that binds the batched first heuristic: each membrane
    system is a chain of dependent item steps (Rule 3 takes one item per
    step), so a pass cannot end before its largest system, packed alone.
    Reported: that system's solo kernel time (CUDA events on the launching
    stream, L2 flushed), its cycles per item at the sampled SM clock, the
    batched kernel's time over it, and the cycles per item of a system of as
    many unit items with one capacity of 1000 (a handful of bins alive: the
    chain's floor, since the kernel's work per item does not grow with the
    bins)."""
    import torch
    from paper_1602_08735_gb300 import instances as I
    h, c, s_ = dict((p[0], p[1:]) for p in PASSES)[name]
    big = int(np.argmax(np.diff(batch.w_off)))
    one = I.from_instances([batch.instance(big)])
    db1 = native.DeviceBatch.from_host(one, device=dev)
    out1 = native.DeviceResult.empty(1, db1.total_items, device=dev)
    assert native.pack_batch(db1, out1, h, c, s_, stream=stream) == 0
    native.kernel_timing_enable(True)
    native.kernel_timing_read()
    for _ in range(reps):
        flush.zero_()
        assert native.pack_batch(db1, out1, h, c, s_, stream=stream) == 0
    t = native.kernel_timing_read()
    native.kernel_timing_enable(False)
    solo = float(np.mean(t))
    m = db1.total_items
    # the chain's floor: the same number of unit items into one capacity of
    # 1000 (at most 2 * ceil(m / 1000) bins ever alive), the same pass
    few = I.from_instances([(np.ones(m, dtype=np.int32), np.array([1000], dtype=np.int32))])
    dbf = native.DeviceBatch.from_host(few, device=dev)
    outf = native.DeviceResult.empty(1, dbf.total_items, device=dev)
    assert native.pack_batch(dbf, outf, h, c, s_, stream=stream) == 0
    native.kernel_timing_enable(True)
    native.kernel_timing_read()
    for _ in range(reps):
        flush.zero_()
        assert native.pack_batch(dbf, outf, h, c, s_, stream=stream) == 0
    tf = native.kernel_timing_read()
    native.kernel_timing_enable(False)
    few_ms = float(np.mean(tf))
    return {"bound": "per-system dependent chain (largest system packed alone)", "pass": name,
            "largest_m": m, "solo_kernel_ms": solo, "sm_mhz": sm_mhz,
            "chain_cycles_per_item": solo * 1e-3 * sm_mhz * 1e6 / m,
            "batched_kernel_ms": kernel_ms, "kernel_over_solo": kernel_ms / solo if solo else None,
            "few_bins": {"items": m, "capacity": 1000, "bins": int(outf.num_bins.cpu()[0]), "kernel_ms": few_ms,
                         "cycles_per_item": few_ms * 1e-3 * sm_mhz * 1e6 / m}}


def serve_stream(native, reqs, rate):
    """Submit reqs at their arrival times (rate None: all at once) and poll
    them all; returns the server's stats and the wall time."""
    items = sum(len(w) for (_, w, _) in reqs)
    with native.Server(device_mem_budget=8 << 30, max_slots=64, lanes=32) as srv:
        t0 = time.perf_counter()
        tickets = []
        for (t_arr, w, B) in reqs:
            if rate is not None:
                now = time.perf_counter() - t0
                if t_arr > now:
                    time.sleep(t_arr - now)
            tickets.append(srv.submit(w, B, 1, 1))
        bad = 0
        for t in tickets:
            rc, _ = srv.poll(t)
            bad += rc != 0
        wall = time.perf_counter() - t0
        st = srv.stats()
    return {"rate_per_s": rate, "requests": len(reqs), "items": items, "failed": bad,
            "p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3, "max_ms": st["max_us"] / 1e3,
            "wait_p50_ms": st["wait_p50_us"] / 1e3, "wait_p99_ms": st["wait_p99_us"] / 1e3,
            "service_p50_ms": st["service_p50_us"] / 1e3, "service_p99_ms": st["service_p99_us"] / 1e3,
            "items_per_s": items / wall, "requests_per_s": len(reqs) / wall, "wall_s": wall,
            "busy_s": st["busy_s"]}


def serving_sweep(native, I, n_req):
    """Config 5 through the continuous-batching server: capacity with every
    request queued at once (requests/s over the server's busy time), then
    Poisson arrivals at 50 %, 90 % and 110 % of that capacity."""
    sat = serve_stream(native, I.config5(seed=5, num_requests=n_req, rate_per_s=1e9), None)
    cap = sat["requests"] / max(sat["busy_s"], 1e-9)
    points = []
    for frac in (0.5, 0.9, 1.1):
        rate = frac * cap
        pt = serve_stream(native, I.config5(seed=5, num_requests=n_req, rate_per_s=rate), rate)
        pt["fraction_of_capacity"] = frac
        points.append(pt)
    return {"pass": "H1-BF per request", "m": "log-uniform [100, 1e5]", "capacity_requests_per_s": cap,
            "capacity_items_per_s": sat["items"] / max(sat["busy_s"], 1e-9), "saturated": sat,
            "points": points}


def variants_side(native, db, dev, stream, flush):
    """One config-3 first-heuristic BF pass with each option (event-timed
    call of the batched entry point, L2 flushed)."""
    import torch
    out = native.DeviceResult.empty(db.N, db.total_items, device=dev)
    res = {}
    for label, kw in (("plain_method", {}), ("presort", dict(flags=native.PRESORT)),
                      ("remark3", dict(flags=native.REMARK3)), ("bounded_K8", dict(max_open=8)),
                      ("bounded_K32", dict(max_open=32))):
        assert native.pack_batch(db, out, 1, 1, stream=stream, **kw) == 0
        e0, e1 = _events(torch)
        ms = 0.0
        for _ in range(3):
            flush.zero_()
            e0.record(stream)
            assert native.pack_batch(db, out, 1, 1, stream=stream, **kw) == 0
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1) / 3
        res[label] = {"ms": ms, "items_per_s": db.total_items / (ms / 1e3),
                      "total_capacity": int(out.total[:db.N].sum().item())}
    return res


def serving_run(native, I, rate, n_req):
    """Config 5: Poisson arrivals through the continuous-batching server."""
    reqs = I.config5(seed=5, num_requests=n_req, rate_per_s=rate)
    items = sum(len(w) for (_, w, _) in reqs)
    with native.Server(device_mem_budget=8 << 30, max_slots=64, lanes=32) as srv:
        t0 = time.perf_counter()
        tickets = []
        for (t_arr, w, B) in reqs:
            now = time.perf_counter() - t0
            if t_arr > now:
                time.sleep(t_arr - now)
            tickets.append(srv.submit(w, B, 1, 1))
        bad = 0
        for t in tickets:
            rc, _ = srv.poll(t)
            bad += rc != 0
        wall = time.perf_counter() - t0
        st = srv.stats()
    return {"rate_per_s": rate, "requests": n_req, "items": items, "failed": bad,
            "p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3, "max_ms": st["max_us"] / 1e3,
            "items_per_s": items / wall, "wall_s": wall,
            "pass": "H1-BF per request", "m": "log-uniform [100, 1e5]"}


# ------------------------------------------------------------------ oracle
KERNEL_OF = {1: "h1w_pack_kernel (first heuristic, one warp per membrane system; two launches side by "
                "side: systems above and up to small_m items, timed from fork to join)",
             2: "h2_pack_kernel_reg (second heuristic, one warp per sublist)"}
KERNEL_SOURCES = {1: ["paper_1602_08735_gb300/csrc/h1w_kernel.cuh", "paper_1602_08735_gb300/csrc/h1_kernel.cuh",
                      "paper_1602_08735_gb300/csrc/device_common.cuh"],
                  2: ["paper_1602_08735_gb300/csrc/h2_kernel.cuh", "paper_1602_08735_gb300/csrc/h2_params.cuh",
                      "paper_1602_08735_gb300/csrc/device_common.cuh"]}
ALU_LANES_PER_SM = 64      # 32-bit integer compare / min / max results per clock per SM


def sources_sha(paths):
    import hashlib
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def roofline_of(torch, dev, kernel_ms, fit_tests):
    """Roofline of the pass whose main kernel runs longest.

    The method's work is the fit test (Rule 4: every bin membrane alive when
    an item arrives tests it; for the second heuristic, in every permutation
    tried), one 32-bit integer compare each, so the bound is the integer ALU:
    peak = SMs x 64 compare results per clock x the SM clock.  achieved =
    fit tests per launch / the kernel's mean event-timed duration.  The
    kernels answer the same questions with far fewer operations (segment
    summaries; fixed register slots), which is why frac can pass 1.
    traffic = DRAM bytes per launch from the committed ncu capture of that
    kernel, or null when its sources changed since the capture."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    f_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sms * ALU_LANES_PER_SM * f_mhz * 1e6 / 1e12
    timed = {k: v for k, v in kernel_ms.items() if v}
    if not timed:
        return None
    name = max(timed, key=timed.get)
    h = dict((p[0], p[1]) for p in PASSES)[name]
    fits = fit_tests[name]["fit_tests"]
    achieved = fits / (timed[name] / 1e3) / 1e12
    traffic = None
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        ent = tr.get(name)
        if ent and ent.get("sources_sha") == sources_sha(KERNEL_SOURCES[h]):
            traffic = ent["dram_bytes_per_launch"]
    except Exception:
        pass
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": KERNEL_OF[h], "pass": name, "kernel_ms": timed[name],
            "fit_tests_per_launch": fits,
            "peak_source": f"derived: {sms} SMs x {ALU_LANES_PER_SM} int32 compare results/clk x {f_mhz:.0f} MHz",
            "kernel_ms_all": kernel_ms,
            "hbm_peak_gbs_measured": peaks.get("hbm_gbs")}


def cpu_baseline(batch, sample_n: int, seed: int = 123):
    """The oracle, as it stands, on a bounded random sample of the workload,
    one instance per host thread across all cores."""
    import oracle
    from paper_1602_08735_gb300 import instances as I
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(batch.N, size=min(sample_n, batch.N), replace=False))
    sub = batch.subset(idx)
    cores = oracle.host_cores()                   # the process's CPU affinity set
    t0 = time.perf_counter()
    for (_, h, c, s) in PASSES:
        oracle.pack_many(sub.w_all, sub.w_off, sub.B_all, sub.B_off, h, c, s, 0, 0, nthreads=cores)
    dt = time.perf_counter() - t0
    items = 4 * sub.total_items
    # one host thread, on the first quarter of the same sample
    one = sub.subset(np.arange(max(1, len(idx) // 4)))
    t1 = time.perf_counter()
    for (_, h, c, s) in PASSES:
        oracle.pack_many(one.w_all, one.w_off, one.B_all, one.B_off, h, c, s, 0, 0, nthreads=1)
    dt1 = time.perf_counter() - t1
    return {"value": items / dt, "unit": "items/s", "cores": cores, "kind": "oracle",
            "nproc": cores, "os_cpu_count": os.cpu_count(),
            "sample": f"{len(idx)} of {batch.N} instances ({sub.total_items} items) x 4 passes "
                      f"(H1 FF/BF/WF, H2 BF), {dt:.2f} s wall",
            "one_core": {"value": 4 * one.total_items / dt1, "unit": "items/s", "cores": 1,
                         "sample": f"{one.N} of those instances ({one.total_items} items) x 4 passes, "
                                   f"{dt1:.2f} s"}}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from paper_1602_08735_gb300 import instances as I
    batch = I.config3(seed=3, N=args.instances)
    sample_n = min(args.cpu_sample, batch.N)
    import oracle
    oracle.build()
    cores = oracle.host_cores()
    rng = np.random.default_rng(7)
    times, items = [], 0
    for k in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(batch.N, size=sample_n, replace=False))
        sub = batch.subset(idx)
        t0 = time.perf_counter()
        for (_, h, c, s) in PASSES:
            oracle.pack_many(sub.w_all, sub.w_off, sub.B_all, sub.B_off, h, c, s, 0, 0, nthreads=cores)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            items += 4 * sub.total_items
    value = items / sum(times)
    line = {
        "impl": "reference", "metric": "items packed/s", "value": value, "unit": "items/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances": batch.N, "sample_instances_per_step": sample_n,
                   "passes": [p[0] for p in PASSES]},
        "cpu_baseline": {"value": value, "unit": "items/s", "cores": cores, "kind": "oracle",
                         "nproc": cores, "os_cpu_count": os.cpu_count(),
                         "sample": f"{sample_n} random instances of {batch.N} per step x 4 passes"},
        "e2e": {"value": value, "unit": "items/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- ours
def rank_batch(native, I, instances, ws, rank):
    """This rank's part of the global batch (config-3 recipe, seed 3,
    instances * ws instances) under the library's longest-first split."""
    from paper_1602_08735_gb300 import shard
    whole = I.config3(seed=3, N=instances * ws)
    part, _ = shard.split(whole, ws, rank)
    return part


def run_ours(args, ws, rank, local):
    import torch

    from paper_1602_08735_gb300 import build as B
    from paper_1602_08735_gb300 import instances as I
    from paper_1602_08735_gb300 import native

    B.build()
    native.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    # one batch of instances x world instances, split over the ranks by the
    # library's LPT split (vsbpp_shard); at one GPU it is config 3 itself
    batch = rank_batch(native, I, args.instances, ws, rank)
    db = native.DeviceBatch.from_host(batch, device=dev)
    outs = [native.DeviceResult.empty(db.N, db.total_items, device=dev) for _ in PASSES]
    tuned = None
    if not args.no_autotune:
        # the library's autotuner picks group size, class split, staging and
        # slot sizing on this batch (BF pass); the plans below use its choice
        t0 = time.perf_counter()
        cfg, best_ms = native.autotune(db, outs[1], 1, 1, stream=stream)
        torch.cuda.synchronize()
        tuned = {"config": cfg, "bf_pass_ms": best_ms, "tuning_s": time.perf_counter() - t0}
    plans = [native.Plan(db.N, db.total_items, db.max_m, h, c, s) for (_, h, c, s) in PASSES]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    # The passes are independent.  Each first-heuristic pass is bound by its
    # largest systems' chains and leaves SMs idle in its tail; the second
    # heuristic needs registers and the integer pipe rather than shared
    # memory, and side by side it is the one that ends last.  So each pass
    # runs on a stream of its own, all four at once, the second heuristic
    # launched first on a high-priority stream (its blocks are placed first
    # as resources free up), then BF, FF, WF (measured: 7.57 ms per step,
    # against 7.95 ms with equal priorities in pass order, 8.39 ms with the
    # first-heuristic passes back to back beside the second heuristic and
    # 9.54 ms with all four back to back).
    pass_streams = [torch.cuda.Stream(device=dev, priority=-1 if p[1] == 2 else 0) for p in PASSES]
    launch_order = ([j for j, p in enumerate(PASSES) if p[1] == 2]
                    + [j for j, p in enumerate(PASSES) if p[0] == "H1-BF"]
                    + [j for j, p in enumerate(PASSES) if p[1] == 1 and p[0] != "H1-BF"])

    def step(evs=None):
        """One step: every pass on its own stream, forked from and joined on
        `stream`.  evs: optional (start, end, per-pass start/end events)."""
        fork = torch.cuda.Event()
        if evs:
            evs[0].record(stream)
        fork.record(stream)
        joins = []
        for j in launch_order:
            st = pass_streams[j]
            st.wait_event(fork)
            if evs:
                evs[2][j][0].record(st)
            plans[j].run(db, outs[j], st)
            if evs:
                evs[2][j][1].record(st)
            e = torch.cuda.Event()
            e.record(st)
            joins.append(e)
        for e in joins:
            stream.wait_event(e)
        if evs:
            evs[1].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    for out, (name, *_r) in zip(outs, PASSES):
        st = out.status[:db.N]
        assert int((st != 0).sum().item()) == 0, f"{name}: instances failed"

    # the method's fit tests in each pass (counters on, one untimed pass)
    native.counters_enable(True)
    native.counters_read(reset=True)
    fit_tests = {}
    for (name, h, c, s), out in zip(PASSES, outs):
        rc = native.pack_batch(db, out, h, c, s, stream=stream)
        assert rc == 0
        fit_tests[name] = native.counters_read(reset=True)
    native.counters_enable(False)

    # ---- timed region: device-resident inputs, graph replays, L2 flushed per step
    mk = lambda: torch.cuda.Event(enable_timing=True)
    ev = [(mk(), mk(), [(mk(), mk()) for _ in PASSES]) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            step(ev[k])
        torch.cuda.synchronize()
    barrier(ws)
    pass_ms = np.zeros(len(PASSES))
    step_ms_local = 0.0
    for k in range(args.steps):
        step_ms_local += ev[k][0].elapsed_time(ev[k][1])
        for j in range(len(PASSES)):
            pass_ms[j] += ev[k][2][j][0].elapsed_time(ev[k][2][j][1])
    pass_ms /= args.steps
    step_ms_local /= args.steps

    # the same passes back to back on one stream (context, untimed region)
    serial_ms = 0.0
    for k in range(args.steps):
        flush.zero_()
        a, b = mk(), mk()
        a.record(stream)
        for pl, out in zip(plans, outs):
            pl.run(db, out, stream)
        b.record(stream)
        torch.cuda.synchronize()
        serial_ms += a.elapsed_time(b)
    serial_ms /= args.steps
    step_ms = max_over_ranks(step_ms_local, ws)
    items_per_step_local = 4 * db.total_items
    items_per_step = sum_over_ranks(items_per_step_local, ws)
    value = items_per_step / (step_ms / 1e3)
    clocks = clk.summary()

    # ---- end to end through the C ABI with host buffers: vsbpp_pack_batch_host
    # takes pinned host CSR arrays, copies them to the device, packs and
    # copies every output back inside the call.  As on the device, the four
    # passes run at once: one host thread per pass, each call on a stream the
    # library lends it alone; host wall clock from the first call to the last
    # return.  The same calls one after another are reported as context.
    from concurrent.futures import ThreadPoolExecutor
    pin = lambda t: t.cpu().pin_memory()
    h_in = [pin(db.w_all), pin(db.w_off), pin(db.B_all), pin(db.B_off)]
    h_out = [native.HostResult(*(torch.empty_like(x, device="cpu").pin_memory() for x in
                                 (o.status, o.bin_of_item, o.bin_type, o.num_bins, o.total))) for o in outs]
    h2d = len(PASSES) * sum(int(x.numel() * x.element_size()) for x in h_in)
    d2h = sum(int(x.numel() * x.element_size()) for o in h_out
              for x in (o.status, o.bin_of_item, o.bin_type, o.num_bins, o.total))
    host_pool = ThreadPoolExecutor(len(PASSES))

    def host_pass(j):
        torch.cuda.set_device(local)                        # the library packs on the calling thread's device
        name, h, c, s_ = PASSES[j]
        return name, native.pack_batch_host(*h_in, h_out[j], h, c, s_, max_m=db.max_m)

    def host_step():
        for name, rc in host_pool.map(host_pass, range(len(PASSES))):
            assert rc == 0, (name, native.strerror(rc))

    e2e_steps = max(1, min(args.steps, 5))
    for _ in range(3):                                      # warm-up: library streams and buffers sized
        host_step()
    e2e_ms = 0.0
    for k in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        host_step()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms = max_over_ranks(e2e_ms / e2e_steps, ws)
    e2e_value = items_per_step / (e2e_ms / 1e3)
    e2e_serial_ms = 0.0
    for j in range(len(PASSES)):                            # warm-up: the lent stream's buffers sized for every pass
        assert host_pass(j)[1] == 0
    for k in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j in range(len(PASSES)):
            assert host_pass(j)[1] == 0
        e2e_serial_ms += (time.perf_counter() - t0) * 1e3
    e2e_serial_ms /= e2e_steps
    host_pool.shutdown()
    for o, d in zip(h_out, outs):                            # the host call's results = the device path's
        assert torch.equal(o.total[:db.N], d.total[:db.N].cpu())
        assert torch.equal(o.bin_of_item, d.bin_of_item.cpu())

    # ---- plain path: one launch per instance, one step
    plain = None
    if not args.no_plain:
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        flush.zero_()
        p0.record(stream)
        for (name, h, c, s), out in zip(PASSES, outs):
            rc = native.pack_plain(db, out, h, c, s, stream=stream)
            assert rc == 0
        p1.record(stream)
        torch.cuda.synchronize()
        plain_ms = max_over_ranks(p0.elapsed_time(p1), ws)
        plain_value = items_per_step / (plain_ms / 1e3)
        plain = {"items_per_s": plain_value, "ms_per_step": plain_ms, "speedup_batched_vs_plain": value / plain_value,
                 "launches_per_step": 2 * db.N * 0 + (3 * (db.N + 3) + 4 * db.N)}

    # ---- main packing kernel of each pass, timed with CUDA events on the
    # launching stream (library hook), L2 flushed before each call
    native.kernel_timing_enable(True)
    native.kernel_timing_read()
    kernel_ms = {}
    for (name, h, c, s), out in zip(PASSES, outs):
        for _ in range(args.steps):
            flush.zero_()
            rc = native.pack_batch(db, out, h, c, s, stream=stream)
            assert rc == 0
        t = native.kernel_timing_read()
        kernel_ms[name] = float(np.mean(t)) if t else None
    native.kernel_timing_enable(False)
    roofline = roofline_of(torch, dev, kernel_ms, fit_tests)
    if roofline:
        roofline["latency"] = latency_roof(native, batch, dev, stream, flush, roofline["pass"],
                                           roofline["kernel_ms"], clocks.get("sm_mhz") or 2070.0,
                                           max(args.steps, 3))

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(batch, args.cpu_sample)

    side = {}
    if not args.no_side:
        side["single_instance"] = single_instance_latency(native, I, dev, stream)
        side["config4"] = config4_pass(native, I, dev, stream, args.config4_instances, args.config4_m)
        side["serving"] = serving_sweep(native, I, args.serve_requests)
        side["variants"] = variants_side(native, db, dev, stream, flush)
        side["exhaustive"] = exhaustive_search(native, I, dev, stream)

    if rank == 0:
        line = {
            "metric": "items packed/s", "value": value, "unit": "items/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances": db.N, "items_per_step": int(items_per_step),
                       "passes": [p[0] for p in PASSES], "l2": "flushed before each timed step",
                       "graph": "each pass is a CUDA-graph replay of the batched persistent launch",
                       "parallelism": f"one batch of {args.instances * ws} instances split over {ws} GPU(s) "
                                      "by the library's longest-first split (vsbpp_shard), no collective",
                       "launch_config": tuned["config"] if tuned else native.get_config(),
                       "autotuned": tuned is not None},
            "autotune": tuned,
            "passes_ms": {p[0]: float(t) for p, t in zip(PASSES, pass_ms)},
            "schedule": "the four passes on four streams at once, each a CUDA-graph replay; H2 launched first on a high-priority stream, then H1 BF, FF, WF",
            "serial_ms_per_step": serial_ms,
            "e2e": {"value": e2e_value, "unit": "items/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "call": "vsbpp_pack_batch_host (pinned host CSR in, host outputs back), one call per pass, the four passes from four host threads at once",
                    "ms_per_step": e2e_ms, "serial_ms_per_step": e2e_serial_ms},
            "gpu_launches": LAUNCHES_PER_STEP * args.steps,
            "plain": plain,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "fit_tests": fit_tests,
            "side": side,
        }
        print(json.dumps(line), flush=True)
    for pl in plans:
        pl.close()


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.profile_once:
        import torch

        from paper_1602_08735_gb300 import build as B
        from paper_1602_08735_gb300 import instances as I
        from paper_1602_08735_gb300 import native
        B.build()
        native.load()
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        stream = torch.cuda.current_stream(dev)
        batch = I.config3(N=args.instances)
        db = native.DeviceBatch.from_host(batch, device=dev)
        out = native.DeviceResult.empty(db.N, db.total_items, device=dev)
        for (name, h, c, s) in PASSES:
            assert native.pack_batch(db, out, h, c, s, stream=stream) == 0, name
        torch.cuda.synchronize()
        print(json.dumps({"profile_once": [p[0] for p in PASSES], "instances": db.N,
                          "items": int(db.total_items)}), flush=True)
        return
    if args.only == "config4":
        import torch
        from paper_1602_08735_gb300 import build as B
        from paper_1602_08735_gb300 import instances as I
        from paper_1602_08735_gb300 import native
        B.build()
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        r = config4_pass(native, I, dev, torch.cuda.current_stream(dev), args.config4_instances,
                         args.config4_m)
        print(json.dumps({"config4": r}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
