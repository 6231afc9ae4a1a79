#!/usr/bin/env python3
"""Benchmark: validating UTF-8 <-> UTF-16LE transcoding on GB300.

Workload (one "step"): the four text profiles (latin, cyrillic, cjk, emoji),
each as a single 1 GiB buffer, transcoded in both directions (UTF-8 ->
UTF-16LE and UTF-16LE -> UTF-8): eight validating transcodes through the C
ABI, inputs resident in HBM before the timed region. Each input is larger
than the 129 MB L2, so no flush is needed between steps.

  value     whole-job input GB/s (1e9 bytes/s) over all ranks, device-timed
  e2e       the same metric through the host-buffer C-ABI calls (input copied
            host->device and output device->host inside the timed region);
            "link_bound": the e2e value the measured host<->device copy rates
            would allow with both directions busy all the time
  roofline  the dominant kernel's algorithmic bytes (input + output) per
            launch / its CUDA-event launch time, against the measured HBM
            copy peak
  cpu_baseline  the oracle (scalar C, one thread) on a bounded prefix sample;
            "parallel": the same sample cut at character boundaries and
            converted on all host cores at once

`--impl reference` times the oracle itself on the host cores (bounded sample
per step) and prints the same JSON line with "impl": "reference".

Multi-GPU (torchrun): every rank transcodes its own eight buffers (different
seeds); no collective on the data path; value = all ranks' input bytes / the
slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import textgen  # noqa: E402

METRIC = "input GB/s, validated UTF-8<->UTF-16LE transcoding (4 profiles x 2 directions x 1 GiB)"
WORKLOAD = ("single 1 GiB buffer per text profile (latin, cyrillic, cjk, emoji), both directions "
            "(UTF-8->UTF-16LE, UTF-16LE->UTF-8), validated")
DIRS = ("utf8_to_utf16le", "utf16le_to_utf8")
KERNEL = "transcode_kernel"      # the one persistent kernel (both directions)
KERNEL_SRC = {"transcode_kernel": ("transcode.cuh", "transcode_256x48.cu")}
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=1 << 30, help="bytes per input buffer")
    ap.add_argument("--profiles", default=",".join(textgen.BENCH_PROFILES))
    ap.add_argument("--e2e-steps", type=int, default=7)
    ap.add_argument("--cpu-sample", type=int, default=256 << 20,
                    help="bytes of each buffer the oracle baseline transcodes")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=["single", "batched", "serving", "latency", "split"],
                    default="single",
                    help="single: 4 profiles x 2 directions x one buffer each (default; the line "
                         "also carries reduced batched, serving and UTF-32 measurements); "
                         "batched: many strings in one persistent graph-captured launch; "
                         "serving: Poisson request arrivals through the serving loop; "
                         "latency: one call's latency and throughput against input size; "
                         "split: every buffer cut across the ranks at character boundaries, "
                         "one all-gather of a 32-byte record per rank")
    ap.add_argument("--strings", type=int, default=200_000, help="batched: number of strings")
    ap.add_argument("--rates", default="0.1,0.25,0.5,0.75,0.9,1.0,1.2",
                    help="serving: arrival rates as fractions of the plain kernel's GB/s")
    ap.add_argument("--serve-seconds", type=float, default=0.5,
                    help="serving: arrival window per rate (seconds)")
    ap.add_argument("--pool-gib", type=float, default=8.0, help="serving: device pool (GiB)")
    ap.add_argument("--slots", type=int, default=2, help="serving: batches in flight")
    ap.add_argument("--batch-total", type=int, default=0,
                    help="batched: scale the string lengths so that they add up to this many "
                         "bytes (0: unscaled, log-uniform 16 B - 1 MiB)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-strings", type=int, default=50_000,
                    help="single: strings of the batched measurement in the default line")
    ap.add_argument("--serve-rates", default="0.1,0.25,0.5,0.75,1.0",
                    help="single: load fractions of the serving measurement in the default line")
    ap.add_argument("--serve-window", type=float, default=0.25,
                    help="single: arrival window per load of the serving measurement (seconds)")
    ap.add_argument("--utf32-size", type=int, default=256 << 20,
                    help="single: UTF-8 bytes per profile for the UTF-32 measurement (0: skip)")
    ap.add_argument("--no-extras", action="store_true",
                    help="single: skip the batched, serving and UTF-32 measurements")
    return ap.parse_args()


def launcher_cmd(argv: list[str], gpus: int, port: int) -> list[str]:
    """The command that runs this benchmark as `gpus` ranks on this node (one
    process per GPU, rendezvous on 127.0.0.1) with the same arguments."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
            f"--nproc-per-node={gpus}", "--master-addr=127.0.0.1", f"--master-port={port}",
            os.path.abspath(__file__), *argv]


def free_port() -> int:
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy read+write)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (6.8 TB/s, earlier GB300 measurement)"


def source_hash(kernel: str) -> str:
    """Hash of the kernel's sources without their // comments and blank lines
    (a comment edit does not change the kernel the counters were taken on)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2212_05098_gb300", "csrc")
    for name in (*KERNEL_SRC[kernel], "common.cuh", "kernels.h"):
        with open(os.path.join(d, name), encoding="utf-8") as f:
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def traffic_record(kernel: str):
    """DRAM bytes per algorithmic byte, per "profile/direction", from the
    committed ncu summary, if it was taken on the kernel source as it is now
    (else {})."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p):
        return {}
    want = source_hash(kernel)
    out = {}
    with open(p) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel and parts[1] == want:
                out[parts[2]] = float(parts[3])
    return out


class ClockSampler:
    """nvidia-smi clocks / throttle reasons every 200 ms (timestamped)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        if not self.samples:
            return None
        inside = [s for t, s in self.samples if t0 - 0.25 <= t <= t1 + 0.25]
        if not inside:
            mid = (t0 + t1) / 2
            inside = [min(self.samples, key=lambda x: abs(x[0] - mid))[1]]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(s[1]) for s in inside if num(s[1]) is not None]
        mx = [num(s[2]) for s in inside if num(s[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in inside for k in range(4)
                          if s[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside)}


def job_rate(local_bytes: float, local_ms: float, world: int, device) -> tuple[float, float]:
    """Whole-job throughput: every rank's bytes over the slowest rank's time.
    Returns (GB/s, slowest time in ms). With world > 1 it all-reduces (SUM of
    bytes, MAX of times) over the default process group."""
    import torch
    b = torch.tensor([float(local_bytes)], dtype=torch.float64, device=device)
    m = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(b, op=dist.ReduceOp.SUM)
        dist.all_reduce(m, op=dist.ReduceOp.MAX)
    ms = float(m.item())
    return float(b.item()) / (ms / 1e3) / 1e9, ms


def gen_inputs(profiles, size, rank, pool):
    cases = []
    for prof in profiles:
        seed = textgen.PROFILE_SEED[prof] + 1000 * rank
        for d in DIRS:
            enc = textgen.UTF8 if d == "utf8_to_utf16le" else textgen.UTF16
            t = textgen.generate(prof, size, enc, seed=seed, executor=pool,
                                 keep_cps=False, keep_lens=False)
            cases.append({"profile": prof, "dir": d, "data": t.data})
    return cases


def host_link_gbs(torch, nbytes):
    """Copy-engine rates between pinned host memory and HBM (GB/s): each
    direction alone, and both at once on two streams."""
    h_a = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h_b = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d_a = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d_b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def run(up, down, reps=3):
        def once():
            if up:
                with torch.cuda.stream(s1):
                    d_a.copy_(h_a, non_blocking=True)
            if down:
                with torch.cuda.stream(s2):
                    h_b.copy_(d_b, non_blocking=True)
        once()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            once()
        torch.cuda.synchronize()
        return nbytes * reps / (time.perf_counter() - t0) / 1e9

    out = {"h2d": run(True, False), "d2h": run(False, True)}
    both = run(True, True)
    out["h2d_concurrent"] = out["d2h_concurrent"] = both
    out["bytes"] = nbytes
    return out


def cpu_baseline(cases, sample_bytes):
    import oracle
    total = 0
    t0 = time.perf_counter()
    for c in cases:
        d = c["data"][: sample_bytes - (sample_bytes % 2)]
        if c["dir"] == "utf8_to_utf16le":
            oracle.utf8_to_utf16le(d)
        else:
            oracle.utf16le_to_utf8(d)
        total += d.size
    dt = time.perf_counter() - t0
    return total, dt


def _char_cuts(data, parts: int, utf16: bool):
    """Byte offsets cutting `data` into `parts` pieces at character boundaries
    (UTF-8: never before a continuation byte; UTF-16LE: never between the
    halves of a surrogate pair)."""
    n = int(data.size)
    unit = 2 if utf16 else 1
    cuts = [0]
    for k in range(1, parts):
        c = max((n * k // parts) // unit * unit, cuts[-1])
        if utf16:
            while c + 1 < n and 0xDC <= int(data[c + 1]) <= 0xDF:
                c += 2
        else:
            while c < n and (int(data[c]) & 0xC0) == 0x80:
                c += 1
        cuts.append(min(c, n))
    cuts.append(n)
    return cuts


def cpu_baseline_parallel(cases, sample_bytes, threads):
    """The same sample, every buffer cut at character boundaries into
    `threads` parts that the oracle converts on `threads` host threads at
    once (its C calls release the GIL). Returns (bytes, seconds)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    jobs = []
    total = 0
    for c in cases:
        d = c["data"][: sample_bytes - (sample_bytes % 2)]
        u16 = c["dir"] != "utf8_to_utf16le"
        cuts = _char_cuts(d, threads, u16)
        f = oracle.utf16le_to_utf8 if u16 else oracle.utf8_to_utf16le
        jobs += [(f, d[a:b]) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
        total += d.size
    with ThreadPoolExecutor(threads) as ex:
        t0 = time.perf_counter()
        list(ex.map(lambda j: j[0](j[1]), jobs))
        dt = time.perf_counter() - t0
    return total, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    profiles = args.profiles.split(",")
    sample = max(2, min(args.size, 16 << 20))
    sample -= sample % 2
    cases = gen_inputs(profiles, sample, 0, None)
    oracle.utf8_to_utf16le(cases[0]["data"][:16])      # build / load
    for _ in range(args.warmup):
        cpu_baseline(cases, sample)
    times = []
    total = 0
    for _ in range(args.steps):
        b, dt = cpu_baseline(cases, sample)
        times.append(dt)
        total += b
    elapsed = sum(times)
    value = total / elapsed / 1e9
    desc = (f"oracle (scalar C, 1 thread) on the first {sample >> 20} MiB of each of the "
            f"{len(cases)} buffers per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8+u16", "data": "synthetic",
        "config": {"workload": WORKLOAD, "bytes_per_buffer": args.size,
                   "sample_bytes_per_buffer": sample, "buffers": len(cases)},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # started as `bench.py --gpus N`: start the N ranks ourselves
        sys.exit(subprocess.call(launcher_cmd(sys.argv[1:], args.gpus, free_port())))
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batched":
        run_batched(args, rank, world, local)
        return
    if args.workload == "serving":
        run_serving(args, rank, world, local)
        return
    if args.workload == "latency":
        run_latency(args, rank, world, local)
        return
    if args.workload == "split":
        run_split(args, rank, world, local)
        return
    # process pool for the generator: started before the first CUDA call
    pool = textgen.process_pool() if args.size >= (64 << 20) else None

    import torch
    import torch.distributed as dist

    import paper_2212_05098_gb300 as gbu

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    profiles = args.profiles.split(",")
    cases = gen_inputs(profiles, args.size, rank, pool)
    if pool is not None:
        pool.shutdown()

    gbu.load()
    ctx = gbu.Context(local)
    ctx.reserve(args.size)
    stream = torch.cuda.Stream()
    results = torch.zeros((len(cases), 4), dtype=torch.int64, device="cuda")
    for i, c in enumerate(cases):
        c["d_in"] = torch.from_numpy(c["data"]).cuda()
        n = c["data"].size
        if c["dir"] == "utf8_to_utf16le":
            c["n"], c["cap"] = n, n
            c["d_out"] = torch.empty(2 * n, dtype=torch.uint8, device="cuda")
        else:
            c["n"], c["cap"] = n // 2, 3 * (n // 2)
            c["d_out"] = torch.empty(c["cap"], dtype=torch.uint8, device="cuda")
        c["res"] = results[i].data_ptr()
    torch.cuda.synchronize()
    sh = stream.cuda_stream

    def launch(c):
        if c["dir"] == "utf8_to_utf16le":
            st = gbu.gbu_utf8_to_utf16le_async(ctx.handle, c["d_in"].data_ptr(), c["n"],
                                               c["d_out"].data_ptr(), c["cap"], c["res"], sh)
        else:
            st = gbu.gbu_utf16le_to_utf8_async(ctx.handle, c["d_in"].data_ptr(), c["n"],
                                               c["d_out"].data_ptr(), c["cap"], c["res"], sh)
        if st != gbu.GBU_OK:
            raise RuntimeError(f"enqueue failed: {gbu.status_name(st)}")

    sampler = ClockSampler(local)
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            for c in cases:
                launch(c)
    stream.synchronize()
    res = results.cpu().numpy()
    for i, c in enumerate(cases):
        st = int(res[i, 0] & 0xFFFFFFFF)
        if st != gbu.GBU_OK:
            raise RuntimeError(f"{c['profile']} {c['dir']}: {gbu.status_name(st)}")
        c["out_len"] = int(res[i, 2])
        ub = 2 if c["dir"] == "utf8_to_utf16le" else 1
        c["alg_bytes"] = c["data"].size + ub * c["out_len"]

    # ---- timed region: K steps, per-launch events on the launching stream ----
    K = args.steps
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in cases] for _ in range(K)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = gbu.gbu_kernel_launch_count()
    t_wall0 = time.time()
    with torch.cuda.stream(stream):
        start.record(stream)
        for k in range(K):
            for i, c in enumerate(cases):
                ev[k][i][0].record(stream)
                launch(c)
                ev[k][i][1].record(stream)
        end.record(stream)
    stream.synchronize()
    t_wall1 = time.time()
    launches = gbu.gbu_kernel_launch_count() - n0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    bytes_step = sum(c["data"].size for c in cases)
    value, ms_total = job_rate(bytes_step * K, start.elapsed_time(end), world, "cuda")
    sampler.stop()
    clocks = sampler.summary(t_wall0, t_wall1)

    # the kernel's roofline over all its launches, with a per-direction split
    peak, peak_src = measured_peak()
    per_dir = {}
    for i, c in enumerate(cases):
        d = per_dir.setdefault(c["dir"], {"ms": 0.0, "bytes": 0, "in_bytes": 0, "launches": 0})
        for k in range(K):
            d["ms"] += ev[k][i][0].elapsed_time(ev[k][i][1])
            d["bytes"] += c["alg_bytes"]
            d["in_bytes"] += c["data"].size
            d["launches"] += 1
    tot_ms = sum(x["ms"] for x in per_dir.values())
    tot_bytes = sum(x["bytes"] for x in per_dir.values())
    tot_in = sum(x["in_bytes"] for x in per_dir.values())
    n_launch = sum(x["launches"] for x in per_dir.values())
    ratios = traffic_record(KERNEL)
    traffic = None
    if all(f"{c['profile']}/{c['dir']}" in ratios for c in cases):
        traffic = sum(ratios[f"{c['profile']}/{c['dir']}"] * c["alg_bytes"] for c in cases) / len(cases)
    achieved = tot_bytes / (tot_ms / 1e3) / 1e9
    directions = {dname: {"achieved_gbs": d["bytes"] / (d["ms"] / 1e3) / 1e9,
                          "frac": d["bytes"] / (d["ms"] / 1e3) / 1e9 / peak,
                          "avg_launch_ms": d["ms"] / d["launches"],
                          "alg_bytes_per_launch": d["bytes"] / d["launches"],
                          "share_of_time": d["ms"] / tot_ms}
                  for dname, d in per_dir.items()}
    roofline = {"kernel": KERNEL, "bound": "hbm", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                "peak_source": peak_src,
                "algorithmic_bytes_per_launch": tot_bytes / n_launch,
                "avg_launch_ms": tot_ms / n_launch}
    per_case = {f"{c['profile']}/{c['dir']}":
                c["data"].size / (statistics.median(ev[k][i][0].elapsed_time(ev[k][i][1])
                                                    for k in range(K)) / 1e3) / 1e9
                for i, c in enumerate(cases)}

    # ---- end to end through the host-buffer C-ABI calls --------------------
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        h2d = sum(c["data"].size for c in cases)
        d2h = sum((2 if c["dir"] == "utf8_to_utf16le" else 1) * c["out_len"] for c in cases)
        outs = {}
        for c in cases:
            ub = 2 if c["dir"] == "utf8_to_utf16le" else 1
            key = c["dir"]
            need = c["cap"] * ub
            if key not in outs or outs[key].numel() < need:
                outs[key] = torch.empty(need, dtype=torch.uint8, pin_memory=True)
            c["h_in"] = torch.from_numpy(c["data"]).pin_memory()
        for _ in range(2):   # untimed passes (scratch sizing, first use of the pinned buffers)
            for c in cases:
                _host_call(gbu, ctx, c, outs, sh)
        if world > 1:
            dist.barrier()
        step_s = []
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for c in cases:
                r = _host_call(gbu, ctx, c, outs, sh)
                if r.status != gbu.GBU_OK or r.out_len != c["out_len"]:
                    raise RuntimeError(f"host call mismatch {r}")
            torch.cuda.synchronize()
            step_s.append(time.perf_counter() - t0)
        # the median step (the host link is shared with other jobs on the node)
        dtt = torch.tensor([statistics.median(step_s)], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(dtt, op=dist.ReduceOp.MAX)
        dt = float(dtt.item())
        e2e = {"value": world * h2d / dt / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "steps": args.e2e_steps, "step_ms": [round(1e3 * x, 2) for x in step_s],
               "api": "gbu_*_host (pinned host buffers)"}
        link = host_link_gbs(torch, 1 << 30)
        # the best e2e value the host link allows: both directions at once, at
        # the concurrent copy rates, and no time for anything else
        t_link = max(h2d / (link["h2d_concurrent"] * 1e9), d2h / (link["d2h_concurrent"] * 1e9))
        e2e["link"] = link
        e2e["link_bound"] = world * h2d / t_link / 1e9
        e2e["frac_of_link_bound"] = e2e["value"] / e2e["link_bound"]

    # validation only (no output, no look-back), same buffers: one untimed
    # pass, then 3 timed passes with an event between calls (per-buffer rates)
    vres = torch.zeros(4, dtype=torch.int64, device="cuda")

    def validate_call(c):
        if c["dir"] == "utf8_to_utf16le":
            gbu.gbu_validate_utf8_async(ctx.handle, c["d_in"].data_ptr(), c["n"],
                                        vres.data_ptr(), sh)
        else:
            gbu.gbu_validate_utf16le_async(ctx.handle, c["d_in"].data_ptr(), c["n"],
                                           vres.data_ptr(), sh)

    with torch.cuda.stream(stream):
        for c in cases:
            validate_call(c)
        vev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * len(cases) + 1)]
        vev[0].record(stream)
        for p in range(3):
            for i, c in enumerate(cases):
                validate_call(c)
                vev[1 + p * len(cases) + i].record(stream)
    stream.synchronize()
    validate_gbs = 3 * bytes_step / (vev[0].elapsed_time(vev[-1]) / 1e3) / 1e9
    validate_per_case = {}
    for i, c in enumerate(cases):
        ms = sum(vev[p * len(cases) + i].elapsed_time(vev[1 + p * len(cases) + i])
                 for p in range(3))
        enc = "utf8" if c["dir"] == "utf8_to_utf16le" else "utf16le"
        validate_per_case[f"{c['profile']}/{enc}"] = 3 * c["data"].size / (ms / 1e3) / 1e9

    # ---- the batched launch, the serving loop and UTF-32 on the same device --
    extras = {}
    if not args.no_extras and world == 1:
        plain_gbs = value / world
        if args.batch_strings > 0:
            b = batched_section(gbu, torch, local, cases, [c["d_in"] for c in cases],
                                args.batch_strings, 4, stream, plain_gbs, 20, 3, 1)
            b.pop("_lay"), b.pop("_is16")
            b["workload"] = (f"{b['strings']} strings (reduced from 200000), lengths log-uniform "
                             "16 B-1 MiB, profiles uniform, direction 50/50, windows of the "
                             "buffers above; one graph-captured launch per step, 20 steps")
            extras["batched"] = b
        rates = [float(x) for x in args.serve_rates.split(",") if x]
        if rates:
            sv = serving_section(gbu, torch, local, cases, [c["d_in"] for c in cases], rates,
                                 args.serve_window, plain_gbs, 8 << 30, 2, 5, min_requests=1000)
            sv["workload"] = (f"Poisson arrivals over {args.serve_window} s per load, sizes "
                              "log-uniform 64 B-16 MiB, 1 % injected errors, windows of the "
                              "buffers above; loads are fractions of this run's value")
            extras["serving"] = sv
        if args.utf32_size > 0:
            extras["utf32"] = utf32_section(gbu, torch, ctx, args.utf32_size, stream,
                                            roofline["frac"])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        b, dt = cpu_baseline(cases, args.cpu_sample)
        cpu = {"value": b / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle (scalar C, 1 thread) on the first "
                         f"{args.cpu_sample >> 20} MiB of each of the {len(cases)} buffers "
                         f"({b / 1e9:.2f} GB total, {dt:.1f} s)"}
        nthreads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        if nthreads and nthreads > 1:
            bp, dtp = cpu_baseline_parallel(cases, args.cpu_sample, nthreads)
            cpu["parallel"] = {"value": bp / dtp / 1e9, "unit": "GB/s", "cores": nthreads,
                               "sample": "the same sample, each buffer cut at character "
                                         f"boundaries into {nthreads} parts converted at once"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": K, "warmup": max(3, args.warmup), "ms_per_step": ms_total / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8+u16", "data": "synthetic (seeded i.i.d. code points per profile)",
            "config": {"workload": WORKLOAD, "bytes_per_buffer": args.size,
                       "buffers": len(cases), "profiles": profiles,
                       "parallelism": f"independent buffers per rank x {world}",
                       "l2": f"inputs {args.size >> 20} MiB each"
                             + (", larger than the 129 MB L2; no flush" if args.size > (129 << 20)
                                else ", NOT larger than L2 (profiling case only)")},
            "roofline": roofline,
            "directions": directions,
            "per_buffer_input_gbs": per_case,
            "per_buffer_output_bytes": {f"{c['profile']}/{c['dir']}":
                                        c["alg_bytes"] - c["data"].size for c in cases},
            "validate_only_input_gbs": validate_gbs,
            "validate_only_per_buffer_gbs": validate_per_case,
            **extras,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def utf32_section(gbu, torch, ctx, size, stream, utf16_frac):
    """UTF-8 <-> UTF-32LE on the two profiles that carry multi-byte
    characters (cjk, emoji), `size` UTF-8 bytes each: per direction the
    median of 5 calls (CUDA events on the call's stream), the roofline
    fraction (input + output bytes) and its ratio to the UTF-16 kernel's
    fraction `utf16_frac` measured in the same run."""
    peak, _ = measured_peak()
    sh = stream.cuda_stream
    out = {}
    for prof in ("cjk", "emoji"):
        t = textgen.generate(prof, size, textgen.UTF8, seed=textgen.PROFILE_SEED[prof],
                             keep_lens=False)
        u8 = t.data
        u32 = np.ascontiguousarray(t.cps, dtype="<u4")
        d8 = torch.from_numpy(u8).cuda()
        d32 = torch.from_numpy(u32.view(np.uint8)).cuda()
        o32 = torch.empty(4 * u8.size, dtype=torch.uint8, device="cuda")
        o8 = torch.empty(4 * u32.size, dtype=torch.uint8, device="cuda")
        calls = {
            "utf8_to_utf32le": (lambda: gbu.gbu_utf8_to_utf32le(
                ctx.handle, d8.data_ptr(), u8.size, o32.data_ptr(), u8.size, sh), u8.size, 4),
            "utf32le_to_utf8": (lambda: gbu.gbu_utf32le_to_utf8(
                ctx.handle, d32.data_ptr(), u32.size, o8.data_ptr(), 4 * u32.size, sh),
                4 * u32.size, 1),
        }
        for name, (call, in_bytes, ub) in calls.items():
            r = call()
            want = u32.size if name == "utf8_to_utf32le" else u8.size
            if r.status != gbu.GBU_OK or r.out_len != want:
                raise RuntimeError(f"utf32 {prof} {name}: {r}")
            ms = []
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                call()
                e1.record(stream)
                stream.synchronize()
                ms.append(e0.elapsed_time(e1))
            m = statistics.median(ms)
            alg = in_bytes + ub * r.out_len
            frac = alg / (m / 1e3) / 1e9 / peak
            out[f"{prof}/{name}"] = {"input_gbs": in_bytes / (m / 1e3) / 1e9, "ms": m,
                                     "alg_bytes": alg, "frac": frac,
                                     "frac_over_utf16_frac": frac / utf16_frac}
        del d8, d32, o32, o8
    out["size_utf8_bytes"] = size
    out["frac_over_utf16_frac_mean"] = float(np.mean(
        [v["frac_over_utf16_frac"] for k, v in out.items() if isinstance(v, dict)]))
    return out


SPLIT_METRIC = ("input GB/s, validated UTF-8<->UTF-16LE transcoding, every 1 GiB buffer cut "
                "across the ranks at character boundaries (4 profiles x 2 directions)")


def run_split(args, rank, world, local):
    """Split workload: every rank holds the same 8 buffers (4 profiles x 2
    directions) and converts its part of each, cut at character boundaries;
    one step = the 8 part launches plus one all-gather (NCCL) of the 8
    result records (32 bytes each) per rank, from which every rank knows its
    output offsets and the buffers' results. Total work is fixed as ranks are
    added (strong scaling)."""
    pool = textgen.process_pool() if args.size >= (64 << 20) else None
    import torch
    import torch.distributed as dist

    import paper_2212_05098_gb300 as gbu
    from paper_2212_05098_gb300 import shard

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    profiles = args.profiles.split(",")
    cases = gen_inputs(profiles, args.size, 0, pool)    # identical buffers on every rank
    if pool is not None:
        pool.shutdown()
    gbu.load()
    ctx = gbu.Context(local)
    ctx.reserve(args.size)
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    results = torch.zeros((len(cases), 4), dtype=torch.int64, device="cuda")
    for i, c in enumerate(cases):
        u16 = c["dir"] == "utf16le_to_utf8"
        cuts = shard.split_points(c["data"], world, u16)
        part = c["data"][cuts[rank]:cuts[rank + 1]]
        c["part_units"] = part.size // 2 if u16 else part.size
        c["d_in"] = torch.from_numpy(np.array(part, copy=True)).cuda()
        c["cap"] = 3 * c["part_units"] if u16 else c["part_units"]
        c["d_out"] = torch.empty(max(1, c["cap"] * (1 if u16 else 2)), dtype=torch.uint8,
                                 device="cuda")
        c["res"] = results[i].data_ptr()
    gathered = torch.zeros((world, len(cases), 4), dtype=torch.int64, device="cuda")

    def step():
        for c in cases:
            f = (gbu.gbu_utf16le_to_utf8_async if c["dir"] == "utf16le_to_utf8"
                 else gbu.gbu_utf8_to_utf16le_async)
            st = f(ctx.handle, c["d_in"].data_ptr() if c["part_units"] else 0, c["part_units"],
                   c["d_out"].data_ptr(), c["cap"], c["res"], sh)
            if st != gbu.GBU_OK:
                raise RuntimeError(f"enqueue failed: {gbu.status_name(st)}")
        if world > 1:
            with torch.cuda.stream(stream):
                dist.all_gather_into_tensor(gathered, results)

    for _ in range(max(3, args.warmup)):
        step()
    stream.synchronize()
    # combine the ranks' records and check them against one whole-buffer call
    rows = gathered.cpu().numpy() if world > 1 else results.cpu().numpy()[None]
    units = [[c["part_units"] for c in cases]]
    if world > 1:
        u = torch.tensor(units[0], dtype=torch.int64, device="cuda")
        ug = torch.zeros((world, len(cases)), dtype=torch.int64, device="cuda")
        dist.all_gather_into_tensor(ug, u)
        units = ug.cpu().tolist()
    whole_ctx = gbu.Context(local)
    for i, c in enumerate(cases):
        parts = [shard.PartResult(int(rows[r, i, 0]) & 0xFFFFFFFF, int(rows[r, i, 1]),
                                  int(rows[r, i, 2])) for r in range(world)]
        _, total = shard.combine(parts, [units[r][i] for r in range(world)])
        if rank == 0:
            d = torch.from_numpy(c["data"]).cuda()
            o = torch.empty(2 * c["data"].size, dtype=torch.uint8, device="cuda")
            if c["dir"] == "utf8_to_utf16le":
                w = gbu.gbu_utf8_to_utf16le(whole_ctx.handle, d.data_ptr(), d.numel(),
                                            o.data_ptr(), d.numel(), sh)
            else:
                w = gbu.gbu_utf16le_to_utf8(whole_ctx.handle, d.data_ptr(), d.numel() // 2,
                                            o.data_ptr(), 3 * (d.numel() // 2), sh)
            if (w.status, w.in_offset, w.out_len) != (total.status, total.in_offset,
                                                      total.out_len):
                raise RuntimeError(f"split result {total} != whole-buffer result {w}")
            del d, o
    whole_ctx.close()
    torch.cuda.empty_cache()

    sampler = ClockSampler(local)
    K = args.steps
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = gbu.gbu_kernel_launch_count()
    t_wall0 = time.time()
    start.record(stream)
    for _ in range(K):
        step()
    end.record(stream)
    stream.synchronize()
    t_wall1 = time.time()
    launches = gbu.gbu_kernel_launch_count() - n0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.stop()
    clocks = sampler.summary(t_wall0, t_wall1)
    whole = sum(c["data"].size for c in cases) * K
    # every rank converts 1/world of each buffer: the job's bytes are the
    # whole buffers once, over the slowest rank's time
    _, ms = job_rate(0.0, start.elapsed_time(end), world, "cuda")
    value = whole / (ms / 1e3) / 1e9
    if rank == 0:
        line = {
            "metric": SPLIT_METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": K, "warmup": max(3, args.warmup), "ms_per_step": ms / K,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "u8+u16", "data": "synthetic (seeded i.i.d. code points per profile)",
            "config": {"workload": f"8 buffers of {args.size} B, each cut into {world} parts "
                                   "at character boundaries",
                       "bytes_per_buffer": args.size, "buffers": len(cases),
                       "parallelism": f"split x {world}, one all-gather of 8 x 32 B per rank "
                                      "per step" if world > 1 else "one rank, no exchange",
                       "l2": "inputs larger than the 129 MB L2; no flush"},
            "cpu_baseline": None, "e2e": None, "clocks": clocks,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


BATCH_METRIC = ("input GB/s, validated UTF-8<->UTF-16LE transcoding of many strings in one "
                "persistent graph-captured launch")


def batched_section(gbu, torch, local, cases, d_corp, n_strings, seed, stream, plain_gbs,
                    steps, warmup, world, batch_total=0, per_string=True):
    """The batched form (one persistent graph-captured launch over many
    strings) on windows of the resident corpora `d_corp` (one per case):
    `n_strings` strings, lengths log-uniform over 16 B - 1 MiB (scaled to
    `batch_total` bytes if given), profile uniform, direction 50/50. Plans,
    autotunes and times `steps` graph launches; `plain_gbs` is the plain
    single-buffer kernel's input GB/s in the same run."""
    from textgen import batch as tbatch
    corpora = [(c["profile"], textgen.UTF8 if c["dir"] == "utf8_to_utf16le" else textgen.UTF16,
                c["data"]) for c in cases]
    lay = tbatch.layout(corpora, n_strings, 16, 1 << 20, seed=seed)
    if batch_total:
        lay = tbatch.layout(corpora, n_strings, 16, 1 << 20, seed=seed,
                            scale=batch_total / lay.total_bytes)
    n_str = lay.nbytes.size
    is16 = np.array([corpora[k][1] == textgen.UTF16 for k in lay.corpus])
    cap_bytes = np.where(is16, 3 * (lay.nbytes // 2), 2 * lay.nbytes)
    out_off = np.zeros(n_str + 1, dtype=np.int64)
    np.cumsum((cap_bytes + 15) // 16 * 16, out=out_off[1:])
    d_out = torch.empty(int(out_off[-1]) + 16, dtype=torch.uint8, device="cuda")
    d_res = torch.zeros(n_str * 24, dtype=torch.uint8, device="cuda")
    base_out = d_out.data_ptr()
    items = []
    for i in range(n_str):
        k = int(lay.corpus[i])
        inp = d_corp[k].data_ptr() + int(lay.start[i])
        if is16[i]:
            n = int(lay.nbytes[i]) // 2
            items.append((inp if n else 0, n, base_out + int(out_off[i]), 3 * n,
                          gbu.GBU_OP_UTF16LE_TO_UTF8))
        else:
            n = int(lay.nbytes[i])
            items.append((inp if n else 0, n, base_out + int(out_off[i]), n,
                          gbu.GBU_OP_UTF8_TO_UTF16LE))
    ctx = gbu.Context(local)
    sh = stream.cuda_stream
    st = gbu.gbu_batch_plan(ctx.handle, items, d_res.data_ptr(), sh)
    if st != gbu.GBU_OK:
        raise RuntimeError(f"batch plan: {gbu.status_name(st)}")
    cache = os.path.join(ROOT, "paper_2212_05098_gb300", "_build", "tune_cache.txt")
    t_tune0 = time.perf_counter()
    st, tune = gbu.gbu_batch_autotune(ctx.handle, sh, cache)
    t_tune = time.perf_counter() - t_tune0
    if st != gbu.GBU_OK:
        raise RuntimeError(f"autotune: {gbu.status_name(st)}")
    for _ in range(max(3, warmup)):
        if gbu.gbu_batch_launch_graph(ctx.handle, sh) != gbu.GBU_OK:
            raise RuntimeError("batch launch failed")
    stream.synchronize()
    res = np.frombuffer(d_res.cpu().numpy().tobytes(),
                        dtype=[("status", "<i4"), ("r", "<u4"), ("off", "<u8"), ("len", "<u8")])
    if (res["status"] != 0).any():
        i = int(np.nonzero(res["status"] != 0)[0][0])
        raise RuntimeError(f"string {i}: {gbu.status_name(int(res['status'][i]))}")
    in_bytes = int(lay.nbytes.sum())
    out_bytes = int((res["len"] * np.where(is16, 1, 2)).sum())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    n0 = gbu.gbu_kernel_launch_count()
    for k in range(steps):
        ev[k][0].record(stream)
        gbu.gbu_batch_launch_graph(ctx.handle, sh)
        ev[k][1].record(stream)
    stream.synchronize()
    launches = gbu.gbu_kernel_launch_count() - n0
    ms_list = [x.elapsed_time(y) for x, y in ev]
    value, ms_total = job_rate(in_bytes * steps, sum(ms_list), world, "cuda")
    out = {"value": value, "unit": "GB/s", "strings": n_str, "input_bytes": in_bytes,
           "output_bytes": out_bytes, "ms_per_launch": ms_total / steps,
           "p50_launch_ms": float(np.percentile(ms_list, 50)),
           "p99_launch_ms": float(np.percentile(ms_list, 99)),
           "tune": {"look_width": tune.look_width, "ctas_per_sm": tune.ctas_per_sm,
                    "chunk_bytes": tune.chunk_bytes, "compute_threads": tune.compute_threads,
                    "autotune_s": round(t_tune, 3)},
           "plain_single_buffer_gbs": plain_gbs,
           "plain_over_batched": plain_gbs / (value / world),
           "frac": (in_bytes + out_bytes) / (ms_total / steps / 1e3) / 1e9 / measured_peak()[0],
           "launches": launches}
    if per_string:
        # the same strings, one plain-kernel launch each
        plain = gbu.Context(local)
        plain.reserve(1 << 20)
        res1 = torch.zeros(4, dtype=torch.int64, device="cuda")
        r1 = res1.data_ptr()

        def one_by_one():
            for (inp, n, outp, cap, op) in items:
                if op == gbu.GBU_OP_UTF8_TO_UTF16LE:
                    gbu.gbu_utf8_to_utf16le_async(plain.handle, inp, n, outp, cap, r1, sh)
                else:
                    gbu.gbu_utf16le_to_utf8_async(plain.handle, inp, n, outp, cap, r1, sh)

        one_by_one()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        one_by_one()
        e1.record(stream)
        stream.synchronize()
        out["per_string_launches"] = {"value": in_bytes / (e0.elapsed_time(e1) / 1e3) / 1e9,
                                      "unit": "GB/s", "ms": e0.elapsed_time(e1),
                                      "host_s": time.perf_counter() - t0, "launches": n_str}
        plain.close()
    out["_lay"], out["_is16"] = lay, is16
    ctx.close()
    return out


def serving_section(gbu, torch, local, cases, d_corp, rates, seconds, plain_gbs, pool_bytes,
                    slots, seed, min_requests=2000):
    """The serving loop at each load in `rates` (fractions of `plain_gbs`):
    Poisson arrivals of requests of log-uniform size over 64 B - 16 MiB
    (windows of the resident corpora, profile uniform, direction 50/50), 1 %
    with one injected error, replayed in real time through the library's
    server. Returns the per-load sustained GB/s and p50/p99 latency."""
    from textgen import batch as tbatch
    corpora = [(c["profile"], textgen.UTF8 if c["dir"] == "utf8_to_utf16le" else textgen.UTF16,
                c["data"]) for c in cases]
    srv = gbu.gbu_server_create(local, int(pool_bytes), slots, 4096)
    if not srv:
        raise RuntimeError("server creation failed")
    mean_bytes = ((16 << 20) - 64) / np.log((16 << 20) / 64)
    sweep = []
    n0 = gbu.gbu_kernel_launch_count()
    for ri, frac in enumerate(rates):
        rate = frac * plain_gbs * 1e9 / mean_bytes          # requests per second
        n_req = int(min(200_000, max(min_requests, rate * seconds)))
        tr = tbatch.serving_trace(corpora, n_req, rate, seed=seed + ri)
        lay = tr.layout
        keep, reqs = [], []
        for i in range(n_req):
            k = int(lay.corpus[i])
            enc = corpora[k][1]
            s0, nb = int(lay.start[i]), int(lay.nbytes[i])
            if tr.error_at[i] >= 0:
                host = tbatch.inject_error(corpora[k][2][s0:s0 + nb], int(tr.error_at[i]), enc)
                dev = torch.from_numpy(host).cuda()
                keep.append(dev)
                ptr = dev.data_ptr()
            else:
                ptr = d_corp[k].data_ptr() + s0
            u16 = enc == textgen.UTF16
            op = gbu.GBU_OP_UTF16LE_TO_UTF8 if u16 else gbu.GBU_OP_UTF8_TO_UTF16LE
            reqs.append((op, ptr if nb else 0, nb // 2 if u16 else nb, 0, 0, i))
        torch.cuda.synchronize()
        st, comp = gbu.gbu_server_replay(srv, reqs, list(tr.t_arrival), 300.0)
        if st != gbu.GBU_OK:
            raise RuntimeError(f"replay: {gbu.status_name(st)}")
        # latency from the scheduled arrival (the replay's clock starts at 0)
        lat = np.array([comp[i].t_done - tr.t_arrival[i] for i in range(n_req)])
        lag = np.array([comp[i].t_submit - tr.t_arrival[i] for i in range(n_req)])
        t_first = float(tr.t_arrival[0])
        t_last = max(comp[i].t_done for i in range(n_req))
        status = np.array([comp[i].result.status for i in range(n_req)])
        n_err = int((tr.error_at >= 0).sum())
        if (status != 0).sum() != n_err or (status[tr.error_at >= 0] == 0).any():
            raise RuntimeError("unexpected request status in the serving run")
        items = np.array([comp[i].batch_items for i in range(n_req)])
        sweep.append({
            "load_frac": frac, "rate_req_s": rate, "requests": n_req,
            "input_bytes": lay.total_bytes, "errors": n_err,
            "sustained_gbs": lay.total_bytes / (t_last - t_first) / 1e9,
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3),
            "mean_batch_items": float(items.mean()),
            "max_submit_lag_ms": float(lag.max() * 1e3),
            "batches": len({comp[i].batch for i in range(n_req)}),
        })
        del keep
    stats = gbu.gbu_server_stats(srv)
    gbu.gbu_server_destroy(srv)
    top = max(sweep, key=lambda x: x["sustained_gbs"])
    return {"sweep": sweep, "sustained_gbs_best": top["sustained_gbs"],
            "p50_ms_at_best": top["p50_ms"], "p99_ms_at_best": top["p99_ms"],
            "plain_single_buffer_gbs": plain_gbs,
            "plain_over_served": plain_gbs / top["sustained_gbs"],
            "pool_bytes": stats.pool_bytes, "pool_high_water": stats.pool_high_water,
            "slots": slots, "launches": gbu.gbu_kernel_launch_count() - n0}


def plain_rate(gbu, torch, local, cases, d_corp, stream, size):
    """Input GB/s of the plain single-buffer kernel on the corpora (3 passes)."""
    plain = gbu.Context(local)
    plain.reserve(size)
    scratch_out = torch.empty(2 * size + 64, dtype=torch.uint8, device="cuda")
    res1 = torch.zeros(4, dtype=torch.int64, device="cuda")
    sh = stream.cuda_stream

    def single():
        for c, d in zip(cases, d_corp):
            if c["dir"] == "utf8_to_utf16le":
                gbu.gbu_utf8_to_utf16le_async(plain.handle, d.data_ptr(), d.numel(),
                                              scratch_out.data_ptr(), d.numel(), res1.data_ptr(), sh)
            else:
                gbu.gbu_utf16le_to_utf8_async(plain.handle, d.data_ptr(), d.numel() // 2,
                                              scratch_out.data_ptr(), 3 * (d.numel() // 2),
                                              res1.data_ptr(), sh)

    single()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        single()
    e1.record(stream)
    stream.synchronize()
    plain.close()
    return 3 * sum(d.numel() for d in d_corp) / (e0.elapsed_time(e1) / 1e3) / 1e9


def run_batched(args, rank, world, local):
    """Batched workload: `--strings` independent strings, lengths log-uniform
    over 16 B - 1 MiB (optionally scaled to `--batch-total` bytes), profile
    uniform over the four, direction 50/50, each a window of that profile's
    corpus (`--size` bytes per profile and encoding) cut at character
    boundaries. One step = one launch of the autotuned batch (CUDA graph).
    Also timed in the same run: the same strings as one plain-kernel launch
    each, and the plain single-buffer kernel on the corpora themselves."""
    pool = textgen.process_pool()
    import torch
    import torch.distributed as dist

    import paper_2212_05098_gb300 as gbu

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    profiles = args.profiles.split(",")
    cases = gen_inputs(profiles, args.size, rank, pool)
    pool.shutdown()
    gbu.load()
    d_corp = [torch.from_numpy(c["data"]).cuda() for c in cases]
    stream = torch.cuda.Stream()
    single_gbs = plain_rate(gbu, torch, local, cases, d_corp, stream, args.size)
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    t_wall0 = time.time()
    b = batched_section(gbu, torch, local, cases, d_corp, args.strings, 4 + 1000 * rank, stream,
                        single_gbs, args.steps, args.warmup, world, args.batch_total)
    t_wall1 = time.time()
    sampler.stop()
    clocks = sampler.summary(t_wall0, t_wall1)
    peak, peak_src = measured_peak()
    ms_launch = b["ms_per_launch"]
    in_bytes, out_bytes = b["input_bytes"], b["output_bytes"]
    roofline = {"kernel": KERNEL, "bound": "hbm",
                "achieved": (in_bytes + out_bytes) / (ms_launch / 1e3) / 1e9, "peak": peak,
                "unit": "GB/s", "frac": (in_bytes + out_bytes) / (ms_launch / 1e3) / 1e9 / peak,
                "traffic": None, "peak_source": peak_src,
                "algorithmic_bytes_per_launch": in_bytes + out_bytes, "avg_launch_ms": ms_launch}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        lay, is16 = b["_lay"], b["_is16"]
        budget, done, t_c = args.cpu_sample, 0, 0.0
        for i in range(lay.nbytes.size):
            if done >= budget:
                break
            d = cases[int(lay.corpus[i])]["data"][int(lay.start[i]):int(lay.start[i] + lay.nbytes[i])]
            t0 = time.perf_counter()
            if is16[i]:
                oracle.utf16le_to_utf8(d)
            else:
                oracle.utf8_to_utf16le(d)
            t_c += time.perf_counter() - t0
            done += d.size
        cpu = {"value": done / t_c / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle (scalar C, 1 thread) on the first strings of the batch, "
                         f"{done / 1e9:.2f} GB, {t_c:.1f} s"}
    if rank == 0:
        line = {
            "metric": BATCH_METRIC, "value": b["value"], "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_launch,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8+u16", "data": "synthetic (windows of seeded per-profile corpora)",
            "config": {"workload": f"{b['strings']} strings, lengths log-uniform 16 B-1 MiB"
                                   + (f" scaled to {args.batch_total} B total" if args.batch_total
                                      else "")
                                   + ", profiles uniform over 4, direction 50/50",
                       "strings": b["strings"], "input_bytes": in_bytes,
                       "output_bytes": out_bytes,
                       "corpus_bytes_per_profile_and_encoding": args.size,
                       "tune": b["tune"],
                       "l2": "inputs read once per step from 8 corpora of "
                             f"{args.size >> 20} MiB; no flush"},
            "roofline": roofline,
            "per_string_launches": b.get("per_string_launches"),
            "plain_single_buffer_gbs": single_gbs,
            "plain_over_batched": b["plain_over_batched"],
            "cpu_baseline": cpu,
            "e2e": None,
            "clocks": clocks,
            "gpu_launches": b["launches"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


SERVE_METRIC = ("sustained input GB/s and p50/p99 request latency, validated UTF-8<->UTF-16LE "
                "transcoding through the serving loop (continuous batching)")


def run_serving(args, rank, world, local):
    """Serving workload: requests of log-uniform size over 64 B - 16 MiB
    (windows of the per-profile corpora, profile uniform, direction 50/50),
    1 % with one injected error, arriving as a Poisson process, replayed in
    real time through the library's serving loop (dispatcher thread,
    continuous batching, admission by bytes against a device pool). For each
    arrival rate (a fraction of the plain kernel's GB/s measured in the same
    run) it reports the sustained input GB/s and the p50/p99 latency from
    arrival to completion."""
    pool = textgen.process_pool()
    import torch
    import torch.distributed as dist

    import paper_2212_05098_gb300 as gbu

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    profiles = args.profiles.split(",")
    cases = gen_inputs(profiles, args.size, rank, pool)
    pool.shutdown()
    gbu.load()
    d_corp = [torch.from_numpy(c["data"]).cuda() for c in cases]
    stream = torch.cuda.Stream()
    plain_gbs = plain_rate(gbu, torch, local, cases, d_corp, stream, args.size)
    sampler = ClockSampler(local)
    t_wall0 = time.time()
    sv = serving_section(gbu, torch, local, cases, d_corp,
                         [float(x) for x in args.rates.split(",")], args.serve_seconds,
                         plain_gbs, args.pool_gib * (1 << 30), args.slots, 5 + 1000 * rank)
    t_wall1 = time.time()
    sampler.stop()
    clocks = sampler.summary(t_wall0, t_wall1)
    if rank == 0:
        line = {
            "metric": SERVE_METRIC, "value": sv["sustained_gbs_best"], "unit": "GB/s",
            "n_gpus": world, "steps": len(sv["sweep"]), "warmup": 0,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8+u16",
            "data": "synthetic (windows of seeded per-profile corpora, 1 % injected errors)",
            "config": {"workload": "Poisson arrivals, sizes log-uniform 64 B-16 MiB, profiles "
                                   "uniform over 4, direction 50/50, 1 % injected errors",
                       "pool_bytes": sv["pool_bytes"], "pool_high_water": sv["pool_high_water"],
                       "slots": args.slots, "max_batch_items": 4096,
                       "rates": "fractions of the plain kernel's GB/s in this run",
                       "latency": "scheduled arrival to completion observed by the dispatcher"},
            "p50_ms_at_best": sv["p50_ms_at_best"], "p99_ms_at_best": sv["p99_ms_at_best"],
            "sweep": sv["sweep"],
            "plain_single_buffer_gbs": plain_gbs,
            "plain_over_served": sv["plain_over_served"],
            "cpu_baseline": None, "e2e": None, "clocks": clocks,
            "gpu_launches": sv["launches"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


LATENCY_METRIC = "latency of one validated transcoding call against input size (mix profile)"
SPIN_CYCLES = 200_000   # ~0.1 ms of GPU clock ahead of every timed call


def run_latency(args, rank, world, local):
    """Small-string regime (the paper's throughput against input length,
    Sec. 8): for input sizes 16 B .. 256 MiB of the mix profile, the median
    device time of one asynchronous call (CUDA events around the call, with
    the stream held behind a short spin while the host enqueues them) and the
    wall time of one synchronous call (launch, wait, read the result), per
    direction; the device time also with the one-launch path off and on
    every kernel shape pinned."""
    import torch

    import paper_2212_05098_gb300 as gbu
    torch.cuda.set_device(local)
    top = min(args.size, 256 << 20)
    t8 = textgen.generate("mix", top, textgen.UTF8, seed=0, keep_cps=False, keep_lens=False).data
    t16 = textgen.generate("mix", top, textgen.UTF16, seed=0, keep_cps=False, keep_lens=False).data
    gbu.load()
    ctx = gbu.Context(local)
    ctx.reserve(top)
    # the same calls with the one-launch path off (every size on the persistent grid)
    ctx_p = gbu.Context(local)
    ctx_p.reserve(top)
    if gbu.gbu_set_tune(ctx_p.handle, 1, 0, 0) != gbu.GBU_OK:
        raise RuntimeError("set_tune failed")
    # and on every kernel shape pinned (the default context picks one by size)
    shapes = gbu.gbu_tune_shapes()
    ctx_s = {}
    for chunk, threads in shapes:
        cs = gbu.Context(local)
        cs.reserve(top)
        if gbu.gbu_set_tune(cs.handle, 1, 0, gbu.GBU_SMALL_MAX_CHUNKS, chunk, threads) != gbu.GBU_OK:
            raise RuntimeError("set_tune failed")
        ctx_s[f"{chunk}x{threads}"] = cs
    small_limit = gbu.GBU_SMALL_MAX_CHUNKS * max(c for c, _ in shapes)
    d8, d16 = torch.from_numpy(t8).cuda(), torch.from_numpy(t16).cuda()
    out = torch.empty(2 * top + 64, dtype=torch.uint8, device="cuda")
    res = torch.zeros(4, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    rows = []
    # floors of the same measurement: an empty launch (torch's spin kernel for
    # one cycle), and a call on an empty input (one 1-thread kernel that
    # writes the result with a system-scope fence)
    def floor_us(launch):
        ts = []
        for _ in range(20):
            with torch.cuda.stream(stream):
                torch.cuda._sleep(SPIN_CYCLES)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            launch()
            e1.record(stream)
            stream.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts) * 1e3

    def empty_kernel():
        with torch.cuda.stream(stream):
            torch.cuda._sleep(1)

    empty_launch_us = floor_us(empty_kernel)
    empty_call_us = floor_us(
        lambda: gbu.gbu_utf8_to_utf16le_async(ctx.handle, 0, 0, 0, 0, res.data_ptr(), sh))
    size = 16
    while size <= top:
        for direction, d in (("utf8_to_utf16le", d8), ("utf16le_to_utf8", d16)):
            n = size if direction == "utf8_to_utf16le" else size // 2

            def call_async(c=ctx):
                if direction == "utf8_to_utf16le":
                    gbu.gbu_utf8_to_utf16le_async(c.handle, d.data_ptr(), n, out.data_ptr(), n,
                                                  res.data_ptr(), sh)
                else:
                    gbu.gbu_utf16le_to_utf8_async(c.handle, d.data_ptr(), n, out.data_ptr(),
                                                  3 * n, res.data_ptr(), sh)

            def device_ms(c, reps):
                for _ in range(3):
                    call_async(c)
                stream.synchronize()
                dev = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    # the stream waits behind a ~0.1 ms spin while the host
                    # enqueues the events and the call, so that the events
                    # time the GPU's work and not the host's launch overhead
                    with torch.cuda.stream(stream):
                        torch.cuda._sleep(SPIN_CYCLES)
                    e0.record(stream)
                    call_async(c)
                    e1.record(stream)
                    stream.synchronize()
                    dev.append(e0.elapsed_time(e1))
                return statistics.median(dev)

            def call_sync():
                if direction == "utf8_to_utf16le":
                    return gbu.gbu_utf8_to_utf16le(ctx.handle, d.data_ptr(), n, out.data_ptr(), n, sh)
                return gbu.gbu_utf16le_to_utf8(ctx.handle, d.data_ptr(), n, out.data_ptr(), 3 * n, sh)

            reps = 20 if size <= (16 << 20) else 5
            shp = gbu.gbu_call_shape(ctx.handle, size)
            path = ("one-launch" if size <= shp.small_chunks * shp.chunk_bytes   # aligned input
                    else "persistent")
            dev_ms = device_ms(ctx, reps)
            pers_ms = device_ms(ctx_p, reps) if size <= small_limit else None
            by_shape = {k: device_ms(cs, reps) * 1e3 for k, cs in ctx_s.items()}
            wall = []
            for _ in range(reps):
                t0 = time.perf_counter()
                r = call_sync()
                wall.append(time.perf_counter() - t0)
            rows.append({"bytes": size, "direction": direction, "status": r.status,
                         "path": path,
                         "shape": f"{shp.chunk_bytes}x{shp.compute_threads}",
                         "device_us": dev_ms * 1e3, "sync_call_us": statistics.median(wall) * 1e6,
                         "device_gbs": size / (dev_ms / 1e3) / 1e9,
                         "device_us_persistent": None if pers_ms is None else pers_ms * 1e3,
                         "device_us_by_shape": by_shape,
                         "best_shape": min(by_shape, key=by_shape.get)})
        size *= 4
    big = [r for r in rows if r["bytes"] == rows[-1]["bytes"]]
    if rank == 0:
        line = {"metric": LATENCY_METRIC, "value": min(r["sync_call_us"] for r in rows),
                "unit": "us (smallest synchronous call)", "n_gpus": world, "steps": len(rows),
                "warmup": 3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "u8+u16", "data": "synthetic (mix profile, seed 0)",
                "config": {"workload": "one call per size, 16 B to 256 MiB by factors of 4",
                           "largest_gbs": {r["direction"]: r["device_gbs"] for r in big},
                           "one_launch_path": "inputs of at most 8 chunks of the call's shape"},
                "device_us_4KiB": {r["direction"]: r["device_us"] for r in rows
                                   if r["bytes"] == 4096},
                "device_us_empty_launch": empty_launch_us,
                "device_us_empty_call": empty_call_us,
                "best_shape_by_size": {f"{r['bytes']}/{r['direction']}": r["best_shape"]
                                       for r in rows},
                "sizes": rows, "gpu_launches": None}
        print(json.dumps(line), flush=True)
    ctx.close()
    ctx_p.close()
    for cs in ctx_s.values():
        cs.close()


def _host_call(gbu, ctx, c, outs, sh):
    out = outs[c["dir"]]
    if c["dir"] == "utf8_to_utf16le":
        return gbu.gbu_utf8_to_utf16le_host(ctx.handle, c["h_in"].data_ptr(), c["n"],
                                            out.data_ptr(), c["cap"], sh)
    return gbu.gbu_utf16le_to_utf8_host(ctx.handle, c["h_in"].data_ptr(), c["n"],
                                        out.data_ptr(), c["cap"], sh)


if __name__ == "__main__":
    main()
