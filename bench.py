#!/usr/bin/env python3
"""Benchmark: validating UTF-8 <-> UTF-16LE transcoding on GB300.

Workload (one "step"): the four text profiles (latin, cyrillic, cjk, emoji),
each as a single 1 GiB buffer, transcoded in both directions (UTF-8 ->
UTF-16LE and UTF-16LE -> UTF-8): eight validating transcodes through the C
ABI, inputs resident in HBM before the timed region. Each input is larger
than the 129 MB L2, so no flush is needed between steps.

  value     whole-job input GB/s (1e9 bytes/s) over all ranks, device-timed
  e2e       the same metric through the host-buffer C-ABI calls (input copied
            host->device and output device->host inside the timed region)
  roofline  the dominant kernel's algorithmic bytes (input + output) per
            launch / its CUDA-event launch time, against the measured HBM
            copy peak
  cpu_baseline  the oracle (scalar C, one thread) on a bounded prefix sample

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
KERNEL_SRC = {"transcode_kernel": "transcode.cu"}
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=1 << 30, help="bytes per input buffer")
    ap.add_argument("--profiles", default=",".join(textgen.BENCH_PROFILES))
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-sample", type=int, default=256 << 20,
                    help="bytes of each buffer the oracle baseline transcodes")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


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
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2212_05098_gb300", "csrc")
    for name in (KERNEL_SRC[kernel], "common.cuh", "kernels.h"):
        with open(os.path.join(d, name), "rb") as f:
            h.update(f.read())
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
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
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
    ms_total = start.elapsed_time(end)
    ms = torch.tensor([ms_total], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    ms_total = float(ms.item())
    sampler.stop()
    clocks = sampler.summary(t_wall0, t_wall1)

    bytes_step = sum(c["data"].size for c in cases)
    value = world * bytes_step * K / (ms_total / 1e3) / 1e9

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
        for c in cases:   # one untimed pass (scratch sizing)
            _host_call(gbu, ctx, c, outs, sh)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for c in cases:
                r = _host_call(gbu, ctx, c, outs, sh)
                if r.status != gbu.GBU_OK or r.out_len != c["out_len"]:
                    raise RuntimeError(f"host call mismatch {r}")
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dtt = torch.tensor([dt], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(dtt, op=dist.ReduceOp.MAX)
        dt = float(dtt.item())
        e2e = {"value": world * h2d * args.e2e_steps / dt / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "steps": args.e2e_steps, "api": "gbu_*_host (pinned host buffers)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        b, dt = cpu_baseline(cases, args.cpu_sample)
        cpu = {"value": b / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle (scalar C, 1 thread) on the first "
                         f"{args.cpu_sample >> 20} MiB of each of the {len(cases)} buffers "
                         f"({b / 1e9:.2f} GB total, {dt:.1f} s)"}

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
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def _host_call(gbu, ctx, c, outs, sh):
    out = outs[c["dir"]]
    if c["dir"] == "utf8_to_utf16le":
        return gbu.gbu_utf8_to_utf16le_host(ctx.handle, c["h_in"].data_ptr(), c["n"],
                                            out.data_ptr(), c["cap"], sh)
    return gbu.gbu_utf16le_to_utf8_host(ctx.handle, c["h_in"].data_ptr(), c["n"],
                                        out.data_ptr(), c["cap"], sh)


if __name__ == "__main__":
    main()
