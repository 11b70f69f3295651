#!/usr/bin/env python
"""Benchmark of the Huffman hot path (histogram -> codebook -> encode ->
decode) on GB300, through the library's C ABI.

One step = the whole path over one synthetic buffer resident in HBM:
huff_histogram_units, huff_build_codebook, huff_encode_units, huff_decode.
The workload is the paper-shaped text of 1 GiB (the scale study of the
paper's ~45 MB English corpus, Section III-A): words from a seeded 50,000-word
vocabulary with Zipf(1.0) frequencies, seed 1, 16384-symbol chunks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is uncompressed bytes per second of the whole
step (GB/s, 1e9 B/s) summed over ranks.  With --gpus N > 1 (launched by
torch.distributed.run) every rank runs its own replica: the path does not
shard, so there is no collective on the data path ("scaling": "weak").
`--impl reference` times the plain CPU oracle on a bounded sample of the same
workload instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Huffman enc/dec GB/s & % HBM roofline; batched vs plain; served p50/p99 ms"
WORKLOAD = "text_1g"
WORKLOAD_DESC = ("synthetic Zipf-word text (50,000-word vocabulary, Zipf(1.0), 5% punctuation, "
                 "newline at 80 chars), 1 GiB, seed 1, 16384-symbol chunks")
REF_SAMPLE = 16 << 20       # bytes per reference-arm step
CPU_SAMPLE = 256 << 20      # bytes of the CPU-baseline sample


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def mark(self, begin: bool):
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        rows = [r.split(", ") for r in out.strip().splitlines() if r.count(",") >= 8]
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, nm in enumerate(names):
                if r[5 + i].strip() == "Active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return
    import oracle
    import synth
    x = synth.text(REF_SAMPLE, 1)  # the first 16 MiB of the 1 GiB workload
    times = []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        st, s = oracle.compress(x)
        st2, back, n = oracle.decode(s)
        dt = time.perf_counter() - t
        assert st == 0 and st2 == 0 and n == x.size
        if i >= args.warmup:
            times.append(dt)
    sec = sum(times) / len(times)
    gbs = x.size / sec / 1e9
    sample = f"first {REF_SAMPLE >> 20} MiB of {WORKLOAD} per step, oracle compress + decode"
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC, "sample_bytes": REF_SAMPLE},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def cpu_baseline(x):
    import oracle
    sample = x[:CPU_SAMPLE]
    t = time.perf_counter()
    st, s = oracle.compress(sample)
    st2, back, n = oracle.decode(s)
    dt = time.perf_counter() - t
    assert st == 0 and st2 == 0 and n == sample.size
    return {"value": sample.size / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"first {CPU_SAMPLE >> 20} MiB of {WORKLOAD}: one oracle compress + decode, "
                      f"1 thread, {dt:.1f} s"}


def run_ours(args):
    import numpy as np
    import torch
    import synth
    import paper_2306_11070_gb300 as hg
    from paper_2306_11070_gb300 import build as nvbuild

    rank, world, local = rank_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    nvbuild.build()
    dev = torch.device("cuda", torch.cuda.current_device())

    x = synth.make(WORKLOAD)
    n = x.size
    base = cpu_baseline(x) if (rank == 0 and world == 1 and not args.no_cpu) else None

    d_x = torch.from_numpy(x).to(dev)
    hist = torch.empty(256, dtype=torch.int64, device=dev)
    uh = torch.empty(hg.huff_unit_hist_size(n), dtype=torch.uint8, device=dev)
    cb = torch.empty(hg.CODEBOOK_BYTES, dtype=torch.uint8, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    cap = hg.huff_max_stream_size(n)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    ob = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = torch.empty(hg.huff_workspace_size(n), dtype=torch.uint8, device=dev)
    dec = torch.empty(n, dtype=torch.uint8, device=dev)
    dn = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    # five events per timed step bracket the four calls (kernels on this stream)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    launches_per_step = 6  # histogram, codebook, unit bits, unit scan, encode, decode

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        hg.huff_histogram_units(d_x, hist, uh)
        if ev:
            ev[1].record(stream)
        hg.huff_build_codebook(hist, cb, st)
        if ev:
            ev[2].record(stream)
        hg.huff_encode_units(d_x, cb, uh, d_out=out, d_out_bytes=ob, d_ws=ws, d_status=st)
        if ev:
            ev[3].record(stream)
        hg.huff_decode(out, cap, d_out=dec, out_cap=n, d_n=dn, d_status=st)
        if ev:
            ev[4].record(stream)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    nbytes = int(ob.item())
    ok = int(st.item()) == 0 and torch.equal(dec, d_x)
    if not ok:
        raise SystemExit(f"bench: round trip failed (status {int(st.item())})")

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier()
    clocks.mark(True)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t_end.record(stream)
    barrier()
    clocks.mark(False)
    elapsed_ms = t_start.elapsed_time(t_end)
    acc = [sum(ev[i].elapsed_time(ev[i + 1]) for ev in evs) for i in range(4)]
    if dist is not None:
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    ms_per_step = elapsed_ms / args.steps

    # end to end through the public API from pinned host memory
    h_x = torch.from_numpy(x).pin_memory()
    h_stream = torch.empty(cap, dtype=torch.uint8).pin_memory()
    h_out = torch.empty(n, dtype=torch.uint8).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        d_x.copy_(h_x, non_blocking=True)
        hg.huff_compress(d_x, d_out=out, d_out_bytes=ob, d_ws=ws, d_status=st)
        size = int(ob.item())  # sync: the caller learns the stream size
        h_stream[:size].copy_(out[:size], non_blocking=True)
        hg.huff_decode(out, size, d_out=dec, out_cap=n, d_n=dn, d_status=st)
        h_out.copy_(dec, non_blocking=True)
        torch.cuda.synchronize()
    e2e_sec = (time.perf_counter() - t0) / e2e_steps
    if dist is not None:
        t = torch.tensor([e2e_sec], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_sec = float(t.item())
    ok = int(st.item()) == 0 and torch.equal(h_out, h_x)
    clk = clocks.stop()
    if not ok:
        raise SystemExit("bench: end-to-end round trip failed")

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    per_k = [a / args.steps for a in acc]  # ms per launch
    names = ["histogram", "codebook", "encode", "decode"]
    alg = [n, 0, n + nbytes, n + nbytes]
    peak, peak_src = load_peaks()
    kern = {nm: {"ms": per_k[i],
                 "gbs_uncompressed": n / (per_k[i] * 1e-3) / 1e9,
                 "gbs_algorithmic": (alg[i] / (per_k[i] * 1e-3) / 1e9) if alg[i] else None}
            for i, nm in enumerate(names)}
    dom = max(range(4), key=lambda i: per_k[i])
    achieved = alg[dom] / (per_k[dom] * 1e-3) / 1e9
    line = {
        "metric": METRIC,
        "value": world * n / (ms_per_step * 1e-3) / 1e9,
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC, "n_bytes": n,
                   "stream_bytes": nbytes, "compression_ratio": nbytes / n,
                   "l2": "inputs larger than L2 (1 GiB vs 129 MB), no flush",
                   "parallelism": f"replicas x{world}"},
        "clocks": clk,
        "e2e": {"value": world * n / e2e_sec / 1e9, "unit": "GB/s", "h2d_bytes_per_step": n,
                "d2h_bytes_per_step": nbytes + n + 8},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": {"kernel": names[dom], "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_src == "measured" else "fallback 6.8 TB/s"},
        "kernels": kern,
        "cpu_baseline": base,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline sample")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
