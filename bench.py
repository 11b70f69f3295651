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
E2E_PASSES = 9  # end-to-end passes of e2e_steps steps; the median is reported
E2E_SETS = 2  # buffer sets the end-to-end pipeline rotates through (3 or 4: slower, 78-102 GB/s)
WORKLOAD_DESC = ("synthetic Zipf-word text (50,000-word vocabulary, Zipf(1.0), 5% punctuation, "
                 "newline at 80 chars), 1 GiB, seed 1, 16384-symbol chunks")
REF_SAMPLE = 16 << 20       # bytes per reference-arm step
CPU_SAMPLE = 256 << 20      # bytes of the CPU-baseline sample


# The paper's own compression latencies (Tables I and II: its ~45 MB text
# corpus on CPU clusters, 4 cores per node, compression only), quoted beside
# the GPU figures as context; they are not a target (other hardware, other
# data, undefined I/O inclusion).
PAPER_CORPUS_MB = 45.0
PAPER_TIMINGS = [
    ("Method 1 (sequential)", "Beta", 1, 7.4105),
    ("Method 1 (sequential)", "Iota", 1, 5.5988),
    ("Method 2 (MPI+OpenMP)", "Beta", 4, 4.754),
    ("Method 2 (UPC)", "Iota", 4, 4.671),
    ("Method 3 (MPI only)", "Beta", 4, 1.219),
    ("Method 3 (MPI only)", "Iota", 2, 0.732),
]


def paper_context(compress_gbs):
    return {"source": "the paper's Tables I-II (compression of a ~45 MB text corpus on CPU "
                      "clusters, 4 cores per node); context only, not a target",
            "rows_mb_per_s": {f"{m} {c} x{k}": round(PAPER_CORPUS_MB / t, 2)
                              for m, c, k, t in PAPER_TIMINGS},
            "ours_compress_gbs": compress_gbs}


def rounded(obj, digits=4):
    """The JSON line's floats to `digits` significant digits (the line stays
    short enough to be kept whole)."""
    if isinstance(obj, float):
        return float(f"{obj:.{digits}g}")
    if isinstance(obj, dict):
        return {k: rounded(v, digits) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [rounded(v, digits) for v in obj]
    return obj


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (a time), via all-reduce; x itself on one
    process.  Works with nccl (device tensor) and gloo (CPU tensor)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbs(world, n_bytes, seconds):
    """Whole-job throughput: every rank processes n_bytes per step, and the
    job's step takes the slowest rank's time."""
    return world * n_bytes / seconds / 1e9


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
    line = {"value": sample.size / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"first {CPU_SAMPLE >> 20} MiB of {WORKLOAD}: one oracle compress + decode, "
                      f"1 thread, {dt:.1f} s"}
    line["segmented_threads"] = cpu_segmented(sample)
    return line


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or ''."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return ""


def cpu_segmented(sample):
    """Reported only: the paper's Method 2 on this host -- the sample cut into
    one segment per core, each compressed with its own codebook and decoded
    by the oracle on its own thread (the oracle's C calls release the GIL)."""
    import platform
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    cores = os.cpu_count() or 1
    seg = (sample.size + cores - 1) // cores
    parts = [sample[i:i + seg] for i in range(0, sample.size, seg)]

    def one(p):
        st, s = oracle.compress(p)
        st2, back, n = oracle.decode(s)
        return st == 0 and st2 == 0 and n == p.size

    t = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        ok = all(ex.map(one, parts))
    dt = time.perf_counter() - t
    assert ok
    return {"value": sample.size / dt / 1e9, "unit": "GB/s", "cores": cores,
            "machine": platform.machine(), "cpu_model": cpu_model(),
            "sample": f"same sample in {len(parts)} segments with their own codebooks, "
                      f"{cores} threads, {dt:.1f} s"}


def measure_batched(hg, synth, torch, count=4096):
    """Config 3: `count` independent text buffers (log-uniform 1 KiB..4 MiB,
    per-buffer seeds), one fused launch per batch (CUDA graph) with
    autotuned chunk size, lanes per buffer and CTAs per SM, vs one plain
    call per buffer on one stream."""
    from concurrent.futures import ThreadPoolExecutor
    sizes = synth.log_uniform_sizes(count, seed=3, lo=1024, hi=4 << 20)
    with ThreadPoolExecutor(16) as ex:
        xs = list(ex.map(lambda i: synth.text(int(sizes[i]), synth.batch_seed(i)), range(count)))
    total = float(sizes.sum())
    ins = [torch.from_numpy(x).cuda() for x in xs]
    # outputs sized for the smallest candidate chunk size, so the tuner may pick it
    outs = [torch.empty(hg.huff_max_stream_size(x.size, 4096), dtype=torch.uint8, device="cuda")
            for x in xs]
    t0 = time.perf_counter()
    probe = hg.BatchPlan(ins, outs, hg.HUFF_BATCH_COMPRESS)
    cbest = probe.autotune(flags=hg.HUFF_TUNE_ROUND_TRIP)
    probe.close()
    tune_c = time.perf_counter() - t0
    plan = hg.BatchPlan(ins, outs, hg.HUFF_BATCH_COMPRESS, cbest)

    def t_ms(fn, reps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            fn()
        e.record()
        torch.cuda.synchronize()
        return s.elapsed_time(e) / reps

    tc = t_ms(plan.run, 10, 3)
    nb = plan.out_bytes.cpu().numpy()
    assert (plan.status.cpu().numpy() == 0).all()
    streams = [outs[i][:int(nb[i])] for i in range(count)]
    decs = [torch.empty(max(x.size, 16), dtype=torch.uint8, device="cuda") for x in xs]
    t0 = time.perf_counter()
    probe = hg.BatchPlan(streams, decs, hg.HUFF_BATCH_DECOMPRESS)
    dbest = probe.autotune()
    probe.close()
    tune_d = time.perf_counter() - t0
    dplan = hg.BatchPlan(streams, decs, hg.HUFF_BATCH_DECOMPRESS, dbest)
    td = t_ms(dplan.run, 10, 3)
    assert (dplan.status.cpu().numpy() == 0).all()
    ok = all(torch.equal(decs[i][:xs[i].size], ins[i]) for i in range(count))
    ws = torch.empty(hg.huff_workspace_size(int(sizes.max())), dtype=torch.uint8, device="cuda")
    obs = torch.zeros(count, dtype=torch.int64, device="cuda")
    sts = torch.zeros(count, dtype=torch.int32, device="cuda")
    dns = torch.zeros(count, dtype=torch.int64, device="cuda")

    def plain_c():
        for i in range(count):
            hg.huff_compress(ins[i], d_out=outs[i], d_out_bytes=obs[i:i + 1], d_ws=ws,
                             d_status=sts[i:i + 1])

    def plain_d():
        for i in range(count):
            hg.huff_decode(streams[i], int(nb[i]), d_out=decs[i], out_cap=xs[i].size,
                           d_n=dns[i:i + 1], d_status=sts[i:i + 1])

    pc = t_ms(plain_c, 2, 1)
    pd = t_ms(plain_d, 2, 1)
    info = plan.info()
    plan.close()
    dplan.close()
    return {"workload": f"{count} text buffers, log-uniform 1 KiB-4 MiB, {total / 2**30:.3f} GiB",
            "graph": info["graph"], "grid": info["grid"], "round_trip_ok": ok,
            "autotuned": {"chunk_symbols": cbest.chunk_symbols,
                          "compress_ctas_per_sm": cbest.ctas_per_sm,
                          "decode_lanes": dbest.decode_lanes,
                          "decompress_ctas_per_sm": dbest.ctas_per_sm,
                          "tune_s": round(tune_c + tune_d, 2)},
            "compress_ms": tc, "compress_gbs": total / tc / 1e6,
            "decompress_ms": td, "decompress_gbs": total / td / 1e6,
            "plain_compress_ms": pc, "plain_decompress_ms": pd,
            "speedup_compress": pc / tc, "speedup_decompress": pd / td}


def measure_method3(hg, synth, torch, oracle=None, n=256 << 20, block=1 << 20,
                    segment=16384):
    """Method 3 (NEXT row): the block-sorting transform of every 1 MiB block of
    256 MiB of synthetic text, its inverse, and the Method 3 container (16 KiB
    segments, one codebook each), timed with CUDA events around the
    synchronous calls; the compression ratio against Method 2 at the same
    segment size and against one codebook; the oracle's transform timed on a
    sample of blocks on the host."""
    x = torch.from_numpy(synth.text(n, 1)).cuda()
    wsb = hg.lib().huff_bwt_workspace_size(n, block)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    last = torch.empty(n, dtype=torch.uint8, device="cuda")
    prim = torch.empty((n + block - 1) // block, dtype=torch.int32, device="cuda")
    back = torch.empty(n, dtype=torch.uint8, device="cuda")

    def t_ms(fn, reps=3, warm=1):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        return float(statistics.median(ts))

    tf = t_ms(lambda: hg.huff_bwt_forward(x, block, d_last=last, d_primary=prim, ws=ws))
    ti = t_ms(lambda: hg.huff_bwt_inverse(last, block, prim, d_out=back, ws=ws))
    ok = bool(torch.equal(back, x))
    del ws
    c, st = hg.huff_m3_compress(x, block, segment)
    tc = t_ms(lambda: hg.huff_m3_compress(x, block, segment), reps=2)
    y, m, st2 = hg.huff_m3_decompress(c)
    td = t_ms(lambda: hg.huff_m3_decompress(c), reps=2)
    ok = ok and int(st.item()) == 0 and int(st2.item()) == 0 and m == n and bool(torch.equal(y, x))
    # with move-to-front after the transform (64 KiB segments suit its output)
    mws = torch.empty(hg.lib().huff_mtf_workspace_size(n, block), dtype=torch.uint8,
                      device="cuda")
    mtf_out = torch.empty(n, dtype=torch.uint8, device="cuda")
    tmf = t_ms(lambda: hg.huff_mtf_forward(last, block, d_out=mtf_out, ws=mws))
    tmi = t_ms(lambda: hg.huff_mtf_inverse(mtf_out, block, d_out=back, ws=mws))
    ok = ok and bool(torch.equal(back, last))
    del mws, mtf_out
    seg_mtf = 65536
    cm, stm = hg.huff_m3_compress(x, block, seg_mtf, stages=hg.HUFF_M3_MTF)
    tcm = t_ms(lambda: hg.huff_m3_compress(x, block, seg_mtf, stages=hg.HUFF_M3_MTF), reps=2)
    ym, mm, stm2 = hg.huff_m3_decompress(cm)
    tdm = t_ms(lambda: hg.huff_m3_decompress(cm), reps=2)
    ok = ok and int(stm.item()) == 0 and int(stm2.item()) == 0 and mm == n and \
        bool(torch.equal(ym, x))
    seg_c, _ = hg.huff_segmented_compress(x, segment)
    one = hg.compress(x)
    out = {"workload": f"synthetic text {n >> 20} MiB (seed 1), {block >> 20} MiB blocks, "
                       f"{segment >> 10} KiB segments",
           "round_trip_ok": ok,
           "forward_ms": tf, "forward_gbs": n / tf / 1e6,
           "inverse_ms": ti, "inverse_gbs": n / ti / 1e6,
           "m3_compress_ms": tc, "m3_compress_gbs": n / tc / 1e6,
           "m3_decompress_ms": td, "m3_decompress_gbs": n / td / 1e6,
           "mtf_forward_gbs": n / tmf / 1e6, "mtf_inverse_gbs": n / tmi / 1e6,
           "m3_mtf_compress_ms": tcm, "m3_mtf_decompress_ms": tdm,
           "ratio_m3_mtf_64k_segments": cm.numel() / n,
           "ratio_m3": c.numel() / n, "ratio_segmented_same_segments": seg_c.numel() / n,
           "ratio_one_codebook": one.numel() / n,
           "bound": "radix-pass bound (stable radix passes and random rank scatters)"}
    if oracle is not None:
        xs = x[:4 * block].cpu().numpy()
        t0 = time.perf_counter()
        L, P = oracle.bwt(xs, block)
        t1 = time.perf_counter()
        oracle.ibwt(L, block, P)
        t2 = time.perf_counter()
        M = oracle.mtf(L, block)
        t3 = time.perf_counter()
        oracle.imtf(M, block)
        t4 = time.perf_counter()
        out["cpu_baseline"] = {"kind": "oracle", "cores": 1,
                               "sample": f"the first 4 blocks ({4 * block >> 20} MiB)",
                               "forward_gbs": xs.size / (t1 - t0) / 1e9,
                               "inverse_gbs": xs.size / (t2 - t1) / 1e9,
                               "mtf_forward_gbs": xs.size / (t3 - t2) / 1e9,
                               "mtf_inverse_gbs": xs.size / (t4 - t3) / 1e9}
    return out


def measure_next_rows(hg, synth, torch, oracle=None):
    """Two next rows of the path on their own workloads: length-limited
    codebooks (12-bit limit) on the 1 GiB geometric stress input, whose
    Huffman codes run to ~29 bits, against the unlimited codebook; and
    per-segment codebooks (Method 2 taken literally) on 256 MiB of text in
    1 MiB segments, with the oracle's container timed on a 16 MiB sample."""
    def t_ms(fn, reps=5, warm=2):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        return float(statistics.median(ts))

    res = {}
    x = torch.from_numpy(synth.make("geometric_1g")).cuda()
    n = x.numel()
    dev = x.device
    h = hg.huff_histogram(x)
    ws = torch.empty(hg.huff_workspace_size(n), dtype=torch.uint8, device=dev)
    buf = torch.empty(hg.huff_max_stream_size(n), dtype=torch.uint8, device=dev)
    ob = torch.zeros(1, dtype=torch.int64, device=dev)
    dn = torch.zeros(1, dtype=torch.int64, device=dev)
    dec = torch.empty(n, dtype=torch.uint8, device=dev)
    rows = {}
    for name, limit in (("huffman", None), ("limited_12", 12)):
        cb, st = (hg.huff_build_codebook(h) if limit is None
                  else hg.huff_build_codebook_limited(h, limit))

        def enc(cb=cb, st=st):
            hg.huff_encode(x, cb, d_out=buf, d_out_bytes=ob, d_ws=ws, d_status=st)

        te = t_ms(enc)
        enc()
        torch.cuda.synchronize()
        nb = int(ob.item())
        td = t_ms(lambda st=st: hg.huff_decode(buf, nb, d_out=dec, out_cap=n, d_n=dn,
                                                d_status=st))
        max_len = int.from_bytes(bytes(cb[1284:1288].cpu().numpy()), "little")
        rows[name] = {"max_len": max_len, "encode_ms": te, "decode_ms": td,
                      "stream_ratio": nb / n,
                      "round_trip_ok": int(st.item()) == 0 and bool(torch.equal(dec, x))}
    res["length_limited"] = {"workload": "geometric_1g (p = 0.5 over 256 bytes, 1 GiB, seed 41)",
                             **rows}
    del x, ws, buf, dec
    torch.cuda.empty_cache()
    n2, seg = 256 << 20, 1 << 20
    x2 = torch.from_numpy(synth.text(n2, 1)).cuda()
    # each call plans its batch on the host and synchronises: ten calls after
    # three warm-up calls, so that the host's allocator has settled
    tc = t_ms(lambda: hg.huff_segmented_compress(x2, seg), reps=10, warm=3)
    c, st = hg.huff_segmented_compress(x2, seg)
    td = t_ms(lambda: hg.huff_segmented_decompress(c), reps=10, warm=3)
    back, m, st2 = hg.huff_segmented_decompress(c)
    torch.cuda.synchronize()
    seg_row = {"workload": "synthetic text 256 MiB (seed 1), 1 MiB segments, own codebook each",
               "compress_ms": tc, "compress_gbs": n2 / tc / 1e6,
               "decompress_ms": td, "decompress_gbs": n2 / td / 1e6,
               "ratio": c.numel() / n2,
               "round_trip_ok": int(st.item()) == 0 and int(st2.item()) == 0 and m == n2
               and bool(torch.equal(back, x2))}
    if oracle is not None:
        sample = x2[:16 << 20].cpu().numpy()
        t0 = time.perf_counter()
        oracle.segmented_compress(sample, seg)
        dt = time.perf_counter() - t0
        seg_row["cpu_baseline"] = {"kind": "oracle", "cores": 1,
                                   "sample": "the first 16 MiB, compress only",
                                   "compress_gbs": sample.size / dt / 1e9}
    res["segmented"] = seg_row
    del x2, c, back
    torch.cuda.empty_cache()
    res["lzss"] = measure_lzss(hg, synth, torch, t_ms, oracle)
    return res


def measure_lzss(hg, synth, torch, t_ms, oracle=None):
    """LZSS Method 2 (Section III-B) with the paper's configuration
    "1024/24/12/8" (window, longest and shortest match, literal block, in
    bits) and the stored-prefix window, on 256 MiB of the bitstream stand-in
    in 64 KiB segments, with pre-allocated buffers (no allocation or host
    synchronisation inside a call)."""
    n, seg = 256 << 20, 64 << 10
    params = hg.LZSS_PAPER
    x = torch.from_numpy(synth.make("bitstream_256m")).cuda()
    L = hg.lib()
    P = hg._lzss_params(params)
    out = torch.empty(L.huff_lzss_max_size(n, seg, P), dtype=torch.uint8, device="cuda")
    ws = torch.empty(L.huff_lzss_workspace_size(n, seg, P), dtype=torch.uint8, device="cuda")
    ob = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")

    def comp():
        hg.huff_lzss_compress(x, seg, params, d_out=out, d_out_bytes=ob, d_ws=ws, d_status=st)

    tc = t_ms(comp, reps=3, warm=1)
    comp()
    torch.cuda.synchronize()
    size = int(ob.item())
    c = out[:size]
    y = torch.empty(n, dtype=torch.uint8, device="cuda")
    dn = torch.zeros(1, dtype=torch.int64, device="cuda")
    st2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    dws = torch.empty(L.huff_lzss_decompress_workspace_size(size), dtype=torch.uint8,
                      device="cuda")

    def decomp():
        hg.huff_lzss_decompress(c, d_out=y, d_n=dn, d_ws=dws, d_status=st2)

    td = t_ms(decomp, reps=3, warm=1)
    decomp()
    torch.cuda.synchronize()
    row = {"workload": "bitstream stand-in 256 MiB (seed 7), 64 KiB segments, 1024/24/12/8, "
                       "stored-prefix window",
           "compress_ms": tc, "compress_gbs": n / tc / 1e6,
           "decompress_ms": td, "decompress_gbs": n / td / 1e6,
           "ratio": size / n,
           "round_trip_ok": int(st.item()) == 0 and int(st2.item()) == 0 and
           int(dn.item()) == n and bool(torch.equal(y, x)),
           "paper_context": "Table V-VI, Method 2 with Dict 2 on 4 cores: adder bitstream "
                            "(763 kB) 43.4% saved in 5.8 s, processor (1.8 MB) 29.1% in 12.11 s"}
    if oracle is not None:
        sample = x[:256 << 10].cpu().numpy()
        t0 = time.perf_counter()
        oracle.lzss_segmented_compress(sample, seg, params)
        dt = time.perf_counter() - t0
        row["cpu_baseline"] = {"kind": "oracle", "cores": 1,
                               "sample": "the first 256 KiB, compress only",
                               "compress_gbs": sample.size / dt / 1e9}
    return row


def measure_served(hg, synth, oracle, torch, loads=(10.0, 20.0, 50.0, 100.0, 150.0, 200.0),
                   seconds=1.0, max_requests=2000):
    """Config 5: open-loop Poisson arrivals of 50/50 compress/decompress
    requests over a pool of 64 text buffers with log-uniform sizes
    4 KiB..16 MiB (streams for decompression pre-made by the oracle), served
    by the continuous-batching loop under an 8 GiB budget, vs the same trace
    served one request at a time through the plain calls."""
    import numpy as np
    rng_sizes = synth.log_uniform_sizes(64, seed=5, lo=4096, hi=16 << 20)
    pool = []
    for i, n in enumerate(rng_sizes):
        x = synth.text(int(n), 7000 + i)
        st, s = oracle.compress(x)
        assert st == 0
        hx = torch.from_numpy(x).pin_memory()
        hs = torch.from_numpy(s).pin_memory()
        pool.append((x, s, hx, hs))
    mean = float(np.mean([p[0].size for p in pool]))
    srv = hg.Server()
    results = []
    # the first pass (the first load, 200 requests) warms the server up and
    # is not reported: its first rounds pay one-time set-up costs
    for idx, load in enumerate((loads[0],) + tuple(loads)):
        warmup = idx == 0
        lam = load * 1e9 / mean
        count = 200 if warmup else min(max_requests, max(200, int(lam * seconds)))
        t_arr, op, _ = synth.poisson_trace(count, seed=5, lam=lam)
        pick = (synth.log_uniform_sizes(count, seed=55, lo=1, hi=64) - 1).astype(np.int64) % 64
        outs = [torch.empty(hg.huff_max_stream_size(pool[j][0].size) if o == 0 else pool[j][0].size,
                            dtype=torch.uint8).pin_memory() for o, j in zip(op, pick)]
        # served, open loop
        import time
        t0 = time.perf_counter()
        tickets, lag = [], []
        for i in range(count):
            while time.perf_counter() - t0 < t_arr[i]:
                pass
            lag.append(time.perf_counter() - t0 - t_arr[i])
            x, s, hx, hs = pool[pick[i]]
            if op[i] == 0:
                tickets.append(srv.submit(hg.HUFF_BATCH_COMPRESS, hx, outs[i]))
            else:
                tickets.append(srv.submit(hg.HUFF_BATCH_DECOMPRESS, hs, outs[i]))
        res = [srv.wait(t, 600000) for t in tickets]
        lat = [r["t_done"] - r["t_submit"] + lg for r, lg in zip(res, lag)]
        span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
        nbytes = sum(pool[j][0].size for j in pick)
        bad = 0
        for i, r in enumerate(res):
            x, s, _, _ = pool[pick[i]]
            ref = s if op[i] == 0 else x
            if r["status"] != 0 or r["out_bytes"] != ref.size or \
                    not np.array_equal(outs[i][:ref.size].numpy(), ref):
                bad += 1
            srv.release(tickets[i])
        # plain, one request at a time, same arrival times
        dev = torch.device("cuda")
        cap = max(hg.huff_max_stream_size(p[0].size) for p in pool)
        d_in = torch.empty(cap, dtype=torch.uint8, device=dev)
        d_out = torch.empty(cap, dtype=torch.uint8, device=dev)
        ws = torch.empty(hg.huff_workspace_size(max(p[0].size for p in pool)), dtype=torch.uint8,
                         device=dev)
        ob = torch.zeros(1, dtype=torch.int64, device=dev)
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        plat = []
        t0 = time.perf_counter()
        for i in range(count):
            now = time.perf_counter() - t0
            if now < t_arr[i]:
                while time.perf_counter() - t0 < t_arr[i]:
                    pass
            x, s, hx, hs = pool[pick[i]]
            if op[i] == 0:
                d_in[:x.size].copy_(hx, non_blocking=True)
                hg.huff_compress(d_in[:x.size], d_out=d_out, d_out_bytes=ob, d_ws=ws, d_status=st)
                m = int(ob.item())
            else:
                d_in[:s.size].copy_(hs, non_blocking=True)
                hg.huff_decode(d_in[:s.size], s.size, d_out=d_out, out_cap=x.size, d_n=ob,
                               d_status=st)
                m = int(ob.item())
            outs[i][:m].copy_(d_out[:m], non_blocking=True)
            torch.cuda.synchronize()
            plat.append(time.perf_counter() - t0 - t_arr[i])
        pspan = time.perf_counter() - t0 - t_arr[0]
        lat_ms = np.array(lat) * 1e3
        plat_ms = np.array(plat) * 1e3
        if warmup:
            continue
        results.append({"offered_gbs": load, "requests": count, "gbs": nbytes / span / 1e9,
                        "p50_ms": float(np.percentile(lat_ms, 50)),
                        "p99_ms": float(np.percentile(lat_ms, 99)),
                        "plain_gbs": nbytes / pspan / 1e9,
                        "plain_p50": float(np.percentile(plat_ms, 50)),
                        "plain_p99": float(np.percentile(plat_ms, 99)),
                        "bad": bad})
    srv.close()
    return {"workload": "Poisson 50/50 compress/decompress, 64 text buffers log-uniform "
                        "4 KiB-16 MiB, 8 GiB budget, 3 rounds in flight",
            "mean_request_bytes": mean, "points": results}


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
    # k_histogram, k_build_codebook, k_unit_bits_hist, k_scan_tile_sums,
    # k_scan_apply, k_encode_mad and k_encode (one of the two returns at once),
    # k_decode
    launches_per_step = 8

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
    elapsed_ms = max_over_ranks(elapsed_ms, dist, dev)
    ms_per_step = elapsed_ms / args.steps

    # end to end through the public API from pinned host memory, pipelined
    # over E2E_SETS buffer sets: later steps' host-to-device copies and
    # earlier steps' device-to-host copies run on their own streams while
    # step k computes
    h_x = torch.from_numpy(x).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    sets = []
    for b in range(E2E_SETS):
        sets.append({
            "d_x": d_x if b == 0 else torch.empty_like(d_x),
            "out": out if b == 0 else torch.empty_like(out),
            "dec": dec if b == 0 else torch.empty_like(dec),
            "ws": ws if b == 0 else torch.empty_like(ws),
            "ob": torch.zeros(1, dtype=torch.int64, device=dev),
            "st": torch.zeros(1, dtype=torch.int32, device=dev),
            "dn": torch.zeros(1, dtype=torch.int64, device=dev),
            "ob_h": torch.zeros(1, dtype=torch.int64).pin_memory(),
            "h_stream": torch.empty(cap, dtype=torch.uint8).pin_memory(),
            "h_out": torch.empty(n, dtype=torch.uint8).pin_memory(),
            "ev_in": torch.cuda.Event(), "ev_c": torch.cuda.Event(),
            "ev_d": torch.cuda.Event(), "ev_done": torch.cuda.Event(),
        })
    s_in, s_comp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

    def enqueue_in_and_compute(k):
        b = sets[k % E2E_SETS]
        with torch.cuda.stream(s_in):
            if k >= E2E_SETS:
                s_in.wait_event(b["ev_done"])  # step k-2 no longer reads this set
            b["d_x"].copy_(h_x, non_blocking=True)
            b["ev_in"].record(s_in)
        with torch.cuda.stream(s_comp):
            s_comp.wait_event(b["ev_in"])
            hg.huff_compress(b["d_x"], d_out=b["out"], d_out_bytes=b["ob"], d_ws=b["ws"],
                             d_status=b["st"], stream=s_comp)
            b["ob_h"].copy_(b["ob"], non_blocking=True)
            b["ev_c"].record(s_comp)
            hg.huff_decode(b["out"], cap, d_out=b["dec"], out_cap=n, d_n=b["dn"],
                           d_status=b["st"], stream=s_comp)
            b["ev_d"].record(s_comp)

    def e2e_pass():
        barrier()
        t0 = time.perf_counter()
        ahead = E2E_SETS - 1  # steps enqueued ahead of the one being copied out
        for j in range(min(ahead, e2e_steps)):
            enqueue_in_and_compute(j)
        for k in range(e2e_steps):
            if k + ahead < e2e_steps:
                enqueue_in_and_compute(k + ahead)
            b = sets[k % E2E_SETS]
            b["ev_c"].synchronize()  # the caller learns the stream size
            size = int(b["ob_h"].item())
            with torch.cuda.stream(s_out):
                s_out.wait_event(b["ev_c"])
                b["h_stream"][:size].copy_(b["out"][:size], non_blocking=True)
                s_out.wait_event(b["ev_d"])
                b["h_out"].copy_(b["dec"], non_blocking=True)
                b["ev_done"].record(s_out)
        torch.cuda.synchronize()
        return max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist, dev)

    # the host link is shared with the machine's other GPUs and tenants, so
    # one pass can land on a busy moment: E2E_PASSES passes, the median kept
    # and every pass reported
    e2e_passes = [e2e_pass() for _ in range(E2E_PASSES)]
    e2e_sec = statistics.median(e2e_passes)
    ok = all(int(b["st"].item()) == 0 for b in sets) and \
        torch.equal(sets[(e2e_steps - 1) % E2E_SETS]["h_out"], h_x)
    del sets
    clk = clocks.stop()
    if not ok:
        raise SystemExit("bench: end-to-end round trip failed")
    del h_x
    # the host-only oracle runs after every GPU timing of the step, so that
    # nothing it leaves behind on the host shares the timed region
    base = cpu_baseline(x) if (rank == 0 and world == 1 and not args.no_cpu) else None
    batched = served = method3 = next_rows = None
    if rank == 0 and not args.no_batched:
        batched = measure_batched(hg, synth, torch)
    if rank == 0 and not args.no_served:
        import oracle
        served = measure_served(hg, synth, oracle, torch)
    if rank == 0 and not args.no_method3:
        m3_oracle = None
        if world == 1 and not args.no_cpu:
            import oracle as m3_oracle
        method3 = measure_method3(hg, synth, torch, m3_oracle)
        next_rows = measure_next_rows(hg, synth, torch, m3_oracle)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    per_k = [a / args.steps for a in acc]  # ms per launch
    names = ["histogram", "codebook", "encode", "decode"]
    alg = [n, 0, n + nbytes, n + nbytes]
    peak, peak_src = load_peaks()
    dom = max(range(4), key=lambda i: per_k[i])
    achieved = alg[dom] / (per_k[dom] * 1e-3) / 1e9
    traffic = profiled_traffic("k_" + names[dom])
    kern = {nm: {"ms": per_k[i],
                 "gbs_algorithmic": (alg[i] / (per_k[i] * 1e-3) / 1e9) if alg[i] else None,
                 "frac": (alg[i] / (per_k[i] * 1e-3) / 1e9 / peak) if alg[i] else None}
            for i, nm in enumerate(names)}
    # the headline evidence (roofline, kernels, batched, served) goes last:
    # readers that keep only the end of a long line still see it
    line = {
        "metric": METRIC,
        "value": job_gbs(world, n, ms_per_step * 1e-3),
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
        "e2e": {"value": job_gbs(world, n, e2e_sec), "unit": "GB/s", "h2d_bytes_per_step": n,
                "passes_gbs": [job_gbs(world, n, t) for t in e2e_passes],
                "d2h_bytes_per_step": nbytes + n + 8,
                "how": f"huff_compress + huff_decode from pinned host memory, {E2E_SETS} buffer "
                       f"sets, copies on their own streams; median of {E2E_PASSES} passes of "
                       f"{e2e_steps} steps"},
        "gpu_launches": launches_per_step * args.steps,
        "cpu_baseline": base,
        "paper_context": paper_context(n / ((per_k[0] + per_k[1] + per_k[2]) * 1e-3) / 1e9),
        "method3": method3,
        "next_rows": next_rows,
        "roofline": {"kernel": names[dom], "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "frac_of_nominal_8tbs": achieved / 8000.0,
                     "traffic_source": "ncu dram bytes per launch of the committed capture"
                     if traffic is not None else "no capture of the current kernel source",
                     "peak_source": f"{peak_src} copy bandwidth (hbm_gbs)"
                     if peak_src == "measured" else "fallback 6.8 TB/s"},
        "kernels": kern,
        "batched": batched,
        "served": served,
    }
    line = rounded(line)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def profiled_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when the kernel's sources changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_text_1g.txt")
    csrc = os.path.join(ROOT, "paper_2306_11070_gb300", "csrc")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        f = ln.split()
        if not f or f[0].startswith("#") or f[0] != kernel:
            continue
        h = hashlib.sha256()
        for name in f[3:]:
            with open(os.path.join(csrc, name), "rb") as fh:
                h.update(fh.read())
        return int(f[1]) if h.hexdigest()[:16] == f[2] else None
    return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline sample")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched measurement")
    ap.add_argument("--no-served", action="store_true", help="skip the served measurement")
    ap.add_argument("--no-method3", action="store_true",
                    help="skip the Method 3 (block-sorting transform) measurement")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
