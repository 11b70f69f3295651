"""GPU parity of the batched engine: every buffer of a batch against the CPU
oracle, byte for byte, and the same buffer compressed alone.

The batch mixes sizes (empty, a few bytes, below and across 16 KiB units and
16384-symbol chunks, up to ~0.3 MiB) and distributions, includes a buffer
whose tree is deeper than 32 bits (its status must be CODE_TOO_LONG while
its neighbours succeed) and, for decompression, corrupt streams whose
statuses must match the oracle's.  Each plan runs twice to check that the
runs are repeatable.
"""
import time

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2306_11070_gb300 as hg
from paper_2306_11070_gb300 import build as nvbuild

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    nvbuild.build()
    hg.lib()


def _fib(k):
    f = [1, 1]
    while len(f) < k:
        f.append(f[-1] + f[-2])
    return f[:k]


def _mixed_inputs():
    gens = [lambda n, s: synth.text(n, s), lambda n, s: synth.zipf_ascii(n, s),
            lambda n, s: synth.uniform(n, s), lambda n, s: synth.geometric(n, s),
            lambda n, s: synth.single(n, 0x41 + s % 20)]
    sizes = [0, 1, 7, 16, 1000, 1024, 4097, 16383, 16384, 16385, 40000, 131072, 300001]
    out = []
    for i, n in enumerate(sizes * 2):
        out.append(gens[i % len(gens)](n, 100 + i))
    out.append(synth.counted(_fib(30), 7))    # 29-bit codes: the wide path
    out.append(synth.counted(_fib(34), 8))    # 33-bit tree: error
    return out


def _dev(x):
    t = torch.zeros(max(x.size, 16), dtype=torch.uint8, device="cuda")
    if x.size:
        t[:x.size] = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return t[:x.size] if x.size else t[:0]


def _compress_batch(xs, cs=16384, params=None):
    ins = [_dev(x) for x in xs]
    outs = [torch.zeros(hg.huff_max_stream_size(x.size, cs), dtype=torch.uint8, device="cuda")
            for x in xs]
    if params is None:
        params = hg.huff_batch_default_params()
        params.chunk_symbols = cs
    plan = hg.BatchPlan(ins, outs, hg.HUFF_BATCH_COMPRESS, params)
    return plan, ins, outs


@pytest.mark.parametrize("cs", [16384, 4096])
def test_batch_compress_matches_oracle_and_single(cs):
    xs = _mixed_inputs()
    plan, ins, outs = _compress_batch(xs, cs)
    for rep in range(2):
        plan.run()
        torch.cuda.synchronize()
        st = plan.status.cpu().numpy()
        nb = plan.out_bytes.cpu().numpy()
        for i, x in enumerate(xs):
            ost, ref = oracle.compress(x, cs)
            assert st[i] == ost, (rep, i, st[i], ost)
            if ost != 0:
                continue
            got = outs[i][:nb[i]].cpu().numpy()
            assert nb[i] == ref.size, (i, nb[i], ref.size)
            assert np.array_equal(got, ref), i
    # and each buffer alone through huff_compress
    for i, x in enumerate(xs[:8]):
        if x.size:
            alone = hg.compress(_dev(x), cs).cpu().numpy()
            assert np.array_equal(alone, outs[i][:alone.size].cpu().numpy())
    info = plan.info()
    assert info["grid"] > 0
    plan.close()


def test_batch_decompress_round_trip_and_corruption():
    xs = [x for x in _mixed_inputs()[:-1]]  # drop the too-long one
    streams = []
    for i, x in enumerate(xs):
        st, s = oracle.compress(x, 1024 if i % 3 == 0 else 16384)
        assert st == 0
        streams.append(s)
    # two corrupt streams: a shifted chunk offset and a Kraft violation
    bad1 = streams[10].copy()
    if (bad1.size - 272) // 8 > 1:
        o = 272 + 8
        bad1[o:o + 8] = np.frombuffer((int.from_bytes(bytes(bad1[o:o + 8]), "little") + 1)
                                      .to_bytes(8, "little"), np.uint8)
    bad2 = streams[4].copy()
    bad2[ord("e")] = 1
    streams += [bad1, bad2]
    xs += [xs[10], xs[4]]
    ins = [_dev(s) for s in streams]
    outs = [torch.zeros(max(x.size, 16), dtype=torch.uint8, device="cuda") for x in xs]
    params = hg.huff_batch_default_params()
    plan = hg.BatchPlan(ins, outs, hg.HUFF_BATCH_DECOMPRESS, params)
    for rep in range(2):
        for o in outs:
            o.zero_()
        plan.run()
        torch.cuda.synchronize()
        st = plan.status.cpu().numpy()
        nb = plan.out_bytes.cpu().numpy()
        for i, (s, x) in enumerate(zip(streams, xs)):
            ost, back, on = oracle.decode(s, cap=outs[i].numel())
            assert st[i] == ost, (rep, i, st[i], ost)
            if ost == 0:
                assert nb[i] == x.size
                assert np.array_equal(outs[i][:x.size].cpu().numpy(), back)
    plan.close()


def test_batch_many_small_buffers_one_chunk_each():
    xs = [synth.text(int(n), 500 + i) for i, n in
          enumerate(synth.log_uniform_sizes(300, seed=9, lo=16, hi=20000))]
    plan, ins, outs = _compress_batch(xs)
    plan.run()
    torch.cuda.synchronize()
    st = plan.status.cpu().numpy()
    nb = plan.out_bytes.cpu().numpy()
    assert (st == 0).all()
    streams = [outs[i][:nb[i]].clone() for i in range(len(xs))]
    for i in range(0, len(xs), 37):
        ost, ref = oracle.compress(xs[i])
        assert np.array_equal(streams[i].cpu().numpy(), ref)
    # round trip through the batched decoder
    dec = [torch.zeros(max(x.size, 16), dtype=torch.uint8, device="cuda") for x in xs]
    dplan = hg.BatchPlan(streams, dec, hg.HUFF_BATCH_DECOMPRESS)
    dplan.run()
    torch.cuda.synchronize()
    assert (dplan.status.cpu().numpy() == 0).all()
    for i, x in enumerate(xs):
        assert np.array_equal(dec[i][:x.size].cpu().numpy(), x), i
    plan.close()
    dplan.close()


@pytest.mark.parametrize("ctas", [0, 1])
def test_batch_few_buffers_and_many_items_per_worker(ctas):
    """Batches far below one wave of items (1-3 buffers) and one buffer with
    many items per worker (6 MiB at one CTA per SM): the ticket loops take
    their next ticket late in the first case and early in the second; every
    stream and every decoded byte must match the oracle."""
    cases = [[synth.text(70000, 41)],
             [synth.text(5, 42), synth.uniform(40000, 43)],
             [synth.geometric(33000, 44), synth.text(1, 45), synth.zipf_ascii(250000, 46)],
             [synth.text(6 << 20, 47)]]
    for xs in cases:
        params = hg.huff_batch_default_params()
        params.chunk_symbols = 4096
        params.ctas_per_sm = ctas
        plan, ins, outs = _compress_batch(xs, 4096, params)
        plan.run()
        torch.cuda.synchronize()
        st = plan.status.cpu().numpy()
        nb = plan.out_bytes.cpu().numpy()
        assert (st == 0).all()
        streams = []
        for i, x in enumerate(xs):
            ost, ref = oracle.compress(x, 4096)
            got = outs[i][:nb[i]]
            assert ost == 0 and np.array_equal(got.cpu().numpy(), ref), i
            streams.append(got.clone())
        for lanes in (1, 64):
            dec = [torch.zeros(max(x.size, 16), dtype=torch.uint8, device="cuda") for x in xs]
            dp = hg.huff_batch_default_params()
            dp.ctas_per_sm = ctas
            dp.decode_lanes = lanes
            dplan = hg.BatchPlan(streams, dec, hg.HUFF_BATCH_DECOMPRESS, dp)
            dplan.run()
            torch.cuda.synchronize()
            assert (dplan.status.cpu().numpy() == 0).all()
            assert (dplan.out_bytes.cpu().numpy() == [x.size for x in xs]).all()
            for i, x in enumerate(xs):
                assert np.array_equal(dec[i][:x.size].cpu().numpy(), x), (lanes, i)
            dplan.close()
        plan.close()


def test_barrier_timeout_reports_status_and_context_survives():
    # The test hook makes every grid barrier wait for one CTA more than the
    # grid holds: the bounded spins run out (no fault, no hang), every buffer
    # reports HUFF_ERR_TIMEOUT, and the GPU context stays usable.
    xs = [synth.text(20000 + 1000 * i, 900 + i) for i in range(8)]
    params = hg.huff_batch_default_params()
    params.barrier_extra = 1
    plan, ins, outs = _compress_batch(xs, params=params)
    t0 = time.time()
    plan.run()
    torch.cuda.synchronize()
    assert time.time() - t0 < 120
    assert (plan.status.cpu().numpy() == hg.HUFF_ERR_TIMEOUT).all()
    plan.close()
    plan2, _, outs2 = _compress_batch(xs)
    plan2.run()
    torch.cuda.synchronize()
    st = plan2.status.cpu().numpy()
    nb = plan2.out_bytes.cpu().numpy()
    assert (st == 0).all()
    for i in (0, 7):
        ost, ref = oracle.compress(xs[i])
        assert np.array_equal(outs2[i][:nb[i]].cpu().numpy(), ref)
    plan2.close()


def test_autotune_decompress_and_round_trip_compress():
    xs = [synth.text(int(n), 700 + i) for i, n in
          enumerate(synth.log_uniform_sizes(96, seed=11, lo=1024, hi=1 << 20))]
    # compress, tuned by compress + decompress time; outputs hold the chosen
    # setting's streams afterwards
    plan, ins, outs = _compress_batch(xs, cs=4096)  # outputs sized for either chunk size
    base = hg.huff_batch_default_params()
    best = plan.autotune(base, flags=hg.HUFF_TUNE_ROUND_TRIP)
    assert best.chunk_symbols in (16384, 4096)
    assert best.decode_lanes in (32, 64, 128, 256)
    plan.close()
    plan2, _, outs2 = _compress_batch(xs, cs=best.chunk_symbols, params=best)
    plan2.run()
    torch.cuda.synchronize()
    nb = plan2.out_bytes.cpu().numpy()
    assert (plan2.status.cpu().numpy() == 0).all()
    for i in range(0, len(xs), 7):
        ost, ref = oracle.compress(xs[i], best.chunk_symbols)
        assert np.array_equal(outs2[i][:nb[i]].cpu().numpy(), ref), i
    # decompress, tuned on those streams; a second call is served from cache
    streams = [outs2[i][:nb[i]].clone() for i in range(len(xs))]
    dec = [torch.zeros(max(x.size, 16), dtype=torch.uint8, device="cuda") for x in xs]
    dplan = hg.BatchPlan(streams, dec, hg.HUFF_BATCH_DECOMPRESS)
    dbest = dplan.autotune()
    t0 = time.time()
    dbest2 = dplan.autotune()
    assert time.time() - t0 < 0.05
    assert (dbest2.decode_lanes, dbest2.ctas_per_sm) == (dbest.decode_lanes, dbest.ctas_per_sm)
    dplan.close()
    tuned = hg.BatchPlan(streams, dec, hg.HUFF_BATCH_DECOMPRESS, dbest)
    tuned.run()
    torch.cuda.synchronize()
    assert (tuned.status.cpu().numpy() == 0).all()
    for i, x in enumerate(xs):
        assert np.array_equal(dec[i][:x.size].cpu().numpy(), x), i
    tuned.close()
    plan2.close()


_TUNE_CHILD = r"""
import json, sys
sys.path.insert(0, "tests")
import numpy as np, torch, synth
import paper_2306_11070_gb300 as hg
xs = [synth.text(int(n), 900 + i) for i, n in
      enumerate(synth.log_uniform_sizes(64, seed=5, lo=4096, hi=1 << 18))]
ins = [torch.from_numpy(x).cuda() for x in xs]
outs = [torch.empty(hg.huff_max_stream_size(x.size), dtype=torch.uint8, device="cuda")
        for x in xs]
p = hg.BatchPlan(ins, outs, hg.HUFF_BATCH_COMPRESS)
p.run()
torch.cuda.synchronize()
nb = p.out_bytes.cpu().numpy()
streams = [outs[i][:nb[i]].clone() for i in range(len(xs))]
dec = [torch.empty(max(x.size, 16), dtype=torch.uint8, device="cuda") for x in xs]
d = hg.BatchPlan(streams, dec, hg.HUFF_BATCH_DECOMPRESS)
b = d.autotune()
print(json.dumps({"decode_lanes": b.decode_lanes, "ctas_per_sm": b.ctas_per_sm}))
"""


def test_autotune_cache_file_round_trip(tmp_path):
    # a first process tunes and appends a JSON line; a second one, given a
    # cache file whose entry was edited to other valid parameters, returns
    # those without tuning: the file is written and read back
    import json
    import os
    import subprocess
    import sys
    cache = tmp_path / "tune.jsonl"
    env = dict(os.environ, HUFF_TUNE_CACHE=str(cache))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r1 = subprocess.run([sys.executable, "-c", _TUNE_CHILD], cwd=root, env=env,
                        capture_output=True, text=True, timeout=600)
    assert r1.returncode == 0, r1.stderr[-2000:]
    first = json.loads(r1.stdout.strip().splitlines()[-1])
    lines = cache.read_text().splitlines()
    assert len(lines) == 1
    entry = json.loads(lines[0])  # a valid JSON object
    assert entry["op"] == hg.HUFF_BATCH_DECOMPRESS
    assert (entry["decode_lanes"], entry["ctas_per_sm"]) == (first["decode_lanes"],
                                                             first["ctas_per_sm"])
    other = 32 if entry["decode_lanes"] != 32 else 64
    entry["decode_lanes"] = other
    entry["ctas_per_sm"] = 1
    cache.write_text(json.dumps(entry) + "\n")
    r2 = subprocess.run([sys.executable, "-c", _TUNE_CHILD], cwd=root, env=env,
                        capture_output=True, text=True, timeout=600)
    assert r2.returncode == 0, r2.stderr[-2000:]
    second = json.loads(r2.stdout.strip().splitlines()[-1])
    assert (second["decode_lanes"], second["ctas_per_sm"]) == (other, 1)
    assert len(cache.read_text().splitlines()) == 1  # served from the file


def test_batched_workload_4096_buffers_matches_oracle():
    """The batched workload itself: 4096 text buffers with log-uniform sizes
    1 KiB..4 MiB (sizes seed 3) and per-buffer seeds, one plan with the
    default parameters and one with 4096-symbol chunks; every stream equals
    the oracle's compress of that buffer, and decompression gives every
    buffer back."""
    from concurrent.futures import ThreadPoolExecutor
    count = 4096
    sizes = synth.log_uniform_sizes(count, seed=3, lo=1024, hi=4 << 20)
    assert sizes.min() >= 1024 and sizes.max() <= 4 << 20
    with ThreadPoolExecutor(16) as ex:
        xs = list(ex.map(lambda i: synth.text(int(sizes[i]), synth.batch_seed(i)), range(count)))
    for cs in (16384, 4096):
        with ThreadPoolExecutor(16) as ex:
            refs = list(ex.map(lambda x: oracle.compress(x, cs), xs))
        plan, ins, outs = _compress_batch(xs, cs)
        plan.run()
        torch.cuda.synchronize()
        st = plan.status.cpu().numpy()
        nb = plan.out_bytes.cpu().numpy()
        assert (st == 0).all()
        for i in range(count):
            ost, ref = refs[i]
            assert ost == oracle.OK
            assert nb[i] == ref.size, i
            assert np.array_equal(outs[i][:ref.size].cpu().numpy(), ref), i
        streams = [outs[i][:int(nb[i])] for i in range(count)]
        decs = [torch.empty(max(x.size, 16), dtype=torch.uint8, device="cuda") for x in xs]
        dplan = hg.BatchPlan(streams, decs, hg.HUFF_BATCH_DECOMPRESS)
        dplan.run()
        torch.cuda.synchronize()
        assert (dplan.status.cpu().numpy() == 0).all()
        for i in range(count):
            assert torch.equal(decs[i][:xs[i].size], ins[i]), i
        plan.close()
        dplan.close()
        del plan, dplan, ins, outs, streams, decs
        torch.cuda.empty_cache()
