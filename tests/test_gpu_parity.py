"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer work, so the bar is bit-exact everywhere: histogram, code lengths and
codes, the whole stream (header, chunk offsets, payload), decoded bytes and
the device status of every error path.  Sizes span several 4096-symbol
encode tiles, several chunks and ragged tails; the full-size workloads are
checked on their whole histogram, codebook and offset table, on sampled
chunk payloads, and by the round trip.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2306_11070_gb300 as hg
from paper_2306_11070_gb300 import build as nvbuild

pytestmark = pytest.mark.gpu
MiB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _lib():
    nvbuild.build()
    hg.lib()
    torch.cuda.init()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_codebook(x_np):
    d = dev(x_np) if x_np.size else torch.empty(0, dtype=torch.uint8, device="cuda")
    h = hg.huff_histogram(d)
    cb, st = hg.huff_build_codebook(h)
    torch.cuda.synchronize()
    return d, h, cb, int(st.item())


def gpu_encode(d, cb, cs=16384, cap=None):
    n = d.numel()
    out_cap = hg.huff_max_stream_size(n, cs) if cap is None else cap
    out = torch.zeros(max(out_cap, 16), dtype=torch.uint8, device="cuda")
    o, ob, st = hg.huff_encode(d, cb, cs, d_out=out, out_cap=out_cap)
    torch.cuda.synchronize()
    return o, int(ob.item()), int(st.item())


def gpu_decode(stream_np_or_t, cap=None):
    s = stream_np_or_t if isinstance(stream_np_or_t, torch.Tensor) else dev(stream_np_or_t)
    if s.numel() == 0:
        s = torch.zeros(16, dtype=torch.uint8, device="cuda")[:0]
    nbytes = s.numel()
    buf = torch.zeros(max(nbytes, 16), dtype=torch.uint8, device="cuda")
    buf[:nbytes] = s
    n_hdr = int.from_bytes(bytes(s[256:264].cpu().numpy()), "little") if nbytes >= 264 else 0
    out_cap = min(n_hdr, 1 << 33) if cap is None else cap
    out = torch.zeros(max(out_cap, 16), dtype=torch.uint8, device="cuda")
    o, n, st = hg.huff_decode(buf, nbytes, d_out=out, out_cap=out_cap)
    torch.cuda.synchronize()
    return o, int(n.item()), int(st.item())


# ------------------------------------------------------------------ inputs
GENS = {
    "zipf": lambda n, s: synth.zipf_ascii(n, s),
    "text": lambda n, s: synth.text(n, s),
    "uniform": lambda n, s: synth.uniform(n, s),
    "geometric": lambda n, s: synth.geometric(n, s),
    "single": lambda n, s: synth.single(n, 0x61),
    "skew4": lambda n, s: synth.geometric_p(n, s, 0.75),
}
SIZES = [1, 2, 15, 16, 17, 31, 32, 33, 4095, 4096, 4097, 16383, 16384, 16385,
         3 * 16384 + 4096 * 2 + 123, 100003, MiB + 7]


# ------------------------------------------------------------------ histogram
@pytest.mark.parametrize("gen", list(GENS))
@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 4096 * 16 + 5, 3 * MiB + 11])
def test_histogram(gen, n):
    x = GENS[gen](n, 7)
    d = dev(x) if n else torch.empty(0, dtype=torch.uint8, device="cuda")
    h = hg.huff_histogram(d).cpu().numpy().view(np.uint64)
    assert np.array_equal(h, oracle.histogram(x))


# ------------------------------------------------------------------ codebook
def _hists(count, seed):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        k = int(rng.integers(1, 257))
        syms = rng.choice(256, size=k, replace=False)
        kind = int(rng.integers(0, 3))
        if kind == 0:
            w = rng.integers(1, 4, size=k)
        elif kind == 1:
            w = rng.integers(1, 1 << 40, size=k)
        else:
            w = np.floor(1e5 * rng.pareto(1.1, size=k)).astype(np.int64) + 1
        h = np.zeros(256, dtype=np.uint64)
        h[syms] = w.astype(np.uint64)
        yield h


def _gpu_cb_from_hist(h):
    dh = torch.from_numpy(h.view(np.int64)).cuda()
    cb, st = hg.huff_build_codebook(dh)
    torch.cuda.synchronize()
    return hg.parse_codebook(cb), int(st.item())


def test_codebook_random_histograms():
    for h in _hists(400, 3):
        (ln, code, nsym, mx), st = _gpu_cb_from_hist(h)
        ost, oln = oracle.code_lengths(h)
        assert st == ost
        if ost != oracle.OK:
            continue
        assert np.array_equal(ln, oln)
        assert np.array_equal(code, oracle.canonical_codes(oln))
        assert nsym == int((h > 0).sum()) and mx == int(oln.max())


def test_codebook_weights_of_2_56_and_more():
    """Weights the packed (weight, byte) key cannot hold take the two-part
    comparison: equal results, ties included (sums stay below 2^64)."""
    rng = np.random.default_rng(11)
    for t in range(60):
        k = int(rng.integers(2, 33))
        syms = rng.choice(256, size=k, replace=False)
        if t % 3 == 0:
            w = rng.integers(1 << 56, 1 << 58, size=k, dtype=np.uint64)
        elif t % 3 == 1:  # ties among huge weights
            w = (np.uint64(1) << np.uint64(56)) * rng.integers(1, 4, size=k).astype(np.uint64)
        else:  # one huge weight among small ones
            w = rng.integers(1, 1000, size=k).astype(np.uint64)
            w[0] = np.uint64(1) << np.uint64(57)
        h = np.zeros(256, dtype=np.uint64)
        h[syms] = w
        (ln, code, nsym, mx), st = _gpu_cb_from_hist(h)
        ost, oln = oracle.code_lengths(h)
        assert st == ost == oracle.OK
        assert np.array_equal(ln, oln)
        assert np.array_equal(code, oracle.canonical_codes(oln))


def test_codebook_fibonacci_boundary():
    f = [1, 1]
    while len(f) < 34:
        f.append(f[-1] + f[-2])
    h = np.zeros(256, dtype=np.uint64)
    h[:33] = f[:33]
    (ln, code, nsym, mx), st = _gpu_cb_from_hist(h)
    ost, oln = oracle.code_lengths(h)
    assert st == 0 and ost == 0 and mx == 32 and np.array_equal(ln, oln)
    assert np.array_equal(code, oracle.canonical_codes(oln))
    h = np.zeros(256, dtype=np.uint64)
    h[:34] = f[:34]
    (_, _, _, _), st = _gpu_cb_from_hist(h)
    assert st == hg.HUFF_ERR_CODE_TOO_LONG == oracle.code_lengths(h)[0]


def test_codebook_empty_and_single():
    (ln, code, nsym, mx), st = _gpu_cb_from_hist(np.zeros(256, dtype=np.uint64))
    assert st == 0 and not ln.any() and nsym == 0 and mx == 0
    h = np.zeros(256, dtype=np.uint64)
    h[77] = 5
    (ln, code, nsym, mx), st = _gpu_cb_from_hist(h)
    assert st == 0 and ln[77] == 1 and code[77] == 0 and nsym == 1 and mx == 1


# ------------------------------------------------------------------ encode / decode
def _check_roundtrip(x, cs=16384):
    d, h, cb, st = gpu_codebook(x)
    assert st == 0
    ln = hg.parse_codebook(cb)[0]
    ost, oln = oracle.code_lengths(oracle.histogram(x))
    assert np.array_equal(ln, oln)
    out, nbytes, st = gpu_encode(d, cb, cs)
    ost, ref, need = oracle.encode(x, oln, cs)
    assert st == 0 and ost == 0
    assert nbytes == need
    got = out[:nbytes].cpu().numpy()
    assert np.array_equal(got, ref)
    back, n, st = gpu_decode(out[:nbytes])
    assert st == 0 and n == x.size
    assert np.array_equal(back[:n].cpu().numpy(), x)


@pytest.mark.parametrize("gen", list(GENS))
@pytest.mark.parametrize("n", SIZES)
def test_stream_bit_exact_and_round_trip(gen, n):
    _check_roundtrip(GENS[gen](n, 11 + n % 97))


@pytest.mark.parametrize("k", [2, 3, 5, 20, 100, 180])
def test_small_alphabets_every_code_group(k):
    """k equally likely byte values (longest codes of 1, 2, 3, 5, 7 and 8
    bits): the encoder's multiply-add groups of 16, 8, 4 and 3 codes, whole
    stream against the oracle over several inner units and a ragged tail."""
    rng = np.random.default_rng(k)
    vals = rng.choice(256, k, replace=False).astype(np.uint8)
    x = vals[rng.integers(0, k, (1 << 20) + 12345)]
    _check_roundtrip(x)


def test_encode_with_uncovered_bytes():
    """Against huff_encode's precondition, code input with bytes that have no
    code (a text codebook, bytes from 128 up planted): the stream is
    unspecified, but the kernels must stay inside their buffers, those bytes
    must count zero bits in the unit offsets and in the coder alike (the
    stream size says so), and the result must be repeatable."""
    n = (2 << 20) + 777
    x = synth.text(n, 31)
    d, h, cb, st = gpu_codebook(x)
    assert st == 0
    ln = hg.parse_codebook(cb)[0]
    assert ln[128:].sum() == 0 and 0 < ln.max() <= 11
    y = x.copy()
    rng = np.random.default_rng(5)
    idx = rng.choice(n, 5000, replace=False)
    y[idx] = rng.integers(128, 256, idx.size, dtype=np.uint8)
    dy = dev(y)
    a1, nb1, st1 = gpu_encode(dy, cb)
    a2, nb2, st2 = gpu_encode(dy, cb)
    assert st1 == 0 and st2 == 0 and nb1 == nb2
    bits = int(ln.astype(np.int64)[y].sum())
    chunks = (n + 16383) // 16384
    assert nb1 == 272 + 8 * chunks + 4 * ((bits + 31) // 32)
    assert torch.equal(a1[:nb1], a2[:nb2])
    # and the covered input still matches the oracle byte for byte
    _check_roundtrip(x)


@pytest.mark.parametrize("shift", [16, 32])
def test_decode_into_offset_output(shift):
    """The decoder stores whole 32-byte groups only where a chunk's output is
    32-byte aligned; an output 16 bytes past an aligned address takes the
    16-byte path in every chunk (and 32 bytes the wide one), same bytes."""
    n = (1 << 20) + 12345
    x = synth.text(n, 21)
    d, h, cb, st = gpu_codebook(x)
    assert st == 0
    out, nbytes, st = gpu_encode(d, cb, 16384)
    assert st == 0
    buf = torch.full((n + 64,), 0xA5, dtype=torch.uint8, device="cuda")
    view = buf[shift:shift + n]
    _, dn, dst = hg.huff_decode(out[:nbytes], d_out=view, out_cap=n)
    torch.cuda.synchronize()
    assert int(dst.item()) == 0 and int(dn.item()) == n
    got = buf.cpu().numpy()
    assert np.array_equal(got[shift:shift + n], x)
    assert (got[:shift] == 0xA5).all() and (got[shift + n:] == 0xA5).all()


@pytest.mark.parametrize("cs", [16, 32, 48, 1024, 4096, 4112, 65536])
def test_chunk_sizes(cs):
    _check_roundtrip(synth.text(5 * 4096 + 77, 5), cs)
    _check_roundtrip(synth.zipf_ascii(3 * 65536 + 5, 6), cs)


@pytest.mark.parametrize("cs", [1 << 20, 1 << 24])
def test_largest_chunks(cs):
    # one or two chunks of up to the largest size: the decoder splits each
    # into 32 self-synchronising sub-segments of up to 512 Ki symbols
    _check_roundtrip(synth.text((1 << 24) + 12345, 8), cs)


def test_empty_input():
    x = np.zeros(0, dtype=np.uint8)
    d, h, cb, st = gpu_codebook(x)
    out, nbytes, st = gpu_encode(d, cb)
    ost, ref, need = oracle.encode(x, np.zeros(256, np.uint8))
    assert st == 0 and nbytes == need == 272
    assert np.array_equal(out[:nbytes].cpu().numpy(), ref)
    back, n, st = gpu_decode(out[:nbytes])
    assert st == 0 and n == 0


@pytest.mark.parametrize("k", [13, 17, 24, 25, 26, 28, 30, 32])
def test_long_codes(k):
    # Fibonacci counts give the deepest trees: codes up to k-1 bits (24 is
    # the longest the fast encoder takes, 12 the longest the decode table holds)
    f = [1, 1]
    while len(f) < k:
        f.append(f[-1] + f[-2])
    x = synth.counted(f[:k], seed=k)
    _check_roundtrip(x)
    _check_roundtrip(x, cs=64)


def test_oracle_stream_decodes_on_gpu():
    x = synth.text(200001, 3)
    st, s = oracle.compress(x, 1024)
    back, n, st = gpu_decode(s)
    assert st == 0 and np.array_equal(back[:n].cpu().numpy(), x)


def test_compress_matches_oracle():
    x = synth.zipf_ascii(MiB, 0)
    got = hg.compress(dev(x)).cpu().numpy()
    st, ref = oracle.compress(x)
    assert np.array_equal(got, ref)


# ------------------------------------------------------------------ error paths
def _corruptions():
    x = synth.text(40000, 21)
    st, s = oracle.compress(x, 1024)
    chunks = (x.size + 1023) // 1024
    o = 272 + 8
    cases = {"short_header": s[:271].copy()}
    t = s.copy(); t[264:268] = np.frombuffer((1000).to_bytes(4, "little"), np.uint8)
    cases["bad_chunk_size"] = t
    t = s.copy(); t[ord("e")] = max(1, int(t[ord("e")]) - 1); cases["kraft_over"] = t
    t = s.copy(); t[ord("e")] = int(t[ord("e")]) + 1; cases["kraft_under"] = t
    t = s.copy(); t[268] ^= 1; cases["max_len_field"] = t
    t = s.copy(); t[0] = 33; cases["len_above_32"] = t
    t = s.copy(); t[256:264] = np.frombuffer((10**12).to_bytes(8, "little"), np.uint8)
    cases["table_too_big"] = t
    t = s.copy()
    t[o:o + 8] = np.frombuffer((int.from_bytes(bytes(t[o:o + 8]), "little") + 1)
                               .to_bytes(8, "little"), np.uint8)
    cases["offset_shifted"] = t
    t = s.copy(); t[272:280] = np.frombuffer((5).to_bytes(8, "little"), np.uint8)
    cases["first_offset"] = t
    t = s.copy(); t[o:o + 8], t[o + 8:o + 16] = t[o + 8:o + 16].copy(), t[o:o + 8].copy()
    cases["offsets_swapped"] = t
    cases["payload_cut"] = s[:272 + 8 * chunks + 8].copy()
    t = s.copy(); t[-1] ^= 0xFF; cases["last_word_flipped"] = t
    t = s.copy(); t[-9] ^= 0x10; cases["payload_bit"] = t
    x1 = synth.single(100, 0x61)
    st, s1 = oracle.compress(x1)
    t = s1.copy(); t[-1] |= 0x80; cases["single_symbol_one_bit"] = t
    return cases


@pytest.mark.parametrize("name", list(_corruptions()))
def test_corrupt_stream_status_matches_oracle(name):
    s = _corruptions()[name]
    ost, oback, on = oracle.decode(s, cap=1 << 20)
    back, n, st = gpu_decode(s, cap=1 << 20)
    assert st == ost, (name, st, ost)
    if ost == 0:  # a change the format cannot detect: both sides decode the same bytes
        assert n == on and np.array_equal(back[:n].cpu().numpy(), oback)


def test_capacity_statuses():
    x = synth.text(100000, 4)
    d, h, cb, st = gpu_codebook(x)
    ln = hg.parse_codebook(cb)[0]
    ost, ref, need = oracle.encode(x, ln)
    out, nbytes, st = gpu_encode(d, cb, cap=need - 1)
    assert st == hg.HUFF_ERR_CAPACITY and nbytes == need
    out, nbytes, st = gpu_encode(d, cb, cap=need)
    assert st == 0 and np.array_equal(out[:need].cpu().numpy(), ref)
    out, nbytes, st = gpu_encode(d, cb, cap=200)
    assert st == hg.HUFF_ERR_CAPACITY
    _, n, st = gpu_decode(ref, cap=x.size - 1)
    assert st == hg.HUFF_ERR_CAPACITY == oracle.decode(ref, cap=x.size - 1)[0] and n == x.size


def test_chain_stops_after_error():
    f = [1, 1]
    while len(f) < 34:
        f.append(f[-1] + f[-2])
    x = synth.counted(f, seed=1)
    d = dev(x)
    out, ob, st = hg.huff_compress(d)
    torch.cuda.synchronize()
    assert int(st.item()) == hg.HUFF_ERR_CODE_TOO_LONG
    assert int(ob.item()) == 0  # the encoder never ran


def test_host_argument_errors():
    d = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(hg.HuffError) as e:
        hg.huff_histogram(d[1:17])  # misaligned
    assert e.value.status == hg.HUFF_ERR_INVALID_ARG
    with pytest.raises(hg.HuffError):
        hg.huff_encode(d, torch.zeros(1288, dtype=torch.uint8, device="cuda"), chunk_symbols=100)


# ------------------------------------------------------------------ full-size workloads
def _full_size_check(x, cs=16384, samples=24):
    """Whole histogram, codebook and offset table against the oracle; sampled
    chunk payloads against the oracle's packing (a fast first failure); then
    the entire stream byte for byte against the oracle's encoder; round trip
    on the GPU."""
    d, h, cb, st = gpu_codebook(x)
    assert np.array_equal(h.cpu().numpy().view(np.uint64), oracle.histogram(x))
    ost, oln = oracle.code_lengths(oracle.histogram(x))
    assert st == ost
    if ost != 0:
        return
    ln, code, nsym, mx = hg.parse_codebook(cb)
    assert np.array_equal(ln, oln) and np.array_equal(code, oracle.canonical_codes(oln))
    out, nbytes, st = gpu_encode(d, cb, cs)
    assert st == 0
    chunks = (x.size + cs - 1) // cs
    st, ooff, total = oracle.chunk_offsets(x, oln, cs)
    assert nbytes == 272 + 8 * chunks + 4 * ((total + 31) // 32)
    head = out[:272 + 8 * chunks].cpu().numpy()
    assert np.array_equal(head[:256], oln)
    off = head[272:].view("<u8")
    assert np.array_equal(off, ooff)
    rng = np.random.default_rng(1)
    pick = sorted(set([0, chunks - 1] + list(rng.integers(0, chunks, size=samples))))
    pay0 = 272 + 8 * chunks
    for c in pick:
        st, w, nb = oracle.pack_bits(x[c * cs:(c + 1) * cs], oln)
        a = int(ooff[c])
        wlo, whi = a // 32, (a + nb + 31) // 32
        gw = out[pay0 + 4 * wlo:pay0 + 4 * whi].cpu().numpy().view("<u4")
        gb = np.unpackbits(gw.astype(">u4").view(np.uint8))[a - 32 * wlo:a - 32 * wlo + nb]
        ob = np.unpackbits(w.astype(">u4").view(np.uint8))[:nb]
        assert np.array_equal(gb, ob), c
    # padding bits after the last code are zero
    lastw = int(out[nbytes - 4:nbytes].cpu().numpy().view("<u4")[0])
    pad = (32 - total % 32) % 32
    assert lastw & ((1 << pad) - 1) == 0
    # the whole stream, byte for byte, against the oracle's encoder
    ost, ref, need = oracle.encode(x, oln, cs)
    assert ost == oracle.OK and need == nbytes
    got = out[:nbytes].cpu().numpy()
    if not np.array_equal(got, ref):
        bad = np.flatnonzero(got != ref)
        raise AssertionError(f"{bad.size} stream bytes differ from the oracle, first at {bad[0]}")
    del got, ref
    back, n, st = gpu_decode(out[:nbytes])
    assert st == 0 and n == x.size
    assert torch.equal(back[:n], d)


@pytest.mark.parametrize("name", ["zipf_ascii_1m", "text_64m", "text_1g", "uniform_1g",
                                  "geometric_1g", "single_1g"])
def test_full_size_workloads(name):
    x = synth.make(name)
    _full_size_check(x)


# ------------------------------------------------------------------ length-limited codebook
def _gpu_cb_limited(h, limit):
    d = torch.from_numpy(np.asarray(h, dtype=np.int64)).cuda()
    cb, st = hg.huff_build_codebook_limited(d, limit)
    torch.cuda.synchronize()
    return hg.parse_codebook(cb), int(st.item())


def test_limited_codebook_matches_oracle():
    rng = np.random.default_rng(23)
    cases = 0
    for trial in range(60):
        k = int(rng.integers(2, 257))
        h = np.zeros(256, dtype=np.uint64)
        syms = rng.choice(256, size=k, replace=False)
        kind = trial % 3
        if kind == 0:
            h[syms] = rng.integers(1, 5, size=k)
        elif kind == 1:
            h[syms] = np.floor(1e6 * rng.pareto(1.2, size=k)).astype(np.uint64) + 1
        else:
            h[syms] = (1 << np.minimum(np.arange(k), 40)).astype(np.uint64)  # deep trees
        for limit in sorted({max(1, int(np.ceil(np.log2(k)))), 9, 12, 16, 32}):
            (ln, code, nsym, mx), st = _gpu_cb_limited(h, limit)
            ost, oln = oracle.code_lengths_limited(h, limit)
            assert st == ost, (trial, limit)
            if ost == 0:
                assert np.array_equal(ln, oln), (trial, limit)
                assert np.array_equal(code, oracle.canonical_codes(oln))
                assert mx == int(oln.max()) <= limit
                cases += 1
    assert cases > 100


def test_limited_codebook_fibonacci_and_errors():
    f = [1, 1]
    while len(f) < 34:
        f.append(f[-1] + f[-2])
    h = np.zeros(256, dtype=np.uint64)
    h[:34] = f
    for limit in (6, 12, 32):
        (ln, code, nsym, mx), st = _gpu_cb_limited(h, limit)
        ost, oln = oracle.code_lengths_limited(h, limit)
        assert st == ost == 0 and np.array_equal(ln, oln) and mx == limit
    (_, _, _, _), st = _gpu_cb_limited(h, 5)                 # 34 > 2^5 bytes
    assert st == hg.HUFF_ERR_CODE_TOO_LONG == oracle.code_lengths_limited(h, 5)[0]
    d = torch.zeros(256, dtype=torch.int64, device="cuda")
    for bad in (0, 33):
        with pytest.raises(hg.HuffError):
            hg.huff_build_codebook_limited(d, bad)


@pytest.mark.parametrize("gen", ["geometric", "text", "uniform"])
def test_limited_stream_round_trip(gen):
    # 12-bit limited codes: every code fits the decoder's table
    x = GENS[gen](300007, 29)
    d = dev(x)
    h = hg.huff_histogram(d)
    cb, st = hg.huff_build_codebook_limited(h, 12)
    out, ob, st = hg.huff_encode(d, cb, d_status=st)
    torch.cuda.synchronize()
    nb = int(ob.item())
    ost, oln = oracle.code_lengths_limited(oracle.histogram(x), 12)
    ost, ref, need = oracle.encode(x, oln)
    assert int(st.item()) == 0 and ost == 0 and nb == need
    assert np.array_equal(out[:nb].cpu().numpy(), ref)
    back, n, st = gpu_decode(out[:nb])
    assert st == 0 and np.array_equal(back[:n].cpu().numpy(), x)


def test_limited_full_size_geometric():
    # the length-limited row on 64 MiB of the geometric stress input (its
    # Huffman codes run to ~29 bits): the whole 12-bit stream equals the
    # oracle's and decodes back
    x = synth.geometric(64 << 20, 41)
    d = dev(x)
    h = hg.huff_histogram(d)
    cb, st = hg.huff_build_codebook_limited(h, 12)
    out, ob, st = hg.huff_encode(d, cb, d_status=st)
    torch.cuda.synchronize()
    nb = int(ob.item())
    ost, oln = oracle.code_lengths_limited(oracle.histogram(x), 12)
    assert max(int(v) for v in oln) == 12
    ost, ref, need = oracle.encode(x, oln)
    assert int(st.item()) == 0 and ost == 0 and nb == need
    assert np.array_equal(out[:nb].cpu().numpy(), ref)
    back, n, st = gpu_decode(out[:nb])
    assert st == 0 and n == x.size and torch.equal(back[:n], d)
