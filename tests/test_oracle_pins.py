"""Pins of the CPU oracle against facts fixed outside it.

Each test checks the oracle against something it does not compute itself:
hand-worked examples of the paper's Method 1 tree (Section III-A), the Kraft
equality of a complete prefix code, brute-force minimum weighted length,
Shannon's bounds, an independently written two-queue construction, the
Fibonacci worst case, the RFC 1951 canonical-code formula, and offsets from
per-chunk counts.  A dropped term, a wrong tie-break, a transposed bit order
or an off-by-one in the chunk table fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from golden_io import all_names, load


def _hist_of(data: bytes):
    return np.bincount(np.frombuffer(data, dtype=np.uint8), minlength=256).astype(np.uint64)


# ---------------------------------------------------------------- worked examples
@pytest.mark.parametrize("name", all_names())
def test_worked_example(name):
    g = load(name)
    x = np.frombuffer(g["input"], dtype=np.uint8)
    h = oracle.histogram(x)
    assert {int(s): int(c) for s, c in enumerate(h) if c} == g["counts"]
    st, ln = oracle.code_lengths(h)
    assert st == oracle.OK
    assert {int(s): int(v) for s, v in enumerate(ln) if v} == g["lengths"]
    code = oracle.canonical_codes(ln)
    for s, bits in g["codes"].items():
        assert format(int(code[s]), f"0{len(bits)}b") == bits
    cs = g["chunk_symbols"]
    st, stream, need = oracle.encode(x, ln, cs)
    assert st == oracle.OK and need == stream.size
    chunks = len(g["offsets"])
    assert stream.size == 272 + 8 * chunks + 4 * len(g["words"])
    hdr = stream[:272]
    assert list(hdr[:256]) == list(ln)
    assert int.from_bytes(bytes(hdr[256:264]), "little") == x.size
    assert int.from_bytes(bytes(hdr[264:268]), "little") == cs
    assert int.from_bytes(bytes(hdr[268:272]), "little") == max(g["lengths"].values())
    off = np.frombuffer(bytes(stream[272:272 + 8 * chunks]), dtype="<u8")
    assert list(off) == g["offsets"]
    words = np.frombuffer(bytes(stream[272 + 8 * chunks:]), dtype="<u4")
    assert [int(w) for w in words] == g["words"]
    st, back, n = oracle.decode(stream)
    assert st == oracle.OK and n == x.size and bytes(back) == g["input"]


def test_abracadabra_payload_bytes_little_endian():
    # word 0x4EAC9C00 stored little-endian: 00 9C AC 4E
    x = np.frombuffer(b"abracadabra", dtype=np.uint8)
    st, stream = oracle.compress(x)
    assert st == oracle.OK
    assert bytes(stream[-4:]) == bytes([0x00, 0x9C, 0xAC, 0x4E])


# ---------------------------------------------------------------- histogram
@pytest.mark.parametrize("n,seed", [(0, 1), (1, 2), (1000, 3), (123457, 4)])
def test_histogram_is_bincount(n, seed):
    x = synth.uniform(n, seed)
    h = oracle.histogram(x)
    assert np.array_equal(h, np.bincount(x, minlength=256).astype(np.uint64))
    assert int(h.sum()) == n


# ---------------------------------------------------------------- code lengths
def _random_hists(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        k = int(rng.integers(2, 257))
        syms = rng.choice(256, size=k, replace=False)
        kind = rng.integers(0, 3)
        if kind == 0:
            w = rng.integers(1, 5, size=k)  # many ties
        elif kind == 1:
            w = rng.integers(1, 10**6, size=k)
        else:
            w = np.floor(1e6 * rng.pareto(1.2, size=k)).astype(np.int64) + 1
        h = np.zeros(256, dtype=np.uint64)
        h[syms] = w.astype(np.uint64)
        out.append(h)
    return out


def test_kraft_equality():
    for h in _random_hists(300, 11):
        st, ln = oracle.code_lengths(h)
        assert st == oracle.OK
        used = ln[h > 0].astype(np.int64)
        assert np.all(used >= 1) and np.all(ln[h == 0] == 0)
        # sum 2^-len == 1 exactly, in integers
        assert sum(1 << (32 - int(v)) for v in used) == 1 << 32


def _min_cost_bruteforce(w):
    k = len(w)
    best = None
    for lens in itertools.product(range(1, k), repeat=k):
        if sum(2.0 ** -l for l in lens) <= 1.0 + 1e-12:
            c = sum(a * b for a, b in zip(w, lens))
            best = c if best is None else min(best, c)
    return best


def test_bruteforce_minimum_weighted_length():
    rng = np.random.default_rng(5)
    for trial in range(60):
        k = int(rng.integers(2, 7 if trial % 3 else 8))
        w = [int(v) for v in rng.integers(1, 50, size=k)]
        h = np.zeros(256, dtype=np.uint64)
        syms = rng.choice(256, size=k, replace=False)
        h[syms] = w
        st, ln = oracle.code_lengths(h)
        assert st == oracle.OK
        got = sum(int(h[s]) * int(ln[s]) for s in syms)
        assert got == _min_cost_bruteforce(w)


def test_shannon_bounds():
    for h in _random_hists(200, 12):
        st, ln = oracle.code_lengths(h)
        p = h[h > 0].astype(np.float64)
        p /= p.sum()
        ent = float(-(p * np.log2(p)).sum())
        avg = float((p * ln[h > 0]).sum())
        assert ent - 1e-9 <= avg < ent + 1 + 1e-9


def _two_queue_lengths(h):
    """Independent construction: leaves sorted by (weight, byte) in one queue,
    merged nodes appended to a second queue; a leaf wins a tie with a merged
    node (its id < 256 <= any merged id)."""
    leaves = sorted((int(h[s]), s) for s in range(256) if h[s] > 0)
    if len(leaves) <= 1:
        return {s: 1 for _, s in leaves}
    merged = []  # (weight, children)
    children = {}
    li = mi = 0

    def take():
        nonlocal li, mi
        if mi >= len(merged) or (li < len(leaves) and leaves[li][0] <= merged[mi][0]):
            li += 1
            return leaves[li - 1][0], ("leaf", leaves[li - 1][1])
        mi += 1
        return merged[mi - 1][0], ("node", mi - 1)

    while (len(leaves) - li) + (len(merged) - mi) > 1:
        wa, a = take()
        wb, b = take()
        children[len(merged)] = (a, b)
        merged.append((wa + wb, None))
    depth = {}
    stack = [(("node", len(merged) - 1), 0)]
    while stack:
        (kind, v), d = stack.pop()
        if kind == "leaf":
            depth[v] = d
        else:
            a, b = children[v]
            stack.append((a, d + 1))
            stack.append((b, d + 1))
    return depth


def test_two_queue_equals_heap():
    for h in _random_hists(300, 13):
        st, ln = oracle.code_lengths(h)
        ref = _two_queue_lengths(h)
        assert {s: int(ln[s]) for s in range(256) if ln[s]} == ref


def _fib(k):
    f = [1, 1]
    while len(f) < k:
        f.append(f[-1] + f[-2])
    return f[:k]


def test_fibonacci_length_boundary():
    # F1..F33 (total 9,227,464) give a chain of depth 32; F1..F34 give 33.
    h = np.zeros(256, dtype=np.uint64)
    h[:33] = _fib(33)
    assert int(h.sum()) == 9227464
    st, ln = oracle.code_lengths(h)
    assert st == oracle.OK and int(ln.max()) == 32
    h = np.zeros(256, dtype=np.uint64)
    h[:34] = _fib(34)
    assert int(h.sum()) == 14930351
    st, _ = oracle.code_lengths(h)
    assert st == oracle.ERR_CODE_TOO_LONG


def test_empty_and_single():
    st, ln = oracle.code_lengths(np.zeros(256, dtype=np.uint64))
    assert st == oracle.OK and not ln.any()
    h = np.zeros(256, dtype=np.uint64)
    h[200] = 7
    st, ln = oracle.code_lengths(h)
    assert st == oracle.OK and ln[200] == 1 and int(ln.sum()) == 1


# ---------------------------------------------------------------- canonical codes
def _deflate_codes(ln):
    """RFC 1951 section 3.2.2: bl_count, next_code, then codes in byte order."""
    bl = [0] * 33
    for v in ln:
        if v:
            bl[int(v)] += 1
    nxt = [0] * 33
    code = 0
    for bits in range(1, 33):
        code = (code + bl[bits - 1]) << 1
        nxt[bits] = code
    out = {}
    for s in range(256):
        if ln[s]:
            out[s] = nxt[int(ln[s])]
            nxt[int(ln[s])] += 1
    return out


def test_canonical_matches_rfc1951_and_is_prefix_free():
    for h in _random_hists(100, 14):
        st, ln = oracle.code_lengths(h)
        code = oracle.canonical_codes(ln)
        ref = _deflate_codes(ln)
        assert {s: int(code[s]) for s in ref} == ref
        words = [format(int(code[s]), f"0{int(ln[s])}b") for s in ref]
        srt = sorted(words)
        for a, b in zip(srt, srt[1:]):
            assert not b.startswith(a)


# ---------------------------------------------------------------- stream layout
@pytest.mark.parametrize("cs", [16, 1024, 16384])
def test_offsets_from_per_chunk_counts(cs):
    x = synth.text(100003, 7)
    st, ln = oracle.code_lengths(oracle.histogram(x))
    st, off, total = oracle.chunk_offsets(x, ln, cs)
    assert st == oracle.OK
    chunks = (x.size + cs - 1) // cs
    per = [int((np.bincount(x[c * cs:(c + 1) * cs], minlength=256) * ln).sum())
           for c in range(chunks)]
    assert list(off) == [0] + list(np.cumsum(per)[:-1])
    assert total == int((oracle.histogram(x) * ln).sum())


def test_payload_independent_of_chunk_size():
    x = synth.zipf_ascii(50001, 3)
    st, ln = oracle.code_lengths(oracle.histogram(x))
    pays = []
    for cs in (16, 48, 4096, 16384):
        st, s, _ = oracle.encode(x, ln, cs)
        chunks = (x.size + cs - 1) // cs
        pays.append(bytes(s[272 + 8 * chunks:]))
    assert all(p == pays[0] for p in pays)


def test_chunk_payload_equals_standalone_packing():
    x = synth.text(70000, 9)
    cs = 16384
    st, ln = oracle.code_lengths(oracle.histogram(x))
    st, s, _ = oracle.encode(x, ln, cs)
    chunks = (x.size + cs - 1) // cs
    off = np.frombuffer(bytes(s[272:272 + 8 * chunks]), dtype="<u8")
    words = np.frombuffer(bytes(s[272 + 8 * chunks:]), dtype="<u4")
    allbits = np.unpackbits(words.astype(">u4").view(np.uint8))
    for c in range(chunks):
        st, w, nb = oracle.pack_bits(x[c * cs:(c + 1) * cs], ln)
        mine = np.unpackbits(w.astype(">u4").view(np.uint8))[:nb]
        assert np.array_equal(allbits[int(off[c]):int(off[c]) + nb], mine)


# ---------------------------------------------------------------- round trip
def _inputs():
    cs = 16384
    sizes = [0, 1, 2, 31, 32, 33, cs - 1, cs, cs + 1, 5 * cs + 7]
    gens = [("zipf", lambda n, s: synth.zipf_ascii(n, s)),
            ("text", lambda n, s: synth.text(n, s)),
            ("uniform", lambda n, s: synth.uniform(n, s)),
            ("geo", lambda n, s: synth.geometric(n, s)),
            ("single", lambda n, s: synth.single(n, 0x61))]
    for name, g in gens:
        for i, n in enumerate(sizes):
            yield f"{name}-{n}", g(n, 100 + i)


@pytest.mark.parametrize("case", list(_inputs()), ids=lambda c: c[0])
def test_round_trip(case):
    _, x = case
    st, s = oracle.compress(x)
    assert st == oracle.OK
    assert s.size <= oracle.max_stream_size(x.size)
    st, back, n = oracle.decode(s)
    assert st == oracle.OK and n == x.size and np.array_equal(back, x)


# ---------------------------------------------------------------- errors
def _stream(n=40000, cs=1024, seed=21):
    x = synth.text(n, seed)
    st, s = oracle.compress(x, cs)
    assert st == oracle.OK
    return x, s.copy(), (n + cs - 1) // cs


def test_capacity_errors():
    x, s, _ = _stream()
    st, _, need = oracle.encode(x, s[:256], 1024, cap=s.size - 1)
    assert st == oracle.ERR_CAPACITY and need == s.size
    st, _, n = oracle.decode(s, cap=x.size - 1)
    assert st == oracle.ERR_CAPACITY and n == x.size


def test_corrupt_streams():
    x, s, chunks = _stream()
    bad = []
    bad.append(s[:271])                                   # shorter than the header
    t = s.copy(); t[264:268] = np.frombuffer((1000).to_bytes(4, "little"), np.uint8); bad.append(t)
    t = s.copy(); t[ord("e")] = max(1, int(t[ord("e")]) - 1); bad.append(t)   # Kraft sum > 1
    t = s.copy(); t[268] ^= 1; bad.append(t)               # longest-length field
    t = s.copy(); t[0] = 33; bad.append(t)                 # length above 32
    t = s.copy(); t[256:264] = np.frombuffer((10**12).to_bytes(8, "little"), np.uint8)
    bad.append(t)                                         # offset table does not fit
    o = 272 + 8
    t = s.copy(); t[o:o + 8] = np.frombuffer((int.from_bytes(bytes(t[o:o + 8]), "little") + 1)
                                             .to_bytes(8, "little"), np.uint8)
    bad.append(t)                                         # chunk 0 ends off its offset
    t = s.copy(); t[272:280] = np.frombuffer((5).to_bytes(8, "little"), np.uint8); bad.append(t)
    t = s.copy(); t[o:o + 8], t[o + 8:o + 16] = t[o + 8:o + 16].copy(), t[o:o + 8].copy()
    bad.append(t)                                         # offsets out of order
    bad.append(s[:272 + 8 * chunks + 8])                  # payload cut short
    for i, t in enumerate(bad):
        st, _, _ = oracle.decode(t, cap=x.size)
        assert st == oracle.ERR_CORRUPT, i


def test_incomplete_code_is_rejected():
    # a = "0", b = "10": Kraft sum 3/4 < 1.  The stream is otherwise well
    # formed (every code read is a valid one), so only the rule "two or more
    # codes fill the code space exactly" rejects it.
    x = np.frombuffer(b"abbaab" * 5, dtype=np.uint8)
    ln = np.zeros(256, dtype=np.uint8)
    ln[ord("a")] = 1
    ln[ord("b")] = 2
    st, s, _ = oracle.encode(x, ln, 16)
    assert st == oracle.OK
    st, _, _ = oracle.decode(s)
    assert st == oracle.ERR_CORRUPT


def test_single_symbol_stream_rejects_a_one_bit():
    x = synth.single(100, 0x61)
    st, s = oracle.compress(x)
    t = s.copy()
    t[-1] |= 0x80  # first payload bit of the only word becomes 1
    st, _, _ = oracle.decode(t)
    assert st == oracle.ERR_CORRUPT


def test_missing_symbol_is_rejected_by_encode():
    x = np.frombuffer(b"abc", dtype=np.uint8)
    ln = np.zeros(256, dtype=np.uint8)
    ln[ord("a")] = 1
    ln[ord("b")] = 1
    st, _, _ = oracle.encode(x, ln, 16384)
    assert st == oracle.ERR_INVALID_ARG


def test_entropy_of_text_workload_is_text_like():
    # the synthetic text stands in for the paper's English corpus: its
    # average code length should be in the 4-5 bit range of English text
    x = synth.text(1 << 20, 1)
    st, ln = oracle.code_lengths(oracle.histogram(x))
    avg = float((oracle.histogram(x) * ln).sum()) / x.size
    assert 4.0 < avg < 5.0
    assert math.isclose(avg, 4.52, abs_tol=0.15)


# ---------------------------------------------------------------- length-limited codes
def test_limited_hand_example():
    # weights 1,1,2,4: Huffman lengths 3,3,2,1; within 2 bits all four take 2
    h = np.zeros(256, dtype=np.uint64)
    h[:4] = [1, 1, 2, 4]
    st, ln = oracle.code_lengths_limited(h, 2)
    assert st == oracle.OK and list(ln[:4]) == [2, 2, 2, 2] and not ln[4:].any()
    st, ln = oracle.code_lengths_limited(h, 3)
    assert st == oracle.OK and list(ln[:4]) == [3, 3, 2, 1]


def _min_cost_limited(w, limit):
    k = len(w)
    best = None
    for lens in itertools.product(range(1, limit + 1), repeat=k):
        if sum(2.0 ** -l for l in lens) <= 1.0 + 1e-12:
            c = sum(a * b for a, b in zip(w, lens))
            best = c if best is None else min(best, c)
    return best


def test_limited_bruteforce_optimal():
    rng = np.random.default_rng(17)
    for trial in range(40):
        k = int(rng.integers(2, 8))
        w = [int(v) for v in rng.integers(1, 60, size=k)]
        if trial % 4 == 0:
            w = [1 << min(j, 20) for j in range(k)]  # deep trees
        h = np.zeros(256, dtype=np.uint64)
        syms = rng.choice(256, size=k, replace=False)
        h[syms] = w
        for limit in range(max(1, math.ceil(math.log2(k))), k):
            st, ln = oracle.code_lengths_limited(h, limit)
            assert st == oracle.OK
            assert int(ln.max()) <= limit and np.all(ln[h > 0] >= 1) and not ln[h == 0].any()
            got = sum(int(h[s]) * int(ln[s]) for s in syms)
            assert got == _min_cost_limited(w, limit), (w, limit)


def test_limited_complete_and_monotone():
    for h in _random_hists(120, 19):
        st, hl = oracle.code_lengths(h)
        k = int((h > 0).sum())
        lo = max(1, math.ceil(math.log2(k)))
        prev = None
        for limit in range(lo, int(hl.max()) + 2):
            st, ln = oracle.code_lengths_limited(h, limit)
            assert st == oracle.OK and int(ln.max()) <= limit
            if k >= 2:
                assert sum(1 << (32 - int(v)) for v in ln[h > 0]) == 1 << 32
            cost = int((h * ln).sum())
            assert prev is None or cost <= prev
            prev = cost
        # a limit the Huffman code already meets leaves it unchanged
        st, ln = oracle.code_lengths_limited(h, int(hl.max()))
        assert np.array_equal(ln, hl)


def test_limited_fibonacci_and_statuses():
    h = np.zeros(256, dtype=np.uint64)
    h[:34] = _fib(34)
    assert oracle.code_lengths(h)[0] == oracle.ERR_CODE_TOO_LONG
    st, ln = oracle.code_lengths_limited(h, 32)
    assert st == oracle.OK and int(ln.max()) == 32
    assert sum(1 << (32 - int(v)) for v in ln[:34]) == 1 << 32
    st, ln = oracle.code_lengths_limited(h, 12)
    assert st == oracle.OK and int(ln.max()) == 12
    h = np.zeros(256, dtype=np.uint64)
    h[:5] = 1
    assert oracle.code_lengths_limited(h, 2)[0] == oracle.ERR_CODE_TOO_LONG   # 5 > 2^2
    assert oracle.code_lengths_limited(h, 0)[0] == oracle.ERR_INVALID_ARG
    assert oracle.code_lengths_limited(h, 33)[0] == oracle.ERR_INVALID_ARG
    h = np.zeros(256, dtype=np.uint64)
    h[9] = 3
    st, ln = oracle.code_lengths_limited(h, 1)
    assert st == oracle.OK and ln[9] == 1 and int(ln.sum()) == 1
    st, ln = oracle.code_lengths_limited(np.zeros(256, dtype=np.uint64), 4)
    assert st == oracle.OK and not ln.any()


# ---------------------------------------------------------------- segmented container
def test_segmented_container_layout():
    x = np.frombuffer(b"abracadabra, the quick brown fox jumps!!", dtype=np.uint8)  # 40 bytes
    st, c = oracle.segmented_compress(x, 16)
    assert st == oracle.OK
    n, seg, count = np.frombuffer(c[:24].tobytes(), "<u8")
    assert (n, seg, count) == (40, 16, 3)
    start = list(np.frombuffer(c[24:56].tobytes(), "<u8"))
    assert start[0] == 64 and all(s % 16 == 0 for s in start[:3]) and start[3] == c.size
    assert not c[56:64].any()
    for i in range(3):
        seg_bytes = x[16 * i:16 * (i + 1)]
        ost, alone = oracle.compress(seg_bytes)
        assert np.array_equal(c[start[i]:start[i] + alone.size], alone)   # its own codebook
        assert not c[start[i] + alone.size:start[i + 1]].any()
        st2, back, m = oracle.decode(c[start[i]:start[i + 1]])
        assert st2 == oracle.OK and bytes(back) == bytes(seg_bytes)
    st, back, n = oracle.segmented_decompress(c)
    assert st == oracle.OK and bytes(back) == bytes(x)


@pytest.mark.parametrize("n,seg", [(0, 16), (5, 16), (4096, 4096), (100003, 16384), (70000, 4096)])
def test_segmented_round_trip(n, seg):
    x = synth.text(n, 31)
    st, c = oracle.segmented_compress(x, seg)
    assert st == oracle.OK
    st, back, m = oracle.segmented_decompress(c)
    assert st == oracle.OK and m == n and np.array_equal(back, x)


def test_segmented_corrupt_containers():
    x = synth.text(50000, 32)
    st, c = oracle.segmented_compress(x, 16384)
    bad = []
    t = c.copy(); t[16:24] = np.frombuffer((5).to_bytes(8, "little"), np.uint8); bad.append(t)   # count
    t = c.copy(); t[8:16] = np.frombuffer((100).to_bytes(8, "little"), np.uint8); bad.append(t)  # segment
    t = c.copy(); t[32:40] = np.frombuffer((int.from_bytes(bytes(t[32:40]), "little") + 16)
                                           .to_bytes(8, "little"), np.uint8); bad.append(t)
    bad.append(c[:-16])                                                                        # cut short
    for i, t in enumerate(bad):
        assert oracle.segmented_decompress(t)[0] == oracle.ERR_CORRUPT, i
    assert oracle.segmented_decompress(c, cap=49999)[0] == oracle.ERR_CAPACITY
