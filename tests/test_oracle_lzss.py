"""Pins of the LZSS oracle (paper Section III-B, Method 1 and Method 2).

The oracle (oracle/lzss_oracle.c) is checked against things other than
itself:
  - hand-worked token streams (tests/golden/lzss/*.txt), each derived by hand
    from the paper's description and the readings Z1-Z5;
  - a closed form: all-zero input with the stored prefix (dictionary 2) is
    the prefix, then maximal matches at distance 1 and a known tail;
  - a token-by-token audit of the code stream on small random inputs: every
    reference must repeat exactly the bits it claims, and a vectorised
    search over all distances (numpy, a different method from the oracle's
    distance loop) must find no longer match and no equally long match at a
    smaller distance; every literal must stand where no match of at least
    the minimum length exists;
  - round trips through the oracle's own decoder (a different procedure);
  - the Method 2 container's layout, read field by field.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lzss")


def _load(name):
    rec = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, _, v = line.partition(":")
            rec[k.strip()] = v.strip()
    p = dict(kv.split("=") for kv in rec["params"].split())
    params = tuple(int(p[k]) for k in ("window", "min_len", "max_len", "block", "dict"))
    return (params, bytes.fromhex(rec["input_hex"]), int(rec["code_bits"]),
            bytes.fromhex(rec["code_hex"]))


def golden_names():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))


@pytest.mark.parametrize("name", golden_names())
def test_golden(name):
    params, x, bits, code = _load(name)
    st, c, nb = oracle.lzss_encode(np.frombuffer(x, np.uint8), params)
    assert st == oracle.OK
    assert nb == bits
    assert bytes(c) == code
    st, y = oracle.lzss_decode(c, nb, len(x), params)
    assert st == oracle.OK and bytes(y) == x


# ------------------------------------------------------------------ stream audit
def _bits(x):
    return np.unpackbits(np.asarray(x, dtype=np.uint8))  # MSB first (Z1)


def _dict_bits(W):
    return _bits(np.arange(W // 8 + 1, dtype=np.uint8))[:W]


def _fields(params):
    W, lmin, lmax, blk, dct = params
    return int(np.log2(W)), int(np.ceil(np.log2(lmax - lmin + 1))) if lmax > lmin else 0


def _longest(seq, p, W, lmin, maxlen, dct):
    """(length, distance) of the best match at p by comparing, for every
    distance at once, the source and the lookahead as 2-D arrays."""
    ds = np.arange(1, W + 1)
    if dct == 2:
        ds = ds[ds <= p]
    if ds.size == 0 or maxlen < lmin:
        return 0, 0
    off = W if dct == 1 else 0  # seq holds the dictionary first under D = 1
    i = np.arange(maxlen)
    src = seq[off + p - ds[:, None] + i[None, :]]
    tgt = seq[off + p + i][None, :]
    eq = src == tgt
    lens = np.where(eq.all(axis=1), maxlen, np.argmin(eq, axis=1))
    best = int(lens.max())
    return best, int(ds[np.flatnonzero(lens == best)[0]])


def _audit(x, params):
    """Walk the oracle's code stream token by token and check each token."""
    W, lmin, lmax, blk, dct = params
    ob, lb = _fields(params)
    st, code, nb = oracle.lzss_encode(x, params)
    assert st == oracle.OK
    cb = _bits(code)[:nb]
    data = _bits(x)
    n = data.size
    seq = np.concatenate([_dict_bits(W), data]) if dct == 1 else data
    q = 0  # read position in the code stream
    p = 0
    if dct == 2:
        raw = min(W, n)
        assert np.array_equal(cb[:raw], data[:raw])  # the first W bits as they are
        q = p = raw
    while p < n:
        r = n - p
        best, dbest = _longest(seq, p, W, lmin, min(lmax, r), dct)
        flag = cb[q]
        q += 1
        if flag:
            d = int("".join(map(str, cb[q:q + ob])) or "0", 2) + 1
            q += ob
            l = (int("".join(map(str, cb[q:q + lb])), 2) if lb else 0) + lmin
            q += lb
            assert lmin <= l <= min(lmax, r)
            assert (best, dbest) == (l, d), (p, best, dbest, l, d)
            p += l
        else:
            assert best < lmin, (p, best)
            k = min(blk, r)
            assert np.array_equal(cb[q:q + k], data[p:p + k])
            q += k
            p += k
    assert q == nb


PARAMS = [(8, 2, 5, 4, 1), (4, 3, 4, 2, 2), (16, 4, 12, 8, 1), (16, 4, 12, 8, 2),
          (32, 3, 8, 3, 2), (64, 6, 9, 5, 1), (64, 12, 24, 8, 2), (128, 12, 24, 8, 1)]


@pytest.mark.parametrize("params", PARAMS)
def test_token_audit_random_inputs(params):
    rng = np.random.default_rng(sum(params))
    for t in range(12):
        m = int(rng.integers(0, 40))
        kind = t % 4
        if kind == 0:
            x = rng.integers(0, 256, m, dtype=np.uint8)
        elif kind == 1:
            x = rng.integers(0, 4, m, dtype=np.uint8)  # long runs of zero bits
        elif kind == 2:
            x = np.tile(rng.integers(0, 256, 3, dtype=np.uint8), m // 3 + 1)[:m]
        else:
            x = synth.bitstream(m, seed=t)
        _audit(np.ascontiguousarray(x, dtype=np.uint8), params)


def test_zeros_closed_form():
    """All-zero input with the stored prefix (dictionary 2): the first W bits
    as they are, then every token a match at distance 1 of Lmax bits (the
    source runs into the zeros being coded), a last shorter match when at
    least Lmin bits are left, else literals of up to B bits."""
    for (W, lmin, lmax, blk) in [(1024, 12, 24, 8), (64, 4, 20, 8), (16, 3, 7, 5), (8, 6, 9, 2)]:
        params = (W, lmin, lmax, blk, 2)
        ob, lb = _fields(params)
        ref = 1 + ob + lb
        for m in (1, 3, 10, 100, 300):
            st, code, nb = oracle.lzss_encode(np.zeros(m, np.uint8), params)
            assert st == oracle.OK
            n = 8 * m
            raw = min(W, n)
            full, rest = divmod(n - raw, lmax)
            expect = raw + full * ref
            if rest >= lmin:
                expect += ref
            else:
                while rest:
                    k = min(blk, rest)
                    expect += 1 + k
                    rest -= k
            assert nb == expect, (params, m)


@pytest.mark.parametrize("gen", ["bitstream", "uniform", "text", "zeros"])
@pytest.mark.parametrize("params", [oracle.PAPER_LZSS, (1024, 12, 24, 8, 1), (256, 6, 16, 8, 2)])
def test_round_trip(gen, params):
    n = 3000
    x = {"bitstream": lambda: synth.bitstream(n, 3), "uniform": lambda: synth.uniform(n, 4),
         "text": lambda: synth.text(n, 5), "zeros": lambda: np.zeros(n, np.uint8)}[gen]()
    st, code, nb = oracle.lzss_encode(x, params)
    assert st == oracle.OK
    st, y = oracle.lzss_decode(code, nb, n, params)
    assert st == oracle.OK and np.array_equal(y, x)
    # a truncated stream is corrupt
    if nb > 1:
        st, _ = oracle.lzss_decode(code, nb - 1, n, params)
        assert st == oracle.ERR_CORRUPT


def test_bad_parameters():
    for params in [(1000, 12, 24, 8, 2), (1024, 0, 24, 8, 2), (1024, 25, 24, 8, 2),
                   (1024, 12, 33, 8, 2), (1024, 12, 24, 0, 2), (1024, 12, 24, 8, 3)]:
        st, _, _ = oracle.lzss_encode(np.zeros(4, np.uint8), params)
        assert st == oracle.ERR_INVALID_ARG


# ------------------------------------------------------------------ Method 2 container
def test_container_layout():
    x = synth.bitstream(10000, 9)
    seg = 4096
    params = oracle.PAPER_LZSS
    st, c = oracle.lzss_segmented_compress(x, seg, params)
    assert st == oracle.OK
    u32 = lambda o: int.from_bytes(bytes(c[o:o + 4]), "little")
    u64 = lambda o: int.from_bytes(bytes(c[o:o + 8]), "little")
    assert u64(0) == x.size and u64(8) == seg
    assert (u32(16), u32(20), u32(24), u32(28), u32(32), u32(36)) == (1024, 12, 24, 8, 2, 0)
    count = u64(40)
    assert count == 3
    pos = (48 + 4 * count + 15) // 16 * 16
    for i in range(count):
        bits = u32(48 + 4 * i)
        m = min(seg, x.size - i * seg)
        st, code, nb = oracle.lzss_encode(x[i * seg:i * seg + m], params)
        assert nb == bits
        nbytes = (bits + 7) // 8
        assert bytes(c[pos:pos + nbytes]) == bytes(code)
        end = (pos + nbytes + 15) // 16 * 16
        assert not c[pos + nbytes:end].any()
        pos = end
    assert pos == c.size
    st, y, n = oracle.lzss_segmented_decompress(c)
    assert st == oracle.OK and n == x.size and np.array_equal(y, x)


def test_container_edge_sizes_and_corruption():
    params = oracle.PAPER_LZSS
    for n in (0, 1, 15, 16, 4096, 4097):
        x = synth.bitstream(n, n + 1)
        st, c = oracle.lzss_segmented_compress(x, 4096, params)
        assert st == oracle.OK
        st, y, nn = oracle.lzss_segmented_decompress(c)
        assert st == oracle.OK and nn == n and np.array_equal(y, x)
    x = synth.bitstream(9000, 2)
    st, c = oracle.lzss_segmented_compress(x, 4096, params)
    bad = c.copy()
    bad[48] ^= 1  # a segment's bit length no longer matches the layout
    assert oracle.lzss_segmented_decompress(bad)[0] == oracle.ERR_CORRUPT
    bad = c.copy()
    bad[16] = 3  # window not a power of two
    assert oracle.lzss_segmented_decompress(bad)[0] == oracle.ERR_CORRUPT
    assert oracle.lzss_segmented_decompress(c[:-16])[0] == oracle.ERR_CORRUPT
    assert oracle.lzss_segmented_decompress(c, cap=100)[0] == oracle.ERR_CAPACITY
