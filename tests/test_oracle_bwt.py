"""Pins of the oracle's Method 3 (Section III-A): the block-sorting transform
of every block before Method 2's coder, and its inverse.

The transform is pinned to things outside the oracle: the worked example of
Burrows and Wheeler's report and hand-worked fixtures (tests/golden/bwt/),
a brute-force sort of explicitly built rotation strings on tiny inputs, and
invariants (a permutation of each block; the inverse gives the input back).
"""
import numpy as np
import pytest

import oracle
import synth
from golden_bwt import all_names, load


def u8(b):
    return np.frombuffer(bytes(b), dtype=np.uint8)


def brute_bwt(x: bytes, block: int):
    """Every rotation written out as a byte string, sorted by (string,
    start): the definition, with Python's own string order."""
    last, prim = bytearray(), []
    for s in range(0, len(x), block):
        b = x[s:s + block]
        m = len(b)
        rows = sorted(range(m), key=lambda j: (b[j:] + b[:j], j))
        last += bytes(b[(j - 1) % m] for j in rows)
        prim.append(rows.index(0))
    return bytes(last), prim


@pytest.mark.parametrize("name", all_names())
def test_golden(name):
    g = load(name)
    L, prim = oracle.bwt(u8(g["input"]), g["block"])
    assert bytes(L) == g["last"]
    assert [int(p) for p in prim] == g["primary"]
    back = oracle.ibwt(u8(g["last"]), g["block"], np.array(g["primary"], dtype=np.uint32))
    assert bytes(back) == g["input"]


def test_bruteforce_tiny_inputs():
    rng = np.random.default_rng(7)
    cases = 0
    for alpha in (1, 2, 3, 4, 256):
        for n in range(1, 14):
            for _ in range(6):
                x = bytes(rng.integers(0, alpha, n, dtype=np.uint8) + (0 if alpha == 256 else 97))
                block = int(rng.integers(1, n + 1))
                L, prim = oracle.bwt(u8(x), block)
                bl, bp = brute_bwt(x, block)
                assert bytes(L) == bl, (x, block)
                assert [int(p) for p in prim] == bp, (x, block)
                cases += 1
    assert cases > 300


def test_unsigned_byte_order():
    # 0x80.. sort above 0x7f (unsigned), so the high byte's rotation is last
    x = bytes([0x7F, 0x80, 0x00])
    L, prim = oracle.bwt(u8(x), 3)
    assert (bytes(L), list(prim)) == brute_bwt(x, 3)
    assert bytes(L) == bytes([0x80, 0x00, 0x7F])


def test_periodic_blocks_keep_start_order():
    for x in (b"aaaaaaa", b"abababab", b"abcabcabc", b"xyxyxyxyxy"):
        L, prim = oracle.bwt(u8(x), len(x))
        assert (bytes(L), list(prim)) == brute_bwt(x, len(x))
        assert bytes(oracle.ibwt(L, len(x), prim)) == x
    L, prim = oracle.bwt(u8(b"aaaa"), 4)
    assert bytes(L) == b"aaaa" and list(prim) == [0]


@pytest.mark.parametrize("block", [1, 2, 7, 64, 1000, 4096])
def test_each_block_is_permuted(block):
    x = synth.text(10000, 3)
    L, prim = oracle.bwt(x, block)
    assert prim.size == (x.size + block - 1) // block
    for s in range(0, x.size, block):
        assert np.array_equal(np.bincount(x[s:s + block], minlength=256),
                              np.bincount(L[s:s + block], minlength=256))
        assert int(prim[s // block]) < min(block, x.size - s)


@pytest.mark.parametrize("kind", ["text", "uniform", "geometric", "single"])
@pytest.mark.parametrize("block", [1, 5, 256, 3000])
def test_inverse_round_trip(kind, block):
    n = 7001
    x = {"text": lambda: synth.text(n, 5), "uniform": lambda: synth.uniform(n, 5),
         "geometric": lambda: synth.geometric(n, 5), "single": lambda: synth.single(n, 5)}[kind]()
    L, prim = oracle.bwt(x, block)
    assert np.array_equal(oracle.ibwt(L, block, prim), x)


def test_transform_groups_equal_bytes_on_text():
    # the property Method 3 relies on: after the transform, equal bytes sit
    # next to each other far more often than in the text itself
    x = synth.text(1 << 16, 11)
    L, _ = oracle.bwt(x, 1 << 16)
    same_x = int(np.count_nonzero(x[1:] == x[:-1]))
    same_l = int(np.count_nonzero(L[1:] == L[:-1]))
    assert same_l > 4 * same_x


def test_empty_and_bad_arguments():
    L, prim = oracle.bwt(np.zeros(0, dtype=np.uint8), 16)
    assert L.size == 0 and prim.size == 0
    with pytest.raises(ValueError):
        oracle.bwt(u8(b"abc"), 0)
    with pytest.raises(ValueError):  # primary index outside its block
        oracle.ibwt(u8(b"abc"), 3, np.array([3], dtype=np.uint32))


def brute_mtf(x: bytes, block: int):
    """Move-to-front with a Python list, the definition written out."""
    out = []
    for s in range(0, len(x), block):
        lst = list(range(256))
        for c in x[s:s + block]:
            j = lst.index(c)
            out.append(j)
            lst.insert(0, lst.pop(j))
    return bytes(out)


def test_mtf_hand_example():
    # Worked by hand, list 0..255 at the start: b (98) sits at 98; then a
    # (97) is at 98 (b moved in front of it); n (110) at 110 (b and a in
    # front, 0..96 and 99..109 before it); then a, n, a at 1 each; a, a at 0
    x = np.frombuffer(b"bananaaa", np.uint8)
    assert list(oracle.mtf(x, 8)) == [98, 98, 110, 1, 1, 1, 0, 0]
    assert bytes(oracle.imtf(oracle.mtf(x, 8), 8)) == b"bananaaa"


def test_mtf_bruteforce_and_round_trip():
    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 300, 1000):
        for alpha in (2, 5, 256):
            x = bytes(rng.integers(0, alpha, n, dtype=np.uint8))
            for block in (1, 3, 64, n):
                m = oracle.mtf(np.frombuffer(x, np.uint8), block)
                assert bytes(m) == brute_mtf(x, block), (n, alpha, block)
                assert bytes(oracle.imtf(m, block)) == x


def test_mtf_after_transform_is_mostly_small():
    # runs of equal bytes become zeros: far more of them after the transform
    # than when the text itself is coded
    x = synth.text(1 << 16, 12)
    L, _ = oracle.bwt(x, 1 << 16)
    m = oracle.mtf(L, 1 << 16)
    raw = oracle.mtf(x, 1 << 16)
    assert np.count_nonzero(m == 0) > 3 * np.count_nonzero(raw == 0)
    assert np.count_nonzero(m < 4) > 0.5 * m.size


@pytest.mark.parametrize("n,block,seg,use_mtf", [(0, 16, 16, False), (1, 1, 16, True),
                                                 (5000, 1000, 2048, False),
                                                 (5000, 1000, 2048, True),
                                                 (70000, 65536, 16384, True)])
def test_m3_container_round_trip(n, block, seg, use_mtf):
    x = synth.text(n, 9)
    st, c = oracle.m3_compress(x, block, seg, mtf_stage=use_mtf)
    assert st == oracle.OK
    count = (n + block - 1) // block
    assert int(np.frombuffer(c[0:8].tobytes(), "<u8")[0]) == n
    assert [int(v) for v in np.frombuffer(c[8:20].tobytes(), "<u4")] == [block, count,
                                                                         int(use_mtf)]
    head = (20 + 4 * count + 15) & ~15
    assert not c[20 + 4 * count:head].any()
    L, prim = oracle.bwt(x, block)
    assert np.array_equal(np.frombuffer(c[20:20 + 4 * count].tobytes(), "<u4"), prim)
    if use_mtf:
        L = oracle.mtf(L, block)
    st2, seg_c = oracle.segmented_compress(L, seg)
    assert np.array_equal(c[head:], seg_c)
    st, y, m = oracle.m3_decompress(c)
    assert st == oracle.OK and m == n and np.array_equal(x, y)


def test_m3_corrupt_containers():
    x = synth.text(3000, 2)
    st, c = oracle.m3_compress(x, 1000, 1024)
    bad = c.copy()
    bad[20:24] = np.frombuffer(np.array([1000], dtype="<u4").tobytes(), np.uint8)  # primary = block
    assert oracle.m3_decompress(bad)[0] == oracle.ERR_CORRUPT
    bad = c.copy()
    bad[12] ^= 1  # block count
    assert oracle.m3_decompress(bad)[0] == oracle.ERR_CORRUPT
    bad = c.copy()
    bad[16] = 2  # unknown stage
    assert oracle.m3_decompress(bad)[0] == oracle.ERR_CORRUPT
    assert oracle.m3_decompress(c[:19])[0] == oracle.ERR_CORRUPT
    assert oracle.m3_decompress(c, cap=2999)[0] == oracle.ERR_CAPACITY
