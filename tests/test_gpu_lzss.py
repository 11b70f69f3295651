"""GPU parity of LZSS Method 2 (segmented LZSS, Section III-B) against the
CPU oracle: containers byte for byte, decoded bytes, statuses.

The oracle searches the window bit by bit (about a second per 64 KiB with a
1024-bit window), so whole-container comparisons use inputs of up to a few
tens of KiB; the 16 MiB case compares sampled segments with the oracle's
Method 1 on the same bytes, and everything with the round trip.
"""
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


def _dev(x):
    t = torch.zeros(max(x.size, 16), dtype=torch.uint8, device="cuda")
    if x.size:
        t[:x.size] = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return t[:x.size]


def _gen(name, n, seed):
    return {"bitstream": lambda: synth.bitstream(n, seed), "uniform": lambda: synth.uniform(n, seed),
            "text": lambda: synth.text(n, seed), "zeros": lambda: np.zeros(n, np.uint8),
            "ones": lambda: np.full(n, 0xFF, np.uint8),
            "periodic": lambda: np.tile(np.array([0xA5, 0x3C, 0x0F], np.uint8), n // 3 + 1)[:n],
            }[name]()


def _roundtrip_vs_oracle(x, seg, params):
    ost, ref = oracle.lzss_segmented_compress(x, seg, params)
    assert ost == oracle.OK
    c, st = hg.huff_lzss_compress(_dev(x), seg, params)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    got = c.cpu().numpy()
    assert got.size == ref.size, (got.size, ref.size)
    if not np.array_equal(got, ref):
        bad = np.flatnonzero(got != ref)
        raise AssertionError(f"{bad.size} container bytes differ, first at {bad[0]}")
    y, n, st = hg.huff_lzss_decompress(c)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and n == x.size
    assert np.array_equal(y.cpu().numpy(), x)
    # the GPU decoder on the oracle's container too
    y2, n2, st2 = hg.huff_lzss_decompress(torch.from_numpy(ref).cuda())
    torch.cuda.synchronize()
    assert int(st2.item()) == 0 and np.array_equal(y2.cpu().numpy(), x)


@pytest.mark.parametrize("gen", ["bitstream", "uniform", "text", "zeros", "ones", "periodic"])
@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 1000, 4096, 9001])
def test_container_matches_oracle_paper_params(gen, n):
    _roundtrip_vs_oracle(_gen(gen, n, n + 3), 4096, hg.LZSS_PAPER)


# windows below 64 bits and above 16384 take the compressor's L1 path, the
# others its shared-memory ring; above 2048 the decompressor reads its
# sources back through L2
@pytest.mark.parametrize("params", [(1024, 12, 24, 8, 1), (8, 2, 5, 4, 1), (4, 3, 4, 2, 2),
                                    (16, 4, 12, 8, 1), (64, 6, 9, 5, 1), (64, 12, 24, 8, 2),
                                    (256, 1, 32, 32, 1), (4096, 16, 32, 8, 2), (32, 3, 3, 1, 2),
                                    (2048, 8, 20, 8, 1), (16384, 12, 24, 8, 1),
                                    (65536, 20, 32, 16, 1),
                                    # the decoder's branch-free step (windows of 32..2048
                                    # bits, stored prefix, literal blocks up to 31 bits):
                                    # 31-bit literals and 32-bit matches, a length field
                                    # of no bits, one-bit matches, short windows
                                    (256, 4, 32, 31, 2), (2048, 1, 1, 16, 2),
                                    (128, 2, 9, 3, 2), (512, 20, 32, 31, 2),
                                    (32, 1, 32, 32, 2)])
@pytest.mark.parametrize("gen", ["bitstream", "text", "periodic"])
def test_container_matches_oracle_other_params(params, gen):
    _roundtrip_vs_oracle(_gen(gen, 3000, sum(params)), 1024, params)


@pytest.mark.parametrize("seg", [16, 48, 4096, 65536])
def test_segment_sizes(seg):
    _roundtrip_vs_oracle(synth.bitstream(20000, seg), seg, hg.LZSS_PAPER)


def test_large_input_sampled_segments():
    """16 MiB of the bitstream stand-in in 64 KiB segments: round trip, and
    three segments' codes equal the oracle's Method 1 on the same bytes."""
    n, seg = 16 << 20, 64 << 10
    x = synth.bitstream(n, 7)
    d = _dev(x)
    c, st = hg.huff_lzss_compress(d, seg, hg.LZSS_PAPER)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    cn = c.cpu().numpy()
    count = n // seg
    bits = cn[48:48 + 4 * count].view("<u4")
    start = (48 + 4 * count + 15) // 16 * 16
    starts = []
    for i in range(count):
        starts.append(start)
        start += ((int(bits[i]) + 7) // 8 + 15) // 16 * 16
    assert start == cn.size
    for i in (0, 97, count - 1):
        ost, code, nb = oracle.lzss_encode(x[i * seg:(i + 1) * seg], hg.LZSS_PAPER)
        assert ost == oracle.OK and nb == int(bits[i])
        assert np.array_equal(cn[starts[i]:starts[i] + code.size], code), i
    y, nn, st = hg.huff_lzss_decompress(c)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and nn == n
    assert torch.equal(y, d)


def test_no_allocation_path():
    """Pre-allocated buffers: nothing is allocated or synchronised inside."""
    x = synth.bitstream(50000, 5)
    d = _dev(x)
    L = hg.lib()
    P = hg._lzss_params(hg.LZSS_PAPER)
    cap = L.huff_lzss_max_size(x.size, 4096, P)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    ws = torch.empty(L.huff_lzss_workspace_size(x.size, 4096, P), dtype=torch.uint8, device="cuda")
    ob = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    hg.huff_lzss_compress(d, 4096, hg.LZSS_PAPER, d_out=out, d_out_bytes=ob, d_ws=ws, d_status=st)
    torch.cuda.synchronize()
    size = int(ob.item())
    ost, ref = oracle.lzss_segmented_compress(x, 4096, hg.LZSS_PAPER)
    assert int(st.item()) == 0 and size == ref.size
    assert np.array_equal(out[:size].cpu().numpy(), ref)
    y = torch.empty(x.size, dtype=torch.uint8, device="cuda")
    dn = torch.zeros(1, dtype=torch.int64, device="cuda")
    dws = torch.empty(L.huff_lzss_decompress_workspace_size(size), dtype=torch.uint8,
                      device="cuda")
    hg.huff_lzss_decompress(out[:size], d_out=y, d_n=dn, d_ws=dws, d_status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and int(dn.item()) == x.size and torch.equal(y, d)


def test_statuses_match_oracle():
    x = synth.bitstream(9000, 2)
    ost, c = oracle.lzss_segmented_compress(x, 4096, hg.LZSS_PAPER)
    cases = {}
    bad = c.copy()
    bad[48] ^= 1
    cases["table_length"] = bad
    bad = c.copy()
    bad[16] = 3
    cases["window_not_power_of_two"] = bad
    cases["truncated"] = c[:-16]
    bad = c.copy()
    bad[40] = 9
    cases["count"] = bad
    # a token's flag flipped inside a segment's code: decodes to something
    # else or runs past the recorded length
    bad = c.copy()
    s0 = (48 + 4 * 3 + 15) // 16 * 16
    bad[s0 + 130] ^= 0x40
    cases["code_bit"] = bad
    for name, cc in cases.items():
        ost, _, _ = oracle.lzss_segmented_decompress(cc)
        y, n, st = hg.huff_lzss_decompress(torch.from_numpy(np.ascontiguousarray(cc)).cuda(),
                                           out_cap=x.size)
        torch.cuda.synchronize()
        got = int(st.item())
        if ost == oracle.OK:  # a flipped bit may still decode to valid tokens
            assert got == 0, name
        else:
            assert got == hg.HUFF_ERR_CORRUPT_STREAM and ost == oracle.ERR_CORRUPT, (name, got, ost)
    y, n, st = hg.huff_lzss_decompress(torch.from_numpy(c).cuda(), out_cap=100)
    torch.cuda.synchronize()
    assert int(st.item()) == hg.HUFF_ERR_CAPACITY


def test_length_field_above_longest_match_mid_segment():
    """A match token far from both ends of a segment (the decoder's
    branch-free step) whose length field is all ones: with 1024/12/24/8 the
    4-bit field then means 27 > 24 bits, so the stream is corrupt for the
    oracle and the GPU alike."""
    x = synth.bitstream(16384, 12)
    params = hg.LZSS_PAPER
    W, lmin, lmax, blk, _ = params
    ob, lb = 10, 4
    ost, c = oracle.lzss_segmented_compress(x, 4096, params)
    assert ost == oracle.OK
    start = (48 + 4 * 4 + 15) // 16 * 16  # segment 0's code
    bits = np.unpackbits(c[start:start + 4096])
    pos, hit = W, None  # tokens begin after the stored prefix
    while pos < 20000:
        if bits[pos]:
            if pos >= 4000:
                hit = pos
                break
            pos += 1 + ob + lb
        else:
            pos += 1 + blk
    assert hit is not None
    bad = c.copy()
    for j in range(hit + 1 + ob, hit + 1 + ob + lb):
        bad[start + j // 8] |= np.uint8(0x80 >> (j % 8))
    ost, _, _ = oracle.lzss_segmented_decompress(bad)
    assert ost == oracle.ERR_CORRUPT
    y, n, st = hg.huff_lzss_decompress(torch.from_numpy(bad).cuda(), out_cap=x.size)
    torch.cuda.synchronize()
    assert int(st.item()) == hg.HUFF_ERR_CORRUPT_STREAM


def test_capacity_and_arguments():
    x = _dev(synth.uniform(5000, 1))
    with pytest.raises(hg.HuffError):
        hg.huff_lzss_compress(x, 100, hg.LZSS_PAPER)  # not a multiple of 16
    with pytest.raises(hg.HuffError):
        hg.huff_lzss_compress(x, 4096, (1000, 12, 24, 8, 2))
    L = hg.lib()
    P = hg._lzss_params(hg.LZSS_PAPER)
    out = torch.empty(64, dtype=torch.uint8, device="cuda")
    ws = torch.empty(L.huff_lzss_workspace_size(5000, 4096, P), dtype=torch.uint8, device="cuda")
    ob = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    hg.huff_lzss_compress(x, 4096, hg.LZSS_PAPER, d_out=out, d_out_bytes=ob, d_ws=ws, d_status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == hg.HUFF_ERR_CAPACITY
