"""GPU parity of Method 3 (Section III-A): the block-sorting transform of
every block, its inverse, the move-to-front stage and the Method 3
container, byte for byte against the oracle, through the C ABI."""
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


def _gen(kind, n, seed):
    if kind == "periodic":
        unit = np.frombuffer(b"abcab", np.uint8)
        return np.resize(unit, n).astype(np.uint8)
    return {"text": synth.text, "uniform": synth.uniform, "geometric": synth.geometric,
            "single": synth.single, "zipf": synth.zipf_ascii}[kind](n, seed)


CASES = [
    ("text", 1, 1), ("text", 5, 16), ("text", 4097, 1), ("text", 4097, 3), ("text", 4097, 64),
    ("text", 100003, 4096), ("text", 100003, 100003), ("text", 100003, 1 << 20),
    ("uniform", 65537, 1000), ("geometric", 65536, 8192), ("zipf", 200000, 65536),
    ("single", 5000, 5000), ("single", 9000, 777), ("periodic", 3000, 3000),
    ("periodic", 10007, 1024),
    # one 3 MiB block: keys of 22 rank bits, so ranges with many groups are
    # too wide for the shared-memory sort and take the global passes
    ("text", 3 << 20, 4 << 20),
]


@pytest.mark.parametrize("kind,n,block", CASES, ids=[f"{k}-{n}-{b}" for k, n, b in CASES])
def test_forward_and_inverse_match_oracle(kind, n, block):
    x = _gen(kind, n, 17)
    ref_last, ref_prim = oracle.bwt(x, block)
    last, prim, st = hg.huff_bwt_forward(_dev(x), block)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(last.cpu().numpy(), ref_last)
    assert np.array_equal(prim.cpu().numpy().astype(np.uint32), ref_prim)
    back, st = hg.huff_bwt_inverse(_dev(ref_last), block,
                                   torch.from_numpy(ref_prim.astype(np.int32)).cuda())
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(back.cpu().numpy(), x)


def test_large_text_blocks():
    # four 1 MiB blocks and a ragged fifth: several radix tiles per block and
    # many doubling rounds
    n, block = (4 << 20) + 12345, 1 << 20
    x = synth.text(n, 23)
    ref_last, ref_prim = oracle.bwt(x, block)
    last, prim, st = hg.huff_bwt_forward(_dev(x), block)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(last.cpu().numpy(), ref_last)
    assert np.array_equal(prim.cpu().numpy().astype(np.uint32), ref_prim)
    back, st = hg.huff_bwt_inverse(last, block, prim)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and np.array_equal(back.cpu().numpy(), x)


def test_inverse_rejects_primary_outside_its_block():
    x = synth.text(3000, 4)
    L, P = oracle.bwt(x, 1000)
    P = P.astype(np.int64)
    P[2] = 1000
    back, st = hg.huff_bwt_inverse(_dev(L), 1000, torch.from_numpy(P.astype(np.int32)).cuda())
    torch.cuda.synchronize()
    assert int(st.item()) == hg.HUFF_ERR_CORRUPT_STREAM


def test_empty_input():
    last, prim, st = hg.huff_bwt_forward(torch.zeros(0, dtype=torch.uint8, device="cuda"), 16)
    torch.cuda.synchronize()
    assert last.numel() == 0 and prim.numel() == 0 and int(st.item()) == 0


MTF_CASES = [("text", 1, 1), ("text", 5000, 1000), ("text", 4096, 4096), ("text", 4097, 4096),
             ("text", 100003, 65536), ("text", 200000, 12345), ("uniform", 70000, 9000),
             ("geometric", 65536, 8192), ("single", 9000, 777), ("periodic", 10007, 1024)]


@pytest.mark.parametrize("kind,n,block", MTF_CASES, ids=[f"{k}-{n}-{b}" for k, n, b in MTF_CASES])
def test_mtf_matches_oracle(kind, n, block):
    # on the transform's output (the stage's real input) and on raw bytes
    x = _gen(kind, n, 31)
    L, _ = oracle.bwt(x, block) if n <= 300000 else (x, None)
    for src in (L, x):
        ref = oracle.mtf(src, block)
        got = hg.huff_mtf_forward(_dev(src), block)
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy(), ref)
        back = hg.huff_mtf_inverse(_dev(ref), block)
        torch.cuda.synchronize()
        assert np.array_equal(back.cpu().numpy(), src)


def test_mtf_large_blocks_in_place():
    n, block = (8 << 20) + 333, 1 << 20
    x = synth.text(n, 37)
    ref = oracle.mtf(x, block)
    d = _dev(x)
    hg.huff_mtf_forward(d, block, d_out=d)  # in place
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), ref)
    hg.huff_mtf_inverse(d, block, d_out=d)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), x)


@pytest.mark.parametrize("kind,n,block,seg,stages", [("text", 0, 16, 16, 0),
                                                     ("text", 70001, 65536, 16384, 0),
                                                     ("text", 70001, 65536, 16384, 1),
                                                     ("zipf", 300000, 100000, 65536, 1),
                                                     ("single", 20000, 4096, 4096, 0),
                                                     ("single", 20000, 4096, 4096, 1)])
def test_m3_container_matches_oracle(kind, n, block, seg, stages):
    x = _gen(kind, n, 29) if n else np.zeros(0, dtype=np.uint8)
    c, st = hg.huff_m3_compress(_dev(x), block, seg, stages=stages)
    torch.cuda.synchronize()
    ost, ref = oracle.m3_compress(x, block, seg, mtf_stage=bool(stages))
    assert int(st.item()) == 0 and ost == 0
    assert np.array_equal(c.cpu().numpy(), ref)
    back, m, st = hg.huff_m3_decompress(c)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and m == n and np.array_equal(back.cpu().numpy(), x)


def test_m3_rejects_bad_containers():
    x = synth.text(50000, 8)
    st, c = oracle.m3_compress(x, 20000, 16384)
    for mutate in ("primary", "count", "stages", "short"):
        t = c.copy()
        if mutate == "primary":
            t[20:24] = np.frombuffer((20000).to_bytes(4, "little"), np.uint8)
        elif mutate == "count":
            t[12] ^= 1
        elif mutate == "stages":
            t[16] = 2
        else:
            t = t[:-16]
        dc = torch.zeros(max(t.size, 16), dtype=torch.uint8, device="cuda")
        dc[:t.size] = torch.from_numpy(t).cuda()
        back, m, st = hg.huff_m3_decompress(dc[:t.size])
        torch.cuda.synchronize()
        assert int(st.item()) != 0, mutate
        assert oracle.m3_decompress(t)[0] != oracle.OK, mutate


def test_full_size_sampled_against_oracle():
    # 64 MiB of text in 1 MiB blocks, the bench's block size: three blocks
    # checked against the oracle one by one (the oracle would take minutes
    # for all), the rest by the round trip through the GPU inverse
    n, block = 64 << 20, 1 << 20
    x = synth.text(n, 1)
    d = _dev(x)
    last, prim, st = hg.huff_bwt_forward(d, block)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    L = last.cpu().numpy()
    P = prim.cpu().numpy().astype(np.uint32)
    for b in (0, 31, 63):
        s = b * block
        ref_l, ref_p = oracle.bwt(x[s:s + block], block)
        assert np.array_equal(L[s:s + block], ref_l), b
        assert int(P[b]) == int(ref_p[0]), b
        ref_m = oracle.mtf(ref_l, block)
        got_m = hg.huff_mtf_forward(last[s:s + block].clone(), block)
        torch.cuda.synchronize()
        assert np.array_equal(got_m.cpu().numpy(), ref_m), b
    back, st = hg.huff_bwt_inverse(last, block, prim)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and torch.equal(back, d)
    c, st = hg.huff_m3_compress(d, block, 65536, stages=hg.HUFF_M3_MTF)
    y, m, st2 = hg.huff_m3_decompress(c)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and int(st2.item()) == 0 and m == n and torch.equal(y, d)
