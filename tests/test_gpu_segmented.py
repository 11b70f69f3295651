"""GPU parity of the segmented container (one codebook per segment, the
paper's Method 2 taken literally): the container bytes equal the oracle's,
containers round-trip, and malformed containers get the oracle's status."""
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


@pytest.mark.parametrize("n,seg,gen", [(0, 16, "text"), (7, 16, "text"), (4096, 4096, "text"),
                                       (100003, 16384, "text"), (1 << 20, 65536, "zipf"),
                                       (300001, 4096, "geo"), (65536, 16, "single")])
def test_segmented_matches_oracle_and_round_trips(n, seg, gen):
    g = {"text": lambda: synth.text(n, 41), "zipf": lambda: synth.zipf_ascii(n, 42),
         "geo": lambda: synth.geometric(n, 43), "single": lambda: synth.single(n, 0x62)}[gen]
    x = g()
    c, st = hg.huff_segmented_compress(_dev(x), seg)
    torch.cuda.synchronize()
    ost, ref = oracle.segmented_compress(x, seg)
    assert int(st.item()) == 0 and ost == 0
    assert np.array_equal(c.cpu().numpy(), ref)
    back, m, st = hg.huff_segmented_decompress(c)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and m == n and np.array_equal(back.cpu().numpy(), x)


def test_segmented_decodes_oracle_containers_and_rejects_bad_ones():
    x = synth.text(50000, 32)
    st, c = oracle.segmented_compress(x, 16384)
    bad = {"ok": c}
    t = c.copy(); t[16:24] = np.frombuffer((5).to_bytes(8, "little"), np.uint8); bad["count"] = t
    t = c.copy(); t[8:16] = np.frombuffer((100).to_bytes(8, "little"), np.uint8); bad["segment"] = t
    t = c.copy(); t[32:40] = np.frombuffer((int.from_bytes(bytes(t[32:40]), "little") + 16)
                                           .to_bytes(8, "little"), np.uint8); bad["start"] = t
    bad["short"] = c[:-16]
    for name, t in bad.items():
        dc = torch.zeros(max(t.size, 16), dtype=torch.uint8, device="cuda")
        dc[:t.size] = torch.from_numpy(t).cuda()
        back, m, st = hg.huff_segmented_decompress(dc[:t.size], out_cap=x.size)
        torch.cuda.synchronize()
        ost, oback, on = oracle.segmented_decompress(t, cap=x.size)
        assert int(st.item()) == ost, name
        if ost == 0:
            assert np.array_equal(back.cpu().numpy(), x)
    back, m, st = hg.huff_segmented_decompress(torch.from_numpy(c).cuda(), out_cap=x.size - 1)
    torch.cuda.synchronize()
    assert int(st.item()) == hg.HUFF_ERR_CAPACITY and m == x.size


def test_segmented_bad_arguments():
    x = torch.zeros(1000, dtype=torch.uint8, device="cuda")
    for seg in (0, 8, 24):
        with pytest.raises(hg.HuffError):
            hg.huff_segmented_compress(x, seg)


def test_segmented_full_size_sampled():
    # 256 MiB of text in 1 MiB segments (the bench's workload): three
    # segments' streams against the oracle's, every start-table entry
    # consistent, and the whole container back through the GPU
    n, seg = 256 << 20, 1 << 20
    x = synth.text(n, 1)
    d = _dev(x)
    c, st = hg.huff_segmented_compress(d, seg)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ch = c.cpu().numpy()
    count = n // seg
    start = np.frombuffer(ch[24:24 + 8 * (count + 1)].tobytes(), "<u8")
    assert int(start[-1]) == ch.size
    for i in (0, 100, count - 1):
        ost, ref = oracle.compress(x[i * seg:(i + 1) * seg])
        s0 = int(start[i])
        assert np.array_equal(ch[s0:s0 + ref.size], ref), i
        assert not ch[s0 + ref.size:int(start[i + 1])].any()
    back, m, st = hg.huff_segmented_decompress(c)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and m == n and torch.equal(back, d)
