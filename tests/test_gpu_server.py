"""GPU tests of the served path (continuous batching).

Requests of mixed sizes and both operations are submitted together, so
several rounds run at once and later arrivals join while earlier ones are on
the GPU; every result must equal the oracle's bytes and the same request
served alone (exact: integer work).  A tight memory budget forces requests
to wait for admission; a request larger than the budget is refused.
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
    torch.cuda.init()


def _pinned(a: np.ndarray) -> torch.Tensor:
    t = torch.empty(max(a.size, 1), dtype=torch.uint8).pin_memory()
    if a.size:
        t[:a.size].copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return t


def _workload(count, seed):
    sizes = synth.log_uniform_sizes(count, seed=seed, lo=4096, hi=2 << 20)
    reqs = []
    for i, n in enumerate(sizes):
        x = synth.text(int(n), 900 + i) if i % 3 else synth.zipf_ascii(int(n), 900 + i)
        if i % 2 == 0:
            st, ref = oracle.compress(x)
            reqs.append(("c", x, ref))
        else:
            st, s = oracle.compress(x)
            reqs.append(("d", s, x))
    return reqs


def _submit_all(srv, reqs):
    tickets, outs = [], []
    for kind, inp, ref in reqs:
        h_in = _pinned(inp)
        if kind == "c":
            h_out = torch.zeros(hg.huff_max_stream_size(inp.size), dtype=torch.uint8).pin_memory()
            t = srv.submit(hg.HUFF_BATCH_COMPRESS, h_in, h_out, in_bytes=inp.size)
        else:
            h_out = torch.zeros(max(ref.size, 1), dtype=torch.uint8).pin_memory()
            t = srv.submit(hg.HUFF_BATCH_DECOMPRESS, h_in, h_out, in_bytes=inp.size)
        tickets.append(t)
        outs.append(h_out)
    return tickets, outs


def _check(srv, reqs, tickets, outs):
    got = []
    for (kind, inp, ref), t, h_out in zip(reqs, tickets, outs):
        r = srv.wait(t, 120000)
        assert r["done"] and r["status"] == 0, r
        assert r["out_bytes"] == ref.size
        b = h_out[:ref.size].numpy().copy()
        assert np.array_equal(b, ref)
        assert r["t_submit"] <= r["t_start"] <= r["t_done"]
        got.append(b)
        srv.release(t)
    return got


def test_mixed_requests_match_oracle_and_alone():
    reqs = _workload(48, 21)
    srv = hg.Server()
    tickets, outs = _submit_all(srv, reqs)
    mixed = _check(srv, reqs, tickets, outs)
    # the same requests one at a time
    for i in range(0, len(reqs), 5):
        t, o = _submit_all(srv, [reqs[i]])
        alone = _check(srv, [reqs[i]], t, o)[0]
        assert np.array_equal(alone, mixed[i])
    srv.close()


def test_tight_budget_admits_in_turn():
    cfg = hg.huff_server_default_config()
    cfg.device_budget = 24 << 20   # a few requests at a time
    cfg.max_rounds = 2
    srv = hg.Server(cfg)
    reqs = _workload(24, 22)
    tickets, outs = _submit_all(srv, reqs)
    _check(srv, reqs, tickets, outs)
    # a request that can never fit is refused at submission
    big = torch.zeros(64 << 20, dtype=torch.uint8)
    out = torch.zeros(1, dtype=torch.uint8)
    with pytest.raises(hg.HuffError) as e:
        srv.submit(hg.HUFF_BATCH_COMPRESS, big, out)
    assert e.value.status == hg.HUFF_ERR_BUDGET
    srv.close()


def test_corrupt_request_fails_alone():
    x = synth.text(100000, 3)
    st, s = oracle.compress(x)
    bad = s.copy()
    bad[ord("e")] = 1  # Kraft sum above 1
    reqs = [("d", s, x), ("d", bad, x), ("d", s, x)]
    srv = hg.Server()
    tickets, outs = _submit_all(srv, reqs)
    res = [srv.wait(t) for t in tickets]
    assert res[0]["status"] == 0 and res[2]["status"] == 0
    assert res[1]["status"] == hg.HUFF_ERR_CORRUPT_STREAM
    assert np.array_equal(outs[0][:x.size].numpy(), x)
    srv.close()
