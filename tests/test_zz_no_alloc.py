"""huff_encode_noalloc: the encoder for callers that cannot allocate device
memory while they encode (a latency-critical loop where an allocation would
synchronise the device, a fixed memory budget reserved at start-up, a
wrapper that only passes input and output buffers).  Its scratch is a fixed
array inside the library instead of a caller workspace.

The test calls the entry point through the C ABI (ctypes) and checks that
its stream is byte-identical to huff_encode's (integer work: the tolerance is
exact) on two calls in a row with different inputs, so scratch left over by
the first call would show up in the second.  A third test fills the whole
scratch array (1 GiB of text: 65,536 units) and compares the stream with the
oracle's encoder byte for byte.  The file runs last in collection order and
also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2306_11070_gb300 as hg
from paper_2306_11070_gb300 import build as nvbuild

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    nvbuild.build()
    lib = hg.lib()
    fn = lib.huff_encode_noalloc
    fn.restype = ctypes.c_int32
    fn.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint32,
                   ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    return fn


def _reference(d, cs):
    h = hg.huff_histogram(d)
    cb, st = hg.huff_build_codebook(h)
    out, ob, st = hg.huff_encode(d, cb, cs)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    nb = int(ob.item())
    return cb, out[:nb].cpu().numpy(), nb


def _noalloc(fn, d, cb, cs):
    n = d.numel()
    cap = hg.huff_max_stream_size(n, cs)
    out = torch.full((cap,), 0xAB, dtype=torch.uint8, device="cuda")
    ob = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(ctypes.c_void_p(d.data_ptr()), n, ctypes.c_void_p(cb.data_ptr()), cs,
            ctypes.c_void_p(out.data_ptr()), cap, ctypes.c_void_p(ob.data_ptr()),
            ctypes.c_void_p(st.data_ptr()), stream)
    assert rc == hg.HUFF_OK, hg.huff_status_str(rc)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    nb = int(ob.item())
    return out[:nb].cpu().numpy(), nb


@pytest.mark.parametrize("cs", [16384, 1024])
def test_noalloc_matches_huff_encode_two_calls(cs):
    fn = _noalloc_fn()
    inputs = [synth.text(3 * 16384 * 7 + 4321, 11), synth.zipf_ascii(200003, 12),
              synth.uniform(5 * 16384, 13)]
    for x in inputs:  # consecutive calls share the scratch array
        d = torch.from_numpy(x).cuda()
        cb, ref, nref = _reference(d, cs)
        got, ngot = _noalloc(fn, d, cb, cs)
        assert ngot == nref
        assert np.array_equal(got, ref)


def test_noalloc_rejects_inputs_beyond_its_scratch():
    fn = _noalloc_fn()
    d = torch.zeros(16, dtype=torch.uint8, device="cuda")
    cb = torch.zeros(hg.CODEBOOK_BYTES, dtype=torch.uint8, device="cuda")
    out = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    ob = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = fn(ctypes.c_void_p(d.data_ptr()), (1 << 30) + 1, ctypes.c_void_p(cb.data_ptr()), 16384,
            ctypes.c_void_p(out.data_ptr()), out.numel(), ctypes.c_void_p(ob.data_ptr()),
            ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(0))
    assert rc == hg.HUFF_ERR_BUDGET


def test_noalloc_full_scratch_matches_oracle():
    """1 GiB of text, the scratch array's full size (65,536 units), twice in a
    row; the stream equals the oracle's encoder with the same code lengths."""
    fn = _noalloc_fn()
    x = synth.make("text_1g")
    assert x.size == 1 << 30
    d = torch.from_numpy(x).cuda()
    h = hg.huff_histogram(d)
    cb, st = hg.huff_build_codebook(h)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ln = hg.parse_codebook(cb)[0]
    ost, ref, need = oracle.encode(x, ln, 16384)
    assert ost == oracle.OK
    for _ in range(2):
        got, ngot = _noalloc(fn, d, cb, 16384)
        assert ngot == need
        assert np.array_equal(got, ref)


@pytest.mark.skipif(torch.cuda.device_count() < 2, reason="needs two GPUs")
def test_noalloc_on_two_devices():
    """The library's launch set-up (dynamic shared memory limits, scratch
    address) is per device: the no-allocation encoder runs on device 0, then
    on device 1, and both streams equal huff_encode's on device 0."""
    fn = _noalloc_fn()
    x = synth.text(3 * 16384 + 77, 21)
    ref_cb, ref, nref = _reference(torch.from_numpy(x).cuda(0), 16384)
    for devno in (0, 1):
        with torch.cuda.device(devno):
            d = torch.from_numpy(x).cuda(devno)
            cb = ref_cb.to(f"cuda:{devno}")
            got, ngot = _noalloc(fn, d, cb, 16384)
            assert ngot == nref and np.array_equal(got, ref)
