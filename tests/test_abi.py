"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/*.h declares; host-only calls agree with the oracle's sizes."""
import glob
import os
import re

import pytest

import oracle
import paper_2306_11070_gb300 as hg
from paper_2306_11070_gb300 import build as nvbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(huff_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    nvbuild.build()
    return hg.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("huff_histogram", "huff_build_codebook", "huff_encode", "huff_decode",
                 "huff_compress", "huff_max_stream_size", "huff_workspace_size",
                 "huff_status_str"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 4095, 4096, 16384, 16385, 10**9, 1 << 30])
@pytest.mark.parametrize("cs", [16, 1024, 16384, 1 << 24])
def test_max_stream_size_matches_oracle(lib, n, cs):
    assert hg.huff_max_stream_size(n, cs) == oracle.max_stream_size(n, cs)


@pytest.mark.parametrize("cs", [0, 8, 17, 100, (1 << 24) + 16])
def test_invalid_chunk_sizes(lib, cs):
    assert hg.huff_max_stream_size(100, cs) == 0
    assert hg.huff_workspace_size(100, cs) == 0


def test_workspace_grows_with_n(lib):
    a = hg.huff_workspace_size(1 << 20)
    b = hg.huff_workspace_size(1 << 30)
    assert 0 < a < b and b % 256 == 0


def test_status_strings(lib):
    for st in range(-8, 1):
        assert hg.huff_status_str(st)
    assert hg.huff_status_str(-4) == "corrupt stream"


def test_product_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2306_11070_gb300")
    files = glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True)
    for f in files:
        if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(f).read()
            assert "import oracle" not in text and "huff_oracle" not in text, f
            assert "from oracle" not in text, f


def test_next_row_sizes_and_argument_checks(lib):
    # host-only paths of the next rows: sizes, and argument errors returned
    # before any device work
    import ctypes
    assert lib.huff_bwt_workspace_size(1 << 20, 0) == 0          # block 0
    assert lib.huff_bwt_workspace_size(1 << 31, 1 << 20) == 0    # above the limit
    a, b = lib.huff_bwt_workspace_size(1 << 20, 1 << 16), lib.huff_bwt_workspace_size(1 << 22, 1 << 16)
    assert 0 < a < b
    assert lib.huff_mtf_workspace_size(1 << 20, 0) == 0
    assert lib.huff_mtf_workspace_size(1 << 20, 4096) > (1 << 20)
    assert lib.huff_m3_max_size(1000, 0, 16, 16384) == 0
    assert lib.huff_m3_max_size(1000, 100, 15, 16384) == 0          # segment not a multiple of 16
    count = 10
    head = (20 + 4 * count + 15) & ~15
    assert lib.huff_m3_max_size(1000, 100, 1024, 16384) == \
        head + lib.huff_segmented_max_size(1000, 1024, 16384)
    st = ctypes.c_int32(0)
    none = ctypes.c_void_p(0)
    # null pointers / zero block: invalid before the device is touched
    assert lib.huff_bwt_forward(none, 16, 0, none, none, none, 0, ctypes.byref(st), none) == \
        hg.HUFF_ERR_INVALID_ARG
    assert lib.huff_mtf_forward(none, 16, 4, none, none, 0, none) == hg.HUFF_ERR_INVALID_ARG
    assert lib.huff_mtf_inverse(none, 16, 0, none, none, 0, none) == hg.HUFF_ERR_INVALID_ARG
    assert lib.huff_m3_compress(none, 16, 4, 16, 16384, 2, none, 0, none, none, 0, none,
                                none) == hg.HUFF_ERR_INVALID_ARG


@pytest.mark.parametrize("params", [(1024, 12, 24, 8, 2), (8, 2, 5, 4, 1), (4096, 16, 32, 8, 1),
                                    (2, 1, 1, 1, 1)])
def test_lzss_sizes_bound_the_oracle(lib, params):
    """huff_lzss_max_size holds the oracle's container on real inputs and its
    own worst-case bound; invalid parameters and segment sizes give 0."""
    import numpy as np
    import synth
    P = hg._lzss_params(params)
    for n, seg in [(0, 16), (1, 16), (100, 16), (3000, 1024), (5000, 4096)]:
        bound = lib.huff_lzss_max_size(n, seg, P)
        assert bound >= oracle.lzss_segmented_max_size(n, seg, params)
        for x in (synth.bitstream(n, 1), synth.uniform(n, 2)):
            st, c = oracle.lzss_segmented_compress(x, seg, params)
            assert st == oracle.OK and c.size <= bound
        assert lib.huff_lzss_workspace_size(n, seg, P) > 0
    assert lib.huff_lzss_max_size(100, 24, P) == 0  # segment not a multiple of 16
    bad = hg._lzss_params((1000, 12, 24, 8, 2))
    assert lib.huff_lzss_max_size(100, 16, bad) == 0
