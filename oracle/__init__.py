"""CPU oracle of the Huffman hot path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.  The CUDA library shares no code
with it.  The arithmetic lives in plain C (``huff_oracle.c``), compiled with
gcc into ``libhuff_oracle.so`` beside it; this module only marshals numpy
arrays.  Each function follows the paper's Huffman Method 1, Method 2 and
Method 3 (Section III-A); see the C file's header for the readings taken
where the paper is silent.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "huff_oracle.c")
_SRC_LZSS = os.path.join(_HERE, "lzss_oracle.c")
_HDR = os.path.join(_HERE, "huff_oracle.h")
_LIB = os.path.join(_HERE, "libhuff_oracle.so")
_lib = None

OK = 0
ERR_INVALID_ARG = -1
ERR_CODE_TOO_LONG = -2
ERR_CAPACITY = -3
ERR_CORRUPT = -4

HEADER_BYTES = 272
MAX_CODE_LEN = 32
DEFAULT_CHUNK = 16384


class LzssParams(ctypes.Structure):
    """oracle_lzss_params: window W (bits), shortest / longest match (bits),
    literal block (bits), dictionary mode (1: counting numbers, 2: the first
    W bits stored)."""
    _fields_ = [("window", ctypes.c_uint32), ("min_len", ctypes.c_uint32),
                ("max_len", ctypes.c_uint32), ("block", ctypes.c_uint32),
                ("dict", ctypes.c_uint32)]


# the paper's LZSS configuration "1024/24/12/8" with the stored-prefix window
PAPER_LZSS = (1024, 12, 24, 8, 2)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction; integer code)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_LZSS), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = f"{_LIB}.tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC, _SRC_LZSS])
        os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    u64 = ctypes.c_uint64
    u32 = ctypes.c_uint32
    lib.oracle_histogram.restype = None
    lib.oracle_histogram.argtypes = [u8p, u64, u64p]
    lib.oracle_code_lengths.restype = ctypes.c_int
    lib.oracle_code_lengths.argtypes = [u64p, u8p]
    lib.oracle_code_lengths_limited.restype = ctypes.c_int
    lib.oracle_code_lengths_limited.argtypes = [u64p, u32, u8p]
    lib.oracle_canonical_codes.restype = None
    lib.oracle_canonical_codes.argtypes = [u8p, u32p]
    lib.oracle_max_stream_size.restype = u64
    lib.oracle_max_stream_size.argtypes = [u64, u32]
    lib.oracle_chunk_offsets.restype = ctypes.c_int
    lib.oracle_chunk_offsets.argtypes = [u8p, u64, u32, u8p, u64p, u64p]
    lib.oracle_pack_bits.restype = ctypes.c_int
    lib.oracle_pack_bits.argtypes = [u8p, u64, u8p, u32p, u64, u64p]
    lib.oracle_encode.restype = ctypes.c_int
    lib.oracle_encode.argtypes = [u8p, u64, u32, u8p, u8p, u64, u64p]
    lib.oracle_compress.restype = ctypes.c_int
    lib.oracle_compress.argtypes = [u8p, u64, u32, u8p, u64, u64p]
    lib.oracle_decode.restype = ctypes.c_int
    lib.oracle_decode.argtypes = [u8p, u64, u8p, u64, u64p]
    lib.oracle_bwt.restype = ctypes.c_int
    lib.oracle_bwt.argtypes = [u8p, u64, u32, u8p, u32p]
    lib.oracle_ibwt.restype = ctypes.c_int
    lib.oracle_ibwt.argtypes = [u8p, u64, u32, u32p, u8p]
    lib.oracle_mtf.restype = ctypes.c_int
    lib.oracle_mtf.argtypes = [u8p, u64, u32, u8p]
    lib.oracle_imtf.restype = ctypes.c_int
    lib.oracle_imtf.argtypes = [u8p, u64, u32, u8p]
    lp = ctypes.POINTER(LzssParams)
    lib.oracle_lzss_params_ok.restype = ctypes.c_int
    lib.oracle_lzss_params_ok.argtypes = [lp]
    lib.oracle_lzss_max_bits.restype = u64
    lib.oracle_lzss_max_bits.argtypes = [u64, lp]
    lib.oracle_lzss_encode.restype = ctypes.c_int
    lib.oracle_lzss_encode.argtypes = [u8p, u64, lp, u8p, u64, u64p]
    lib.oracle_lzss_decode.restype = ctypes.c_int
    lib.oracle_lzss_decode.argtypes = [u8p, u64, lp, u8p, u64]
    lib.oracle_lzss_segmented_max_size.restype = u64
    lib.oracle_lzss_segmented_max_size.argtypes = [u64, u64, lp]
    lib.oracle_lzss_segmented_compress.restype = ctypes.c_int
    lib.oracle_lzss_segmented_compress.argtypes = [u8p, u64, u64, lp, u8p, u64, u64p]
    lib.oracle_lzss_segmented_decompress.restype = ctypes.c_int
    lib.oracle_lzss_segmented_decompress.argtypes = [u8p, u64, u8p, u64, u64p]
    return lib

def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def use_library(path: str):
    """Route every call of this module to another build of ``huff_oracle.c``
    (the mutation tests compile copies with one planted mistake) for the
    duration of the ``with`` block."""
    global _lib
    saved = _load()
    _lib = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _bytes(x) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.uint8)).reshape(-1)
    return a if a.size else np.zeros(1, dtype=np.uint8)[:0]


def histogram(x) -> np.ndarray:
    """Byte counts, u64[256] (Method 1's probability-of-occurrence step)."""
    a = _bytes(x)
    h = np.zeros(256, dtype=np.uint64)
    _load().oracle_histogram(_p(a, ctypes.c_uint8), a.size, _p(h, ctypes.c_uint64))
    return h


def code_lengths(hist):
    """(status, len u8[256]) from the (weight, id)-ordered merge tree."""
    h = np.ascontiguousarray(np.asarray(hist, dtype=np.uint64))
    assert h.size == 256
    ln = np.zeros(256, dtype=np.uint8)
    st = _load().oracle_code_lengths(_p(h, ctypes.c_uint64), _p(ln, ctypes.c_uint8))
    return st, ln


def code_lengths_limited(hist, limit: int):
    """(status, len u8[256]): optimal code lengths of at most `limit` bits
    (the Huffman lengths when they fit, else package-merge)."""
    h = np.ascontiguousarray(np.asarray(hist, dtype=np.uint64))
    assert h.size == 256
    ln = np.zeros(256, dtype=np.uint8)
    st = _load().oracle_code_lengths_limited(_p(h, ctypes.c_uint64), limit,
                                             _p(ln, ctypes.c_uint8))
    return st, ln


def canonical_codes(lengths) -> np.ndarray:
    ln = np.ascontiguousarray(np.asarray(lengths, dtype=np.uint8))
    code = np.zeros(256, dtype=np.uint32)
    _load().oracle_canonical_codes(_p(ln, ctypes.c_uint8), _p(code, ctypes.c_uint32))
    return code


def max_stream_size(n: int, cs: int = DEFAULT_CHUNK) -> int:
    return int(_load().oracle_max_stream_size(n, cs))


def chunk_offsets(x, lengths, cs: int = DEFAULT_CHUNK):
    """(status, off u64[C], total_bits) of the concatenated codes."""
    a = _bytes(x)
    ln = np.ascontiguousarray(np.asarray(lengths, dtype=np.uint8))
    chunks = (a.size + cs - 1) // cs if cs else 0
    off = np.zeros(max(chunks, 1), dtype=np.uint64)
    tb = ctypes.c_uint64(0)
    st = _load().oracle_chunk_offsets(_p(a, ctypes.c_uint8), a.size, cs, _p(ln, ctypes.c_uint8),
                                      _p(off, ctypes.c_uint64), ctypes.byref(tb))
    return st, off[:chunks], int(tb.value)


def pack_bits(x, lengths):
    """(status, u32 words, bits): the codes of x concatenated MSB first from bit 0."""
    a = _bytes(x)
    ln = np.ascontiguousarray(np.asarray(lengths, dtype=np.uint8))
    nwords = (a.size * MAX_CODE_LEN + 31) // 32
    words = np.zeros(max(nwords, 1), dtype=np.uint32)
    bits = ctypes.c_uint64(0)
    st = _load().oracle_pack_bits(_p(a, ctypes.c_uint8), a.size, _p(ln, ctypes.c_uint8),
                                  _p(words, ctypes.c_uint32), words.size, ctypes.byref(bits))
    nb = int(bits.value)
    return st, words[:(nb + 31) // 32], nb


def encode(x, lengths, cs: int = DEFAULT_CHUNK, cap: int | None = None):
    """(status, stream bytes, needed bytes) for a given codebook (lengths)."""
    a = _bytes(x)
    ln = np.ascontiguousarray(np.asarray(lengths, dtype=np.uint8))
    if cap is None:
        cap = max_stream_size(a.size, cs) if cs else HEADER_BYTES
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    ob = ctypes.c_uint64(0)
    st = _load().oracle_encode(_p(a, ctypes.c_uint8), a.size, cs, _p(ln, ctypes.c_uint8),
                               _p(out, ctypes.c_uint8), cap, ctypes.byref(ob))
    need = int(ob.value)
    return st, (out[:need] if st == OK else out[:0]), need


def compress(x, cs: int = DEFAULT_CHUNK, cap: int | None = None):
    """(status, stream bytes): histogram + lengths + canonical codes + encode."""
    a = _bytes(x)
    if cap is None:
        cap = max_stream_size(a.size, cs) if cs else HEADER_BYTES
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    ob = ctypes.c_uint64(0)
    st = _load().oracle_compress(_p(a, ctypes.c_uint8), a.size, cs, _p(out, ctypes.c_uint8),
                                 cap, ctypes.byref(ob))
    return st, (out[:int(ob.value)] if st == OK else out[:0])


def decode(stream, cap: int | None = None):
    """(status, decoded bytes, n from the header)."""
    s = _bytes(stream)
    if cap is None:
        cap = int.from_bytes(bytes(s[256:264]), "little") if s.size >= 264 else 0
        cap = min(cap, 1 << 34)
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    n = ctypes.c_uint64(0)
    st = _load().oracle_decode(_p(s, ctypes.c_uint8), s.size, _p(out, ctypes.c_uint8), cap,
                               ctypes.byref(n))
    nn = int(n.value)
    return st, (out[:nn] if st == OK else out[:0]), nn


# ---------------------------------------------------------------- segmented container
def _al16(v: int) -> int:
    return (v + 15) & ~15


def segmented_compress(x, segment_bytes: int, cs: int = DEFAULT_CHUNK):
    """(status, container bytes): the paper's Method 2 taken literally
    (Section III-A) -- the input cut into segments with ids, each segment
    compressed alone with its own codebook by `compress`, the streams laid
    out behind a header and a start table (layout in include/huff.h:
    n, segment_bytes, count, start[0..count], streams at multiples of 16,
    zero bytes between them)."""
    a = _bytes(x)
    n = a.size
    if segment_bytes < 16 or segment_bytes % 16:
        return ERR_INVALID_ARG, np.zeros(0, dtype=np.uint8)
    count = (n + segment_bytes - 1) // segment_bytes if n else 0
    streams = []
    for i in range(count):
        st, s = compress(a[i * segment_bytes:(i + 1) * segment_bytes], cs)
        if st != OK:
            return st, np.zeros(0, dtype=np.uint8)
        streams.append(s)
    header = _al16(24 + 8 * (count + 1))
    start = [header]
    for s in streams:
        start.append(start[-1] + _al16(s.size))
    out = np.zeros(start[-1], dtype=np.uint8)
    out[0:24] = np.frombuffer(np.array([n, segment_bytes, count], dtype="<u8").tobytes(),
                              np.uint8)
    out[24:24 + 8 * (count + 1)] = np.frombuffer(np.array(start, dtype="<u8").tobytes(),
                                                 np.uint8)
    for i, s in enumerate(streams):
        out[start[i]:start[i] + s.size] = s
    return OK, out


def segmented_decompress(c, cap: int | None = None):
    """(status, decoded bytes, n): validate the header and start table,
    decode every segment with `decode` and check it decodes to its own
    size; any failure is ERR_CORRUPT, n > cap is ERR_CAPACITY."""
    c = _bytes(c)
    empty = np.zeros(0, dtype=np.uint8)
    if c.size < 32:
        return ERR_CORRUPT, empty, 0
    n, seg, count = (int(v) for v in np.frombuffer(c[:24].tobytes(), "<u8"))
    if seg < 16 or seg % 16 or count != ((n + seg - 1) // seg if n else 0) or \
            count > (c.size - 32) // 8:
        return ERR_CORRUPT, empty, 0
    start = [int(v) for v in np.frombuffer(c[24:24 + 8 * (count + 1)].tobytes(), "<u8")]
    if start[0] != _al16(24 + 8 * (count + 1)) or start[-1] > c.size or \
            any(s % 16 for s in start[:-1]) or any(b < a for a, b in zip(start, start[1:])):
        return ERR_CORRUPT, empty, 0
    if cap is not None and n > cap:
        return ERR_CAPACITY, empty, n
    out = np.zeros(n, dtype=np.uint8)
    for i in range(count):
        want = seg if i + 1 < count else n - (count - 1) * seg
        st, back, m = decode(c[start[i]:start[i + 1]], cap=want)
        if st != OK or m != want:
            return ERR_CORRUPT, empty, n
        out[i * seg:i * seg + want] = back
    return OK, out, n


def bwt(x, block: int):
    """Method 3's block-sorting transform of every `block`-byte block:
    (last column bytes, primary index per block)."""
    a = _bytes(x)
    n = a.size
    count = (n + block - 1) // block if block > 0 else 0
    L = np.zeros(n, dtype=np.uint8)
    prim = np.zeros(max(count, 1), dtype=np.uint32)
    st = _load().oracle_bwt(_p(a, ctypes.c_uint8), n, block, _p(L, ctypes.c_uint8),
                            _p(prim, ctypes.c_uint32))
    if st != OK:
        raise ValueError(f"oracle_bwt status {st}")
    return L, prim[:count]


def ibwt(L, block: int, primary):
    """Inverse of :func:`bwt`."""
    a = _bytes(L)
    n = a.size
    count = (n + block - 1) // block if block > 0 else 0
    prim = np.ascontiguousarray(primary, dtype=np.uint32)
    if prim.size < count:
        raise ValueError("one primary index per block is needed")
    if prim.size == 0:
        prim = np.zeros(1, dtype=np.uint32)
    out = np.zeros(n, dtype=np.uint8)
    st = _load().oracle_ibwt(_p(a, ctypes.c_uint8), n, block, _p(prim, ctypes.c_uint32),
                             _p(out, ctypes.c_uint8))
    if st != OK:
        raise ValueError(f"oracle_ibwt status {st}")
    return out


def mtf(x, block: int):
    """Move-to-front coding of every `block`-byte block (list 0..255 at each
    block start)."""
    a = _bytes(x)
    out = np.zeros(a.size, dtype=np.uint8)
    st = _load().oracle_mtf(_p(a, ctypes.c_uint8), a.size, block, _p(out, ctypes.c_uint8))
    if st != OK:
        raise ValueError(f"oracle_mtf status {st}")
    return out


def imtf(idx, block: int):
    """Inverse of :func:`mtf`."""
    a = _bytes(idx)
    out = np.zeros(a.size, dtype=np.uint8)
    st = _load().oracle_imtf(_p(a, ctypes.c_uint8), a.size, block, _p(out, ctypes.c_uint8))
    if st != OK:
        raise ValueError(f"oracle_imtf status {st}")
    return out


# ---------------------------------------------------------------- Method 3 container
def m3_compress(x, block: int, segment_bytes: int, cs: int = DEFAULT_CHUNK, mtf_stage: bool = False):
    """(status, container bytes): Method 3 (Section III-A) -- the
    block-sorting transform of every `block`-byte block, optionally
    move-to-front coding of every block, then Method 2's segmented coder (one
    codebook per segment) over the result.  Layout (include/huff.h): n (u64),
    block (u32), count (u32), stages (u32: bit 0 = move-to-front), one u32
    primary index per block, zero bytes up to a multiple of 16, then the
    segmented container."""
    a = _bytes(x)
    n = a.size
    empty = np.zeros(0, dtype=np.uint8)
    if block < 1 or block >= 1 << 32:
        return ERR_INVALID_ARG, empty
    L, prim = bwt(a, block)
    if mtf_stage:
        L = mtf(L, block)
    st, seg = segmented_compress(L, segment_bytes, cs)
    if st != OK:
        return st, empty
    count = prim.size
    head = _al16(20 + 4 * count)
    out = np.zeros(head + seg.size, dtype=np.uint8)
    out[0:8] = np.frombuffer(np.array([n], dtype="<u8").tobytes(), np.uint8)
    out[8:20] = np.frombuffer(np.array([block, count, 1 if mtf_stage else 0], dtype="<u4")
                              .tobytes(), np.uint8)
    out[20:20 + 4 * count] = np.frombuffer(prim.astype("<u4").tobytes(), np.uint8)
    out[head:] = seg
    return OK, out


def m3_decompress(c, cap: int | None = None):
    """(status, bytes, n): validate the header (stages other than bit 0 are
    corrupt), decode the segmented container, check it holds n bytes and
    every primary index lies inside its block, undo move-to-front if it was
    applied, then invert the transform."""
    c = _bytes(c)
    empty = np.zeros(0, dtype=np.uint8)
    if c.size < 20:
        return ERR_CORRUPT, empty, 0
    n = int(np.frombuffer(c[0:8].tobytes(), "<u8")[0])
    block, count, stages = (int(v) for v in np.frombuffer(c[8:20].tobytes(), "<u4"))
    if block < 1 or count != (n + block - 1) // block or stages > 1 or \
            20 + 4 * count > c.size:
        return ERR_CORRUPT, empty, 0
    if cap is not None and n > cap:
        return ERR_CAPACITY, empty, n
    prim = np.frombuffer(c[20:20 + 4 * count].tobytes(), "<u4").astype(np.uint32)
    for i in range(count):
        if int(prim[i]) >= min(block, n - i * block):
            return ERR_CORRUPT, empty, n
    head = _al16(20 + 4 * count)
    st, L, m = segmented_decompress(c[head:], cap=n)
    if st != OK or m != n:
        return ERR_CORRUPT, empty, n
    if stages & 1:
        L = imtf(L, block)
    return OK, ibwt(L, block, prim), n


# ---------------------------------------------------------------- LZSS (Section III-B)
def _lzss_params(params):
    w, lmin, lmax, blk, dct = params
    return LzssParams(w, lmin, lmax, blk, dct)


def lzss_encode(x, params=PAPER_LZSS):
    """LZSS Method 1 of one segment: (status, code bytes, code bits).
    params = (window, min_len, max_len, block, dict)."""
    a = _bytes(x)
    P = _lzss_params(params)
    lib = _load()
    if not lib.oracle_lzss_params_ok(ctypes.byref(P)):
        return ERR_INVALID_ARG, np.zeros(0, np.uint8), 0
    cap = (int(lib.oracle_lzss_max_bits(a.size, ctypes.byref(P))) + 7) // 8
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    bits = ctypes.c_uint64(0)
    st = lib.oracle_lzss_encode(_p(a, ctypes.c_uint8), a.size, ctypes.byref(P),
                                _p(out, ctypes.c_uint8), cap, ctypes.byref(bits))
    nb = int(bits.value)
    return st, out[:(nb + 7) // 8], nb


def lzss_decode(code, bits: int, m: int, params=PAPER_LZSS):
    """Inverse of :func:`lzss_encode` for an m-byte segment: (status, bytes)."""
    c = _bytes(code)
    if c.size == 0:
        c = np.zeros(1, np.uint8)
    P = _lzss_params(params)
    out = np.zeros(max(m, 1), dtype=np.uint8)
    st = _load().oracle_lzss_decode(_p(c, ctypes.c_uint8), bits, ctypes.byref(P),
                                    _p(out, ctypes.c_uint8), m)
    return st, out[:m]


def lzss_segmented_max_size(n: int, seg: int, params=PAPER_LZSS) -> int:
    P = _lzss_params(params)
    return int(_load().oracle_lzss_segmented_max_size(n, seg, ctypes.byref(P)))


def lzss_segmented_compress(x, seg: int, params=PAPER_LZSS):
    """LZSS Method 2: (status, container bytes)."""
    a = _bytes(x)
    P = _lzss_params(params)
    cap = lzss_segmented_max_size(a.size, seg, params)
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    ob = ctypes.c_uint64(0)
    st = _load().oracle_lzss_segmented_compress(_p(a, ctypes.c_uint8), a.size, seg,
                                                ctypes.byref(P), _p(out, ctypes.c_uint8), cap,
                                                ctypes.byref(ob))
    return st, (out[:int(ob.value)] if st == OK else out[:0])


def lzss_segmented_decompress(c, cap: int | None = None):
    """Inverse of :func:`lzss_segmented_compress`: (status, bytes, n)."""
    a = _bytes(c)
    if cap is None:
        cap = int.from_bytes(bytes(a[0:8]), "little") if a.size >= 8 else 0
        cap = min(cap, 1 << 34)
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    n = ctypes.c_uint64(0)
    st = _load().oracle_lzss_segmented_decompress(_p(a, ctypes.c_uint8), a.size,
                                                  _p(out, ctypes.c_uint8), cap, ctypes.byref(n))
    nn = int(n.value)
    return st, (out[:nn] if st == OK else out[:0]), nn
