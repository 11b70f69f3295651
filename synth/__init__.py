"""Seeded synthetic inputs for the tests and the benchmark.

The generators live in ``synth.c`` (splitmix64 streams, no Huffman
arithmetic) and are compiled with gcc into ``libhuffsynth.so`` beside it on
first use.  The same seeded inputs feed both the CPU oracle and the CUDA
path; nothing here computes any part of the method.

Workloads (sizes, distributions and seeds):

* ``zipf_ascii``: bytes i.i.d. Zipf(s=1.1) over the 96 codes 32..127, rank
  order equal to byte order (1 MiB, seed 0 in the small parity case).
* ``text``: synthetic English-like text of the scale of the paper's ~45 MB
  corpus (Section III-A): 50,000 random lowercase words, Zipf(1.0) word
  frequencies, punctuation after 5% of words, a newline once a line reaches
  80 characters (64 MiB and 1 GiB, seed 1).
* ``uniform`` / ``geometric`` / ``single``: the distribution stress inputs
  (uniform bytes, P(k) = 2^-(k+1), one repeated byte 0x61; seeds 40, 41).
* ``bitstream``: a stand-in for the FPGA configuration bitstreams the
  paper's LZSS section codes (Section III-B; not available): zero runs,
  repeated frame templates with a few flipped bits, random stretches
  (256 MiB, seed 7, in 64 KiB segments for the GPU LZSS measurement).
* ``log_uniform_sizes`` and ``batch_seed``: the sizes and per-buffer seeds of
  the batched workload (4096 buffers, 1 KiB..4 MiB, sizes seed 3).
* ``poisson_trace``: open-loop arrivals for the served workload (seed 5).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libhuffsynth.so")
_lib = None

MiB = 1 << 20
GiB = 1 << 30


def build(force: bool = False) -> str:
    """Compile synth.c into libhuffsynth.so (gcc, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = f"{_LIB}.tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.synth_splitmix64.restype = ctypes.c_uint64
        lib.synth_splitmix64.argtypes = [ctypes.c_uint64]
        lib.synth_zipf_ascii.restype = ctypes.c_int
        lib.synth_zipf_ascii.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double]
        lib.synth_text.restype = ctypes.c_int
        lib.synth_text.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64]
        for name in ("synth_uniform", "synth_geometric"):
            fn = getattr(lib, name)
            fn.restype = None
            fn.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_geometric_p.restype = None
        lib.synth_geometric_p.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double]
        lib.synth_bitstream.restype = ctypes.c_int
        lib.synth_bitstream.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_shuffle.restype = None
        lib.synth_shuffle.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_log_uniform_sizes.restype = None
        lib.synth_log_uniform_sizes.argtypes = [u64p, ctypes.c_uint32, ctypes.c_uint64,
                                                ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_poisson_trace.restype = None
        lib.synth_poisson_trace.argtypes = [f64p, u8p, u64p, ctypes.c_uint32, ctypes.c_uint64,
                                            ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _out(n: int, out: np.ndarray | None) -> np.ndarray:
    if out is None:
        return np.empty(int(n), dtype=np.uint8)
    assert out.dtype == np.uint8 and out.flags.c_contiguous and out.size >= n
    return out


def splitmix64(state: int) -> int:
    """One splitmix64 output for the given state (state advanced once)."""
    return int(_load().synth_splitmix64(ctypes.c_uint64(state & (2**64 - 1))))


def zipf_ascii(n: int, seed: int = 0, s: float = 1.1, out=None) -> np.ndarray:
    a = _out(n, out)
    if _load().synth_zipf_ascii(_ptr(a, ctypes.c_uint8), n, seed, s) != 0:
        raise MemoryError("synth_zipf_ascii")
    return a[:n]


def text(n: int, seed: int = 1, out=None) -> np.ndarray:
    a = _out(n, out)
    if _load().synth_text(_ptr(a, ctypes.c_uint8), n, seed) != 0:
        raise MemoryError("synth_text")
    return a[:n]


def uniform(n: int, seed: int = 40, out=None) -> np.ndarray:
    a = _out(n, out)
    _load().synth_uniform(_ptr(a, ctypes.c_uint8), n, seed)
    return a[:n]


def geometric(n: int, seed: int = 41, out=None) -> np.ndarray:
    a = _out(n, out)
    _load().synth_geometric(_ptr(a, ctypes.c_uint8), n, seed)
    return a[:n]


def geometric_p(n: int, seed: int, p: float, out=None) -> np.ndarray:
    a = _out(n, out)
    _load().synth_geometric_p(_ptr(a, ctypes.c_uint8), n, seed, p)
    return a[:n]


def bitstream(n: int, seed: int = 7, out=None) -> np.ndarray:
    """Stand-in for FPGA configuration bitstreams (LZSS inputs): zero runs,
    templates repeated with a few flipped bits, random stretches."""
    a = _out(n, out)
    if _load().synth_bitstream(_ptr(a, ctypes.c_uint8), n, seed) != 0:
        raise MemoryError("synth_bitstream")
    return a[:n]


def single(n: int, byte: int = 0x61, out=None) -> np.ndarray:
    a = _out(n, out)
    a[:n] = byte
    return a[:n]


def shuffle(a: np.ndarray, seed: int) -> np.ndarray:
    """Seeded Fisher-Yates shuffle of a uint8 array, in place."""
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    _load().synth_shuffle(_ptr(a, ctypes.c_uint8), a.size, seed)
    return a


def counted(counts, seed: int) -> np.ndarray:
    """Bytes with exactly counts[b] copies of byte b, in seeded random order
    (for example Fibonacci counts, the deepest possible code tree)."""
    counts = [int(c) for c in counts]
    a = np.repeat(np.arange(len(counts), dtype=np.uint8), counts)
    return shuffle(np.ascontiguousarray(a), seed)


def log_uniform_sizes(count: int, seed: int = 3, lo: int = 1024, hi: int = 4 * MiB) -> np.ndarray:
    s = np.empty(count, dtype=np.uint64)
    _load().synth_log_uniform_sizes(_ptr(s, ctypes.c_uint64), count, seed, lo, hi)
    return s


def batch_seed(i: int) -> int:
    """Seed of buffer i in the batched workload: splitmix64(1 xor (i + 1))."""
    return splitmix64(1 ^ (i + 1))


def poisson_trace(count: int, seed: int = 5, lam: float = 5000.0,
                  lo: int = 4096, hi: int = 16 * MiB):
    """Arrival times (s), ops (0 = compress, 1 = decompress) and sizes."""
    t = np.empty(count, dtype=np.float64)
    op = np.empty(count, dtype=np.uint8)
    s = np.empty(count, dtype=np.uint64)
    _load().synth_poisson_trace(_ptr(t, ctypes.c_double), _ptr(op, ctypes.c_uint8),
                                _ptr(s, ctypes.c_uint64), count, seed, lam, lo, hi)
    return t, op, s


# Named single-buffer workloads: name -> (generator, size, seed)
WORKLOADS = {
    "zipf_ascii_1m": (zipf_ascii, 1 * MiB, 0),
    "text_64m": (text, 64 * MiB, 1),
    "text_1g": (text, 1 * GiB, 1),
    "uniform_1g": (uniform, 1 * GiB, 40),
    "geometric_1g": (geometric, 1 * GiB, 41),
    "single_1g": (lambda n, seed, out=None: single(n, 0x61, out=out), 1 * GiB, 42),
    "bitstream_256m": (bitstream, 256 * MiB, 7),
}


def make(name: str, n: int | None = None, out=None) -> np.ndarray:
    """Generate a named workload (optionally at another size n)."""
    gen, size, seed = WORKLOADS[name]
    size = size if n is None else n
    return gen(size, seed, out=out)
