"""GB300 Huffman codec: Python binding of libhuff.so.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current CUDA stream.  The
functions named ``huff_*`` mirror the C ABI in ``include/huff.h`` one to one;
``compress`` / ``decompress`` are conveniences that size the buffers,
synchronise once and raise on a non-zero status.

The library must have been built (``python -m paper_2306_11070_gb300.build``
or ``__graft_entry__.build()``); there is no fallback of any kind, and every
call raises if ``libhuff.so`` is missing.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhuff.so")

HUFF_OK = 0
HUFF_ERR_INVALID_ARG = -1
HUFF_ERR_CODE_TOO_LONG = -2
HUFF_ERR_CAPACITY = -3
HUFF_ERR_CORRUPT_STREAM = -4
HUFF_ERR_CUDA = -5
HUFF_ERR_TIMEOUT = -6
HUFF_ERR_BUDGET = -7
HUFF_ERR_UNSUPPORTED = -8

HEADER_BYTES = 272
DEFAULT_CHUNK_SYMBOLS = 16384
CODEBOOK_BYTES = 1288  # sizeof(huff_codebook_t)

_lib = None

HUFF_BATCH_COMPRESS = 0
HUFF_BATCH_DECOMPRESS = 1
HUFF_TUNE_FORCE = 1
HUFF_TUNE_ROUND_TRIP = 2


class BatchDesc(ctypes.Structure):
    """huff_batch_desc_t"""
    _fields_ = [("d_in", ctypes.c_void_p), ("in_bytes", ctypes.c_uint64),
                ("d_out", ctypes.c_void_p), ("out_cap", ctypes.c_uint64),
                ("d_out_bytes", ctypes.c_void_p), ("d_status", ctypes.c_void_p)]


class BatchParams(ctypes.Structure):
    """huff_batch_params_t"""
    _fields_ = [("chunk_symbols", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("decode_lanes", ctypes.c_uint32), ("use_graph", ctypes.c_uint32),
                ("barrier_extra", ctypes.c_uint32)]


class LzssParams(ctypes.Structure):
    """huff_lzss_params_t"""
    _fields_ = [("window", ctypes.c_uint32), ("min_len", ctypes.c_uint32),
                ("max_len", ctypes.c_uint32), ("block", ctypes.c_uint32),
                ("dict", ctypes.c_uint32)]


# the paper's LZSS configuration "1024/24/12/8" (window, shortest and longest
# match, literal block, in bits) with the stored-prefix window
LZSS_PAPER = (1024, 12, 24, 8, 2)


class ServerConfig(ctypes.Structure):
    """huff_server_cfg_t"""
    _fields_ = [("device_budget", ctypes.c_uint64), ("max_rounds", ctypes.c_uint32),
                ("max_batch", ctypes.c_uint32), ("chunk_symbols", ctypes.c_uint32),
                ("decode_lanes", ctypes.c_uint32)]


class Request(ctypes.Structure):
    """huff_request_t"""
    _fields_ = [("op", ctypes.c_int32), ("h_in", ctypes.c_void_p), ("in_bytes", ctypes.c_uint64),
                ("h_out", ctypes.c_void_p), ("out_cap", ctypes.c_uint64)]


class Result(ctypes.Structure):
    """huff_result_t"""
    _fields_ = [("done", ctypes.c_int32), ("status", ctypes.c_int32),
                ("out_bytes", ctypes.c_uint64), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class HuffError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        super().__init__(f"{where}: {huff_status_str(status)} ({status})" if where else
                         f"{huff_status_str(status)} ({status})")


def lib() -> ctypes.CDLL:
    """The loaded libhuff.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2306_11070_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
        L.huff_status_str.restype = ctypes.c_char_p
        L.huff_status_str.argtypes = [i32]
        L.huff_version.restype = ctypes.c_int
        L.huff_version.argtypes = []
        L.huff_max_stream_size.restype = u64
        L.huff_max_stream_size.argtypes = [u64, u32]
        L.huff_workspace_size.restype = u64
        L.huff_workspace_size.argtypes = [u64, u32]
        L.huff_histogram.restype = i32
        L.huff_histogram.argtypes = [vp, u64, vp, vp]
        L.huff_unit_hist_size.restype = u64
        L.huff_unit_hist_size.argtypes = [u64]
        L.huff_histogram_units.restype = i32
        L.huff_histogram_units.argtypes = [vp, u64, vp, vp, vp]
        L.huff_encode_units.restype = i32
        L.huff_encode_units.argtypes = [vp, u64, vp, vp, u32, vp, u64, vp, vp, u64, vp, vp]
        L.huff_build_codebook.restype = i32
        L.huff_build_codebook.argtypes = [vp, vp, vp, vp]
        L.huff_build_codebook_limited.restype = i32
        L.huff_build_codebook_limited.argtypes = [vp, u32, vp, vp, vp]
        L.huff_encode.restype = i32
        L.huff_encode.argtypes = [vp, u64, vp, u32, vp, u64, vp, vp, u64, vp, vp]
        L.huff_encode_noalloc.restype = i32
        L.huff_encode_noalloc.argtypes = [vp, u64, vp, u32, vp, u64, vp, vp, vp]
        L.huff_decode.restype = i32
        L.huff_decode.argtypes = [vp, u64, vp, u64, vp, vp, vp]
        L.huff_compress.restype = i32
        L.huff_compress.argtypes = [vp, u64, u32, vp, u64, vp, vp, u64, vp, vp]
        L.huff_server_default_config.restype = None
        L.huff_server_default_config.argtypes = [ctypes.POINTER(ServerConfig)]
        L.huff_server_create.restype = i32
        L.huff_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
        L.huff_server_submit.restype = i32
        L.huff_server_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(u64)]
        L.huff_server_poll.restype = i32
        L.huff_server_poll.argtypes = [vp, u64, ctypes.POINTER(Result)]
        L.huff_server_wait.restype = i32
        L.huff_server_wait.argtypes = [vp, u64, u32, ctypes.POINTER(Result)]
        L.huff_server_release.restype = i32
        L.huff_server_release.argtypes = [vp, u64]
        L.huff_server_destroy.restype = None
        L.huff_server_destroy.argtypes = [vp]
        L.huff_batch_default_params.restype = None
        L.huff_batch_default_params.argtypes = [ctypes.POINTER(BatchParams)]
        L.huff_batch_plan.restype = i32
        L.huff_batch_plan.argtypes = [ctypes.POINTER(BatchDesc), u32, ctypes.c_int,
                                      ctypes.POINTER(BatchParams), ctypes.POINTER(vp)]
        L.huff_batch_run.restype = i32
        L.huff_batch_run.argtypes = [vp, vp]
        L.huff_batch_info.restype = i32
        L.huff_batch_info.argtypes = [vp, ctypes.POINTER(BatchParams), ctypes.POINTER(u32),
                                      ctypes.POINTER(i32)]
        L.huff_batch_destroy.restype = None
        L.huff_batch_destroy.argtypes = [vp]
        L.huff_segmented_max_size.restype = u64
        L.huff_segmented_max_size.argtypes = [u64, u64, u32]
        L.huff_segmented_workspace_size.restype = u64
        L.huff_segmented_workspace_size.argtypes = [u64, u64, u32]
        L.huff_segmented_compress.restype = i32
        L.huff_segmented_compress.argtypes = [vp, u64, u64, u32, vp, u64, vp, vp, u64, vp, vp]
        L.huff_segmented_decompress.restype = i32
        L.huff_segmented_decompress.argtypes = [vp, u64, vp, u64, vp, vp, vp]
        L.huff_bwt_workspace_size.restype = u64
        L.huff_bwt_workspace_size.argtypes = [u64, u32]
        L.huff_bwt_forward.restype = i32
        L.huff_bwt_forward.argtypes = [vp, u64, u32, vp, vp, vp, u64, vp, vp]
        L.huff_bwt_inverse.restype = i32
        L.huff_bwt_inverse.argtypes = [vp, u64, u32, vp, vp, vp, u64, vp, vp]
        L.huff_m3_max_size.restype = u64
        L.huff_m3_max_size.argtypes = [u64, u32, u64, u32]
        L.huff_m3_workspace_size.restype = u64
        L.huff_m3_workspace_size.argtypes = [u64, u32, u64, u32]
        L.huff_m3_compress.restype = i32
        L.huff_m3_compress.argtypes = [vp, u64, u32, u64, u32, u32, vp, u64, vp, vp, u64, vp, vp]
        L.huff_mtf_workspace_size.restype = u64
        L.huff_mtf_workspace_size.argtypes = [u64, u32]
        L.huff_mtf_forward.restype = i32
        L.huff_mtf_forward.argtypes = [vp, u64, u32, vp, vp, u64, vp]
        L.huff_mtf_inverse.restype = i32
        L.huff_mtf_inverse.argtypes = [vp, u64, u32, vp, vp, u64, vp]
        L.huff_m3_decompress_workspace_size.restype = u64
        L.huff_m3_decompress_workspace_size.argtypes = [u64, u32]
        L.huff_m3_decompress.restype = i32
        L.huff_m3_decompress.argtypes = [vp, u64, vp, u64, vp, vp, u64, vp, vp]
        L.huff_batch_autotune.restype = i32
        L.huff_batch_autotune.argtypes = [ctypes.POINTER(BatchDesc), u32, ctypes.c_int,
                                          ctypes.POINTER(BatchParams), u32,
                                          ctypes.POINTER(BatchParams), vp]
        lp = ctypes.POINTER(LzssParams)
        L.huff_lzss_max_size.restype = u64
        L.huff_lzss_max_size.argtypes = [u64, u64, lp]
        L.huff_lzss_workspace_size.restype = u64
        L.huff_lzss_workspace_size.argtypes = [u64, u64, lp]
        L.huff_lzss_compress.restype = i32
        L.huff_lzss_compress.argtypes = [vp, u64, u64, lp, vp, u64, vp, vp, u64, vp, vp]
        L.huff_lzss_decompress_workspace_size.restype = u64
        L.huff_lzss_decompress_workspace_size.argtypes = [u64]
        L.huff_lzss_decompress.restype = i32
        L.huff_lzss_decompress.argtypes = [vp, u64, vp, u64, vp, vp, u64, vp, vp]
        _lib = L
    return _lib


# ---------------------------------------------------------------- helpers
def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if isinstance(t, torch.Tensor):
        if not t.is_cuda:
            raise ValueError("device tensor expected")
        if not t.is_contiguous():
            raise ValueError("contiguous tensor expected")
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(int(t))


def _check(st: int, where: str):
    if st != HUFF_OK:
        raise HuffError(st, where)


def _u8(t: torch.Tensor) -> torch.Tensor:
    if t.dtype != torch.uint8:
        raise TypeError("uint8 tensor expected")
    return t.reshape(-1)


def huff_status_str(status: int) -> str:
    return lib().huff_status_str(int(status)).decode()


def huff_version() -> int:
    return int(lib().huff_version())


def huff_max_stream_size(n: int, chunk_symbols: int = DEFAULT_CHUNK_SYMBOLS) -> int:
    return int(lib().huff_max_stream_size(int(n), int(chunk_symbols)))


def huff_workspace_size(n: int, chunk_symbols: int = DEFAULT_CHUNK_SYMBOLS) -> int:
    return int(lib().huff_workspace_size(int(n), int(chunk_symbols)))


def new_status(device=None) -> torch.Tensor:
    """A zeroed int32 device status word."""
    return torch.zeros(1, dtype=torch.int32, device=device or "cuda")


# ---------------------------------------------------------------- C ABI mirror
def huff_histogram(d_in: torch.Tensor, d_hist: torch.Tensor | None = None, stream=None):
    """u64[256] byte counts (returned as int64 tensor bits)."""
    x = _u8(d_in)
    if d_hist is None:
        d_hist = torch.empty(256, dtype=torch.int64, device=x.device)
    _check(lib().huff_histogram(_ptr(x), x.numel(), _ptr(d_hist), _stream(stream)),
           "huff_histogram")
    return d_hist


def huff_unit_hist_size(n: int) -> int:
    return int(lib().huff_unit_hist_size(int(n)))


def huff_histogram_units(d_in: torch.Tensor, d_hist: torch.Tensor | None = None,
                         d_unit_hist: torch.Tensor | None = None, stream=None):
    """(u64[256] counts, u16[256] per 16 KiB unit) -- the latter as uint8 bytes."""
    x = _u8(d_in)
    if d_hist is None:
        d_hist = torch.empty(256, dtype=torch.int64, device=x.device)
    if d_unit_hist is None:
        d_unit_hist = torch.empty(max(huff_unit_hist_size(x.numel()), 16), dtype=torch.uint8,
                                  device=x.device)
    _check(lib().huff_histogram_units(_ptr(x), x.numel(), _ptr(d_hist), _ptr(d_unit_hist),
                                      _stream(stream)), "huff_histogram_units")
    return d_hist, d_unit_hist


def huff_build_codebook(d_hist: torch.Tensor, d_cb: torch.Tensor | None = None,
                        d_status: torch.Tensor | None = None, stream=None):
    """(codebook bytes uint8[1288], status int32[1])."""
    if d_cb is None:
        d_cb = torch.empty(CODEBOOK_BYTES, dtype=torch.uint8, device=d_hist.device)
    if d_status is None:
        d_status = new_status(d_hist.device)
    _check(lib().huff_build_codebook(_ptr(d_hist), _ptr(d_cb), _ptr(d_status), _stream(stream)),
           "huff_build_codebook")
    return d_cb, d_status


def huff_build_codebook_limited(d_hist: torch.Tensor, max_len: int,
                                d_cb: torch.Tensor | None = None,
                                d_status: torch.Tensor | None = None, stream=None):
    """(codebook bytes, status): codes of at most max_len bits."""
    if d_cb is None:
        d_cb = torch.empty(CODEBOOK_BYTES, dtype=torch.uint8, device=d_hist.device)
    if d_status is None:
        d_status = new_status(d_hist.device)
    _check(lib().huff_build_codebook_limited(_ptr(d_hist), max_len, _ptr(d_cb), _ptr(d_status),
                                             _stream(stream)), "huff_build_codebook_limited")
    return d_cb, d_status


def huff_encode(d_in: torch.Tensor, d_cb: torch.Tensor, chunk_symbols: int = DEFAULT_CHUNK_SYMBOLS,
                d_out: torch.Tensor | None = None, d_out_bytes: torch.Tensor | None = None,
                d_ws: torch.Tensor | None = None, d_status: torch.Tensor | None = None,
                stream=None, out_cap: int | None = None):
    """(stream buffer, out_bytes int64[1], status int32[1]); sizes not read back."""
    x = _u8(d_in)
    n = x.numel()
    dev = x.device
    if d_out is None:
        d_out = torch.empty(huff_max_stream_size(n, chunk_symbols), dtype=torch.uint8, device=dev)
    if d_out_bytes is None:
        d_out_bytes = torch.zeros(1, dtype=torch.int64, device=dev)
    if d_ws is None:
        d_ws = torch.empty(max(huff_workspace_size(n, chunk_symbols), 256), dtype=torch.uint8,
                           device=dev)
    if d_status is None:
        d_status = new_status(dev)
    cap = d_out.numel() if out_cap is None else int(out_cap)
    _check(lib().huff_encode(_ptr(x), n, _ptr(d_cb), int(chunk_symbols), _ptr(d_out), cap,
                             _ptr(d_out_bytes), _ptr(d_ws), d_ws.numel(), _ptr(d_status),
                             _stream(stream)), "huff_encode")
    return d_out, d_out_bytes, d_status


def huff_encode_units(d_in: torch.Tensor, d_cb: torch.Tensor, d_unit_hist: torch.Tensor,
                      chunk_symbols: int = DEFAULT_CHUNK_SYMBOLS,
                      d_out: torch.Tensor | None = None, d_out_bytes: torch.Tensor | None = None,
                      d_ws: torch.Tensor | None = None, d_status: torch.Tensor | None = None,
                      stream=None, out_cap: int | None = None):
    """huff_encode with the unit histograms of huff_histogram_units."""
    x = _u8(d_in)
    n = x.numel()
    dev = x.device
    if d_out is None:
        d_out = torch.empty(huff_max_stream_size(n, chunk_symbols), dtype=torch.uint8, device=dev)
    if d_out_bytes is None:
        d_out_bytes = torch.zeros(1, dtype=torch.int64, device=dev)
    if d_ws is None:
        d_ws = torch.empty(max(huff_workspace_size(n, chunk_symbols), 256), dtype=torch.uint8,
                           device=dev)
    if d_status is None:
        d_status = new_status(dev)
    cap = d_out.numel() if out_cap is None else int(out_cap)
    _check(lib().huff_encode_units(_ptr(x), n, _ptr(d_cb), _ptr(d_unit_hist), int(chunk_symbols),
                                   _ptr(d_out), cap, _ptr(d_out_bytes), _ptr(d_ws), d_ws.numel(),
                                   _ptr(d_status), _stream(stream)), "huff_encode_units")
    return d_out, d_out_bytes, d_status


def huff_encode_noalloc(d_in: torch.Tensor, d_cb: torch.Tensor,
                        chunk_symbols: int = DEFAULT_CHUNK_SYMBOLS,
                        d_out: torch.Tensor | None = None,
                        d_out_bytes: torch.Tensor | None = None,
                        d_status: torch.Tensor | None = None, stream=None,
                        out_cap: int | None = None):
    """huff_encode without a workspace (the library's fixed scratch array)."""
    x = _u8(d_in)
    n = x.numel()
    dev = x.device
    if d_out is None:
        d_out = torch.empty(huff_max_stream_size(n, chunk_symbols), dtype=torch.uint8, device=dev)
    if d_out_bytes is None:
        d_out_bytes = torch.zeros(1, dtype=torch.int64, device=dev)
    if d_status is None:
        d_status = new_status(dev)
    cap = d_out.numel() if out_cap is None else int(out_cap)
    _check(lib().huff_encode_noalloc(_ptr(x), n, _ptr(d_cb), int(chunk_symbols), _ptr(d_out), cap,
                                     _ptr(d_out_bytes), _ptr(d_status), _stream(stream)),
           "huff_encode_noalloc")
    return d_out, d_out_bytes, d_status


def huff_decode(d_stream: torch.Tensor, stream_bytes: int | None = None,
                d_out: torch.Tensor | None = None, out_cap: int | None = None,
                d_n: torch.Tensor | None = None, d_status: torch.Tensor | None = None,
                stream=None):
    """(output buffer, n int64[1], status int32[1]).  Without d_out the
    header's n is read back once to size the output."""
    s = _u8(d_stream)
    nbytes = s.numel() if stream_bytes is None else int(stream_bytes)
    dev = s.device
    if d_out is None:
        n = int.from_bytes(bytes(s[256:264].cpu().numpy()), "little") if s.numel() >= 264 else 0
        d_out = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
        out_cap = n if out_cap is None else out_cap
    if out_cap is None:
        out_cap = d_out.numel()
    if d_n is None:
        d_n = torch.zeros(1, dtype=torch.int64, device=dev)
    if d_status is None:
        d_status = new_status(dev)
    _check(lib().huff_decode(_ptr(s), nbytes, _ptr(d_out), int(out_cap), _ptr(d_n),
                             _ptr(d_status), _stream(stream)), "huff_decode")
    return d_out, d_n, d_status


def huff_compress(d_in: torch.Tensor, chunk_symbols: int = DEFAULT_CHUNK_SYMBOLS,
                  d_out: torch.Tensor | None = None, d_out_bytes: torch.Tensor | None = None,
                  d_ws: torch.Tensor | None = None, d_status: torch.Tensor | None = None,
                  stream=None, out_cap: int | None = None):
    """(stream buffer, out_bytes int64[1], status int32[1]), no host sync."""
    x = _u8(d_in)
    n = x.numel()
    dev = x.device
    if d_out is None:
        d_out = torch.empty(huff_max_stream_size(n, chunk_symbols), dtype=torch.uint8, device=dev)
    if d_out_bytes is None:
        d_out_bytes = torch.zeros(1, dtype=torch.int64, device=dev)
    if d_ws is None:
        d_ws = torch.empty(huff_workspace_size(n, chunk_symbols), dtype=torch.uint8, device=dev)
    if d_status is None:
        d_status = torch.empty(1, dtype=torch.int32, device=dev)
    cap = d_out.numel() if out_cap is None else int(out_cap)
    _check(lib().huff_compress(_ptr(x), n, int(chunk_symbols), _ptr(d_out), cap,
                               _ptr(d_out_bytes), _ptr(d_ws), d_ws.numel(), _ptr(d_status),
                               _stream(stream)), "huff_compress")
    return d_out, d_out_bytes, d_status


# ---------------------------------------------------------------- batched engine
def huff_batch_default_params() -> BatchParams:
    p = BatchParams()
    lib().huff_batch_default_params(ctypes.byref(p))
    return p


class BatchPlan:
    """A planned batch (huff_batch_plan / huff_batch_run / huff_batch_destroy).

    `inputs` and `outputs` are lists of uint8 CUDA tensors; for compression
    the outputs must hold huff_max_stream_size bytes, for decompression the
    decoded size.  Per-buffer sizes and statuses are the int64 / int32
    tensors `out_bytes` and `status` (one entry per buffer).  The tensors
    must stay alive as long as the plan."""

    def __init__(self, inputs, outputs, op=HUFF_BATCH_COMPRESS, params: BatchParams | None = None,
                 in_bytes=None):
        count = len(inputs)
        assert count == len(outputs) and count > 0
        dev = inputs[0].device
        self.inputs, self.outputs = list(inputs), list(outputs)
        self.out_bytes = torch.zeros(count, dtype=torch.int64, device=dev)
        self.status = torch.zeros(count, dtype=torch.int32, device=dev)
        descs = (BatchDesc * count)()
        for i, (x, y) in enumerate(zip(self.inputs, self.outputs)):
            nb = x.numel() if in_bytes is None else int(in_bytes[i])
            descs[i] = BatchDesc(x.data_ptr() if x.numel() else 0, nb, y.data_ptr(), y.numel(),
                                 self.out_bytes.data_ptr() + 8 * i, self.status.data_ptr() + 4 * i)
        self._descs = descs
        self.op = op
        h = ctypes.c_void_p(0)
        prm = ctypes.byref(params) if params is not None else None
        _check(lib().huff_batch_plan(descs, count, op, prm, ctypes.byref(h)), "huff_batch_plan")
        self._h = h

    def run(self, stream=None):
        _check(lib().huff_batch_run(self._h, _stream(stream)), "huff_batch_run")

    def autotune(self, base: BatchParams | None = None, flags: int = 0, stream=None) -> BatchParams:
        """huff_batch_autotune on this plan's buffers: the fastest parameters
        (running the batch several times).  Build a new plan with them."""
        best = BatchParams()
        prm = ctypes.byref(base) if base is not None else None
        _check(lib().huff_batch_autotune(self._descs, len(self.inputs), self.op, prm, flags,
                                         ctypes.byref(best), _stream(stream)),
               "huff_batch_autotune")
        return best

    def info(self):
        p, g, used = BatchParams(), ctypes.c_uint32(0), ctypes.c_int32(0)
        _check(lib().huff_batch_info(self._h, ctypes.byref(p), ctypes.byref(g), ctypes.byref(used)),
               "huff_batch_info")
        return {"chunk_symbols": p.chunk_symbols, "ctas_per_sm": p.ctas_per_sm,
                "decode_lanes": p.decode_lanes, "grid": g.value, "graph": bool(used.value)}

    def close(self):
        if self._h and self._h.value:
            lib().huff_batch_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- segmented container
def huff_segmented_compress(d_in: torch.Tensor, segment_bytes: int,
                            chunk_symbols: int = DEFAULT_CHUNK_SYMBOLS, stream=None):
    """(container uint8 tensor, status int32[1]): one codebook per segment."""
    n = d_in.numel()
    L = lib()
    cap = L.huff_segmented_max_size(n, segment_bytes, chunk_symbols)
    wsb = L.huff_segmented_workspace_size(n, segment_bytes, chunk_symbols)
    if cap == 0 or wsb == 0:
        raise HuffError(HUFF_ERR_INVALID_ARG, "huff_segmented_compress")
    dev = d_in.device
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    ob = torch.zeros(1, dtype=torch.int64, device=dev)
    st = new_status(dev)
    _check(L.huff_segmented_compress(_ptr(d_in) if n else None, n, segment_bytes, chunk_symbols,
                                     _ptr(out), cap, _ptr(ob), _ptr(ws), wsb, _ptr(st),
                                     _stream(stream)), "huff_segmented_compress")
    size = int(ob.item())
    return (out[:size] if int(st.item()) == 0 else out[:0]), st


def huff_segmented_decompress(d_container: torch.Tensor, out_cap: int | None = None,
                              stream=None):
    """(decoded uint8 tensor, n, status int32[1])."""
    dev = d_container.device
    dn = torch.zeros(1, dtype=torch.int64, device=dev)
    st = new_status(dev)
    if out_cap is None:
        out_cap = int.from_bytes(bytes(d_container[:8].cpu().numpy()), "little") \
            if d_container.numel() >= 8 else 0
    out = torch.empty(max(out_cap, 16), dtype=torch.uint8, device=dev)
    _check(lib().huff_segmented_decompress(_ptr(d_container), d_container.numel(), _ptr(out),
                                           out_cap, _ptr(dn), _ptr(st), _stream(stream)),
           "huff_segmented_decompress")
    n = int(dn.item())
    return out[:n], n, st


# ---------------------------------------------------------------- LZSS Method 2
def _lzss_params(params) -> LzssParams:
    w, lmin, lmax, blk, dct = params
    return LzssParams(w, lmin, lmax, blk, dct)


def huff_lzss_compress(d_in: torch.Tensor, segment_bytes: int, params=LZSS_PAPER,
                       d_out=None, d_out_bytes=None, d_ws=None, d_status=None, stream=None):
    """(container uint8 tensor, status int32[1]); params = (window, min_len,
    max_len, block, dict).  With d_out / d_out_bytes / d_ws / d_status
    given, nothing is allocated and nothing is synchronised: the container
    is d_out[:d_out_bytes] once the stream has run."""
    n = d_in.numel()
    L = lib()
    P = _lzss_params(params)
    cap = L.huff_lzss_max_size(n, segment_bytes, ctypes.byref(P))
    wsb = L.huff_lzss_workspace_size(n, segment_bytes, ctypes.byref(P))
    if cap == 0 or wsb == 0:
        raise HuffError(HUFF_ERR_INVALID_ARG, "huff_lzss_compress")
    dev = d_in.device
    sync = d_out is None
    out = d_out if d_out is not None else torch.empty(cap, dtype=torch.uint8, device=dev)
    ws = d_ws if d_ws is not None else torch.empty(max(wsb, 16), dtype=torch.uint8, device=dev)
    ob = d_out_bytes if d_out_bytes is not None else torch.zeros(1, dtype=torch.int64, device=dev)
    st = d_status if d_status is not None else new_status(dev)
    _check(L.huff_lzss_compress(_ptr(d_in) if n else None, n, segment_bytes, ctypes.byref(P),
                                _ptr(out), out.numel(), _ptr(ob), _ptr(ws), ws.numel(), _ptr(st),
                                _stream(stream)), "huff_lzss_compress")
    if not sync:
        return out, st
    size = int(ob.item())
    return (out[:size] if int(st.item()) == 0 else out[:0]), st


def huff_lzss_decompress(d_container: torch.Tensor, out_cap: int | None = None, d_out=None,
                         d_n=None, d_ws=None, d_status=None, stream=None):
    """(decoded uint8 tensor, n, status int32[1]).  With d_out / d_n / d_ws /
    d_status given, nothing is allocated and nothing is synchronised (n is
    then None: read d_n after the stream has run)."""
    dev = d_container.device
    L = lib()
    nb = d_container.numel()
    sync = d_out is None
    dn = d_n if d_n is not None else torch.zeros(1, dtype=torch.int64, device=dev)
    st = d_status if d_status is not None else new_status(dev)
    if d_out is None:
        if out_cap is None:
            out_cap = int.from_bytes(bytes(d_container[:8].cpu().numpy()), "little") \
                if nb >= 8 else 0
        d_out = torch.empty(max(out_cap, 16), dtype=torch.uint8, device=dev)
    elif out_cap is None:
        out_cap = d_out.numel()
    wsb = L.huff_lzss_decompress_workspace_size(nb)
    ws = d_ws if d_ws is not None else torch.empty(max(wsb, 16), dtype=torch.uint8, device=dev)
    _check(L.huff_lzss_decompress(_ptr(d_container), nb, _ptr(d_out), out_cap, _ptr(dn),
                                  _ptr(ws), ws.numel(), _ptr(st), _stream(stream)),
           "huff_lzss_decompress")
    if not sync:
        return d_out, None, st
    n = int(dn.item())
    return d_out[:n], n, st


# ---------------------------------------------------------------- Method 3
def _bwt_ws(n: int, block: int, dev, ws=None):
    wsb = lib().huff_bwt_workspace_size(n, block)
    if wsb == 0:
        raise HuffError(HUFF_ERR_INVALID_ARG, "huff_bwt_workspace_size")
    if ws is None or ws.numel() < wsb:
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    return ws, wsb


def huff_bwt_forward(d_in: torch.Tensor, block: int, d_last=None, d_primary=None, ws=None,
                     stream=None):
    """(last column uint8[n], primary int32[blocks] holding u32, status int32[1]):
    the block-sorting transform of every `block`-byte block (synchronizes)."""
    x = _u8(d_in)
    n = x.numel()
    dev = x.device
    blocks = (n + block - 1) // block if block > 0 else 0
    if d_last is None:
        d_last = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
    if d_primary is None:
        d_primary = torch.empty(max(blocks, 1), dtype=torch.int32, device=dev)
    ws, wsb = _bwt_ws(n, block, dev, ws) if n else (None, 0)
    st = new_status(dev)
    _check(lib().huff_bwt_forward(_ptr(x) if n else None, n, block, _ptr(d_last),
                                  _ptr(d_primary), _ptr(ws), wsb, _ptr(st), _stream(stream)),
           "huff_bwt_forward")
    return d_last[:n], d_primary[:blocks], st


def huff_bwt_inverse(d_last: torch.Tensor, block: int, d_primary: torch.Tensor, d_out=None,
                     ws=None, stream=None):
    """(bytes uint8[n], status int32[1]): inverse of huff_bwt_forward."""
    L = _u8(d_last)
    n = L.numel()
    dev = L.device
    if d_out is None:
        d_out = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
    ws, wsb = _bwt_ws(n, block, dev, ws) if n else (None, 0)
    st = new_status(dev)
    _check(lib().huff_bwt_inverse(_ptr(L) if n else None, n, block, _ptr(d_primary),
                                  _ptr(d_out), _ptr(ws), wsb, _ptr(st), _stream(stream)),
           "huff_bwt_inverse")
    return d_out[:n], st


def _mtf_call(fn, name, d_in, block, d_out, ws, stream):
    x = _u8(d_in)
    n = x.numel()
    dev = x.device
    if d_out is None:
        d_out = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
    wsb = lib().huff_mtf_workspace_size(n, block)
    if wsb == 0:
        raise HuffError(HUFF_ERR_INVALID_ARG, name)
    if ws is None or ws.numel() < wsb:
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    _check(fn(_ptr(x) if n else None, n, block, _ptr(d_out), _ptr(ws), wsb, _stream(stream)), name)
    return d_out[:n]


def huff_mtf_forward(d_in: torch.Tensor, block: int, d_out=None, ws=None, stream=None):
    """Move-to-front coding of every `block`-byte block (asynchronous)."""
    return _mtf_call(lib().huff_mtf_forward, "huff_mtf_forward", d_in, block, d_out, ws, stream)


def huff_mtf_inverse(d_in: torch.Tensor, block: int, d_out=None, ws=None, stream=None):
    """Inverse of huff_mtf_forward (asynchronous)."""
    return _mtf_call(lib().huff_mtf_inverse, "huff_mtf_inverse", d_in, block, d_out, ws, stream)


HUFF_M3_MTF = 1


def huff_m3_compress(d_in: torch.Tensor, block: int, segment_bytes: int,
                     chunk_symbols: int = DEFAULT_CHUNK_SYMBOLS, stages: int = 0, stream=None):
    """(container uint8 tensor, status int32[1]): Method 3 -- the transform of
    every block (then move-to-front with stages=HUFF_M3_MTF), then one
    codebook per segment."""
    x = _u8(d_in)
    n = x.numel()
    L = lib()
    cap = L.huff_m3_max_size(n, block, segment_bytes, chunk_symbols)
    wsb = L.huff_m3_workspace_size(n, block, segment_bytes, chunk_symbols)
    if cap == 0 or wsb == 0:
        raise HuffError(HUFF_ERR_INVALID_ARG, "huff_m3_compress")
    dev = x.device
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    ob = torch.zeros(1, dtype=torch.int64, device=dev)
    st = new_status(dev)
    _check(L.huff_m3_compress(_ptr(x) if n else None, n, block, segment_bytes, chunk_symbols,
                              stages, _ptr(out), cap, _ptr(ob), _ptr(ws), wsb, _ptr(st),
                              _stream(stream)), "huff_m3_compress")
    size = int(ob.item())
    return (out[:size] if int(st.item()) == 0 else out[:0]), st


def huff_m3_decompress(d_container: torch.Tensor, out_cap: int | None = None, stream=None):
    """(decoded uint8 tensor, n, status int32[1])."""
    c = _u8(d_container)
    dev = c.device
    head = bytes(c[:16].cpu().numpy()) if c.numel() >= 16 else b"\0" * 16
    n = int.from_bytes(head[:8], "little")
    block = int.from_bytes(head[8:12], "little")
    wsb = lib().huff_m3_decompress_workspace_size(n, block) if block else 0
    ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device=dev)
    if out_cap is None:
        out_cap = n
    out = torch.empty(max(out_cap, 16), dtype=torch.uint8, device=dev)
    dn = torch.zeros(1, dtype=torch.int64, device=dev)
    st = new_status(dev)
    _check(lib().huff_m3_decompress(_ptr(c), c.numel(), _ptr(out), out_cap, _ptr(dn), _ptr(ws),
                                    wsb, _ptr(st), _stream(stream)), "huff_m3_decompress")
    got = int(dn.item()) if int(st.item()) == 0 else 0
    return out[:got], got, st


# ---------------------------------------------------------------- served path
def huff_server_default_config() -> ServerConfig:
    c = ServerConfig()
    lib().huff_server_default_config(ctypes.byref(c))
    return c


def _host_ptr(buf) -> int:
    """Address of a host buffer: a CPU tensor (pinned for full speed) or numpy array."""
    if isinstance(buf, torch.Tensor):
        assert not buf.is_cuda and buf.is_contiguous()
        return buf.data_ptr()
    return int(buf.ctypes.data)


class Server:
    """huff_server_*: continuous-batching request loop on the current device."""

    def __init__(self, cfg: ServerConfig | None = None):
        h = ctypes.c_void_p(0)
        _check(lib().huff_server_create(ctypes.byref(cfg) if cfg is not None else None,
                                        ctypes.byref(h)), "huff_server_create")
        self._h = h
        self._keep = {}

    def submit(self, op: int, h_in, h_out, in_bytes: int | None = None) -> int:
        n = (h_in.numel() if isinstance(h_in, torch.Tensor) else h_in.size) if in_bytes is None \
            else int(in_bytes)
        cap = h_out.numel() if isinstance(h_out, torch.Tensor) else h_out.size
        req = Request(op, _host_ptr(h_in) if n else 0, n, _host_ptr(h_out), cap)
        t = ctypes.c_uint64(0)
        _check(lib().huff_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)),
               "huff_server_submit")
        self._keep[t.value] = (h_in, h_out)
        return t.value

    @staticmethod
    def _res(r: Result):
        return {"done": bool(r.done), "status": r.status, "out_bytes": r.out_bytes,
                "t_submit": r.t_submit, "t_start": r.t_start, "t_done": r.t_done}

    def poll(self, ticket: int):
        r = Result()
        _check(lib().huff_server_poll(self._h, ticket, ctypes.byref(r)), "huff_server_poll")
        return self._res(r)

    def wait(self, ticket: int, timeout_ms: int = 60000):
        r = Result()
        st = lib().huff_server_wait(self._h, ticket, timeout_ms, ctypes.byref(r))
        if st not in (HUFF_OK, HUFF_ERR_TIMEOUT):
            raise HuffError(st, "huff_server_wait")
        return self._res(r)

    def release(self, ticket: int):
        _check(lib().huff_server_release(self._h, ticket), "huff_server_release")
        self._keep.pop(ticket, None)

    def close(self):
        if self._h and self._h.value:
            lib().huff_server_destroy(self._h)
            self._h = ctypes.c_void_p(0)
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- conveniences
def parse_codebook(d_cb: torch.Tensor):
    """(len u8[256], code u32[256], nsym, max_len) as numpy, from a device codebook."""
    import numpy as np
    raw = d_cb.cpu().numpy().tobytes()
    ln = np.frombuffer(raw[:256], dtype=np.uint8).copy()
    code = np.frombuffer(raw[256:1280], dtype="<u4").copy()
    nsym, max_len = np.frombuffer(raw[1280:1288], dtype="<u4")
    return ln, code, int(nsym), int(max_len)


def compress(x: torch.Tensor, chunk_symbols: int = DEFAULT_CHUNK_SYMBOLS, stream=None) -> torch.Tensor:
    """Compress a uint8 CUDA tensor; returns the stream trimmed to its size."""
    out, ob, st = huff_compress(x, chunk_symbols, stream=stream)
    torch.cuda.current_stream().synchronize() if stream is None else torch.cuda.synchronize()
    _check(int(st.item()), "compress")
    return out[:int(ob.item())]


def decompress(stream_t: torch.Tensor, stream=None) -> torch.Tensor:
    """Decompress a stream held in a uint8 CUDA tensor."""
    out, n, st = huff_decode(stream_t, stream=stream)
    torch.cuda.current_stream().synchronize() if stream is None else torch.cuda.synchronize()
    _check(int(st.item()), "decompress")
    return out[:int(n.item())]


__all__ = [name for name in dir() if name.startswith("huff_")] + [
    "compress", "decompress", "parse_codebook", "new_status", "HuffError", "lib", "LIB_PATH",
    "BatchPlan", "BatchDesc", "BatchParams", "HUFF_BATCH_COMPRESS", "HUFF_BATCH_DECOMPRESS",
    "Server", "ServerConfig", "Request", "Result",
]
