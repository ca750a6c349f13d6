"""Thin ctypes binding of the fpsnr C ABI (include/fpsnr.h).

The functions below carry the C names and only marshal arguments: device
buffers are passed as integer device pointers (e.g. ``tensor.data_ptr()``),
streams as integer handles (``torch.cuda.Stream.cuda_stream``).  Every step of
the method runs in the CUDA library; there is no CPU fallback: ``load()``
raises if libfpsnr.so has not been built.

``Plan`` is a convenience wrapper over torch tensors (torch supplies device
memory and streams only).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfpsnr.so")

FPSNR_OK = 0
FPSNR_EINVAL = -1
FPSNR_ENOMEM = -2
FPSNR_ECUDA = -3
FPSNR_ENONFINITE = -4
FPSNR_ECAPACITY = -5
FPSNR_ECORRUPT = -6
FPSNR_ETIMEOUT = -7
FPSNR_MAX_PSNR = 180.0

# every function include/fpsnr.h declares
EXPORTS = ("fpsnr_default_opts", "fpsnr_plan", "fpsnr_plan_set_psnr", "fpsnr_plan_eb_rel",
           "fpsnr_plan_points", "fpsnr_max_compressed_bytes", "fpsnr_compress",
           "fpsnr_decompress", "fpsnr_psnr", "fpsnr_plan_codes", "fpsnr_plan_destroy",
           "fpsnr_strerror", "fpsnr_plan_profile", "fpsnr_plan_profile_read",
           "fpsnr_stage_name", "fpsnr_psnr_static", "fpsnr_compress_batch",
           "fpsnr_decompress_batch", "fpsnr_plan_set_tuning", "fpsnr_plan_get_tuning",
           "fpsnr_autotune", "fpsnr_server_create", "fpsnr_server_submit", "fpsnr_server_poll",
           "fpsnr_server_wait", "fpsnr_server_drain", "fpsnr_server_get_stats",
           "fpsnr_server_now", "fpsnr_server_destroy", "fpsnr_server_take_any",
           "fpsnr_blob_info", "fpsnr_plan_from_blob", "fpsnr_plan_set_wait_limit")
FPSNR_EAGAIN = -8
FPSNR_REQ_COMPRESS = 0
FPSNR_REQ_DECOMPRESS = 1
FPSNR_PSNR_STATIC_MAX_POINTS = 1 << 28
FPSNR_NSTAGES = 18

_lock = threading.Lock()
_lib = None


class FpsnrError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {fpsnr_strerror(code)} ({code})" if what else
                         f"{fpsnr_strerror(code)} ({code})")


class fpsnr_opts(C.Structure):
    _fields_ = [("radius", C.c_int), ("chunk", C.c_int), ("lmax", C.c_int),
                ("lorenzo_dims", C.c_int), ("psnr_mode", C.c_int), ("lossless", C.c_int)]


class fpsnr_stats(C.Structure):
    _fields_ = [("target_psnr", C.c_double), ("eb_rel", C.c_double), ("eb_abs", C.c_double),
                ("vr", C.c_double), ("psnr_model", C.c_double), ("sse", C.c_double),
                ("mse", C.c_double), ("psnr_actual", C.c_double), ("bytes", C.c_uint64),
                ("n_outlier", C.c_uint64), ("n_verbatim", C.c_uint64), ("n_sym", C.c_uint64),
                ("xmin", C.c_float), ("xmax", C.c_float), ("flags", C.c_uint32),
                ("status", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


STATS_BYTES = C.sizeof(fpsnr_stats)


class fpsnr_server_opts(C.Structure):
    _fields_ = [("hbm_budget", C.c_uint64), ("max_batch", C.c_int), ("streams", C.c_int)]


class fpsnr_request(C.Structure):
    _fields_ = [("kind", C.c_int), ("ndim", C.c_int), ("dims", C.c_uint64 * 3),
                ("target_psnr_db", C.c_double), ("opts", fpsnr_opts), ("d_in", C.c_void_p),
                ("in_bytes", C.c_uint64), ("d_out", C.c_void_p), ("out_cap", C.c_uint64),
                ("arrival_us", C.c_double)]


class fpsnr_result(C.Structure):
    _fields_ = [("status", C.c_int), ("out_bytes", C.c_uint64), ("stats", fpsnr_stats),
                ("arrival_us", C.c_double), ("start_us", C.c_double), ("done_us", C.c_double)]


class fpsnr_server_stats(C.Structure):
    _fields_ = [("completed", C.c_uint64), ("failed", C.c_uint64), ("batches", C.c_uint64),
                ("p50_us", C.c_double), ("p99_us", C.c_double), ("max_us", C.c_double),
                ("plans", C.c_uint64), ("plan_bytes", C.c_uint64), ("bytes_in", C.c_uint64),
                ("plans_created", C.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class fpsnr_blob_header(C.Structure):
    _fields_ = [("ndim", C.c_int), ("lorenzo_dims", C.c_int), ("dims", C.c_uint64 * 3),
                ("points", C.c_uint64), ("target_psnr", C.c_double), ("eb_rel", C.c_double),
                ("eb_abs", C.c_double), ("vr", C.c_double), ("xmin", C.c_float),
                ("xmax", C.c_float), ("flags", C.c_uint32), ("radius", C.c_int),
                ("chunk", C.c_int), ("lmax", C.c_int), ("lossless", C.c_int),
                ("raw_bytes", C.c_uint64), ("n_outlier", C.c_uint64), ("n_verbatim", C.c_uint64)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["dims"] = [int(v) for v in self.dims]
        return d


class fpsnr_tuning(C.Structure):
    _fields_ = [("chunk", C.c_int), ("pq_tile_x", C.c_int), ("band_rows", C.c_int),
                ("dec_threads", C.c_int), ("ms", C.c_double), ("bytes", C.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def load(path: str = LIB_PATH):
    """Load libfpsnr.so (raises if it is missing: build it first)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} not found: run paper_1805_07384_gb300/build.py "
                               "(or __graft_entry__.build()) first")
        L = C.CDLL(path)
        P, U64, D = C.c_void_p, C.c_uint64, C.c_double
        L.fpsnr_default_opts.argtypes = [C.POINTER(fpsnr_opts)]
        L.fpsnr_plan.argtypes = [C.POINTER(P), C.c_int, C.POINTER(U64), D, C.POINTER(fpsnr_opts)]
        L.fpsnr_plan_set_psnr.argtypes = [P, D]
        L.fpsnr_plan_eb_rel.argtypes = [P]
        L.fpsnr_plan_eb_rel.restype = D
        L.fpsnr_plan_points.argtypes = [P]
        L.fpsnr_plan_points.restype = U64
        L.fpsnr_max_compressed_bytes.argtypes = [P]
        L.fpsnr_max_compressed_bytes.restype = U64
        L.fpsnr_compress.argtypes = [P, P, P, U64, P, P, P]
        L.fpsnr_decompress.argtypes = [P, P, U64, P, U64, P, P]
        L.fpsnr_compress_batch.argtypes = [P, P, P, P, P, P, C.c_int, P]
        L.fpsnr_decompress_batch.argtypes = [P, P, P, P, P, C.c_int, P]
        L.fpsnr_psnr.argtypes = [P, P, U64, C.POINTER(D), C.POINTER(D), C.POINTER(D), P]
        L.fpsnr_psnr_static.argtypes = [P, P, U64, C.POINTER(D), C.POINTER(D), C.POINTER(D), P]
        L.fpsnr_plan_codes.argtypes = [P]
        L.fpsnr_plan_codes.restype = P
        L.fpsnr_plan_destroy.argtypes = [P]
        L.fpsnr_plan_destroy.restype = None
        L.fpsnr_strerror.argtypes = [C.c_int]
        L.fpsnr_strerror.restype = C.c_char_p
        L.fpsnr_plan_profile.argtypes = [P, C.c_int]
        L.fpsnr_plan_profile_read.argtypes = [P, C.POINTER(D), C.POINTER(U64), C.c_int]
        L.fpsnr_stage_name.argtypes = [C.c_int]
        L.fpsnr_stage_name.restype = C.c_char_p
        L.fpsnr_server_create.argtypes = [C.POINTER(fpsnr_server_opts), C.POINTER(P)]
        L.fpsnr_server_submit.argtypes = [P, C.POINTER(fpsnr_request), C.POINTER(U64)]
        L.fpsnr_server_poll.argtypes = [P, U64, C.POINTER(fpsnr_result)]
        L.fpsnr_server_wait.argtypes = [P, U64, C.POINTER(fpsnr_result), D]
        L.fpsnr_server_take_any.argtypes = [P, C.POINTER(U64), C.POINTER(fpsnr_result)]
        L.fpsnr_server_drain.argtypes = [P, D]
        L.fpsnr_server_get_stats.argtypes = [P, C.POINTER(fpsnr_server_stats)]
        L.fpsnr_server_now.argtypes = [P]
        L.fpsnr_server_now.restype = D
        L.fpsnr_server_destroy.argtypes = [P]
        L.fpsnr_server_destroy.restype = None
        L.fpsnr_plan_set_tuning.argtypes = [P, C.POINTER(fpsnr_tuning)]
        L.fpsnr_plan_get_tuning.argtypes = [P, C.POINTER(fpsnr_tuning)]
        L.fpsnr_autotune.argtypes = [C.c_int, C.POINTER(U64), D, C.POINTER(fpsnr_opts), P, D,
                                     C.POINTER(fpsnr_tuning), P]
        L.fpsnr_blob_info.argtypes = [P, U64, C.POINTER(fpsnr_blob_header), P]
        L.fpsnr_plan_from_blob.argtypes = [C.POINTER(P), C.POINTER(fpsnr_blob_header)]
        L.fpsnr_plan_set_wait_limit.argtypes = [P, C.c_uint32, C.c_int]
        _lib = L
        return L


# ---------------------------------------------------------------------------
# the C functions, same names
# ---------------------------------------------------------------------------

def fpsnr_default_opts() -> fpsnr_opts:
    o = fpsnr_opts()
    load().fpsnr_default_opts(C.byref(o))
    return o


def fpsnr_plan(ndim: int, dims, target_psnr_db: float, opts: fpsnr_opts | None = None):
    """dims x-fastest; returns the plan handle (int) or raises FpsnrError."""
    vals = [int(d) for d in dims]
    vals += [1] * max(0, 3 - len(vals))
    arr = (C.c_uint64 * len(vals))(*vals)
    h = C.c_void_p()
    rc = load().fpsnr_plan(C.byref(h), int(ndim), arr, float(target_psnr_db),
                           C.byref(opts) if opts is not None else None)
    if rc:
        raise FpsnrError(rc, "fpsnr_plan")
    return h.value


def fpsnr_plan_set_psnr(plan, target_psnr_db: float) -> int:
    return load().fpsnr_plan_set_psnr(plan, float(target_psnr_db))


def fpsnr_plan_eb_rel(plan) -> float:
    return load().fpsnr_plan_eb_rel(plan)


def fpsnr_plan_points(plan) -> int:
    return load().fpsnr_plan_points(plan)


def fpsnr_max_compressed_bytes(plan) -> int:
    return load().fpsnr_max_compressed_bytes(plan)


def fpsnr_compress(plan, d_in: int, d_out: int, out_cap: int, d_out_bytes: int = 0,
                   d_stats: int = 0, stream: int = 0) -> int:
    return load().fpsnr_compress(plan, d_in, d_out, int(out_cap), d_out_bytes or None,
                                 d_stats or None, stream or None)


def fpsnr_decompress(plan, d_blob: int, blob_bytes: int, d_out: int, n_out: int,
                     d_status: int = 0, stream: int = 0) -> int:
    return load().fpsnr_decompress(plan, d_blob, int(blob_bytes), d_out, int(n_out),
                                   d_status or None, stream or None)


def _ptr_array(vals):
    return (C.c_void_p * len(vals))(*[int(v) if v else None for v in vals])


def _same_length(n, **lists):
    for name, v in lists.items():
        if len(v) != n:
            raise ValueError(f"{name} has {len(v)} entries for {n} plans")


def fpsnr_compress_batch(plans, d_in, d_out, out_cap, d_out_bytes: int = 0, d_stats: int = 0,
                         stream: int = 0) -> int:
    """Lists of plan handles, input/output device pointers and capacities."""
    n = len(plans)
    _same_length(n, d_in=d_in, d_out=d_out, out_cap=out_cap)
    caps = (C.c_uint64 * n)(*[int(c) for c in out_cap])
    return load().fpsnr_compress_batch(_ptr_array(plans), _ptr_array(d_in), _ptr_array(d_out),
                                       caps, d_out_bytes or None, d_stats or None, n,
                                       stream or None)


def fpsnr_decompress_batch(plans, d_blob, blob_bytes, d_out, d_status: int = 0,
                           stream: int = 0) -> int:
    n = len(plans)
    _same_length(n, d_blob=d_blob, blob_bytes=blob_bytes, d_out=d_out)
    nb = (C.c_uint64 * n)(*[int(b) for b in blob_bytes])
    return load().fpsnr_decompress_batch(_ptr_array(plans), _ptr_array(d_blob), nb,
                                         _ptr_array(d_out), d_status or None, n, stream or None)


def fpsnr_psnr(d_x: int, d_xr: int, n: int, stream: int = 0):
    """Returns (psnr_db, mse, vr); raises FpsnrError on failure."""
    p, m, v = C.c_double(), C.c_double(), C.c_double()
    rc = load().fpsnr_psnr(d_x, d_xr, int(n), C.byref(p), C.byref(m), C.byref(v), stream or None)
    if rc:
        raise FpsnrError(rc, "fpsnr_psnr")
    return p.value, m.value, v.value


def fpsnr_psnr_static(d_x: int, d_xr: int, n: int, stream: int = 0):
    """Allocation-free fpsnr_psnr: returns (psnr_db, mse, vr); raises FpsnrError."""
    p, m, v = C.c_double(), C.c_double(), C.c_double()
    rc = load().fpsnr_psnr_static(d_x, d_xr, int(n), C.byref(p), C.byref(m), C.byref(v),
                                  stream or None)
    if rc:
        raise FpsnrError(rc, "fpsnr_psnr_static")
    return p.value, m.value, v.value


def fpsnr_blob_info(blob: int, blob_bytes: int, stream: int = 0) -> fpsnr_blob_header:
    """Header of the blob at `blob` (device or host pointer); raises FpsnrError."""
    h = fpsnr_blob_header()
    rc = load().fpsnr_blob_info(blob, int(blob_bytes), C.byref(h), stream or None)
    if rc:
        raise FpsnrError(rc, "fpsnr_blob_info")
    return h


def fpsnr_plan_from_blob(header: fpsnr_blob_header):
    """Plan handle (int) that decompresses blobs with this header; raises FpsnrError."""
    p = C.c_void_p()
    rc = load().fpsnr_plan_from_blob(C.byref(p), C.byref(header))
    if rc:
        raise FpsnrError(rc, "fpsnr_plan_from_blob")
    return p.value


def fpsnr_plan_set_wait_limit(plan, spins: int, test_unmet: int = 0) -> int:
    return load().fpsnr_plan_set_wait_limit(plan, int(spins), int(test_unmet))


def fpsnr_plan_codes(plan) -> int:
    return load().fpsnr_plan_codes(plan)


def fpsnr_plan_destroy(plan) -> None:
    load().fpsnr_plan_destroy(plan)


def fpsnr_strerror(code: int) -> str:
    return load().fpsnr_strerror(int(code)).decode()


def fpsnr_plan_profile(plan, enable: bool) -> int:
    return load().fpsnr_plan_profile(plan, 1 if enable else 0)


def fpsnr_plan_profile_read(plan):
    """{stage name: (milliseconds, launches)} since the last read."""
    ms = (C.c_double * FPSNR_NSTAGES)()
    ln = (C.c_uint64 * FPSNR_NSTAGES)()
    rc = load().fpsnr_plan_profile_read(plan, ms, ln, FPSNR_NSTAGES)
    if rc:
        raise FpsnrError(rc, "fpsnr_plan_profile_read")
    return {fpsnr_stage_name(i): (ms[i], int(ln[i])) for i in range(FPSNR_NSTAGES)}


def fpsnr_stage_name(stage: int) -> str:
    return load().fpsnr_stage_name(int(stage)).decode()


# ---------------------------------------------------------------------------
# torch convenience wrapper
# ---------------------------------------------------------------------------

def _check(t, name, dtype, numel=None, min_numel=None, device=None):
    """Argument checks of the torch wrappers, before anything is enqueued (the
    C side sees bare pointers and sizes and cannot check a tensor's type,
    layout or device)."""
    if not getattr(t, "is_cuda", False):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError(f"{name} has {t.numel()} elements, needs at least {min_numel}")


def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def fpsnr_plan_set_tuning(plan, t: fpsnr_tuning) -> int:
    return load().fpsnr_plan_set_tuning(plan, C.byref(t))


def fpsnr_plan_get_tuning(plan) -> fpsnr_tuning:
    t = fpsnr_tuning()
    rc = load().fpsnr_plan_get_tuning(plan, C.byref(t))
    if rc:
        raise FpsnrError(rc, "fpsnr_plan_get_tuning")
    return t


def fpsnr_autotune(ndim: int, dims, target_psnr_db: float, opts, d_sample: int,
                   max_size_increase: float, stream: int) -> fpsnr_tuning:
    """dims x-fastest; d_sample a device pointer; returns fpsnr_tuning or raises."""
    vals = [int(d) for d in dims] + [1] * max(0, 3 - len(dims))
    arr = (C.c_uint64 * len(vals))(*vals)
    t = fpsnr_tuning()
    rc = load().fpsnr_autotune(int(ndim), arr, float(target_psnr_db),
                               C.byref(opts) if opts is not None else None, d_sample,
                               float(max_size_increase), C.byref(t), stream)
    if rc:
        raise FpsnrError(rc, "fpsnr_autotune")
    return t


def autotune(sample, target_psnr_db: float, max_size_increase: float = 0.01, radius: int = 32768,
             chunk: int = 256, lmax: int = 27, lorenzo_dims: int = 0, stream=None) -> dict:
    """Chunk size and launch shapes for fields shaped like `sample` (a float32
    CUDA tensor, numpy C-order shape) at this target; see fpsnr_autotune."""
    import torch
    _check(sample, "sample", torch.float32)
    o = fpsnr_default_opts()
    o.radius, o.chunk, o.lmax, o.lorenzo_dims = radius, chunk, lmax, lorenzo_dims
    shape = tuple(sample.shape)
    return fpsnr_autotune(len(shape), list(reversed(shape)), target_psnr_db, o, sample.data_ptr(),
                          max_size_increase, _stream_handle(stream)).as_dict()


def parse_stats(raw) -> dict:
    """fpsnr_stats from a uint8 tensor/bytes of STATS_BYTES bytes."""
    b = bytes(raw.cpu().numpy().tobytes()) if hasattr(raw, "cpu") else bytes(raw)
    return fpsnr_stats.from_buffer_copy(b[:STATS_BYTES]).as_dict()


class Plan:
    """Owns one C plan for fields of one shape (numpy/torch C-order shape)."""

    def __init__(self, shape, target_psnr_db: float, radius: int = 32768, chunk: int = 256,
                 lmax: int = 27, lorenzo_dims: int = 0, psnr_mode: int = 0, lossless: int = 0):
        import torch
        self.shape = tuple(int(s) for s in shape)
        self.n = int(math.prod(self.shape))
        o = fpsnr_default_opts()
        o.radius, o.chunk, o.lmax, o.lorenzo_dims = radius, chunk, lmax, lorenzo_dims
        o.psnr_mode, o.lossless = psnr_mode, lossless
        self.opts = o
        self.handle = fpsnr_plan(len(self.shape), list(reversed(self.shape)), target_psnr_db, o)
        self.target = float(target_psnr_db)
        self.max_bytes = fpsnr_max_compressed_bytes(self.handle)
        self.device = torch.device("cuda", torch.cuda.current_device())

    @classmethod
    def from_blob(cls, blob, blob_bytes: int, stream=None) -> "Plan":
        """A plan for decompressing `blob` (uint8 CUDA tensor holding blob_bytes
        bytes), built from the blob's own header (fpsnr_blob_info and
        fpsnr_plan_from_blob): nothing else about the field is needed."""
        import torch
        _check(blob, "blob", torch.uint8)
        if not 0 <= int(blob_bytes) <= blob.numel():
            raise ValueError(f"blob_bytes {int(blob_bytes)} outside the blob's {blob.numel()} bytes")
        h = fpsnr_blob_info(blob.data_ptr(), int(blob_bytes), _stream_handle(stream))
        self = cls.__new__(cls)
        self.header = h.as_dict()
        self.shape = tuple(int(h.dims[i]) for i in reversed(range(h.ndim)))
        self.n = int(h.points)
        o = fpsnr_default_opts()
        o.radius, o.chunk, o.lmax, o.lorenzo_dims = h.radius, h.chunk, h.lmax, h.lorenzo_dims
        o.lossless = h.lossless
        self.opts = o
        self.handle = fpsnr_plan_from_blob(h)
        self.target = float(h.target_psnr)
        self.max_bytes = fpsnr_max_compressed_bytes(self.handle)
        self.device = blob.device
        return self

    def set_psnr(self, target_psnr_db: float) -> None:
        rc = fpsnr_plan_set_psnr(self.handle, target_psnr_db)
        if rc:
            raise FpsnrError(rc, "fpsnr_plan_set_psnr")
        self.target = float(target_psnr_db)

    def alloc_out(self):
        import torch
        return torch.empty(self.max_bytes, dtype=torch.uint8, device=self.device)

    def compress(self, x, out=None, nbytes=None, stats=None, stream=None):
        """Enqueue compression of x (float32 CUDA tensor of the plan's shape).
        Returns (out, nbytes, stats) device tensors: nbytes is int64[1] holding
        the blob size, stats is uint8[STATS_BYTES] (see parse_stats)."""
        import torch
        _check(x, "x", torch.float32, numel=self.n)
        out = self.alloc_out() if out is None else out
        nbytes = torch.zeros(1, dtype=torch.int64, device=x.device) if nbytes is None else nbytes
        stats = torch.zeros(STATS_BYTES, dtype=torch.uint8, device=x.device) if stats is None else stats
        _check(out, "out", torch.uint8, device=x.device)
        _check(nbytes, "nbytes", torch.int64, min_numel=1, device=x.device)
        _check(stats, "stats", torch.uint8, min_numel=STATS_BYTES, device=x.device)
        rc = fpsnr_compress(self.handle, x.data_ptr(), out.data_ptr(), out.numel(),
                            nbytes.data_ptr(), stats.data_ptr(), _stream_handle(stream))
        if rc:
            raise FpsnrError(rc, "fpsnr_compress")
        return out, nbytes, stats

    def decompress(self, blob, blob_bytes: int, out=None, status=None, stream=None):
        """Enqueue decompression; returns (float32 tensor of the plan's shape,
        int32[1] device status)."""
        import torch
        _check(blob, "blob", torch.uint8)
        if not 0 <= int(blob_bytes) <= blob.numel():
            raise ValueError(f"blob_bytes {int(blob_bytes)} outside the blob's {blob.numel()} bytes")
        out = torch.empty(self.shape, dtype=torch.float32, device=blob.device) if out is None else out
        status = torch.zeros(1, dtype=torch.int32, device=blob.device) if status is None else status
        _check(out, "out", torch.float32, numel=self.n, device=blob.device)
        _check(status, "status", torch.int32, min_numel=1, device=blob.device)
        rc = fpsnr_decompress(self.handle, blob.data_ptr(), int(blob_bytes), out.data_ptr(), self.n,
                              status.data_ptr(), _stream_handle(stream))
        if rc:
            raise FpsnrError(rc, "fpsnr_decompress")
        return out, status

    def set_tuning(self, t: dict) -> None:
        """Launch shapes from a tuning dict (autotune's, or hand-written); the
        chunk must match the plan's (pass chunk=... at construction)."""
        tt = fpsnr_tuning()
        for k in ("chunk", "pq_tile_x", "band_rows", "dec_threads"):
            setattr(tt, k, int(t.get(k, 0)))
        rc = fpsnr_plan_set_tuning(self.handle, tt)
        if rc:
            raise FpsnrError(rc, "fpsnr_plan_set_tuning")

    def get_tuning(self) -> dict:
        return fpsnr_plan_get_tuning(self.handle).as_dict()

    def codes(self):
        """Copy of the uint16 symbols of the last compression (int16 tensor)."""
        import torch
        ptr = fpsnr_plan_codes(self.handle)

        class _View:
            pass

        v = _View()
        v.__cuda_array_interface__ = {"shape": (self.n,), "typestr": "<i2",
                                      "data": (int(ptr), False), "version": 3}
        torch.cuda.synchronize()
        return torch.as_tensor(v, device=self.device).clone()

    def close(self):
        if getattr(self, "handle", None):
            fpsnr_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def compress_batch(plans, xs, outs=None, nbytes=None, stats=None, stream=None):
    """Compress fields xs[i] with plans[i] in one batched call.  Returns (outs,
    nbytes int64[count], stats uint8[count, STATS_BYTES]) device tensors."""
    import torch
    n = len(plans)
    _same_length(n, xs=xs)
    if n == 0:
        raise ValueError("empty batch")
    dev = xs[0].device
    outs = [p.alloc_out() for p in plans] if outs is None else outs
    nbytes = torch.zeros(n, dtype=torch.int64, device=dev) if nbytes is None else nbytes
    stats = (torch.zeros((n, STATS_BYTES), dtype=torch.uint8, device=dev)
             if stats is None else stats)
    _same_length(n, outs=outs)
    for i, (p, x, o) in enumerate(zip(plans, xs, outs)):
        _check(x, f"xs[{i}]", torch.float32, numel=p.n, device=dev)
        _check(o, f"outs[{i}]", torch.uint8, device=dev)
    _check(nbytes, "nbytes", torch.int64, min_numel=n, device=dev)
    _check(stats, "stats", torch.uint8, min_numel=n * STATS_BYTES, device=dev)
    rc = fpsnr_compress_batch([p.handle for p in plans], [x.data_ptr() for x in xs],
                              [o.data_ptr() for o in outs], [o.numel() for o in outs],
                              nbytes.data_ptr(), stats.data_ptr(), _stream_handle(stream))
    if rc:
        raise FpsnrError(rc, "fpsnr_compress_batch")
    return outs, nbytes, stats


def decompress_batch(plans, blobs, blob_bytes=None, outs=None, status=None, stream=None):
    """Decompress blobs[i] with plans[i] in one batched call.  blob_bytes
    defaults to each buffer's size.  Returns (outs, status int32[count])."""
    import torch
    n = len(plans)
    _same_length(n, blobs=blobs)
    if n == 0:
        raise ValueError("empty batch")
    dev = blobs[0].device
    outs = ([torch.empty(p.shape, dtype=torch.float32, device=dev) for p in plans]
            if outs is None else outs)
    status = torch.zeros(n, dtype=torch.int32, device=dev) if status is None else status
    blob_bytes = [b.numel() for b in blobs] if blob_bytes is None else [int(v) for v in blob_bytes]
    _same_length(n, outs=outs, blob_bytes=blob_bytes)
    for i, (p, b, nb, o) in enumerate(zip(plans, blobs, blob_bytes, outs)):
        _check(b, f"blobs[{i}]", torch.uint8, device=dev)
        if not 0 <= nb <= b.numel():
            raise ValueError(f"blob_bytes[{i}] = {nb} outside the blob's {b.numel()} bytes")
        _check(o, f"outs[{i}]", torch.float32, numel=p.n, device=dev)
    _check(status, "status", torch.int32, min_numel=n, device=dev)
    rc = fpsnr_decompress_batch([p.handle for p in plans], [b.data_ptr() for b in blobs],
                                blob_bytes, [o.data_ptr() for o in outs], status.data_ptr(),
                                _stream_handle(stream))
    if rc:
        raise FpsnrError(rc, "fpsnr_decompress_batch")
    return outs, status


def psnr(x, xr, stream=None):
    """(PSNR dB, MSE, vr) of reconstruction xr against x (CUDA float32 tensors)."""
    import torch
    _check(x, "x", torch.float32)
    _check(xr, "xr", torch.float32, numel=x.numel(), device=x.device)
    return fpsnr_psnr(x.data_ptr(), xr.data_ptr(), x.numel(), _stream_handle(stream))


# ---------------------------------------------------------------------------
# request server
# ---------------------------------------------------------------------------

def _result_dict(r: fpsnr_result) -> dict:
    return {"status": r.status, "out_bytes": r.out_bytes, "stats": r.stats.as_dict(),
            "arrival_us": r.arrival_us, "start_us": r.start_us, "done_us": r.done_us}


class Server:
    """fpsnr_server_* over torch tensors.  Keeps each request's tensors alive
    until its result has been taken."""

    def __init__(self, hbm_budget: int = 8 << 30, max_batch: int = 16, streams: int = 4):
        o = fpsnr_server_opts(int(hbm_budget), int(max_batch), int(streams))
        h = C.c_void_p()
        rc = load().fpsnr_server_create(C.byref(o), C.byref(h))
        if rc:
            raise FpsnrError(rc, "fpsnr_server_create")
        self.handle = h.value
        self._keep = {}

    def now(self) -> float:
        return load().fpsnr_server_now(self.handle)

    def _submit(self, kind, shape, d_in, in_bytes, d_out, out_cap, psnr, arrival_us, keep,
                radius, chunk, lmax, lorenzo_dims) -> int:
        r = fpsnr_request()
        r.kind = kind
        dims = list(reversed([int(v) for v in shape]))
        r.ndim = len(dims)
        for i, d in enumerate(dims):
            r.dims[i] = d
        r.target_psnr_db = float(psnr)
        r.opts.radius, r.opts.chunk, r.opts.lmax, r.opts.lorenzo_dims = radius, chunk, lmax, lorenzo_dims
        r.d_in, r.in_bytes, r.d_out, r.out_cap = d_in, int(in_bytes), d_out, int(out_cap)
        r.arrival_us = float(arrival_us)
        t = C.c_uint64()
        rc = load().fpsnr_server_submit(self.handle, C.byref(r), C.byref(t))
        if rc:
            raise FpsnrError(rc, "fpsnr_server_submit")
        self._keep[t.value] = keep
        return t.value

    def submit_compress(self, x, psnr: float, out, arrival_us: float = 0.0, radius: int = 32768,
                        chunk: int = 256, lmax: int = 27, lorenzo_dims: int = 0) -> int:
        """Queue compression of x (float32 CUDA tensor) into out (uint8 CUDA tensor)."""
        import torch
        _check(x, "x", torch.float32)
        _check(out, "out", torch.uint8, device=x.device)
        return self._submit(FPSNR_REQ_COMPRESS, x.shape, x.data_ptr(), 0, out.data_ptr(),
                            out.numel(), psnr, arrival_us, (x, out), radius, chunk, lmax,
                            lorenzo_dims)

    def submit_decompress(self, blob, nbytes: int, out, arrival_us: float = 0.0,
                          radius: int = 32768, chunk: int = 256, lmax: int = 27,
                          lorenzo_dims: int = 0) -> int:
        """Queue decompression of blob (uint8 CUDA tensor) into out (float32
        CUDA tensor of the field's shape)."""
        import torch
        _check(blob, "blob", torch.uint8)
        if not 0 <= int(nbytes) <= blob.numel():
            raise ValueError(f"nbytes {int(nbytes)} outside the blob's {blob.numel()} bytes")
        _check(out, "out", torch.float32, device=blob.device)
        return self._submit(FPSNR_REQ_DECOMPRESS, out.shape, blob.data_ptr(), nbytes,
                            out.data_ptr(), 4 * out.numel(), 60.0, arrival_us, (blob, out),
                            radius, chunk, lmax, lorenzo_dims)

    def poll(self, ticket: int):
        r = fpsnr_result()
        rc = load().fpsnr_server_poll(self.handle, ticket, C.byref(r))
        if rc == FPSNR_EAGAIN:
            return None
        if rc:
            raise FpsnrError(rc, "fpsnr_server_poll")
        self._keep.pop(ticket, None)
        return _result_dict(r)

    def take_any(self):
        """(ticket, result) of the oldest completed request not yet taken, or None."""
        r = fpsnr_result()
        t = C.c_uint64()
        rc = load().fpsnr_server_take_any(self.handle, C.byref(t), C.byref(r))
        if rc == FPSNR_EAGAIN:
            return None
        if rc:
            raise FpsnrError(rc, "fpsnr_server_take_any")
        self._keep.pop(t.value, None)
        return t.value, _result_dict(r)

    def wait(self, ticket: int, timeout: float = 120.0) -> dict:
        r = fpsnr_result()
        rc = load().fpsnr_server_wait(self.handle, ticket, C.byref(r), float(timeout))
        if rc:
            raise FpsnrError(rc, "fpsnr_server_wait")
        self._keep.pop(ticket, None)
        return _result_dict(r)

    def drain(self, timeout: float = 600.0) -> None:
        rc = load().fpsnr_server_drain(self.handle, float(timeout))
        if rc:
            raise FpsnrError(rc, "fpsnr_server_drain")

    def stats(self) -> dict:
        st = fpsnr_server_stats()
        rc = load().fpsnr_server_get_stats(self.handle, C.byref(st))
        if rc:
            raise FpsnrError(rc, "fpsnr_server_get_stats")
        return st.as_dict()

    def close(self) -> None:
        if getattr(self, "handle", None):
            load().fpsnr_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
