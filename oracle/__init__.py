"""CPU oracle for fixed-PSNR lossy compression -- TEST INFRASTRUCTURE ONLY.

Plain single-threaded C (``fpsnr_oracle.c``, built with ``-O2 -ffp-contract=off``)
behind ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the CUDA library never does, and
this package imports nothing from it.

Each wrapper names the part of the paper it follows (Tao et al., "Fixed-PSNR
Lossy Compression for Scientific Data"):

* ``eb_rel_from_psnr`` -- Eq. 8;  ``psnr_model`` -- Eq. 7
* ``plan_scalars`` -- eb_abs = eb_rel * vr (Sec. IV, after Eq. 7), bin width 2 eb
* ``lattice`` -- prediction + uniform quantization (Sec. II-A, Sec. III, Sec. IV)
* ``huffman_lengths`` / ``canonical_codes`` -- SZ's Huffman stage (Sec. II-A)
* ``compress`` / ``decompress`` -- the whole pipeline and its inverse (Sec. III, Eq. 1)
* ``fine_hist`` / ``pred_mse`` / ``refine_eb`` -- the optional bound refinement on the
  field's empirical PDF (Eq. 3); ``sum_exact`` -- the exactly rounded sum of its terms
* ``psnr`` -- Eq. 4-5 (sign of Eq. 5 read as 20 log10 vr - 10 log10 MSE)
* ``classic_sz`` -- comparison path predicting from reconstructed values (Sec. III)

Parity status of every function: pinned (see tests/test_oracle_pins.py) except
``classic_sz``, whose exact bytes are "parity unpinned": the paper prints no
output of SZ 1.4 to compare with; only its invariants (pointwise bound, PSNR
model) are checked.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fpsnr_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENONFINITE, ECORRUPT = 0, -1, -2, -4, -6
FLAG_CONSTANT, FLAG_LATTICE_OFF = 1, 2
HEADER_BYTES = 128


# gcc flags of the oracle library: no FMA contraction, IEEE arithmetic
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared"]

# A test may point this variable at another build of fpsnr_oracle.c (the
# mutation test loads copies with one deliberate mistake each, to show that
# the pins catch it); unset, the library is built and loaded from here.
LIB_ENV = "FPSNR_ORACLE_LIB"


def compile_library(src: str, out: str) -> None:
    subprocess.run(["gcc", *CFLAGS, "-o", out, src, "-lm"], check=True)


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        compile_library(_SRC, tmp)
        os.replace(tmp, _SO)
    return _SO


class Scalars(C.Structure):
    _fields_ = [("eb_rel", C.c_double), ("eb_abs", C.c_double), ("vr", C.c_double),
                ("xmin", C.c_float), ("xmax", C.c_float), ("s", C.c_float),
                ("inv", C.c_float), ("thr", C.c_float), ("flags", C.c_uint32)]


class Stats(C.Structure):
    _fields_ = [("target_psnr", C.c_double), ("eb_rel", C.c_double), ("eb_abs", C.c_double),
                ("vr", C.c_double), ("psnr_model", C.c_double), ("sse", C.c_double),
                ("mse", C.c_double), ("psnr_actual", C.c_double), ("bytes", C.c_uint64),
                ("n_outlier", C.c_uint64), ("n_verbatim", C.c_uint64), ("n_sym", C.c_uint64),
                ("xmin", C.c_float), ("xmax", C.c_float), ("s", C.c_float), ("inv", C.c_float),
                ("thr", C.c_float), ("flags", C.c_uint32), ("status", C.c_int32),
                ("pad", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(os.environ.get(LIB_ENV) or build())
            L = _lib
            P = C.c_void_p
            L.or_eb_rel_from_psnr.restype = C.c_double
            L.or_eb_rel_from_psnr.argtypes = [C.c_double]
            L.or_psnr_model.restype = C.c_double
            L.or_psnr_model.argtypes = [C.c_double, C.c_double]
            L.or_range.argtypes = [P, C.c_uint64, P, P]
            L.or_plan_scalars.restype = None
            L.or_plan_scalars.argtypes = [C.c_double, C.c_float, C.c_float, C.c_uint64, P]
            L.or_lattice.argtypes = [P, C.c_int, P, C.c_int, P, C.c_int32, P, P, P, P, P, P, P, P]
            L.or_inverse_lorenzo.restype = None
            L.or_inverse_lorenzo.argtypes = [P, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64]
            L.or_huffman_lengths.argtypes = [P, C.c_uint32, C.c_int, P]
            L.or_canonical_codes.restype = C.c_uint32
            L.or_canonical_codes.argtypes = [P, C.c_uint32, P, P]
            L.or_compress.argtypes = [P, C.c_int, P, C.c_int, C.c_double, C.c_int, C.c_int,
                                      C.c_int, C.POINTER(C.c_void_p), P, P]
            L.or_compress_mode.argtypes = [P, C.c_int, P, C.c_int, C.c_double, C.c_int, C.c_int,
                                           C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p), P, P]
            L.or_zrle_wrap.argtypes = [P, C.c_uint64, C.POINTER(C.c_void_p), P]
            L.or_zrle_unwrap.argtypes = [P, C.c_uint64, C.POINTER(C.c_void_p), P]
            L.or_fine_hist.restype = None
            L.or_fine_hist.argtypes = [P, C.c_uint64, C.c_float, C.c_double, P]
            L.or_pred_mse.restype = C.c_double
            L.or_pred_mse.argtypes = [P, C.c_uint64, C.c_double]
            L.or_sum_exact.restype = C.c_double
            L.or_sum_exact.argtypes = [P, P, C.c_uint32]
            L.or_refine_eb.restype = C.c_double
            L.or_refine_eb.argtypes = [P, C.c_uint64, C.c_double, C.c_double, C.c_double]
            L.or_decompress.argtypes = [P, C.c_uint64, P, C.c_uint64]
            L.or_blob_info.argtypes = [P, C.c_uint64, P, P]
            L.or_free.restype = None
            L.or_free.argtypes = [P]
            L.or_sse.restype = C.c_double
            L.or_sse.argtypes = [P, P, C.c_uint64]
            L.or_psnr.argtypes = [P, P, C.c_uint64, P, P, P]
            L.or_classic_sz.argtypes = [P, C.c_int, P, C.c_int, C.c_double, C.c_int, P, P, P]
        return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dims(shape) -> np.ndarray:
    """numpy C-order shape -> dims array, x (last numpy axis) first."""
    return np.array(list(reversed(shape)) + [1] * (3 - len(shape)), dtype=np.uint64)


def eb_rel_from_psnr(psnr_db: float) -> float:
    return lib().or_eb_rel_from_psnr(float(psnr_db))


def psnr_model(vr: float, eb_abs: float) -> float:
    return lib().or_psnr_model(float(vr), float(eb_abs))


def value_range(x: np.ndarray):
    x = np.ascontiguousarray(x, dtype=np.float32)
    lo, hi = C.c_float(), C.c_float()
    rc = lib().or_range(_ptr(x), x.size, C.byref(lo), C.byref(hi))
    return rc, lo.value, hi.value


def plan_scalars(eb_rel: float, xmin: float, xmax: float, n: int) -> Scalars:
    s = Scalars()
    lib().or_plan_scalars(float(eb_rel), float(xmin), float(xmax), int(n), C.byref(s))
    return s


def lattice(x: np.ndarray, scalars: Scalars, radius: int, lorenzo_dims: int = 0):
    """Codes, outliers, verbatims and SSE of the lattice predictor."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    ndim = x.ndim
    ld = lorenzo_dims or ndim
    n = x.size
    codes = np.zeros(max(n, 1), np.uint16)
    oi = np.zeros(max(n, 1), np.uint32)
    od = np.zeros(max(n, 1), np.int32)
    vi = np.zeros(max(n, 1), np.uint32)
    vb = np.zeros(max(n, 1), np.uint32)
    no, nv, sse = C.c_uint64(), C.c_uint64(), C.c_double()
    dims = _dims(x.shape)
    rc = lib().or_lattice(_ptr(x), ndim, _ptr(dims), ld, C.byref(scalars), int(radius), _ptr(codes),
                          _ptr(oi), _ptr(od), C.byref(no), _ptr(vi), _ptr(vb), C.byref(nv),
                          C.byref(sse))
    if rc:
        raise RuntimeError(f"or_lattice failed: {rc}")
    return dict(codes=codes[:n].reshape(x.shape), out_idx=oi[:no.value].copy(),
                out_delta=od[:no.value].copy(), vb_idx=vi[:nv.value].copy(),
                vb_bits=vb[:nv.value].copy(), sse=sse.value)


def inverse_lorenzo(v: np.ndarray, lorenzo_dims: int) -> np.ndarray:
    """d-dimensional inclusive prefix sums of an int64 array (returns a copy)."""
    v = np.ascontiguousarray(v, dtype=np.int64).copy()
    shape = v.shape
    n = v.size
    if lorenzo_dims == 1:
        nx, ny, nz = n, 1, 1
    elif lorenzo_dims == 2:
        nx = shape[-1]
        ny, nz = (n // nx if nx else 0), 1
    else:
        nx, ny = shape[-1], shape[-2]
        nz = n // (nx * ny) if nx * ny else 0
    lib().or_inverse_lorenzo(_ptr(v), lorenzo_dims, nx, ny, nz)
    return v


def huffman_lengths(counts, lmax: int) -> np.ndarray:
    counts = np.ascontiguousarray(counts, dtype=np.uint32)
    lens = np.zeros(max(counts.size, 1), np.uint8)
    rc = lib().or_huffman_lengths(_ptr(counts), counts.size, int(lmax), _ptr(lens))
    if rc:
        raise ValueError(f"or_huffman_lengths failed: {rc}")
    return lens[:counts.size]


def canonical_codes(lens):
    lens = np.ascontiguousarray(lens, dtype=np.uint8)
    codes = np.zeros(max(lens.size, 1), np.uint32)
    order = np.zeros(max(lens.size, 1), np.uint32)
    n = lib().or_canonical_codes(_ptr(lens), lens.size, _ptr(codes), _ptr(order))
    return codes[:lens.size], order[:n]


def compress(x: np.ndarray, psnr_db: float, radius: int = 32768, chunk: int = 256,
             lmax: int = 27, lorenzo_dims: int = 0, psnr_mode: int = 0, lossless: int = 0):
    """Returns (blob bytes, stats dict); raises on a nonzero status.  psnr_mode
    1 refines eb from the fine histogram (or_refine_eb); lossless 1 wraps the
    blob in the zero-run container when that is smaller (or_zrle_wrap)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    dims = _dims(x.shape)
    out = C.c_void_p()
    nbytes = C.c_uint64()
    st = Stats()
    rc = lib().or_compress_mode(_ptr(x), x.ndim, _ptr(dims), int(lorenzo_dims), float(psnr_db),
                                int(psnr_mode), int(lossless), int(radius), int(chunk), int(lmax),
                                C.byref(out),
                                C.byref(nbytes), C.byref(st))
    if rc:
        raise ValueError(f"or_compress failed with status {rc}")
    try:
        blob = C.string_at(out.value, nbytes.value)
    finally:
        lib().or_free(out)
    return blob, st.as_dict()


def compress_status(x: np.ndarray, psnr_db: float, **kw) -> int:
    """Status code of or_compress (0 = OK) without raising."""
    try:
        compress(x, psnr_db, **kw)
        return OK
    except ValueError as e:
        return int(str(e).rsplit(" ", 1)[-1])


def decompress(blob: bytes, shape) -> np.ndarray:
    n = int(np.prod(shape)) if len(shape) else 1
    out = np.zeros(max(n, 1), np.float32)
    buf = np.frombuffer(blob, dtype=np.uint8)
    rc = lib().or_decompress(_ptr(buf), len(blob), _ptr(out), n)
    if rc:
        raise ValueError(f"or_decompress failed with status {rc}")
    return out[:n].reshape(shape)


def decompress_status(blob: bytes, n: int) -> int:
    out = np.zeros(max(n, 1), np.float32)
    buf = np.frombuffer(blob, dtype=np.uint8)
    return lib().or_decompress(_ptr(buf), len(blob), _ptr(out), n)


def sse(x: np.ndarray, xr: np.ndarray) -> float:
    x = np.ascontiguousarray(x, dtype=np.float32)
    xr = np.ascontiguousarray(xr, dtype=np.float32)
    return lib().or_sse(_ptr(x), _ptr(xr), x.size)


def psnr(x: np.ndarray, xr: np.ndarray):
    """(PSNR dB, MSE, vr) per Eq. 4-5."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    xr = np.ascontiguousarray(xr, dtype=np.float32)
    p, m, v = C.c_double(), C.c_double(), C.c_double()
    rc = lib().or_psnr(_ptr(x), _ptr(xr), x.size, C.byref(p), C.byref(m), C.byref(v))
    if rc:
        raise ValueError(f"or_psnr failed with status {rc}")
    return p.value, m.value, v.value


def classic_sz(x: np.ndarray, psnr_db: float, radius: int = 32768, lorenzo_dims: int = 0):
    """(reconstruction, unpredictable count, PSNR) of the classic sequential path."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    xr = np.zeros_like(x)
    dims = _dims(x.shape)
    nu, p = C.c_uint64(), C.c_double()
    rc = lib().or_classic_sz(_ptr(x), x.ndim, _ptr(dims), int(lorenzo_dims), float(psnr_db),
                             int(radius), _ptr(xr), C.byref(nu), C.byref(p))
    if rc:
        raise ValueError(f"or_classic_sz failed with status {rc}")
    return xr, nu.value, p.value


def parse_blob(blob: bytes) -> dict:
    """Split a blob into its header fields and sections (pure byte slicing)."""
    b = np.frombuffer(blob, dtype=np.uint8)
    u32 = lambda o: int(np.frombuffer(blob, np.uint32, 1, o)[0])
    f32 = lambda o: float(np.frombuffer(blob, np.float32, 1, o)[0])
    f64 = lambda o: float(np.frombuffer(blob, np.float64, 1, o)[0])
    h = dict(magic=u32(0), version=u32(4), ndim=u32(8), lorenzo_dims=u32(12),
             dims=[int(v) for v in np.frombuffer(blob, np.uint64, 3, 16)],
             target_psnr=f64(40), eb_rel=f64(48), eb_abs=f64(56), vr=f64(64), xmin=f32(72),
             xmax=f32(76), s=f32(80), inv=f32(84), thr=f32(88), flags=u32(92), radius=u32(96),
             chunk=u32(100), lmax=u32(104), n_sym=u32(108), n_chunks=u32(112),
             stream_words=u32(116), n_outlier=u32(120), n_verbatim=u32(124))
    pad = lambda v: (v + 15) & ~15
    o_cb = HEADER_BYTES
    o_ct = o_cb + pad(4 * h["n_sym"])
    o_st = o_ct + pad(4 * h["n_chunks"])
    o_ou = o_st + pad(4 * h["stream_words"])
    o_vb = o_ou + pad(8 * h["n_outlier"])
    end = o_vb + pad(8 * h["n_verbatim"])
    h["codebook"] = np.frombuffer(blob, np.uint32, h["n_sym"], o_cb)
    h["chunk_table"] = np.frombuffer(blob, np.uint32, h["n_chunks"], o_ct)
    h["stream"] = np.frombuffer(blob, np.uint32, h["stream_words"], o_st)
    ou = np.frombuffer(blob, np.uint32, 2 * h["n_outlier"], o_ou).reshape(-1, 2)
    vb = np.frombuffer(blob, np.uint32, 2 * h["n_verbatim"], o_vb).reshape(-1, 2)
    h["out_idx"], h["out_delta"] = ou[:, 0], ou[:, 1].view(np.int32)
    h["vb_idx"], h["vb_bits"] = vb[:, 0], vb[:, 1]
    h["total"] = end
    del b
    return h


FINE_BINS = 4096


def fine_hist(x: np.ndarray, xmin: float, vr: float) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    h = np.zeros(FINE_BINS, np.uint32)
    lib().or_fine_hist(_ptr(x), x.size, C.c_float(xmin), float(vr), _ptr(h))
    return h


def pred_mse(h: np.ndarray, n: int, r: float) -> float:
    """Eq. 3's predicted MSE over vr^2 for the relative bound r = eb / vr."""
    h = np.ascontiguousarray(h, dtype=np.uint32)
    return lib().or_pred_mse(_ptr(h), int(n), float(r))


def sum_exact(h, t) -> float:
    """sum(h[i] * t[i]) for uint32 counts and finite non-negative float32
    terms, computed exactly and rounded once to the nearest double."""
    h = np.ascontiguousarray(h, dtype=np.uint32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    assert h.size == t.size
    return lib().or_sum_exact(_ptr(h), _ptr(t), h.size)


def refine_eb(h: np.ndarray, n: int, vr: float, eb0: float, mse_rel: float) -> float:
    """Largest eb in [eb0/4, 64 eb0] with pred_mse(h, n, eb / vr) <= mse_rel."""
    h = np.ascontiguousarray(h, dtype=np.uint32)
    return lib().or_refine_eb(_ptr(h), int(n), float(vr), float(eb0), float(mse_rel))


def _zcall(fn, data: bytes) -> bytes:
    buf = np.frombuffer(data, dtype=np.uint8).copy() if data else np.zeros(1, np.uint8)
    out = C.c_void_p()
    nb = C.c_uint64()
    rc = fn(_ptr(buf), len(data), C.byref(out), C.byref(nb))
    if rc:
        raise ValueError(f"lossless layer failed with status {rc}")
    try:
        return C.string_at(out.value, nb.value)
    finally:
        lib().or_free(out)


def zrle_wrap(raw: bytes) -> bytes:
    return _zcall(lib().or_zrle_wrap, raw)


def zrle_unwrap(data: bytes) -> bytes:
    return _zcall(lib().or_zrle_unwrap, data)
