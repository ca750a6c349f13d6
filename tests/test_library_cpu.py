"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every function include/fpsnr.h declares, and rejects bad arguments
before touching the device."""
import math
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_1805_07384_gb300 import build, fpsnr
    build.build()
    return fpsnr


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fpsnr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fpsnr_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    L = lib.load()
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(lib.EXPORTS)


def test_strerror_and_defaults(lib):
    assert lib.fpsnr_strerror(0) == "ok"
    for code in (-1, -2, -3, -4, -5, -6, -7):
        assert lib.fpsnr_strerror(code) not in ("ok", "unknown error")
    assert lib.fpsnr_strerror(-99) == "unknown error"
    o = lib.fpsnr_default_opts()
    assert (o.radius, o.chunk, o.lmax, o.lorenzo_dims) == (32768, 256, 27, 0)


@pytest.mark.parametrize("ndim,dims,psnr,kw", [
    (0, [4], 80.0, {}), (4, [2, 2, 2, 2], 80.0, {}), (2, [4, 4], 0.0, {}),
    (2, [4, 4], -3.0, {}), (2, [4, 4], 180.5, {}), (2, [4, 4], math.nan, {}),
    (2, [4, 4], math.inf, {}), (2, [4, 4], 80.0, {"radius": 0}),
    (2, [4, 4], 80.0, {"radius": 40000}), (2, [4, 4], 80.0, {"chunk": 33}),
    (2, [4, 4], 80.0, {"chunk": 16}), (2, [4, 4], 80.0, {"lmax": 15}),
    (2, [4, 4], 80.0, {"lmax": 28, "radius": 2}), (2, [4, 4], 80.0, {"lorenzo_dims": 3}),
    (3, [2**16, 2**16, 2], 80.0, {}),
])
def test_plan_rejects_bad_arguments(lib, ndim, dims, psnr, kw):
    o = lib.fpsnr_default_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    with pytest.raises(lib.FpsnrError) as e:
        lib.fpsnr_plan(ndim, dims, psnr, o)
    assert e.value.code == lib.FPSNR_EINVAL


def test_null_handles(lib):
    assert lib.fpsnr_max_compressed_bytes(None) == 0
    assert lib.fpsnr_plan_points(None) == 0
    assert math.isnan(lib.fpsnr_plan_eb_rel(None))
    assert lib.fpsnr_plan_set_psnr(None, 80.0) == lib.FPSNR_EINVAL
    assert lib.fpsnr_compress(None, 0, 0, 0) == lib.FPSNR_EINVAL
    assert lib.fpsnr_decompress(None, 0, 0, 0, 0) == lib.FPSNR_EINVAL
    lib.fpsnr_plan_destroy(None)
