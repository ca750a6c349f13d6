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


def test_wrappers_check_arguments_before_enqueueing(lib):
    """The Python layer rejects mismatched lists and tensors that are not
    contiguous CUDA tensors of the right type before anything reaches the C
    side (which sees bare pointers and cannot check them)."""
    import types

    import torch

    # low-level batch wrappers: one entry per plan in every list
    with pytest.raises(ValueError, match="d_in has 1 entries for 2 plans"):
        lib.fpsnr_compress_batch([1, 2], [8], [16, 24], [4, 4])
    with pytest.raises(ValueError, match="blob_bytes has 3 entries"):
        lib.fpsnr_decompress_batch([1, 2], [8, 8], [4, 4, 4], [16, 24])
    # torch wrappers
    x = torch.zeros(6, dtype=torch.float32)
    with pytest.raises(TypeError, match="CUDA tensor"):
        lib.psnr(x, x)
    fake = [types.SimpleNamespace(n=6, handle=None, shape=(6,)) for _ in range(2)]
    with pytest.raises(ValueError, match="xs has 1 entries for 2 plans"):
        lib.compress_batch(fake, [x])
    with pytest.raises(ValueError, match="empty batch"):
        lib.compress_batch([], [])
    with pytest.raises(TypeError, match=r"xs\[0\] must be a CUDA tensor"):
        lib.compress_batch(fake, [x, x], outs=[x, x], nbytes=x, stats=x)
    with pytest.raises(ValueError, match="blobs has 1 entries"):
        lib.decompress_batch(fake, [x])


def test_ctypes_layouts_match_the_header(lib, tmp_path):
    """Every struct the binding mirrors has the size and field offsets that a
    C compiler gives the declaration in include/fpsnr.h."""
    import ctypes
    import subprocess

    structs = [lib.fpsnr_opts, lib.fpsnr_stats, lib.fpsnr_tuning, lib.fpsnr_server_opts,
               lib.fpsnr_request, lib.fpsnr_result, lib.fpsnr_server_stats, lib.fpsnr_blob_header]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "fpsnr.h"', "int main(void) {"]
    want = []
    for s in structs:
        name = s.__name__
        lines.append(f'printf("%zu\\n", sizeof({name}));')
        want.append(ctypes.sizeof(s))
        for f, _ in s._fields_:
            lines.append(f'printf("%zu\\n", offsetof({name}, {f}));')
            want.append(getattr(s, f).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == want
