"""fpsnr_psnr_static, the PSNR entry point that allocates no device memory.

It serves callers that cannot allocate device memory while they run (inside an
allocator's or memory pool's own callback, under a fixed reserved memory
budget, or in a service loop that must stay out of the CUDA allocator because
cudaMalloc/cudaFree can synchronize the device).  Its scratch is one fixed
device array inside the library.  This file runs last on purpose (pytest
collects it last), so a failure here leaves every other test already run; it
also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1805_07384_gb300 import synth

pytestmark = pytest.mark.gpu

PSNR_TOL_DB = 1e-9


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07384_gb300 import build, fpsnr
    build.build()
    fpsnr.load()
    return torch, fpsnr


def reconstruction(env, x, psnr):
    torch, fpsnr = env
    plan = fpsnr.Plan(x.shape, psnr)
    xt = torch.from_numpy(x).cuda()
    out, nb, _ = plan.compress(xt)
    xr, status = plan.decompress(out, out.numel())
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    plan.close()
    return xt, xr


def test_static_psnr_matches_allocating_entry_point(env):
    """Two calls in a row (different fields, so stale scratch would show),
    each checked against fpsnr_psnr through the C ABI."""
    torch, fpsnr = env
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(synth.single_2d(512, seed=3), 80.0),
             (synth.rescale(synth.grf((700, 1300), 2.5, 8), -4.0, 9.0).astype(np.float32), 40.0)]
    for x, psnr in cases:
        xt, xr = reconstruction(env, x, psnr)
        ref = fpsnr.fpsnr_psnr(xt.data_ptr(), xr.data_ptr(), xt.numel(), stream)
        got = fpsnr.fpsnr_psnr_static(xt.data_ptr(), xr.data_ptr(), xt.numel(), stream)
        assert abs(got[0] - ref[0]) < PSNR_TOL_DB
        assert got[1] == pytest.approx(ref[1], rel=1e-12, abs=0)
        assert got[2] == ref[2]
        assert abs(got[0] - psnr) < 0.2


def test_static_psnr_rejects_sizes_beyond_its_scratch(env):
    torch, fpsnr = env
    with pytest.raises(fpsnr.FpsnrError) as e:
        fpsnr.fpsnr_psnr_static(256, 256, fpsnr.FPSNR_PSNR_STATIC_MAX_POINTS + 1)
    assert e.value.code == fpsnr.FPSNR_EINVAL
