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
    each checked against fpsnr_psnr through the C ABI and against the oracle's
    PSNR of the same arrays; neither call changes the device's free memory."""
    import oracle
    torch, fpsnr = env
    stream = torch.cuda.current_stream().cuda_stream
    # the first call on a device loads the library's array onto it (the memory
    # it holds until the process exits); the calls measured below come after
    warm = torch.ones(8, device="cuda")
    fpsnr.fpsnr_psnr_static(warm.data_ptr(), warm.data_ptr(), 8, stream)
    cases = [(synth.single_2d(512, seed=3), 80.0),
             (synth.rescale(synth.grf((700, 1300), 2.5, 8), -4.0, 9.0).astype(np.float32), 40.0)]
    for x, psnr in cases:
        xt, xr = reconstruction(env, x, psnr)
        ref = fpsnr.fpsnr_psnr(xt.data_ptr(), xr.data_ptr(), xt.numel(), stream)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        got = fpsnr.fpsnr_psnr_static(xt.data_ptr(), xr.data_ptr(), xt.numel(), stream)
        assert torch.cuda.mem_get_info()[0] == free0
        assert abs(got[0] - ref[0]) < PSNR_TOL_DB
        assert got[1] == pytest.approx(ref[1], rel=1e-12, abs=0)
        assert got[2] == ref[2]
        op, om, ov = oracle.psnr(x, xr.cpu().numpy())
        assert abs(got[0] - op) < PSNR_TOL_DB and got[2] == ov
        assert got[1] == pytest.approx(om, rel=1e-12, abs=0)
        assert abs(got[0] - psnr) < 0.2


def test_static_psnr_tails_alignment_and_empty(env):
    """An odd point count (the scalar tail), pointers 4 bytes past a 16-byte
    boundary (the kernel without vector loads) and n = 0."""
    import oracle
    torch, fpsnr = env
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(21)
    n = 1_000_003
    x = rng.standard_normal(n + 1).astype(np.float32)
    xr = (x + 1e-3 * rng.standard_normal(n + 1)).astype(np.float32)
    xt, rt = torch.from_numpy(x).cuda(), torch.from_numpy(xr).cuda()
    for off, m in ((0, n), (1, n), (1, n - 2), (0, 7)):
        pa, pb = xt.data_ptr() + 4 * off, rt.data_ptr() + 4 * off
        got = fpsnr.fpsnr_psnr_static(pa, pb, m, stream)
        ref = fpsnr.fpsnr_psnr(pa, pb, m, stream)
        op, om, ov = oracle.psnr(x[off:off + m], xr[off:off + m])
        assert abs(got[0] - ref[0]) < PSNR_TOL_DB and abs(got[0] - op) < PSNR_TOL_DB, (off, m)
        assert got[1] == pytest.approx(om, rel=1e-12, abs=0) and got[2] == ov
    assert fpsnr.fpsnr_psnr_static(0, 0, 0, stream) == (float("inf"), 0.0, 0.0)


def test_static_psnr_at_its_largest_size(env):
    """Exactly FPSNR_PSNR_STATIC_MAX_POINTS points (2 GiB of inputs, the most
    partials the array holds), against fpsnr_psnr."""
    torch, fpsnr = env
    stream = torch.cuda.current_stream().cuda_stream
    n = fpsnr.FPSNR_PSNR_STATIC_MAX_POINTS
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    x = torch.rand(n, generator=g, device="cuda", dtype=torch.float32)
    xr = x + 1e-4 * torch.randn(n, generator=g, device="cuda", dtype=torch.float32)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got = fpsnr.fpsnr_psnr_static(x.data_ptr(), xr.data_ptr(), n, stream)
    assert torch.cuda.mem_get_info()[0] == free0
    ref = fpsnr.fpsnr_psnr(x.data_ptr(), xr.data_ptr(), n, stream)
    assert abs(got[0] - ref[0]) < PSNR_TOL_DB
    assert got[1] == pytest.approx(ref[1], rel=1e-12, abs=0) and got[2] == ref[2]
    del x, xr
    torch.cuda.empty_cache()


def test_static_psnr_rejects_sizes_beyond_its_scratch(env):
    torch, fpsnr = env
    with pytest.raises(fpsnr.FpsnrError) as e:
        fpsnr.fpsnr_psnr_static(256, 256, fpsnr.FPSNR_PSNR_STATIC_MAX_POINTS + 1)
    assert e.value.code == fpsnr.FPSNR_EINVAL
