"""Batched multi-field launches (fpsnr_compress_batch / fpsnr_decompress_batch):
every field's bytes and reconstruction equal those of a separate call and the
oracle's, for a batch that mixes shapes, predictor dimensions, targets,
radii, chunk sizes and degenerate fields, and for batches larger than one
launch covers."""
import numpy as np
import pytest

from paper_1805_07384_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(oracle):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07384_gb300 import build, fpsnr
    build.build()
    fpsnr.load()
    return torch, fpsnr, oracle


def mixed_cases():
    rng = np.random.default_rng(5)
    cases = [
        (synth.single_2d(256, 1), 80.0, dict()),
        (synth.smooth_3d((20, 30, 44), 2), 60.0, dict()),
        (synth.smooth_1d(5000, 3), 100.0, dict()),
        (synth.uniform_noise((90, 130), 4), 120.0, dict()),          # large alphabet
        (np.full((33, 17), 1.5, np.float32), 80.0, dict()),          # constant
        (synth.single_2d(128, 6), 40.0, dict(radius=4, lmax=10)),    # outliers
        (synth.smooth_3d((9, 12, 16), 7), 90.0, dict(lorenzo_dims=2)),
        (synth.single_2d(200, 8)[:, :150].copy(), 70.0, dict(chunk=64)),
    ]
    return cases


def check_batch(env, cases):
    torch, fpsnr, oracle = env
    plans = [fpsnr.Plan(x.shape, p, **kw) for x, p, kw in cases]
    xs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x, _, _ in cases]
    outs, nbytes, stats = fpsnr.compress_batch(plans, xs)
    torch.cuda.synchronize()
    nb = nbytes.cpu().tolist()
    for i, (x, p, kw) in enumerate(cases):
        st = fpsnr.parse_stats(stats[i])
        assert st["status"] == 0, (i, st["status"])
        ob, ost = oracle.compress(x, p, **kw)
        blob = outs[i][: nb[i]].cpu().numpy().tobytes()
        assert blob == ob, f"field {i}: bytes differ from the oracle"
    recs, status = fpsnr.decompress_batch(plans, outs, nb)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0] * len(cases)
    for i, (x, p, kw) in enumerate(cases):
        ob, _ = oracle.compress(x, p, **kw)
        oxr = oracle.decompress(ob, x.shape)
        assert np.array_equal(recs[i].cpu().numpy().view(np.uint32), oxr.view(np.uint32)), i
    return plans, xs, outs, nb


def test_batch_mixed_fields(env):
    check_batch(env, mixed_cases())


def test_batch_equals_single_calls_and_repeats(env):
    torch, fpsnr, _ = env
    cases = mixed_cases()
    plans, xs, outs, nb = check_batch(env, cases)
    # the same plans again, one field at a time
    for i, pl in enumerate(plans):
        out, n1, _ = pl.compress(xs[i])
        torch.cuda.synchronize()
        assert int(n1.item()) == nb[i]
        assert torch.equal(out[: nb[i]], outs[i][: nb[i]])
    # and batched once more (state left by single calls is clean)
    check_batch(env, cases)


def test_batch_larger_than_one_launch(env):
    cases = [(synth.single_2d(64, s), 40.0 + 2 * s, dict()) for s in range(40)]
    check_batch(env, cases)


def test_batch_error_stays_in_its_field(env):
    torch, fpsnr, oracle = env
    good = synth.single_2d(96, 2)
    bad = good.copy()
    bad[5, 5] = np.nan
    plans = [fpsnr.Plan(good.shape, 80.0) for _ in range(3)]
    xs = [torch.from_numpy(a).cuda() for a in (good, bad, good)]
    outs, nbytes, stats = fpsnr.compress_batch(plans, xs)
    torch.cuda.synchronize()
    sts = [fpsnr.parse_stats(stats[i])["status"] for i in range(3)]
    assert sts == [0, fpsnr.FPSNR_ENONFINITE, 0]
    ob, _ = oracle.compress(good, 80.0)
    nb = nbytes.cpu().tolist()
    assert nb[1] == 0
    for i in (0, 2):
        assert outs[i][: nb[i]].cpu().numpy().tobytes() == ob


def test_batch_rejects_repeated_plan(env):
    torch, fpsnr, _ = env
    x = torch.zeros((16, 16), device="cuda")
    pl = fpsnr.Plan((16, 16), 80.0)
    out = pl.alloc_out()
    rc = fpsnr.fpsnr_compress_batch([pl.handle, pl.handle], [x.data_ptr()] * 2,
                                    [out.data_ptr()] * 2, [out.numel()] * 2)
    assert rc == fpsnr.FPSNR_EINVAL


def test_profiler_counts_every_launch(env):
    """The launch count the benchmark reports is the number of library kernels:
    a batch of 2D fields (band path) takes range, predictor, ranks, codebook,
    the encoder's three kernels, emit and finalize to compress (9), and
    decode setup, decode, outlier scatter, band sum, carry and scan, patch and
    status to decompress (8)."""
    torch, fpsnr, _ = env
    xs = [torch.from_numpy(synth.single_2d(256, s)).cuda() for s in (1, 2)]
    plans = [fpsnr.Plan(tuple(x.shape), p) for x, p in zip(xs, (60.0, 100.0))]
    outs, nb, st = fpsnr.compress_batch(plans, xs)
    fpsnr.decompress_batch(plans, outs)
    torch.cuda.synchronize()
    fpsnr.fpsnr_plan_profile(plans[0].handle, True)
    fpsnr.fpsnr_plan_profile_read(plans[0].handle)
    fpsnr.compress_batch(plans, xs, outs=outs)
    comp = sum(v[1] for v in fpsnr.fpsnr_plan_profile_read(plans[0].handle).values())
    recs, status = fpsnr.decompress_batch(plans, outs)
    dec = sum(v[1] for v in fpsnr.fpsnr_plan_profile_read(plans[0].handle).values())
    torch.cuda.synchronize()
    fpsnr.fpsnr_plan_profile(plans[0].handle, False)
    assert all(int(s) == 0 for s in status.cpu())
    assert (comp, dec) == (9, 8)


def test_wrappers_reject_bad_tensors(env):
    """Wrong dtype, layout, size or capacity raises in Python before anything
    is enqueued; the plan is still usable afterwards."""
    torch, fpsnr, _ = env
    p = fpsnr.Plan((33, 47), 60.0)
    x = torch.rand(33, 47, device="cuda")
    with pytest.raises(TypeError, match="must be torch.float32"):
        p.compress(x.double())
    with pytest.raises(ValueError, match="contiguous"):
        p.compress(torch.rand(47, 33, device="cuda").t())
    with pytest.raises(ValueError, match="elements"):
        p.compress(torch.rand(10, device="cuda"))
    with pytest.raises(TypeError, match="out must be torch.uint8"):
        p.compress(x, out=torch.empty(p.max_bytes, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError, match="stats has"):
        p.compress(x, stats=torch.zeros(4, dtype=torch.uint8, device="cuda"))
    out, nb, st = p.compress(x)
    torch.cuda.synchronize()
    n = int(nb.item())
    with pytest.raises(ValueError, match="outside the blob"):
        p.decompress(out, out.numel() + 1)
    with pytest.raises(TypeError, match="out must be torch.float32"):
        p.decompress(out, n, out=torch.empty(33 * 47, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError, match="xs has 1 entries for 2 plans"):
        fpsnr.compress_batch([p, p], [x])
    with pytest.raises(ValueError, match=r"blob_bytes\[0\]"):
        fpsnr.decompress_batch([p], [out], blob_bytes=[out.numel() + 16])
    with pytest.raises(ValueError, match="elements"):
        fpsnr.psnr(x, torch.rand(5, device="cuda"))
    xr, status = p.decompress(out, n)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert (xr - x).abs().max().item() <= fpsnr.parse_stats(st)["eb_abs"]
    p.close()
