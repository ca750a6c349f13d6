"""Decompression from the blob alone (fpsnr_blob_info, fpsnr_plan_from_blob):
the header is read back from the bytes of plain blobs and of the lossless
container, a plan is made from it, and the reconstruction equals the
oracle's, for every predictor dimension, non-default options and degenerate
fields.  Corrupt or truncated headers are refused on the host."""
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


def cases():
    rng = np.random.default_rng(31)
    flat = synth.single_2d(300, 4).copy()
    flat[40:260, 30:280] = flat.min()  # long zero runs at 40 dB: the container wins
    return [
        (synth.single_2d(256, 1), 80.0, dict()),
        (synth.smooth_3d((20, 30, 44), 2), 60.0, dict(radius=512, chunk=128, lmax=16)),
        (synth.smooth_1d(5000, 3), 100.0, dict(chunk=64)),
        (synth.smooth_3d((9, 17, 33), 5), 70.0, dict(lorenzo_dims=2)),
        (np.full((40, 50), 2.5, np.float32), 80.0, dict()),
        (flat, 40.0, dict(lossless=1)),
        (rng.uniform(-1, 1, (64, 64)).astype(np.float32), 90.0, dict(lossless=1)),
    ]


def test_decompress_knowing_only_the_bytes(env):
    torch, fpsnr, oracle = env
    containers = 0
    for i, (x, psnr, kw) in enumerate(cases()):
        plan = fpsnr.Plan(x.shape, psnr, **kw)
        out, nb, _ = plan.compress(torch.from_numpy(np.ascontiguousarray(x)).cuda())
        torch.cuda.synchronize()
        n = int(nb.item())
        blob = out[:n].clone()  # only the bytes travel on
        plan.close()
        del out
        ob, _ = oracle.compress(x, psnr, **kw)
        raw = oracle.zrle_unwrap(ob) if kw.get("lossless") else ob
        containers += raw != ob
        h = fpsnr.fpsnr_blob_info(blob.data_ptr(), n).as_dict()
        ph = oracle.parse_blob(raw)
        assert h["ndim"] == x.ndim and tuple(reversed(h["dims"][:x.ndim])) == x.shape, i
        assert h["points"] == x.size and h["raw_bytes"] == len(raw), i
        assert h["lossless"] == int(raw != ob), i
        for k in ("lorenzo_dims", "radius", "chunk", "lmax", "flags", "n_outlier", "n_verbatim"):
            assert h[k] == ph[k], (i, k)
        for k in ("target_psnr", "eb_rel", "eb_abs", "vr", "xmin", "xmax"):
            assert h[k] == ph[k], (i, k)
        # the same header from host memory
        assert fpsnr.fpsnr_blob_info(np.frombuffer(ob, np.uint8).ctypes.data, n).as_dict() == h
        p2 = fpsnr.Plan.from_blob(blob, n)
        assert p2.shape == x.shape
        xr, status = p2.decompress(blob, n)
        torch.cuda.synchronize()
        assert int(status.item()) == 0, i
        oxr = oracle.decompress(ob, x.shape)
        assert np.array_equal(xr.cpu().numpy().view(np.uint32), oxr.view(np.uint32)), i
        p2.close()
    assert containers >= 1


def test_blob_info_refuses_bad_headers(env):
    torch, fpsnr, oracle = env
    x = synth.single_2d(64, 2)
    ob, _ = oracle.compress(x, 60.0)
    good = np.frombuffer(ob, np.uint8).copy()

    def code(buf, n=None):
        try:
            fpsnr.fpsnr_blob_info(buf.ctypes.data, len(buf) if n is None else n)
            return 0
        except fpsnr.FpsnrError as e:
            return e.code

    assert code(good) == 0
    bad = good.copy()
    bad[0] ^= 1  # magic
    assert code(bad) == fpsnr.FPSNR_ECORRUPT
    bad = good.copy()
    bad[8] = 4  # ndim 4
    assert code(bad) == fpsnr.FPSNR_ECORRUPT
    assert code(good, 100) == fpsnr.FPSNR_ECORRUPT       # shorter than the header
    assert code(good, len(ob) - 16) == fpsnr.FPSNR_ECORRUPT  # sections cut off
    flat = cases()[5][0]
    zb, _ = oracle.compress(flat, 40.0, lossless=1)
    zc = np.frombuffer(zb, np.uint8).copy()
    assert zc[:4].tobytes() == b"FPZ1" and code(zc) == 0
    bad = zc.copy()
    bad[36] ^= 0x40  # the first segment's end offset
    assert code(bad) == fpsnr.FPSNR_ECORRUPT
    bad = zc.copy()
    bad[8] ^= 1  # the expanded size no longer matches the header inside
    assert code(bad) == fpsnr.FPSNR_ECORRUPT
