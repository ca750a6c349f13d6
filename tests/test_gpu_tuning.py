"""Launch shapes and the autotuner.

Tile shapes split the work differently but must never change a byte or a
float: every shape is checked against the default plan and the oracle.  The
autotuner's chunk size does change the bytes (it is a header field), so a
tuned plan is checked against the oracle run at the chunk it picked.
"""
import numpy as np
import pytest

from paper_1805_07384_gb300 import synth
from test_gpu_parity import check_case, env, field_for  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _run(env, plan, xt):
    torch, fpsnr, _ = env
    out, nb, st = plan.compress(xt)
    n = int(nb.item())
    rec, status = plan.decompress(out, n)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return out[:n].cpu().numpy().tobytes(), rec.cpu().numpy(), fpsnr.parse_stats(st)


@pytest.mark.parametrize("shape,psnr", [((300, 2100), 80.0), ((97, 5000), 120.0), ((70, 1031), 40.0)])
def test_tiles_keep_bytes(env, shape, psnr):
    torch, fpsnr, oracle = env
    x = field_for(shape, 31)
    xt = torch.from_numpy(x).cuda()
    base = fpsnr.Plan(shape, psnr)
    blob0, rec0, _ = _run(env, base, xt)
    ob, _ = oracle.compress(x, psnr)
    assert blob0 == ob
    for key, vals in (("pq_tile_x", (128, 256, 512, 1024)), ("band_rows", (16, 32, 64)),
                      ("dec_threads", (128, 256, 512))):
        for v in vals:
            plan = fpsnr.Plan(shape, psnr)
            plan.set_tuning({key: v})
            assert plan.get_tuning()[key] == v
            blob, rec, _ = _run(env, plan, xt)
            assert blob == blob0, (key, v)
            assert np.array_equal(rec.view(np.uint32), rec0.view(np.uint32)), (key, v)
    # all three at once, away from the defaults
    plan = fpsnr.Plan(shape, psnr)
    plan.set_tuning({"pq_tile_x": 128, "band_rows": 64, "dec_threads": 512})
    blob, rec, _ = _run(env, plan, xt)
    assert blob == blob0 and np.array_equal(rec.view(np.uint32), rec0.view(np.uint32))


def test_set_tuning_rejects(env):
    torch, fpsnr, _ = env
    p2 = fpsnr.Plan((64, 300), 60.0, chunk=256)
    p3 = fpsnr.Plan((8, 16, 32), 60.0)
    p2wide = fpsnr.Plan((4, 9000), 60.0)
    for plan, t in ((p2, {"chunk": 512}), (p2, {"pq_tile_x": 64}), (p2, {"band_rows": 8}),
                    (p2, {"dec_threads": 384}), (p3, {"pq_tile_x": 256}), (p3, {"band_rows": 32}),
                    (p2wide, {"band_rows": 16})):
        before = plan.get_tuning()
        with pytest.raises(fpsnr.FpsnrError) as e:
            plan.set_tuning(t)
        assert e.value.code == -1
        assert plan.get_tuning() == before
    p2.set_tuning({"chunk": 256, "pq_tile_x": 256})
    p3.set_tuning({"dec_threads": 128})


@pytest.mark.parametrize("shape,psnr,ld", [((400, 1800), 60.0, 0), ((24, 40, 72), 100.0, 0),
                                           ((200000,), 80.0, 0)])
def test_autotune_parity(env, shape, psnr, ld):
    torch, fpsnr, oracle = env
    x = synth.smooth_3d(shape, 7) if len(shape) == 3 else field_for(shape, 9)
    xt = torch.from_numpy(x).cuda()
    t = fpsnr.autotune(xt, psnr, max_size_increase=0.02, lorenzo_dims=ld)
    assert t["chunk"] in (64, 128, 256, 512, 1024, 2048)
    assert t["ms"] > 0 and t["bytes"] > 0
    # the cache answers the same without timing again
    assert fpsnr.autotune(xt, psnr, max_size_increase=0.02, lorenzo_dims=ld) == t
    plan = fpsnr.Plan(shape, psnr, chunk=t["chunk"], lorenzo_dims=ld)
    plan.set_tuning(t)
    _, st, blob = check_case(env, x, psnr, chunk=t["chunk"], ld=ld, plan=plan)
    assert st["bytes"] == t["bytes"]
    # within the size tolerance of every other chunk size
    for c in (64, 128, 256, 512, 1024, 2048):
        ob, _ = oracle.compress(x, psnr, chunk=c, lorenzo_dims=ld)
        assert t["bytes"] <= len(ob) * 1.02 + 1
