"""Request server: continuous batching over cached plans.

Every result must be identical whether a request runs alone or inside a mix of
other shapes, targets and kinds; the HBM budget must bound the cached plans;
arrival times must be honoured; device statuses must reach the caller.
"""
import numpy as np
import pytest

from paper_1805_07384_gb300 import synth
from test_gpu_parity import env, field_for  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

CASES = [((300, 700), 80.0), ((20, 30, 40), 100.0), ((50000,), 60.0), ((64, 64), 40.0),
         ((300, 700), 120.0), ((9, 130, 7), 70.0), ((1800, 360), 90.0)]


def _field(shape, seed):
    if len(shape) == 3:
        return synth.smooth_3d(shape, seed)
    return field_for(shape, seed)


def _inputs(torch, fpsnr):
    xs = [torch.from_numpy(_field(s, 40 + i)).cuda() for i, (s, _) in enumerate(CASES)]
    caps = [fpsnr.Plan(s, p).max_bytes for s, p in CASES]
    return xs, caps


def test_server_alone_equals_mix(env):
    torch, fpsnr, oracle = env
    xs, caps = _inputs(torch, fpsnr)
    srv = fpsnr.Server(hbm_budget=16 << 30, max_batch=8, streams=3)
    # alone: one request at a time
    alone_blobs, alone_recs = [], []
    for (shape, psnr), x, cap in zip(CASES, xs, caps):
        out = torch.empty(cap, dtype=torch.uint8, device="cuda")
        r = srv.wait(srv.submit_compress(x, psnr, out))
        assert r["status"] == 0, r
        blob = out[:r["out_bytes"]].clone()
        alone_blobs.append(blob)
        rec = torch.empty(shape, dtype=torch.float32, device="cuda")
        r2 = srv.wait(srv.submit_decompress(blob, r["out_bytes"], rec))
        assert r2["status"] == 0
        alone_recs.append(rec)
    # the same against a direct plan call and the oracle
    for (shape, psnr), x, blob in zip(CASES, xs, alone_blobs):
        p = fpsnr.Plan(shape, psnr)
        out, nb, _ = p.compress(x)
        torch.cuda.synchronize()
        assert out[:int(nb.item())].cpu().numpy().tobytes() == blob.cpu().numpy().tobytes()
    ob, _ = oracle.compress(xs[0].cpu().numpy(), CASES[0][1])
    assert alone_blobs[0].cpu().numpy().tobytes() == ob
    # in the mix: every compress and decompress arriving at once, twice over
    tickets = []
    at = srv.now() + 50000.0
    for rep in range(2):
        for i, ((shape, psnr), x, cap) in enumerate(zip(CASES, xs, caps)):
            out = torch.empty(cap, dtype=torch.uint8, device="cuda")
            tickets.append(("c", i, out, srv.submit_compress(x, psnr, out, arrival_us=at)))
            rec = torch.empty(shape, dtype=torch.float32, device="cuda")
            blob = alone_blobs[i]
            tickets.append(("d", i, rec, srv.submit_decompress(blob, blob.numel(), rec, arrival_us=at)))
    for kind, i, buf, t in tickets:
        r = srv.wait(t)
        assert r["status"] == 0, (kind, i, r)
        if kind == "c":
            assert r["out_bytes"] == alone_blobs[i].numel()
            assert torch.equal(buf[:r["out_bytes"]], alone_blobs[i]), i
        else:
            assert torch.equal(buf.view(torch.int32), alone_recs[i].view(torch.int32)), i
    st = srv.stats()
    assert st["completed"] == 2 * len(CASES) + 4 * len(CASES) and st["failed"] == 0
    assert st["batches"] < st["completed"]  # requests were fused
    assert st["p99_us"] >= st["p50_us"] > 0
    srv.close()


def test_server_budget(env):
    torch, fpsnr, _ = env
    shape = (500, 800)
    x = torch.from_numpy(field_for(shape, 5)).cuda()
    probe = fpsnr.Plan(shape, 80.0)
    cap = probe.max_bytes
    slab = None
    srv = fpsnr.Server(hbm_budget=1 << 40, max_batch=4, streams=2)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    srv.wait(srv.submit_compress(x, 80.0, out))
    slab = srv.stats()["plan_bytes"]
    srv.close()
    # room for one plan only: requests of the shape run one after another
    srv = fpsnr.Server(hbm_budget=int(slab * 1.5), max_batch=4, streams=2)
    outs = [torch.empty(cap, dtype=torch.uint8, device="cuda") for _ in range(4)]
    ts = [srv.submit_compress(x, 60.0 + 10 * i, o) for i, o in enumerate(outs)]
    res = [srv.wait(t) for t in ts]
    assert all(r["status"] == 0 for r in res)
    st = srv.stats()
    assert st["plans"] == 1 and st["plan_bytes"] <= int(slab * 1.5)
    # the requests that waited for the busy plan allocated nothing meanwhile
    assert st["plans_created"] == 1
    # a different shape evicts the idle plan
    y = torch.from_numpy(field_for((400, 900), 6)).cuda()
    o2 = torch.empty(fpsnr.Plan((400, 900), 80.0).max_bytes, dtype=torch.uint8, device="cuda")
    assert srv.wait(srv.submit_compress(y, 80.0, o2))["status"] == 0
    assert srv.stats()["plans"] == 1 and srv.stats()["plans_created"] == 2
    srv.close()
    # no room for the plan at all
    srv = fpsnr.Server(hbm_budget=int(slab // 2), max_batch=4, streams=1)
    r = srv.wait(srv.submit_compress(x, 80.0, outs[0]))
    assert r["status"] == fpsnr.FPSNR_ENOMEM
    assert srv.stats()["failed"] == 1
    srv.close()


def test_server_arrival_and_errors(env):
    torch, fpsnr, _ = env
    shape = (128, 256)
    x = torch.from_numpy(field_for(shape, 8)).cuda()
    cap = fpsnr.Plan(shape, 80.0).max_bytes
    srv = fpsnr.Server(hbm_budget=4 << 30, max_batch=4, streams=2)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    at = srv.now() + 30000.0
    t = srv.submit_compress(x, 80.0, out, arrival_us=at)
    assert srv.poll(t) is None
    r = srv.wait(t)
    assert r["status"] == 0 and r["arrival_us"] == pytest.approx(at) and r["start_us"] >= at
    with pytest.raises(fpsnr.FpsnrError):
        srv.poll(t)  # already taken
    with pytest.raises(fpsnr.FpsnrError):
        srv.poll(10 ** 9)  # never issued
    # output too small: the device status comes back
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    assert srv.wait(srv.submit_compress(x, 80.0, small))["status"] == fpsnr.FPSNR_ECAPACITY
    # corrupt blob
    good = out[:r["out_bytes"]].clone()
    bad = good.clone()
    bad[4] ^= 0x5A
    rec = torch.empty(shape, dtype=torch.float32, device="cuda")
    assert srv.wait(srv.submit_decompress(bad, bad.numel(), rec))["status"] == fpsnr.FPSNR_ECORRUPT
    assert srv.wait(srv.submit_decompress(good, good.numel(), rec))["status"] == 0
    # misaligned input is refused at submission
    with pytest.raises(fpsnr.FpsnrError):
        srv._submit(fpsnr.FPSNR_REQ_DECOMPRESS, shape, good.data_ptr() + 4, 100, rec.data_ptr(),
                    rec.numel() * 4, 60.0, 0.0, None, 32768, 256, 27, 0)
    # results in completion order
    ts = {srv.submit_compress(x, 50.0 + 10 * i, torch.empty(cap, dtype=torch.uint8, device="cuda")): i
          for i in range(5)}
    srv.drain()
    got = []
    while True:
        item = srv.take_any()
        if item is None:
            break
        got.append(item)
    assert sorted(t for t, _ in got) == sorted(ts) and all(r["status"] == 0 for _, r in got)
    assert [r["done_us"] for _, r in got] == sorted(r["done_us"] for _, r in got)
    srv.close()
