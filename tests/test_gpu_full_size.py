"""The workloads at their full sizes, through the batched calls the
benchmark uses.

Hurricane-like fields (100 x 500 x 500, 25 M points): all 13 (the vortex
field, the two spiked ones, every target from 30 to 120 dB) in one batch,
bytes and floats checked against the oracle.  NYX-like fields (512^3, 134 M
points): the six of the benchmark in its launch configuration (three
sub-batches on concurrent streams); every point satisfies |x - x'| <= eb and
the reported PSNR equals the standalone reduction's; the lognormal density
at 40 dB and a velocity component at 80 dB match the oracle byte for byte and
float for float.  Climate-like fields: the 24 of the 2D benchmark in its
launch configuration.
"""
import math

import numpy as np
import pytest

from paper_1805_07384_gb300 import synth
from test_gpu_parity import env  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _batch(env, fields, psnrs):
    torch, fpsnr, _ = env
    plans = [fpsnr.Plan(tuple(x.shape), p) for x, p in zip(fields, psnrs)]
    xs = [x if hasattr(x, "is_cuda") else torch.from_numpy(np.ascontiguousarray(x)).cuda()
          for x in fields]
    outs, nb, st = fpsnr.compress_batch(plans, xs)
    recs, status = fpsnr.decompress_batch(plans, outs)
    torch.cuda.synchronize()
    stats = [fpsnr.parse_stats(st[i]) for i in range(len(fields))]
    assert all(s["status"] == 0 for s in stats)
    assert all(int(status[i].item()) == 0 for i in range(len(fields)))
    return plans, xs, outs, nb, stats, recs


def _properties(env, x, xr, st):
    torch, fpsnr, _ = env
    err = (x.double() - xr.double()).abs().max().item()
    assert err <= st["eb_abs"]
    p, _, vr = fpsnr.psnr(x, xr)
    assert vr == st["vr"]
    assert (math.isinf(p) and math.isinf(st["psnr_actual"])) or abs(p - st["psnr_actual"]) < 1e-9


def _against_oracle(env, x_np, psnr, blob, rec, st):
    """Bytes, floats, counts and the error sum of one field against the oracle."""
    torch, fpsnr, oracle = env
    ob, ost = oracle.compress(x_np, psnr)
    assert blob.numel() == len(ob) and blob.cpu().numpy().tobytes() == ob
    oxr = oracle.decompress(ob, x_np.shape)
    assert np.array_equal(rec.cpu().numpy().view(np.uint32), oxr.view(np.uint32))
    assert st["n_outlier"] == ost["n_outlier"] and st["n_verbatim"] == ost["n_verbatim"]
    assert st["sse"] == pytest.approx(ost["sse"], rel=1e-12, abs=0)


def test_hurricane_full_size(env):
    torch, fpsnr, oracle = env
    fields, meta = synth.hurricane_batch(13, device=torch.device("cuda"))
    assert fields[0].shape == (100, 500, 500) and meta[0]["vortex"]
    assert sum(m["spikes"] > 0 for m in meta) == 2
    psnrs = [m["psnr"] for m in meta]
    assert sorted(set(psnrs)) == [30.0 + 10 * k for k in range(10)]
    plans, xs, outs, nb, stats, recs = _batch(env, fields, psnrs)
    for i in range(len(fields)):
        _properties(env, xs[i], recs[i], stats[i])
        _against_oracle(env, xs[i].cpu().numpy(), psnrs[i], outs[i][:int(nb[i].item())], recs[i],
                        stats[i])


def _bench_layout(env, xs, psnrs, nsub=3):
    """Fields dealt by decreasing target into `nsub` sub-batches, each
    compressed and decompressed by one batched call on its own stream, the
    streams concurrent (the benchmark's launch configuration)."""
    torch, fpsnr, _ = env
    F = len(xs)
    dealt = sorted(range(F), key=lambda i: (-psnrs[i], i))
    groups = [sorted(dealt[g::nsub]) for g in range(nsub)]
    plans = [fpsnr.Plan(tuple(x.shape), p) for x, p in zip(xs, psnrs)]
    streams = [torch.cuda.Stream() for _ in groups]
    res = {}
    torch.cuda.synchronize()
    for s, idx in zip(streams, groups):
        with torch.cuda.stream(s):
            gp = [plans[i] for i in idx]
            outs, nb, st = fpsnr.compress_batch(gp, [xs[i] for i in idx], stream=s)
            recs, status = fpsnr.decompress_batch(gp, outs, stream=s)
            res[tuple(idx)] = (outs, nb, st, recs, status)
    torch.cuda.synchronize()
    got = {}
    for idx, (outs, nb, st, recs, status) in res.items():
        for k, i in enumerate(idx):
            s = fpsnr.parse_stats(st[k])
            assert s["status"] == 0 and int(status[k].item()) == 0, i
            _properties(env, xs[i], recs[k], s)
            got[i] = (outs[k][:int(nb[k].item())], recs[k], s)
    return plans, got


def test_cosmology_full_size(env):
    torch, fpsnr, oracle = env
    fields, kinds = synth.cosmology_fields(512, seed=3, device=torch.device("cuda"))
    xs = [f.contiguous() for f in fields]
    del fields
    psnrs = [(40.0, 60.0, 80.0)[i % 3] for i in range(6)]
    plans, got = _bench_layout(env, xs, psnrs)
    assert kinds[0] == "density" and psnrs[0] == 40.0
    assert kinds[2] == "velocity" and psnrs[2] == 80.0
    for i in (0, 2):
        blob, rec, st = got[i]
        _against_oracle(env, xs[i].cpu().numpy(), psnrs[i], blob, rec, st)
    for p in plans:
        p.close()


def test_climate_batch_in_bench_configuration(env):
    """The benchmark's workload in its launch configuration: 24 fields of
    1800x3600 at the mixed targets, dealt into 3 sub-batches by decreasing
    target, each compressed and decompressed by one batched call on its own
    stream, the three streams concurrent.  Every field meets its bound and
    reports the standalone PSNR; three sampled fields (a 120 dB one, a 40 dB
    one and the one with a constant rectangle) match the oracle byte for byte
    and float for float."""
    torch, fpsnr, oracle = env
    F = 24
    fields, meta = synth.climate_batch(F)
    psnrs = [synth.mixed_psnr(i) for i in range(F)]
    xs = [torch.from_numpy(f).cuda() for f in fields]
    plans, got = _bench_layout(env, xs, psnrs)
    const = [i for i, m in enumerate(meta) if m["const_rect"]][0]
    sample = sorted({next(i for i in range(F) if psnrs[i] == 120.0),
                     next(i for i in range(F) if psnrs[i] == 40.0), const})
    for i in sample:
        blob, rec, s = got[i]
        _against_oracle(env, fields[i], psnrs[i], blob, rec, s)
