"""Failure handling on the GPU without a fault: every wait of one thread block
on another has an iteration limit, after which the kernel records
FPSNR_ETIMEOUT in the device status and returns.  The test makes the waits
run out on purpose (fpsnr_plan_set_wait_limit's test switch: the look-back
scans wait for a flag that no block ever sets), reads the status on the host,
and then checks that the same plan, stream and context still decompress
correctly."""
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


# 1D: look-back along the one row (about 250 tiles); wide 2D rows: look-back
# along x, then along y between segments of 16 rows
CASES = [(synth.smooth_1d(1 << 20, 7), 90.0),
         (synth.rescale(synth.grf((40, 9001), 3.0, 9), -1.0, 1.0).astype(np.float32), 70.0)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_unmet_waits_time_out_and_the_plan_recovers(env, case):
    torch, fpsnr, oracle = env
    x, psnr = CASES[case]
    plan = fpsnr.Plan(x.shape, psnr)
    out, nb, st = plan.compress(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    n = int(nb.item())
    assert fpsnr.parse_stats(st)["status"] == 0
    assert fpsnr.fpsnr_plan_set_wait_limit(plan.handle, 2000, 1) == 0
    xr, status = plan.decompress(out, n)
    torch.cuda.synchronize()  # the kernels returned: the waits gave up
    assert int(status.item()) == fpsnr.FPSNR_ETIMEOUT
    # back to the default limit: the same plan decodes the same blob exactly
    assert fpsnr.fpsnr_plan_set_wait_limit(plan.handle, 0, 0) == 0
    xr, status = plan.decompress(out, n)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ob, _ = oracle.compress(x, psnr)
    assert out[:n].cpu().numpy().tobytes() == ob
    oxr = oracle.decompress(ob, x.shape)
    assert np.array_equal(xr.cpu().numpy().view(np.uint32), oxr.view(np.uint32))
    plan.close()


def test_wait_limit_arguments(env):
    torch, fpsnr, _ = env
    plan = fpsnr.Plan((100,), 60.0)
    assert fpsnr.fpsnr_plan_set_wait_limit(plan.handle, 5, 2) == fpsnr.FPSNR_EINVAL
    assert fpsnr.fpsnr_plan_set_wait_limit(0, 5, 0) == fpsnr.FPSNR_EINVAL
    assert fpsnr.fpsnr_plan_set_wait_limit(plan.handle, 1 << 20, 0) == 0
    plan.close()
