"""Parity of the CUDA path with the CPU oracle, through the C ABI.

Bit-exact: symbols, compressed bytes, reconstructed floats (integer, byte and
float-bit work).  Achieved PSNR: within 1e-9 dB of the oracle's.  Cases span
several tiles with ragged tails, every predictor dimension, outlier-forcing
radii, chunk sizes, large alphabets (global-memory Huffman path), the length
limit, and the degenerate fields (constant, empty, non-finite, denormal range).
"""
import math

import numpy as np
import pytest

from paper_1805_07384_gb300 import synth

pytestmark = pytest.mark.gpu

PSNR_TOL_DB = 1e-9


@pytest.fixture(scope="module")
def env(oracle):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07384_gb300 import build, fpsnr
    build.build()
    fpsnr.load()
    return torch, fpsnr, oracle


def run_gpu(env, x, psnr, radius=32768, chunk=256, lmax=27, ld=0, plan=None, psnr_mode=0):
    torch, fpsnr, _ = env
    plan = plan or fpsnr.Plan(x.shape, psnr, radius=radius, chunk=chunk, lmax=lmax,
                              lorenzo_dims=ld, psnr_mode=psnr_mode)
    plan.set_psnr(psnr)
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out, nb, st = plan.compress(xt)
    torch.cuda.synchronize()
    stats = fpsnr.parse_stats(st)
    nbytes = int(nb.item())
    blob = out[:nbytes].cpu().numpy().tobytes()
    return plan, xt, out, nbytes, stats, blob


def check_case(env, x, psnr, radius=32768, chunk=256, lmax=27, ld=0, plan=None, psnr_mode=0):
    torch, fpsnr, oracle = env
    plan, xt, out, nbytes, st, blob = run_gpu(env, x, psnr, radius, chunk, lmax, ld, plan, psnr_mode)
    assert st["status"] == 0, fpsnr.fpsnr_strerror(st["status"])
    ob, ost = oracle.compress(x, psnr, radius=radius, chunk=chunk, lmax=lmax, lorenzo_dims=ld,
                              psnr_mode=psnr_mode)
    # symbols
    if x.size and not (ost["flags"] & oracle.FLAG_CONSTANT) and psnr_mode == 0:
        s = oracle.plan_scalars(ost["eb_rel"], ost["xmin"], ost["xmax"], x.size)
        lat = oracle.lattice(x, s, radius, lorenzo_dims=ld)
        gcodes = plan.codes().cpu().numpy().view(np.uint16)
        assert np.array_equal(gcodes, lat["codes"].ravel()), "symbols differ"
    # bytes
    assert nbytes == len(ob), (nbytes, len(ob))
    if blob != ob:
        gh, oh = oracle.parse_blob(blob), oracle.parse_blob(ob)
        for k in ("n_sym", "n_chunks", "stream_words", "n_outlier", "n_verbatim", "flags"):
            assert gh[k] == oh[k], k
        for k in ("codebook", "chunk_table", "stream", "out_idx", "out_delta", "vb_idx", "vb_bits"):
            assert np.array_equal(gh[k], oh[k]), k
        assert blob[:128] == ob[:128], "header differs"
        assert False, "bytes differ"
    # reconstruction
    xr, status = plan.decompress(out, nbytes)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    oxr = oracle.decompress(ob, x.shape)
    assert np.array_equal(xr.cpu().numpy().view(np.uint32), oxr.view(np.uint32)), "floats differ"
    # PSNR (Eq. 4-5)
    if x.size:
        op, omse, ovr = oracle.psnr(x, oxr)
        gp, gmse, gvr = fpsnr.psnr(xt, xr)
        assert gvr == ovr
        if math.isinf(op):
            assert math.isinf(gp) and math.isinf(st["psnr_actual"])
        else:
            assert abs(gp - op) < PSNR_TOL_DB
            assert abs(st["psnr_actual"] - op) < PSNR_TOL_DB
            assert st["sse"] == pytest.approx(ost["sse"], rel=1e-12, abs=0)
    assert st["n_outlier"] == ost["n_outlier"] and st["n_verbatim"] == ost["n_verbatim"]
    assert st["eb_abs"] == ost["eb_abs"] and st["vr"] == ost["vr"]
    return plan, st, ost


# ---------------------------------------------------------------------------
# histogram-refined bound (psnr_mode 1)
# ---------------------------------------------------------------------------

def _refine_fields():
    dens, kinds = synth.cosmology_fields(40, seed=3)
    rng = np.random.default_rng(12)
    return [("density", dens[0]), ("temperature", dens[5]), ("velocity", dens[2]),
            ("climate", field_for((300, 700), 13)),
            ("lognormal1d", np.exp(1.5 * rng.standard_normal(100003)).astype(np.float32)),
            ("uniform", rng.uniform(-2.0, 7.0, (64, 1000)).astype(np.float32)),
            # ranges near 2^100 and 2^-80: Eq. 3 is evaluated in units of vr
            ("lognormal_x2^90", (np.exp(1.5 * rng.standard_normal((50, 600))) * 2.0 ** 90).astype(np.float32)),
            ("lognormal_x2^-90", (np.exp(1.5 * rng.standard_normal((50, 600))) * 2.0 ** -90).astype(np.float32))]


@pytest.mark.parametrize("psnr", [30.0, 40.0, 50.0, 80.0])
def test_parity_refined_eb(env, psnr):
    """Bytes, floats and PSNR with the refined bound: the device must reach the
    oracle's eb bit for bit (same histogram, same float terms, both sums exact
    and rounded once)."""
    for name, x in _refine_fields():
        _, st, ost = check_case(env, x, psnr, psnr_mode=1)
        assert st["eb_abs"] == ost["eb_abs"] and st["eb_rel"] == ost["eb_rel"], name


def test_refined_eb_batch_and_constant(env):
    """Refined and plain fields mixed in one batch; a constant field is left alone."""
    torch, fpsnr, oracle = env
    fields = [x for _, x in _refine_fields()] + [np.full((40, 50), 3.5, np.float32)]
    modes = [1, 0, 1, 1, 0, 1, 1, 0, 1][:len(fields) - 1] + [1]
    plans = [fpsnr.Plan(x.shape, 35.0, psnr_mode=m) for x, m in zip(fields, modes)]
    xs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in fields]
    outs, nb, st = fpsnr.compress_batch(plans, xs)
    torch.cuda.synchronize()
    for i, (x, m) in enumerate(zip(fields, modes)):
        ob, _ = oracle.compress(x, 35.0, psnr_mode=m)
        n = int(nb[i].item())
        assert outs[i][:n].cpu().numpy().tobytes() == ob, i


# ---------------------------------------------------------------------------
# value ranges far from 1: the error sums stay exact (squares in units of the
# bound's exponent on compression, of the largest difference seen in the
# standalone reduction)
# ---------------------------------------------------------------------------

def _extreme_fields():
    rng = np.random.default_rng(17)
    g = synth.rescale(synth.grf((70, 300), 3.0, 4), 0.0, 1.0)
    ln = np.exp(1.5 * rng.standard_normal((60, 333)))
    return [("lognormal_x2^90", (ln * 2.0 ** 90).astype(np.float32)),
            ("lognormal_x2^-90", (ln * 2.0 ** -90).astype(np.float32)),
            ("mixing_ratio_1e-9", (1e-9 + 1e-9 * g).astype(np.float32)),
            ("offset_1e30", (1e30 * (1.0 + 1e-3 * g)).astype(np.float32)),
            ("grf_x2^120", (g * 2.0 ** 120 - 2.0 ** 119).astype(np.float32))]


@pytest.mark.parametrize("psnr", [40.0, 120.0, 170.0])
def test_parity_extreme_ranges(env, psnr):
    for name, x in _extreme_fields():
        _, st, ost = check_case(env, x, psnr)
        assert math.isfinite(st["sse"]), name


# ---------------------------------------------------------------------------
# shapes x predictor dimensions
# ---------------------------------------------------------------------------

SHAPES = [
    ((1,), 1), ((7,), 1), ((1000,), 1), ((100003,), 1),
    ((1, 1), 2), ((1, 517), 2), ((517, 1), 2), ((33, 47), 2), ((64, 64), 2), ((257, 511), 2),
    ((130, 1031), 2), ((9, 130), 1),
    ((1, 1, 1), 3), ((2, 3, 5), 3), ((17, 33, 65), 3), ((9, 130, 7), 3), ((40, 40, 40), 3),
    ((5, 9, 300), 2), ((4, 6, 33), 1),
    # 2D rows of 8*G columns per thread (G = 2, 4) and rows wider than one block
    ((40, 2056), 2), ((37, 5000), 2), ((11, 8200), 2), ((9, 9001), 2),
    # 3D tiles of 32 planes x 16/G rows: several slabs and bands with partial
    # last ones, 4G columns per thread (G = 1, 2, 4) as vectors or one by one,
    # and rows wider than a tile covers (look-back scans)
    ((70, 37, 64), 3), ((33, 17, 130), 3), ((65, 20, 500), 3), ((3, 300, 16), 3),
    ((34, 19, 520), 3), ((5, 25, 1000), 3), ((6, 11, 530), 3), ((35, 9, 1030), 3), ((4, 13, 2048), 3),
    ((3, 6, 1200), 3), ((2, 3, 2100), 3),
]


def field_for(shape, seed):
    if len(shape) == 3 and min(shape) > 1:
        return synth.smooth_3d(shape, seed)
    if len(shape) == 1:
        return synth.smooth_1d(shape[0], seed) if shape[0] > 2 else \
            np.linspace(-1, 1, shape[0]).astype(np.float32)
    g = synth.grf(shape, 3.0, seed) if min(shape) > 1 else \
        np.random.default_rng(seed).standard_normal(shape).cumsum(axis=-1)
    return synth.rescale(g, -1.0, 1.0).astype(np.float32)


@pytest.mark.parametrize("shape,ld", SHAPES, ids=lambda v: str(v))
@pytest.mark.parametrize("psnr", [40.0, 80.0, 120.0])
def test_parity_shapes(env, shape, ld, psnr):
    x = field_for(shape, 3 + len(shape))
    check_case(env, x, psnr, ld=ld)


@pytest.mark.parametrize("radius,lmax", [(4, 27), (2, 27), (64, 8), (300, 12)])
@pytest.mark.parametrize("shape,ld", [((200, 301), 2), ((6000,), 1), ((12, 20, 36), 3)])
def test_parity_small_radius_outliers(env, radius, lmax, shape, ld):
    """Tiny radii force outliers; small lmax forces the length-limit rebuild."""
    x = field_for(shape, 21)
    _, st, _ = check_case(env, x, 60.0, radius=radius, lmax=lmax, ld=ld)
    if radius <= 4:
        assert st["n_outlier"] > 0


@pytest.mark.parametrize("chunk", [32, 64, 224, 4096, 65536])
def test_parity_chunk_sizes(env, chunk):
    x = field_for((123, 457), 5)
    check_case(env, x, 90.0, chunk=chunk)


@pytest.mark.parametrize("psnr", [60.0, 100.0, 150.0])
def test_parity_large_alphabet(env, psnr):
    """White noise: thousands of symbols (global-memory Huffman path) and, at
    high PSNR, residuals beyond the radius."""
    x = synth.uniform_noise((300, 400), 11)
    _, st, _ = check_case(env, x, psnr)
    if psnr == 100:
        assert st["n_sym"] > 4096
    if psnr == 150:
        assert st["n_outlier"] > x.size // 2


def test_parity_affine_offsets(env):
    """Climate-like value offsets: float32 spacing near 1e5 vs a tiny range."""
    g = synth.rescale(synth.grf((180, 360), 2.5, 9), -1, 1)
    for scale, offset in ((1e-3, 1e5), (1e4, -3e-3), (2.0, 7.0)):
        x = (offset + scale * g).astype(np.float32)
        for psnr in (40.0, 100.0):
            check_case(env, x, psnr)


def test_parity_repeated_calls_same_plan(env):
    """Plan state (bitmaps, counters, look-back flags) is clean between calls."""
    torch, fpsnr, oracle = env
    shape = (150, 270)
    plan = fpsnr.Plan(shape, 80.0)
    for i, psnr in enumerate((80.0, 150.0, 40.0, 150.0, 120.0)):
        x = synth.uniform_noise(shape, i) if i % 2 else field_for(shape, 30 + i)
        check_case(env, x, psnr, plan=plan)


# ---------------------------------------------------------------------------
# degenerate fields and data-dependent errors
# ---------------------------------------------------------------------------

def test_constant_field(env):
    x = np.full((70, 33), -2.5, np.float32)
    _, st, _ = check_case(env, x, 80.0)
    assert st["bytes"] == 128 and st["flags"] == 1 and math.isinf(st["psnr_actual"])


def test_empty_field(env):
    torch, fpsnr, oracle = env
    x = np.zeros((0, 17), np.float32)
    plan, xt, out, nbytes, st, blob = run_gpu(env, x, 80.0)
    ob, _ = oracle.compress(x, 80.0)
    assert blob == ob and nbytes == 128


def test_lattice_off_denormals(env):
    x = (np.arange(4000, dtype=np.float32) * np.float32(1e-45)).reshape(40, 100)
    _, st, _ = check_case(env, x, 150.0)
    assert st["flags"] == 2


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_nonfinite_input(env, bad):
    torch, fpsnr, oracle = env
    x = field_for((64, 80), 2)
    x[17, 33] = bad
    plan, xt, out, nbytes, st, blob = run_gpu(env, x, 80.0)
    assert st["status"] == fpsnr.FPSNR_ENONFINITE and nbytes == 0
    # the plan stays usable
    check_case(env, field_for((64, 80), 2), 80.0, plan=plan)


def test_capacity_too_small(env):
    torch, fpsnr, oracle = env
    x = field_for((100, 100), 4)
    plan = fpsnr.Plan(x.shape, 80.0)
    xt = torch.from_numpy(x).cuda()
    for cap in (0, 64, 200, 3000):
        out = torch.zeros(max(cap, 16), dtype=torch.uint8, device="cuda")
        nb = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = torch.zeros(fpsnr.STATS_BYTES, dtype=torch.uint8, device="cuda")
        rc = fpsnr.fpsnr_compress(plan.handle, xt.data_ptr(), out.data_ptr(), cap, nb.data_ptr(),
                                  st.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert rc == 0
        s = fpsnr.parse_stats(st)
        assert s["status"] == fpsnr.FPSNR_ECAPACITY and int(nb.item()) == 0
        assert torch.all(out[cap:] == 0)
    check_case(env, x, 80.0, plan=plan)


def test_corrupt_blobs(env):
    torch, fpsnr, oracle = env
    x = field_for((90, 120), 6)
    plan, xt, out, nbytes, st, blob = run_gpu(env, x, 80.0)
    good = out[:nbytes].clone()

    def status_of(buf, nb):
        _, status = plan.decompress(buf, nb)
        torch.cuda.synchronize()
        return int(status.item())

    assert status_of(good, nbytes) == 0
    assert status_of(good, 100) == fpsnr.FPSNR_ECORRUPT          # truncated header
    assert status_of(good, nbytes - 16) == fpsnr.FPSNR_ECORRUPT  # truncated sections
    for off in (0, 4, 8, 16, 96, 100, 108, 112, 116):           # header fields
        b = good.clone()
        b[off] ^= 0x5A
        assert status_of(b, nbytes) == fpsnr.FPSNR_ECORRUPT, off
    b = good.clone()
    b[128 + 1] ^= 0xFF  # codebook entry order / length
    assert status_of(b, nbytes) in (fpsnr.FPSNR_ECORRUPT, 0)
    # random stream damage never faults; status is either ok (garbage) or corrupt
    rng = np.random.default_rng(0)
    for _ in range(5):
        b = good.clone()
        pos = int(rng.integers(200, nbytes))
        b[pos] ^= int(rng.integers(1, 255))
        assert status_of(b, nbytes) in (0, fpsnr.FPSNR_ECORRUPT)
    # shape mismatch with the plan
    other = fpsnr.Plan((90, 121), 80.0)
    _, status = other.decompress(good, nbytes)
    torch.cuda.synchronize()
    assert int(status.item()) == fpsnr.FPSNR_ECORRUPT
    assert status_of(good, nbytes) == 0


@pytest.mark.parametrize("psnr", [30.0, 110.0])
def test_decoder_chunk_overrun_is_corrupt(env, psnr):
    """A chunk whose table entry leaves it no stream words must be reported as
    corrupt (its codes would read past its words), in both decoding modes: at
    30 dB the codes are short and go in pairs, at 110 dB most are longer than
    the 12-bit table and go one by one."""
    torch, fpsnr, _ = env
    x = field_for((300, 500), 8)
    plan, xt, out, nbytes, st, blob = run_gpu(env, x, psnr)
    assert st["status"] == 0
    bits = 8.0 * nbytes / x.size
    assert (bits < 3.0) if psnr == 30.0 else (bits > 9.0), bits
    good = out[:nbytes].clone()
    _, status = plan.decompress(good, nbytes)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    off_ct = 128 + ((4 * st["n_sym"] + 15) & ~15)
    tab = np.frombuffer(blob[off_ct:off_ct + 4 * 64], np.uint32)
    for c in (0, 17, 40):  # chunk c + 1 starts where chunk c starts: c owns no words
        b = good.clone()
        b[off_ct + 4 * (c + 1):off_ct + 4 * (c + 2)] = torch.from_numpy(
            np.array([tab[c]], np.uint32).view(np.uint8).copy()).cuda()
        _, status = plan.decompress(b, nbytes)
        torch.cuda.synchronize()
        assert int(status.item()) == fpsnr.FPSNR_ECORRUPT, c
    _, status = plan.decompress(good, nbytes)
    torch.cuda.synchronize()
    assert int(status.item()) == 0


def test_corrupt_outlier_list(env):
    """The outlier list is checked against the decoded symbols: an index past
    the field, two entries out of order, or an entry moved off its symbol 0
    (leaving a symbol 0 without an entry) are all reported as corrupt."""
    torch, fpsnr, oracle = env
    x = field_for((90, 120), 7)
    plan, xt, out, nbytes, st, blob = run_gpu(env, x, 80.0, radius=16)
    h = oracle.parse_blob(blob)
    no = h["n_outlier"]
    assert no >= 3
    pad = lambda v: (v + 15) & ~15
    o_ou = 128 + pad(4 * h["n_sym"]) + pad(4 * h["n_chunks"]) + pad(4 * h["stream_words"])
    good = out[:nbytes].clone()
    idx = h["out_idx"].astype(np.int64)

    def status_with(entries):
        b = good.clone()
        words = b[o_ou:o_ou + 8 * no].view(torch.int32).view(-1, 2)
        for i, v in entries:
            words[i, 0] = int(v)
        _, status = plan.decompress(b, nbytes)
        torch.cuda.synchronize()
        return int(status.item())

    assert status_with([]) == 0
    assert status_with([(1, x.size + 5)]) == fpsnr.FPSNR_ECORRUPT              # past the field
    assert status_with([(0, idx[1]), (1, idx[0])]) == fpsnr.FPSNR_ECORRUPT     # out of order
    # an entry moved to the next point when that point is not an outlier
    moved = [i for i in range(no) if (i + 1 == no or idx[i] + 1 < idx[i + 1])]
    assert moved
    i = moved[0]
    assert status_with([(i, idx[i] + 1)]) == fpsnr.FPSNR_ECORRUPT
    _, status = plan.decompress(good, nbytes)
    torch.cuda.synchronize()
    assert int(status.item()) == 0


# ---------------------------------------------------------------------------
# workload shapes
# ---------------------------------------------------------------------------

def test_single_2d_512_80db(env):
    """512x512 GRF (P ~ k^-3) at 80 dB, R = 32768: bit-exact and on the model."""
    x = synth.single_2d()
    _, st, ost = check_case(env, x, 80.0)
    assert abs(st["psnr_actual"] - 80.0) < 0.05


@pytest.mark.parametrize("psnr", [40.0, 60.0, 80.0, 100.0, 120.0])
def test_single_2d_sweep(env, psnr):
    check_case(env, synth.single_2d(), psnr)


def test_climate_fields_full_size(env):
    """Three full 1800x3600 climate-like fields, including the one with a
    constant rectangle, at three of the sweep's targets."""
    fields, meta = synth.climate_batch(24)
    pick = [i for i, m in enumerate(meta) if m["const_rect"]][:1] + [0, 7]
    for j, i in enumerate(pick):
        check_case(env, fields[i], synth.PSNR_SWEEP_2D[(2 * j + i) % 5])


def test_hurricane_like_reduced(env):
    """3D fields with the hurricane generator's structure at reduced size
    (vortex mean, spikes, anisotropy), 3D predictor, PSNR 30..120."""
    fields, meta = synth.hurricane_batch(count=4, nz=20, ny=60, nx=70)
    for i, x in enumerate(fields):
        check_case(env, x, 30.0 + 30.0 * i)


def test_cosmology_like_reduced(env):
    """Lognormal (heavy-tailed) and velocity fields at 48^3."""
    fields, kinds = synth.cosmology_fields(n=48)
    for i, x in enumerate(fields):
        check_case(env, x, (40.0, 60.0, 80.0)[i % 3])


# ---------------------------------------------------------------------------
# optional lossless container
# ---------------------------------------------------------------------------

def _flat_field(shape, seed):
    x = field_for(shape, seed).copy()
    x[:, : shape[1] // 2] = x.min()  # a flat region: long runs of the zero residual
    return x


@pytest.mark.parametrize("case", [((300, 700), 30.0), ((300, 700), 40.0), ((257, 511), 60.0),
                                  ((300, 700), 100.0), ((12, 20, 36), 40.0)])
def test_parity_lossless(env, case):
    torch, fpsnr, oracle = env
    shape, psnr = case
    x = synth.smooth_3d(shape, 4) if len(shape) == 3 else _flat_field(shape, 17)
    ob, ost = oracle.compress(x, psnr, lossless=1)
    plain, _ = oracle.compress(x, psnr)
    plan = fpsnr.Plan(shape, psnr, lossless=1)
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out, nb, st = plan.compress(xt)
    torch.cuda.synchronize()
    n = int(nb.item())
    s = fpsnr.parse_stats(st)
    assert s["status"] == 0 and s["bytes"] == n == len(ob)
    assert out[:n].cpu().numpy().tobytes() == ob
    oxr = oracle.decompress(ob, x.shape)
    xr, status = plan.decompress(out, n)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert np.array_equal(xr.cpu().numpy().view(np.uint32), oxr.view(np.uint32))
    # a lossless plan also reads plain blobs; a plain plan refuses containers
    pb = torch.from_numpy(np.frombuffer(plain, np.uint8).copy()).cuda()
    xr2, status = plan.decompress(pb, len(plain))
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and torch.equal(xr2, xr)
    if ob[:4] == b"FPZ1":
        assert len(ob) < len(plain)
        xr3, status = fpsnr.Plan(shape, psnr).decompress(out, n)
        torch.cuda.synchronize()
        assert int(status.item()) == fpsnr.FPSNR_ECORRUPT
        # damaged containers are caught, never a fault
        for off in (4, 16, 20, 33, 40):
            b = out[:n].clone()
            b[off] ^= 0x5A
            _, status = plan.decompress(b, n)
            torch.cuda.synchronize()
            assert int(status.item()) == fpsnr.FPSNR_ECORRUPT, off
        _, status = plan.decompress(out, n)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
    else:
        assert ob == plain


def test_lossless_batch_mixed(env):
    torch, fpsnr, oracle = env
    fields = [_flat_field((200, 400), 21), field_for((200, 400), 22), _flat_field((150, 300), 23)]
    flags = [1, 0, 1]
    plans = [fpsnr.Plan(x.shape, 40.0, lossless=f) for x, f in zip(fields, flags)]
    xs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in fields]
    outs, nb, st = fpsnr.compress_batch(plans, xs)
    recs, status = fpsnr.decompress_batch(plans, outs)
    torch.cuda.synchronize()
    for i, (x, f) in enumerate(zip(fields, flags)):
        ob, _ = oracle.compress(x, 40.0, lossless=f)
        n = int(nb[i].item())
        assert outs[i][:n].cpu().numpy().tobytes() == ob, i
        assert int(status[i].item()) == 0
        assert np.array_equal(recs[i].cpu().numpy().view(np.uint32),
                              oracle.decompress(ob, x.shape).view(np.uint32)), i
