"""Mutation check of the oracle's pins: each case plants one plausible mistake
in a copy of oracle/fpsnr_oracle.c (a dropped term, a wrong sign, index,
rounding or bound, a transposed operand), builds it, and runs the pins of
tests/test_oracle_pins.py against it.  Every mutant must make at least one pin
fail; a survivor names a part of the oracle that no pin constrains.

The mistakes are planted on the CPU only, in a temporary copy; the oracle's
own source and library are not touched.  Each mutation keeps every array
access in bounds, so a mutant fails by wrong results, not by a crash.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

from conftest import ROOT

SRC = os.path.join(ROOT, "oracle", "fpsnr_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# name, text of the oracle, replacement (the text must occur exactly once)
MUTANTS = [
    # Eq. 8 and Eq. 7 (Sec. IV)
    ("eq8_drops_sqrt3", "return sqrt(3.0) * pow(10.0, -psnr_db / 20.0);",
     "return pow(10.0, -psnr_db / 20.0);"),
    ("eq8_exponent_over_10", "return sqrt(3.0) * pow(10.0, -psnr_db / 20.0);",
     "return sqrt(3.0) * pow(10.0, -psnr_db / 10.0);"),
    ("eq7_sign_of_log3", "return 20.0 * log10(vr / eb_abs) + 10.0 * log10(3.0);",
     "return 20.0 * log10(vr / eb_abs) - 10.0 * log10(3.0);"),
    # Eq. 5 as read (20 log10 vr - 10 log10 MSE)
    ("eq5_sign_of_mse", "return 20.0 * log10(vr) - 10.0 * log10(mse);",
     "return 20.0 * log10(vr) + 10.0 * log10(mse);"),
    # value range and plan scalars (Sec. IV, bin width 2 eb)
    ("vr_drops_xmin", "p->vr = (double)xmax - (double)xmin;", "p->vr = (double)xmax;"),
    ("bin_width_eb", "double two_eb = 2.0 * p->eb_abs;", "double two_eb = p->eb_abs;"),
    ("threshold_not_below_eb", "float t = (f > 0.0f) ? nextafterf(f, 0.0f) : 0.0f;",
     "float t = f;"),
    # prequantization and reconstruction (Sec. III-IV, midpoint)
    ("prequant_truncates", "return (int32_t)rintf(t);", "return (int32_t)t;"),
    ("prequant_without_anchor", "float t = x - p->xmin;", "float t = x;"),
    ("reconstruct_at_bin_edge", "return fmaf((float)q, p->s, p->xmin);",
     "return fmaf((float)q + 0.5f, p->s, p->xmin);"),
    # Lorenzo residuals (Sec. II-A)
    ("lorenzo_1d_wrong_neighbour", "int64_t prev = (i > 0) ? (int64_t)q[i - 1] : 0;",
     "int64_t prev = (i > 1) ? (int64_t)q[i - 2] : 0;"),
    ("lorenzo_2d_corner_sign", "if (ld == 2) return Q(0, 0, 0) - Q(0, 0, 1) - Q(0, 1, 0) + Q(0, 1, 1);",
     "if (ld == 2) return Q(0, 0, 0) - Q(0, 0, 1) - Q(0, 1, 0) - Q(0, 1, 1);"),
    ("lorenzo_2d_transposed_term",
     "if (ld == 2) return Q(0, 0, 0) - Q(0, 0, 1) - Q(0, 1, 0) + Q(0, 1, 1);",
     "if (ld == 2) return Q(0, 0, 0) - Q(0, 0, 1) - Q(0, 0, 2) + Q(0, 1, 1);"),
    ("lorenzo_3d_drops_corner", "Q(1, 1, 0) - Q(1, 1, 1);", "Q(1, 1, 0);"),
    # symbols and outliers
    ("symbol_offset", "codes[i] = (uint16_t)(d + radius);",
     "codes[i] = (uint16_t)(d + radius - 1);"),
    ("outlier_bound_too_tight", "if (d > -(int64_t)radius && d < (int64_t)radius) {",
     "if (d > -(int64_t)radius && d < (int64_t)radius - 1) {"),
    # verbatim test and error sums (Eq. 4)
    ("verbatim_threshold_doubled", "if (!(fabsf(diff) <= p->thr)) {",
     "if (!(fabsf(diff) <= 2.0f * p->thr)) {"),
    ("sse_counts_verbatim_points",
     "            nv++;\n        } else {\n            sq_add(&acc, x[i], xr);\n        }",
     "            nv++;\n        }\n        sq_add(&acc, x[i], xr);"),
    ("sse_drops_compensation", "static double sq_total(const sq_acc* a) { return a->s + a->c; }",
     "static double sq_total(const sq_acc* a) { return a->s; }"),
    # Huffman construction and canonical codes
    ("huffman_internal_wins_ties",
     "if (li < n && (ii >= next || wt[li] <= wt[ii])) pick[j] = li++;",
     "if (li < n && (ii >= next || wt[li] < wt[ii])) pick[j] = li++;"),
    ("length_limit_quarters_counts", "if (w[s] > 0) w[s] = (w[s] >> 1) > 0 ? (w[s] >> 1) : 1;",
     "if (w[s] > 0) w[s] = (w[s] >> 2) > 0 ? (w[s] >> 2) : 1;"),
    ("canonical_codes_not_extended", "if (i > 0) c = (c + 1) << (v[i].len - v[i - 1].len);",
     "if (i > 0) c = (c + 1);"),
    ("stream_lsb_first", "w |= 1u << (31 - (bitpos % 32));", "w |= 1u << (bitpos % 32);"),
    # decompression (Eq. 1: prefix sums invert the residuals)
    ("decode_symbol_offset", "v[i] = sym ? (int64_t)sym - (int64_t)radius : 0;",
     "v[i] = sym ? (int64_t)sym - (int64_t)radius + 1 : 0;"),
    ("decode_outliers_dropped", "v[idx] = (int32_t)get32(blob, off_ou + 8ull * i + 4);",
     "v[idx] = 0;"),
    ("decode_verbatims_not_patched", "memcpy(&out[idx], &b, 4);", "(void)b;"),
    ("inverse_lorenzo_skips_second_row", "for (uint64_t y = 1; y < ny; y++)",
     "for (uint64_t y = 2; y < ny; y++)"),
    # histogram-refined bound (Eq. 3)
    ("pred_mse_drops_bin_variance", "term[j] = e * e + w212;", "term[j] = e * e;"),
    ("pred_mse_floors", "float q = rintf(c / df);", "float q = floorf(c / df);"),
    ("refine_bisection_reversed",
     "if (or_pred_mse(h, n, mid / vr) <= mse_rel) lo = mid;\n        else hi = mid;",
     "if (or_pred_mse(h, n, mid / vr) <= mse_rel) hi = mid;\n        else lo = mid;"),
    # the exact sum of Eq. 3's terms: another grouping or rounding of it
    ("pred_mse_sequential_double_sum", "return or_sum_exact(h, term, OR_FINE_BINS) / (double)n;",
     "double s = 0.0;\n    for (int j = 0; j < OR_FINE_BINS; j++) s += (double)h[j] * (double)term[j];\n"
     "    return s / (double)n;"),
    ("pred_mse_blocked_pairwise_sum", "return or_sum_exact(h, term, OR_FINE_BINS) / (double)n;",
     "double part[1024];\n    for (int g = 0; g < 1024; g++) {\n        double a = 0.0;\n"
     "        for (int k = 0; k < 4; k++) a += (double)h[4 * g + k] * (double)term[4 * g + k];\n"
     "        part[g] = a;\n    }\n    for (int s2 = 512; s2 >= 1; s2 >>= 1)\n"
     "        for (int i = 0; i < s2; i++) part[i] += part[i + s2];\n    return part[0] / (double)n;"),
    ("exact_sum_truncates", "if (round && (sticky || (mant & 1u))) mant++;", "(void)round;"),
    ("exact_sum_ties_away", "if (round && (sticky || (mant & 1u))) mant++;", "if (round) mant++;"),
    ("exact_sum_drops_sticky", "for (int p = low - 2; p >= 0 && !sticky; p--) sticky = BIT(p);",
     "(void)0;"),
    ("refine_bracket_narrowed", "double lo = eb0 * 0.25, hi = eb0 * 64.0;",
     "double lo = eb0 * 0.25, hi = eb0 * 4.0;"),
    ("refine_gate_at_4_fine_bins", "p.eb_abs * (double)OR_FINE_BINS >= 8.0 * p.vr",
     "p.eb_abs * (double)OR_FINE_BINS >= 2.0 * p.vr"),
    ("fine_hist_rounds", "int b = (int)u; /* truncation toward zero; u >= 0 */",
     "int b = (int)(u + 0.5f);"),
    # range, degenerate fields, plan
    ("nonfinite_not_rejected", "if (!isfinite(v)) return OR_ENONFINITE;", "(void)0;"),
    ("min_tracks_max", "if (i == 0 || v < lo) lo = v;", "if (i == 0 || v > lo) lo = v;"),
    ("constant_field_not_detected", "if (n == 0 || p->vr == 0.0) {", "if (n == 0) {"),
    ("eb_not_scaled_by_vr", "scalars_for_eb(eb_rel * p->vr, p);", "scalars_for_eb(eb_rel, p);"),
    ("eq7_range_term_halved", "return 20.0 * log10(vr / eb_abs) + 10.0 * log10(3.0);",
     "return 10.0 * log10(vr / eb_abs) + 10.0 * log10(3.0);"),
    # lists, single-symbol code, prefix sums over planes
    ("outlier_residual_negated", "out_delta[no] = (int32_t)d; }", "out_delta[no] = (int32_t)-d; }"),
    ("verbatim_bits_flipped", "vb_bits[nv] = b; }", "vb_bits[nv] = b ^ 1u; }"),
    ("single_symbol_length_2", "if (w[s] > 0) len[s] = 1;", "if (w[s] > 0) len[s] = 2;"),
    ("inverse_lorenzo_skips_second_plane", "for (uint64_t z = 1; z < nz; z++)",
     "for (uint64_t z = 2; z < nz; z++)"),
    # zero-run container
    ("zero_run_length_off_by_one", "uint64_t v = k - 1;", "uint64_t v = k;"),
    ("zero_run_codes_equal_size_segments", "rawflag[sg] = c >= len;", "rawflag[sg] = c > len;"),
    ("container_kept_when_larger", "if (total >= raw_bytes) {", "if (total > raw_bytes + 64) {"),
]


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    import oracle

    src = open(SRC).read()
    d = tmp_path_factory.mktemp("oracle_mutants")
    jobs = {}
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, f"{name}: mutation site not found once in the oracle"
        c = d / f"{name}.c"
        c.write_text(src.replace(old, new))
        jobs[name] = (str(c), str(d / f"lib_{name}.so"))
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        list(ex.map(lambda j: oracle.compile_library(*j), jobs.values()))
    return {name: so for name, (_, so) in jobs.items()}


def _run_pins(lib):
    import oracle

    env = dict(os.environ, **{oracle.LIB_ENV: lib})
    return subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_pins_pass_on_the_unchanged_source(tmp_path):
    """Control: the same procedure on an unmodified copy passes every pin."""
    import oracle

    lib = str(tmp_path / "lib_control.so")
    oracle.compile_library(SRC, lib)
    r = _run_pins(lib)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_mutant(mutant_libs, name):
    r = _run_pins(mutant_libs[name])
    # exit status 1: the pins ran and at least one failed (not a crash or a
    # collection error)
    assert r.returncode == 1, f"{name} survived the pins (exit {r.returncode}):\n{r.stdout[-2000:]}"
