/*
 * fpsnr_oracle.c -- plain, slow, single-threaded CPU oracle for fixed-PSNR
 * lossy compression (Tao, Di, Liang, Chen, Cappello, "Fixed-PSNR Lossy
 * Compression for Scientific Data").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or constant with the
 * CUDA library: the byte format below is written out here independently.
 *
 * Build flags: -O2 -ffp-contract=off (no FMA contraction: every float
 * operation is rounded on its own, exactly as written; the one fused
 * multiply-add of the reconstruction is an explicit fmaf()).
 *
 * What each function follows:
 *   or_eb_rel_from_psnr ... Eq. 8 (Sec. IV): eb_rel = sqrt(3) * 10^(-PSNR/20)
 *   or_psnr_model ........ Eq. 7 (Sec. IV): PSNR = 20 log10(vr/eb) + 10 log10 3
 *   or_range ............. vr = value range of the original data (Sec. IV,
 *                          definition under Eq. 5), max - min in FP64
 *   or_plan_scalars ...... eb_abs = eb_rel * vr (Sec. IV, under Eq. 7);
 *                          SZ bin width 2*eb_abs (Sec. IV, before Eq. 7)
 *   or_lattice ........... steps 1-2 of the prediction-based pipeline
 *                          (Sec. II-A, Sec. III): uniform quantization with
 *                          midpoint reconstruction (Sec. IV, Eq. 2-3 setting)
 *                          and the Lorenzo predictor (Sec. II-A), run on the
 *                          integer lattice q = round((x - xmin) / 2eb)
 *   or_huffman_lengths ... the customized Huffman coding of SZ step 2
 *                          (Sec. II-A); tie-break and length-limit rule are
 *                          this library's reading (the paper is silent)
 *   or_compress / or_decompress ... the whole pipeline and its inverse
 *                          (Sec. III: decompression rebuilds the prediction
 *                          errors, then the data point by point, Eq. 1)
 *   or_fine_hist / or_pred_mse / or_refine_eb ... optional eb refinement:
 *                          Eq. 3 evaluated on the field's empirical PDF (a
 *                          fine histogram) instead of a PDF taken constant
 *                          over each quantization bin, then the largest eb
 *                          whose predicted MSE meets the target (Sec. V notes
 *                          the constant-PDF estimate degrades as bins widen;
 *                          Sec. VI leaves low targets to future work); the
 *                          sum of Eq. 3's terms is exact, rounded once
 *                          (or_sum_exact)
 *   or_zrle_wrap / or_zrle_unwrap ... optional lossless layer over the finished
 *                          blob, standing in for SZ's lossless step 3 (Sec. II-A,
 *                          "optional"; the paper names GZIP): zero-byte runs
 *                          coded per 1 KiB segment
 *   or_sse / or_psnr ..... MSE, NRMSE and PSNR definitions (Eq. 4-5, with the
 *                          sign of Eq. 5 read as PSNR = 20 log10 vr - 10 log10 MSE)
 *   or_classic_sz ........ comparison path: the classic sequential predictor
 *                          that predicts from already-reconstructed values
 *                          (Sec. III, the argument for X_pred = X~_pred)
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_ENONFINITE (-4)
#define OR_ECORRUPT (-6)

#define OR_MAGIC 0x31535046u /* bytes "FPS1" */
#define OR_VERSION 1u
#define OR_HEADER_BYTES 128u
#define OR_FLAG_CONSTANT 1u
#define OR_FLAG_LATTICE_OFF 2u

/* ------------------------------------------------------------------------ */
/* Eq. 8 and Eq. 7                                                           */
/* ------------------------------------------------------------------------ */

/* Eq. 8: value-range-based relative error bound for a target PSNR (dB). */
double or_eb_rel_from_psnr(double psnr_db) { return sqrt(3.0) * pow(10.0, -psnr_db / 20.0); }

/* Eq. 7: PSNR the model predicts for SZ run at absolute bound eb on range vr. */
double or_psnr_model(double vr, double eb_abs) {
    return 20.0 * log10(vr / eb_abs) + 10.0 * log10(3.0);
}

/* ------------------------------------------------------------------------ */
/* value range                                                               */
/* ------------------------------------------------------------------------ */

/* min and max of the float field; returns OR_ENONFINITE if any NaN/Inf. */
int or_range(const float* x, uint64_t n, float* xmin, float* xmax) {
    float lo = 0.0f, hi = 0.0f;
    for (uint64_t i = 0; i < n; i++) {
        float v = x[i];
        if (!isfinite(v)) return OR_ENONFINITE;
        if (i == 0 || v < lo) lo = v;
        if (i == 0 || v > hi) hi = v;
    }
    *xmin = lo;
    *xmax = hi;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* plan scalars: eb, bin width, threshold                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    double eb_rel, eb_abs, vr;
    float xmin, xmax;
    float s;   /* (float)(2 eb): width of one quantization bin */
    float inv; /* (float)(1 / (2 eb)) */
    float thr; /* largest float T with T + half an ulp above T < eb */
    uint32_t flags;
} or_scalars;

/* largest float not above v (v finite, >= 0) */
static float round_down_to_float(double v) {
    float f = (float)v; /* round to nearest */
    if ((double)f > v) f = nextafterf(f, 0.0f);
    return f;
}

/* Bin width, its inverse and the verbatim threshold for absolute bound eb_abs
 * (the caller has checked that the field is not constant). */
static void scalars_for_eb(double eb_abs, or_scalars* p) {
    p->eb_abs = eb_abs;
    double two_eb = 2.0 * p->eb_abs;
    float s = (float)two_eb;
    float inv = (float)(1.0 / two_eb);
    if (!(s > 0.0f) || isinf(inv) || !(p->vr <= (double)FLT_MAX)) {
        /* the lattice cannot be represented in float32: every q is 0 */
        p->flags = OR_FLAG_LATTICE_OFF;
        s = 0.0f;
        inv = 0.0f;
    }
    p->s = s;
    p->inv = inv;
    float f = round_down_to_float(p->eb_abs);
    float t = (f > 0.0f) ? nextafterf(f, 0.0f) : 0.0f;
    p->thr = t > 0.0f ? t : 0.0f;
}

void or_plan_scalars(double eb_rel, float xmin, float xmax, uint64_t n, or_scalars* p) {
    memset(p, 0, sizeof(*p));
    p->eb_rel = eb_rel;
    p->xmin = xmin;
    p->xmax = xmax;
    p->vr = (double)xmax - (double)xmin;
    if (n == 0 || p->vr == 0.0) {
        /* constant (or empty) field: nothing to quantize, exact reconstruction */
        p->flags = OR_FLAG_CONSTANT;
        p->eb_abs = 0.0;
        return;
    }
    scalars_for_eb(eb_rel * p->vr, p);
}

/* ------------------------------------------------------------------------ */
/* optional eb refinement from the empirical PDF (Eq. 3)                     */
/* ------------------------------------------------------------------------ */

#define OR_FINE_BINS 4096   /* bins of the fine histogram over [xmin, xmax] */
#define OR_BISECT_STEPS 16

/* Fine histogram of the field: bin = trunc((x - xmin) * kinv) in float32,
 * kinv = (float)(K / vr), clamped to [0, K - 1]. */
void or_fine_hist(const float* x, uint64_t n, float xmin, double vr, uint32_t* h) {
    const float kinv = (float)((double)OR_FINE_BINS / vr);
    memset(h, 0, OR_FINE_BINS * sizeof(uint32_t));
    for (uint64_t i = 0; i < n; i++) {
        float u = (x[i] - xmin) * kinv;
        int b = (int)u; /* truncation toward zero; u >= 0 */
        if (b < 0) b = 0;
        if (b > OR_FINE_BINS - 1) b = OR_FINE_BINS - 1;
        h[b]++;
    }
}

/* Exact sum of k products h[i] * t[i] (h counts, t finite non-negative
 * floats), rounded once to the nearest double (ties to even).  Every float is
 * an integer multiple of 2^-149, and h * t < 2^32 * 2^128, so the products
 * are added without rounding as integers in units of 2^OR_SUM_LSB, in
 * OR_SUM_LIMBS 32-bit limbs (enough for 4096 terms with room to spare), and
 * the total is rounded to 53 bits at the end.  The order of the terms does
 * not matter: integer addition is exact. */
#define OR_SUM_LIMBS 12
#define OR_SUM_LSB (-172) /* 2^-149 = 2^23 * 2^-172, the smallest float's mantissa times 2^-172 */
double or_sum_exact(const uint32_t* h, const float* t, uint32_t k) {
    uint32_t acc[OR_SUM_LIMBS];
    memset(acc, 0, sizeof(acc));
    for (uint32_t i = 0; i < k; i++) {
        if (h[i] == 0 || t[i] == 0.0f) continue;
        int e;
        const float m = frexpf(t[i], &e); /* t = m 2^e, m in [0.5, 1) */
        const uint64_t mant = (uint64_t)ldexpf(m, 24); /* t = mant 2^(e - 24), mant < 2^24 */
        uint64_t prod = (uint64_t)h[i] * mant; /* < 2^56 */
        int shift = e - 24 - OR_SUM_LSB; /* bit position of prod's lowest bit, >= 0 */
        int limb = shift / 32, bit = shift % 32;
        /* add prod << bit into limbs limb, limb + 1, ... with carries */
        uint64_t carry = 0;
        uint64_t piece[3] = {(prod << bit) & 0xffffffffull, (prod >> (32 - bit)) & 0xffffffffull,
                             bit ? (prod >> (64 - bit)) : 0};
        if (bit == 0) piece[1] = (prod >> 32) & 0xffffffffull;
        for (int j = limb; j < OR_SUM_LIMBS; j++) {
            uint64_t v = (uint64_t)acc[j] + carry + (j - limb < 3 ? piece[j - limb] : 0);
            acc[j] = (uint32_t)v;
            carry = v >> 32;
            if (j - limb >= 2 && carry == 0) break;
        }
    }
    /* highest set bit */
    int top = -1;
    for (int j = OR_SUM_LIMBS - 1; j >= 0 && top < 0; j--)
        for (int b = 31; b >= 0; b--)
            if ((acc[j] >> b) & 1u) { top = 32 * j + b; break; }
    if (top < 0) return 0.0;
#define BIT(p) ((int)((acc[(p) / 32] >> ((p) % 32)) & 1u))
    /* the 53 bits from the top down, then the round bit and the sticky bits */
    const int low = top - 52 > 0 ? top - 52 : 0;
    uint64_t mant = 0;
    for (int p = top; p >= low; p--) mant = (mant << 1) | (uint64_t)BIT(p);
    if (low > 0) {
        const int round = BIT(low - 1);
        int sticky = 0;
        for (int p = low - 2; p >= 0 && !sticky; p--) sticky = BIT(p);
        if (round && (sticky || (mant & 1u))) mant++; /* 2^53 is still exact */
    }
#undef BIT
    return ldexp((double)mant, low + OR_SUM_LSB);
}

/* Eq. 3 with the PDF taken constant over each fine bin rather than over each
 * quantization bin, in units of the value range (Eq. 3 is scale invariant, and
 * in these units every term is a moderate float whatever the field's range):
 * with midpoint reconstruction on the lattice of step 2r (r = eb / vr)
 * anchored at xmin, the fine bin j, of width w = 1/K and centre
 * c = (j + 1/2) w, contributes h_j (e^2 + w^2 / 12), e = c - 2r round(c / 2r).
 * Per-bin terms in float32; their sum exact, rounded once (or_sum_exact).
 * Returns the predicted MSE over vr^2. */
double or_pred_mse(const uint32_t* h, uint64_t n, double r) {
    const double w = 1.0 / (double)OR_FINE_BINS;
    const float df = (float)(2.0 * r);
    const float w212 = (float)(w * w / 12.0);
    float term[OR_FINE_BINS];
    for (int j = 0; j < OR_FINE_BINS; j++) {
        float c = (float)(((double)j + 0.5) * w);
        float q = rintf(c / df);
        float e = c - q * df;
        term[j] = e * e + w212;
    }
    return or_sum_exact(h, term, OR_FINE_BINS) / (double)n;
}

/* Largest eb in [eb0 / 4, 64 eb0] whose predicted MSE over vr^2 does not
 * exceed mse_rel = 10^(-PSNR/10), by OR_BISECT_STEPS bisections on the
 * geometric midpoint. */
double or_refine_eb(const uint32_t* h, uint64_t n, double vr, double eb0, double mse_rel) {
    double lo = eb0 * 0.25, hi = eb0 * 64.0;
    if (or_pred_mse(h, n, lo / vr) > mse_rel) return lo;
    if (or_pred_mse(h, n, hi / vr) <= mse_rel) return hi;
    for (int it = 0; it < OR_BISECT_STEPS; it++) {
        double mid = sqrt(lo * hi);
        if (or_pred_mse(h, n, mid / vr) <= mse_rel) lo = mid;
        else hi = mid;
    }
    return lo;
}

/* ------------------------------------------------------------------------ */
/* Lorenzo predictor on the integer lattice                                  */
/* ------------------------------------------------------------------------ */

/* prequantization of one value: q = round_half_even((x - xmin) * inv) */
static int32_t prequant(float x, const or_scalars* p) {
    if (p->flags & OR_FLAG_LATTICE_OFF) return 0;
    float t = x - p->xmin;
    t = t * p->inv;
    return (int32_t)rintf(t);
}

/* midpoint reconstruction of lattice point q */
static float dequant(int32_t q, const or_scalars* p) { return fmaf((float)q, p->s, p->xmin); }

/* logical shape seen by a d-dimensional Lorenzo predictor: the d-1 fastest
 * axes are kept and all slower axes are merged into the slowest one. */
static void lorenzo_shape(int ndim, const uint64_t* dims, int ld, uint64_t* nx, uint64_t* ny,
                          uint64_t* nz) {
    uint64_t n = 1;
    for (int i = 0; i < ndim; i++) n *= dims[i];
    if (ld == 1) {
        *nx = n; *ny = 1; *nz = 1;
    } else if (ld == 2) {
        *nx = dims[0]; *ny = dims[0] ? n / dims[0] : 0; *nz = 1;
    } else {
        *nx = dims[0]; *ny = dims[1]; *nz = (dims[0] && dims[1]) ? n / (dims[0] * dims[1]) : 0;
    }
}

/* Lorenzo residual of the lattice field q, neighbours outside the field = 0.
 * 1D: q[i] - q[i-1]
 * 2D: q[r][c] - q[r][c-1] - q[r-1][c] + q[r-1][c-1]
 * 3D: 7-neighbour inclusion-exclusion. */
static int64_t lorenzo_residual(const int32_t* q, int ld, uint64_t nx, uint64_t ny, uint64_t i) {
    uint64_t x = i % nx;
    uint64_t y = (i / nx) % ny;
    uint64_t z = i / (nx * ny);
#define Q(dz, dy, dx)                                                                       \
    (((dz) > z || (dy) > y || (dx) > x) ? (int64_t)0                                        \
                                        : (int64_t)q[((z - (dz)) * ny + (y - (dy))) * nx + \
                                                     (x - (dx))])
    if (ld == 1) {
        int64_t prev = (i > 0) ? (int64_t)q[i - 1] : 0;
        return (int64_t)q[i] - prev;
    }
    if (ld == 2) return Q(0, 0, 0) - Q(0, 0, 1) - Q(0, 1, 0) + Q(0, 1, 1);
    return Q(0, 0, 0) - Q(0, 0, 1) - Q(0, 1, 0) - Q(1, 0, 0) + Q(0, 1, 1) + Q(1, 0, 1) +
           Q(1, 1, 0) - Q(1, 1, 1);
#undef Q
}

/* Eq. 4 sums the squared point errors; the definition fixes no order of
 * summation, so the oracle computes the sum as exactly as FP64 allows: each
 * difference is split exactly (TwoSum), each square is exact up to the dl^2
 * term (FMA TwoProd plus the 2*dh*dl cross term), and the running sum is
 * compensated (Neumaier).  A plain running FP64 sum drifts by ~1e-12 relative
 * over 1e5 points, more than the 1e-9 dB the PSNR comparisons are held to. */
typedef struct { double s, c; } sq_acc;

static void sq_add(sq_acc* a, float x, float xr) {
    double u = (double)x, v = -(double)xr;
    double dh = u + v, bb = dh - u;
    double dl = (u - (dh - bb)) + (v - bb);
    double p = dh * dh;
    double pe = fma(dh, dh, -p) + 2.0 * dh * dl;
    double t = a->s + p;
    if (fabs(a->s) >= fabs(p)) a->c += (a->s - t) + p;
    else a->c += (p - t) + a->s;
    a->s = t;
    a->c += pe;
}

static double sq_total(const sq_acc* a) { return a->s + a->c; }

/* Steps 1-2 on every point.  Outputs:
 *   codes[i]      = delta + R if |delta| < R, else 0 (outlier marker)
 *   out_idx/out_delta  the outliers, ascending idx      (may be NULL: count only)
 *   vb_idx/vb_bits     the verbatim points, ascending idx
 *   *sse          = sum over points of (x - x')^2 (sq_add), x' the value the
 *                   decompressor will produce (verbatim points reproduce x)
 * For ld==1 the field is flat; see lorenzo_shape for 2 and 3. */
int or_lattice(const float* x, int ndim, const uint64_t* dims, int ld, const or_scalars* p,
               int32_t radius, uint16_t* codes, uint32_t* out_idx, int32_t* out_delta,
               uint64_t* n_out, uint32_t* vb_idx, uint32_t* vb_bits, uint64_t* n_vb,
               double* sse) {
    uint64_t nx, ny, nz;
    lorenzo_shape(ndim, dims, ld, &nx, &ny, &nz);
    uint64_t n = nx * ny * nz;
    int32_t* q = (int32_t*)malloc((n ? n : 1) * sizeof(int32_t));
    if (!q) return OR_ENOMEM;
    for (uint64_t i = 0; i < n; i++) q[i] = prequant(x[i], p);
    uint64_t no = 0, nv = 0;
    sq_acc acc = {0.0, 0.0};
    for (uint64_t i = 0; i < n; i++) {
        int64_t d = lorenzo_residual(q, ld, nx, ny, i);
        if (d > -(int64_t)radius && d < (int64_t)radius) {
            codes[i] = (uint16_t)(d + radius);
        } else {
            codes[i] = 0;
            if (out_idx) { out_idx[no] = (uint32_t)i; out_delta[no] = (int32_t)d; }
            no++;
        }
        float xr = dequant(q[i], p);
        float diff = x[i] - xr;
        if (!(fabsf(diff) <= p->thr)) {
            if (vb_idx) { uint32_t b; memcpy(&b, &x[i], 4); vb_idx[nv] = (uint32_t)i; vb_bits[nv] = b; }
            nv++;
        } else {
            sq_add(&acc, x[i], xr);
        }
    }
    free(q);
    *n_out = no;
    *n_vb = nv;
    *sse = sq_total(&acc);
    return OR_OK;
}

/* Inverse of the zero-padded Lorenzo residual: inclusive prefix sums along
 * every axis of the predictor's shape (textbook identity: the d-dimensional
 * difference operator is inverted by d nested running sums). */
void or_inverse_lorenzo(int64_t* v, int ld, uint64_t nx, uint64_t ny, uint64_t nz) {
    uint64_t n = nx * ny * nz;
    if (ld == 1) {
        for (uint64_t i = 1; i < n; i++) v[i] += v[i - 1];
        return;
    }
    for (uint64_t z = 0; z < nz; z++)
        for (uint64_t y = 0; y < ny; y++)
            for (uint64_t x = 1; x < nx; x++) v[(z * ny + y) * nx + x] += v[(z * ny + y) * nx + x - 1];
    for (uint64_t z = 0; z < nz; z++)
        for (uint64_t y = 1; y < ny; y++)
            for (uint64_t x = 0; x < nx; x++) v[(z * ny + y) * nx + x] += v[(z * ny + y - 1) * nx + x];
    if (ld == 3)
        for (uint64_t z = 1; z < nz; z++)
            for (uint64_t y = 0; y < ny; y++)
                for (uint64_t x = 0; x < nx; x++)
                    v[(z * ny + y) * nx + x] += v[((z - 1) * ny + y) * nx + x];
}

/* ------------------------------------------------------------------------ */
/* Huffman code lengths (two-queue construction) and canonical codes         */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t w; uint32_t sym; } or_leaf;

static int leaf_cmp(const void* a, const void* b) {
    const or_leaf* x = (const or_leaf*)a;
    const or_leaf* y = (const or_leaf*)b;
    if (x->w != y->w) return x->w < y->w ? -1 : 1;
    return x->sym < y->sym ? -1 : (x->sym > y->sym ? 1 : 0);
}

/* One Huffman construction over weights w (symbols with w == 0 get no code).
 * Leaves are taken in ascending (weight, symbol) order; internal nodes are
 * queued in creation order; when the two queue heads weigh the same, the
 * leaf is taken first.  Returns the maximum length, or -1 on ENOMEM. */
static int huffman_once(const uint64_t* w, uint32_t nsym, uint8_t* len) {
    uint32_t n = 0;
    for (uint32_t s = 0; s < nsym; s++) len[s] = 0;
    for (uint32_t s = 0; s < nsym; s++) n += (w[s] > 0);
    if (n == 0) return 0;
    if (n == 1) {
        for (uint32_t s = 0; s < nsym; s++)
            if (w[s] > 0) len[s] = 1;
        return 1;
    }
    or_leaf* lv = (or_leaf*)malloc(n * sizeof(or_leaf));
    uint64_t* wt = (uint64_t*)malloc((2 * (size_t)n - 1) * sizeof(uint64_t));
    uint32_t* par = (uint32_t*)malloc((2 * (size_t)n - 1) * sizeof(uint32_t));
    uint32_t* dep = (uint32_t*)malloc((2 * (size_t)n - 1) * sizeof(uint32_t));
    if (!lv || !wt || !par || !dep) { free(lv); free(wt); free(par); free(dep); return -1; }
    uint32_t k = 0;
    for (uint32_t s = 0; s < nsym; s++)
        if (w[s] > 0) { lv[k].w = w[s]; lv[k].sym = s; k++; }
    qsort(lv, n, sizeof(or_leaf), leaf_cmp);
    for (uint32_t i = 0; i < n; i++) wt[i] = lv[i].w;
    uint32_t li = 0, ii = n, next = n, total = 2 * n - 1;
    while (next < total) {
        uint32_t pick[2];
        for (int j = 0; j < 2; j++) {
            if (li < n && (ii >= next || wt[li] <= wt[ii])) pick[j] = li++;
            else pick[j] = ii++;
        }
        wt[next] = wt[pick[0]] + wt[pick[1]];
        par[pick[0]] = next;
        par[pick[1]] = next;
        next++;
    }
    dep[total - 1] = 0;
    for (uint32_t i = total - 1; i-- > 0;) dep[i] = dep[par[i]] + 1;
    int maxlen = 0;
    for (uint32_t i = 0; i < n; i++) {
        len[lv[i].sym] = (uint8_t)dep[i];
        if ((int)dep[i] > maxlen) maxlen = (int)dep[i];
    }
    free(lv); free(wt); free(par); free(dep);
    return maxlen;
}

/* Code lengths for counts[nsym], limited to lmax bits: while the longest code
 * exceeds lmax, every nonzero count c becomes max(1, c >> 1) and the tree is
 * rebuilt.  Returns OR_OK, OR_EINVAL if lmax cannot hold the alphabet. */
int or_huffman_lengths(const uint32_t* counts, uint32_t nsym, int lmax, uint8_t* len) {
    uint64_t* w = (uint64_t*)malloc((nsym ? nsym : 1) * sizeof(uint64_t));
    if (!w) return OR_ENOMEM;
    uint32_t used = 0;
    for (uint32_t s = 0; s < nsym; s++) { w[s] = counts[s]; used += counts[s] > 0; }
    if (used > 1 && (lmax >= 63 || ((uint64_t)1 << lmax) < used)) { free(w); return OR_EINVAL; }
    for (;;) {
        int m = huffman_once(w, nsym, len);
        if (m < 0) { free(w); return OR_ENOMEM; }
        if (m <= lmax) break;
        for (uint32_t s = 0; s < nsym; s++)
            if (w[s] > 0) w[s] = (w[s] >> 1) > 0 ? (w[s] >> 1) : 1;
    }
    free(w);
    return OR_OK;
}

typedef struct { uint32_t len, sym; } or_lsym;
static int lsym_cmp(const void* a, const void* b) {
    const or_lsym* x = (const or_lsym*)a;
    const or_lsym* y = (const or_lsym*)b;
    if (x->len != y->len) return x->len < y->len ? -1 : 1;
    return x->sym < y->sym ? -1 : (x->sym > y->sym ? 1 : 0);
}

/* Canonical codes: symbols with a code, in ascending (length, symbol) order,
 * get consecutive code values; moving to a longer length appends zeros.
 * order_out (optional) receives the symbols in that order; returns count. */
uint32_t or_canonical_codes(const uint8_t* len, uint32_t nsym, uint32_t* code,
                            uint32_t* order_out) {
    uint32_t n = 0;
    for (uint32_t s = 0; s < nsym; s++) { code[s] = 0; n += len[s] > 0; }
    if (n == 0) return 0;
    or_lsym* v = (or_lsym*)malloc(n * sizeof(or_lsym));
    if (!v) return 0;
    uint32_t k = 0;
    for (uint32_t s = 0; s < nsym; s++)
        if (len[s]) { v[k].len = len[s]; v[k].sym = s; k++; }
    qsort(v, n, sizeof(or_lsym), lsym_cmp);
    uint64_t c = 0;
    for (uint32_t i = 0; i < n; i++) {
        if (i > 0) c = (c + 1) << (v[i].len - v[i - 1].len);
        code[v[i].sym] = (uint32_t)c;
        if (order_out) order_out[i] = v[i].sym;
    }
    free(v);
    return n;
}

/* ------------------------------------------------------------------------ */
/* byte format                                                               */
/* ------------------------------------------------------------------------ */
/*
 * header, 128 bytes, little-endian:
 *   0 u32 magic "FPS1"   4 u32 version   8 u32 ndim   12 u32 lorenzo dims
 *  16 u64 dims[3] (x fastest, unused = 1)
 *  40 f64 target PSNR   48 f64 eb_rel   56 f64 eb_abs   64 f64 vr
 *  72 f32 xmin  76 f32 xmax  80 f32 s  84 f32 inv  88 f32 thr  92 u32 flags
 *  96 u32 radius 100 u32 chunk 104 u32 lmax 108 u32 n_sym 112 u32 n_chunks
 * 116 u32 stream_words 120 u32 n_outlier 124 u32 n_verbatim
 * then, each section padded to a multiple of 16 bytes:
 *   codebook    n_sym u32 entries (len << 16 | sym), canonical order
 *   chunk table n_chunks u32 word offsets into the stream
 *   stream      stream_words u32 words; codes MSB-first; every chunk of
 *               `chunk` symbols starts on a fresh word
 *   outliers    n_outlier pairs (u32 idx, i32 delta), ascending idx
 *   verbatims   n_verbatim pairs (u32 idx, u32 float bits), ascending idx
 */

static uint64_t pad16(uint64_t b) { return (b + 15u) & ~(uint64_t)15u; }

static void put32(uint8_t* b, uint64_t off, uint32_t v) { memcpy(b + off, &v, 4); }
static void put64(uint8_t* b, uint64_t off, uint64_t v) { memcpy(b + off, &v, 8); }
static void putf64(uint8_t* b, uint64_t off, double v) { memcpy(b + off, &v, 8); }
static void putf32(uint8_t* b, uint64_t off, float v) { memcpy(b + off, &v, 4); }
static uint32_t get32(const uint8_t* b, uint64_t off) { uint32_t v; memcpy(&v, b + off, 4); return v; }
static uint64_t get64(const uint8_t* b, uint64_t off) { uint64_t v; memcpy(&v, b + off, 8); return v; }
static double getf64(const uint8_t* b, uint64_t off) { double v; memcpy(&v, b + off, 8); return v; }
static float getf32(const uint8_t* b, uint64_t off) { float v; memcpy(&v, b + off, 4); return v; }

typedef struct {
    double target_psnr, eb_rel, eb_abs, vr, psnr_model, sse, mse, psnr_actual;
    uint64_t bytes, n_outlier, n_verbatim, n_sym;
    float xmin, xmax, s, inv, thr;
    uint32_t flags;
    int32_t status;
    int32_t pad;
} or_stats;

void or_free(void* p) { free(p); }

static double psnr_from(double vr, double mse) {
    if (mse == 0.0) return INFINITY;
    return 20.0 * log10(vr) - 10.0 * log10(mse);
}

/* Compress a float32 field at a target PSNR.  dims are x fastest.  On success
 * *out receives a malloc'd blob of *out_bytes bytes (free with or_free). */
/* ------------------------------------------------------------------------ */
/* optional lossless layer (SZ step 3)                                       */
/* ------------------------------------------------------------------------ */
/* Container "FPZ1" around a finished blob:
 *   0  u32 magic 0x315A5046 ("FPZ1")    4  u32 version 1
 *   8  u64 raw blob bytes              16  u32 segment bytes (1024)
 *  20  u32 segments                    24  8 zero bytes
 *  32  u32 offsets[segments + 1]: start of every segment's data relative to
 *      the data section (bit 31: the segment is stored raw); the last entry
 *      is the data length; zero-padded to 16 bytes
 *      data section: every segment coded on its own, zero-padded to 16 bytes
 * A segment is coded byte by byte: a nonzero byte is copied; a run of k zero
 * bytes (k >= 1, as long as it lasts inside the segment) becomes 0x00 and
 * k - 1 in LEB128 (7 bits per byte, low first, bit 7 = more).  A segment whose
 * code is not shorter than the segment is stored raw.  The container is used
 * only when it is smaller than the blob; otherwise the blob stays as it is. */

#define OR_ZMAGIC 0x315A5046u
#define OR_ZSEG 1024u

static uint64_t zrle_code(const uint8_t* in, uint64_t len, uint8_t* out) {
    uint64_t o = 0, i = 0;
    while (i < len) {
        if (in[i] != 0) {
            if (out) out[o] = in[i];
            o++;
            i++;
            continue;
        }
        uint64_t k = 0;
        while (i + k < len && in[i + k] == 0) k++;
        if (out) out[o] = 0;
        o++;
        uint64_t v = k - 1;
        while (v >= 128) {
            if (out) out[o] = (uint8_t)((v & 127u) | 128u);
            o++;
            v >>= 7;
        }
        if (out) out[o] = (uint8_t)v;
        o++;
        i += k;
    }
    return o;
}

static uint64_t pad16o(uint64_t b) { return (b + 15u) & ~(uint64_t)15u; }

/* Wraps `raw` in the container when that is smaller; *out is malloc'd (free
 * with or_free) and holds either the container or a copy of raw. */
int or_zrle_wrap(const uint8_t* raw, uint64_t raw_bytes, uint8_t** out, uint64_t* out_bytes) {
    uint64_t nseg = (raw_bytes + OR_ZSEG - 1) / OR_ZSEG;
    uint64_t* off = (uint64_t*)malloc((nseg + 1) * sizeof(uint64_t));
    uint8_t* rawflag = (uint8_t*)malloc(nseg ? nseg : 1);
    if (!off || !rawflag) { free(off); free(rawflag); return OR_ENOMEM; }
    uint64_t data = 0;
    for (uint64_t sg = 0; sg < nseg; sg++) {
        uint64_t b = sg * OR_ZSEG, len = raw_bytes - b < OR_ZSEG ? raw_bytes - b : OR_ZSEG;
        uint64_t c = zrle_code(raw + b, len, NULL);
        rawflag[sg] = c >= len;
        off[sg] = data;
        data += rawflag[sg] ? len : c;
    }
    off[nseg] = data;
    uint64_t dstart = 32 + pad16o(4 * (nseg + 1));
    uint64_t total = dstart + pad16o(data);
    uint8_t* o;
    if (total >= raw_bytes) {
        o = (uint8_t*)malloc(raw_bytes ? raw_bytes : 1);
        if (!o) { free(off); free(rawflag); return OR_ENOMEM; }
        memcpy(o, raw, raw_bytes);
        *out = o;
        *out_bytes = raw_bytes;
        free(off);
        free(rawflag);
        return OR_OK;
    }
    o = (uint8_t*)calloc(total, 1);
    if (!o) { free(off); free(rawflag); return OR_ENOMEM; }
    put32(o, 0, OR_ZMAGIC);
    put32(o, 4, 1u);
    put64(o, 8, raw_bytes);
    put32(o, 16, OR_ZSEG);
    put32(o, 20, (uint32_t)nseg);
    for (uint64_t sg = 0; sg <= nseg; sg++)
        put32(o, 32 + 4 * sg, (uint32_t)off[sg] | ((sg < nseg && rawflag[sg]) ? 0x80000000u : 0u));
    for (uint64_t sg = 0; sg < nseg; sg++) {
        uint64_t b = sg * OR_ZSEG, len = raw_bytes - b < OR_ZSEG ? raw_bytes - b : OR_ZSEG;
        if (rawflag[sg]) memcpy(o + dstart + off[sg], raw + b, len);
        else zrle_code(raw + b, len, o + dstart + off[sg]);
    }
    free(off);
    free(rawflag);
    *out = o;
    *out_bytes = total;
    return OR_OK;
}

/* Inverse of or_zrle_wrap for a container (magic "FPZ1"); a buffer without
 * the magic is returned as a copy.  OR_ECORRUPT on any inconsistency. */
int or_zrle_unwrap(const uint8_t* c, uint64_t bytes, uint8_t** raw, uint64_t* raw_bytes) {
    *raw = NULL;
    *raw_bytes = 0;
    if (bytes < 4 || get32(c, 0) != OR_ZMAGIC) {
        uint8_t* o = (uint8_t*)malloc(bytes ? bytes : 1);
        if (!o) return OR_ENOMEM;
        memcpy(o, c, bytes);
        *raw = o;
        *raw_bytes = bytes;
        return OR_OK;
    }
    if (bytes < 32 || get32(c, 4) != 1u || get32(c, 16) != OR_ZSEG) return OR_ECORRUPT;
    uint64_t rb = get64(c, 8), nseg = get32(c, 20);
    if (nseg != (rb + OR_ZSEG - 1) / OR_ZSEG) return OR_ECORRUPT;
    uint64_t dstart = 32 + pad16o(4 * (nseg + 1));
    if (dstart > bytes) return OR_ECORRUPT;
    uint64_t dlen = get32(c, 32 + 4 * nseg) & 0x7FFFFFFFu;
    if (dstart + dlen > bytes) return OR_ECORRUPT;
    uint8_t* o = (uint8_t*)malloc(rb ? rb : 1);
    if (!o) return OR_ENOMEM;
    for (uint64_t sg = 0; sg < nseg; sg++) {
        uint32_t e0 = get32(c, 32 + 4 * sg), e1 = get32(c, 32 + 4 * (sg + 1));
        uint64_t a = e0 & 0x7FFFFFFFu, z = e1 & 0x7FFFFFFFu;
        uint64_t b = sg * OR_ZSEG, len = rb - b < OR_ZSEG ? rb - b : OR_ZSEG;
        if (a > z || z > dlen) { free(o); return OR_ECORRUPT; }
        const uint8_t* in = c + dstart + a;
        if (e0 & 0x80000000u) {
            if (z - a != len) { free(o); return OR_ECORRUPT; }
            memcpy(o + b, in, len);
            continue;
        }
        uint64_t i = 0, w = 0;
        while (i < z - a) {
            uint8_t v = in[i++];
            if (v != 0) {
                if (w >= len) { free(o); return OR_ECORRUPT; }
                o[b + w++] = v;
                continue;
            }
            uint64_t k = 0;
            int sh = 0;
            for (;;) {
                if (i >= z - a || sh > 28) { free(o); return OR_ECORRUPT; }
                uint8_t t = in[i++];
                k |= (uint64_t)(t & 127u) << sh;
                sh += 7;
                if (!(t & 128u)) break;
            }
            k += 1;
            if (w + k > len) { free(o); return OR_ECORRUPT; }
            memset(o + b + w, 0, k);
            w += k;
        }
        if (w != len) { free(o); return OR_ECORRUPT; }
    }
    *raw = o;
    *raw_bytes = rb;
    return OR_OK;
}

/* psnr_mode 0: eb from Eq. 8; 1: eb refined from the fine histogram (above)
 * when Eq. 8's quantization bin spans at least 16 fine bins. */
int or_compress_mode(const float* x, int ndim, const uint64_t* dims_in, int lorenzo_dims,
                     double target_psnr, int psnr_mode, int lossless, int radius, int chunk,
                     int lmax, uint8_t** out, uint64_t* out_bytes, or_stats* st) {
    or_stats dummy;
    if (!st) st = &dummy;
    memset(st, 0, sizeof(*st));
    *out = NULL;
    *out_bytes = 0;
    if (ndim < 1 || ndim > 3 || !(target_psnr > 0.0) || !(target_psnr <= 180.0) ||
        radius < 1 || radius > 32768 || chunk < 1 || lmax < 1 || lmax > 27 ||
        psnr_mode < 0 || psnr_mode > 1 || lossless < 0 || lossless > 1)
        return st->status = OR_EINVAL;
    int ld = lorenzo_dims ? lorenzo_dims : ndim;
    if (ld < 1 || ld > ndim) return st->status = OR_EINVAL;
    uint64_t dims[3] = {1, 1, 1};
    uint64_t n = 1;
    for (int i = 0; i < ndim; i++) { dims[i] = dims_in[i]; n *= dims[i]; }
    if (n > 0xFFFFFFFFull) return st->status = OR_EINVAL;
    uint32_t nsym = 2u * (uint32_t)radius;
    if (((uint64_t)1 << lmax) < nsym) return st->status = OR_EINVAL;

    float xmin = 0.0f, xmax = 0.0f;
    if (or_range(x, n, &xmin, &xmax) != OR_OK) return st->status = OR_ENONFINITE;
    or_scalars p;
    or_plan_scalars(or_eb_rel_from_psnr(target_psnr), xmin, xmax, n, &p);
    /* the fine histogram resolves the PDF inside a quantization bin only when
     * the bin spans at least 16 fine bins (2 eb >= 16 vr / K); narrower bins
     * are Eq. 6's setting and keep Eq. 8's eb.  A constant field, or one whose
     * lattice is off (x - xmin may overflow float), is left as it is. */
    if (psnr_mode == 1 && p.flags == 0 && p.eb_abs * (double)OR_FINE_BINS >= 8.0 * p.vr) {
        uint32_t* fh = (uint32_t*)malloc(OR_FINE_BINS * sizeof(uint32_t));
        if (!fh) return st->status = OR_ENOMEM;
        or_fine_hist(x, n, xmin, p.vr, fh);
        const double mse_rel = pow(10.0, -target_psnr / 10.0);
        const double eb = or_refine_eb(fh, n, p.vr, p.eb_abs, mse_rel);
        free(fh);
        p.flags = 0;
        p.eb_rel = eb / p.vr;
        scalars_for_eb(eb, &p);
    }

    uint16_t* codes = (uint16_t*)malloc((n ? n : 1) * sizeof(uint16_t));
    uint32_t* oi = (uint32_t*)malloc((n ? n : 1) * 4);
    int32_t* od = (int32_t*)malloc((n ? n : 1) * 4);
    uint32_t* vi = (uint32_t*)malloc((n ? n : 1) * 4);
    uint32_t* vb = (uint32_t*)malloc((n ? n : 1) * 4);
    uint32_t* hist = (uint32_t*)calloc(nsym, 4);
    uint8_t* len = (uint8_t*)calloc(nsym, 1);
    uint32_t* code = (uint32_t*)calloc(nsym, 4);
    uint32_t* order = (uint32_t*)calloc(nsym, 4);
    int rc = OR_OK;
    uint8_t* blob = NULL;
    if (!codes || !oi || !od || !vi || !vb || !hist || !len || !code || !order) { rc = OR_ENOMEM; goto done; }

    uint64_t no = 0, nv = 0, nchunks = 0, words = 0;
    uint32_t nused = 0;
    double sse = 0.0;
    uint32_t* chunk_off = NULL;
    if (!(p.flags & OR_FLAG_CONSTANT)) {
        rc = or_lattice(x, ndim, dims, ld, &p, radius, codes, oi, od, &no, vi, vb, &nv, &sse);
        if (rc) goto done;
        for (uint64_t i = 0; i < n; i++) hist[codes[i]]++;
        rc = or_huffman_lengths(hist, nsym, lmax, len);
        if (rc) goto done;
        nused = or_canonical_codes(len, nsym, code, order);
        nchunks = (n + (uint64_t)chunk - 1) / (uint64_t)chunk;
        chunk_off = (uint32_t*)malloc((nchunks ? nchunks : 1) * 4);
        if (!chunk_off) { rc = OR_ENOMEM; goto done; }
        for (uint64_t c = 0; c < nchunks; c++) {
            uint64_t bits = 0;
            uint64_t e = (c + 1) * (uint64_t)chunk;
            if (e > n) e = n;
            for (uint64_t i = c * (uint64_t)chunk; i < e; i++) bits += len[codes[i]];
            chunk_off[c] = (uint32_t)words;
            words += (bits + 31) / 32;
        }
    }
    uint64_t off_cb = OR_HEADER_BYTES;
    uint64_t off_ct = off_cb + pad16(4ull * nused);
    uint64_t off_st = off_ct + pad16(4ull * nchunks);
    uint64_t off_ou = off_st + pad16(4ull * words);
    uint64_t off_vb = off_ou + pad16(8ull * no);
    uint64_t total = off_vb + pad16(8ull * nv);
    blob = (uint8_t*)calloc(total, 1);
    if (!blob) { rc = OR_ENOMEM; goto done; }

    put32(blob, 0, OR_MAGIC);
    put32(blob, 4, OR_VERSION);
    put32(blob, 8, (uint32_t)ndim);
    put32(blob, 12, (uint32_t)ld);
    for (int i = 0; i < 3; i++) put64(blob, 16 + 8 * i, dims[i]);
    putf64(blob, 40, target_psnr);
    putf64(blob, 48, p.eb_rel);
    putf64(blob, 56, p.eb_abs);
    putf64(blob, 64, p.vr);
    putf32(blob, 72, p.xmin);
    putf32(blob, 76, p.xmax);
    putf32(blob, 80, p.s);
    putf32(blob, 84, p.inv);
    putf32(blob, 88, p.thr);
    put32(blob, 92, p.flags);
    put32(blob, 96, (uint32_t)radius);
    put32(blob, 100, (uint32_t)chunk);
    put32(blob, 104, (uint32_t)lmax);
    put32(blob, 108, nused);
    put32(blob, 112, (uint32_t)nchunks);
    put32(blob, 116, (uint32_t)words);
    put32(blob, 120, (uint32_t)no);
    put32(blob, 124, (uint32_t)nv);
    for (uint32_t i = 0; i < nused; i++) put32(blob, off_cb + 4ull * i, ((uint32_t)len[order[i]] << 16) | order[i]);
    for (uint64_t c = 0; c < nchunks; c++) put32(blob, off_ct + 4 * c, chunk_off[c]);
    /* MSB-first bit writer, restarted on a word boundary for every chunk */
    for (uint64_t c = 0; c < nchunks; c++) {
        uint64_t bitpos = (uint64_t)chunk_off[c] * 32;
        uint64_t e = (c + 1) * (uint64_t)chunk;
        if (e > n) e = n;
        for (uint64_t i = c * (uint64_t)chunk; i < e; i++) {
            uint32_t cw = code[codes[i]];
            int l = len[codes[i]];
            for (int b = l - 1; b >= 0; b--) {
                if ((cw >> b) & 1u) {
                    uint64_t wi = bitpos / 32;
                    uint32_t w = get32(blob, off_st + 4 * wi);
                    w |= 1u << (31 - (bitpos % 32));
                    put32(blob, off_st + 4 * wi, w);
                }
                bitpos++;
            }
        }
    }
    for (uint64_t i = 0; i < no; i++) { put32(blob, off_ou + 8 * i, oi[i]); put32(blob, off_ou + 8 * i + 4, (uint32_t)od[i]); }
    for (uint64_t i = 0; i < nv; i++) { put32(blob, off_vb + 8 * i, vi[i]); put32(blob, off_vb + 8 * i + 4, vb[i]); }

    st->target_psnr = target_psnr;
    st->eb_rel = p.eb_rel;
    st->eb_abs = p.eb_abs;
    st->vr = p.vr;
    st->psnr_model = (p.flags & OR_FLAG_CONSTANT) ? INFINITY : or_psnr_model(p.vr, p.eb_abs);
    st->sse = sse;
    st->mse = n ? sse / (double)n : 0.0;
    st->psnr_actual = psnr_from(p.vr, st->mse);
    st->bytes = total;
    st->n_outlier = no;
    st->n_verbatim = nv;
    st->n_sym = nused;
    st->xmin = p.xmin; st->xmax = p.xmax; st->s = p.s; st->inv = p.inv; st->thr = p.thr;
    st->flags = p.flags;
    if (lossless) {
        uint8_t* wrapped = NULL;
        uint64_t wb = 0;
        rc = or_zrle_wrap(blob, total, &wrapped, &wb);
        if (rc) goto done;
        free(blob);
        blob = wrapped;
        total = wb;
        st->bytes = wb;
    }
    *out = blob;
    *out_bytes = total;
    blob = NULL;
    free(chunk_off);
done:
    free(blob); free(codes); free(oi); free(od); free(vi); free(vb);
    free(hist); free(len); free(code); free(order);
    st->status = rc;
    return rc;
}

int or_compress(const float* x, int ndim, const uint64_t* dims_in, int lorenzo_dims,
                double target_psnr, int radius, int chunk, int lmax, uint8_t** out,
                uint64_t* out_bytes, or_stats* st) {
    return or_compress_mode(x, ndim, dims_in, lorenzo_dims, target_psnr, 0, 0, radius, chunk,
                            lmax, out, out_bytes, st);
}

/* Parse a blob's header (first 128 bytes): dims and counts.  Returns OR_OK or
 * OR_ECORRUPT. */
int or_blob_info(const uint8_t* blob, uint64_t bytes, uint64_t* dims, uint32_t* counts) {
    if (bytes < OR_HEADER_BYTES || get32(blob, 0) != OR_MAGIC || get32(blob, 4) != OR_VERSION)
        return OR_ECORRUPT;
    for (int i = 0; i < 3; i++) dims[i] = get64(blob, 16 + 8 * i);
    for (int i = 0; i < 5; i++) counts[i] = get32(blob, 108 + 4 * i);
    return OR_OK;
}

/* Decompress a blob into n floats.  Bit-serial canonical Huffman decoding,
 * outlier deltas put back, prefix sums, midpoint reconstruction, verbatim
 * values restored. */
static int decompress_raw(const uint8_t* blob, uint64_t bytes, float* out, uint64_t n_out);

/* A container (or_zrle_wrap) is unwrapped first. */
int or_decompress(const uint8_t* blob, uint64_t bytes, float* out, uint64_t n_out) {
    if (bytes >= 4 && get32(blob, 0) == OR_ZMAGIC) {
        uint8_t* raw = NULL;
        uint64_t rb = 0;
        int rc = or_zrle_unwrap(blob, bytes, &raw, &rb);
        if (rc == OR_OK) rc = decompress_raw(raw, rb, out, n_out);
        free(raw);
        return rc;
    }
    return decompress_raw(blob, bytes, out, n_out);
}

static int decompress_raw(const uint8_t* blob, uint64_t bytes, float* out, uint64_t n_out) {
    if (bytes < OR_HEADER_BYTES || get32(blob, 0) != OR_MAGIC || get32(blob, 4) != OR_VERSION)
        return OR_ECORRUPT;
    int ndim = (int)get32(blob, 8);
    int ld = (int)get32(blob, 12);
    if (ndim < 1 || ndim > 3 || ld < 1 || ld > ndim) return OR_ECORRUPT;
    uint64_t dims[3];
    uint64_t n = 1;
    for (int i = 0; i < 3; i++) { dims[i] = get64(blob, 16 + 8 * i); n *= dims[i]; }
    if (n != n_out || n > 0xFFFFFFFFull) return OR_ECORRUPT;
    or_scalars p;
    memset(&p, 0, sizeof(p));
    p.xmin = getf32(blob, 72);
    p.s = getf32(blob, 80);
    p.flags = get32(blob, 92);
    (void)getf64(blob, 64);
    uint32_t radius = get32(blob, 96), chunk = get32(blob, 100), lmax = get32(blob, 104);
    uint32_t nused = get32(blob, 108), nchunks = get32(blob, 112), words = get32(blob, 116);
    uint32_t no = get32(blob, 120), nv = get32(blob, 124);
    if (p.flags & OR_FLAG_CONSTANT) {
        for (uint64_t i = 0; i < n; i++) out[i] = p.xmin;
        return OR_OK;
    }
    if (radius < 1 || radius > 32768 || chunk < 1 || lmax < 1 || lmax > 27 || nused == 0 ||
        nused > 2 * radius || (uint64_t)nchunks != (n + chunk - 1) / chunk)
        return OR_ECORRUPT;
    uint64_t off_cb = OR_HEADER_BYTES;
    uint64_t off_ct = off_cb + pad16(4ull * nused);
    uint64_t off_st = off_ct + pad16(4ull * nchunks);
    uint64_t off_ou = off_st + pad16(4ull * words);
    uint64_t off_vb = off_ou + pad16(8ull * no);
    uint64_t total = off_vb + pad16(8ull * nv);
    if (total > bytes) return OR_ECORRUPT;

    /* canonical decoding tables */
    uint32_t count[33] = {0}, first_code[33] = {0}, first_index[33] = {0};
    uint32_t* syms = (uint32_t*)malloc(nused * 4);
    int64_t* v = (int64_t*)malloc((n ? n : 1) * sizeof(int64_t));
    if (!syms || !v) { free(syms); free(v); return OR_ENOMEM; }
    int rc = OR_OK;
    uint32_t prev_len = 0;
    for (uint32_t i = 0; i < nused; i++) {
        uint32_t e = get32(blob, off_cb + 4ull * i);
        uint32_t l = e >> 16, s = e & 0xFFFFu;
        if (l < 1 || l > lmax || s >= 2 * radius || l < prev_len) { rc = OR_ECORRUPT; goto done; }
        prev_len = l;
        syms[i] = s;
        count[l]++;
    }
    {
        uint32_t code = 0, idx = 0;
        for (uint32_t l = 1; l <= 32; l++) {
            code = (code + (l > 1 ? count[l - 1] : 0)) << (l > 1 ? 1 : 0);
            first_code[l] = code;
            first_index[l] = idx;
            idx += count[l];
        }
    }
    for (uint32_t c = 0; c < nchunks && rc == OR_OK; c++) {
        uint64_t w0 = get32(blob, off_ct + 4ull * c);
        uint64_t w1 = (c + 1 < nchunks) ? get32(blob, off_ct + 4ull * (c + 1)) : words;
        if (w0 > w1 || w1 > words) { rc = OR_ECORRUPT; break; }
        uint64_t bitpos = w0 * 32, bitend = w1 * 32;
        uint64_t e = (uint64_t)(c + 1) * chunk;
        if (e > n) e = n;
        for (uint64_t i = (uint64_t)c * chunk; i < e; i++) {
            uint32_t code = 0;
            int found = 0;
            for (uint32_t l = 1; l <= lmax; l++) {
                if (bitpos >= bitend) break;
                uint32_t w = get32(blob, off_st + 4 * (bitpos / 32));
                code = (code << 1) | ((w >> (31 - (bitpos % 32))) & 1u);
                bitpos++;
                if (code - first_code[l] < count[l]) {
                    uint32_t sym = syms[first_index[l] + (code - first_code[l])];
                    v[i] = sym ? (int64_t)sym - (int64_t)radius : 0;
                    found = 1;
                    break;
                }
            }
            if (!found) { rc = OR_ECORRUPT; break; }
        }
    }
    if (rc) goto done;
    for (uint32_t i = 0; i < no; i++) {
        uint32_t idx = get32(blob, off_ou + 8ull * i);
        if (idx >= n) { rc = OR_ECORRUPT; goto done; }
        v[idx] = (int32_t)get32(blob, off_ou + 8ull * i + 4);
    }
    {
        uint64_t nx, ny, nz;
        lorenzo_shape(ndim, dims, ld, &nx, &ny, &nz);
        or_inverse_lorenzo(v, ld, nx, ny, nz);
    }
    for (uint64_t i = 0; i < n; i++) out[i] = dequant((int32_t)v[i], &p);
    for (uint32_t i = 0; i < nv; i++) {
        uint32_t idx = get32(blob, off_vb + 8ull * i);
        uint32_t b = get32(blob, off_vb + 8ull * i + 4);
        if (idx >= n) { rc = OR_ECORRUPT; goto done; }
        memcpy(&out[idx], &b, 4);
    }
done:
    free(syms);
    free(v);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* distortion                                                                */
/* ------------------------------------------------------------------------ */

/* Eq. 4: sum of squared errors (sq_add). */
double or_sse(const float* x, const float* xr, uint64_t n) {
    sq_acc acc = {0.0, 0.0};
    for (uint64_t i = 0; i < n; i++) sq_add(&acc, x[i], xr[i]);
    return sq_total(&acc);
}

/* Eq. 4-5: MSE, vr from the original x, PSNR = 20 log10 vr - 10 log10 MSE. */
int or_psnr(const float* x, const float* xr, uint64_t n, double* psnr, double* mse, double* vr) {
    float lo, hi;
    if (n == 0) { *psnr = INFINITY; *mse = 0.0; *vr = 0.0; return OR_OK; }
    int rc = or_range(x, n, &lo, &hi);
    if (rc) return rc;
    *vr = (double)hi - (double)lo;
    *mse = or_sse(x, xr, n) / (double)n;
    *psnr = psnr_from(*vr, *mse);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* comparison path: classic sequential prediction from reconstructed values  */
/* ------------------------------------------------------------------------ */

/* Predict every point by the Lorenzo predictor over already-reconstructed
 * neighbours (in FP64), quantize the prediction error into bins of width
 * 2 eb (index = round(err / 2eb)), reconstruct at the bin midpoint, and keep
 * the value exactly (unpredictable) when the index leaves (-R, R) or the
 * reconstruction misses the bound.  Writes the reconstruction to xr. */
int or_classic_sz(const float* x, int ndim, const uint64_t* dims_in, int lorenzo_dims,
                  double target_psnr, int radius, float* xr, uint64_t* n_unpred,
                  double* psnr_actual) {
    int ld = lorenzo_dims ? lorenzo_dims : ndim;
    uint64_t dims[3] = {1, 1, 1};
    uint64_t n = 1;
    for (int i = 0; i < ndim; i++) { dims[i] = dims_in[i]; n *= dims[i]; }
    float lo, hi;
    if (or_range(x, n, &lo, &hi) != OR_OK) return OR_ENONFINITE;
    double vr = (double)hi - (double)lo;
    double eb = or_eb_rel_from_psnr(target_psnr) * vr;
    uint64_t nx, ny, nz;
    lorenzo_shape(ndim, dims, ld, &nx, &ny, &nz);
    uint64_t unp = 0;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t xi = i % nx, yi = (i / nx) % ny, zi = i / (nx * ny);
#define R(dz, dy, dx)                                                           \
    (((dz) > zi || (dy) > yi || (dx) > xi)                                      \
         ? 0.0                                                                  \
         : (double)xr[((zi - (dz)) * ny + (yi - (dy))) * nx + (xi - (dx))])
        double pred;
        if (ld == 1) pred = i > 0 ? (double)xr[i - 1] : 0.0;
        else if (ld == 2) pred = R(0, 0, 1) + R(0, 1, 0) - R(0, 1, 1);
        else pred = R(0, 0, 1) + R(0, 1, 0) + R(1, 0, 0) - R(0, 1, 1) - R(1, 0, 1) - R(1, 1, 0) + R(1, 1, 1);
#undef R
        int ok = 0;
        if (eb > 0.0) {
            double k = nearbyint(((double)x[i] - pred) / (2.0 * eb));
            if (fabs(k) < (double)radius) {
                float rec = (float)(pred + k * 2.0 * eb);
                if (fabs((double)x[i] - (double)rec) <= eb) { xr[i] = rec; ok = 1; }
            }
        }
        if (!ok) { xr[i] = x[i]; unp++; }
    }
    *n_unpred = unp;
    double mse = n ? or_sse(x, xr, n) / (double)n : 0.0;
    *psnr_actual = psnr_from(vr, mse);
    return OR_OK;
}
