// compress.cu -- the compression chain of the fixed-PSNR method on sm_103a.
//
//   k_range_plan   value range vr = max - min (Sec. IV, under Eq. 5) and the
//                  error bound eb_abs = eb_rel * vr (Sec. IV, after Eq. 7),
//                  bin width 2 eb (Sec. IV, before Eq. 7)
//   k_pq           prequantization onto the integer lattice + Lorenzo residual
//                  (Sec. II-A step 1, Sec. III) + uniform quantization into
//                  symbols (Sec. IV) + verbatim test + histogram + outlier
//                  staging + exact squared-error partials (Eq. 4)
//   k_rank_popc    order-preserving compaction ranks for outliers/verbatims
//   (k_codebook    Huffman code, huffman.cu)
//   k_enc_pack     warp-cooperative MSB-first bit packing of every chunk into
//                  its own scratch slot (SZ step 2, Sec. II-A)
//   k_enc_scan     chunk word offsets and section layout
//   k_enc_copy     chunk words placed in the stream, chunk table
//   k_emit         outliers and verbatims written in index order
//   k_finalize     header, size, statistics
#include <float.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace fp {

// ---------------------------------------------------------------------------
// value range and plan scalars
// ---------------------------------------------------------------------------

// Bin width s = (float)(2 eb), its inverse, the verbatim threshold (the float
// just below rd(eb)) and the lattice-off flag for absolute bound eb on a
// non-constant field of range vr.
__device__ void scalars_for_eb(double eb, double vr, float* s_out, float* inv_out, float* thr_out,
                               uint32_t* flags) {
    const double two_eb = __dmul_rn(2.0, eb);
    float s = __double2float_rn(two_eb);
    float inv = __double2float_rn(__ddiv_rn(1.0, two_eb));
    *flags = 0;
    if (!(s > 0.0f) || isinf(inv) || !(vr <= (double)FLT_MAX)) {
        *flags = kFlagLatticeOff;
        s = 0.0f;
        inv = 0.0f;
    }
    const float f = __double2float_rd(eb);
    const float t = f > 0.0f ? __int_as_float(__float_as_int(f) - 1) : 0.0f;
    *s_out = s;
    *inv_out = inv;
    *thr_out = t > 0.0f ? t : 0.0f;
}

struct RangeArgs {
    const float* x;
    uint64_t n;
    DevParams* par;
    float* part;
    uint32_t* hist;
    uint32_t nsym;
    double eb_rel, target;
    uint64_t cap;
    bool vec;  // x is 16-byte aligned
};

__global__ void __launch_bounds__(512) k_range_plan(const __grid_constant__ Batch<RangeArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const RangeArgs& A = B.a[fld];
    const uint32_t bid = blockIdx.x - B.off[fld], nblk = B.off[fld + 1] - B.off[fld];
    const float* __restrict__ x = A.x;
    const uint64_t n = A.n;
    DevParams* par = A.par;
    float* part = A.part;
    uint32_t* hist = A.hist;
    const uint32_t nsym = A.nsym;
    const bool VEC = A.vec;
    const uint32_t tid = threadIdx.x;
    const uint64_t gtid = (uint64_t)bid * blockDim.x + tid;
    const uint64_t gsz = (uint64_t)nblk * blockDim.x;
    for (uint64_t i = gtid; i < nsym; i += gsz) hist[i] = 0u;

    float lo = FLT_MAX, hi = -FLT_MAX;
    int nf = 0;
    if (VEC) {
        const float4* x4 = reinterpret_cast<const float4*>(x);
        const uint64_t n4 = n >> 2;
        // four independent 16-byte loads in flight per thread
        for (uint64_t i0 = gtid; i0 < n4; i0 += 4 * gsz) {
            float4 v[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint64_t i = i0 + k * gsz;
                v[k] = i < n4 ? __ldcs(x4 + i) : v[0];
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                nf |= !isfinite(v[k].x) | !isfinite(v[k].y) | !isfinite(v[k].z) | !isfinite(v[k].w);
                lo = fminf(lo, fminf(fminf(v[k].x, v[k].y), fminf(v[k].z, v[k].w)));
                hi = fmaxf(hi, fmaxf(fmaxf(v[k].x, v[k].y), fmaxf(v[k].z, v[k].w)));
            }
        }
        for (uint64_t i = (n4 << 2) + gtid; i < n; i += gsz) {
            float v = x[i];
            nf |= !isfinite(v);
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
    } else {
        for (uint64_t i = gtid; i < n; i += gsz) {
            float v = x[i];
            nf |= !isfinite(v);
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        nf |= __shfl_xor_sync(0xffffffffu, nf, o);
    }
    __shared__ float slo[16], shi[16];
    __shared__ int snf[16];
    __shared__ bool last;
    if ((tid & 31) == 0) { slo[tid >> 5] = lo; shi[tid >> 5] = hi; snf[tid >> 5] = nf; }
    __syncthreads();
    if (tid == 0) {
        for (uint32_t w = 1; w < (blockDim.x >> 5); w++) {
            lo = fminf(lo, slo[w]); hi = fmaxf(hi, shi[w]); nf |= snf[w];
        }
        part[3 * bid] = lo;
        part[3 * bid + 1] = hi;
        part[3 * bid + 2] = nf ? 1.0f : 0.0f;
        __threadfence();
        last = (atomicAdd(&par->done_range, 1u) == nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    lo = FLT_MAX; hi = -FLT_MAX; nf = 0;
    for (uint32_t b = tid; b < nblk; b += blockDim.x) {
        lo = fminf(lo, __ldcg(part + 3 * b));
        hi = fmaxf(hi, __ldcg(part + 3 * b + 1));
        nf |= __ldcg(part + 3 * b + 2) != 0.0f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        nf |= __shfl_xor_sync(0xffffffffu, nf, o);
    }
    __syncthreads();
    if ((tid & 31) == 0) { slo[tid >> 5] = lo; shi[tid >> 5] = hi; snf[tid >> 5] = nf; }
    __syncthreads();
    if (tid != 0) return;
    for (uint32_t w = 1; w < (blockDim.x >> 5); w++) {
        lo = fminf(lo, slo[w]); hi = fmaxf(hi, shi[w]); nf |= snf[w];
    }
    if (n == 0) { lo = 0.0f; hi = 0.0f; }
    double vr = (double)hi - (double)lo;
    uint32_t flags = 0;
    int status = 0;
    double eb = 0.0;
    float s = 0.0f, inv = 0.0f, thr = 0.0f;
    if (nf) {
        status = FPSNR_ENONFINITE;
        flags = kFlagError;
    } else if (n == 0 || vr == 0.0) {
        flags = kFlagConstant;
    } else {
        eb = __dmul_rn(A.eb_rel, vr);
        scalars_for_eb(eb, vr, &s, &inv, &thr, &flags);
    }
    par->kinv = vr > 0.0 ? __double2float_rn(__ddiv_rn((double)kFineBins, vr)) : 0.0f;
    par->vr = vr;
    par->eb_abs = eb;
    par->eb_rel = A.eb_rel;
    par->target_psnr = A.target;
    par->sse = 0.0;
    par->xmin = lo;
    par->xmax = hi;
    par->s = s;
    par->inv = inv;
    par->thr = thr;
    par->flags = flags;
    par->status = status;
    par->n_out = 0;
    par->n_vb = 0;
    par->n_sym = 0;
    par->stream_words = 0;
    par->cap = A.cap;
    par->off_cb = kHeaderBytes;
    par->off_ct = par->off_st = par->off_ou = par->off_vb = par->total = kHeaderBytes;
    par->done_range = 0;
    par->sym_lo = 0xffffffffu;
    par->sym_hi = 0u;
}

// ---------------------------------------------------------------------------
// optional error-bound refinement from the field's empirical PDF (Eq. 3)
// ---------------------------------------------------------------------------
//
// Eq. 8 takes the quantization error as uniform over every bin (Eq. 6).  With
// psnr_mode 1 the bound is refined on a kFineBins-bin histogram of the field:
// every fine bin contributes h (e^2 + w^2/12), e the lattice error of its
// centre, w its width, and a fixed bisection finds the largest eb whose
// predicted MSE meets the target.  Only when Eq. 8's bin spans at least 16
// fine bins.  Eq. 3 is scale invariant, so it is evaluated in units of the
// value range (w = 1/K, bin centres (j + 1/2)/K, lattice step 2 eb/vr, target
// 10^(-PSNR/10)): every float term is then a moderate number whatever the
// field's range.  Per-bin terms are computed in float with explicit
// round-to-nearest intrinsics; their weighted sum is exact and rounded once,
// so the result does not depend on how the sum is split among threads.

__device__ __forceinline__ bool refine_applies(const DevParams* par) {
    return par->flags == 0 && __dmul_rn(par->eb_abs, (double)kFineBins) >= __dmul_rn(8.0, par->vr);
}

struct FineArgs {
    const float* x;
    DevParams* par;
    uint32_t* fh;
    uint64_t n;
    bool vec;
};

// Fine histogram: bin = trunc((x - xmin) * kinv) in float, clamped to [0, K - 1].
__global__ void __launch_bounds__(512) k_fine_hist(const __grid_constant__ Batch<FineArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const FineArgs& A = B.a[fld];
    const uint32_t bid = blockIdx.x - B.off[fld], nblk = B.off[fld + 1] - B.off[fld];
    const DevParams* par = A.par;
    if (!refine_applies(par)) return;
    __shared__ uint32_t sh[kFineBins];
    for (uint32_t i = threadIdx.x; i < (uint32_t)kFineBins; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    const float xmin = par->xmin, kinv = par->kinv;
    auto bin = [&](float v) {
        const float u = __fmul_rn(__fsub_rn(v, xmin), kinv);
        const int b = __float2int_rz(u);
        atomicAdd(&sh[min(max(b, 0), kFineBins - 1)], 1u);
    };
    const uint64_t gtid = (uint64_t)bid * blockDim.x + threadIdx.x;
    const uint64_t gsz = (uint64_t)nblk * blockDim.x;
    const float* __restrict__ x = A.x;
    if (A.vec) {
        const float4* x4 = reinterpret_cast<const float4*>(x);
        const uint64_t n4 = A.n >> 2;
        for (uint64_t i = gtid; i < n4; i += gsz) {
            const float4 v = __ldcs(x4 + i);
            bin(v.x); bin(v.y); bin(v.z); bin(v.w);
        }
        for (uint64_t i = (n4 << 2) + gtid; i < A.n; i += gsz) bin(x[i]);
    } else {
        for (uint64_t i = gtid; i < A.n; i += gsz) bin(x[i]);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < (uint32_t)kFineBins; i += blockDim.x)
        if (sh[i]) atomicAdd(&A.fh[i], sh[i]);
}

struct RefineArgs {
    DevParams* par;
    uint32_t* fh;
    uint64_t n;
    double mse_rel;  // 10^(-target / 10), from the host
};

constexpr int kRefineThreads = 1024;
constexpr int kBisectSteps = 16;

// Unsigned 128-bit integer as two 64-bit halves.
struct U128 {
    uint64_t lo, hi;
};

__device__ __forceinline__ U128 u128_add(U128 a, U128 b) {
    U128 r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
    return r;
}

// p << s for p < 2^56 and 0 <= s < 72.
__device__ __forceinline__ U128 u128_shl(uint64_t p, uint32_t s) {
    U128 r;
    if (s == 0) {
        r.lo = p;
        r.hi = 0;
    } else if (s < 64) {
        r.lo = p << s;
        r.hi = p >> (64 - s);
    } else {
        r.lo = 0;
        r.hi = p << (s - 64);
    }
    return r;
}

// Nearest double (ties to even) to v * 2^e (v < 2^127, result within the
// normal range).
__device__ double u128_to_double_rn(U128 v, int e) {
    if (v.hi == 0 && v.lo < (1ull << 53)) return __dmul_rn((double)v.lo, ldexp(1.0, e));
    const int top = v.hi ? 127 - __clzll((long long)v.hi) : 63 - __clzll((long long)v.lo);
    const int sh = top - 52;  // >= 1: bits below sh are rounded off
    uint64_t mant;
    if (sh < 64) mant = (v.lo >> sh) | (sh ? (v.hi << (64 - sh)) : 0ull);
    else mant = v.hi >> (sh - 64);
    const int rb = sh - 1;  // round bit position
    const uint32_t round = (uint32_t)((rb < 64 ? (v.lo >> rb) : (v.hi >> (rb - 64))) & 1ull);
    bool sticky;
    if (rb == 0) sticky = false;
    else if (rb < 64) sticky = (v.lo & ((1ull << rb) - 1ull)) != 0ull;
    else if (rb == 64) sticky = v.lo != 0ull;
    else sticky = v.lo != 0ull || (v.hi & ((1ull << (rb - 64)) - 1ull)) != 0ull;
    if (round && (sticky || (mant & 1ull))) mant++;  // 2^53 is exact
    return __dmul_rn((double)mant, ldexp(1.0, sh + e));
}

// One block per field: the bisection of Eq. 3's predicted MSE, then the plan
// scalars for the refined bound.  Clears the fine histogram for the next call.
//
// The weighted sum of the terms is exact.  Every term is at least w212 =
// fl(w^2/12) (a float e^2 >= 0 plus w212, rounded), so all terms are integer
// multiples of u = 2^E0, the unit in the last place of w212.  A term is below
// (111 + 1/K)^2 (|e| <= max(c, step / 2) and the step 2 eb / vr <= 128 sqrt(3)),
// about 2^42 w212, so term / u < 2^66 and, with sum(h) = n < 2^32, the total
// is an integer below 2^98 in units of u: each thread adds its products as
// 128-bit integers, the block adds those, and the total is rounded to a
// double once.
__global__ void __launch_bounds__(kRefineThreads) k_eb_refine(const __grid_constant__ Batch<RefineArgs> B) {
    const RefineArgs& A = B.a[blockIdx.x];
    DevParams* par = A.par;
    if (!refine_applies(par)) return;
    static_assert(kFineBins == 4 * kRefineThreads, "4 fine bins per thread");
    __shared__ uint64_t part_lo[kRefineThreads / 32], part_hi[kRefineThreads / 32];
    __shared__ double s_pred;
    const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    uint32_t h[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        h[k] = A.fh[4 * t + k];
        A.fh[4 * t + k] = 0u;
    }
    const double vr = par->vr, eb0 = par->eb_abs;
    const double w = 1.0 / (double)kFineBins;
    const float w212 = __double2float_rn(__ddiv_rn(__dmul_rn(w, w), 12.0));
    // exponent field of w212 (a normal float): terms are multiples of 2^E0
    const int bw = (int)((__float_as_uint(w212) >> 23) & 0xffu);
    const int E0 = (bw > 0 ? bw : 1) - 150;
    float c[4];
#pragma unroll
    for (int k = 0; k < 4; k++) c[k] = __double2float_rn(__dmul_rn(__dadd_rn((double)(4 * t + k), 0.5), w));
    const double nd = (double)A.n;
    auto pred = [&](double eb) -> double {
        const float df = __double2float_rn(__dmul_rn(2.0, __ddiv_rn(eb, vr)));
        U128 acc = {0ull, 0ull};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float q = rintf(__fdiv_rn(c[k], df));
            const float e = __fsub_rn(c[k], __fmul_rn(q, df));
            const float term = __fadd_rn(__fmul_rn(e, e), w212);
            const uint32_t bits = __float_as_uint(term);
            const int bt = (int)((bits >> 23) & 0xffu);
            const uint64_t mant = (uint64_t)((bits & 0x7fffffu) | (bt ? 0x800000u : 0u));
            // term = mant 2^(max(bt, 1) - 150); the shift stays below 66 (see above)
            const int s = (bt > 0 ? bt : 1) - 150 - E0;
            const uint32_t sh = (uint32_t)min(max(s, 0), 71);
            acc = u128_add(acc, u128_shl((uint64_t)h[k] * mant, sh));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            U128 other;
            other.lo = __shfl_xor_sync(0xffffffffu, acc.lo, o);
            other.hi = __shfl_xor_sync(0xffffffffu, acc.hi, o);
            acc = u128_add(acc, other);
        }
        __syncthreads();  // the previous evaluation's result has been read
        if (lane == 0) {
            part_lo[warp] = acc.lo;
            part_hi[warp] = acc.hi;
        }
        __syncthreads();
        if (t == 0) {
            U128 tot = {0ull, 0ull};
            for (int i = 0; i < kRefineThreads / 32; i++) tot = u128_add(tot, U128{part_lo[i], part_hi[i]});
            s_pred = __ddiv_rn(u128_to_double_rn(tot, E0), nd);
        }
        __syncthreads();
        return s_pred;
    };
    const double target = A.mse_rel;
    double lo = __dmul_rn(eb0, 0.25), hi = __dmul_rn(eb0, 64.0), eb;
    if (pred(lo) > target) {
        eb = lo;
    } else if (pred(hi) <= target) {
        eb = hi;
    } else {
        for (int it = 0; it < kBisectSteps; it++) {
            const double mid = __dsqrt_rn(__dmul_rn(lo, hi));
            if (pred(mid) <= target) lo = mid;
            else hi = mid;
        }
        eb = lo;
    }
    if (t == 0) {
        float s, inv, thr;
        uint32_t flags;
        scalars_for_eb(eb, vr, &s, &inv, &thr, &flags);
        par->eb_abs = eb;
        par->eb_rel = __ddiv_rn(eb, vr);
        par->s = s;
        par->inv = inv;
        par->thr = thr;
        par->flags = flags;
    }
}

// ---------------------------------------------------------------------------
// fused prequantize + Lorenzo + quantize + verbatim test + histogram
// ---------------------------------------------------------------------------

struct PQArgs {
    const float* x;
    DevParams* par;
    uint16_t* codes;
    uint32_t* hist;
    uint2* stage_out;
    uint2* stage_vb;
    uint32_t* bm_out;
    uint32_t* bm_vb;
    double* sse_part;
    uint64_t n;
    uint32_t vx, vy, vz, zs;
    uint32_t nbx, nby;
    int radius;
};

constexpr int kHistWin = 4096;

__device__ __forceinline__ int32_t prequant(float x, float xmin, float inv, bool off) {
    return off ? 0 : __float2int_rn(__fmul_rn(__fsub_rn(x, xmin), inv));
}

// MODE 1: flat 1D predictor over a (rows x vx) traversal, left neighbour of a
//         row start is the previous row's last point, no upper-row term.
// MODE 2: 2D predictor on (vz rows) x vx, TY must be 1 (vy == 1).
// MODE 3: 3D predictor on vz x vy x vx with TY rows per tile, plus a halo
//         warp for the row above the tile.
// A warp covers SEG consecutive segments of 128 columns of a tile row, 4
// points per lane in each, so a thread handles 4 * SEG points of every row.
// Register budget: the two-segment kernel keeps all of its state (124
// registers, 4 blocks per SM: capping it spills inside the row loop); the
// one-segment kernels are held to 7 blocks of 128 threads per SM (2D) or
// 4 blocks of 256 (3D).
template <int MODE, int TX, int TY, bool VEC, int SEG>
__global__ void __launch_bounds__(TX / (4 * SEG) * (TY + (MODE == 3 ? 1 : 0)),
                                  SEG == 2 ? (MODE == 2 && VEC ? 5 : 1) : (MODE == 3 ? 3 : 896 / (TX / (4 * SEG) * TY)))
    k_pq(const __grid_constant__ Batch<PQArgs> B) {
    constexpr int TPR = TX / (4 * SEG);  // threads per tile row
    // MODE 3 adds a halo warp (threadIdx.y == 0) that only forms the row
    // differences of the row above the tile
    constexpr int NT = TPR * (TY + (MODE == 3 ? 1 : 0));
    constexpr int NP = 4 * SEG;          // points per thread per row
    static_assert(TPR % 32 == 0, "whole warps per tile row");
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const PQArgs& a = B.a[fld];
    const float* __restrict__ x = a.x;
    DevParams* par = a.par;
    const uint32_t flags = par->flags;
    if (flags & (kFlagConstant | kFlagError)) return;
    const float xmin = par->xmin, inv = par->inv, s = par->s, thr0 = par->thr;
    // The reconstruction test and the exact error sums run in units of 2^k,
    // k the exponent of the bound when it lies outside [2^-40, 2^40] (else 0):
    // a non-verbatim error is below the bound, so its square stays a normal
    // float for any range.  Scaling by a power of two is exact, so the test's
    // decisions are those of the unscaled arithmetic (|x| <= 2^24 vr keeps
    // every scaled value below 2^54); the block's sum is scaled back in FP64.
    int ke = 0;
    {
        const int bt = (int)((__float_as_uint(thr0) >> 23) & 0xffu);  // 0: subnormal
        if (thr0 > 0.0f && (bt < 127 - 40 || bt >= 127 + 40)) ke = min(max(bt - 127, -126), 126);
        // a nonzero xmin must stay a normal float once scaled (else the
        // reconstruction's rounding could differ from the unscaled one)
        const int bx = (int)((__float_as_uint(xmin) >> 23) & 0xffu);
        if (xmin != 0.0f && bx - ke < 1) ke = 0;
    }
    const float ssc = __uint_as_float((uint32_t)(127 - ke) << 23);  // 2^-k
    const float2 ssc2 = make_float2(ssc, ssc);
    // -x' 2^-k = fma(q, -s 2^-k, -xmin 2^-k) rounds to exactly the scaled, negated reconstruction
    const float ns = __fmul_rn(-s, ssc), nxmin = __fmul_rn(-xmin, ssc), thr = __fmul_rn(thr0, ssc);
    const float2 ns2 = make_float2(ns, ns), nxmin2s = make_float2(nxmin, nxmin);
    const float2 nxmin2 = make_float2(-xmin, -xmin), inv2 = make_float2(inv, inv);  // unscaled, for prequantization
    const bool off = (flags & kFlagLatticeOff) != 0;
    const int R = a.radius;

    // histogram window, then one spill slot per lane for points counted elsewhere
    __shared__ __align__(16) uint32_t shist[kHistWin + 32];
    __shared__ int32_t sL1[(MODE == 3) ? 2 : 1][(MODE == 3) ? TY + 1 : 1][(MODE == 3) ? TX : 1];
    __shared__ double ssum[NT / 32];

    const uint32_t tid = threadIdx.y * TPR + threadIdx.x;
    for (uint32_t i = tid; i < (kHistWin + 32) / 4; i += NT)
        reinterpret_cast<uint4*>(shist)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();

    const uint32_t b = blockIdx.x - B.off[fld];
    const uint32_t bx = b % a.nbx;
    const uint32_t by = (b / a.nbx) % a.nby;
    const uint32_t bz = b / (a.nbx * a.nby);
    const uint32_t x0 = bx * TX, y0 = by * TY, z0 = bz * a.zs;
    const uint32_t z1 = min(z0 + a.zs, a.vz);
    const uint32_t lane = tid & 31u;
    // column of the thread's first point within the tile; segment j adds 128 j
    const uint32_t cb = (threadIdx.x >> 5) * (128u * SEG) + 4u * lane;
    const uint32_t xb = x0 + cb;
    const uint32_t xw = xb - 4u * lane;  // the warp's first column
    // MODE 3: warp row threadIdx.y holds row y0 + threadIdx.y - 1 (row y0 - 1
    // for the halo warp, which exists only when y0 > 0)
    const uint32_t y = (MODE == 3) ? y0 + threadIdx.y - 1u : y0 + threadIdx.y;
    const uint32_t vx = a.vx;
    const bool yin = (MODE == 3) ? (threadIdx.y == 0 ? y0 > 0 : y < a.vy) : true;
    // histogram window [wlo, wlo + kHistWin) around the zero residual; the
    // unsigned difference code - wlo wraps for codes below the window
    const uint32_t wlo = (uint32_t)(R - kHistWin / 2);

    // A row of the tile: 4 * SEG points per thread and, for lane 0, the left
    // neighbour of its first point.  Rows are fetched one ahead of their use.
    struct Row {
        float v[NP];
        float l;
        bool hl;
    };
    auto row_limit = [&](uint64_t rowbase) -> uint32_t {
        // MODE 1 rows are consecutive runs of vx points; only the last is short
        return (MODE == 1) ? (uint32_t)min((uint64_t)vx, a.n - rowbase) : vx;
    };
    auto load_row = [&](const float* xrow, uint64_t rowbase, bool rowin, uint32_t lim, Row& r) {
#pragma unroll
        for (int j = 0; j < SEG; j++) {
            const uint32_t xj = xb + 128u * j;
            if (VEC && rowin && xj + 3 < lim) {
                const float4 v = __ldcs(reinterpret_cast<const float4*>(xrow + xj));
                r.v[4 * j] = v.x; r.v[4 * j + 1] = v.y; r.v[4 * j + 2] = v.z; r.v[4 * j + 3] = v.w;
            } else {
#pragma unroll
                for (int k = 0; k < 4; k++) r.v[4 * j + k] = (rowin && xj + k < lim) ? xrow[xj + k] : 0.0f;
            }
        }
        r.l = 0.0f;
        r.hl = false;
        if (lane == 0 && rowin) {
            if (xb > 0) {
                // a warp that starts past the row end needs nothing: its points are outside
                if (xb <= lim) {
                    r.l = xrow[xb - 1];
                    r.hl = true;
                }
            } else if (MODE == 1 && rowbase > 0) {
                r.l = x[rowbase - 1];
                r.hl = true;
            }
        }
    };
    auto fetch = [&](uint32_t z, Row& r) {
        const uint64_t rowbase = ((uint64_t)z * a.vy + (yin ? y : 0u)) * vx;
        load_row(x + rowbase, rowbase, yin, row_limit(rowbase), r);
    };
    // row differences of 4 * SEG lattice values whose left neighbour (of the
    // warp's first point) is ql0: segment j > 0 of lane 0 continues from lane
    // 31's segment j - 1
    auto row_diff = [&](const int32_t (&q)[NP], int32_t ql0, int32_t (&L1)[NP]) {
        int32_t ql = __shfl_up_sync(0xffffffffu, q[3], 1);
        if (lane == 0) ql = ql0;
        L1[0] = q[0] - ql;
#pragma unroll
        for (int k = 1; k < 4; k++) L1[k] = q[k] - q[k - 1];
#pragma unroll
        for (int j = 1; j < SEG; j++) {
            const int32_t send = lane == 31u ? q[4 * j - 1] : q[4 * j + 3];
            const int32_t qj = __shfl_sync(0xffffffffu, send, (lane + 31u) & 31u);
            L1[4 * j] = q[4 * j] - qj;
#pragma unroll
            for (int k = 1; k < 4; k++) L1[4 * j + k] = q[4 * j + k] - q[4 * j + k - 1];
        }
    };

    int32_t L2prev[NP];
#pragma unroll
    for (int i = 0; i < NP; i++) L2prev[i] = 0;
    FF2 acc = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
    uint32_t glo = 0xffffffffu, ghi = 0u;  // nonzero symbols counted outside the window
    int buf = 0;
    Row cur, nxt;

    // One row.  FULL: every point of the warp lies inside the row (a uniform
    // branch per warp), so no point needs a bounds flag.
    auto row = [&](uint32_t z, auto full_tag, auto scaled_tag) {
        constexpr bool FULL = decltype(full_tag)::value;
        constexpr bool SCALED = decltype(scaled_tag)::value;
        const uint64_t rowbase = ((uint64_t)z * a.vy + y) * vx;
        const uint32_t lim = row_limit(rowbase);
        bool in[NP];
        int32_t q[NP];
        // prequantization two points at a time: fl(fl(x - xmin) * inv) in each
        // lane (an add feeding a product: nothing to contract), then rounded
        // to the nearest integer
#pragma unroll
        for (int i = 0; i < NP; i += 2) {
            const float2 pv = __fmul2_rn(__fadd2_rn(make_float2(cur.v[i], cur.v[i + 1]), nxmin2), inv2);
#pragma unroll
            for (int k = 0; k < 2; k++) {
                in[i + k] = FULL || (yin && (xb + 128u * ((i + k) / 4) + ((i + k) % 4) < lim));
                q[i + k] = (in[i + k] && !off) ? __float2int_rn(k ? pv.y : pv.x) : 0;
            }
        }
        // Reconstruction, verbatim test and exact squared error, two points at a
        // time.  The two-segment kernels do this first, so that their 8 inputs
        // die before the residuals are formed (5 blocks per SM without spills;
        // the rare staging path reloads a verbatim point's bits); the others
        // after the histogram.  The halo warp and the warm-up plane above the
        // slab count nothing.
        constexpr bool EARLY = SEG == 2;
        uint32_t vbm = 0u;  // bit i: point i is stored verbatim
        auto recon = [&]() {
#pragma unroll
            for (int i = 0; i < NP; i += 2) {
                const float2 x2 = make_float2(cur.v[i], cur.v[i + 1]);
                const float2 xv = SCALED ? __fmul2_rn(x2, ssc2) : x2;
                const float2 nxr = __ffma2_rn(make_float2(__int2float_rn(q[i]), __int2float_rn(q[i + 1])), ns2,
                                              nxmin2s);
                const float2 df = __fadd2_rn(xv, nxr);  // fl(x - x') per point
                const bool v0 = in[i] && !(fabsf(df.x) <= thr);
                const bool v1 = in[i + 1] && !(fabsf(df.y) <= thr);
                ff2_add_sq_diff(acc, xv, nxr, df, in[i] && !v0, in[i + 1] && !v1);
                vbm |= (v0 ? 1u << i : 0u) | (v1 ? 2u << i : 0u);
            }
        };
        if constexpr (EARLY) {
            if (z >= z0 && (MODE != 3 || threadIdx.y != 0)) recon();
        }
        int32_t L1[NP];
        row_diff(q, cur.hl ? prequant(cur.l, xmin, inv, off) : 0, L1);

        int32_t L2[NP];
        if (MODE == 3) {
            // every warp row's differences along x (zero for a missing halo
            // row); the row above's come back after the barrier
#pragma unroll
            for (int i = 0; i < NP; i++) sL1[buf][threadIdx.y][cb + 128u * (i / 4) + (i % 4)] = L1[i];
            __syncthreads();
            if (threadIdx.y == 0) {  // the halo warp is done with this plane
                buf ^= 1;
                return;
            }
#pragma unroll
            for (int i = 0; i < NP; i++) L2[i] = L1[i] - sL1[buf][threadIdx.y - 1][cb + 128u * (i / 4) + (i % 4)];
            buf ^= 1;
        } else {
#pragma unroll
            for (int i = 0; i < NP; i++) L2[i] = L1[i];
        }

        if (z >= z0) {
            int32_t d[NP];
            uint32_t code[NP];
#pragma unroll
            for (int i = 0; i < NP; i++) {
                d[i] = (MODE == 1) ? L2[i] : L2[i] - L2prev[i];
                // |d| < R  <=>  d + R - 1 in [0, 2R - 2]
                const uint32_t u = (uint32_t)(d[i] + (R - 1));
                code[i] = u < (uint32_t)(2 * R - 1) ? u + 1u : 0u;
            }
            uint16_t* crow = a.codes + rowbase;
#pragma unroll
            for (int j = 0; j < SEG; j++) {
                const uint32_t xj = xb + 128u * j;
                if (VEC && in[4 * j + 3]) {
                    uint2 pk;
                    pk.x = code[4 * j] | (code[4 * j + 1] << 16);
                    pk.y = code[4 * j + 2] | (code[4 * j + 3] << 16);
                    *reinterpret_cast<uint2*>(crow + xj) = pk;
                } else {
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        if (in[4 * j + k]) crow[xj + k] = (uint16_t)code[4 * j + k];
                }
            }
            // histogram: every point adds to its window bin, or to the lane's
            // spill slot when it is outside the window (or outside the row);
            // codes outside the window then go to the global counters
            bool spill = false;
#pragma unroll
            for (int i = 0; i < NP; i++) {
                const uint32_t bin = code[i] - wlo;
                const bool win = in[i] && bin < (uint32_t)kHistWin;
                atomicAdd(&shist[win ? bin : kHistWin + lane], 1u);
                spill |= in[i] && !win;
            }
            if (__any_sync(0xffffffffu, spill)) {
#pragma unroll
                for (int i = 0; i < NP; i++) {
                    if (in[i] && code[i] - wlo >= (uint32_t)kHistWin) {
                        atomicAdd(&a.hist[code[i]], 1u);
                        if (code[i]) {
                            glo = min(glo, code[i]);
                            ghi = max(ghi, code[i]);
                        }
                    }
                }
            }
            if constexpr (!EARLY) recon();
            // outliers: a symbol 0
            bool ol[NP];
            bool rare = vbm != 0u;
#pragma unroll
            for (int i = 0; i < NP; i++) {
                ol[i] = in[i] && code[i] == 0u;
                rare |= ol[i];
            }
            // outliers and verbatims are rare: one vote per row decides whether any
            // lane of the warp needs the order-preserving staging below
            if (__any_sync(0xffffffffu, rare)) {
                // one slot reservation per list for the whole warp row: outlier
                // count in the low half, verbatim count in the high half
                uint32_t mine = 0;
#pragma unroll
                for (int i = 0; i < NP; i++) mine += (ol[i] ? 1u : 0u) + (((vbm >> i) & 1u) ? 0x10000u : 0u);
                uint32_t incl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= (uint32_t)o) incl += y;
                }
                const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
                uint32_t bo = 0, bv = 0;
                if (lane == 0) {
                    if (tot & 0xffffu) bo = atomicAdd(&par->n_out, tot & 0xffffu);
                    if (tot >> 16) bv = atomicAdd(&par->n_vb, tot >> 16);
                }
                const uint32_t ex = incl - mine;
                uint32_t so = __shfl_sync(0xffffffffu, bo, 0) + (ex & 0xffffu);
                uint32_t sv = __shfl_sync(0xffffffffu, bv, 0) + (ex >> 16);
#pragma unroll
                for (int i = 0; i < NP; i++) {
                    const uint32_t gi = (uint32_t)rowbase + xb + 128u * (i / 4) + (i % 4);
                    if (ol[i]) {
                        a.stage_out[so++] = make_uint2(gi, (uint32_t)d[i]);
                        atomicOr(&a.bm_out[gi >> 5], 1u << (gi & 31u));
                    }
                    if ((vbm >> i) & 1u) {
                        // the two-segment kernels reload the bits (rare)
                        a.stage_vb[sv++] = make_uint2(gi, __float_as_uint(EARLY ? x[gi] : cur.v[i]));
                        atomicOr(&a.bm_vb[gi >> 5], 1u << (gi & 31u));
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NP; i++) L2prev[i] = L2[i];
    };

    const uint32_t zstart = (MODE != 1 && z0 > 0) ? z0 - 1 : z0;
    // a warp whose first column is past the row end has no point in any row
    // (MODE 3 keeps every warp for the block barriers of its loop)
    const uint32_t zlast = (MODE != 3 && xw >= vx) ? zstart : z1;
    if (zstart < zlast) fetch(zstart, nxt);
    // one copy of the loop per scaling (uniform over the block)
    auto rows = [&](auto scaled_tag) {
        for (uint32_t z = zstart; z < zlast; z++) {
            cur = nxt;
            if (z + 1 < zlast) fetch(z + 1, nxt);
            // MODE 3: the halo warp of the first band has no row (yin false)
            if ((MODE != 3 || yin) && xw + 128u * SEG <= row_limit(((uint64_t)z * a.vy + y) * vx))
                row(z, std::true_type{}, scaled_tag);
            else
                row(z, std::false_type{}, scaled_tag);
        }
    };
    if (ke != 0) rows(std::true_type{});
    else rows(std::false_type{});

    // flush the histogram window (and take the block's symbol range from it)
    // and the squared-error partial
    __syncthreads();
    for (uint32_t i = tid; i < kHistWin / 4; i += NT) {
        const uint4 c4 = reinterpret_cast<const uint4*>(shist)[i];
        if ((c4.x | c4.y | c4.z | c4.w) == 0u) continue;
        const uint32_t cs[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (cs[k]) {
                const uint32_t sym = wlo + 4u * i + k;
                atomicAdd(&a.hist[sym], cs[k]);
                if (sym) {
                    glo = min(glo, sym);
                    ghi = max(ghi, sym);
                }
            }
        }
    }
    double tot = block_sum_double(ff2_to_double(acc), ssum);
    if (tid == 0) a.sse_part[b] = __dmul_rn(tot, __longlong_as_double((long long)(1023 + 2 * ke) << 52));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        glo = min(glo, __shfl_xor_sync(0xffffffffu, glo, o));
        ghi = max(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
    }
    if (lane == 0 && glo <= ghi) {
        atomicMin(&par->sym_lo, glo);
        atomicMax(&par->sym_hi, ghi);
    }
}

// ---------------------------------------------------------------------------
// order-preserving ranks: popcount prefix of the membership bitmaps
// ---------------------------------------------------------------------------

struct RankArgs {
    const DevParams* par;
    const uint32_t* bm;
    uint32_t* wpre;
    uint32_t* bpre;
    uint64_t nwords;
    uint32_t nbmblk;
};

// 2 * ceil(nbmblk / 4) blocks per field: list (outliers, verbatims) x four
// bitmap blocks of 1024 words, 4 consecutive words per thread; each bitmap
// block's words get their exclusive popcount prefix within that bitmap block,
// and the bitmap block its total.
__global__ void __launch_bounds__(1024) k_rank_popc(const __grid_constant__ Batch<RankArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const RankArgs& A = B.a[fld];
    const uint32_t bid = blockIdx.x - B.off[fld];
    const DevParams* par = A.par;
    const uint32_t* bm = A.bm;
    uint32_t* wpre = A.wpre;
    uint32_t* bpre = A.bpre;
    const uint64_t nwords = A.nwords;
    const uint32_t nbmblk = A.nbmblk;
    const uint32_t nb4 = (nbmblk + 3u) / 4u;
    const uint32_t list = bid / nb4;
    const uint32_t blk4 = bid % nb4;
    const uint32_t cnt = list == 0 ? par->n_out : par->n_vb;
    if (cnt == 0 || (par->flags & (kFlagConstant | kFlagError))) return;
    __shared__ uint32_t sh[33];
    __shared__ uint32_t sseg[4];
    const uint64_t w0 = (uint64_t)blk4 * 4096u + 4u * threadIdx.x;  // the thread's first word
    const uint32_t* b = bm + list * nwords;
    uint32_t v[4], c = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        v[k] = w0 + k < nwords ? b[w0 + k] : 0u;
        c += __popc(v[k]);
    }
    uint32_t total;
    const uint32_t ex = block_excl_scan(c, sh, &total);
    // bitmap block seg (256 threads) starts at thread 256 seg
    const uint32_t seg = threadIdx.x >> 8;
    if ((threadIdx.x & 255u) == 0u) sseg[seg] = ex;
    __syncthreads();
    // only words holding a set bit are ever looked up (k_emit): the others stay unwritten
    uint32_t e = ex - sseg[seg];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (w0 + k < nwords && v[k]) wpre[list * nwords + w0 + k] = e;
        e += __popc(v[k]);
    }
    if ((threadIdx.x & 255u) == 0u && blk4 * 4u + seg < nbmblk)
        bpre[list * nbmblk + blk4 * 4u + seg] = (seg < 3u ? sseg[seg + 1] : total) - sseg[seg];
}

// ---------------------------------------------------------------------------
// encoder: packing into per-chunk slots, offsets, placement
// ---------------------------------------------------------------------------

static __device__ __forceinline__ uint64_t pad16(uint64_t b) { return (b + 15u) & ~(uint64_t)15u; }

constexpr int kEncWarps = 8;                  // warps of an encoder block
constexpr int kEncCpw = kEncTile / kEncWarps;  // consecutive chunks each warp packs
static_assert(kEncTile <= 32 && kEncTile % kEncWarps == 0, "a tile's chunk prefix is one warp scan");
constexpr int kPieceWords = (256 * kMaxLmax + 31) / 32 + 2;

struct EncArgs {
    DevParams* par;
    const uint16_t* codes;
    const uint32_t* enc;
    uint8_t* out;
    uint64_t n;
    uint32_t chunk;
    uint64_t nchunks;
    uint32_t ntiles;
    uint32_t slot_words;    // scratch words per chunk: enough for chunk * lmax bits
    uint32_t* scratch;      // [nchunks * slot_words] every chunk packed from its slot's start
    uint32_t* chunk_words;  // [nchunks] words of every chunk
    uint32_t* tile_sum;     // [ntiles] words of every tile, then their exclusive prefix
};

// Encoder, three launches with no inter-block waiting:
//   k_enc_pack  one block per tile of kEncTile chunks, kEncCpw consecutive
//               chunks per warp: MSB-first packing into each chunk's own
//               scratch slot (chunks start on word boundaries, so a chunk's
//               words do not depend on where it lands): pieces of 256 symbols
//               (8 per lane, loaded one piece ahead) are OR-ed into a per-warp
//               shared-memory word buffer, full words go out coalesced and the
//               partial last word carries into the next piece.  The chunk's
//               word count and its tile's total are recorded.
//   k_enc_scan  one block per field: exclusive prefix of the tile totals, the
//               section layout and the capacity check
//   k_enc_copy  one block per tile: word offsets (tile prefix + in-tile
//               prefix), chunk table entries, and the words of each warp's
//               kEncCpw chunks copied from their slots into the stream by
//               that warp.  Every write is checked against the output
//               capacity.
// The codes are read and looked up once; the packed stream (a fraction of
// their bytes) is written twice and read once.
__global__ void __launch_bounds__(kEncWarps * 32) k_enc_pack(const __grid_constant__ Batch<EncArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const EncArgs& a = B.a[fld];
    const uint32_t t = blockIdx.x - B.off[fld];
    if (a.par->flags & (kFlagConstant | kFlagError)) return;
    __shared__ uint32_t sbuf[kEncWarps][kPieceWords];
    __shared__ uint32_t s_words[kEncWarps];
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    // the warp's chunks: kEncCpw consecutive ones of the tile
    const uint64_t cw0 = (uint64_t)t * kEncTile + (uint64_t)wib * kEncCpw;
    const uint64_t cw1 = min(cw0 + kEncCpw, a.nchunks);
    uint32_t* buf = sbuf[wib];
    uint32_t warp_words = 0;
    // the arguments the loops use, in registers (else reloaded from the
    // parameter space inside them)
    const uint32_t* __restrict__ enc = a.enc;
    const uint16_t* __restrict__ codes = a.codes;
    const uint64_t nn = a.n;
    const uint32_t chunk = a.chunk;
    // The codes of a piece are loaded one piece ahead (16 bytes a lane), so the
    // load of the next piece is in flight while this one is packed.
    auto chunk_end = [&](uint64_t c) { return min((c + 1) * chunk, nn); };
    uint4 nxt = make_uint4(0u, 0u, 0u, 0u);
    auto prefetch = [&](uint64_t c, uint64_t pb) {
        const uint64_t i = pb + 8u * lane;
        if (c < cw1 && i + 8 <= chunk_end(c)) nxt = *reinterpret_cast<const uint4*>(codes + i);
    };
    if (cw0 < cw1) prefetch(cw0, cw0 * a.chunk);
    for (uint64_t c = cw0; c < cw1; c++) {
        const uint64_t beg = c * a.chunk;
        const uint64_t end = chunk_end(c);
        uint32_t* dst = a.scratch + c * a.slot_words;
        uint32_t carry = 0;  // partial word (bits from previous pieces)
        uint32_t cbits = 0;  // valid bits in carry (< 32)
        uint32_t wpos = 0;   // words of the chunk written so far
        for (uint64_t pb = beg; pb < end; pb += 256u) {
            const uint4 v = nxt;
            // the next piece: further in this chunk, else the warp's next chunk
            if (pb + 256u < end) prefetch(c, pb + 256u);
            else prefetch(c + 1, (c + 1) * a.chunk);
            uint32_t cw[8], cl[8];
            uint32_t mybits = 0;
            const uint64_t i = pb + 8u * lane;
            if (i + 8 <= end) {
                const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const uint32_t e0 = __ldg(enc + (wv[k] & 0xffffu));
                    const uint32_t e1 = __ldg(enc + (wv[k] >> 16));
                    cw[2 * k] = e0 >> 5; cl[2 * k] = e0 & 31u;
                    cw[2 * k + 1] = e1 >> 5; cl[2 * k + 1] = e1 & 31u;
                }
            } else {
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const uint32_t e = (i + k < end) ? __ldg(enc + codes[i + k]) : 0u;
                    cw[k] = e >> 5; cl[k] = e & 31u;
                }
            }
#pragma unroll
            for (int k = 0; k < 8; k++) mybits += cl[k];
            uint32_t incl = mybits;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (uint32_t)o) incl += y;
            }
            const uint32_t piece_bits = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t nw = (cbits + piece_bits + 31u) >> 5;
            for (uint32_t k = lane; k < nw; k += 32) buf[k] = 0u;
            __syncwarp();
            if (lane == 0) buf[0] = carry;
            __syncwarp();
            // the lane's bits start at bit bp of buf
            const uint32_t bp = cbits + incl - mybits;  // bit position in buf
            if (__all_sync(0xffffffffu, mybits <= 64u)) {
                // every lane's codes fit 64 bits: concatenated in two registers by
                // funnel shifts, left-aligned, then OR-ed into the (at most three)
                // words they cover
                uint32_t ah = 0u, al = 0u;
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    ah = __funnelshift_l(al, ah, cl[k]);  // cl <= 27
                    al = (al << cl[k]) | cw[k];            // cw < 2^cl
                }
                if (mybits) {
                    uint32_t hi, lo;
                    if (mybits <= 32u) {
                        hi = al << (32u - mybits);
                        lo = 0u;
                    } else {
                        hi = __funnelshift_l(al, ah, 64u - mybits);
                        lo = al << (64u - mybits);
                    }
                    const uint32_t o = bp & 31u, w = bp >> 5;
                    const uint32_t nwd = (o + mybits + 31u) >> 5;  // words covered: 1..3
                    atomicOr(&buf[w], hi >> o);
                    if (nwd > 1u) atomicOr(&buf[w + 1], __funnelshift_r(lo, hi, o));
                    if (nwd > 2u) atomicOr(&buf[w + 2], lo << (32u - o));  // o > 0 here
                }
            } else if (mybits <= 128u) {
                // up to 128 bits: the same in four registers, left-aligned by a
                // word shift and a bit shift, then OR-ed into up to five words
                uint32_t a3 = 0u, a2 = 0u, a1 = 0u, a0 = 0u;
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const uint32_t l = cl[k];
                    a3 = __funnelshift_l(a2, a3, l);
                    a2 = __funnelshift_l(a1, a2, l);
                    a1 = __funnelshift_l(a0, a1, l);
                    a0 = (a0 << l) | cw[k];
                }
                if (mybits) {
                    const uint32_t sh = 128u - mybits, q = sh >> 5, r = sh & 31u;
                    const uint32_t b3 = q == 0u ? a3 : (q == 1u ? a2 : (q == 2u ? a1 : a0));
                    const uint32_t b2 = q == 0u ? a2 : (q == 1u ? a1 : (q == 2u ? a0 : 0u));
                    const uint32_t b1 = q == 0u ? a1 : (q == 1u ? a0 : 0u);
                    const uint32_t b0 = q == 0u ? a0 : 0u;
                    const uint32_t v3 = __funnelshift_l(b2, b3, r), v2 = __funnelshift_l(b1, b2, r);
                    const uint32_t v1 = __funnelshift_l(b0, b1, r), v0 = b0 << r;
                    const uint32_t o = bp & 31u, w = bp >> 5;
                    const uint32_t nwd = (o + mybits + 31u) >> 5;  // words covered: 1..5
                    atomicOr(&buf[w], v3 >> o);
                    if (nwd > 1u) atomicOr(&buf[w + 1], __funnelshift_r(v2, v3, o));
                    if (nwd > 2u) atomicOr(&buf[w + 2], __funnelshift_r(v1, v2, o));
                    if (nwd > 3u) atomicOr(&buf[w + 3], __funnelshift_r(v0, v1, o));
                    if (nwd > 4u) atomicOr(&buf[w + 4], v0 << (32u - o));  // o > 0 here
                }
            } else {
                // the codes are assembled in a 64-bit register (left-aligned,
                // after bp % 32 bits of the word that belong to earlier lanes)
                // and OR-ed in a word at a time
                uint32_t w = bp >> 5, nbit = bp & 31u;
                unsigned long long acc = 0ull;
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const uint32_t l = cl[k];
                    // cw == 0 when l == 0, so the masked shift is harmless then
                    acc |= (unsigned long long)cw[k] << ((64u - nbit - l) & 63u);
                    nbit += l;
                    if (nbit >= 32u) {
                        atomicOr(&buf[w], (uint32_t)(acc >> 32));
                        acc <<= 32;
                        nbit -= 32u;
                        w++;
                    }
                }
                if (nbit > (bp & 31u) || (nbit && w > (bp >> 5))) atomicOr(&buf[w], (uint32_t)(acc >> 32));
            }
            __syncwarp();
            const uint32_t tot = cbits + piece_bits;
            const uint32_t full = tot >> 5;
            for (uint32_t k = lane; k < full; k += 32) dst[wpos + k] = buf[k];
            carry = (tot & 31u) ? buf[full] : 0u;
            cbits = tot & 31u;
            wpos += full;
            __syncwarp();
        }
        if (cbits) {
            if (lane == 0) dst[wpos] = carry;
            wpos++;
        }
        if (lane == 0) a.chunk_words[c] = wpos;
        warp_words += wpos;
    }
    if (lane == 0) s_words[wib] = warp_words;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t sum = 0;
        for (int w = 0; w < kEncWarps; w++) sum += s_words[w];
        a.tile_sum[t] = sum;
    }
}

__global__ void __launch_bounds__(1024) k_enc_scan(const __grid_constant__ Batch<EncArgs> B) {
    const EncArgs& a = B.a[blockIdx.x];  // one block per field
    DevParams* par = a.par;
    if (par->flags & (kFlagConstant | kFlagError)) return;
    __shared__ uint32_t sh[33];
    constexpr int IPT = 4;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < a.ntiles; base += 1024u * IPT) {
        const uint32_t i0 = base + threadIdx.x * IPT;
        uint32_t v[IPT], sum = 0;
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            v[k] = (i0 + k < a.ntiles) ? a.tile_sum[i0 + k] : 0u;
            sum += v[k];
        }
        uint32_t total;
        uint32_t ex = block_excl_scan(sum, sh, &total) + carry;
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            if (i0 + k < a.ntiles) a.tile_sum[i0 + k] = ex;
            ex += v[k];
        }
        carry += total;
    }
    if (threadIdx.x == 0) {
        const uint64_t off_st = par->off_ct + pad16(4ull * a.nchunks);
        const uint64_t off_ou = off_st + pad16(4ull * carry);
        const uint64_t off_vb = off_ou + pad16(8ull * par->n_out);
        const uint64_t total = off_vb + pad16(8ull * par->n_vb);
        par->stream_words = carry;
        par->off_st = off_st;
        par->off_ou = off_ou;
        par->off_vb = off_vb;
        par->total = total;
        if (total > par->cap) set_error(par, FPSNR_ECAPACITY);
    }
}

// One block per tile: the word offsets of the tile's chunks (tile prefix plus
// the prefix of their word counts, in shared memory), the chunk table, then
// the words of every warp's kEncCpw chunks copied by that warp (the words of a
// tile are contiguous in the stream).
__global__ void __launch_bounds__(kEncWarps * 32) k_enc_copy(const __grid_constant__ Batch<EncArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const EncArgs& a = B.a[fld];
    const uint32_t t = blockIdx.x - B.off[fld];
    DevParams* par = a.par;
    if (par->flags & (kFlagConstant | kFlagError)) return;  // uniform over the block
    __shared__ uint32_t pre[kEncTile + 1];
    const uint64_t c0 = (uint64_t)t * kEncTile;
    const uint32_t nch = (uint32_t)min((uint64_t)kEncTile, a.nchunks - c0);
    const uint64_t cap = par->cap;
    const uint64_t off_ct = par->off_ct;
    const uint64_t off_st = par->off_st;
    const uint32_t tile_off = a.tile_sum[t];  // words of all earlier tiles
    if (threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x;
        const uint32_t w = lane < nch ? a.chunk_words[c0 + lane] : 0u;
        uint32_t incl = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (lane < (uint32_t)kEncTile) pre[lane] = incl - w;  // pre[nch..] = the tile's total
        if (lane == 31) pre[kEncTile] = incl;
        if (lane < nch && off_ct + 4ull * (c0 + lane + 1) <= cap)
            reinterpret_cast<uint32_t*>(a.out + off_ct)[c0 + lane] = tile_off + incl - w;
    }
    __syncthreads();
    const uint32_t total = pre[nch];
    uint32_t* stream = reinterpret_cast<uint32_t*>(a.out + off_st) + tile_off;
    // words that fit the output (the layout already flagged a short buffer)
    const uint64_t room = off_st + 4ull * tile_off <= cap ? (cap - off_st - 4ull * tile_off) / 4ull : 0ull;
    const uint32_t lim = (uint32_t)min((uint64_t)total, room);
    // each warp copies the words of the kEncCpw chunks its pack warp packed
    // (contiguous in the stream)
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t k0 = min((threadIdx.x >> 5) * (uint32_t)kEncCpw, nch);
    const uint32_t k1 = min(k0 + (uint32_t)kEncCpw, nch);
    const uint32_t wend = min(pre[k1], lim);
    for (uint32_t w = pre[k0] + lane; w < wend; w += 32) {
        uint32_t k = k0;  // the chunk holding word w: the last k with pre[k] <= w
#pragma unroll
        for (int i = 1; i < kEncCpw; i++) k += (k0 + i < k1 && pre[k0 + i] <= w) ? 1u : 0u;
        stream[w] = __ldcs(a.scratch + (c0 + k) * a.slot_words + (w - pre[k]));
    }
}

// Outliers and verbatims in ascending index: rank = number of set bitmap bits
// before the index.
struct EmitArgs {
    const DevParams* par;
    const uint2* stage_out;
    const uint2* stage_vb;
    const uint32_t* bm;
    const uint32_t* wpre;
    const uint32_t* bpre;
    uint8_t* out;
    uint64_t nwords;
    uint32_t nbmblk;
    uint32_t G;  // blocks per list
};

__global__ void __launch_bounds__(256) k_emit(const __grid_constant__ Batch<EmitArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const EmitArgs& A = B.a[fld];
    const uint32_t bid = blockIdx.x - B.off[fld];
    const DevParams* par = A.par;
    const uint2* stage_out = A.stage_out;
    const uint2* stage_vb = A.stage_vb;
    const uint32_t* bm = A.bm;
    const uint32_t* wpre = A.wpre;
    const uint32_t* bpre = A.bpre;
    uint8_t* out = A.out;
    const uint64_t nwords = A.nwords;
    const uint32_t nbmblk = A.nbmblk;
    if (par->flags & (kFlagConstant | kFlagError)) return;
    const uint32_t list = bid / A.G;
    const uint32_t lb = bid % A.G;
    const uint32_t cnt = list == 0 ? par->n_out : par->n_vb;
    const uint2* stage = list == 0 ? stage_out : stage_vb;
    uint2* dst = reinterpret_cast<uint2*>(out + (list == 0 ? par->off_ou : par->off_vb));
    const uint32_t* b = bm + list * nwords;
    const uint32_t* wp = wpre + list * nwords;
    const uint32_t* bp = bpre + list * nbmblk;
    for (uint32_t i = lb * blockDim.x + threadIdx.x; i < cnt; i += A.G * blockDim.x) {
        uint2 e = stage[i];
        const uint32_t idx = e.x, w = idx >> 5;
        const uint32_t r = bp[w >> 10] + wp[w] + __popc(b[w] & ((1u << (idx & 31u)) - 1u));
        dst[r] = e;
    }
}

struct FinArgs {
    DevParams* par;
    uint32_t* bm;
    const uint2* stage_out;
    const uint2* stage_vb;
    uint8_t* out;
    uint64_t* out_bytes;
    fpsnr_stats* stats;
    int ndim, ld;
    uint64_t d0, d1, d2, n;
    int radius, chunk, lmax;
    uint64_t nchunks, nwords;
    uint32_t G;  // blocks per field
};

__global__ void __launch_bounds__(256) k_finalize(const __grid_constant__ Batch<FinArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const FinArgs& A = B.a[fld];
    const uint32_t bid = blockIdx.x - B.off[fld];
    DevParams* par = A.par;
    uint32_t* bm = A.bm;
    const uint2* stage_out = A.stage_out;
    const uint2* stage_vb = A.stage_vb;
    uint8_t* out = A.out;
    uint64_t* out_bytes = A.out_bytes;
    fpsnr_stats* stats = A.stats;
    const int ndim = A.ndim, ld = A.ld;
    const uint64_t d0 = A.d0, d1 = A.d1, d2 = A.d2, n = A.n;
    const int radius = A.radius, chunk = A.chunk, lmax = A.lmax;
    const uint64_t nchunks = A.nchunks, nwords = A.nwords;
    // clear the membership bitmaps (only the words that were set)
    const uint32_t no = par->n_out, nv = par->n_vb;
    for (uint32_t i = bid * blockDim.x + threadIdx.x; i < no; i += A.G * blockDim.x)
        bm[stage_out[i].x >> 5] = 0u;
    for (uint32_t i = bid * blockDim.x + threadIdx.x; i < nv; i += A.G * blockDim.x)
        bm[nwords + (stage_vb[i].x >> 5)] = 0u;
    if (bid != 0 || threadIdx.x != 0) return;

    uint32_t flags = par->flags;
    if ((flags & kFlagConstant) && !(flags & kFlagError) && par->cap < kHeaderBytes) {
        par->status = FPSNR_ECAPACITY;  // even the header does not fit
        flags |= kFlagError;
        par->flags = flags;
    }
    const bool err = (flags & kFlagError) != 0;
    const bool cst = (flags & kFlagConstant) != 0;
    const uint64_t total = err ? 0 : par->total;
    if (!err) {
        uint8_t* h = out;
        auto put32 = [&](int o, uint32_t v) { *reinterpret_cast<uint32_t*>(h + o) = v; };
        auto put64 = [&](int o, uint64_t v) { *reinterpret_cast<uint64_t*>(h + o) = v; };
        auto putd = [&](int o, double v) { *reinterpret_cast<double*>(h + o) = v; };
        auto putf = [&](int o, float v) { *reinterpret_cast<float*>(h + o) = v; };
        put32(0, kMagic);
        put32(4, kVersion);
        put32(8, (uint32_t)ndim);
        put32(12, (uint32_t)ld);
        put64(16, d0);
        put64(24, d1);
        put64(32, d2);
        putd(40, par->target_psnr);
        putd(48, par->eb_rel);
        putd(56, par->eb_abs);
        putd(64, par->vr);
        putf(72, par->xmin);
        putf(76, par->xmax);
        putf(80, par->s);
        putf(84, par->inv);
        putf(88, par->thr);
        put32(92, flags & ~kFlagError);
        put32(96, (uint32_t)radius);
        put32(100, (uint32_t)chunk);
        put32(104, (uint32_t)lmax);
        put32(108, cst ? 0u : par->n_sym);
        put32(112, cst ? 0u : (uint32_t)nchunks);
        put32(116, cst ? 0u : par->stream_words);
        put32(120, cst ? 0u : par->n_out);
        put32(124, cst ? 0u : par->n_vb);
        if (!cst) {
            // zero the padding that rounds every section up to 16 bytes
            auto zero = [&](uint64_t from, uint64_t to) {
                for (uint64_t o = from; o < to; o += 4) *reinterpret_cast<uint32_t*>(h + o) = 0u;
            };
            zero(kHeaderBytes + 4ull * par->n_sym, par->off_ct);
            zero(par->off_ct + 4ull * nchunks, par->off_st);
            zero(par->off_st + 4ull * par->stream_words, par->off_ou);
            zero(par->off_ou + 8ull * par->n_out, par->off_vb);
            zero(par->off_vb + 8ull * par->n_vb, par->total);
        }
    }
    if (out_bytes) *out_bytes = total;
    if (stats) {
        fpsnr_stats s;
        s.target_psnr = par->target_psnr;
        s.eb_rel = par->eb_rel;
        s.eb_abs = par->eb_abs;
        s.vr = par->vr;
        s.psnr_model = cst ? __longlong_as_double(0x7ff0000000000000ll)
                           : 20.0 * log10(par->vr / par->eb_abs) + 10.0 * log10(3.0);
        s.sse = par->sse;
        s.mse = n ? par->sse / (double)n : 0.0;
        s.psnr_actual = (s.mse == 0.0) ? __longlong_as_double(0x7ff0000000000000ll)
                                       : 20.0 * log10(par->vr) - 10.0 * log10(s.mse);
        s.bytes = total;
        s.n_outlier = cst ? 0 : par->n_out;
        s.n_verbatim = cst ? 0 : par->n_vb;
        s.n_sym = cst ? 0 : par->n_sym;
        s.xmin = par->xmin;
        s.xmax = par->xmax;
        s.flags = flags & ~kFlagError;
        s.status = par->status;
        *stats = s;
    }
}

// ---------------------------------------------------------------------------
// host launcher
// ---------------------------------------------------------------------------

#define FP_LAUNCH_CHECK()                                          \
    do {                                                           \
        if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA; \
    } while (0)

// Launches one k_pq variant over the fields of a batch that use it.
template <int MODE, int TX, int TY, int SEG>
static void launch_pq_t(Batch<PQArgs>& b, uint32_t blocks, bool vec, cudaStream_t st) {
    const dim3 blk(TX / (4 * SEG), TY + (MODE == 3 ? 1 : 0));  // MODE 3: plus the halo warp
    if (vec) k_pq<MODE, TX, TY, true, SEG><<<blocks, blk, 0, st>>>(b);
    else k_pq<MODE, TX, TY, false, SEG><<<blocks, blk, 0, st>>>(b);
}

static void launch_pq_variant(int mode, int tx, Batch<PQArgs>& b, uint32_t blocks, bool vec,
                              cudaStream_t st) {
    if (mode == 1) launch_pq_t<1, 1024, 1, 2>(b, blocks, vec, st);
    else if (mode == 3) launch_pq_t<3, 128, 8, 1>(b, blocks, vec, st);
    else if (tx == 128) launch_pq_t<2, 128, 1, 1>(b, blocks, vec, st);
    else if (tx == 256) launch_pq_t<2, 256, 1, 1>(b, blocks, vec, st);
    else if (tx == 512) launch_pq_t<2, 512, 1, 1>(b, blocks, vec, st);
    else launch_pq_t<2, 1024, 1, 2>(b, blocks, vec, st);
}

// Small grid-stride kernels (emit, finalize) use this many blocks per field:
// about four per SM over the batch (the outlier / verbatim lists can hold a
// tenth of the points at 120 dB).
static uint32_t small_blocks(const fpsnr_plan_s* p, int count) {
    const uint32_t g = (uint32_t)std::max(1, 4 * p->sm_count / std::max(1, count));
    return std::min<uint32_t>(g, 256);
}

int launch_compress_batch(fpsnr_plan_s* const* P, const float* const* d_in, void* const* d_out,
                          const uint64_t* caps, uint64_t* d_out_bytes, fpsnr_stats* d_stats,
                          int count, cudaStream_t st) {
    if (count <= 0) return FPSNR_OK;
    if (count > kMaxBatch) {
        for (int b0 = 0; b0 < count; b0 += kMaxBatch) {
            const int c = std::min(kMaxBatch, count - b0);
            int rc = launch_compress_batch(P + b0, d_in + b0, d_out + b0, caps + b0,
                                           d_out_bytes ? d_out_bytes + b0 : nullptr,
                                           d_stats ? d_stats + b0 : nullptr, c, st);
            if (rc) return rc;
        }
        return FPSNR_OK;
    }
    fp::Profiler& prof = P[0]->prof;  // batched launches are attributed to the first plan
    uint32_t blocks[kMaxBatch];

    // ---- range + plan scalars ----
    {
        Batch<RangeArgs> b;
        b.count = (uint32_t)count;
        for (int f = 0; f < count; f++) {
            const fpsnr_plan_s* p = P[f];
            const Workspace& w = p->w;
            b.a[f] = RangeArgs{d_in[f], p->n, w.par, w.range_part, w.hist, p->nsym, p->eb_rel,
                               p->target_psnr, caps[f],
                               ((uintptr_t)d_in[f] & 15u) == 0};
            blocks[f] = p->n_range_blocks;
        }
        const uint32_t tot = batch_offsets(b, blocks);
        StageScope sc(prof, kStRange, st);
        k_range_plan<<<tot, 512, 0, st>>>(b);
    }
    FP_LAUNCH_CHECK();

    // ---- optional bound refinement (psnr_mode 1) ----
    {
        Batch<FineArgs> bf;
        Batch<RefineArgs> br;
        bf.count = br.count = 0;
        uint32_t fblocks[kMaxBatch], rblocks[kMaxBatch];
        for (int f = 0; f < count; f++) {
            const fpsnr_plan_s* p = P[f];
            if (p->psnr_mode != 1 || p->n == 0) continue;
            fblocks[bf.count] = p->n_range_blocks;
            rblocks[br.count] = 1;
            bf.a[bf.count++] = FineArgs{d_in[f], p->w.par, p->w.fine_hist, p->n,
                                        ((uintptr_t)d_in[f] & 15u) == 0};
            br.a[br.count++] = RefineArgs{p->w.par, p->w.fine_hist, p->n, p->mse_rel};
        }
        if (bf.count) {
            const uint32_t tf = batch_offsets(bf, fblocks);
            const uint32_t tr = batch_offsets(br, rblocks);
            StageScope sc(prof, kStRefine, st);
            k_fine_hist<<<tf, 512, 0, st>>>(bf);
            k_eb_refine<<<tr, kRefineThreads, 0, st>>>(br);
            sc.more(1);
        }
    }
    FP_LAUNCH_CHECK();

    // ---- predictor: one launch per kernel variant present in the batch ----
    {
        Batch<PQArgs> b;
        bool done[kMaxBatch] = {};
        for (int f0 = 0; f0 < count; f0++) {
            if (done[f0] || P[f0]->n == 0) continue;
            const PQGeom& g0 = P[f0]->pq;
            const bool vec0 = g0.vec && ((uintptr_t)d_in[f0] & 15u) == 0;
            b.count = 0;
            for (int f = f0; f < count; f++) {
                const fpsnr_plan_s* p = P[f];
                const PQGeom& g = p->pq;
                const bool vec = g.vec && ((uintptr_t)d_in[f] & 15u) == 0;
                if (done[f] || p->n == 0 || g.mode != g0.mode || g.tx != g0.tx || vec != vec0) continue;
                done[f] = true;
                const Workspace& w = p->w;
                PQArgs a;
                a.x = d_in[f];
                a.par = w.par;
                a.codes = w.codes;
                a.hist = w.hist;
                a.stage_out = w.stage_out;
                a.stage_vb = w.stage_vb;
                a.bm_out = w.bm;
                a.bm_vb = w.bm + p->nwords;
                a.sse_part = w.sse_part;
                a.n = p->n;
                a.vx = g.vx;
                a.vy = g.vy;
                a.vz = g.vz;
                a.zs = (uint32_t)g.zs;
                a.nbx = g.nbx;
                a.nby = g.nby;
                a.radius = p->radius;
                blocks[b.count] = g.nblocks;
                b.a[b.count++] = a;
            }
            const uint32_t tot = batch_offsets(b, blocks);
            StageScope sc(prof, kStPq, st);
            launch_pq_variant(g0.mode, g0.tx, b, tot, vec0, st);
            FP_LAUNCH_CHECK();
        }
    }

    // ---- order-preserving ranks of outliers / verbatims ----
    {
        Batch<RankArgs> b;
        b.count = (uint32_t)count;
        for (int f = 0; f < count; f++) {
            const fpsnr_plan_s* p = P[f];
            const Workspace& w = p->w;
            b.a[f] = RankArgs{w.par, w.bm, w.wpre, w.bpre, p->nwords, (uint32_t)p->nbmblk};
            blocks[f] = p->n ? 2u * (((uint32_t)p->nbmblk + 3u) / 4u) : 0u;
        }
        const uint32_t tot = batch_offsets(b, blocks);
        if (tot) {
            StageScope sc(prof, kStRank, st);
            k_rank_popc<<<tot, 1024, 0, st>>>(b);
            FP_LAUNCH_CHECK();
        }
    }

    // ---- codebook ----
    int rc = launch_codebook_batch(P, d_out, count, st);
    if (rc) return rc;

    // ---- encoder: chunk words, tile prefix, packing ----
    {
        Batch<EncArgs> b;
        b.count = (uint32_t)count;
        for (int f = 0; f < count; f++) {
            const fpsnr_plan_s* p = P[f];
            const Workspace& w = p->w;
            EncArgs e;
            e.par = w.par;
            e.codes = w.codes;
            e.enc = w.enc;
            e.out = reinterpret_cast<uint8_t*>(d_out[f]);
            e.n = p->n;
            e.chunk = (uint32_t)p->chunk;
            e.nchunks = p->nchunks;
            e.ntiles = (uint32_t)((p->nchunks + kEncTile - 1) / kEncTile);
            e.slot_words = p->enc_slot_words;
            e.scratch = w.enc_scratch;
            e.chunk_words = w.chunk_off;
            e.tile_sum = w.enc_tiles;
            b.a[f] = e;
            blocks[f] = p->n ? e.ntiles : 0u;
        }
        const uint32_t tot = batch_offsets(b, blocks);
        if (tot) {
            StageScope sc(prof, kStEncode, st);
            k_enc_pack<<<tot, kEncWarps * 32, 0, st>>>(b);
            FP_LAUNCH_CHECK();
            for (int f = 0; f <= count; f++) b.off[f] = (uint32_t)f;
            k_enc_scan<<<count, 1024, 0, st>>>(b);
            FP_LAUNCH_CHECK();
            batch_offsets(b, blocks);
            k_enc_copy<<<tot, kEncWarps * 32, 0, st>>>(b);
            FP_LAUNCH_CHECK();
            sc.more(2);
        }
    }

    // ---- outliers / verbatims in index order ----
    {
        Batch<EmitArgs> b;
        b.count = (uint32_t)count;
        for (int f = 0; f < count; f++) {
            const fpsnr_plan_s* p = P[f];
            const Workspace& w = p->w;
            const uint32_t G = small_blocks(p, count);
            b.a[f] = EmitArgs{w.par, w.stage_out, w.stage_vb, w.bm, w.wpre, w.bpre,
                              reinterpret_cast<uint8_t*>(d_out[f]), p->nwords, (uint32_t)p->nbmblk, G};
            blocks[f] = p->n ? 2 * G : 0u;
        }
        const uint32_t tot = batch_offsets(b, blocks);
        if (tot) {
            StageScope sc(prof, kStEmit, st);
            k_emit<<<tot, 256, 0, st>>>(b);
            FP_LAUNCH_CHECK();
        }
    }

    // ---- header, size, statistics, bitmap clearing ----
    {
        Batch<FinArgs> b;
        b.count = (uint32_t)count;
        for (int f = 0; f < count; f++) {
            const fpsnr_plan_s* p = P[f];
            const Workspace& w = p->w;
            FinArgs a;
            a.par = w.par;
            a.bm = w.bm;
            a.stage_out = w.stage_out;
            a.stage_vb = w.stage_vb;
            a.out = reinterpret_cast<uint8_t*>(d_out[f]);
            a.out_bytes = d_out_bytes ? d_out_bytes + f : nullptr;
            a.stats = d_stats ? d_stats + f : nullptr;
            a.ndim = p->ndim;
            a.ld = p->ld;
            a.d0 = p->dims[0];
            a.d1 = p->dims[1];
            a.d2 = p->dims[2];
            a.n = p->n;
            a.radius = p->radius;
            a.chunk = p->chunk;
            a.lmax = p->lmax;
            a.nchunks = p->nchunks;
            a.nwords = p->nwords;
            a.G = small_blocks(p, count);
            b.a[f] = a;
            blocks[f] = a.G;
        }
        const uint32_t tot = batch_offsets(b, blocks);
        StageScope sc(prof, kStFinalize, st);
        k_finalize<<<tot, 256, 0, st>>>(b);
        FP_LAUNCH_CHECK();
    }
    // optional lossless container around the finished blobs
    return launch_zr_wrap(P, d_out, d_out_bytes, d_stats, count, st);
}

}  // namespace fp
