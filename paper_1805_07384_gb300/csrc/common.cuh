// common.cuh -- internal declarations shared by the fpsnr CUDA translation units.
//
// The plan owns one device slab carved into the arrays of `Workspace`.  The
// per-call scalars (value range, error bound, counters, section offsets,
// status) live in one `DevParams` record on the device, so that a whole
// compress or decompress call is a chain of kernels on one stream with no
// host round trip.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fpsnr.h"

namespace fp {

constexpr uint32_t kMagic = 0x31535046u;  // bytes "FPS1"
constexpr uint32_t kVersion = 1u;
constexpr uint32_t kHeaderBytes = 128u;
constexpr uint32_t kFlagConstant = 1u;     // vr == 0 (or empty): header only
constexpr uint32_t kFlagLatticeOff = 2u;   // bin width not representable: q = 0
constexpr uint32_t kFlagError = 1u << 31;  // internal: a device-side error occurred
constexpr int kMaxRadius = 32768;
constexpr int kMaxSym = 2 * kMaxRadius;
constexpr int kMaxLmax = 27;
constexpr int kFineBins = 4096;  // fine histogram of the bound refinement (psnr_mode 1)
constexpr uint32_t kZrSeg = 1024;          // lossless container: bytes per segment
constexpr uint32_t kZrMagic = 0x315A5046u;  // bytes "FPZ1"
constexpr int kEncTile = 32;        // chunks per encoder tile
constexpr int kLutBits = 12;        // decode look-up table width
constexpr uint32_t kLutLen = 0x20u;  // table entry flag: length only, symbol by canonical index
constexpr uint32_t kLutSlow = 0x40u; // table entry flag: not a whole code of <= kLutBits bits
constexpr uint32_t kSpinLimit = 1u << 22;

// Per-call device record.  Written by kernels, read by later kernels.
struct DevParams {
    double vr, eb_abs, eb_rel, target_psnr;
    double sse;
    float xmin, xmax, s, inv, thr;
    uint32_t flags;
    int32_t status;
    uint32_t n_out, n_vb;     // staged outlier / verbatim counts
    uint32_t n_sym;           // Huffman symbols in use
    uint32_t stream_words;
    uint32_t done_range;      // self-resetting last-block counter
    uint32_t sym_lo, sym_hi;  // smallest / largest nonzero symbol seen by the predictor
    // look-back epoch of the inverse-Lorenzo scans, advanced on the device by
    // the first kernel of every decompress call (so a captured CUDA graph
    // replays correctly)
    uint32_t dec_epoch;
    float kinv;               // (float)(kFineBins / vr): fine-histogram bin scale
    // lossless container: wrap decision and sizes; unwrap outcome and raw length
    uint32_t zr_use, zr_bad;
    uint64_t zr_total, zr_dstart, zr_raw;
    uint64_t cap;             // output capacity of this call
    uint64_t off_cb, off_ct, off_st, off_ou, off_vb, total;
    // decompression: header fields of the blob being decoded
    uint32_t d_radius, d_chunk, d_lmax, d_nsym, d_nchunks, d_words, d_nout, d_nvb;
    uint32_t d_zero;  // symbols 0 (outliers) met by the first residual pass
    uint32_t d_count[32], d_first_code[32], d_first_index[32];
};

// Device arrays carved from the plan's slab.
struct Workspace {
    DevParams* par;
    uint32_t* hist;         // [nsym] symbol counts
    uint32_t* enc;          // [nsym] (code << 5) | len, 0 = unused
    uint8_t* len_sym;       // [nsym] code length per symbol
    uint16_t* codes;        // [n] symbols
    uint32_t* chunk_off;    // [nchunks] words per chunk, then exclusive word offsets
    uint2* stage_out;       // [n] (idx, delta) in discovery order
    uint2* stage_vb;        // [n] (idx, float bits) in discovery order
    uint32_t* bm;           // [2][nwords] membership bitmaps (kept all-zero between calls)
    uint32_t* wpre;         // [2][nwords] in-block exclusive popcount prefix (words with a set bit only)
    uint32_t* bpre;         // [2][nbmblk] block totals, then exclusive prefix
    double* sse_part;       // [n_pq_blocks]
    float* range_part;      // [3][n_range_blocks]
    // Huffman construction scratch
    unsigned long long* hlist;  // [nsym] used symbols (count << 16 | symbol), ascending symbol
    unsigned long long* hbuf1;  // [nsym] sort ping-pong
    unsigned long long* hbuf2;  // [nsym] sort ping-pong
    uint32_t* hpar;             // [2*nsym] parent of every node
    // decoding tables
    uint32_t* dlut;  // [1 << kLutBits] decode table
    uint16_t* dsyms; // [kMaxSym]
    // inverse-Lorenzo look-back state
    uint32_t* lb_flags;  // [n_lb_tiles]
    uint32_t* lb_vals;   // [2][n_lb_tiles * lb_width] aggregate, inclusive
    uint32_t* lb_ctr;    // [8] dynamic tile counters (pairs: counter, done)
    uint32_t* enc_tiles; // [enc_tiles] words per encoder tile, then their exclusive prefix
    uint32_t* enc_scratch;  // [nchunks * enc_slot_words] packed chunks before placement
    uint32_t* bsum;      // [nbands * nx] 2D band column sums (band geometry only)
    uint32_t* vcb;       // 3D tiles: [nz][nbands][nx] band column sums of every plane
    uint32_t* vds;       // 3D tiles: [nslabs][ny][nx] slab sums of every row
    uint32_t* vts;       // 3D tiles: [nslabs][nbands][nx] column sums of every tile
    uint32_t* fine_hist; // [kFineBins] bound refinement histogram (kept zero between calls)
    uint8_t* zr_scratch; // lossless plans: container (compress) / expanded blob (decompress)
    uint32_t* zr_seg;    // lossless plans: per-segment lengths, then offsets
};

// Launch geometry of the predict-quantize kernel.
struct PQGeom {
    int mode;          // 1: flat 1D, 2: rows x nx, 3: nz x ny x nx
    int tx, ty, zs;    // tile width (x), tile height (y), planes per block
    uint32_t vx, vy, vz;  // predictor view (x fastest)
    uint32_t nbx, nby, nbz;
    uint32_t nblocks;
    bool vec;          // rows start on 16-byte boundaries
};

// Geometry of one inverse-Lorenzo scan pass.
// 2D inverse Lorenzo by bands of rows, used when a row fits one block.
constexpr uint32_t kBandMaxNx = 8192;  // 256 threads x 8 columns x G (G <= 4)
constexpr uint32_t kBandRows = 32;     // rows per band
struct BandGeom {
    bool on;
    uint32_t nx, rows, tr, nbands;
    int g;     // 8 * g columns per thread
    bool vec;  // nx % 8 == 0: symbol rows and output rows start on 16-byte boundaries
};

// 3D inverse Lorenzo by tiles of tz planes x ty rows x the whole row, used
// when a row fits one block (nx <= kVolMaxNx): reduce, carry, scan.  A block
// has 16 warps; a row takes wpr of them (cpl columns per lane), so a tile has
// ty = 16 / wpr rows.
constexpr uint32_t kVolMaxNx = 2048;  // 4 warps x 32 lanes x 16 columns
constexpr uint32_t kVolSlab = 32;     // planes per slab
struct VolGeom {
    bool on;
    uint32_t nx, ny, nz, ty, tz, nbands, nslabs;
    int cpl;   // columns per lane: 4 (nx <= 128), 8 (<= 256), 16
    int wpr;   // warps per row: 1 (nx <= 512), 2 (<= 1024), 4 (<= 2048)
    bool vec;  // nx % 4 == 0: rows of floats start on 16-byte boundaries
};

struct ScanPass {
    int kind;          // 0: contiguous rows, 1: strided (middle axis)
    uint32_t A, L, B;  // outer count, scan length, inner count (B = 1 for contiguous)
    uint32_t tiles;
    int ipt;           // contiguous: items per thread; strided: rows per tile
    int tb;            // strided: columns per tile
    bool vec;          // rows of int32 values start on 16-byte boundaries
    bool vec16;        // rows of 16-bit symbols start on 16-byte boundaries
    bool final_pass;
    int ctr_slot;      // which lb_ctr pair
    uint64_t val_off;  // offset (in tiles) into the look-back arrays
};

}  // namespace fp

namespace fp {
enum Stage {
    kStRange = 0, kStPq, kStRank, kStCodebook, kStBandSum, kStBandCarry, kStEncode, kStEmit,
    kStFinalize, kStDsetup, kStDecode, kStRefine, kStScanX, kStScanY, kStScanFinal, kStPatch,
    kStZrWrap, kStZrUnwrap
};

// Host-side launch counters and optional per-launch CUDA events.
struct Profiler {
    bool on = false;
    uint64_t launches[FPSNR_NSTAGES] = {};
    struct Rec { int stage; cudaEvent_t a, b; };
    Rec* recs = nullptr;
    size_t nrec = 0, cap = 0;
    cudaEvent_t* pool = nullptr;
    size_t npool = 0, used = 0;
    cudaEvent_t take();
    void begin(int stage, cudaStream_t st, cudaEvent_t* a);
    void end(int stage, cudaStream_t st, cudaEvent_t a);
    void release();
};
}  // namespace fp

struct fpsnr_plan_s {
    int device;
    int ndim, ld;
    uint64_t dims[3];
    uint64_t n;
    double target_psnr, eb_rel;
    int radius, chunk, lmax;
    int psnr_mode;    // 0: eb from Eq. 8; 1: refined from the fine histogram
    int lossless;     // 1: wrap blobs in the zero-run container when smaller
    uint64_t zr_scratch_cap, zr_seg_cap;
    double mse_rel;   // 10^(-target / 10) (the target MSE over vr^2)
    uint32_t nsym;
    uint64_t nchunks, nwords, nbmblk;
    fp::PQGeom pq;
    uint32_t n_range_blocks;
    int n_passes;
    fp::ScanPass pass[3];
    fp::BandGeom band;
    fp::VolGeom vol;
    uint64_t lb_tiles_total, lb_width;
    uint64_t enc_tiles;
    uint32_t enc_slot_words;  // scratch words per chunk (chunk * lmax bits)
    void* slab;
    size_t slab_bytes;
    fp::Workspace w;
    int sm_count;
    int cb_smem;               // dynamic shared memory of the codebook kernel
    int dec_threads;           // decoder block size: 0 chosen per launch, or 128 / 512
    uint32_t spin_limit;       // polls before an inter-block wait gives up (FPSNR_ETIMEOUT)
    uint32_t wait_skew;        // test switch: look-back waits expect an epoch no block publishes
    uint32_t pq_blocks_cap;    // predictor blocks the workspace holds partials for (any tile width)
    uint32_t band_cap;         // band sums the workspace holds (band height 16)
    fp::Profiler prof;
};

// Brackets the kernel launches of one stage with the plan's profiler; the
// scope counts one launch, more() the stage's further launches.
struct StageScope {
    fp::Profiler& pr;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    StageScope(fp::Profiler& p, int s, cudaStream_t stream) : pr(p), stage(s), st(stream) {
        pr.begin(stage, st, &a);
    }
    void more(int k) { pr.launches[stage] += (uint64_t)k; }
    ~StageScope() { pr.end(stage, st, a); }
};

namespace fp {

// ---- batched launches ----
// A batch runs one kernel launch per stage for up to kMaxBatch fields.  The
// per-field arguments travel in the kernel parameter (a __grid_constant__
// table, so no device memory and nothing to re-upload when a graph replays);
// block b belongs to the field f with off[f] <= b < off[f + 1].
constexpr int kMaxBatch = 32;

template <class A>
struct Batch {
    uint32_t count;
    uint32_t off[kMaxBatch + 1];
    A a[kMaxBatch];
};

// Host: fills off[] from per-field block counts; returns the total.
template <class A>
inline uint32_t batch_offsets(Batch<A>& b, const uint32_t* blocks) {
    uint32_t t = 0;
    for (uint32_t f = 0; f < b.count; f++) {
        b.off[f] = t;
        t += blocks[f];
    }
    b.off[b.count] = t;
    return t;
}

#ifdef __CUDACC__
// Field of block `bid`: the largest f with off[f] <= bid (fields with no
// blocks are skipped because a later field starts at the same offset).
__device__ __forceinline__ uint32_t batch_field(const uint32_t* off, uint32_t count, uint32_t bid) {
    uint32_t lo = 0, hi = count;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= bid) lo = mid;
        else hi = mid;
    }
    return lo;
}
#endif

// ---- host-side launchers ----
int launch_compress_batch(fpsnr_plan_s* const* plans, const float* const* d_in,
                          void* const* d_out, const uint64_t* caps, uint64_t* d_out_bytes,
                          fpsnr_stats* d_stats, int count, cudaStream_t st);
int launch_codebook_batch(fpsnr_plan_s* const* plans, void* const* d_out, int count,
                          cudaStream_t st);
int launch_decompress_batch(fpsnr_plan_s* const* plans, const void* const* d_blob,
                            const uint64_t* bytes, float* const* d_out, int* d_status, int count,
                            cudaStream_t st);
int codebook_smem_bytes();
// PSNR reduction (psnr.cu): scratch = 16-byte zeroed counter, 32-byte result,
// then one partial per block.
int psnr_enqueue(const float* d_x, const float* d_xr, uint64_t n, void* scratch, unsigned blocks,
                 cudaStream_t st);
int psnr_finish(const void* h_result, double* psnr_db, double* mse, double* vr, uint64_t n);
size_t psnr_scratch_bytes_for(unsigned blocks);
constexpr size_t kPsnrResultOffset = 16;
constexpr size_t kPsnrResultBytes = 24;
int codebook_prepare();
int decode_prepare(const fpsnr_plan_s* p);
// lossless container (lossless.cu)
int launch_zr_wrap(fpsnr_plan_s* const* plans, void* const* d_out, uint64_t* d_out_bytes,
                   fpsnr_stats* d_stats, int count, cudaStream_t st);
int launch_zr_unwrap(fpsnr_plan_s* const* plans, const void* const* d_blob, const uint64_t* bytes,
                     int count, cudaStream_t st);

// ---- device helpers ----
#ifdef __CUDACC__

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Sets the device status once (first error wins) and raises the error flag.
__device__ __forceinline__ void set_error(DevParams* par, int code) {
    atomicCAS(reinterpret_cast<int*>(&par->status), 0, code);
    atomicOr(&par->flags, kFlagError);
}

// Block-wide exclusive scan of one uint32 per thread (blockDim.x multiple of 32,
// at most 1024).  `sh` needs 33 words.  Returns the exclusive prefix; *total
// receives the block sum.  Contains __syncthreads.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* sh, uint32_t* total) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? sh[lane] : 0u;
        uint32_t s = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= (uint32_t)o) s += y;
        }
        if (lane < nw) sh[lane] = s - w;
        if (lane == nw - 1) sh[32] = s;
    }
    __syncthreads();
    uint32_t r = sh[warp] + x - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

// Error-free transformations on float32 (Knuth TwoSum, FMA-based TwoProd).
// Every operation is an explicit round-to-nearest intrinsic so that the
// compiler neither contracts nor reassociates them.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ double ff_to_double(const FF& a) { return (double)a.hi + (double)a.lo; }

// Sum of squared differences for any float range: the difference is split
// exactly (TwoSum) in the inputs' own units, and its two parts are scaled by
// 2^-e before the exact square is accumulated in float-float, e a unit kept
// above every difference seen so far (|dh| < 2^(e+1)).  When a larger
// difference arrives the unit rises and the float-float sum so far moves to an
// FP64 spill (a rare branch), so squares neither overflow nor lose their low
// parts to underflow.  Total = spill + float-float sum * 2^(2e).
struct SqSum {
    FF acc;
    double spill;
    int e;      // the unit's exponent
    float sc;   // 2^-e
    float lim;  // 2^(e + 1)
};

__device__ __forceinline__ void sq_init(SqSum& q) {
    q.acc = FF{0.0f, 0.0f};
    q.spill = 0.0;
    q.e = -100;  // differences of floats are 0 or at least 2^-149
    q.sc = __uint_as_float((uint32_t)(127 + 100) << 23);
    q.lim = __uint_as_float((uint32_t)(127 - 99) << 23);
}

__device__ __forceinline__ double sq_unit2(int e) {
    return __longlong_as_double((long long)(1023 + 2 * e) << 52);  // 2^(2e)
}

__device__ __forceinline__ void sq_add(SqSum& q, float a, float b) {
    // exact a - b = dh + dl
    const float nb = -b;
    const float dh = __fadd_rn(a, nb);
    const float bb = __fsub_rn(dh, a);
    const float dl = __fadd_rn(__fsub_rn(a, __fsub_rn(dh, bb)), __fsub_rn(nb, bb));
    if (!(fabsf(dh) < q.lim)) {
        // raise the unit above |dh| (an infinite or NaN dh takes the top unit)
        q.spill = __dadd_rn(q.spill, __dmul_rn(ff_to_double(q.acc), sq_unit2(q.e)));
        q.acc = FF{0.0f, 0.0f};
        const int bd = (int)((__float_as_uint(dh) >> 23) & 0xffu);
        q.e = min(max(q.e, bd - 127 + 1), 126);
        q.sc = __uint_as_float((uint32_t)(127 - q.e) << 23);
        q.lim = q.e < 126 ? __uint_as_float((uint32_t)(127 + q.e + 1) << 23) : __int_as_float(0x7f800000);
    }
    const float h = __fmul_rn(dh, q.sc), l = __fmul_rn(dl, q.sc);
    // (h + l)^2 = p + e with the 2 h l cross term (l^2 is below the precision kept)
    const float p = __fmul_rn(h, h);
    float er = __fmaf_rn(h, h, -p);
    er = __fmaf_rn(__fadd_rn(h, h), l, er);
    const float t = __fadd_rn(q.acc.hi, p);
    const float tb = __fsub_rn(t, q.acc.hi);
    const float err = __fadd_rn(__fsub_rn(q.acc.hi, __fsub_rn(t, tb)), __fsub_rn(p, tb));
    q.acc.hi = t;
    q.acc.lo = __fadd_rn(q.acc.lo, __fadd_rn(err, er));
}

__device__ __forceinline__ double sq_total(const SqSum& q) {
    return __dadd_rn(q.spill, __dmul_rn(ff_to_double(q.acc), sq_unit2(q.e)));
}

// Two independent float-float accumulators in the packed f32x2 lanes.  The
// subtractions are fma(x, -1, y): the product is exact, so each is the single
// rounding of y - x, as a subtraction would be.
struct FF2 {
    float2 hi, lo;
};

__device__ __forceinline__ float2 f2_sub(float2 y, float2 x) {
    return __ffma2_rn(x, make_float2(-1.0f, -1.0f), y);
}

// acc += (a - b)^2 in each lane, given nb = -b and dh = fl(a + nb); a lane
// whose keep flag is false adds exactly zero (whatever a and b hold).
__device__ __forceinline__ void ff2_add_sq_diff(FF2& acc, float2 a, float2 nb, float2 dh, bool keep0,
                                                bool keep1) {
    // exact a - b = dh + dl (TwoSum)
    const float2 bb = f2_sub(dh, a);
    const float2 dl = __fadd2_rn(f2_sub(a, f2_sub(dh, bb)), f2_sub(nb, bb));
    // d^2 = p + e with np = -p (FMA TwoProd, plus the 2 dh dl cross term)
    const float2 ndh = __fmul2_rn(dh, make_float2(-1.0f, -1.0f));
    float2 np = __fmul2_rn(dh, ndh);
    float2 e = __ffma2_rn(dh, dh, np);
    e = __ffma2_rn(__fadd2_rn(dh, dh), dl, e);
    // np reaches the adds below only through these selects: a __fmul2_rn result
    // that feeds a __fadd2_rn directly was measured to be fused into one fma,
    // which would fold e into err and count it twice
    np.x = keep0 ? np.x : 0.0f;
    np.y = keep1 ? np.y : 0.0f;
    e.x = keep0 ? e.x : 0.0f;
    e.y = keep1 ? e.y : 0.0f;
    // acc.hi + p = t + err (TwoSum; p - tb is formed as -(np + tb))
    const float2 t = f2_sub(acc.hi, np);
    const float2 tb = f2_sub(t, acc.hi);
    const float2 err = f2_sub(f2_sub(acc.hi, f2_sub(t, tb)), __fadd2_rn(np, tb));
    acc.hi = t;
    acc.lo = __fadd2_rn(acc.lo, __fadd2_rn(err, e));
}

__device__ __forceinline__ double ff2_to_double(const FF2& a) {
    return ((double)a.hi.x + (double)a.lo.x) + ((double)a.hi.y + (double)a.lo.y);
}

// Deterministic block reduction of one double per thread (fixed tree order).
// `sh` needs blockDim.x/32 doubles.  Result valid in thread 0.
__device__ __forceinline__ double block_sum_double(double v, double* sh) {
    const uint32_t tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    const uint32_t lane = tid & 31u, warp = tid >> 5;
    const uint32_t nw = (blockDim.x * blockDim.y * blockDim.z) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (tid == 0)
        for (uint32_t i = 0; i < nw; i++) r += sh[i];
    return r;
}

// ---- TMA bulk copies (cp.async.bulk) completing on an mbarrier ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive once and announce `bytes` of asynchronous transactions.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
                 "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy; dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         unsigned long long* mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* mbar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_u32(mbar)), "r"(phase) : "memory");
    return ok != 0;
}

// Bounded wait for phase `phase` of an mbarrier; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* mbar, uint32_t phase,
                                                  uint32_t limit = kSpinLimit) {
    for (uint32_t it = 0; it < limit; it++)
        if (mbar_try_wait(mbar, phase)) return true;
    return false;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Decoupled look-back over tiles [first, t): one warp inspects 32 predecessors
// per round trip.  Each tile publishes flags[tile] = epoch << 2 | state with
// state 1 (its own aggregate in agg[tile]) or 2 (inclusive prefix in inc[tile]).
// Waits (at most `limit` polls per round trip) until every inspected
// predecessor has published under `epoch`, adds the aggregates of those nearer
// than the nearest inclusive prefix plus that prefix, and stops there.
// Returns the exclusive prefix of tile t in every lane; on a timeout sets
// FPSNR_ETIMEOUT and returns what it has.
__device__ __forceinline__ uint32_t warp_lookback(const uint32_t* flags, const uint32_t* agg,
                                                  const uint32_t* inc, uint32_t t, uint32_t first,
                                                  uint32_t epoch, uint32_t limit, DevParams* par) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t carry = 0;
    int64_t hi = (int64_t)t - 1;
    while (hi >= (int64_t)first) {
        const int64_t p = hi - lane;
        const bool valid = p >= (int64_t)first;
        uint32_t st = 0;
        for (uint32_t it = 0;; it++) {
            if (valid && st == 0) {
                const uint32_t f = ld_acquire(flags + p);
                if ((f >> 2) == epoch && (f & 3u)) st = f & 3u;
            }
            if (__all_sync(0xffffffffu, !valid || st != 0)) break;
            if (it >= limit) {
                if (lane == 0) set_error(par, FPSNR_ETIMEOUT);
                return __shfl_sync(0xffffffffu, carry, 0);
            }
            __nanosleep(32);
        }
        const uint32_t pmask = __ballot_sync(0xffffffffu, valid && st == 2u);
        const uint32_t stop = pmask ? (uint32_t)(__ffs(pmask) - 1) : 32u;
        uint32_t v = 0;
        if (valid && lane <= stop) v = (st == 2u) ? __ldcg(inc + p) : __ldcg(agg + p);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        carry += v;
        if (pmask) break;
        hi -= 32;
    }
    return carry;
}

#endif  // __CUDACC__

}  // namespace fp
