/*
 * fpsnr.h -- C ABI of the GB300 fixed-PSNR lossy compressor.
 *
 * Method: Tao, Di, Liang, Chen, Cappello, "Fixed-PSNR Lossy Compression for
 * Scientific Data".  The caller states a target PSNR; the library derives the
 * value-range-relative error bound from it (Eq. 8, Sec. IV), multiplies it by
 * the field's value range (eb_abs = eb_rel * vr, Sec. IV after Eq. 7), runs a
 * prediction-based compressor at that bound (Sec. II-A steps 1-2, Sec. III),
 * and reports the PSNR the reconstruction actually reaches (Eq. 4-5).
 *
 * Every step runs on the GPU in this library's own sm_103a kernels.  All
 * pointers named d_* are device pointers on the plan's device; h_* are host
 * pointers.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  No function throws; every function returns 0 (FPSNR_OK) or a
 * negative FPSNR_E* code for errors known when the work is enqueued.  Errors
 * that depend on the data (non-finite input, output too small, corrupt blob)
 * are written to a device status word and are visible after the stream is
 * synchronized.
 *
 * Data layout: a field is a dense float32 array of 1 to 3 dimensions, C order
 * with x the fastest axis; dims[0] = nx, dims[1] = ny, dims[2] = nz.
 * At most 2^32 - 1 points per field.
 *
 * Compressed byte format (little-endian; every section padded to 16 bytes):
 *   header, 128 bytes:
 *     0 u32 magic "FPS1"  4 u32 version (1)  8 u32 ndim  12 u32 lorenzo dims
 *    16 u64 dims[3] (x fastest, unused = 1)
 *    40 f64 target PSNR  48 f64 eb_rel  56 f64 eb_abs  64 f64 vr
 *    72 f32 xmin  76 f32 xmax  80 f32 s = (float)(2 eb_abs)
 *    84 f32 inv = (float)(1 / (2 eb_abs))  88 f32 thr (verbatim threshold)
 *    92 u32 flags (1 = constant field, 2 = lattice off)
 *    96 u32 radius R  100 u32 chunk C  104 u32 lmax  108 u32 n_sym
 *   112 u32 n_chunks  116 u32 stream_words  120 u32 n_outlier  124 u32 n_verbatim
 *   codebook:   n_sym u32 entries (len << 16 | symbol), ascending (len, symbol)
 *   chunk table: n_chunks u32 word offsets into the stream
 *   stream:     stream_words u32 words, canonical Huffman codes MSB-first;
 *               each chunk of C symbols starts on a fresh word
 *   outliers:   n_outlier (u32 index, i32 residual), ascending index
 *   verbatims:  n_verbatim (u32 index, u32 float bits), ascending index
 * Symbols: residual delta of the integer lattice q = round((x - xmin) * inv)
 * under the zero-padded Lorenzo predictor; symbol = delta + R when
 * |delta| < R, else 0 and the residual travels in the outlier list.  A point
 * whose reconstruction fmaf((float)q, s, xmin) misses the bound travels
 * verbatim.
 */
#ifndef FPSNR_H
#define FPSNR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FPSNR_OK 0
#define FPSNR_EINVAL (-1)     /* bad argument (ndim, dims, PSNR, options, alignment) */
#define FPSNR_ENOMEM (-2)     /* device allocation failed while planning */
#define FPSNR_ECUDA (-3)      /* a CUDA call or kernel launch failed */
#define FPSNR_ENONFINITE (-4) /* (device status) input holds NaN or Inf */
#define FPSNR_ECAPACITY (-5)  /* (device status) compressed size exceeds out_cap */
#define FPSNR_ECORRUPT (-6)   /* (device status) blob malformed or mismatched */
#define FPSNR_ETIMEOUT (-7)   /* (device status) an inter-block wait gave up */
#define FPSNR_EAGAIN (-8)     /* (server) the request has not completed yet */

/* Limits on the target PSNR: 0 < target <= FPSNR_MAX_PSNR dB.  Above 180 dB
 * the integer lattice of a 3D residual could overflow int32. */
#define FPSNR_MAX_PSNR 180.0

typedef struct fpsnr_plan_s* fpsnr_plan_t;

/* Options; fpsnr_default_opts fills the defaults shown. */
typedef struct {
    int radius;       /* R, 1..32768: residuals in (-R, R) are Huffman symbols (32768) */
    int chunk;        /* C, symbols per independently decodable chunk, 32..65536 (256) */
    int lmax;         /* longest Huffman code in bits, 1..27, 2^lmax >= 2R (27) */
    int lorenzo_dims; /* predictor dimension d, 0 = ndim; d < ndim merges the
                         slowest axes into the slowest predictor axis */
    int psnr_mode;    /* 0: eb from Eq. 8 (0).  1: refine eb on the field's
                         empirical PDF: Eq. 3 evaluated on a 4096-bin histogram
                         of the values (each fine bin contributes its count x
                         (e^2 + w^2/12), e the lattice error of its centre, w
                         its width), and the largest eb in [eb8/4, 64 eb8] whose
                         predicted MSE meets the target, by 16 geometric
                         bisections; only when Eq. 8's bin 2 eb8 spans at least
                         16 fine bins (targets below about 59 dB), else eb8.
                         Eq. 3 is evaluated in units of the value range (bin
                         centres (j + 1/2)/4096, target 10^(-PSNR/10)), each
                         term in float and their weighted sum exactly, rounded
                         once to FP64.
                         Costs one more pass over the input.  The blob records
                         the eb used; decompression is unchanged. */
    int lossless;     /* 0: none (0).  1: optional lossless layer (the paper's
                         optional lossless step, Sec. II-A): the finished blob
                         is wrapped in the container below when that is
                         smaller, else left as it is.  A plan with lossless 1
                         decompresses both forms; a plan with 0 only plain
                         blobs.  Its workspace grows by about the largest blob.
                         Container "FPZ1": u32 magic 0x315A5046, u32 version 1,
                         u64 blob bytes, u32 segment bytes (1024), u32 segments
                         S, 8 zero bytes; u32 offsets[S + 1] (start of every
                         segment's data in the data section, bit 31 = stored
                         raw; the last entry is the data length), zero-padded
                         to 16 bytes; the data section, zero-padded to 16 bytes.
                         A segment is coded byte by byte: a nonzero byte is
                         copied, a run of k zero bytes becomes 0x00 and k - 1
                         in LEB128; it is stored raw when the code is not
                         shorter. */
} fpsnr_opts;

/* Per-call statistics, written by fpsnr_compress to device memory. */
typedef struct {
    double target_psnr; /* dB, as planned */
    double eb_rel;      /* Eq. 8 */
    double eb_abs;      /* eb_rel * vr */
    double vr;          /* max - min of the input, FP64 */
    double psnr_model;  /* Eq. 7 at eb_abs (equals the target up to rounding) */
    double sse;         /* sum of squared reconstruction errors, FP64 */
    double mse;         /* sse / n */
    double psnr_actual; /* 20 log10 vr - 10 log10 mse; +inf when mse == 0 */
    uint64_t bytes;     /* compressed size, 0 on error */
    uint64_t n_outlier; /* residuals outside (-R, R) */
    uint64_t n_verbatim;/* points stored as raw floats */
    uint64_t n_sym;     /* Huffman symbols in use */
    float xmin, xmax;
    uint32_t flags;     /* 1 constant field, 2 lattice off */
    int32_t status;     /* FPSNR_OK or a device-side error code */
} fpsnr_stats;

/* Fill *opts with the defaults.  Returns FPSNR_OK, or FPSNR_EINVAL if NULL. */
int fpsnr_default_opts(fpsnr_opts* opts);

/* Create a plan for fields of one shape on the current CUDA device.  The
 * plan evaluates Eq. 8 (Sec. IV) on the host in FP64: eb_rel =
 * sqrt(3) 10^(-PSNR/20), the bound relative to the value range that makes the
 * uniform quantizer's MSE (Eq. 6-7) meet the target; eb_abs = eb_rel * vr is
 * formed on the device once the range is known.
 *   ndim 1..3; dims[ndim], x fastest, each >= 0 (a zero extent gives an empty
 *   field); target_psnr_db in (0, FPSNR_MAX_PSNR]; opts NULL = defaults.
 * The plan owns all device scratch (about 20 bytes per point, one cudaMalloc;
 * creating a plan synchronises the device once, destroying it too) and is not
 * thread-safe: one call at a time per plan (calls on one stream serialize).
 * Arguments are checked before any device call.
 * Returns FPSNR_OK, FPSNR_EINVAL, FPSNR_ENOMEM or FPSNR_ECUDA. */
int fpsnr_plan(fpsnr_plan_t* out, int ndim, const uint64_t* dims, double target_psnr_db,
               const fpsnr_opts* opts);

/* Change the plan's target PSNR (Eq. 8, Sec. IV, is re-evaluated on the host;
 * no allocation).  Returns FPSNR_OK or FPSNR_EINVAL. */
int fpsnr_plan_set_psnr(fpsnr_plan_t plan, double target_psnr_db);

/* eb_rel of the plan's current target (Eq. 8), computed on the host in FP64. */
double fpsnr_plan_eb_rel(fpsnr_plan_t plan);

/* Number of points of the plan's shape. */
uint64_t fpsnr_plan_points(fpsnr_plan_t plan);

/* Upper bound on the compressed size of any field of the plan's shape. */
uint64_t fpsnr_max_compressed_bytes(fpsnr_plan_t plan);

/* Compress d_in (n float32 points of the plan's shape) into d_out: the value
 * range vr (Sec. IV, under Eq. 5), eb_abs = eb_rel * vr (Sec. IV, after Eq. 7),
 * prediction by the Lorenzo predictor and uniform quantization with bins of
 * width 2 eb_abs (Sec. II-A steps 1-2, Sec. IV), Huffman coding of the
 * quantization codes (Sec. II-A step 2), and the reconstruction error the
 * decompressor will reproduce, summed into the achieved PSNR (Eq. 4-5; Sec.
 * III shows the error of the data equals the error of the prediction
 * residuals, Eq. 1, so it is known at compression time).
 *   d_in: 4-byte aligned; d_out: 16-byte aligned, out_cap bytes.
 *   d_out_bytes (device, may be NULL): receives the blob size, 0 on error.
 *   d_stats (device, may be NULL): receives fpsnr_stats.
 * Asynchronous on `stream`; no host synchronization, no allocation.
 * Enqueue errors: FPSNR_EINVAL, FPSNR_ECUDA.  Device status: FPSNR_ENONFINITE,
 * FPSNR_ECAPACITY (nothing beyond out_cap is written). */
int fpsnr_compress(fpsnr_plan_t plan, const float* d_in, void* d_out, uint64_t out_cap,
                   uint64_t* d_out_bytes, fpsnr_stats* d_stats, void* stream);

/* Decompress a blob produced for a field of the plan's shape (Sec. III: the
 * quantization codes are decoded, the prediction residuals rebuilt, and the
 * data recovered from them by inverting the Lorenzo predictor, Eq. 1; the
 * midpoint of each bin is the reconstructed value, Sec. IV).  A caller that
 * holds only the blob gets a fitting plan from fpsnr_blob_info and
 * fpsnr_plan_from_blob.
 *   d_blob: 16-byte aligned, blob_bytes long; d_out: n_out floats, 16-byte
 *   aligned, n_out == fpsnr_plan_points(plan).  d_out is also used as int32
 *   scratch while decoding.  d_status (device, may be NULL) receives
 *   FPSNR_OK or FPSNR_ECORRUPT (bad header, shape mismatch, malformed stream).
 * Asynchronous on `stream`; no allocation. */
int fpsnr_decompress(fpsnr_plan_t plan, const void* d_blob, uint64_t blob_bytes, float* d_out,
                     uint64_t n_out, int* d_status, void* stream);

/* Header of a compressed blob, as fpsnr_blob_info reads it (the byte format
 * above; for the lossless container, the header of the blob inside it). */
typedef struct {
    int ndim;             /* 1..3 */
    int lorenzo_dims;     /* predictor dimension the blob was made with */
    uint64_t dims[3];     /* x fastest; unused = 1 */
    uint64_t points;      /* dims[0] * dims[1] * dims[2] */
    double target_psnr;   /* dB, as planned */
    double eb_rel, eb_abs, vr;
    float xmin, xmax;
    uint32_t flags;       /* 1 constant field, 2 lattice off */
    int radius, chunk, lmax;
    int lossless;         /* 1: the bytes are the "FPZ1" container */
    uint64_t raw_bytes;   /* size of the plain blob (inside the container, if any) */
    uint64_t n_outlier, n_verbatim;
} fpsnr_blob_header;

/* Reads the header of a blob (device or host memory, blob_bytes long), so
 * that a caller holding only the bytes can plan their decompression (the
 * workflow of Sec. IV ends with the compressed data alone; the decompressor
 * must recover everything else from it).  For the lossless container it
 * expands the first segment on the host.  Copies at most a few KiB to the
 * host on `stream` and synchronizes it; allocates nothing.
 * Returns FPSNR_OK, FPSNR_EINVAL (null pointer), FPSNR_ECORRUPT (not a blob
 * of this library, or a header no plan can take) or FPSNR_ECUDA. */
int fpsnr_blob_info(const void* blob, uint64_t blob_bytes, fpsnr_blob_header* info, void* stream);

/* Creates a plan that decompresses blobs with this header: the blob's shape,
 * predictor dimension, radius, chunk size, code-length limit and target, and
 * opts.lossless set when the blob is a container.  As fpsnr_plan otherwise
 * (allocates the plan's workspace, synchronizes the device once).
 * Returns FPSNR_OK, FPSNR_EINVAL, FPSNR_ENOMEM or FPSNR_ECUDA. */
int fpsnr_plan_from_blob(fpsnr_plan_t* out, const fpsnr_blob_header* info);

/* Batched compression (Sec. II-A, III, IV per field, as fpsnr_compress):
 * `count` fields, each with its own plan (shape, target
 * PSNR, options), compressed by one kernel launch per stage, so that stages
 * bound by latency (Huffman construction, look-back chains, small kernels)
 * overlap across fields.  plans, d_in, d_out, out_cap: host arrays of `count`
 * entries (pointers as for fpsnr_compress; the plans must be distinct and on
 * the current device).  d_out_bytes: device array of `count` u64 (may be NULL);
 * d_stats: device array of `count` fpsnr_stats (may be NULL).  Results equal
 * those of `count` separate fpsnr_compress calls.  Any count is accepted;
 * launches cover at most 32 fields each.  Asynchronous, no allocation.
 * Returns FPSNR_OK, FPSNR_EINVAL or FPSNR_ECUDA. */
int fpsnr_compress_batch(const fpsnr_plan_t* plans, const float* const* d_in, void* const* d_out,
                         const uint64_t* out_cap, uint64_t* d_out_bytes, fpsnr_stats* d_stats,
                         int count, void* stream);

/* Batched decompression (Sec. III, Eq. 1, per field as fpsnr_decompress), the
 * counterpart of fpsnr_compress_batch: host arrays
 * plans, d_blob, blob_bytes, d_out of `count` entries; d_status: device array
 * of `count` ints (may be NULL).  Asynchronous, no allocation. */
int fpsnr_decompress_batch(const fpsnr_plan_t* plans, const void* const* d_blob,
                           const uint64_t* blob_bytes, float* const* d_out, int* d_status,
                           int count, void* stream);

/* Distortion of a reconstruction (Eq. 4-5, Sec. IV): vr = max - min of d_x (FP64),
 * MSE = sum((x - xr)^2) / n with exact squares accumulated to FP64,
 * PSNR = 20 log10 vr - 10 log10 MSE (+inf when MSE == 0), log10 on the host.
 *   d_x, d_xr: n float32 points each, 4-byte aligned.
 * Synchronous: returns after the result is on the host.  Allocates a small
 * scratch (under 64 KB) with cudaMallocAsync on `stream` and frees it.
 * Returns FPSNR_OK, FPSNR_EINVAL, FPSNR_ENONFINITE (NaN/Inf in d_x) or
 * FPSNR_ECUDA. */
int fpsnr_psnr(const float* d_x, const float* d_xr, uint64_t n, double* h_psnr_db,
               double* h_mse, double* h_vr, void* stream);

/* PSNR of a reconstruction (Eq. 4-5) without allocating device memory.  There
 * is no counterpart in the paper: this entry point exists for callers that cannot
 * allocate device memory while they run, such as code inside a device memory
 * allocator's or memory pool's own callback (allocating there would re-enter
 * the allocator), processes held to a fixed memory budget reserved up front,
 * and latency-critical service loops that must stay out of the CUDA allocator
 * (cudaMalloc and cudaFree can synchronize the whole device).
 * It computes the same quantities as fpsnr_psnr with the same kernel; its
 * scratch is one fixed 64 KiB device array inside this library, which every
 * GPU that loads the library holds until the process exits.
 *   n <= FPSNR_PSNR_STATIC_MAX_POINTS (2^28 points, 1 GiB of float32); a
 *   larger n returns FPSNR_EINVAL without touching the device.
 *   The two entry points split the points among threads and blocks
 *   differently (512 x 256 points per block here, a grid capped at four
 *   blocks per SM there), so their float-float partial sums round
 *   differently: the MSE agrees to about 1e-12 relative, the PSNR to about
 *   1e-11 dB.
 * The first call on each device looks up the array's device address with that
 * device current and keeps it for the process; make that first call before
 * any stream capture.  A cudaDeviceReset of that device (which unloads the
 * library's module, and with it the array) leaves the kept address stale:
 * after a reset this entry point must not be called again.  All calls
 * share the one array, which keeps the last call's contents; each call clears
 * the part that must start at zero.  Calls that overlap on the GPU (from two
 * host threads, or on two streams of one device) race on the array: the
 * caller must serialize them.  Synchronous, like fpsnr_psnr.
 * Returns FPSNR_OK, FPSNR_EINVAL, FPSNR_ENONFINITE or FPSNR_ECUDA. */
#define FPSNR_PSNR_STATIC_MAX_POINTS (1ull << 28)
int fpsnr_psnr_static(const float* d_x, const float* d_xr, uint64_t n, double* h_psnr_db,
                      double* h_mse, double* h_vr, void* stream);

/* Launch shapes and chunk size of a plan.  The paper fixes none of these: the
 * chunk size C (symbols per independently decodable Huffman chunk, a header
 * field) trades decoder parallelism against one u32 offset per chunk in the
 * stream; the tile shapes change only how the work is split over blocks, never
 * the bytes.
 *   chunk        symbols per chunk (0: keep the plan's)
 *   pq_tile_x    2D predictor tile width: 128, 256, 512 or 1024 points (0: by row length)
 *   band_rows    2D decompression band height: 16, 32 or 64 rows (0: 32); only
 *                for 2D fields with rows of at most 8192 points
 *   dec_threads  decoder block size: 128, 256 or 512 (0: chosen per launch)
 *   ms, bytes    filled by fpsnr_autotune: best compress + decompress time of the
 *                sample (milliseconds) and its compressed size at `chunk` */
typedef struct {
    int chunk;
    int pq_tile_x;
    int band_rows;
    int dec_threads;
    double ms;
    uint64_t bytes;
} fpsnr_tuning;

/* Applies the launch shapes of `t` to the plan (t->chunk must be 0 or equal
 * the plan's chunk; a plan's chunk is fixed when it is created).  Values that
 * do not apply to the plan's shape, or are not in the lists above, return
 * FPSNR_EINVAL and leave the plan unchanged.  Not while a call on the plan is
 * in flight. */
int fpsnr_plan_set_tuning(fpsnr_plan_t plan, const fpsnr_tuning* t);
int fpsnr_plan_get_tuning(fpsnr_plan_t plan, fpsnr_tuning* t);

/* Failure handling.  Every wait of one thread block on another (the
 * decoupled look-back of the scans that invert the predictor for 1D fields and
 * for rows wider than one tile, and the decoder's wait for its table copy)
 * polls at most `spins` times (0: the default, 2^22; each poll sleeps about
 * 32 ns), then records FPSNR_ETIMEOUT in the device status and returns, so
 * that a wait that cannot end leaves an error, not a hung GPU.  test_unmet = 1
 * makes the look-back waits expect a flag that no block ever sets, so that
 * every such wait runs out: for tests of this path (the output is then
 * meaningless and the status FPSNR_ETIMEOUT); 0 for normal use.  Not while a
 * call on the plan is in flight.  Returns FPSNR_OK or FPSNR_EINVAL. */
int fpsnr_plan_set_wait_limit(fpsnr_plan_t plan, uint32_t spins, int test_unmet);

/* Autotuner: picks the chunk size and launch shapes for fields of this shape,
 * target and options by timing compress + decompress of `d_sample` (a device
 * field of that shape, 4-byte aligned) on `stream`.  It tries chunk sizes
 * 64..2048 (and opts->chunk), keeps those whose compressed size is within
 * (1 + max_size_increase) of the smallest, takes the fastest of them, then
 * tunes pq_tile_x, band_rows and dec_threads one at a time at that chunk.
 * Each candidate is timed as the best of 3 runs after a warm-up, with CUDA
 * events.  Results are cached for the process by (shape, target, options,
 * max_size_increase); a cached answer returns without touching the device.
 * Synchronous; allocates temporary device buffers and plans.
 * Returns FPSNR_OK, FPSNR_EINVAL, FPSNR_ENOMEM or FPSNR_ECUDA (or the status
 * a sample compression reported, e.g. FPSNR_ENONFINITE). */
int fpsnr_autotune(int ndim, const uint64_t* dims, double target_psnr_db, const fpsnr_opts* opts,
                   const float* d_sample, double max_size_increase, fpsnr_tuning* out,
                   void* stream);

/* ------------------------------------------------------------------------
 * Request server (no counterpart in the paper, which compresses one field per
 * call).  A worker thread takes compress and decompress requests for fields of
 * any shape and target as they arrive, keeps plans (and so their device
 * workspace, tables and codebooks) cached per (shape, options), admits a
 * request only while the plans it needs fit an HBM budget, and fuses the
 * admitted requests of one kind into batched launches (fpsnr_compress_batch /
 * fpsnr_decompress_batch) on a few streams, continuously: each stream holds
 * one batch in flight, and as soon as a stream is free the requests that have
 * arrived leave together (a batch never waits to fill).  Results are identical
 * to a plain call on the same field (every kernel is deterministic and per
 * field).
 * ------------------------------------------------------------------------ */
typedef struct fpsnr_server_s* fpsnr_server_t;

/* hbm_budget   bytes of device memory the server's cached plans may hold (the
 *              caller's input and output buffers are not counted); idle plans
 *              are evicted least recently used first to admit others; a request
 *              whose plan alone exceeds the budget fails with FPSNR_ENOMEM
 * max_batch    requests fused into one launch (1..32)
 * streams      CUDA streams the worker launches on (1..16) */
typedef struct {
    uint64_t hbm_budget;
    int max_batch;
    int streams;
} fpsnr_server_opts;

#define FPSNR_REQ_COMPRESS 0
#define FPSNR_REQ_DECOMPRESS 1

/* kind         FPSNR_REQ_COMPRESS or FPSNR_REQ_DECOMPRESS
 * ndim, dims   field shape, x fastest (as fpsnr_plan)
 * target_psnr_db, opts   as fpsnr_plan (opts.radius 0 means the defaults);
 *              decompression uses opts and dims to pick the plan, and the blob
 *              must have been made with them
 * d_in         compress: float32 field (4-byte aligned); decompress: blob
 *              (16-byte aligned) of in_bytes bytes
 * d_out        compress: blob buffer of out_cap bytes; decompress: float32
 *              output of the field's points (both 16-byte aligned)
 * arrival_us   when the request may start, in microseconds of the server's
 *              clock (fpsnr_server_now); 0 means at submission.  Latency is
 *              measured from arrival_us when it is set (a request submitted
 *              after its arrival time counts the lateness), else from
 *              submission.
 * Buffers stay owned by the caller and must stay valid until the request
 * completes. */
typedef struct {
    int kind;
    int ndim;
    uint64_t dims[3];
    double target_psnr_db;
    fpsnr_opts opts;
    const void* d_in;
    uint64_t in_bytes;
    void* d_out;
    uint64_t out_cap;
    double arrival_us;
} fpsnr_request;

/* status       FPSNR_OK or the request's error (launch errors, or the device
 *              status the compression / decompression reported)
 * out_bytes    compress: blob size
 * stats        compress: the field's fpsnr_stats
 * arrival_us, start_us, done_us   server clock: admitted arrival, launch
 *              enqueued, completion observed by the worker */
typedef struct {
    int status;
    uint64_t out_bytes;
    fpsnr_stats stats;
    double arrival_us, start_us, done_us;
} fpsnr_result;

/* completed / failed   requests finished since creation (failed: status != 0)
 * batches              launches (each one batched compress or decompress call)
 * p50_us, p99_us, max_us   latency (done - arrival) over completed requests
 * plans, plan_bytes    plans cached now and the device memory they hold
 * bytes_in             original field bytes of completed requests
 * plans_created        plans allocated since creation (a request that waits
 *                      for room allocates nothing until its plan fits) */
typedef struct {
    uint64_t completed, failed, batches;
    double p50_us, p99_us, max_us;
    uint64_t plans, plan_bytes;
    uint64_t bytes_in;
    uint64_t plans_created;
} fpsnr_server_stats;

/* Creates a server on the current device (its worker thread starts at once).
 * Returns FPSNR_OK, FPSNR_EINVAL, FPSNR_ENOMEM or FPSNR_ECUDA. */
int fpsnr_server_create(const fpsnr_server_opts* opts, fpsnr_server_t* out);
/* Queues a request; *ticket identifies it.  Thread-safe; never blocks on the
 * GPU.  Returns FPSNR_OK or FPSNR_EINVAL (bad shape, options or alignment). */
int fpsnr_server_submit(fpsnr_server_t s, const fpsnr_request* r, uint64_t* ticket);
/* Result of a completed request (each result can be taken once): FPSNR_OK with
 * *res filled, FPSNR_EAGAIN if it is still pending, FPSNR_EINVAL for a ticket
 * never issued or already taken. */
int fpsnr_server_poll(fpsnr_server_t s, uint64_t ticket, fpsnr_result* res);
/* The oldest completed result not yet taken, in completion order: FPSNR_OK
 * with *ticket and *res filled, or FPSNR_EAGAIN when none is waiting. */
int fpsnr_server_take_any(fpsnr_server_t s, uint64_t* ticket, fpsnr_result* res);
/* Blocks until the request completes or timeout_s elapses (FPSNR_ETIMEOUT). */
int fpsnr_server_wait(fpsnr_server_t s, uint64_t ticket, fpsnr_result* res, double timeout_s);
/* Blocks until every submitted request has completed. */
int fpsnr_server_drain(fpsnr_server_t s, double timeout_s);
int fpsnr_server_get_stats(fpsnr_server_t s, fpsnr_server_stats* st);
/* Microseconds since the server was created (its clock for arrival times). */
double fpsnr_server_now(fpsnr_server_t s);
/* Completes every queued request, then frees the plans, streams and thread. */
void fpsnr_server_destroy(fpsnr_server_t s);

/* Device pointer to the uint16 symbol array (n entries) the last
 * fpsnr_compress on this plan produced; valid until the next call on the plan.
 * For inspection and tests. */
const uint16_t* fpsnr_plan_codes(fpsnr_plan_t plan);

/* Stage profiler.  The library's kernels are grouped into FPSNR_NSTAGES
 * stages (fpsnr_stage_name gives each name).  Kernel launches per stage are
 * always counted on the host (a stage call can launch several kernels).  With
 * fpsnr_plan_profile(plan, 1) every stage call is also bracketed by CUDA
 * events on its stream; fpsnr_plan_profile_read synchronizes those events,
 * adds each stage's total milliseconds and kernel launch count since the last
 * read into ms[i] and launches[i] (arrays of nstages entries, either may be
 * NULL), and resets the counters.  Recording adds one event pair per stage
 * call; it does not change what the kernels compute.
 * Returns FPSNR_OK, FPSNR_EINVAL or FPSNR_ECUDA. */
#define FPSNR_NSTAGES 18
int fpsnr_plan_profile(fpsnr_plan_t plan, int enable);
int fpsnr_plan_profile_read(fpsnr_plan_t plan, double* ms, uint64_t* launches, int nstages);
const char* fpsnr_stage_name(int stage);

/* Release the plan and its device scratch (synchronizes the device first). */
void fpsnr_plan_destroy(fpsnr_plan_t plan);

/* Static string for an FPSNR_* code. */
const char* fpsnr_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* FPSNR_H */
