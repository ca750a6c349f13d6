// api.cu -- C ABI entry points: plan creation (validation, launch geometry,
// device scratch), compress / decompress dispatch, error strings.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "common.cuh"
#include "plan.cuh"

namespace {

using fp::PQGeom;
using fp::ScanPass;

bool psnr_ok(double t) { return t > 0.0 && t <= FPSNR_MAX_PSNR; }

double eb_rel_of(double psnr) { return sqrt(3.0) * pow(10.0, -psnr / 20.0); }  // Eq. 8

uint64_t cdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// Carves a slab into 256-byte aligned arrays; first pass only measures.
struct Carver {
    uint8_t* base;
    size_t off = 0;
    template <class T>
    T* take(uint64_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += (size_t)count * sizeof(T);
        return p;
    }
};

void carve(fpsnr_plan_s* p, uint8_t* base, size_t* total) {
    Carver c{base};
    fp::Workspace& w = p->w;
    const uint64_t n = std::max<uint64_t>(p->n, 1);
    w.par = c.take<fp::DevParams>(1);
    w.hist = c.take<uint32_t>(p->nsym);
    w.enc = c.take<uint32_t>(p->nsym);
    w.len_sym = c.take<uint8_t>(p->nsym);
    w.codes = c.take<uint16_t>(n + 8);
    w.chunk_off = c.take<uint32_t>(std::max<uint64_t>(p->nchunks, 1));
    w.stage_out = c.take<uint2>(n);
    w.stage_vb = c.take<uint2>(n);
    w.bm = c.take<uint32_t>(2 * std::max<uint64_t>(p->nwords, 1));
    w.wpre = c.take<uint32_t>(2 * std::max<uint64_t>(p->nwords, 1));
    w.bpre = c.take<uint32_t>(2 * std::max<uint64_t>(p->nbmblk, 1));
    w.sse_part = c.take<double>(std::max<uint32_t>(p->pq_blocks_cap, 1));
    w.range_part = c.take<float>(3 * (uint64_t)p->n_range_blocks);
    w.hlist = c.take<unsigned long long>(p->nsym);
    w.hbuf1 = c.take<unsigned long long>(p->nsym);
    w.hbuf2 = c.take<unsigned long long>(p->nsym);
    w.hpar = c.take<uint32_t>(2ull * p->nsym);
    w.dlut = c.take<uint32_t>(1u << fp::kLutBits);
    w.dsyms = c.take<uint16_t>(fp::kMaxSym);
    w.lb_flags = c.take<uint32_t>(std::max<uint64_t>(p->lb_tiles_total, 1));
    w.lb_vals = c.take<uint32_t>(2 * std::max<uint64_t>(p->lb_tiles_total, 1) * p->lb_width);
    w.lb_ctr = c.take<uint32_t>(8);
    w.enc_tiles = c.take<uint32_t>(std::max<uint64_t>(p->enc_tiles, 1));
    w.enc_scratch = c.take<uint32_t>(std::max<uint64_t>(p->nchunks * p->enc_slot_words, 1));
    w.bsum = c.take<uint32_t>(p->band.on ? (uint64_t)p->band_cap * p->band.nx : 1);
    const fp::VolGeom& v = p->vol;
    w.vcb = c.take<uint32_t>(v.on ? (uint64_t)v.nz * v.nbands * v.nx : 1);
    w.vds = c.take<uint32_t>(v.on ? (uint64_t)v.nslabs * v.ny * v.nx : 1);
    w.vts = c.take<uint32_t>(v.on ? (uint64_t)v.nslabs * v.nbands * v.nx : 1);
    w.fine_hist = c.take<uint32_t>(fp::kFineBins);
    w.zr_scratch = c.take<uint8_t>(p->lossless ? p->zr_scratch_cap : 16);
    w.zr_seg = c.take<uint32_t>(p->lossless ? p->zr_seg_cap : 1);
    *total = (c.off + 255) & ~(size_t)255;
}

// Predictor geometry.  2D fields take a tile width tx of 128, 256 or 512 points
// (0: by row length); each block walks max(4, 8192 / tx) rows.  Returns false if
// the grid would be too large.
bool pq_geometry(fpsnr_plan_s* p, int tx) {
    const uint64_t* d = p->dims;
    const uint64_t n = p->n;
    PQGeom& g = p->pq;
    if (p->ld == 1) {
        g.mode = 1; g.tx = 1024; g.ty = 1; g.zs = 16;
        g.vx = 1024; g.vy = 1; g.vz = (uint32_t)std::max<uint64_t>(cdiv(n, 1024), 1);
    } else if (p->ld == 2) {
        const uint64_t nx = d[0], rows = nx ? n / nx : 0;
        g.mode = 2; g.ty = 1;
        g.tx = tx ? tx : (nx <= 128 ? 128 : (nx <= 256 ? 256 : (nx <= 512 ? 512 : 1024)));
        g.zs = std::max(64, 32768 / g.tx);  // rows per block: one warm-up row each
        g.vx = (uint32_t)nx; g.vy = 1; g.vz = (uint32_t)rows;
    } else {
        // slabs of 64 planes: a block re-derives one plane above its slab
        g.mode = 3; g.tx = 128; g.ty = 8; g.zs = 64;
        g.vx = (uint32_t)d[0]; g.vy = (uint32_t)d[1]; g.vz = (uint32_t)d[2];
    }
    g.vec = (g.vx % 4) == 0;
    g.nbx = g.nby = g.nbz = g.nblocks = 0;
    if (n > 0) {
        g.nbx = (uint32_t)cdiv(g.vx, g.tx);
        g.nby = (uint32_t)cdiv(g.vy, g.ty);
        g.nbz = (uint32_t)cdiv(g.vz, g.zs);
        const uint64_t nb = (uint64_t)g.nbx * g.nby * g.nbz;
        if (nb > 0x7FFFFFFFull) return false;
        g.nblocks = (uint32_t)nb;
    }
    return true;
}

// 2D inverse-Lorenzo band height (16, 32 or 64 rows).
void band_rows(fpsnr_plan_s* p, uint32_t tr) {
    p->band.tr = tr;
    p->band.nbands = (uint32_t)cdiv(p->band.rows, tr);
}

ScanPass contig_pass(uint64_t rows, uint64_t W, bool final_pass) {
    ScanPass s{};
    s.kind = 0;
    s.A = (uint32_t)rows;
    s.L = (uint32_t)W;
    s.B = 1;
    s.ipt = W <= 1024 ? 4 : (W <= 2048 ? 8 : 16);
    s.tiles = (uint32_t)(rows * cdiv(W, 256ull * s.ipt));
    s.tb = 1;
    s.vec = (W % 4) == 0;
    s.vec16 = rows == 1 || (W % 8) == 0;
    s.final_pass = final_pass;
    return s;
}

ScanPass strided_pass(uint64_t A, uint64_t L, uint64_t B, bool final_pass) {
    ScanPass s{};
    s.kind = 1;
    s.A = (uint32_t)A;
    s.L = (uint32_t)L;
    s.B = (uint32_t)B;
    s.vec = (B % 4) == 0;
    s.tb = s.vec ? 1024 : 256;
    s.ipt = 16;
    s.tiles = (uint32_t)(cdiv(L, 16) * A * cdiv(B, (uint64_t)s.tb));
    s.final_pass = final_pass;
    return s;
}

// Runs `fn` with the plans' device current (all plans of one call share it).
template <class F>
int on_device(int device, F fn) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return FPSNR_ECUDA;
    if (cur != device && cudaSetDevice(device) != cudaSuccess) return FPSNR_ECUDA;
    int rc = fn();
    if (cur != device) cudaSetDevice(cur);
    return rc;
}

}  // namespace

namespace fp {

cudaEvent_t Profiler::take() {
    if (used == npool) {
        size_t nn = npool ? 2 * npool : 256;
        cudaEvent_t* np_ = static_cast<cudaEvent_t*>(realloc(pool, nn * sizeof(cudaEvent_t)));
        if (!np_) return nullptr;
        pool = np_;
        for (size_t i = npool; i < nn; i++)
            if (cudaEventCreate(&pool[i]) != cudaSuccess) { nn = i; break; }
        npool = nn;
        if (used == npool) return nullptr;
    }
    return pool[used++];
}

void Profiler::begin(int stage, cudaStream_t st, cudaEvent_t* a) {
    launches[stage]++;
    *a = nullptr;
    if (!on) return;
    *a = take();
    if (*a) cudaEventRecord(*a, st);
}

void Profiler::end(int stage, cudaStream_t st, cudaEvent_t a) {
    if (!on || !a) return;
    cudaEvent_t b = take();
    if (!b) return;
    cudaEventRecord(b, st);
    if (nrec == cap) {
        size_t nc = cap ? 2 * cap : 256;
        Rec* nr = static_cast<Rec*>(realloc(recs, nc * sizeof(Rec)));
        if (!nr) return;
        recs = nr;
        cap = nc;
    }
    recs[nrec++] = Rec{stage, a, b};
}

void Profiler::release() {
    for (size_t i = 0; i < npool; i++) cudaEventDestroy(pool[i]);
    free(pool);
    free(recs);
    pool = nullptr;
    recs = nullptr;
    npool = used = nrec = cap = 0;
}

}  // namespace fp

extern "C" {

static const char* kStageNames[FPSNR_NSTAGES] = {
    "range_plan", "predict_quantize", "rank_popc", "codebook", "band_sum", "band_carry",
    "encode", "emit", "finalize", "decode_setup", "decode", "eb_refine", "scan_x", "scan_y",
    "scan_final_dequant", "patch", "lossless_wrap", "lossless_unwrap"};

const char* fpsnr_stage_name(int stage) {
    return (stage >= 0 && stage < FPSNR_NSTAGES) ? kStageNames[stage] : "unknown";
}

int fpsnr_plan_profile(fpsnr_plan_t p, int enable) {
    if (!p) return FPSNR_EINVAL;
    p->prof.on = enable != 0;
    return FPSNR_OK;
}

int fpsnr_plan_profile_read(fpsnr_plan_t p, double* ms, uint64_t* launches, int nstages) {
    if (!p || nstages < 0) return FPSNR_EINVAL;
    fp::Profiler& pr = p->prof;
    int rc = FPSNR_OK;
    for (int i = 0; i < nstages && i < FPSNR_NSTAGES; i++) {
        if (ms) ms[i] = 0.0;
        if (launches) launches[i] = pr.launches[i];
    }
    for (size_t r = 0; r < pr.nrec; r++) {
        float t = 0.0f;
        if (cudaEventSynchronize(pr.recs[r].b) != cudaSuccess ||
            cudaEventElapsedTime(&t, pr.recs[r].a, pr.recs[r].b) != cudaSuccess) {
            rc = FPSNR_ECUDA;
            continue;
        }
        if (ms && pr.recs[r].stage < nstages) ms[pr.recs[r].stage] += t;
    }
    pr.nrec = 0;
    pr.used = 0;
    for (int i = 0; i < FPSNR_NSTAGES; i++) pr.launches[i] = 0;
    return rc;
}

int fpsnr_default_opts(fpsnr_opts* o) {
    if (!o) return FPSNR_EINVAL;
    o->radius = 32768;
    o->chunk = 256;
    o->lmax = 27;
    o->lorenzo_dims = 0;
    o->psnr_mode = 0;
    o->lossless = 0;
    return FPSNR_OK;
}

const char* fpsnr_strerror(int code) {
    switch (code) {
        case FPSNR_OK: return "ok";
        case FPSNR_EINVAL: return "invalid argument";
        case FPSNR_ENOMEM: return "device memory allocation failed";
        case FPSNR_ECUDA: return "CUDA error";
        case FPSNR_ENONFINITE: return "input contains NaN or Inf";
        case FPSNR_ECAPACITY: return "output buffer too small";
        case FPSNR_ECORRUPT: return "compressed stream is corrupt or does not match the plan";
        case FPSNR_ETIMEOUT: return "inter-block wait timed out";
        case FPSNR_EAGAIN: return "request not completed yet";
        default: return "unknown error";
    }
}

int fpsnr_plan(fpsnr_plan_t* out, int ndim, const uint64_t* dims, double target_psnr_db,
               const fpsnr_opts* opts) {
    if (!out) return FPSNR_EINVAL;
    *out = nullptr;
    fpsnr_plan_s* p = nullptr;
    int rc = fp::plan_layout(&p, ndim, dims, target_psnr_db, opts);
    if (rc != FPSNR_OK) return rc;
    rc = fp::plan_allocate(p);
    if (rc != FPSNR_OK) return rc;
    *out = p;
    return FPSNR_OK;
}

}  // extern "C"

namespace fp {

int plan_layout(fpsnr_plan_s** out, int ndim, const uint64_t* dims, double target_psnr_db,
                const fpsnr_opts* opts) {
    *out = nullptr;
    if (ndim < 1 || ndim > 3 || !dims || !psnr_ok(target_psnr_db)) return FPSNR_EINVAL;
    fpsnr_opts o;
    fpsnr_default_opts(&o);
    if (opts) o = *opts;
    const int ld = o.lorenzo_dims ? o.lorenzo_dims : ndim;
    if (ld < 1 || ld > ndim) return FPSNR_EINVAL;
    if (o.radius < 1 || o.radius > fp::kMaxRadius) return FPSNR_EINVAL;
    if (o.chunk < 32 || o.chunk > 65536 || (o.chunk % 32) != 0) return FPSNR_EINVAL;
    if (o.lmax < 1 || o.lmax > fp::kMaxLmax || (1ull << o.lmax) < 2ull * o.radius) return FPSNR_EINVAL;
    if (o.psnr_mode != 0 && o.psnr_mode != 1) return FPSNR_EINVAL;
    if (o.lossless != 0 && o.lossless != 1) return FPSNR_EINVAL;
    uint64_t d[3] = {1, 1, 1};
    uint64_t n = 1;
    for (int i = 0; i < ndim; i++) {
        d[i] = dims[i];
        if (d[i] > 0xFFFFFFFFull) return FPSNR_EINVAL;
        n *= d[i];
        if (n > 0xFFFFFFFFull) return FPSNR_EINVAL;
    }
    fpsnr_plan_s* p = new (std::nothrow) fpsnr_plan_s();
    if (!p) return FPSNR_ENOMEM;
    p->ndim = ndim;
    p->ld = ld;
    memcpy(p->dims, d, sizeof(d));
    p->n = n;
    p->target_psnr = target_psnr_db;
    p->eb_rel = eb_rel_of(target_psnr_db);
    p->mse_rel = pow(10.0, -target_psnr_db / 10.0);
    p->psnr_mode = o.psnr_mode;
    p->lossless = o.lossless;
    p->spin_limit = fp::kSpinLimit;
    p->wait_skew = 0;
    p->radius = o.radius;
    p->chunk = o.chunk;
    p->lmax = o.lmax;
    p->nsym = 2u * (uint32_t)o.radius;
    p->nchunks = cdiv(n, (uint64_t)o.chunk);
    p->nwords = cdiv(n, 32);
    p->nbmblk = cdiv(p->nwords, 1024);
    p->enc_tiles = cdiv(p->nchunks, fp::kEncTile);
    p->enc_slot_words = (uint32_t)cdiv((uint64_t)p->chunk * (uint64_t)p->lmax, 32);
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
        delete p;
        return FPSNR_ECUDA;
    }

    // predictor geometry; the workspace holds partials for any 2D tile width
    if (!pq_geometry(p, 0)) { delete p; return FPSNR_EINVAL; }
    p->pq_blocks_cap = p->pq.nblocks;
    if (ld == 2 && n > 0) {
        const int tx0 = p->pq.tx;
        for (int tx : {128, 256, 512, 1024}) {
            if (!pq_geometry(p, tx)) { delete p; return FPSNR_EINVAL; }
            p->pq_blocks_cap = std::max(p->pq_blocks_cap, p->pq.nblocks);
        }
        pq_geometry(p, tx0);
    }
    p->n_range_blocks = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(cdiv(n, 512ull * 16),
                                                                            2ull * p->sm_count));

    // inverse-Lorenzo passes
    p->n_passes = 0;
    p->band = fp::BandGeom{};
    p->vol = fp::VolGeom{};
    if (n > 0) {
        if (ld == 1) {
            p->pass[p->n_passes++] = contig_pass(1, n, true);
        } else if (ld == 2 && d[0] <= fp::kBandMaxNx) {
            const uint64_t nx = d[0], rows = n / nx;
            fp::BandGeom& b = p->band;
            b.on = true;
            b.nx = (uint32_t)nx;
            b.rows = (uint32_t)rows;
            band_rows(p, fp::kBandRows);
            p->band_cap = (uint32_t)cdiv(rows, 16);
            b.g = nx <= 2048 ? 1 : (nx <= 4096 ? 2 : 4);
            b.vec = (nx % 8) == 0;
        } else if (ld == 2) {
            const uint64_t nx = d[0], rows = n / nx;
            p->pass[p->n_passes++] = contig_pass(rows, nx, false);
            p->pass[p->n_passes++] = strided_pass(1, rows, nx, true);
        } else if (d[0] <= fp::kVolMaxNx) {
            fp::VolGeom& v = p->vol;
            v.on = true;
            v.nx = (uint32_t)d[0];
            v.ny = (uint32_t)d[1];
            v.nz = (uint32_t)(n / (d[0] * d[1]));
            v.cpl = v.nx <= 128 ? 4 : (v.nx <= 256 ? 8 : 16);
            v.wpr = v.nx <= 512 ? 1 : (v.nx <= 1024 ? 2 : 4);
            v.ty = 16u / (uint32_t)v.wpr;
            v.tz = fp::kVolSlab;
            v.nbands = (uint32_t)cdiv(v.ny, v.ty);
            v.nslabs = (uint32_t)cdiv(v.nz, v.tz);
            v.vec = (v.nx % 4u) == 0;
        } else {
            p->pass[p->n_passes++] = contig_pass(d[2] * d[1], d[0], false);
            p->pass[p->n_passes++] = strided_pass(d[2], d[1], d[0], false);
            p->pass[p->n_passes++] = strided_pass(1, d[2], d[1] * d[0], true);
        }
    }
    p->lb_tiles_total = 0;
    p->lb_width = 1;
    for (int i = 0; i < p->n_passes; i++) {
        p->pass[i].val_off = p->lb_tiles_total;
        p->pass[i].ctr_slot = i;
        p->lb_tiles_total += p->pass[i].tiles;
        p->lb_width = std::max<uint64_t>(p->lb_width, (uint64_t)p->pass[i].tb);
    }

    if (p->lossless) {
        p->zr_scratch_cap = (fpsnr_max_compressed_bytes(p) + 15) & ~(uint64_t)15;
        p->zr_seg_cap = cdiv(p->zr_scratch_cap, fp::kZrSeg) + 1;
    }
    size_t bytes = 0;
    carve(p, nullptr, &bytes);
    p->slab_bytes = bytes;
    *out = p;
    return FPSNR_OK;
}

int plan_allocate(fpsnr_plan_s* p) {
    size_t bytes = p->slab_bytes;
    void* slab = nullptr;
    if (cudaMalloc(&slab, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return FPSNR_ENOMEM;
    }
    p->slab = slab;
    carve(p, reinterpret_cast<uint8_t*>(slab), &bytes);
    const fp::Workspace& w = p->w;
    bool ok = cudaMemset(w.par, 0, sizeof(fp::DevParams)) == cudaSuccess &&
              cudaMemset(w.bm, 0, 2 * std::max<uint64_t>(p->nwords, 1) * 4) == cudaSuccess &&
              cudaMemset(w.lb_flags, 0, std::max<uint64_t>(p->lb_tiles_total, 1) * 4) == cudaSuccess &&
              cudaMemset(w.lb_ctr, 0, 8 * 4) == cudaSuccess &&
              cudaMemset(w.fine_hist, 0, fp::kFineBins * 4) == cudaSuccess &&

              fp::codebook_prepare() == FPSNR_OK && fp::decode_prepare(p) == FPSNR_OK &&
              cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
        cudaFree(slab);
        delete p;
        return FPSNR_ECUDA;
    }
    p->cb_smem = fp::codebook_smem_bytes();
    return FPSNR_OK;
}

}  // namespace fp

extern "C" {

int fpsnr_plan_set_psnr(fpsnr_plan_t p, double target_psnr_db) {
    if (!p || !psnr_ok(target_psnr_db)) return FPSNR_EINVAL;
    p->target_psnr = target_psnr_db;
    p->eb_rel = eb_rel_of(target_psnr_db);
    p->mse_rel = pow(10.0, -target_psnr_db / 10.0);
    return FPSNR_OK;
}

double fpsnr_plan_eb_rel(fpsnr_plan_t p) { return p ? p->eb_rel : NAN; }

uint64_t fpsnr_plan_points(fpsnr_plan_t p) { return p ? p->n : 0; }

uint64_t fpsnr_max_compressed_bytes(fpsnr_plan_t p) {
    if (!p) return 0;
    auto pad = [](uint64_t b) { return (b + 15u) & ~(uint64_t)15u; };
    const uint64_t words = cdiv(p->n * (uint64_t)p->lmax, 32) + p->nchunks;
    return fp::kHeaderBytes + pad(4ull * p->nsym) + pad(4ull * p->nchunks) + pad(4ull * words) +
           pad(8ull * p->n) + pad(8ull * p->n);
}

int fpsnr_compress(fpsnr_plan_t p, const float* d_in, void* d_out, uint64_t out_cap,
                   uint64_t* d_out_bytes, fpsnr_stats* d_stats, void* stream) {
    return fpsnr_compress_batch(&p, &d_in, &d_out, &out_cap, d_out_bytes, d_stats, 1, stream);
}

int fpsnr_compress_batch(const fpsnr_plan_t* plans, const float* const* d_in, void* const* d_out,
                         const uint64_t* out_cap, uint64_t* d_out_bytes, fpsnr_stats* d_stats,
                         int count, void* stream) {
    if (count < 0 || (count > 0 && (!plans || !d_in || !d_out || !out_cap))) return FPSNR_EINVAL;
    if (count == 0) return FPSNR_OK;
    for (int i = 0; i < count; i++) {
        const fpsnr_plan_s* p = plans[i];
        if (!p || !d_out[i] || (p->n > 0 && !d_in[i])) return FPSNR_EINVAL;
        if (((uintptr_t)d_in[i] & 3u) || ((uintptr_t)d_out[i] & 15u)) return FPSNR_EINVAL;
        if (p->device != plans[0]->device) return FPSNR_EINVAL;
        for (int j = 0; j < i; j++)
            if (plans[j] == p) return FPSNR_EINVAL;  // a plan's scratch serves one field at a time
    }
    return on_device(plans[0]->device, [&] {
        return fp::launch_compress_batch(const_cast<fpsnr_plan_s* const*>(plans), d_in, d_out, out_cap,
                                         d_out_bytes, d_stats, count,
                                         reinterpret_cast<cudaStream_t>(stream));
    });
}

int fpsnr_decompress(fpsnr_plan_t p, const void* d_blob, uint64_t blob_bytes, float* d_out,
                     uint64_t n_out, int* d_status, void* stream) {
    if (!p || n_out != p->n) return FPSNR_EINVAL;
    return fpsnr_decompress_batch(&p, &d_blob, &blob_bytes, &d_out, d_status, 1, stream);
}

int fpsnr_decompress_batch(const fpsnr_plan_t* plans, const void* const* d_blob,
                           const uint64_t* blob_bytes, float* const* d_out, int* d_status,
                           int count, void* stream) {
    if (count < 0 || (count > 0 && (!plans || !d_blob || !blob_bytes || !d_out))) return FPSNR_EINVAL;
    if (count == 0) return FPSNR_OK;
    for (int i = 0; i < count; i++) {
        const fpsnr_plan_s* p = plans[i];
        if (!p || !d_blob[i] || (p->n > 0 && !d_out[i])) return FPSNR_EINVAL;
        if (((uintptr_t)d_blob[i] & 15u) || ((uintptr_t)d_out[i] & 15u)) return FPSNR_EINVAL;
        if (p->device != plans[0]->device) return FPSNR_EINVAL;
        for (int j = 0; j < i; j++)
            if (plans[j] == p) return FPSNR_EINVAL;
    }
    return on_device(plans[0]->device, [&] {
        return fp::launch_decompress_batch(const_cast<fpsnr_plan_s* const*>(plans), d_blob, blob_bytes,
                                           d_out, d_status, count,
                                           reinterpret_cast<cudaStream_t>(stream));
    });
}

int fpsnr_plan_set_tuning(fpsnr_plan_t p, const fpsnr_tuning* t) {
    if (!p || !t) return FPSNR_EINVAL;
    if (t->chunk != 0 && t->chunk != p->chunk) return FPSNR_EINVAL;
    const int tx = t->pq_tile_x, tr = t->band_rows, dt = t->dec_threads;
    if (tx != 0 && (tx != 128 && tx != 256 && tx != 512 && tx != 1024)) return FPSNR_EINVAL;
    if (tx != 0 && p->ld != 2) return FPSNR_EINVAL;
    if (tr != 0 && (tr != 16 && tr != 32 && tr != 64)) return FPSNR_EINVAL;
    if (tr != 0 && !p->band.on) return FPSNR_EINVAL;
    if (dt != 0 && dt != 128 && dt != 256 && dt != 512) return FPSNR_EINVAL;
    if (p->ld == 2 && p->n > 0) {
        const int keep = p->pq.tx;
        if (!pq_geometry(p, tx) || p->pq.nblocks > p->pq_blocks_cap) {
            pq_geometry(p, keep);
            return FPSNR_EINVAL;
        }
    }
    if (p->band.on) band_rows(p, tr ? (uint32_t)tr : fp::kBandRows);
    p->dec_threads = dt;
    return FPSNR_OK;
}

int fpsnr_plan_set_wait_limit(fpsnr_plan_t p, uint32_t spins, int test_unmet) {
    if (!p || (test_unmet != 0 && test_unmet != 1)) return FPSNR_EINVAL;
    p->spin_limit = spins ? spins : fp::kSpinLimit;
    p->wait_skew = (uint32_t)test_unmet;
    return FPSNR_OK;
}

int fpsnr_plan_get_tuning(fpsnr_plan_t p, fpsnr_tuning* t) {
    if (!p || !t) return FPSNR_EINVAL;
    memset(t, 0, sizeof(*t));
    t->chunk = p->chunk;
    t->pq_tile_x = p->ld == 2 ? p->pq.tx : 0;
    t->band_rows = p->band.on ? (int)p->band.tr : 0;
    t->dec_threads = p->dec_threads;
    return FPSNR_OK;
}

// ---- reading a blob's header (host) ----

static uint32_t rd_u32(const uint8_t* b) {
    return (uint32_t)b[0] | ((uint32_t)b[1] << 8) | ((uint32_t)b[2] << 16) | ((uint32_t)b[3] << 24);
}
static uint64_t rd_u64(const uint8_t* b) { return (uint64_t)rd_u32(b) | ((uint64_t)rd_u32(b + 4) << 32); }
static double rd_f64(const uint8_t* b) {
    double v;
    memcpy(&v, b, 8);
    return v;
}
static float rd_f32(const uint8_t* b) {
    float v;
    memcpy(&v, b, 4);
    return v;
}

// Copies `bytes` bytes at offset `off` of the caller's blob (device or host
// memory) to the host and waits for them.
static int blob_read(const void* blob, uint64_t off, void* dst, uint64_t bytes, cudaStream_t st) {
    if (cudaMemcpyAsync(dst, static_cast<const uint8_t*>(blob) + off, bytes, cudaMemcpyDefault, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return FPSNR_ECUDA;
    }
    return FPSNR_OK;
}

// Header fields of a plain blob (kHeaderBytes bytes); FPSNR_ECORRUPT unless
// they describe a field this library can plan.
static int parse_header(const uint8_t* h, fpsnr_blob_header* info) {
    if (rd_u32(h) != fp::kMagic || rd_u32(h + 4) != fp::kVersion) return FPSNR_ECORRUPT;
    info->ndim = (int)rd_u32(h + 8);
    info->lorenzo_dims = (int)rd_u32(h + 12);
    uint64_t n = 1;
    for (int i = 0; i < 3; i++) info->dims[i] = rd_u64(h + 16 + 8 * i);
    if (info->ndim < 1 || info->ndim > 3 || info->lorenzo_dims < 1 || info->lorenzo_dims > info->ndim)
        return FPSNR_ECORRUPT;
    for (int i = 0; i < 3; i++) {
        if (i >= info->ndim && info->dims[i] != 1) return FPSNR_ECORRUPT;
        if (info->dims[i] > 0xFFFFFFFFull) return FPSNR_ECORRUPT;
        n *= info->dims[i];
        if (n > 0xFFFFFFFFull) return FPSNR_ECORRUPT;
    }
    info->target_psnr = rd_f64(h + 40);
    info->eb_rel = rd_f64(h + 48);
    info->eb_abs = rd_f64(h + 56);
    info->vr = rd_f64(h + 64);
    info->xmin = rd_f32(h + 72);
    info->xmax = rd_f32(h + 76);
    info->flags = rd_u32(h + 92);
    info->radius = (int)rd_u32(h + 96);
    info->chunk = (int)rd_u32(h + 100);
    info->lmax = (int)rd_u32(h + 104);
    info->n_outlier = rd_u32(h + 120);
    info->n_verbatim = rd_u32(h + 124);
    info->points = n;
    auto pad = [](uint64_t b) { return (b + 15u) & ~(uint64_t)15u; };
    info->raw_bytes = fp::kHeaderBytes;
    if (!(info->flags & fp::kFlagConstant))
        info->raw_bytes += pad(4ull * rd_u32(h + 108)) + pad(4ull * rd_u32(h + 112)) +
                           pad(4ull * rd_u32(h + 116)) + pad(8ull * rd_u32(h + 120)) +
                           pad(8ull * rd_u32(h + 124));
    if ((info->flags & ~3u) != 0 || !psnr_ok(info->target_psnr) || info->radius < 1 ||
        info->radius > fp::kMaxRadius || info->chunk < 32 || info->chunk > 65536 ||
        (info->chunk % 32) != 0 || info->lmax < 1 || info->lmax > fp::kMaxLmax ||
        (1ull << info->lmax) < 2ull * (uint64_t)info->radius)
        return FPSNR_ECORRUPT;
    return FPSNR_OK;
}

int fpsnr_blob_info(const void* blob, uint64_t blob_bytes, fpsnr_blob_header* info, void* stream) {
    if (!blob || !info) return FPSNR_EINVAL;
    memset(info, 0, sizeof(*info));
    if (blob_bytes < 32) return FPSNR_ECORRUPT;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint8_t head[fp::kHeaderBytes];
    const uint64_t first = std::min<uint64_t>(blob_bytes, fp::kHeaderBytes);
    int rc = blob_read(blob, 0, head, first, st);
    if (rc) return rc;
    if (rd_u32(head) != fp::kZrMagic) {
        if (blob_bytes < fp::kHeaderBytes) return FPSNR_ECORRUPT;
        rc = parse_header(head, info);
        if (rc) return rc;
        return info->raw_bytes <= blob_bytes ? FPSNR_OK : FPSNR_ECORRUPT;
    }
    // lossless container: expand its first segment, which holds the header
    const uint64_t raw = rd_u64(head + 8);
    const uint64_t nseg = rd_u32(head + 20);
    const uint64_t dstart = 32 + ((4 * (nseg + 1) + 15) & ~(uint64_t)15);
    if (rd_u32(head + 4) != 1u || rd_u32(head + 16) != fp::kZrSeg || raw < fp::kHeaderBytes ||
        nseg != (raw + fp::kZrSeg - 1) / fp::kZrSeg || dstart > blob_bytes)
        return FPSNR_ECORRUPT;
    uint8_t offs[8];
    if ((rc = blob_read(blob, 32, offs, 8, st))) return rc;
    const uint32_t e0 = rd_u32(offs), e1 = rd_u32(offs + 4);
    const uint64_t lo = e0 & 0x7FFFFFFFu, hi = e1 & 0x7FFFFFFFu;
    const uint32_t len = (uint32_t)std::min<uint64_t>(fp::kZrSeg, raw);
    if (lo > hi || hi - lo > fp::kZrSeg || dstart + hi > blob_bytes) return FPSNR_ECORRUPT;
    uint8_t code[fp::kZrSeg], seg[fp::kZrSeg];
    if (hi > lo && (rc = blob_read(blob, dstart + lo, code, hi - lo, st))) return rc;
    const uint64_t clen = hi - lo;
    if (e0 & 0x80000000u) {
        if (clen != len) return FPSNR_ECORRUPT;
        memcpy(seg, code, len);
    } else {
        // a nonzero byte stands for itself; 0x00 and LEB128 k - 1 for k zeros
        uint64_t i = 0;
        uint32_t w = 0;
        while (i < clen) {
            const uint8_t v = code[i++];
            if (v) {
                if (w >= len) return FPSNR_ECORRUPT;
                seg[w++] = v;
                continue;
            }
            uint32_t k = 0;
            for (int sh = 0;; sh += 7) {
                if (i >= clen || sh > 28) return FPSNR_ECORRUPT;
                const uint8_t t = code[i++];
                k |= (uint32_t)(t & 127u) << sh;
                if (!(t & 128u)) break;
            }
            if ((uint64_t)w + k + 1 > len) return FPSNR_ECORRUPT;
            memset(seg + w, 0, k + 1);
            w += k + 1;
        }
        if (w != len) return FPSNR_ECORRUPT;
    }
    rc = parse_header(seg, info);
    if (rc) return rc;
    info->lossless = 1;
    return info->raw_bytes == raw ? FPSNR_OK : FPSNR_ECORRUPT;
}

int fpsnr_plan_from_blob(fpsnr_plan_t* out, const fpsnr_blob_header* info) {
    if (!out || !info) return FPSNR_EINVAL;
    *out = nullptr;
    fpsnr_opts o;
    fpsnr_default_opts(&o);
    o.radius = info->radius;
    o.chunk = info->chunk;
    o.lmax = info->lmax;
    o.lorenzo_dims = info->lorenzo_dims;
    o.lossless = info->lossless ? 1 : 0;
    return fpsnr_plan(out, info->ndim, info->dims, info->target_psnr, &o);
}

const uint16_t* fpsnr_plan_codes(fpsnr_plan_t p) { return p ? p->w.codes : nullptr; }

void fpsnr_plan_destroy(fpsnr_plan_t p) {
    if (!p) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    p->prof.release();
    cudaFree(p->slab);
    if (cur != p->device && cur >= 0) cudaSetDevice(cur);
    delete p;
}

}  // extern "C"
