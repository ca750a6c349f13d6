// tune.cu -- autotuner for the chunk size and launch shapes (no counterpart in
// the paper, whose compressor runs on CPUs: these are the GPU decoder's
// chunking and the kernels' tile shapes).
//
// The chunk size C changes the compressed bytes (one u32 offset per chunk; C
// is a header field) and the decoder's parallelism (one thread per chunk), so
// it is chosen as the fastest C whose compressed size stays within a tolerance
// of the smallest.  Tile shapes never change the bytes and are chosen purely by
// time, one parameter at a time.  Timing is compress + decompress of a sample
// field, best of 3 runs after a warm-up, CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fpsnr.h"

namespace {

std::mutex g_mu;
std::map<std::string, fpsnr_tuning> g_cache;

struct Buffers {
    void* blob = nullptr;
    float* rec = nullptr;
    uint64_t* nbytes = nullptr;
    fpsnr_stats* stats = nullptr;
    int* status = nullptr;
    uint64_t cap = 0;
    ~Buffers() {
        cudaFree(blob);
        cudaFree(rec);
        cudaFree(nbytes);
        cudaFree(stats);
        cudaFree(status);
    }
};

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Compress + decompress of the sample: the warm-up run checks both statuses
// and gives the compressed size, then the best of `reps` timed runs.
int measure(fpsnr_plan_t p, const float* d_sample, uint64_t n, Buffers& b, Events& ev,
            cudaStream_t st, double* ms, uint64_t* bytes) {
    auto once = [&]() -> int {
        int rc = fpsnr_compress(p, d_sample, b.blob, b.cap, b.nbytes, b.stats, st);
        if (rc) return rc;
        // the blob is at most `cap` bytes; the decoder checks every section against it
        return fpsnr_decompress(p, b.blob, b.cap, b.rec, n, b.status, st);
    };
    int rc = once();
    if (rc) return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FPSNR_ECUDA;
    fpsnr_stats hs;
    int hstatus = 0;
    if (cudaMemcpy(&hs, b.stats, sizeof(hs), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&hstatus, b.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(bytes, b.nbytes, sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return FPSNR_ECUDA;
    if (hs.status) return hs.status;
    if (hstatus) return hstatus;
    double best = INFINITY;
    for (int r = 0; r < 3; r++) {
        if (cudaEventRecord(ev.a, st) != cudaSuccess) return FPSNR_ECUDA;
        rc = once();
        if (rc) return rc;
        if (cudaEventRecord(ev.b, st) != cudaSuccess || cudaEventSynchronize(ev.b) != cudaSuccess)
            return FPSNR_ECUDA;
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, ev.a, ev.b) != cudaSuccess) return FPSNR_ECUDA;
        best = std::min(best, (double)t);
    }
    *ms = best;
    return FPSNR_OK;
}

}  // namespace

extern "C" int fpsnr_autotune(int ndim, const uint64_t* dims, double target_psnr_db,
                              const fpsnr_opts* opts, const float* d_sample,
                              double max_size_increase, fpsnr_tuning* out, void* stream) {
    if (!out || !dims || !d_sample || ndim < 1 || ndim > 3 || !(max_size_increase >= 0.0) ||
        ((uintptr_t)d_sample & 3u))
        return FPSNR_EINVAL;
    fpsnr_opts o;
    fpsnr_default_opts(&o);
    if (opts) o = *opts;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FPSNR_ECUDA;
    uint64_t d[3] = {1, 1, 1}, n = 1;
    for (int i = 0; i < ndim; i++) {
        d[i] = dims[i];
        n *= d[i];
    }
    char key[256];
    snprintf(key, sizeof(key), "%d|%d|%llu,%llu,%llu|%.17g|%d,%d,%d,%d,%d,%d|%.17g", dev, ndim,
             (unsigned long long)d[0], (unsigned long long)d[1], (unsigned long long)d[2],
             target_psnr_db, o.radius, o.chunk, o.lmax, o.lorenzo_dims, o.psnr_mode, o.lossless,
             max_size_increase);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            *out = it->second;
            return FPSNR_OK;
        }
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    std::vector<int> chunks = {64, 128, 256, 512, 1024, 2048};
    if (std::find(chunks.begin(), chunks.end(), o.chunk) == chunks.end()) chunks.push_back(o.chunk);
    std::sort(chunks.begin(), chunks.end());

    // buffers sized for the smallest chunk (the largest worst-case blob)
    Buffers b;
    {
        fpsnr_opts oc = o;
        oc.chunk = chunks.front();
        fpsnr_plan_t p = nullptr;
        int rc = fpsnr_plan(&p, ndim, d, target_psnr_db, &oc);
        if (rc) return rc;
        b.cap = fpsnr_max_compressed_bytes(p);
        fpsnr_plan_destroy(p);
    }
    if (cudaMalloc(&b.blob, b.cap) != cudaSuccess ||
        cudaMalloc(&b.rec, std::max<uint64_t>(n, 1) * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&b.nbytes, sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&b.stats, sizeof(fpsnr_stats)) != cudaSuccess ||
        cudaMalloc(&b.status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return FPSNR_ENOMEM;
    }
    Events ev;
    if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess)
        return FPSNR_ECUDA;

    // chunk size: fastest within the size tolerance of the smallest blob
    std::vector<double> cms(chunks.size());
    std::vector<uint64_t> cbytes(chunks.size());
    for (size_t i = 0; i < chunks.size(); i++) {
        fpsnr_opts oc = o;
        oc.chunk = chunks[i];
        fpsnr_plan_t p = nullptr;
        int rc = fpsnr_plan(&p, ndim, d, target_psnr_db, &oc);
        if (rc) return rc;
        rc = measure(p, d_sample, n, b, ev, st, &cms[i], &cbytes[i]);
        fpsnr_plan_destroy(p);
        if (rc) return rc;
    }
    const uint64_t smallest = *std::min_element(cbytes.begin(), cbytes.end());
    size_t pick = 0;
    double pick_ms = INFINITY;
    for (size_t i = 0; i < chunks.size(); i++) {
        if ((double)cbytes[i] <= (double)smallest * (1.0 + max_size_increase) && cms[i] < pick_ms) {
            pick = i;
            pick_ms = cms[i];
        }
    }

    // launch shapes at that chunk, one parameter at a time
    fpsnr_opts oc = o;
    oc.chunk = chunks[pick];
    fpsnr_plan_t p = nullptr;
    int rc = fpsnr_plan(&p, ndim, d, target_psnr_db, &oc);
    if (rc) return rc;
    fpsnr_tuning cur;
    fpsnr_plan_get_tuning(p, &cur);
    cur.dec_threads = 0;
    double best_ms = pick_ms;
    uint64_t best_bytes = cbytes[pick];
    const bool has_tx = cur.pq_tile_x != 0, has_band = cur.band_rows != 0;
    for (int param = 0; param < 3 && rc == FPSNR_OK; param++) {
        std::vector<int> vals;
        if (param == 0 && has_tx) vals = {128, 256, 512, 1024};
        if (param == 1 && has_band) vals = {16, 32, 64};
        if (param == 2) vals = {128, 256, 512};
        for (int v : vals) {
            fpsnr_tuning t = cur;
            if (param == 0) t.pq_tile_x = v;
            if (param == 1) t.band_rows = v;
            if (param == 2) t.dec_threads = v;
            if (fpsnr_plan_set_tuning(p, &t) != FPSNR_OK) continue;
            double ms = 0.0;
            uint64_t by = 0;
            rc = measure(p, d_sample, n, b, ev, st, &ms, &by);
            if (rc) break;
            if (ms < best_ms) {
                best_ms = ms;
                best_bytes = by;
                cur = t;
            }
        }
    }
    fpsnr_plan_destroy(p);
    if (rc) return rc;
    cur.chunk = chunks[pick];
    cur.ms = best_ms;
    cur.bytes = best_bytes;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = cur;
    }
    *out = cur;
    return FPSNR_OK;
}
