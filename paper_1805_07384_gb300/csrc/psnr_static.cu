// psnr_static.cu -- fpsnr_psnr_static: the PSNR reduction with no device
// allocation, for callers that cannot allocate device memory while they run
// (code inside an allocator's or memory pool's own callback, processes held to
// a fixed memory budget, service loops that must stay out of the CUDA
// allocator because cudaMalloc/cudaFree can synchronize the device).
//
// The scratch of the reduction (a zeroed block counter, the result and one
// partial per block) lives in the file-scope device array below.  Host code
// cannot use the array's name as a device address, so the first call on each
// device looks the address up with that device current and caches it.  Every
// call shares the array: calls that overlap on the GPU race on it.
#include <math.h>

#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kScratchBytes = 64 * 1024;
constexpr uint64_t kPointsPerBlock = 512ull * 256;  // threads x points per thread
constexpr uint64_t kMaxBlocks = FPSNR_PSNR_STATIC_MAX_POINTS / kPointsPerBlock;
constexpr int kMaxDevices = 256;

static __device__ __align__(256) unsigned char g_psnr_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices];

// Device address of g_psnr_scratch on the current device (looked up once).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FPSNR_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_psnr_scratch) != cudaSuccess || !p) return FPSNR_ECUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return FPSNR_OK;
}

}  // namespace

extern "C" int fpsnr_psnr_static(const float* d_x, const float* d_xr, uint64_t n,
                                 double* h_psnr_db, double* h_mse, double* h_vr, void* stream) {
    if (n > 0 && (!d_x || !d_xr)) return FPSNR_EINVAL;
    if ((((uintptr_t)d_x | (uintptr_t)d_xr) & 3u) != 0) return FPSNR_EINVAL;
    if (n > FPSNR_PSNR_STATIC_MAX_POINTS) return FPSNR_EINVAL;
    if (n == 0) {
        if (h_psnr_db) *h_psnr_db = INFINITY;
        if (h_mse) *h_mse = 0.0;
        if (h_vr) *h_vr = 0.0;
        return FPSNR_OK;
    }
    const unsigned blocks = (unsigned)((n + kPointsPerBlock - 1) / kPointsPerBlock);
    static_assert(kMaxBlocks * 24 + 48 <= kScratchBytes, "scratch holds every partial");
    if (blocks > kMaxBlocks || fp::psnr_scratch_bytes_for(blocks) > kScratchBytes)
        return FPSNR_EINVAL;
    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // the block counter must start at zero; the rest is overwritten before use
    if (cudaMemsetAsync(scratch, 0, fp::kPsnrResultOffset, st) != cudaSuccess) return FPSNR_ECUDA;
    rc = fp::psnr_enqueue(d_x, d_xr, n, scratch, blocks, st);
    if (rc) return rc;
    alignas(8) unsigned char host[32];
    if (cudaMemcpyAsync(host, static_cast<unsigned char*>(scratch) + fp::kPsnrResultOffset,
                        fp::kPsnrResultBytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FPSNR_ECUDA;
    return fp::psnr_finish(host, h_psnr_db, h_mse, h_vr, n);
}
