// psnr.cu -- distortion of a reconstruction (Eq. 4-5 of Sec. IV):
// vr = max - min of the original field, MSE = sum (x - x')^2 / n,
// PSNR = 20 log10 vr - 10 log10 MSE.
//
// One pass over both arrays: per point the difference is made exact with a
// float32 TwoSum, scaled by a per-thread power-of-two unit that follows the
// largest difference seen (so that squares stay normal floats for any range,
// see SqSum), its square made exact with an FMA TwoProd, and both parts are
// accumulated in float-float per thread; threads and blocks combine in FP64 in
// a fixed order, so the result does not depend on scheduling.  The log10 is
// taken on the host.
#include <float.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace fp {

struct PsnrPart {
    double sse;
    float lo, hi;
    int nf;
    int pad;
};

template <bool VEC>
__global__ void __launch_bounds__(512) k_psnr(const float* __restrict__ x,
                                              const float* __restrict__ xr, uint64_t n,
                                              PsnrPart* part, uint32_t* done, PsnrPart* result) {
    const uint32_t tid = threadIdx.x;
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + tid;
    const uint64_t gsz = (uint64_t)gridDim.x * blockDim.x;
    float lo = FLT_MAX, hi = -FLT_MAX;
    int nf = 0;
    SqSum acc;
    sq_init(acc);
    uint64_t tail = 0;
    if (VEC) {
        const float4* x4 = reinterpret_cast<const float4*>(x);
        const float4* r4 = reinterpret_cast<const float4*>(xr);
        const uint64_t n4 = n >> 2;
        for (uint64_t i = gtid; i < n4; i += gsz) {
            const float4 a = __ldcs(x4 + i), b = __ldcs(r4 + i);
            nf |= !isfinite(a.x) | !isfinite(a.y) | !isfinite(a.z) | !isfinite(a.w);
            lo = fminf(lo, fminf(fminf(a.x, a.y), fminf(a.z, a.w)));
            hi = fmaxf(hi, fmaxf(fmaxf(a.x, a.y), fmaxf(a.z, a.w)));
            sq_add(acc, a.x, b.x);
            sq_add(acc, a.y, b.y);
            sq_add(acc, a.z, b.z);
            sq_add(acc, a.w, b.w);
        }
        tail = n4 << 2;
    }
    for (uint64_t i = tail + gtid; i < n; i += gsz) {
        const float a = x[i], b = xr[i];
        nf |= !isfinite(a);
        lo = fminf(lo, a);
        hi = fmaxf(hi, a);
        sq_add(acc, a, b);
    }
    __shared__ double sdbl[16];
    __shared__ float slo[16], shi[16];
    __shared__ int snf[16];
    __shared__ bool last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        nf |= __shfl_xor_sync(0xffffffffu, nf, o);
    }
    if ((tid & 31) == 0) { slo[tid >> 5] = lo; shi[tid >> 5] = hi; snf[tid >> 5] = nf; }
    const double bs = block_sum_double(sq_total(acc), sdbl);
    if (tid == 0) {
        for (uint32_t w = 1; w < (blockDim.x >> 5); w++) {
            lo = fminf(lo, slo[w]); hi = fmaxf(hi, shi[w]); nf |= snf[w];
        }
        PsnrPart pp;
        pp.sse = bs;
        pp.lo = lo;
        pp.hi = hi;
        pp.nf = nf;
        pp.pad = 0;
        part[blockIdx.x] = pp;
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || tid != 0) return;
    __threadfence();
    PsnrPart r;
    r.sse = 0.0;
    r.lo = FLT_MAX;
    r.hi = -FLT_MAX;
    r.nf = 0;
    r.pad = 0;
    for (uint32_t b = 0; b < gridDim.x; b++) {  // fixed order
        r.sse += __ldcg(&part[b].sse);
        r.lo = fminf(r.lo, __ldcg(&part[b].lo));
        r.hi = fmaxf(r.hi, __ldcg(&part[b].hi));
        r.nf |= __ldcg(&part[b].nf);
    }
    *result = r;
    *done = 0;
}

// Scratch layout: [0] done counter (u32, padded to 16 B), [1] result, then partials.
static size_t psnr_scratch_bytes(unsigned blocks) { return 16 + 32 + (size_t)blocks * sizeof(PsnrPart); }

size_t psnr_scratch_bytes_for(unsigned blocks) {
    static_assert(sizeof(PsnrPart) == kPsnrResultBytes, "result layout");
    return psnr_scratch_bytes(blocks);
}

int psnr_blocks(uint64_t n, int sm_count) {
    uint64_t want = (n + 512ull * 16 - 1) / (512ull * 16);
    want = std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sm_count * 4));
    return (int)want;
}

int psnr_enqueue(const float* d_x, const float* d_xr, uint64_t n, void* scratch, unsigned blocks,
                 cudaStream_t st) {
    uint8_t* s = reinterpret_cast<uint8_t*>(scratch);
    uint32_t* done = reinterpret_cast<uint32_t*>(s);
    PsnrPart* result = reinterpret_cast<PsnrPart*>(s + 16);
    PsnrPart* part = reinterpret_cast<PsnrPart*>(s + 48);
    const bool vec = (((uintptr_t)d_x | (uintptr_t)d_xr) & 15u) == 0;
    if (vec) k_psnr<true><<<blocks, 512, 0, st>>>(d_x, d_xr, n, part, done, result);
    else k_psnr<false><<<blocks, 512, 0, st>>>(d_x, d_xr, n, part, done, result);
    return cudaGetLastError() == cudaSuccess ? FPSNR_OK : FPSNR_ECUDA;
}

int psnr_finish(const void* h_result, double* psnr_db, double* mse, double* vr, uint64_t n) {
    const PsnrPart* r = reinterpret_cast<const PsnrPart*>(h_result);
    if (r->nf) return FPSNR_ENONFINITE;
    const double v = (double)r->hi - (double)r->lo;
    const double m = r->sse / (double)n;
    if (vr) *vr = v;
    if (mse) *mse = m;
    if (psnr_db) *psnr_db = (m == 0.0) ? INFINITY : 20.0 * log10(v) - 10.0 * log10(m);
    return FPSNR_OK;
}

}  // namespace fp

extern "C" int fpsnr_psnr(const float* d_x, const float* d_xr, uint64_t n, double* h_psnr_db,
                          double* h_mse, double* h_vr, void* stream) {
    if (n > 0 && (!d_x || !d_xr)) return FPSNR_EINVAL;
    if ((((uintptr_t)d_x | (uintptr_t)d_xr) & 3u) != 0) return FPSNR_EINVAL;
    if (n == 0) {
        if (h_psnr_db) *h_psnr_db = INFINITY;
        if (h_mse) *h_mse = 0.0;
        if (h_vr) *h_vr = 0.0;
        return FPSNR_OK;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FPSNR_ECUDA;
    const unsigned blocks = (unsigned)fp::psnr_blocks(n, sms);
    const size_t bytes = fp::psnr_scratch_bytes(blocks);
    void* scratch = nullptr;
    if (cudaMallocAsync(&scratch, bytes, st) != cudaSuccess) return FPSNR_ECUDA;
    int rc = FPSNR_OK;
    fp::PsnrPart host;
    if (cudaMemsetAsync(scratch, 0, 16, st) != cudaSuccess) rc = FPSNR_ECUDA;
    if (!rc) rc = fp::psnr_enqueue(d_x, d_xr, n, scratch, blocks, st);
    if (!rc && cudaMemcpyAsync(&host, reinterpret_cast<uint8_t*>(scratch) + 16, sizeof(host),
                               cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = FPSNR_ECUDA;
    if (cudaFreeAsync(scratch, st) != cudaSuccess && !rc) rc = FPSNR_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = FPSNR_ECUDA;
    if (rc) return rc;
    return fp::psnr_finish(&host, h_psnr_db, h_mse, h_vr, n);
}
