// lossless.cu -- optional lossless layer over the finished blob, standing in
// for SZ's optional lossless step 3 (Sec. II-A; the paper names GZIP).
//
// Container "FPZ1" (layout in include/fpsnr.h, opts.lossless): the blob is
// cut into 1 KiB segments, each coded on its own -- a nonzero byte is copied,
// a run of k zero bytes becomes 0x00 and k - 1 in LEB128 -- or stored raw when
// its code is not shorter; the container replaces the blob only when smaller.
// Huffman spends at least one bit per symbol, so flat regions at low targets
// leave long zero runs in the stream; elsewhere the stream is close to
// incompressible and the blob stays as it is.
//
//   wrap:   k_zr_size (one thread per segment: coded length)
//           k_zr_layout (one block per field: offsets by scan, the decision)
//           k_zr_write (one thread per segment, into the plan's scratch)
//           k_zr_copy (scratch -> caller's buffer, size and stats updated)
//   unwrap: k_zr_expand (one thread per segment, into the plan's scratch; a
//           plain blob is copied) -- decompression then reads the scratch
#include "common.cuh"

namespace fp {

__device__ __forceinline__ uint32_t ldb(const uint8_t* p, uint64_t o) {
    return (uint32_t)p[o] | ((uint32_t)p[o + 1] << 8) | ((uint32_t)p[o + 2] << 16) |
           ((uint32_t)p[o + 3] << 24);
}
__device__ __forceinline__ void stb(uint8_t* p, uint64_t o, uint32_t v) {
    p[o] = (uint8_t)v;
    p[o + 1] = (uint8_t)(v >> 8);
    p[o + 2] = (uint8_t)(v >> 16);
    p[o + 3] = (uint8_t)(v >> 24);
}

// Code of one segment; returns its length and writes it to `out` if given.
__device__ uint32_t zr_code(const uint8_t* __restrict__ in, uint32_t len, uint8_t* __restrict__ out) {
    uint32_t o = 0, i = 0;
    while (i < len) {
        const uint8_t b = in[i];
        if (b) {
            if (out) out[o] = b;
            o++;
            i++;
            continue;
        }
        uint32_t k = 1;
        while (i + k < len && in[i + k] == 0) k++;
        if (out) out[o] = 0;
        o++;
        uint32_t v = k - 1;
        while (v >= 128u) {
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

struct ZrArgs {
    DevParams* par;
    uint8_t* blob;        // caller's buffer: the finished blob (wrap) or the input (unwrap)
    uint64_t in_bytes;    // unwrap: bytes the caller passed
    uint8_t* scratch;     // plan scratch: the container (wrap) or the raw blob (unwrap)
    uint64_t scratch_cap;
    uint32_t* seg;        // per segment: coded length, then offset | raw bit
    uint64_t seg_cap;     // segments the table holds
    uint64_t* out_bytes;  // wrap: caller's size word (may be null)
    fpsnr_stats* stats;   // wrap: caller's stats (may be null)
};

__device__ __forceinline__ bool zr_wrap_applies(const DevParams* par) {
    return !(par->flags & kFlagError) && par->status == 0;
}

__global__ void __launch_bounds__(256) k_zr_size(const __grid_constant__ Batch<ZrArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const ZrArgs& a = B.a[fld];
    if (!zr_wrap_applies(a.par)) return;
    const uint64_t total = a.par->total;
    const uint64_t nseg = (total + kZrSeg - 1) / kZrSeg;
    if (nseg > a.seg_cap) return;  // the layout kernel leaves the blob as it is
    const uint64_t g = (uint64_t)(blockIdx.x - B.off[fld]) * blockDim.x + threadIdx.x;
    const uint64_t gs = (uint64_t)(B.off[fld + 1] - B.off[fld]) * blockDim.x;
    for (uint64_t s = g; s < nseg; s += gs) {
        const uint64_t b = s * kZrSeg;
        const uint32_t len = (uint32_t)min((uint64_t)kZrSeg, total - b);
        const uint32_t c = zr_code(a.blob + b, len, nullptr);
        a.seg[s] = c >= len ? (len | 0x80000000u) : c;
    }
}

// one block per field: exclusive scan of the segment lengths into offsets
// (bit 31 kept), container size, and whether the container is used
__global__ void __launch_bounds__(1024) k_zr_layout(const __grid_constant__ Batch<ZrArgs> B) {
    const ZrArgs& a = B.a[blockIdx.x];
    DevParams* par = a.par;
    __shared__ uint32_t sh[33];
    __shared__ unsigned long long s_base;
    if (threadIdx.x == 0) {
        s_base = 0;
        par->zr_use = 0;
    }
    __syncthreads();
    if (!zr_wrap_applies(par)) return;
    const uint64_t total = par->total;
    const uint64_t nseg = (total + kZrSeg - 1) / kZrSeg;
    if (nseg > a.seg_cap) return;
    for (uint64_t s0 = 0; s0 < nseg; s0 += blockDim.x) {
        const uint64_t s = s0 + threadIdx.x;
        const uint32_t e = s < nseg ? a.seg[s] : 0u;
        const uint32_t len = e & 0x7FFFFFFFu;
        uint32_t tot;
        const uint32_t ex = block_excl_scan(len, sh, &tot);
        if (s < nseg) a.seg[s] = (uint32_t)(s_base + ex) | (e & 0x80000000u);
        __syncthreads();
        if (threadIdx.x == 0) s_base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const uint64_t data = s_base;
        a.seg[nseg] = (uint32_t)data;
        const uint64_t dstart = 32 + ((4 * (nseg + 1) + 15) & ~(uint64_t)15);
        const uint64_t ctotal = dstart + ((data + 15) & ~(uint64_t)15);
        const bool use = ctotal < total && ctotal <= a.scratch_cap;
        par->zr_use = use ? 1u : 0u;
        par->zr_total = ctotal;
        par->zr_dstart = dstart;
    }
}

__global__ void __launch_bounds__(256) k_zr_write(const __grid_constant__ Batch<ZrArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const ZrArgs& a = B.a[fld];
    const DevParams* par = a.par;
    if (!par->zr_use) return;
    const uint64_t total = par->total, ctotal = par->zr_total, dstart = par->zr_dstart;
    const uint64_t nseg = (total + kZrSeg - 1) / kZrSeg;
    const uint64_t g = (uint64_t)(blockIdx.x - B.off[fld]) * blockDim.x + threadIdx.x;
    const uint64_t gs = (uint64_t)(B.off[fld + 1] - B.off[fld]) * blockDim.x;
    uint8_t* c = a.scratch;
    if (g == 0) {
        stb(c, 0, kZrMagic);
        stb(c, 4, 1u);
        stb(c, 8, (uint32_t)total);
        stb(c, 12, (uint32_t)(total >> 32));
        stb(c, 16, kZrSeg);
        stb(c, 20, (uint32_t)nseg);
        stb(c, 24, 0u);
        stb(c, 28, 0u);
    }
    // offset table and its padding
    for (uint64_t s = g; s < (dstart - 32) / 4; s += gs) stb(c, 32 + 4 * s, s <= nseg ? a.seg[s] : 0u);
    // data padding
    const uint64_t data = a.seg[nseg];
    for (uint64_t o = dstart + data + g; o < ctotal; o += gs) c[o] = 0;
    for (uint64_t s = g; s < nseg; s += gs) {
        const uint32_t e = a.seg[s];
        const uint64_t b = s * kZrSeg;
        const uint32_t len = (uint32_t)min((uint64_t)kZrSeg, total - b);
        uint8_t* dst = c + dstart + (e & 0x7FFFFFFFu);
        if (e & 0x80000000u) {
            for (uint32_t i = 0; i < len; i++) dst[i] = a.blob[b + i];
        } else {
            zr_code(a.blob + b, len, dst);
        }
    }
}

__global__ void __launch_bounds__(256) k_zr_copy(const __grid_constant__ Batch<ZrArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const ZrArgs& a = B.a[fld];
    const DevParams* par = a.par;
    if (!par->zr_use) return;
    const uint64_t ctotal = par->zr_total;
    const uint64_t g = (uint64_t)(blockIdx.x - B.off[fld]) * blockDim.x + threadIdx.x;
    const uint64_t gs = (uint64_t)(B.off[fld + 1] - B.off[fld]) * blockDim.x;
    // both buffers are 16-byte aligned and the container is a multiple of 16 bytes
    const uint4* src = reinterpret_cast<const uint4*>(a.scratch);
    uint4* dst = reinterpret_cast<uint4*>(a.blob);
    for (uint64_t i = g; i < ctotal / 16; i += gs) dst[i] = src[i];
    if (g == 0) {
        if (a.out_bytes) *a.out_bytes = ctotal;
        if (a.stats) a.stats->bytes = ctotal;
    }
}

// Unwrap into the plan's scratch.  A plain blob (no container magic) is
// copied; a container is expanded segment by segment.  The outcome goes to
// par->zr_bad (the header check that follows must not clear it) and the raw
// length to par->zr_raw.
__global__ void __launch_bounds__(256) k_zr_expand(const __grid_constant__ Batch<ZrArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const ZrArgs& a = B.a[fld];
    DevParams* par = a.par;
    const uint8_t* c = a.blob;
    const uint64_t bytes = a.in_bytes;
    const uint64_t g = (uint64_t)(blockIdx.x - B.off[fld]) * blockDim.x + threadIdx.x;
    const uint64_t gs = (uint64_t)(B.off[fld + 1] - B.off[fld]) * blockDim.x;
    auto bad = [&]() { atomicOr(&par->zr_bad, 1u); };
    if (bytes < 4 || ldb(c, 0) != kZrMagic) {
        // plain blob: copy what fits (the header check sees the true length)
        const uint64_t m = min(bytes, a.scratch_cap);
        for (uint64_t i = g; i < m; i += gs) a.scratch[i] = c[i];
        if (g == 0) par->zr_raw = m;
        return;
    }
    if (bytes < 32) {
        if (g == 0) bad();
        return;
    }
    const uint64_t rb = (uint64_t)ldb(c, 8) | ((uint64_t)ldb(c, 12) << 32);
    const uint64_t nseg = ldb(c, 20);
    const uint64_t dstart = 32 + ((4 * (nseg + 1) + 15) & ~(uint64_t)15);
    const bool hdr_ok = ldb(c, 4) == 1u && ldb(c, 16) == kZrSeg && rb <= a.scratch_cap &&
                        nseg == (rb + kZrSeg - 1) / kZrSeg && dstart <= bytes &&
                        dstart + (ldb(c, 32 + 4 * nseg) & 0x7FFFFFFFu) <= bytes;
    if (!hdr_ok) {
        if (g == 0) bad();
        return;
    }
    if (g == 0) par->zr_raw = rb;
    const uint64_t dlen = ldb(c, 32 + 4 * nseg) & 0x7FFFFFFFu;
    for (uint64_t s = g; s < nseg; s += gs) {
        const uint32_t e0 = ldb(c, 32 + 4 * s), e1 = ldb(c, 32 + 4 * (s + 1));
        const uint64_t lo = e0 & 0x7FFFFFFFu, hi = e1 & 0x7FFFFFFFu;
        const uint64_t b = s * kZrSeg;
        const uint32_t len = (uint32_t)min((uint64_t)kZrSeg, rb - b);
        if (lo > hi || hi > dlen) {
            bad();
            continue;
        }
        const uint8_t* in = c + dstart + lo;
        const uint64_t clen = hi - lo;
        uint8_t* out = a.scratch + b;
        if (e0 & 0x80000000u) {
            if (clen != len) {
                bad();
                continue;
            }
            for (uint32_t i = 0; i < len; i++) out[i] = in[i];
            continue;
        }
        uint64_t i = 0;
        uint32_t w = 0;
        bool ok = true;
        while (ok && i < clen) {
            const uint8_t v = in[i++];
            if (v) {
                if (w >= len) ok = false;
                else out[w++] = v;
                continue;
            }
            uint32_t k = 0;
            int sh = 0;
            for (;;) {
                if (i >= clen || sh > 28) {
                    ok = false;
                    break;
                }
                const uint8_t t = in[i++];
                k |= (uint32_t)(t & 127u) << sh;
                sh += 7;
                if (!(t & 128u)) break;
            }
            if (!ok) break;
            if ((uint64_t)w + k + 1 > len) {
                ok = false;
                break;
            }
            for (uint32_t j = 0; j <= k; j++) out[w++] = 0;
        }
        if (!ok || w != len) bad();
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static uint32_t zr_blocks(const fpsnr_plan_s* p) {
    const uint64_t segs = (p->zr_scratch_cap + kZrSeg - 1) / kZrSeg;
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((segs + 255) / 256, 64));
}

int launch_zr_wrap(fpsnr_plan_s* const* P, void* const* d_out, uint64_t* d_out_bytes,
                   fpsnr_stats* d_stats, int count, cudaStream_t st) {
    Batch<ZrArgs> b, b1;
    b.count = b1.count = 0;
    uint32_t blocks[kMaxBatch], ones[kMaxBatch];
    for (int f = 0; f < count; f++) {
        const fpsnr_plan_s* p = P[f];
        if (!p->lossless || p->n == 0) continue;
        const Workspace& w = p->w;
        ZrArgs a{w.par, reinterpret_cast<uint8_t*>(d_out[f]), 0, w.zr_scratch, p->zr_scratch_cap,
                 w.zr_seg, p->zr_seg_cap, d_out_bytes ? d_out_bytes + f : nullptr,
                 d_stats ? d_stats + f : nullptr};
        blocks[b.count] = zr_blocks(p);
        ones[b1.count] = 1;
        b.a[b.count++] = a;
        b1.a[b1.count++] = a;
    }
    if (!b.count) return FPSNR_OK;
    const uint32_t tot = batch_offsets(b, blocks);
    batch_offsets(b1, ones);
    StageScope sc(P[0]->prof, kStZrWrap, st);
    k_zr_size<<<tot, 256, 0, st>>>(b);
    k_zr_layout<<<b1.count, 1024, 0, st>>>(b1);
    k_zr_write<<<tot, 256, 0, st>>>(b);
    k_zr_copy<<<tot, 256, 0, st>>>(b);
    sc.more(3);
    return cudaGetLastError() == cudaSuccess ? FPSNR_OK : FPSNR_ECUDA;
}

int launch_zr_unwrap(fpsnr_plan_s* const* P, const void* const* d_blob, const uint64_t* bytes,
                     int count, cudaStream_t st) {
    Batch<ZrArgs> b;
    b.count = 0;
    uint32_t blocks[kMaxBatch];
    for (int f = 0; f < count; f++) {
        const fpsnr_plan_s* p = P[f];
        if (!p->lossless || p->n == 0) continue;
        const Workspace& w = p->w;
        blocks[b.count] = zr_blocks(p);
        b.a[b.count++] = ZrArgs{w.par, const_cast<uint8_t*>(reinterpret_cast<const uint8_t*>(d_blob[f])),
                                bytes[f], w.zr_scratch, p->zr_scratch_cap, w.zr_seg, p->zr_seg_cap,
                                nullptr, nullptr};
    }
    if (!b.count) return FPSNR_OK;
    const uint32_t tot = batch_offsets(b, blocks);
    StageScope sc(P[0]->prof, kStZrUnwrap, st);
    k_zr_expand<<<tot, 256, 0, st>>>(b);
    return cudaGetLastError() == cudaSuccess ? FPSNR_OK : FPSNR_ECUDA;
}

}  // namespace fp
