// decompress.cu -- inverse of the compression chain (Sec. III: rebuild the
// prediction errors, then the data; Eq. 1 holds because the residuals are
// reproduced exactly).
//
//   k_dsetup        header validation against the plan, canonical decoding
//                   tables and an 11-bit look-up table
//   k_decode        one thread per chunk, canonical Huffman decode into int32
//                   residuals (written into the output buffer)
//   k_scatter       outlier residuals put back
//   k_scan_contig   inclusive prefix sum along x (rows), decoupled look-back
//                   between tiles of one row
//   k_scan_strided  inclusive prefix sum along y or z, decoupled look-back
//                   between row segments; the last pass also dequantizes:
//                   x' = fmaf((float)q, s, xmin) (midpoint reconstruction,
//                   Sec. IV)
//   k_patch         verbatim points restored
//
// The prefix sums run in modular uint32 arithmetic: intermediate partial sums
// may leave the int32 range, but every final lattice value is in [0, 2^31),
// so the modular result is exact.
#include "common.cuh"

namespace fp {

__device__ __forceinline__ uint32_t rd32(const uint8_t* b, uint64_t o) {
    return *reinterpret_cast<const uint32_t*>(b + o);
}
__device__ __forceinline__ uint64_t rd64(const uint8_t* b, uint64_t o) {
    return *reinterpret_cast<const uint64_t*>(b + o);
}
static __device__ __forceinline__ uint64_t pad16d(uint64_t b) { return (b + 15u) & ~(uint64_t)15u; }

__global__ void __launch_bounds__(1024) k_dsetup(DevParams* par, const uint8_t* __restrict__ blob,
                                                 uint64_t bytes, int ndim, int ld, uint64_t d0,
                                                 uint64_t d1, uint64_t d2, uint64_t n,
                                                 uint32_t chunk, uint64_t nchunks, uint32_t* lut,
                                                 uint16_t* syms) {
    __shared__ int s_ok;
    __shared__ uint32_t s_cnt[32];
    __shared__ unsigned long long s_kraft;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) {
        int ok = bytes >= kHeaderBytes;
        uint32_t flags = 0, radius = 0, ch = 0, lmax = 0, nsym = 0, nck = 0, words = 0, no = 0, nv = 0;
        if (ok) {
            ok = rd32(blob, 0) == kMagic && rd32(blob, 4) == kVersion &&
                 rd32(blob, 8) == (uint32_t)ndim && rd32(blob, 12) == (uint32_t)ld &&
                 rd64(blob, 16) == d0 && rd64(blob, 24) == d1 && rd64(blob, 32) == d2;
            flags = rd32(blob, 92);
            radius = rd32(blob, 96);
            ch = rd32(blob, 100);
            lmax = rd32(blob, 104);
            nsym = rd32(blob, 108);
            nck = rd32(blob, 112);
            words = rd32(blob, 116);
            no = rd32(blob, 120);
            nv = rd32(blob, 124);
            ok = ok && (flags & ~3u) == 0;
        }
        const bool cst = ok && (flags & kFlagConstant);
        if (ok && !cst) {
            ok = radius >= 1 && radius <= (uint32_t)kMaxRadius && ch == chunk && lmax >= 1 &&
                 lmax <= (uint32_t)kMaxLmax && nsym >= 1 && nsym <= 2 * radius &&
                 (uint64_t)nck == nchunks && no <= n && nv <= n;
        }
        uint64_t off_ct = kHeaderBytes, off_st = kHeaderBytes, off_ou = kHeaderBytes,
                 off_vb = kHeaderBytes, total = kHeaderBytes;
        if (ok && !cst) {
            off_ct = kHeaderBytes + pad16d(4ull * nsym);
            off_st = off_ct + pad16d(4ull * nck);
            off_ou = off_st + pad16d(4ull * words);
            off_vb = off_ou + pad16d(8ull * no);
            total = off_vb + pad16d(8ull * nv);
            ok = total <= bytes;
        }
        par->xmin = ok ? *reinterpret_cast<const float*>(blob + 72) : 0.0f;
        par->s = ok ? *reinterpret_cast<const float*>(blob + 80) : 0.0f;
        par->flags = ok ? flags : kFlagError;
        par->status = ok ? 0 : FPSNR_ECORRUPT;
        par->d_radius = radius;
        par->d_chunk = ch;
        par->d_lmax = lmax;
        par->d_nsym = cst ? 0 : nsym;
        par->d_nchunks = nck;
        par->d_words = words;
        par->d_nout = cst ? 0 : no;
        par->d_nvb = cst ? 0 : nv;
        par->off_ct = off_ct;
        par->off_st = off_st;
        par->off_ou = off_ou;
        par->off_vb = off_vb;
        par->total = total;
        s_ok = ok && !cst;
        s_kraft = 0;
    }
    if (tid < 32) s_cnt[tid] = 0;
    __syncthreads();
    if (!s_ok) return;
    const uint32_t nsym = par->d_nsym, lmax = par->d_lmax, radius = par->d_radius;
    const uint32_t* cb = reinterpret_cast<const uint32_t*>(blob + kHeaderBytes);
    int bad = 0;
    unsigned long long kraft = 0;
    for (uint32_t i = tid; i < nsym; i += blockDim.x) {
        const uint32_t e = cb[i];
        const uint32_t l = e >> 16, s = e & 0xffffu;
        if (l < 1 || l > lmax || s >= 2 * radius || (i > 0 && cb[i - 1] >= e)) bad = 1;
        else {
            atomicAdd(&s_cnt[l], 1u);
            kraft += 1ull << (kMaxLmax - l);
        }
        syms[i] = (uint16_t)s;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kraft += __shfl_xor_sync(0xffffffffu, kraft, o);
    if ((tid & 31) == 0) atomicAdd(&s_kraft, kraft);
    bad = __syncthreads_or(bad);
    if (tid == 0) {
        if (bad || s_kraft > (1ull << kMaxLmax)) {
            set_error(par, FPSNR_ECORRUPT);
        }
        uint32_t code = 0, idx = 0;
        for (uint32_t l = 1; l < 32; l++) {
            if (l > 1) code = (code + s_cnt[l - 1]) << 1;
            par->d_count[l] = s_cnt[l];
            par->d_first_code[l] = code;
            par->d_first_index[l] = idx;
            idx += s_cnt[l];
        }
        par->d_count[0] = 0;
        par->d_first_code[0] = 0;
        par->d_first_index[0] = 0;
    }
    for (uint32_t i = tid; i < (1u << kLutBits); i += blockDim.x) lut[i] = 0u;
    __syncthreads();
    if (par->flags & kFlagError) return;
    for (uint32_t i = tid; i < nsym; i += blockDim.x) {
        const uint32_t e = cb[i];
        const uint32_t l = e >> 16, s = e & 0xffffu;
        if (l <= (uint32_t)kLutBits) {
            const uint32_t code = par->d_first_code[l] + (i - par->d_first_index[l]);
            const uint32_t b0 = code << (kLutBits - l), cnt = 1u << (kLutBits - l);
            if (code < (1u << l))
                for (uint32_t j = 0; j < cnt; j++) lut[b0 + j] = (s << 8) | l;
        }
    }
}

// One thread decodes one chunk of `chunk` symbols into int32 residuals.
__global__ void __launch_bounds__(256) k_decode(DevParams* par, const uint8_t* __restrict__ blob,
                                                const uint32_t* __restrict__ lut_g,
                                                const uint16_t* __restrict__ syms,
                                                int32_t* __restrict__ out, uint64_t n,
                                                uint32_t chunk, uint64_t nchunks) {
    __shared__ uint32_t slut[1u << kLutBits];
    __shared__ uint32_t s_cnt[32], s_fc[32], s_fi[32];
    const uint32_t flags = par->flags;
    if (flags & kFlagError) return;
    const bool cst = (flags & kFlagConstant) != 0;
    if (!cst) {
        for (uint32_t i = threadIdx.x; i < (1u << kLutBits); i += blockDim.x) slut[i] = lut_g[i];
        if (threadIdx.x < 32) {
            s_cnt[threadIdx.x] = par->d_count[threadIdx.x];
            s_fc[threadIdx.x] = par->d_first_code[threadIdx.x];
            s_fi[threadIdx.x] = par->d_first_index[threadIdx.x];
        }
    }
    __syncthreads();
    const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchunks) return;
    const uint64_t beg = c * chunk;
    const uint64_t end = min(beg + chunk, n);
    if (cst) {
        for (uint64_t i = beg; i < end; i++) out[i] = 0;
        return;
    }
    const uint32_t R = par->d_radius, lmax = par->d_lmax, words = par->d_words;
    const uint32_t* tab = reinterpret_cast<const uint32_t*>(blob + par->off_ct);
    const uint32_t* stream = reinterpret_cast<const uint32_t*>(blob + par->off_st);
    const uint32_t w0 = tab[c];
    const uint32_t w1 = (c + 1 < nchunks) ? tab[c + 1] : words;
    if (w0 > w1 || w1 > words) { set_error(par, FPSNR_ECORRUPT); return; }
    uint64_t buf = 0;
    uint32_t nb = 0, wi = w0;
    for (uint64_t i = beg; i < end; i++) {
        while (nb <= 32 && wi < w1) {
            buf |= (uint64_t)__ldg(stream + wi) << (32 - nb);
            wi++;
            nb += 32;
        }
        const uint32_t e = slut[(uint32_t)(buf >> (64 - kLutBits))];
        uint32_t l = e & 0xffu, sym = e >> 8;
        if (l == 0) {
            for (l = kLutBits + 1; l <= lmax; l++) {
                const uint32_t code = (uint32_t)(buf >> (64 - l));
                const uint32_t k = code - s_fc[l];
                if (k < s_cnt[l]) { sym = syms[s_fi[l] + k]; break; }
            }
            if (l > lmax) { set_error(par, FPSNR_ECORRUPT); return; }
        }
        if (l > nb) { set_error(par, FPSNR_ECORRUPT); return; }
        buf <<= l;
        nb -= l;
        out[i] = sym ? (int32_t)sym - (int32_t)R : 0;
    }
}

__global__ void __launch_bounds__(256) k_scatter(DevParams* par, const uint8_t* __restrict__ blob,
                                                 int32_t* out, uint64_t n) {
    if (par->flags & kFlagError) return;
    const uint32_t no = par->d_nout;
    const uint2* ol = reinterpret_cast<const uint2*>(blob + par->off_ou);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < no; i += gridDim.x * blockDim.x) {
        const uint2 e = ol[i];
        if (e.x >= n) { set_error(par, FPSNR_ECORRUPT); return; }
        out[e.x] = (int32_t)e.y;
    }
}

__global__ void __launch_bounds__(256) k_patch(DevParams* par, const uint8_t* __restrict__ blob,
                                               float* out, uint64_t n) {
    if (par->flags & kFlagError) return;
    const uint32_t nv = par->d_nvb;
    const uint2* vl = reinterpret_cast<const uint2*>(blob + par->off_vb);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
        const uint2 e = vl[i];
        if (e.x >= n) { set_error(par, FPSNR_ECORRUPT); return; }
        out[e.x] = __uint_as_float(e.y);
    }
}

__global__ void k_status(const DevParams* par, int* status) { *status = par->status; }

// ---------------------------------------------------------------------------
// decoupled look-back helpers
// ---------------------------------------------------------------------------

constexpr uint32_t kStA = 1u, kStP = 2u;

// Waits (bounded) for tile `p` of this epoch to publish; returns its state
// (kStA or kStP), or 0 after a timeout (the tile then counts as zero).
__device__ __forceinline__ uint32_t wait_flag(const uint32_t* flags, uint64_t p, uint32_t epoch,
                                              DevParams* par) {
    for (uint32_t it = 0; it < kSpinLimit; it++) {
        const uint32_t f = ld_acquire(flags + p);
        if ((f >> 2) == epoch && (f & 3u)) return f & 3u;
        __nanosleep(64);
    }
    set_error(par, FPSNR_ETIMEOUT);
    return 0;
}

struct ScanArgs {
    DevParams* par;
    uint32_t* data;
    uint32_t A, L, B;       // (outer, scan length, inner)
    uint32_t nbt;           // strided: column tiles
    uint32_t tpr;           // contiguous: tiles per row
    uint32_t tiles;
    uint32_t* flags;        // [tiles]
    uint32_t* agg;          // [tiles * width]
    uint32_t* inc;          // [tiles * width]
    uint32_t* ctr;          // [2]: tile counter, done counter
    uint32_t epoch;
};

__device__ __forceinline__ void tile_done(uint32_t* ctr, uint32_t tiles) {
    if (atomicAdd(ctr + 1, 1u) == tiles - 1) {
        ctr[0] = 0;
        ctr[1] = 0;
    }
}

// Contiguous rows: each tile is 256*IPT consecutive points of one row.
template <int IPT, bool FINAL, bool VEC>
__global__ void __launch_bounds__(256) k_scan_contig(ScanArgs a) {
    __shared__ uint32_t sh[33];
    __shared__ uint32_t s_id, s_carry;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) s_id = atomicAdd(a.ctr, 1u);
    __syncthreads();
    const uint32_t id = s_id;
    const uint32_t row = id / a.tpr, t = id % a.tpr;
    const uint32_t W = a.L;
    const uint64_t rbase = (uint64_t)row * W;
    const uint32_t c0 = t * (256u * IPT) + tid * IPT;
    uint32_t v[IPT];
    if (VEC && c0 + IPT <= W) {
#pragma unroll
        for (int k = 0; k < IPT; k += 4) {
            uint4 q = *reinterpret_cast<const uint4*>(a.data + rbase + c0 + k);
            v[k] = q.x; v[k + 1] = q.y; v[k + 2] = q.z; v[k + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < IPT; k++) v[k] = (c0 + k < W) ? a.data[rbase + c0 + k] : 0u;
    }
#pragma unroll
    for (int k = 1; k < IPT; k++) v[k] += v[k - 1];
    uint32_t agg;
    const uint32_t ex = block_excl_scan(v[IPT - 1], sh, &agg);
    uint32_t carry = 0;
    if (a.tpr > 1) {
        if (tid == 0) {
            if (t == 0) {
                a.inc[id] = agg;
                __threadfence();
                st_release(a.flags + id, (a.epoch << 2) | kStP);
            } else {
                a.agg[id] = agg;
                __threadfence();
                st_release(a.flags + id, (a.epoch << 2) | kStA);
                uint64_t p = id - 1;
                for (;;) {
                    const uint32_t st = wait_flag(a.flags, p, a.epoch, a.par);
                    if (st == kStP) { carry += __ldcg(a.inc + p); break; }
                    if (st == 0) break;
                    carry += __ldcg(a.agg + p);
                    p--;
                }
                a.inc[id] = carry + agg;
                __threadfence();
                st_release(a.flags + id, (a.epoch << 2) | kStP);
            }
            s_carry = carry;
        }
        __syncthreads();
        carry = s_carry;
    }
    const uint32_t add = ex + carry;
    if (FINAL) {
        const DevParams* par = a.par;
        const float s = par->s, xmin = par->xmin;
        float* outf = reinterpret_cast<float*>(a.data);
        float f[IPT];
#pragma unroll
        for (int k = 0; k < IPT; k++) f[k] = __fmaf_rn(__int2float_rn((int32_t)(v[k] + add)), s, xmin);
        if (VEC && c0 + IPT <= W) {
#pragma unroll
            for (int k = 0; k < IPT; k += 4)
                *reinterpret_cast<float4*>(outf + rbase + c0 + k) = make_float4(f[k], f[k + 1], f[k + 2], f[k + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < IPT; k++)
                if (c0 + k < W) outf[rbase + c0 + k] = f[k];
        }
    } else {
        if (VEC && c0 + IPT <= W) {
#pragma unroll
            for (int k = 0; k < IPT; k += 4)
                *reinterpret_cast<uint4*>(a.data + rbase + c0 + k) =
                    make_uint4(v[k] + add, v[k + 1] + add, v[k + 2] + add, v[k + 3] + add);
        } else {
#pragma unroll
            for (int k = 0; k < IPT; k++)
                if (c0 + k < W) a.data[rbase + c0 + k] = v[k] + add;
        }
    }
    if (tid == 0) tile_done(a.ctr, a.tiles);
}

// Strided scan along the middle axis of (A, L, B): a tile is SEG consecutive
// rows of the scan axis by 256*CPT consecutive inner columns.
template <int SEG, int CPT, bool FINAL>
__global__ void __launch_bounds__(256) k_scan_strided(ScanArgs a) {
    constexpr uint32_t TB = 256u * CPT;
    __shared__ uint32_t s_id, s_st;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) s_id = atomicAdd(a.ctr, 1u);
    __syncthreads();
    const uint32_t id = s_id;
    const uint32_t bt = id % a.nbt;
    const uint32_t oa = (id / a.nbt) % a.A;
    const uint32_t seg = id / (a.nbt * a.A);
    const uint32_t col = bt * TB + tid * CPT;
    const uint32_t r0 = seg * SEG;
    const bool colin = col < a.B;  // CPT divides B when CPT > 1
    uint32_t v[SEG][CPT];
#pragma unroll
    for (int r = 0; r < SEG; r++) {
        const uint32_t row = r0 + r;
        const uint64_t off = ((uint64_t)oa * a.L + row) * a.B + col;
        if (colin && row < a.L) {
            if (CPT == 4) {
                uint4 q = *reinterpret_cast<const uint4*>(a.data + off);
                v[r][0] = q.x; v[r][CPT > 1 ? 1 : 0] = q.y; v[r][CPT > 2 ? 2 : 0] = q.z; v[r][CPT > 3 ? 3 : 0] = q.w;
            } else {
#pragma unroll
                for (int k = 0; k < CPT; k++) v[r][k] = a.data[off + k];
            }
        } else {
#pragma unroll
            for (int k = 0; k < CPT; k++) v[r][k] = 0u;
        }
    }
#pragma unroll
    for (int r = 1; r < SEG; r++)
#pragma unroll
        for (int k = 0; k < CPT; k++) v[r][k] += v[r - 1][k];
    uint32_t carry[CPT];
#pragma unroll
    for (int k = 0; k < CPT; k++) carry[k] = 0;
    const uint64_t vb = (uint64_t)id * TB + tid * CPT;
    if (seg == 0) {
#pragma unroll
        for (int k = 0; k < CPT; k++) a.inc[vb + k] = v[SEG - 1][k];
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(a.flags + id, (a.epoch << 2) | kStP);
    } else {
#pragma unroll
        for (int k = 0; k < CPT; k++) a.agg[vb + k] = v[SEG - 1][k];
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(a.flags + id, (a.epoch << 2) | kStA);
        const uint32_t step = a.nbt * a.A;
        uint64_t p = id;
        for (;;) {
            p -= step;
            if (tid == 0) s_st = wait_flag(a.flags, p, a.epoch, a.par);
            __syncthreads();
            const uint32_t st = s_st;
            __syncthreads();
            if (st == 0) break;
            const uint32_t* src = (st == kStP) ? a.inc : a.agg;
            const uint64_t pb = p * TB + tid * CPT;
#pragma unroll
            for (int k = 0; k < CPT; k++) carry[k] += __ldcg(src + pb + k);
            if (st == kStP) break;
        }
#pragma unroll
        for (int k = 0; k < CPT; k++) a.inc[vb + k] = carry[k] + v[SEG - 1][k];
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(a.flags + id, (a.epoch << 2) | kStP);
    }
    const DevParams* par = a.par;
    const float s = par->s, xmin = par->xmin;
#pragma unroll
    for (int r = 0; r < SEG; r++) {
        const uint32_t row = r0 + r;
        if (!colin || row >= a.L) continue;
        const uint64_t off = ((uint64_t)oa * a.L + row) * a.B + col;
        if (FINAL) {
            float* outf = reinterpret_cast<float*>(a.data);
            float f[CPT];
#pragma unroll
            for (int k = 0; k < CPT; k++)
                f[k] = __fmaf_rn(__int2float_rn((int32_t)(v[r][k] + carry[k])), s, xmin);
            if (CPT == 4)
                *reinterpret_cast<float4*>(outf + off) =
                    make_float4(f[0], f[CPT > 1 ? 1 : 0], f[CPT > 2 ? 2 : 0], f[CPT > 3 ? 3 : 0]);
            else
#pragma unroll
                for (int k = 0; k < CPT; k++) outf[off + k] = f[k];
        } else {
            if (CPT == 4)
                *reinterpret_cast<uint4*>(a.data + off) =
                    make_uint4(v[r][0] + carry[0], v[r][CPT > 1 ? 1 : 0] + carry[CPT > 1 ? 1 : 0],
                               v[r][CPT > 2 ? 2 : 0] + carry[CPT > 2 ? 2 : 0],
                               v[r][CPT > 3 ? 3 : 0] + carry[CPT > 3 ? 3 : 0]);
            else
#pragma unroll
                for (int k = 0; k < CPT; k++) a.data[off + k] = v[r][k] + carry[k];
        }
    }
    if (tid == 0) tile_done(a.ctr, a.tiles);
}

// ---------------------------------------------------------------------------
// host launcher
// ---------------------------------------------------------------------------

template <int IPT, bool FINAL>
static void launch_contig_t(const ScanArgs& a, bool vec, cudaStream_t st) {
    if (vec) k_scan_contig<IPT, FINAL, true><<<a.tiles, 256, 0, st>>>(a);
    else k_scan_contig<IPT, FINAL, false><<<a.tiles, 256, 0, st>>>(a);
}

template <bool FINAL>
static void launch_contig(const ScanArgs& a, int ipt, bool vec, cudaStream_t st) {
    if (ipt == 4) launch_contig_t<4, FINAL>(a, vec, st);
    else if (ipt == 8) launch_contig_t<8, FINAL>(a, vec, st);
    else launch_contig_t<16, FINAL>(a, vec, st);
}

int launch_decompress(fpsnr_plan_s* p, const void* d_blob, uint64_t bytes, float* d_out,
                      int* d_status, cudaStream_t st) {
    const Workspace& w = p->w;
    const uint8_t* blob = reinterpret_cast<const uint8_t*>(d_blob);
    {
    StageScope sc(p->prof, kStDsetup, st);
    k_dsetup<<<1, 1024, 0, st>>>(w.par, blob, bytes, p->ndim, p->ld, p->dims[0], p->dims[1],
                                 p->dims[2], p->n, (uint32_t)p->chunk, p->nchunks, w.dlut, w.dsyms);
    }
    if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA;
    if (p->n > 0) {
        int32_t* out = reinterpret_cast<int32_t*>(d_out);
        const unsigned gdec = (unsigned)((p->nchunks + 255) / 256);
        {
        StageScope sc(p->prof, kStDecode, st);
        k_decode<<<gdec, 256, 0, st>>>(w.par, blob, w.dlut, w.dsyms, out, p->n, (uint32_t)p->chunk,
                                       p->nchunks);
        }
        {
        StageScope sc(p->prof, kStScatter, st);
        k_scatter<<<(unsigned)p->sm_count, 256, 0, st>>>(w.par, blob, out, p->n);
        }
        if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA;
        p->epoch = (p->epoch + 1) & 0x3fffffffu;
        if (p->epoch == 0) p->epoch = 1;
        for (int i = 0; i < p->n_passes; i++) {
            const ScanPass& sp = p->pass[i];
            ScanArgs a;
            a.par = w.par;
            a.data = reinterpret_cast<uint32_t*>(d_out);
            a.A = sp.A;
            a.L = sp.L;
            a.B = sp.B;
            a.tiles = sp.tiles;
            a.flags = w.lb_flags + sp.val_off;
            a.agg = w.lb_vals + sp.val_off * p->lb_width;
            a.inc = w.lb_vals + (p->lb_tiles_total + sp.val_off) * p->lb_width;
            a.ctr = w.lb_ctr + 2 * sp.ctr_slot;
            a.epoch = p->epoch;
            StageScope sc(p->prof, sp.final_pass ? kStScanFinal : (i == 0 ? kStScanX : kStScanY), st);
            if (sp.kind == 0) {
                a.tpr = (sp.L + 256u * sp.ipt - 1) / (256u * sp.ipt);
                a.nbt = 1;
                if (sp.final_pass) launch_contig<true>(a, sp.ipt, sp.vec, st);
                else launch_contig<false>(a, sp.ipt, sp.vec, st);
            } else {
                a.tpr = 1;
                a.nbt = (sp.B + sp.tb - 1) / sp.tb;
                if (sp.vec) {
                    if (sp.final_pass) k_scan_strided<16, 4, true><<<sp.tiles, 256, 0, st>>>(a);
                    else k_scan_strided<16, 4, false><<<sp.tiles, 256, 0, st>>>(a);
                } else {
                    if (sp.final_pass) k_scan_strided<16, 1, true><<<sp.tiles, 256, 0, st>>>(a);
                    else k_scan_strided<16, 1, false><<<sp.tiles, 256, 0, st>>>(a);
                }
            }
            if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA;
        }
        StageScope sc(p->prof, kStPatch, st);
        k_patch<<<(unsigned)p->sm_count, 256, 0, st>>>(w.par, blob, d_out, p->n);
    }
    if (d_status) k_status<<<1, 1, 0, st>>>(w.par, d_status);
    return cudaGetLastError() == cudaSuccess ? FPSNR_OK : FPSNR_ECUDA;
}

}  // namespace fp
