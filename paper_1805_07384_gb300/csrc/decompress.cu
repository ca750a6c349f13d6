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
#include <algorithm>

#include "common.cuh"

namespace fp {

__device__ __forceinline__ uint32_t rd32(const uint8_t* b, uint64_t o) {
    return *reinterpret_cast<const uint32_t*>(b + o);
}
__device__ __forceinline__ uint64_t rd64(const uint8_t* b, uint64_t o) {
    return *reinterpret_cast<const uint64_t*>(b + o);
}
static __device__ __forceinline__ uint64_t pad16d(uint64_t b) { return (b + 15u) & ~(uint64_t)15u; }

struct DsetupArgs {
    DevParams* par;
    const uint8_t* blob;
    uint64_t bytes;
    int ndim, ld;
    uint64_t d0, d1, d2, n;
    uint32_t chunk;
    uint64_t nchunks;
    uint32_t* lut;
    uint16_t* syms;
    uint32_t* lb_ctr;
};

// one block per field
__global__ void __launch_bounds__(1024) k_dsetup(const __grid_constant__ Batch<DsetupArgs> B) {
    const DsetupArgs& A = B.a[blockIdx.x];
    DevParams* par = A.par;
    const uint8_t* __restrict__ blob = A.blob;
    const uint64_t bytes = A.bytes;
    const int ndim = A.ndim, ld = A.ld;
    const uint64_t d0 = A.d0, d1 = A.d1, d2 = A.d2, n = A.n;
    const uint32_t chunk = A.chunk;
    const uint64_t nchunks = A.nchunks;
    uint32_t* lut = A.lut;
    uint16_t* syms = A.syms;
    uint32_t* lb_ctr = A.lb_ctr;
    __shared__ int s_ok;
    __shared__ uint32_t s_cnt[32];
    __shared__ unsigned long long s_kraft;
    const uint32_t tid = threadIdx.x;
    // the scans' tile counters start every call at zero (see k_scan_contig)
    if (tid < 8) lb_ctr[tid] = 0;
    if (tid == 0) {
        const uint32_t e = (par->dec_epoch + 1) & 0x3fffffffu;
        par->dec_epoch = e ? e : 1u;
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
    __syncthreads();
    if (par->flags & kFlagError) return;
    // every table entry v (the next kLutBits bits) finds its code length as the
    // first length whose canonical range ends above v (ranges are contiguous and
    // ascending); prefixes of longer codes get 0
    const uint32_t lm = min(lmax, (uint32_t)kLutBits);
    for (uint32_t v = tid; v < (1u << kLutBits); v += blockDim.x) {
        const unsigned long long w = (unsigned long long)v << (32 - kLutBits);
        uint32_t e = 0;
        for (uint32_t l = 1; l <= lm; l++) {
            const unsigned long long lje =
                (unsigned long long)(par->d_first_code[l] + par->d_count[l]) << (32 - l);
            if (w < lje) {
                const uint32_t code = v >> (kLutBits - l);
                const uint32_t k = code - par->d_first_code[l];
                if (k < par->d_count[l]) e = ((uint32_t)syms[par->d_first_index[l] + k] << 8) | l;
                break;
            }
        }
        lut[v] = e;
    }
}

// One thread decodes one chunk of `chunk` symbols into int32 residuals.  The
// block's chunks are consecutive, so their words form one contiguous range of
// the stream: the block copies it into shared memory with coalesced loads and
// every thread then reads its bits from there.  The serial chain per symbol is
// one look-up-table read plus a few shifts: the next stream word is fetched
// into a register ahead of the refill, 8 residuals are decoded into registers
// and written as two 16-byte stores into the thread's own chunk.  Codes longer
// than the table are located by comparing the left-justified window with the
// end of each length's canonical range.
constexpr int kDecThreads = 256;  // chunks per decode block
constexpr int kMaxDynSmem = 227 * 1024;

// STAGED = false (chunks too large for the window to fit shared memory): the
// words are read from global memory directly.
struct DecArgs {
    DevParams* par;
    const uint8_t* blob;
    const uint32_t* lut_g;
    const uint16_t* syms;
    int32_t* out;
    uint64_t n;
    uint32_t chunk;
    uint64_t nchunks;
    uint32_t win_cap;
};

template <bool STAGED, int THREADS>
__global__ void __launch_bounds__(THREADS) k_decode(const __grid_constant__ Batch<DecArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const DecArgs& A = B.a[fld];
    const uint32_t bid = blockIdx.x - B.off[fld];
    DevParams* par = A.par;
    const uint8_t* __restrict__ blob = A.blob;
    const uint32_t* __restrict__ lut_g = A.lut_g;
    const uint16_t* __restrict__ syms = A.syms;
    int32_t* __restrict__ out = A.out;
    const uint64_t n = A.n;
    const uint32_t chunk = A.chunk;
    const uint64_t nchunks = A.nchunks;
    const uint32_t win_cap = A.win_cap;
    extern __shared__ __align__(16) uint32_t dsw[];
    uint32_t* slut = dsw;                   // 1 << kLutBits entries
    uint32_t* sw = dsw + (1u << kLutBits);  // the block's stream words (from a 16-byte boundary)
    __shared__ uint32_t s_fc[32], s_fi[32];
    __shared__ unsigned long long s_lje[33];
    __shared__ uint32_t s_ws, s_we, s_bad;
    __shared__ __align__(8) unsigned long long s_mbar;
    const uint32_t flags = par->flags;
    if (flags & kFlagError) return;
    const bool cst = (flags & kFlagConstant) != 0;
    const uint64_t cb0 = (uint64_t)bid * THREADS;
    const uint64_t c = cb0 + threadIdx.x;
    const uint64_t cb1 = min(cb0 + THREADS, nchunks);
    if (cst) {
        if (c < nchunks) {
            const uint64_t beg = c * chunk, end = min(beg + chunk, n);
            for (uint64_t i = beg; i < end; i++) out[i] = 0;
        }
        return;
    }
    const uint32_t words = par->d_words;
    const uint32_t* tab = reinterpret_cast<const uint32_t*>(blob + par->off_ct);
    const uint32_t* stream = reinterpret_cast<const uint32_t*>(blob + par->off_st);
    if (threadIdx.x < 32) {
        const uint32_t l = threadIdx.x;
        s_fc[l] = par->d_first_code[l];
        s_fi[l] = par->d_first_index[l];
        // end of length l's codes, left-justified in 32 bits (2^32 once the code is complete)
        s_lje[l] = l ? (unsigned long long)(par->d_first_code[l] + par->d_count[l]) << (32 - l) : 0ull;
    }
    if (threadIdx.x == 0) {
        s_lje[32] = ~0ull;
        const uint32_t ws = tab[cb0];
        const uint32_t we = (cb1 < nchunks) ? tab[cb1] : words;
        // a non-monotone table cannot come from the encoder
        const bool bad = ws > we || we > words;
        if (bad) set_error(par, FPSNR_ECORRUPT);
        s_bad = bad;
        s_ws = bad ? 0 : ws;
        s_we = bad ? 0 : we;
        mbar_init(&s_mbar, 1);
    }
    __syncthreads();
    if (s_bad) return;
    const uint32_t ws = s_ws, we = s_we;
    // the window is staged only when it fits; otherwise this block reads global memory
    const bool staged = STAGED && (((we + 3u) & ~3u) - (ws & ~3u)) <= win_cap + 4u;
    // the look-up table and the 16-byte aligned cover of the window arrive by two
    // bulk copies (the stream section is padded to 16 bytes, so the cover stays in it)
    const uint32_t ws_al = ws & ~3u;
    const uint32_t win_bytes = staged ? (((we + 3u) & ~3u) - ws_al) * 4u : 0u;
    if (threadIdx.x == 0) {
        const uint32_t lut_bytes = (1u << kLutBits) * 4u;
        mbar_arrive_expect_tx(&s_mbar, lut_bytes + win_bytes);
        bulk_g2s(slut, lut_g, lut_bytes, &s_mbar);
        if (win_bytes) bulk_g2s(sw, stream + ws_al, win_bytes, &s_mbar);
    }
    if (!mbar_wait_bounded(&s_mbar, 0)) {
        // never expected; record it, let the copies land, then leave
        set_error(par, FPSNR_ETIMEOUT);
        mbar_wait_bounded(&s_mbar, 0);
        return;
    }
    if (c >= nchunks) return;
    const uint64_t beg = c * chunk;
    const uint32_t cnt = (uint32_t)(min(beg + chunk, n) - beg);
    const int32_t R = (int32_t)par->d_radius;
    const uint32_t lmax = par->d_lmax;
    const uint32_t w0 = tab[c];
    const uint32_t w1 = (c + 1 < nchunks) ? tab[c + 1] : words;
    if (w0 > w1 || w0 < ws || w1 > we) { set_error(par, FPSNR_ECORRUPT); return; }
    auto word = [&](uint32_t k) -> uint32_t { return staged ? sw[k - ws_al] : __ldg(stream + k); };
    uint64_t buf = 0;
    uint32_t nb = 0, wi = w0;
    // the next two words are always in flight (a global load takes several
    // refills' worth of symbols to arrive)
    uint32_t nxt = wi < w1 ? word(wi) : 0u;
    uint32_t nxt2 = wi + 1 < w1 ? word(wi + 1) : 0u;
    bool bad = false;
    // decodes one residual; sets `bad` on a malformed stream
    auto one = [&]() -> int32_t {
        if (nb <= 32 && wi < w1) {
            buf |= (uint64_t)nxt << (32 - nb);
            nb += 32;
            wi++;
            nxt = nxt2;
            nxt2 = wi + 1 < w1 ? word(wi + 1) : 0u;
        }
        const uint32_t e = slut[(uint32_t)(buf >> (64 - kLutBits))];
        uint32_t l = e & 0xffu, sym = e >> 8;
        if (l == 0) {
            const uint32_t w32 = (uint32_t)(buf >> 32);
            l = kLutBits + 1;
            while (l <= lmax && (unsigned long long)w32 >= s_lje[l]) l++;
            if (l > lmax) { bad = true; l = 0; sym = 0; }
            else sym = syms[s_fi[l] + ((w32 >> (32 - l)) - s_fc[l])];
        }
        if (l > nb) { bad = true; l = 0; }
        buf <<= l;
        nb -= l;
        return sym ? (int32_t)sym - R : 0;
    };
    int32_t* dst = out + beg;
    const uint32_t cnt8 = cnt & ~7u;
    for (uint32_t i = 0; i < cnt8; i += 8) {
        int32_t o[8];
#pragma unroll
        for (int k = 0; k < 8; k++) o[k] = one();
        if (bad) { set_error(par, FPSNR_ECORRUPT); return; }
        int4* d4 = reinterpret_cast<int4*>(dst + i);
        d4[0] = make_int4(o[0], o[1], o[2], o[3]);
        d4[1] = make_int4(o[4], o[5], o[6], o[7]);
    }
    for (uint32_t i = cnt8; i < cnt; i++) {
        const int32_t v = one();
        if (bad) { set_error(par, FPSNR_ECORRUPT); return; }
        dst[i] = v;
    }
}

struct SmallArgs {
    DevParams* par;
    const uint8_t* blob;
    void* out;
    uint64_t n;
    uint32_t G;       // blocks per field
    int* status;      // k_status only
};

__global__ void __launch_bounds__(256) k_scatter(const __grid_constant__ Batch<SmallArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const SmallArgs& A = B.a[fld];
    const uint32_t bid = blockIdx.x - B.off[fld];
    DevParams* par = A.par;
    if (par->flags & kFlagError) return;
    const uint32_t no = par->d_nout;
    const uint2* ol = reinterpret_cast<const uint2*>(A.blob + par->off_ou);
    int32_t* out = reinterpret_cast<int32_t*>(A.out);
    for (uint32_t i = bid * blockDim.x + threadIdx.x; i < no; i += A.G * blockDim.x) {
        const uint2 e = ol[i];
        if (e.x >= A.n) { set_error(par, FPSNR_ECORRUPT); return; }
        out[e.x] = (int32_t)e.y;
    }
}

__global__ void __launch_bounds__(256) k_patch(const __grid_constant__ Batch<SmallArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const SmallArgs& A = B.a[fld];
    const uint32_t bid = blockIdx.x - B.off[fld];
    DevParams* par = A.par;
    if (par->flags & kFlagError) return;
    const uint32_t nv = par->d_nvb;
    const uint2* vl = reinterpret_cast<const uint2*>(A.blob + par->off_vb);
    float* out = reinterpret_cast<float*>(A.out);
    for (uint32_t i = bid * blockDim.x + threadIdx.x; i < nv; i += A.G * blockDim.x) {
        const uint2 e = vl[i];
        if (e.x >= A.n) { set_error(par, FPSNR_ECORRUPT); return; }
        out[e.x] = __uint_as_float(e.y);
    }
}

// one thread per field
__global__ void k_status(const __grid_constant__ Batch<SmallArgs> B) {
    const SmallArgs& A = B.a[blockIdx.x];
    if (threadIdx.x == 0 && A.status) *A.status = A.par->status;
}

// ---------------------------------------------------------------------------
// decoupled look-back helpers
// ---------------------------------------------------------------------------

constexpr uint32_t kStA = 1u, kStP = 2u;

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
};

__device__ __forceinline__ void tile_done(uint32_t* ctr, uint32_t tiles) {
    if (atomicAdd(ctr + 1, 1u) == tiles - 1) {
        ctr[0] = 0;
        ctr[1] = 0;
    }
}

// Contiguous rows: each tile is 256*IPT consecutive points of one row.
template <int IPT, bool FINAL, bool VEC>
__global__ void __launch_bounds__(256) k_scan_contig(const __grid_constant__ Batch<ScanArgs> B) {
    const ScanArgs& a = B.a[batch_field(B.off, B.count, blockIdx.x)];
    __shared__ uint32_t sh[33];
    __shared__ uint32_t s_id, s_carry;
    const uint32_t tid = threadIdx.x;
    const uint32_t epoch = a.par->dec_epoch;
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
        if (tid < 32) {
            if (tid == 0) {
                if (t == 0) a.inc[id] = agg;
                else a.agg[id] = agg;
                __threadfence();
                st_release(a.flags + id, (epoch << 2) | (t == 0 ? kStP : kStA));
            }
            if (t > 0) {
                carry = warp_lookback(a.flags, a.agg, a.inc, id, id - t, epoch, a.par);
                if (tid == 0) {
                    a.inc[id] = carry + agg;
                    __threadfence();
                    st_release(a.flags + id, (epoch << 2) | kStP);
                }
            }
            if (tid == 0) s_carry = carry;
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
__global__ void __launch_bounds__(256) k_scan_strided(const __grid_constant__ Batch<ScanArgs> B) {
    const ScanArgs& a = B.a[batch_field(B.off, B.count, blockIdx.x)];
    constexpr uint32_t TB = 256u * CPT;
    __shared__ uint32_t s_id, s_st;
    const uint32_t tid = threadIdx.x;
    const uint32_t epoch = a.par->dec_epoch;
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
        if (tid == 0) st_release(a.flags + id, (epoch << 2) | kStP);
    } else {
#pragma unroll
        for (int k = 0; k < CPT; k++) a.agg[vb + k] = v[SEG - 1][k];
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(a.flags + id, (epoch << 2) | kStA);
        // warp 0 inspects up to 32 earlier segments of this column strip per round
        // trip; every thread then adds their vectors up to the nearest inclusive one
        const uint32_t step = a.nbt * a.A;
        int64_t shi = (int64_t)seg - 1;
        for (;;) {
            if (tid < 32) {
                const int64_t sp = shi - tid;
                const bool valid = sp >= 0;
                const uint64_t pt = valid ? (uint64_t)id - (uint64_t)(seg - sp) * step : 0;
                uint32_t st = 0;
                bool timeout = false;
                for (uint32_t it = 0;; it++) {
                    if (valid && st == 0) {
                        const uint32_t f = ld_acquire(a.flags + pt);
                        if ((f >> 2) == epoch && (f & 3u)) st = f & 3u;
                    }
                    if (__all_sync(0xffffffffu, !valid || st != 0)) break;
                    if (it >= kSpinLimit) { timeout = true; break; }
                    __nanosleep(32);
                }
                const uint32_t pmask = __ballot_sync(0xffffffffu, valid && st == kStP);
                const uint32_t nvalid = __popc(__ballot_sync(0xffffffffu, valid));
                if (tid == 0) {
                    if (timeout) set_error(a.par, FPSNR_ETIMEOUT);
                    // number of segments to add, and whether the last one is inclusive
                    s_st = timeout ? 0u : (pmask ? ((uint32_t)__ffs(pmask) | 0x80000000u) : nvalid);
                }
            }
            __syncthreads();
            const uint32_t code = s_st;
            __syncthreads();
            const uint32_t cnt = code & 0x7fffffffu;
            for (uint32_t j = 0; j < cnt; j++) {
                const uint64_t pt = (uint64_t)id - (uint64_t)(seg - (shi - (int64_t)j)) * step;
                const bool last_inc = (code & 0x80000000u) && j + 1 == cnt;
                const uint32_t* src = last_inc ? a.inc : a.agg;
                const uint64_t pb = pt * TB + tid * CPT;
#pragma unroll
                for (int k = 0; k < CPT; k++) carry[k] += __ldcg(src + pb + k);
            }
            if (code == 0u || (code & 0x80000000u)) break;
            shi -= 32;
            if (shi < 0) break;
        }
#pragma unroll
        for (int k = 0; k < CPT; k++) a.inc[vb + k] = carry[k] + v[SEG - 1][k];
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(a.flags + id, (epoch << 2) | kStP);
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
static void launch_contig_t(const Batch<ScanArgs>& b, uint32_t tiles, bool vec, cudaStream_t st) {
    if (vec) k_scan_contig<IPT, FINAL, true><<<tiles, 256, 0, st>>>(b);
    else k_scan_contig<IPT, FINAL, false><<<tiles, 256, 0, st>>>(b);
}

template <bool FINAL>
static void launch_contig(const Batch<ScanArgs>& b, uint32_t tiles, int ipt, bool vec,
                          cudaStream_t st) {
    if (ipt == 4) launch_contig_t<4, FINAL>(b, tiles, vec, st);
    else if (ipt == 8) launch_contig_t<8, FINAL>(b, tiles, vec, st);
    else launch_contig_t<16, FINAL>(b, tiles, vec, st);
}

// Shared-memory stream window of one decode block: room for its chunks at up
// to 16 bits per symbol (a chunk may need ceil(chunk * lmax / 32) words; a block
// whose window is larger reads its words from global memory instead).  Keeping
// the window small keeps several blocks resident per SM.
uint32_t decode_window_words(const fpsnr_plan_s* p) {
    const uint32_t bits = (uint32_t)std::min(p->lmax, 16);
    return (uint32_t)(kDecThreads * (((uint64_t)p->chunk * bits + 31) / 32));
}

// LUT + window + 4 words of slack for rounding the window to 16-byte bounds
int decode_smem_bytes(const fpsnr_plan_s* p) {
    return (int)(((1u << kLutBits) + decode_window_words(p) + 8) * 4);
}

// Largest dynamic shared memory the staged decoder can take on this device:
// the per-block opt-in limit minus the kernel's static shared memory.
static int decode_smem_limit() {
    static int limit = -1;
    if (limit < 0) {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, k_decode<false, kDecThreads>) != cudaSuccess)
            return 0;
        limit = std::min(kMaxDynSmem, optin - (int)fa.sharedSizeBytes);
    }
    return limit;
}

// The attribute belongs to the kernel, not to a plan: set it to the largest
// size any plan can ask for.
int decode_prepare(const fpsnr_plan_s*) { return decode_smem_limit() > 0 ? FPSNR_OK : FPSNR_ECUDA; }

static uint32_t small_blocks_d(const fpsnr_plan_s* p, int count) {
    const int g = std::max(1, p->sm_count / std::max(1, count));
    return (uint32_t)std::min(g, 64);
}

int launch_decompress_batch(fpsnr_plan_s* const* P, const void* const* d_blob,
                            const uint64_t* bytes, float* const* d_out, int* d_status, int count,
                            cudaStream_t st) {
    if (count <= 0) return FPSNR_OK;
    if (count > kMaxBatch) {
        for (int b0 = 0; b0 < count; b0 += kMaxBatch) {
            const int c = std::min(kMaxBatch, count - b0);
            int rc = launch_decompress_batch(P + b0, d_blob + b0, bytes + b0, d_out + b0,
                                             d_status ? d_status + b0 : nullptr, c, st);
            if (rc) return rc;
        }
        return FPSNR_OK;
    }
    fp::Profiler& prof = P[0]->prof;  // batched launches are attributed to the first plan
    uint32_t blocks[kMaxBatch];
    {
        Batch<DsetupArgs> b;
        b.count = (uint32_t)count;
        for (int f = 0; f < count; f++) {
            const fpsnr_plan_s* p = P[f];
            const Workspace& w = p->w;
            b.a[f] = DsetupArgs{w.par, reinterpret_cast<const uint8_t*>(d_blob[f]), bytes[f],
                                p->ndim, p->ld, p->dims[0], p->dims[1], p->dims[2], p->n,
                                (uint32_t)p->chunk, p->nchunks, w.dlut, w.dsyms, w.lb_ctr};
            b.off[f] = (uint32_t)f;
        }
        b.off[count] = (uint32_t)count;
        StageScope sc(prof, kStDsetup, st);
        k_dsetup<<<count, 1024, 0, st>>>(b);
        if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA;
    }
    // decode: one launch per (staged, shared-memory size) group
    {
        bool done[kMaxBatch] = {};
        for (int f0 = 0; f0 < count; f0++) {
            if (done[f0] || P[f0]->n == 0) continue;
            const int smem0 = decode_smem_bytes(P[f0]);
            Batch<DecArgs> b;
            b.count = 0;
            for (int f = f0; f < count; f++) {
                const fpsnr_plan_s* p = P[f];
                if (done[f] || p->n == 0 || decode_smem_bytes(p) != smem0) continue;
                done[f] = true;
                const Workspace& w = p->w;
                blocks[b.count] = (uint32_t)((p->nchunks + kDecThreads - 1) / kDecThreads);
                b.a[b.count++] = DecArgs{w.par, reinterpret_cast<const uint8_t*>(d_blob[f]), w.dlut,
                                         w.dsyms, reinterpret_cast<int32_t*>(d_out[f]), p->n,
                                         (uint32_t)p->chunk, p->nchunks, decode_window_words(p)};
            }
            const uint32_t tot = batch_offsets(b, blocks);
            StageScope sc(prof, kStDecode, st);
            // every thread streams its own chunk from global memory (two words in
            // flight); only the look-up table is staged in shared memory
            k_decode<false, kDecThreads><<<tot, kDecThreads, (1u << kLutBits) * 4 + 64, st>>>(b);
            if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA;
        }
    }
    Batch<SmallArgs> sb;
    sb.count = (uint32_t)count;
    for (int f = 0; f < count; f++) {
        const fpsnr_plan_s* p = P[f];
        sb.a[f] = SmallArgs{p->w.par, reinterpret_cast<const uint8_t*>(d_blob[f]), d_out[f], p->n,
                            small_blocks_d(p, count), d_status ? d_status + f : nullptr};
        blocks[f] = p->n ? sb.a[f].G : 0u;
    }
    const uint32_t small_tot = batch_offsets(sb, blocks);
    if (small_tot) {
        StageScope sc(prof, kStScatter, st);
        k_scatter<<<small_tot, 256, 0, st>>>(sb);
        if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA;
    }
    // inverse Lorenzo passes, grouped by pass index and kernel variant
    for (int i = 0; i < 3; i++) {
        bool done[kMaxBatch] = {};
        for (int f0 = 0; f0 < count; f0++) {
            const fpsnr_plan_s* p0 = P[f0];
            if (done[f0] || p0->n == 0 || p0->n_passes <= i) continue;
            const ScanPass& s0 = p0->pass[i];
            Batch<ScanArgs> b;
            b.count = 0;
            for (int f = f0; f < count; f++) {
                const fpsnr_plan_s* p = P[f];
                if (done[f] || p->n == 0 || p->n_passes <= i) continue;
                const ScanPass& sp = p->pass[i];
                if (sp.kind != s0.kind || sp.ipt != s0.ipt || sp.vec != s0.vec ||
                    sp.final_pass != s0.final_pass)
                    continue;
                done[f] = true;
                const Workspace& w = p->w;
                ScanArgs a;
                a.par = w.par;
                a.data = reinterpret_cast<uint32_t*>(d_out[f]);
                a.A = sp.A;
                a.L = sp.L;
                a.B = sp.B;
                a.tiles = sp.tiles;
                a.flags = w.lb_flags + sp.val_off;
                a.agg = w.lb_vals + sp.val_off * p->lb_width;
                a.inc = w.lb_vals + (p->lb_tiles_total + sp.val_off) * p->lb_width;
                a.ctr = w.lb_ctr + 2 * sp.ctr_slot;
                if (sp.kind == 0) {
                    a.tpr = (sp.L + 256u * sp.ipt - 1) / (256u * sp.ipt);
                    a.nbt = 1;
                } else {
                    a.tpr = 1;
                    a.nbt = (sp.B + sp.tb - 1) / sp.tb;
                }
                blocks[b.count] = sp.tiles;
                b.a[b.count++] = a;
            }
            const uint32_t tot = batch_offsets(b, blocks);
            StageScope sc(prof, s0.final_pass ? kStScanFinal : (i == 0 ? kStScanX : kStScanY), st);
            if (s0.kind == 0) {
                if (s0.final_pass) launch_contig<true>(b, tot, s0.ipt, s0.vec, st);
                else launch_contig<false>(b, tot, s0.ipt, s0.vec, st);
            } else if (s0.vec) {
                if (s0.final_pass) k_scan_strided<16, 4, true><<<tot, 256, 0, st>>>(b);
                else k_scan_strided<16, 4, false><<<tot, 256, 0, st>>>(b);
            } else {
                if (s0.final_pass) k_scan_strided<16, 1, true><<<tot, 256, 0, st>>>(b);
                else k_scan_strided<16, 1, false><<<tot, 256, 0, st>>>(b);
            }
            if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA;
        }
    }
    if (small_tot) {
        StageScope sc(prof, kStPatch, st);
        k_patch<<<small_tot, 256, 0, st>>>(sb);
        if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA;
    }
    if (d_status) {
        for (int f = 0; f < count; f++) sb.off[f] = (uint32_t)f;
        sb.off[count] = (uint32_t)count;
        k_status<<<count, 32, 0, st>>>(sb);
    }
    return cudaGetLastError() == cudaSuccess ? FPSNR_OK : FPSNR_ECUDA;
}

}  // namespace fp
