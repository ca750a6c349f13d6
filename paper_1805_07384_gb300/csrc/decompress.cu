// decompress.cu -- inverse of the compression chain (Sec. III: rebuild the
// prediction errors, then the data; Eq. 1 holds because the residuals are
// reproduced exactly).
//
//   k_dsetup        header validation against the plan, canonical decoding
//                   tables and a look-up table over the next kLutBits bits
//   k_decode        one thread per chunk, canonical Huffman decode into the
//                   16-bit symbols (the plan's symbol buffer): a bit-position
//                   window over three registers fed by a per-thread cp.async
//                   ring, codes in pairs through the table for fields whose
//                   codes are short
//   2D fields up to kBandMaxNx columns (reduce, then scan, over bands of rows):
//     k_band_sum    column sums of the residuals of every band
//     k_band_carry  exclusive prefix of those sums over the bands
//     k_band_scan   per band: the carry row's prefix along x seeds the column
//                   sums, then every row's prefix along x is added to them;
//                   dequantization x' = fmaf((float)q, s, xmin) (midpoint
//                   reconstruction, Sec. IV) is fused into the write
//   3D fields up to kVolMaxNx columns (tiles of 32 planes x a band of rows):
//     k_vol_sum     per tile: column sums per plane, slab sums per row, and
//                   the tile's column totals
//     k_vol_carry   exclusive prefixes of those sums over bands and slabs
//     k_vol_scan    per tile, plane by plane (planes staged by bulk copies):
//                   column prefix, then row prefix, dequantized on the write
//   other shapes (1D, wider 2D and 3D):
//     k_scan_contig   inclusive prefix sum along x (rows), decoupled look-back
//                     between tiles of one row; the first pass reads symbols
//     k_scan_strided  inclusive prefix sum along y or z, decoupled look-back
//                     between row segments; the last pass dequantizes
//   k_patch         verbatim points restored
//
// Symbol 0 marks an outlier.  After decoding, k_out_scatter checks the outlier
// list against the symbols (strictly increasing indices, each at a symbol 0)
// and writes every outlier's residual at its index in the caller's output
// buffer, which holds nothing else until the last pass writes the floats;
// every pass that turns symbols into residuals then reads an outlier's
// residual with one load, before the same thread writes that point.  The
// first such pass counts the symbols 0 and k_patch checks that there are as
// many as outliers.  The prefix sums run in modular uint32 arithmetic: intermediate
// partial sums may leave the int32 range, but every final lattice value is in
// [0, 2^31), so the modular result is exact.
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
    bool zr;  // the blob is the plan's unwrapped copy: its length and verdict are on the device
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
    const uint64_t bytes = A.zr ? par->zr_raw : A.bytes;
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
    if (tid == 0) par->d_zero = 0u;
    if (tid == 0) {
        const uint32_t e = (par->dec_epoch + 1) & 0x3fffffffu;
        par->dec_epoch = e ? e : 1u;
        // a container that failed to expand is corrupt whatever the copy holds
        const bool zr_bad = A.zr && par->zr_bad != 0u;
        if (A.zr) par->zr_bad = 0u;
        int ok = bytes >= kHeaderBytes && !zr_bad;
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
    // Table over the next kLutBits bits.  Canonical code ranges tile the
    // left-justified code space in order of length, so prefix v (a) holds one
    // whole code of length l <= kLutBits: entry (sym << 8) | l; (b) lies inside
    // the range of a single length l > kLutBits: entry kLutSlow | kLutLen | l
    // (the decoder finds the symbol from its canonical index); or (c) straddles
    // the ranges of several lengths or has no code: entry kLutSlow (the decoder
    // searches the range ends).  Case (c) holds for at most one prefix per
    // length boundary.
    for (uint32_t v = tid; v < (1u << kLutBits); v += blockDim.x) {
        const unsigned long long w = (unsigned long long)v << (32 - kLutBits);
        uint32_t e = kLutSlow;
        for (uint32_t l = 1; l <= lmax; l++) {
            const unsigned long long lje =
                (unsigned long long)(par->d_first_code[l] + par->d_count[l]) << (32 - l);
            if (w < lje) {
                if (l <= (uint32_t)kLutBits) {
                    const uint32_t code = v >> (kLutBits - l);
                    const uint32_t k = code - par->d_first_code[l];
                    if (k < par->d_count[l]) e = ((uint32_t)syms[par->d_first_index[l] + k] << 8) | l;
                } else if (w + (1ull << (32 - kLutBits)) <= lje) {
                    e = kLutSlow | kLutLen | l;
                }
                break;
            }
        }
        lut[v] = e;
    }
}

// One thread decodes one chunk of `chunk` symbols, reading the stream by bit
// position p: the next 32 bits are a funnel shift of the two words that hold
// bit p.  The thread keeps three consecutive words of its chunk in registers
// (a, b, c) and moves on by one word whenever p crosses a word boundary (no
// step takes more than 27 bits, the longest code).  The words come from a
// ring of kDecRing aligned quads in shared memory that cp.async fills three
// quads ahead of the one being read (an asynchronous copy holds no register,
// and shared memory per thread stays small whatever the stream's density).
// Codes go in pairs when the code's long lengths are rare: a table read over
// the next kLutBits bits gives the first code's length and symbol, a second
// read at the window shifted by that length gives the second's, and when both
// are whole codes of at most kLutBits bits (no kLutSlow flag) a byte permute
// packs both symbols.  Otherwise, and for every code of a field whose long
// codes are frequent, codes are decoded one by one: a longer code takes its
// symbol from its canonical index (kLutLen), and a prefix shared by several
// lengths is resolved by comparing the window with the end of each length's
// canonical range.  A chunk that consumes more bits than it owns, or meets a
// prefix no code has, is corrupt.
constexpr int kDecRing = 8;  // stream quads in a thread's ring (power of two)
// a field decodes codes in pairs when its mean code length, estimated as the
// sum over lengths l of l * count[l] * 2^-l (a code of l bits stands for a
// probability near 2^-l), is below this many bits
constexpr float kDecPairBits = 5.0f;

// Asynchronous 16-byte copy global -> shared memory through L2 (both 16-byte
// aligned), one commit group per copy, and waits on the thread's own groups.
__device__ __forceinline__ void cp_async16(uint32_t* dst, const uint32_t* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copies quad q of the stream into the ring slot it maps to (nothing past
// the section's qend quads) and closes a copy group.
template <int THREADS>
__device__ __forceinline__ void dec_issue(uint32_t* ring, const uint32_t* __restrict__ stream, uint32_t qend,
                                          uint32_t q) {
    if (q < qend) cp_async16(ring + (q & (kDecRing - 1)) * (4u * THREADS), stream + 4u * q);
    cp_async_commit();
}

// dynamic shared memory of a THREADS-wide decode block: the table, then the
// stream rings
constexpr uint32_t dec_smem(int threads) {
    return ((1u << kLutBits) + 4u * kDecRing * (uint32_t)threads) * 4u;
}
// blocks per SM that the shared memory admits (227 KB, 1 KB reserved a block)
constexpr int dec_min_blocks(int threads) { return (int)((227u * 1024u) / (dec_smem(threads) + 1536u)); }

struct DecArgs {
    DevParams* par;
    uint32_t spin_limit;  // polls of the table copy's mbarrier before giving up
    const uint8_t* blob;
    const uint32_t* lut_g;
    const uint16_t* syms;
    uint16_t* out;  // [n] decoded symbols
    uint64_t n;
    uint32_t chunk;
    uint64_t nchunks;
};

// Decodes the cnt symbols of the chunk that owns stream words [w0, w1) into
// dst; false when the chunk is corrupt (it reads past its words, or meets a
// prefix no code has).  ring is the thread's first ring word; quads of the
// 16-byte padded section end at qend.  The caller has issued quads
// w0 / 4 .. w0 / 4 + kDecRing - 1 (dec_issue), one copy group each.
// Every code step is free of branches but for rare long-code cases, so the
// lanes of a warp stay together: the window slides by a predicated move, and
// the ring is refilled once per group of 8 codes.  A group moves the window
// by at most 8 x 27 bits (7 words, 2 quads), so two copies per group keep the
// ring kDecRing - 1 quads ahead of the quad of word a, and the words a group
// reads (up to 9 words past a) lie in quads issued two groups earlier: all
// but the four newest copy groups have landed.
template <int THREADS, bool PAIRS>
__device__ __forceinline__ bool dec_chunk(uint32_t* ring, const uint32_t* __restrict__ stream, uint32_t qend,
                                          uint32_t w0, uint32_t w1, uint32_t cnt, uint16_t* __restrict__ dst,
                                          const uint32_t* __restrict__ lut, const uint32_t* __restrict__ base,
                                          const unsigned long long* __restrict__ lje,
                                          const uint16_t* __restrict__ syms, uint32_t lmax) {
    // word w of the stream sits in slot (w / 4) mod kDecRing of the ring
    auto word = [&](uint32_t w) -> uint32_t {
        return ring[((w >> 2) & (kDecRing - 1)) * (4u * THREADS) + (w & 3u)];
    };
    uint32_t qi = (w0 >> 2) + kDecRing - 1;  // last quad issued
    cp_async_wait<kDecRing - 2>();           // quads w0 / 4 and w0 / 4 + 1 landed
    uint32_t a = word(w0), b = word(w0 + 1), c = word(w0 + 2);
    uint32_t p = 0;   // bits consumed since word w0
    uint32_t wr = 0;  // a holds word w0 + wr
    bool bad = false;
    auto refill = [&]() {
        const uint32_t want = ((w0 + wr) >> 2) + kDecRing - 1;
#pragma unroll
        for (int r = 0; r < 2; r++) {
            if (qi < want) {
                qi++;
                if (qi < qend) cp_async16(ring + (qi & (kDecRing - 1)) * (4u * THREADS), stream + 4u * qi);
            }
            cp_async_commit();
        }
        cp_async_wait<4>();
    };
    // p moved by at most 27 bits: slide the three words along by at most one
    auto step = [&]() {
        const bool cross = (p >> 5) != wr;
        wr += cross ? 1u : 0u;
        a = cross ? b : a;
        b = cross ? c : b;
        if (cross) c = word(w0 + wr + 2);
    };
    // one code of any length
    auto one = [&]() -> uint32_t {
        const uint32_t win = __funnelshift_l(b, a, p);  // bits p .. p + 31 of the chunk
        const uint32_t e = lut[win >> (32 - kLutBits)];
        uint32_t l = e & 31u;
        uint32_t sym = e >> 8;
        if (e == kLutSlow) {
            // a prefix shared by several lengths (or by none): the first length
            // whose canonical range ends above the window, by a fixed number of
            // bisection steps over kLutBits + 1 .. lmax
            uint32_t lo = kLutBits + 1, hi = lmax;
            bad |= (unsigned long long)win >= lje[lmax];  // no code has this prefix
#pragma unroll
            for (int it = 0; it < 5; it++) {
                if (lo < hi) {
                    const uint32_t m = (lo + hi) >> 1;
                    if ((unsigned long long)win < lje[m]) hi = m;
                    else lo = m + 1;
                }
            }
            l = lo;
        }
        // a code longer than kLutBits bits: its symbol from its canonical index,
        // off the dependency chain of the next code's position
        if (e & kLutSlow) sym = __ldg(&syms[(base[l] + (win >> (32 - l))) & 0xffffu]);
        p += l;
        step();
        return sym;
    };
    const uint32_t cnt8 = cnt & ~7u;
    uint4 prev = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t i = 0; i < cnt8; i += 8) {
        refill();
        uint32_t s[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if constexpr (PAIRS) {
                const uint32_t win = __funnelshift_l(b, a, p);
                const uint32_t e1 = lut[win >> (32 - kLutBits)];
                const uint32_t e2 = lut[(win << (e1 & 31u)) >> (32 - kLutBits)];
                if (((e1 | e2) & kLutSlow) == 0u) {
                    s[k] = __byte_perm(e1, e2, 0x6521);  // bits 8..23 of each entry
                    p += (e1 & 31u) + (e2 & 31u);
                    step();
                    continue;
                }
            }
            const uint32_t s0 = one();
            s[k] = s0 | (one() << 16);
        }
        // each group is stored after the next one is decoded: the symbol loads of
        // long codes land meanwhile
        if (i) *reinterpret_cast<uint4*>(dst + i - 8) = prev;
        prev = make_uint4(s[0], s[1], s[2], s[3]);
    }
    if (cnt8) *reinterpret_cast<uint4*>(dst + cnt8 - 8) = prev;
    if (cnt8 < cnt) {
        refill();
        for (uint32_t i = cnt8; i < cnt; i++) dst[i] = (uint16_t)one();
    }
    return !bad && p <= 32u * (w1 - w0);
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, dec_min_blocks(THREADS)) k_decode(const __grid_constant__ Batch<DecArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const DecArgs& A = B.a[fld];
    const uint32_t bid = blockIdx.x - B.off[fld];
    DevParams* par = A.par;
    const uint64_t n = A.n;
    const uint32_t chunk = A.chunk;
    const uint64_t nchunks = A.nchunks;
    extern __shared__ __align__(16) uint32_t slut[];  // decode table, then the stream rings
    __shared__ uint32_t s_base[32];  // first index - first code of every length (mod 2^32)
    __shared__ unsigned long long s_lje[33];
    __shared__ uint32_t s_pairs;     // codes longer than kLutBits bits are rare
    __shared__ __align__(8) unsigned long long s_mbar;
    // constant fields have no stream: their residuals are all zero
    if (par->flags & (kFlagError | kFlagConstant)) return;
    const uint32_t words = par->d_words;
    const uint32_t* __restrict__ tab = reinterpret_cast<const uint32_t*>(A.blob + par->off_ct);
    const uint32_t* __restrict__ stream = reinterpret_cast<const uint32_t*>(A.blob + par->off_st);
    // the chunk's first quads are in flight while the block sets up its table
    const uint64_t c = (uint64_t)bid * THREADS + threadIdx.x;
    const bool live = c < nchunks;
    uint32_t w0 = 0u, w1 = 0u;
    bool sane = false;
    uint32_t* ring = slut + (1u << kLutBits) + 4u * threadIdx.x;
    const uint32_t qend = (words + 3u) >> 2;  // quads in the 16-byte padded section
    if (live) {
        w0 = tab[c];
        w1 = (c + 1 < nchunks) ? tab[c + 1] : words;
        // (a chunk owns fewer than 2^22 words: 65536 codes of <= 27 bits)
        sane = w0 <= w1 && w1 <= words && w1 - w0 < (1u << 22);
        if (sane) {
#pragma unroll
            for (uint32_t r = 0; r < (uint32_t)kDecRing; r++) dec_issue<THREADS>(ring, stream, qend, (w0 >> 2) + r);
        }
    }
    if (threadIdx.x < 32) {
        const uint32_t l = threadIdx.x;
        const uint32_t cl = par->d_count[l];
        s_base[l] = par->d_first_index[l] - par->d_first_code[l];
        // end of length l's codes, left-justified in 32 bits (2^32 once the code is complete)
        s_lje[l] = l ? (unsigned long long)(par->d_first_code[l] + cl) << (32 - l) : 0ull;
        float m = ldexpf((float)(cl * l), -(int)l);
#pragma unroll
        for (int o = 16; o; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
        if (l == 0) s_pairs = m < kDecPairBits;
    }
    if (threadIdx.x == 0) {
        s_lje[32] = ~0ull;
        mbar_init(&s_mbar, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t lut_bytes = (1u << kLutBits) * 4u;
        mbar_arrive_expect_tx(&s_mbar, lut_bytes);
        bulk_g2s(slut, A.lut_g, lut_bytes, &s_mbar);
    }
    if (!mbar_wait_bounded(&s_mbar, 0, A.spin_limit)) {
        // never expected; record it, let the copies land (bounded), then leave
        set_error(par, FPSNR_ETIMEOUT);
        mbar_wait_bounded(&s_mbar, 0);
        cp_async_wait<0>();
        return;
    }
    if (!live) return;
    if (!sane) {
        set_error(par, FPSNR_ECORRUPT);
        return;
    }
    const uint64_t beg = c * chunk;
    const uint32_t cnt = (uint32_t)(min(beg + chunk, n) - beg);
    const bool ok = s_pairs ? dec_chunk<THREADS, true>(ring, stream, qend, w0, w1, cnt, A.out + beg, slut, s_base,
                                                        s_lje, A.syms, par->d_lmax)
                            : dec_chunk<THREADS, false>(ring, stream, qend, w0, w1, cnt, A.out + beg, slut, s_base,
                                                         s_lje, A.syms, par->d_lmax);
    // copies still in flight land before the block's shared memory is released
    cp_async_wait<0>();
    if (!ok) set_error(par, FPSNR_ECORRUPT);
}

// Residual of point `idx` from its symbol: code - R, or for symbol 0 (an
// outlier) the residual k_out_scatter placed at idx.
__device__ __forceinline__ uint32_t residual_of(uint32_t code, uint32_t R, uint32_t idx,
                                                const uint32_t* __restrict__ od) {
    return code ? code - R : od[idx];
}

// Loads IPT consecutive 16-bit values (IPT a multiple of 4; p 8-byte aligned,
// and 16-byte aligned when IPT >= 8).
template <int IPT>
__device__ __forceinline__ void load_syms(const uint16_t* __restrict__ p, uint32_t (&v)[IPT]) {
    if constexpr (IPT == 4) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        v[0] = q.x & 0xffffu; v[1] = q.x >> 16; v[2] = q.y & 0xffffu; v[3] = q.y >> 16;
    } else {
#pragma unroll
        for (int k = 0; k < IPT; k += 8) {
            const uint4 q = *reinterpret_cast<const uint4*>(p + k);
            v[k] = q.x & 0xffffu; v[k + 1] = q.x >> 16;
            v[k + 2] = q.y & 0xffffu; v[k + 3] = q.y >> 16;
            v[k + 4] = q.z & 0xffffu; v[k + 5] = q.z >> 16;
            v[k + 6] = q.w & 0xffffu; v[k + 7] = q.w >> 16;
        }
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

__global__ void __launch_bounds__(256) k_patch(const __grid_constant__ Batch<SmallArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const SmallArgs& A = B.a[fld];
    const uint32_t bid = blockIdx.x - B.off[fld];
    DevParams* par = A.par;
    if (par->flags & kFlagError) return;
    // every symbol 0 had an outlier entry: as many of them as entries
    if (bid == 0 && threadIdx.x == 0 && par->d_zero != par->d_nout) set_error(par, FPSNR_ECORRUPT);
    const uint32_t nv = par->d_nvb;
    const uint2* vl = reinterpret_cast<const uint2*>(A.blob + par->off_vb);
    float* out = reinterpret_cast<float*>(A.out);
    for (uint32_t i = bid * blockDim.x + threadIdx.x; i < nv; i += A.G * blockDim.x) {
        const uint2 e = vl[i];
        if (e.x >= A.n) { set_error(par, FPSNR_ECORRUPT); return; }
        out[e.x] = __uint_as_float(e.y);
    }
}

struct ScatterArgs {
    DevParams* par;
    const uint8_t* blob;
    const uint16_t* syms;  // decoded symbols
    uint32_t* od;          // the caller's output buffer: outlier residuals at their indices
    uint64_t n;
    uint32_t G;            // blocks per field
};

// Outlier residuals placed at their point indices, after checking the list
// against the decoded symbols; any mismatch means the blob is corrupt.
__global__ void __launch_bounds__(256) k_out_scatter(const __grid_constant__ Batch<ScatterArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const ScatterArgs& A = B.a[fld];
    const uint32_t bid = blockIdx.x - B.off[fld];
    DevParams* par = A.par;
    if (par->flags & (kFlagError | kFlagConstant)) return;
    const uint32_t no = par->d_nout;
    const uint2* __restrict__ ol = reinterpret_cast<const uint2*>(A.blob + par->off_ou);
    for (uint32_t i = bid * blockDim.x + threadIdx.x; i < no; i += A.G * blockDim.x) {
        const uint2 e = ol[i];
        const bool ok = e.x < A.n && (i + 1 == no || e.x < ol[i + 1].x) && A.syms[e.x] == 0;
        if (!ok) {
            set_error(par, FPSNR_ECORRUPT);
            return;
        }
        A.od[e.x] = e.y;
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
    uint32_t* data;         // int32 lattice values in the output buffer (later passes)
    const uint16_t* syms;   // decoded symbols (first pass)
    const uint8_t* blob;    // outlier list (first pass)
    uint32_t A, L, B;       // (outer, scan length, inner)
    uint32_t nbt;           // strided: column tiles
    uint32_t tpr;           // contiguous: tiles per row
    uint32_t tiles;
    uint32_t* flags;        // [tiles]
    uint32_t* agg;          // [tiles * width]
    uint32_t* inc;          // [tiles * width]
    uint32_t* ctr;          // [2]: tile counter, done counter
    uint32_t spin_limit;    // polls per look-back round trip before giving up
    uint32_t skew;          // 0; a test sets 1: predecessors are awaited under an epoch never published
};

__device__ __forceinline__ void tile_done(uint32_t* ctr, uint32_t tiles) {
    if (atomicAdd(ctr + 1, 1u) == tiles - 1) {
        ctr[0] = 0;
        ctr[1] = 0;
    }
}

// Contiguous rows: each tile is 256*IPT consecutive points of one row.  SYM:
// the input is the decoded symbols (first pass), else int32 values in place.
template <int IPT, bool FINAL, bool VEC, bool SYM>
__global__ void __launch_bounds__(256) k_scan_contig(const __grid_constant__ Batch<ScanArgs> B) {
    const ScanArgs& a = B.a[batch_field(B.off, B.count, blockIdx.x)];
    __shared__ uint32_t sh[33];
    __shared__ uint32_t s_id, s_carry;
    const uint32_t tid = threadIdx.x;
    DevParams* par = a.par;
    const uint32_t epoch = par->dec_epoch;
    if (tid == 0) s_id = atomicAdd(a.ctr, 1u);
    __syncthreads();
    const uint32_t id = s_id;
    const uint32_t row = id / a.tpr, t = id % a.tpr;
    const uint32_t W = a.L;
    const uint64_t rbase = (uint64_t)row * W;
    const uint32_t c0 = t * (256u * IPT) + tid * IPT;
    uint32_t v[IPT];
    if (SYM) {
        const uint32_t flags = par->flags;
        if (flags & kFlagConstant) {
#pragma unroll
            for (int k = 0; k < IPT; k++) v[k] = 0u;
        } else {
            const uint32_t R = par->d_radius;
            const uint32_t* od = a.data;  // outlier residuals, read before this thread writes
            uint32_t nzero = 0;           // symbols 0, checked against the list by k_patch
            if (VEC && c0 + IPT <= W) {
                load_syms<IPT>(a.syms + rbase + c0, v);
#pragma unroll
                for (int k = 0; k < IPT; k++) {
                    nzero += v[k] == 0u;
                    v[k] = residual_of(v[k], R, (uint32_t)(rbase + c0 + k), od);
                }
            } else {
#pragma unroll
                for (int k = 0; k < IPT; k++) {
                    const uint32_t sym = (c0 + k < W) ? a.syms[rbase + c0 + k] : 1u;
                    nzero += sym == 0u;
                    v[k] = (c0 + k < W) ? residual_of(sym, R, (uint32_t)(rbase + c0 + k), od) : 0u;
                }
            }
            if (nzero) atomicAdd(&par->d_zero, nzero);
        }
    } else if (VEC && c0 + IPT <= W) {
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
                carry = warp_lookback(a.flags, a.agg, a.inc, id, id - t, epoch + a.skew,
                                      a.spin_limit, par);
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
                        if ((f >> 2) == epoch + a.skew && (f & 3u)) st = f & 3u;
                    }
                    if (__all_sync(0xffffffffu, !valid || st != 0)) break;
                    if (it >= a.spin_limit) { timeout = true; break; }
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
// 2D inverse Lorenzo over bands of rows: reduce, then scan
// ---------------------------------------------------------------------------
//
// With S the 2D inclusive prefix sum of the residuals, band b (rows r0..r1-1)
// needs only S(r0 - 1, .), which is the prefix along x of E_b, the sum of the
// residuals of all rows above r0 per column.  E_b is the exclusive prefix over
// bands of every band's column sums, so three launches with no waiting between
// blocks give the exact 2D sum: column sums per band, their prefix over bands,
// then per band the row prefixes added on top of the carry row.  Each thread
// owns 8*G consecutive columns; a row of up to 2048*G columns is one block.

struct BandArgs {
    DevParams* par;
    const uint16_t* syms;  // [rows * nx] decoded symbols
    const uint8_t* blob;   // outlier list
    uint32_t* bsum;        // [nbands * nx] column sums, then their exclusive prefix over bands
    float* out;            // [rows * nx]
    uint32_t nx, rows, tr, nbands;
};

// Residuals of columns c0 .. c0 + 8G - 1 of row r (zero past the row end).
template <int G, bool VEC>
__device__ __forceinline__ void band_row_residuals(const BandArgs& a, uint32_t r, uint32_t c0,
                                                   uint32_t R, const uint32_t* __restrict__ od,
                                                   uint32_t (&d)[8 * G], uint32_t& nzero) {
    const uint64_t base = (uint64_t)r * a.nx;
    if (VEC) {
#pragma unroll
        for (int g = 0; g < G; g++) {
            const uint32_t cg = c0 + 8u * g;
            uint32_t v[8];
            if (cg < a.nx) {
                load_syms<8>(a.syms + base + cg, v);
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    nzero += v[k] == 0u;
                    v[k] = residual_of(v[k], R, (uint32_t)(base + cg + k), od);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 8; k++) v[k] = 0u;
            }
#pragma unroll
            for (int k = 0; k < 8; k++) d[8 * g + k] = v[k];
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8 * G; k++) {
            const uint32_t sym = (c0 + k < a.nx) ? a.syms[base + c0 + k] : 1u;
            nzero += sym == 0u;
            d[k] = (c0 + k < a.nx) ? residual_of(sym, R, (uint32_t)(base + c0 + k), od) : 0u;
        }
    }
}

// Raw symbols of row r for columns [c0, c0 + 8G) as G 16-byte loads (VEC rows:
// nx a multiple of 8); groups past the row end read nothing.
template <int G>
__device__ __forceinline__ void band_row_load(const BandArgs& a, uint32_t r, uint32_t c0, uint4 (&q)[G]) {
    const uint64_t base = (uint64_t)r * a.nx;
#pragma unroll
    for (int g = 0; g < G; g++) {
        const uint32_t cg = c0 + 8u * g;
        q[g] = cg < a.nx ? *reinterpret_cast<const uint4*>(a.syms + base + cg) : make_uint4(0u, 0u, 0u, 0u);
    }
}

// Residuals of row r from the raw symbols of band_row_load.
template <int G>
__device__ __forceinline__ void band_row_convert(const BandArgs& a, uint32_t r, uint32_t c0,
                                                 const uint4 (&q)[G], uint32_t R,
                                                 const uint32_t* __restrict__ od,
                                                 uint32_t (&d)[8 * G]) {
    const uint64_t base = (uint64_t)r * a.nx;
#pragma unroll
    for (int g = 0; g < G; g++) {
        const uint32_t cg = c0 + 8u * g;
        const uint32_t v[8] = {q[g].x & 0xffffu, q[g].x >> 16, q[g].y & 0xffffu, q[g].y >> 16,
                               q[g].z & 0xffffu, q[g].z >> 16, q[g].w & 0xffffu, q[g].w >> 16};
#pragma unroll
        for (int k = 0; k < 8; k++)
            d[8 * g + k] = cg < a.nx ? residual_of(v[k], R, (uint32_t)(base + cg + k), od) : 0u;
    }
}

// one block per band: column sums of the band's residuals
template <int G, bool VEC>
__global__ void __launch_bounds__(256) k_band_sum(const __grid_constant__ Batch<BandArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const BandArgs& a = B.a[fld];
    const uint32_t band = blockIdx.x - B.off[fld];
    DevParams* par = a.par;
    const uint32_t flags = par->flags;
    if (flags & kFlagError) return;
    const uint32_t c0 = threadIdx.x * 8u * G;
    if (c0 >= a.nx) return;
    uint32_t acc[8 * G];
#pragma unroll
    for (int k = 0; k < 8 * G; k++) acc[k] = 0u;
    if (!(flags & kFlagConstant)) {
        const uint32_t R = par->d_radius;
        const uint32_t* __restrict__ od = reinterpret_cast<const uint32_t*>(a.out);
        const uint32_t r0 = band * a.tr, r1 = min(r0 + a.tr, a.rows);
        uint32_t nzero = 0;  // symbols 0 (outliers), checked against the list by k_patch
        for (uint32_t r = r0; r < r1; r++) {
            uint32_t d[8 * G];
            band_row_residuals<G, VEC>(a, r, c0, R, od, d, nzero);
#pragma unroll
            for (int k = 0; k < 8 * G; k++) acc[k] += d[k];
        }
        if (nzero) atomicAdd(&par->d_zero, nzero);
    }
    uint32_t* dst = a.bsum + (uint64_t)band * a.nx;
#pragma unroll
    for (int k = 0; k < 8 * G; k++)
        if (c0 + k < a.nx) dst[c0 + k] = acc[k];
}

// one thread per column: exclusive prefix over the bands, in place
__global__ void __launch_bounds__(256) k_band_carry(const __grid_constant__ Batch<BandArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const BandArgs& a = B.a[fld];
    if (a.par->flags & kFlagError) return;
    const uint32_t col = (blockIdx.x - B.off[fld]) * blockDim.x + threadIdx.x;
    if (col >= a.nx) return;
    uint32_t* p = a.bsum + col;
    const uint64_t st = a.nx;
    uint32_t acc = 0u;
    uint32_t b = 0;
    for (; b + 8 <= a.nbands; b += 8) {
        uint32_t t[8];
#pragma unroll
        for (int k = 0; k < 8; k++) t[k] = p[(uint64_t)(b + k) * st];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            p[(uint64_t)(b + k) * st] = acc;
            acc += t[k];
        }
    }
    for (; b < a.nbands; b++) {
        const uint32_t t = p[(uint64_t)b * st];
        p[(uint64_t)b * st] = acc;
        acc += t;
    }
}

// Inclusive prefix along the block's columns of one row given per thread:
// thread-local prefix plus the block's exclusive scan of the thread totals.
template <int G>
__device__ __forceinline__ void band_row_prefix(uint32_t (&d)[8 * G], uint32_t* sh) {
#pragma unroll
    for (int k = 1; k < 8 * G; k++) d[k] += d[k - 1];
    uint32_t tot;
    const uint32_t ex = block_excl_scan(d[8 * G - 1], sh, &tot);
#pragma unroll
    for (int k = 0; k < 8 * G; k++) d[k] += ex;
}

// one block per band: carry row, then every row's prefix, dequantized
template <int G, bool VEC>
__global__ void __launch_bounds__(256) k_band_scan(const __grid_constant__ Batch<BandArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const BandArgs& a = B.a[fld];
    const uint32_t band = blockIdx.x - B.off[fld];
    DevParams* par = a.par;
    __shared__ uint32_t sh[33];
    const uint32_t flags = par->flags;
    if (flags & kFlagError) return;
    const bool cst = (flags & kFlagConstant) != 0;
    const uint32_t c0 = threadIdx.x * 8u * G;
    const float s = par->s, xmin = par->xmin;
    const uint32_t R = par->d_radius;
    // outlier residuals, each read before this thread writes the point's float
    const uint32_t* od = reinterpret_cast<const uint32_t*>(a.out);
    // S(r0 - 1, .) = prefix along x of the carry row
    uint32_t col[8 * G];
    {
        const uint32_t* e = a.bsum + (uint64_t)band * a.nx;
#pragma unroll
        for (int k = 0; k < 8 * G; k++) col[k] = (c0 + k < a.nx) ? e[c0 + k] : 0u;
        band_row_prefix<G>(col, sh);
    }
    const uint32_t r0 = band * a.tr, r1 = min(r0 + a.tr, a.rows);
    const bool live = !cst && c0 < a.nx;
    // VEC: the next row's symbols are loaded before this row's block scan
    uint4 qn[G];
    if (VEC && live && r0 < r1) band_row_load<G>(a, r0, c0, qn);
    for (uint32_t r = r0; r < r1; r++) {
        uint32_t d[8 * G];
        if (!live) {
#pragma unroll
            for (int k = 0; k < 8 * G; k++) d[k] = 0u;
        } else if (VEC) {
            uint4 q[G];
#pragma unroll
            for (int g = 0; g < G; g++) q[g] = qn[g];
            if (r + 1 < r1) band_row_load<G>(a, r + 1, c0, qn);
            band_row_convert<G>(a, r, c0, q, R, od, d);
        } else {
            uint32_t unused = 0;  // counted by k_band_sum
            band_row_residuals<G, VEC>(a, r, c0, R, od, d, unused);
        }
        band_row_prefix<G>(d, sh);
        float f[8 * G];
#pragma unroll
        for (int k = 0; k < 8 * G; k++) {
            col[k] += d[k];
            f[k] = __fmaf_rn(__int2float_rn((int32_t)col[k]), s, xmin);
        }
        float* o = a.out + (uint64_t)r * a.nx + c0;
        if (VEC) {
#pragma unroll
            for (int g = 0; g < 2 * G; g++)
                if (c0 + 4u * g < a.nx)
                    *reinterpret_cast<float4*>(o + 4 * g) =
                        make_float4(f[4 * g], f[4 * g + 1], f[4 * g + 2], f[4 * g + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < 8 * G; k++)
                if (c0 + k < a.nx) o[k] = f[k];
        }
    }
}

// ---------------------------------------------------------------------------
// 3D inverse Lorenzo over tiles of planes x rows: reduce, carry, scan
// ---------------------------------------------------------------------------
//
// q is the 3D inclusive prefix sum of the residuals.  The field is cut into
// tiles of tz planes (a slab s) by ty rows (a band b) by the whole row.  For a
// point (z, y, x) of tile (s, b), with z0 and y0 the tile's first plane and
// row, the column sum
//   A(z, y, x) = sum of the residuals at (z', y', x) with z' <= z and y' <= y
// splits into four parts:
//   K[s][b][x]                                z' < z0,  y' < y0
//   sum over y0 <= y' <= y of E[s][y'][x]     z' < z0,  y0 <= y' <= y
//   sum over z0 <= z' <= z of F[z'][b][x]     z0 <= z' <= z,  y' < y0
//   the tile's own residuals                  z0 <= z' <= z,  y0 <= y' <= y
// and q(z, y, x) is the prefix of A(z, y, .) along x.  E (per row, over the
// earlier slabs), F (per plane, over the earlier bands) and K (per tile, over
// both) are exclusive prefixes of the slab sums of every row, the band column
// sums of every plane and the column sums of every tile, which one reading of
// the residuals gives.  Three launches with no waiting between blocks:
//   k_vol_sum    one block per tile: the three kinds of sums
//   k_vol_carry  their exclusive prefixes, in place
//   k_vol_scan   one block per tile, plane by plane: the column prefix along
//                y (plus F) by one thread per column, then A of every row in
//                the registers of the warp that owns the row, its prefix along
//                x by warp shuffles, and x' = fmaf((float)q, s, xmin) on the
//                write
// Both tile kernels stage each plane's rows of the tile (one contiguous range
// of symbols) in shared memory with a bulk copy two planes ahead.  The
// symbols are read twice and the floats written once.  All sums are modular
// uint32 (every final q is in [0, 2^31)).

struct VolArgs {
    DevParams* par;
    const uint16_t* syms;  // [nz][ny][nx] decoded symbols (the buffer holds 8 more)
    float* out;            // [nz][ny][nx]; outlier residuals (u32) at their indices until written
    uint32_t* cb;          // [nz][nbands][nx] band column sums of every plane -> F
    uint32_t* ds;          // [nslabs][ny][nx] slab sums of every row -> E
    uint32_t* ts;          // [nslabs][nbands][nx] column sums of every tile -> K
    uint32_t nx, ny, nz, tz, nbands, nslabs;
    uint32_t nF, nE;       // k_vol_carry: blocks of its first two roles
    uint32_t spin_limit;   // polls of a plane's copy before giving up
};

constexpr uint32_t kVolSymBytes = 16384 + 32;  // one plane of a tile: 8192 symbols + alignment

// Shared-memory staging of a tile's planes: two buffers of symbols at `base`
// (kVolSymBytes apart), each filled by one bulk copy completing on its own
// mbarrier.  Thread 0 counts the copies it issues to each buffer; every
// thread counts the ones it has waited for.
struct VolStage {
    uint8_t* base;
    unsigned long long* mbar;  // [2]
    uint32_t issued0, issued1;
    uint32_t waited0, waited1;
    __device__ __forceinline__ const uint16_t* buf(int which) const {
        return reinterpret_cast<const uint16_t*>(base + (which ? kVolSymBytes : 0u));
    }
};

// Byte range of plane z's rows [y0, y1) of the tile, widened to 16-byte
// boundaries (the symbol buffer holds 16 bytes past the field's end).
__device__ __forceinline__ void vol_plane_range(const VolArgs& a, uint32_t z, uint32_t y0, uint32_t y1,
                                                uint64_t* from, uint32_t* bytes, uint32_t* skew) {
    const uint64_t b0 = 2ull * ((uint64_t)z * a.ny + y0) * a.nx;
    const uint64_t b1 = 2ull * ((uint64_t)z * a.ny + y1) * a.nx;
    const uint64_t lo = b0 & ~15ull, hi = (b1 + 15ull) & ~15ull;
    *from = lo;
    *bytes = (uint32_t)(hi - lo);
    *skew = (uint32_t)((b0 - lo) >> 1);  // symbols before the tile's first one
}

// Thread 0: start the copy of plane z into buffer `which`.
__device__ __forceinline__ void vol_issue(const VolArgs& a, VolStage& st, int which, uint32_t z,
                                          uint32_t y0, uint32_t y1) {
    uint64_t from;
    uint32_t bytes, skew;
    vol_plane_range(a, z, y0, y1, &from, &bytes, &skew);
    // earlier generic reads of the buffer are ordered before the copy's writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    unsigned long long* mb = st.mbar + which;
    mbar_arrive_expect_tx(mb, bytes);
    bulk_g2s(st.base + (which ? kVolSymBytes : 0u), reinterpret_cast<const uint8_t*>(a.syms) + from, bytes, mb);
    if (which) st.issued1++;
    else st.issued0++;
}

// Every thread: wait (at most `limit` polls) for the next copy into buffer
// `which`; false if it did not land in time (it then stays counted as
// outstanding, for vol_drain).
__device__ __forceinline__ bool vol_wait(VolStage& st, int which, uint32_t limit) {
    const uint32_t k = which ? st.waited1 : st.waited0;
    if (!mbar_wait_bounded(st.mbar + which, k & 1u, limit)) return false;
    if (which) st.waited1++;
    else st.waited0++;
    return true;
}

// After a timeout: thread 0 waits (bounded) for every copy still in flight,
// so that none lands after the block has left.
__device__ __forceinline__ void vol_drain(const VolStage& st) {
    if (threadIdx.x != 0) return;
    for (uint32_t k = st.waited0; k < st.issued0; k++) mbar_wait_bounded(st.mbar, k & 1u);
    for (uint32_t k = st.waited1; k < st.issued1; k++) mbar_wait_bounded(st.mbar + 1, k & 1u);
}

template <int CPL, int WPR>
__global__ void __launch_bounds__(512) k_vol_sum(const __grid_constant__ Batch<VolArgs> B) {
    constexpr uint32_t TY = 16 / WPR;
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const VolArgs& a = B.a[fld];
    const uint32_t t = blockIdx.x - B.off[fld];
    DevParams* par = a.par;
    const uint32_t flags = par->flags;
    if (flags & kFlagError) return;  // uniform over the block
    extern __shared__ __align__(16) uint8_t vsm[];
    __shared__ __align__(8) unsigned long long s_mbar[2];
    const uint32_t s = t / a.nbands, b = t % a.nbands;
    const uint32_t z0 = s * a.tz, z1 = min(z0 + a.tz, a.nz);
    const uint32_t y0 = b * TY, y1 = min(y0 + TY, a.ny), nrows = y1 - y0;
    const bool cst = (flags & kFlagConstant) != 0;
    VolStage st{vsm, s_mbar, 0u, 0u, 0u, 0u};
    if (threadIdx.x == 0) {
        mbar_init(&s_mbar[0], 1);
        mbar_init(&s_mbar[1], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0 && !cst) {
        vol_issue(a, st, 0, z0, y0, y1);
        if (z0 + 1 < z1) vol_issue(a, st, 1, z0 + 1, y0, y1);
    }
    const uint32_t R = par->d_radius;
    const uint32_t* __restrict__ od = reinterpret_cast<const uint32_t*>(a.out);
    uint32_t dacc[WPR][TY], tacc[WPR];
#pragma unroll
    for (int q = 0; q < WPR; q++) {
        tacc[q] = 0u;
#pragma unroll
        for (uint32_t r = 0; r < TY; r++) dacc[q][r] = 0u;
    }
    uint32_t nzero = 0;  // symbols 0 (outliers), checked against the list by k_patch
    for (uint32_t z = z0; z < z1; z++) {
        const int which = (int)((z - z0) & 1u);
        const bool late = !cst && !vol_wait(st, which, a.spin_limit);
        uint64_t from;
        uint32_t bytes, skew;
        vol_plane_range(a, z, y0, y1, &from, &bytes, &skew);
        const uint16_t* sb = st.buf(which) + skew;
#pragma unroll
        for (int q = 0; q < WPR; q++) {
            const uint32_t j = threadIdx.x + 512u * q;
            if (j >= a.nx) continue;
            uint32_t cs = 0u, zeros = 0u;  // bit r: row r holds a symbol 0 (an outlier)
            if (!cst) {
#pragma unroll
                for (uint32_t r = 0; r < TY; r++) {
                    if (r < nrows) {
                        const uint32_t sym = sb[r * a.nx + j];
                        zeros |= (sym == 0u ? 1u : 0u) << r;
                        cs += sym - R;
                        dacc[q][r] += sym - R;
                    }
                }
                if (zeros) {  // rare: an outlier's residual replaces its symbol's -R
                    nzero += __popc(zeros);
#pragma unroll
                    for (uint32_t r = 0; r < TY; r++) {
                        if ((zeros >> r) & 1u) {
                            const uint32_t fix = od[((uint64_t)z * a.ny + y0 + r) * a.nx + j] + R;
                            cs += fix;
                            dacc[q][r] += fix;
                        }
                    }
                }
            }
            a.cb[((uint64_t)z * a.nbands + b) * a.nx + j] = cs;
            tacc[q] += cs;
        }
        if (__syncthreads_or(late)) {  // every thread is done with the buffer
            if (threadIdx.x == 0) set_error(par, FPSNR_ETIMEOUT);
            vol_drain(st);
            return;
        }
        if (threadIdx.x == 0 && !cst && z + 2 < z1) vol_issue(a, st, which, z + 2, y0, y1);
    }
    if (nzero) atomicAdd(&par->d_zero, nzero);
#pragma unroll
    for (int q = 0; q < WPR; q++) {
        const uint32_t j = threadIdx.x + 512u * q;
        if (j >= a.nx) continue;
#pragma unroll
        for (uint32_t r = 0; r < TY; r++)
            if (r < nrows) a.ds[((uint64_t)s * a.ny + y0 + r) * a.nx + j] = dacc[q][r];
        a.ts[((uint64_t)s * a.nbands + b) * a.nx + j] = tacc[q];
    }
}

// count values at p, p + stride, ... replaced by their exclusive prefix
__device__ __forceinline__ void excl_prefix_strided(uint32_t* p, uint32_t count, uint64_t stride) {
    uint32_t acc = 0u, i = 0;
    // 16 loads in flight at a time (the sums are latency-bound, not bandwidth-bound)
    for (; i + 16 <= count; i += 16) {
        uint32_t v[16];
#pragma unroll
        for (int k = 0; k < 16; k++) v[k] = p[(uint64_t)(i + k) * stride];
#pragma unroll
        for (int k = 0; k < 16; k++) {
            p[(uint64_t)(i + k) * stride] = acc;
            acc += v[k];
        }
    }
    for (; i + 8 <= count; i += 8) {
        uint32_t v[8];
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = p[(uint64_t)(i + k) * stride];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            p[(uint64_t)(i + k) * stride] = acc;
            acc += v[k];
        }
    }
    for (; i < count; i++) {
        const uint32_t v = p[(uint64_t)i * stride];
        p[(uint64_t)i * stride] = acc;
        acc += v;
    }
}

// Three roles by block: F (one thread per plane and column: over the bands),
// E (one thread per row and column: over the slabs), K (32 columns per block:
// over the slabs, then, after a block barrier, over the bands).
__global__ void __launch_bounds__(256) k_vol_carry(const __grid_constant__ Batch<VolArgs> B) {
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const VolArgs& a = B.a[fld];
    const uint32_t t = blockIdx.x - B.off[fld];
    if (a.par->flags & kFlagError) return;  // uniform over the block
    if (t < a.nF) {
        const uint64_t i = (uint64_t)t * 256u + threadIdx.x;  // z * nx + x
        if (i >= (uint64_t)a.nz * a.nx) return;
        const uint64_t z = i / a.nx, x = i % a.nx;
        excl_prefix_strided(a.cb + z * a.nbands * a.nx + x, a.nbands, a.nx);
    } else if (t < a.nF + a.nE) {
        const uint64_t i = (uint64_t)(t - a.nF) * 256u + threadIdx.x;  // y * nx + x
        if (i >= (uint64_t)a.ny * a.nx) return;
        excl_prefix_strided(a.ds + i, a.nslabs, (uint64_t)a.ny * a.nx);
    } else {
        const uint32_t x = (t - a.nF - a.nE) * 32u + (threadIdx.x & 31u), r = threadIdx.x >> 5;
        if (x < a.nx)
            for (uint32_t b = r; b < a.nbands; b += 8)
                excl_prefix_strided(a.ts + (uint64_t)b * a.nx + x, a.nslabs, (uint64_t)a.nbands * a.nx);
        __syncthreads();  // every thread of the block reaches it
        if (x < a.nx)
            for (uint32_t s = r; s < a.nslabs; s += 8)
                excl_prefix_strided(a.ts + (uint64_t)s * a.nbands * a.nx + x, a.nbands, a.nx);
    }
}

// Word of column j in a row of the column-prefix buffer: groups of 4 words
// (one 128-bit read of a lane) are permuted within each run of 8 groups, so
// that both the column threads' writes and the lanes' 128-bit reads of a row
// are free of bank conflicts.
__device__ __forceinline__ uint32_t vol_swz(uint32_t j) {
    const uint32_t c = j >> 2;
    return ((c ^ ((c >> 3) & 7u)) << 2) | (j & 3u);
}

template <int CPL, int WPR, bool FV>
__global__ void __launch_bounds__(512, 2) k_vol_scan(const __grid_constant__ Batch<VolArgs> B) {
    constexpr uint32_t TY = 16 / WPR;
    constexpr uint32_t RS = 32u * CPL * WPR;  // words per row of the column-prefix buffer
    const uint32_t fld = batch_field(B.off, B.count, blockIdx.x);
    const VolArgs& a = B.a[fld];
    const uint32_t t = blockIdx.x - B.off[fld];
    DevParams* par = a.par;
    const uint32_t flags = par->flags;
    if (flags & kFlagError) return;  // uniform over the block
    extern __shared__ __align__(16) uint8_t vsm[];
    __shared__ __align__(8) unsigned long long s_mbar[2];
    __shared__ uint32_t wt[2][16];  // WPR > 1: warp totals of a row's parts
    uint32_t* D0 = reinterpret_cast<uint32_t*>(vsm + 2 * kVolSymBytes);
    uint32_t* D1 = D0 + TY * RS;
    const uint32_t s = t / a.nbands, b = t % a.nbands;
    const uint32_t z0 = s * a.tz, z1 = min(z0 + a.tz, a.nz);
    const uint32_t y0 = b * TY, y1 = min(y0 + TY, a.ny), nrows = y1 - y0;
    const bool cst = (flags & kFlagConstant) != 0;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    VolStage st{vsm, s_mbar, 0u, 0u, 0u, 0u};
    if (threadIdx.x == 0) {
        mbar_init(&s_mbar[0], 1);
        mbar_init(&s_mbar[1], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0 && !cst) {
        vol_issue(a, st, 0, z0, y0, y1);
        if (z0 + 1 < z1) vol_issue(a, st, 1, z0 + 1, y0, y1);
    }
    const uint32_t R = par->d_radius;
    const float sc = par->s, xmin = par->xmin;
    // outlier residuals, each read by a column thread before the barrier that
    // precedes the float write of its point
    const uint32_t* __restrict__ od = reinterpret_cast<const uint32_t*>(a.out);

    // A(z0 - 1, y, .) of the band's rows, by the column threads into D1
#pragma unroll
    for (int q = 0; q < WPR; q++) {
        const uint32_t j = threadIdx.x + 512u * q;
        if (j >= RS) continue;
        uint32_t run = j < a.nx ? a.ts[((uint64_t)s * a.nbands + b) * a.nx + j] : 0u;
#pragma unroll
        for (uint32_t r = 0; r < TY; r++) {
            if (j < a.nx && r < nrows) run += a.ds[((uint64_t)s * a.ny + y0 + r) * a.nx + j];
            D1[r * RS + vol_swz(j)] = run;
        }
    }
    __syncthreads();
    const uint32_t row = warp / WPR;  // the row this warp owns in phase B
    const uint32_t c0 = (warp % WPR) * 32u * CPL + lane * CPL;
    uint32_t P[CPL];
#pragma unroll
    for (int k = 0; k < CPL; k += 4) {
        const uint4 v = *reinterpret_cast<const uint4*>(D1 + row * RS + vol_swz(c0 + k));
        P[k] = v.x; P[k + 1] = v.y; P[k + 2] = v.z; P[k + 3] = v.w;
    }
    // F of the next plane, loaded a plane ahead by the column threads
    uint32_t fn[WPR];
#pragma unroll
    for (int q = 0; q < WPR; q++) {
        const uint32_t j = threadIdx.x + 512u * q;
        fn[q] = (j < a.nx && z0 < z1) ? a.cb[((uint64_t)z0 * a.nbands + b) * a.nx + j] : 0u;
    }
    for (uint32_t z = z0; z < z1; z++) {
        const int which = (int)((z - z0) & 1u);
        uint32_t* D = which ? D1 : D0;
        const bool late = !cst && !vol_wait(st, which, a.spin_limit);
        uint64_t from;
        uint32_t bytes, skew;
        vol_plane_range(a, z, y0, y1, &from, &bytes, &skew);
        const uint16_t* sb = st.buf(which) + skew;
        // phase A: per column, F plus the prefix over the band's rows
#pragma unroll
        for (int q = 0; q < WPR; q++) {
            const uint32_t j = threadIdx.x + 512u * q;
            if (j >= RS) continue;
            const uint32_t f0 = fn[q];
            fn[q] = (j < a.nx && z + 1 < z1) ? a.cb[((uint64_t)(z + 1) * a.nbands + b) * a.nx + j] : 0u;
            uint32_t* dcol = D + vol_swz(j);
            if (j >= a.nx) {
#pragma unroll
                for (uint32_t r = 0; r < TY; r++) dcol[r * RS] = 0u;
                continue;
            }
            uint32_t c = f0, zeros = 0u;  // bit r: row r holds a symbol 0 (an outlier)
#pragma unroll
            for (uint32_t r = 0; r < TY; r++) {
                if (r < nrows && !cst) {
                    const uint32_t sym = sb[r * a.nx + j];
                    zeros |= (sym == 0u ? 1u : 0u) << r;
                    c += sym - R;
                }
                dcol[r * RS] = c;
            }
            if (zeros) {  // rare: the column again, with the outliers' residuals
                c = f0;
#pragma unroll
                for (uint32_t r = 0; r < TY; r++) {
                    if (r < nrows) {
                        const uint32_t sym = sb[r * a.nx + j];
                        c += sym ? sym - R : od[((uint64_t)z * a.ny + y0 + r) * a.nx + j];
                    }
                    dcol[r * RS] = c;
                }
            }
        }
        if (__syncthreads_or(late)) {
            if (threadIdx.x == 0) set_error(par, FPSNR_ETIMEOUT);
            vol_drain(st);
            return;
        }
        if (threadIdx.x == 0 && !cst && z + 2 < z1) vol_issue(a, st, which, z + 2, y0, y1);
        // phase B: the warp's row, A = A(z - 1) + this plane's column prefix,
        // then its prefix along x
        uint32_t v[CPL];
#pragma unroll
        for (int k = 0; k < CPL; k += 4) {
            const uint4 cq = *reinterpret_cast<const uint4*>(D + row * RS + vol_swz(c0 + k));
            P[k] += cq.x; P[k + 1] += cq.y; P[k + 2] += cq.z; P[k + 3] += cq.w;
        }
        v[0] = P[0];
#pragma unroll
        for (int k = 1; k < CPL; k++) v[k] = v[k - 1] + P[k];
        const uint32_t tot = v[CPL - 1];
        uint32_t incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        uint32_t ex = incl - tot;
        if constexpr (WPR > 1) {
            if (lane == 31u) wt[which][warp] = incl;
            __syncthreads();
            for (uint32_t p = 0; p < warp % WPR; p++) ex += wt[which][row * WPR + p];
        }
        if (row < nrows) {
            const uint64_t rb = ((uint64_t)z * a.ny + y0 + row) * a.nx;
            float f[CPL];
#pragma unroll
            for (int k = 0; k < CPL; k++) f[k] = __fmaf_rn(__int2float_rn((int32_t)(v[k] + ex)), sc, xmin);
            float* o = a.out + rb + c0;
            if (FV && c0 + CPL <= a.nx) {
#pragma unroll
                for (int k = 0; k < CPL; k += 4)
                    *reinterpret_cast<float4*>(o + k) = make_float4(f[k], f[k + 1], f[k + 2], f[k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < CPL; k++)
                    if (c0 + k < a.nx) o[k] = f[k];
            }
        }
    }
}

// dynamic shared memory of the tile kernels
constexpr uint32_t vol_sum_smem() { return 2 * kVolSymBytes; }
template <int CPL, int WPR>
constexpr uint32_t vol_scan_smem() { return 2 * kVolSymBytes + 2 * (16 / WPR) * 32u * CPL * WPR * 4u; }

// ---------------------------------------------------------------------------
// host launcher
// ---------------------------------------------------------------------------

template <int IPT, bool FINAL, bool SYM>
static void launch_contig_t(const Batch<ScanArgs>& b, uint32_t tiles, bool vec, cudaStream_t st) {
    if (vec) k_scan_contig<IPT, FINAL, true, SYM><<<tiles, 256, 0, st>>>(b);
    else k_scan_contig<IPT, FINAL, false, SYM><<<tiles, 256, 0, st>>>(b);
}

template <bool FINAL, bool SYM>
static void launch_contig(const Batch<ScanArgs>& b, uint32_t tiles, int ipt, bool vec,
                          cudaStream_t st) {
    if (ipt == 4) launch_contig_t<4, FINAL, SYM>(b, tiles, vec, st);
    else if (ipt == 8) launch_contig_t<8, FINAL, SYM>(b, tiles, vec, st);
    else launch_contig_t<16, FINAL, SYM>(b, tiles, vec, st);
}

template <int G, bool VEC>
static void launch_band_t(const Batch<BandArgs>& b, const uint32_t* nb, const uint32_t* ncol,
                          fp::Profiler& prof, cudaStream_t st) {
    Batch<BandArgs> bb = b;
    const uint32_t tb = batch_offsets(bb, nb);
    {
        StageScope sc(prof, kStBandSum, st);
        k_band_sum<G, VEC><<<tb, 256, 0, st>>>(bb);
    }
    Batch<BandArgs> bc = b;
    const uint32_t tc = batch_offsets(bc, ncol);
    {
        StageScope sc(prof, kStBandCarry, st);
        k_band_carry<<<tc, 256, 0, st>>>(bc);
    }
    {
        StageScope sc(prof, kStScanFinal, st);
        k_band_scan<G, VEC><<<tb, 256, 0, st>>>(bb);
    }
}

template <bool VEC>
static void launch_band(const Batch<BandArgs>& b, const uint32_t* nb, const uint32_t* ncol, int g,
                        fp::Profiler& prof, cudaStream_t st) {
    if (g == 1) launch_band_t<1, VEC>(b, nb, ncol, prof, st);
    else if (g == 2) launch_band_t<2, VEC>(b, nb, ncol, prof, st);
    else launch_band_t<4, VEC>(b, nb, ncol, prof, st);
}

template <int CPL, int WPR, bool FV>
static void launch_vol_t(const Batch<VolArgs>& b, const uint32_t* ntile, const uint32_t* ncarry,
                         fp::Profiler& prof, cudaStream_t st) {
    Batch<VolArgs> bt = b;
    const uint32_t tt = batch_offsets(bt, ntile);
    {
        StageScope sc(prof, kStBandSum, st);
        k_vol_sum<CPL, WPR><<<tt, 512, vol_sum_smem(), st>>>(bt);
    }
    Batch<VolArgs> bc = b;
    const uint32_t tc = batch_offsets(bc, ncarry);
    {
        StageScope sc(prof, kStBandCarry, st);
        k_vol_carry<<<tc, 256, 0, st>>>(bc);
    }
    {
        StageScope sc(prof, kStScanFinal, st);
        k_vol_scan<CPL, WPR, FV><<<tt, 512, vol_scan_smem<CPL, WPR>(), st>>>(bt);
    }
}

template <bool FV>
static void launch_vol(const Batch<VolArgs>& b, const uint32_t* ntile, const uint32_t* ncarry, int cpl,
                       int wpr, fp::Profiler& prof, cudaStream_t st) {
    if (wpr == 4) launch_vol_t<16, 4, FV>(b, ntile, ncarry, prof, st);
    else if (wpr == 2) launch_vol_t<16, 2, FV>(b, ntile, ncarry, prof, st);
    else if (cpl == 16) launch_vol_t<16, 1, FV>(b, ntile, ncarry, prof, st);
    else if (cpl == 8) launch_vol_t<8, 1, FV>(b, ntile, ncarry, prof, st);
    else launch_vol_t<4, 1, FV>(b, ntile, ncarry, prof, st);
}

template <int CPL, int WPR, bool FV>
static bool vol_attrs() {
    return cudaFuncSetAttribute(k_vol_scan<CPL, WPR, FV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)vol_scan_smem<CPL, WPR>()) == cudaSuccess;
}

template <int T>
static bool decode_attrs() {
    return cudaFuncSetAttribute(k_decode<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dec_smem(T)) == cudaSuccess &&
           cudaFuncSetAttribute(k_decode<T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100) ==
               cudaSuccess;
}

// Called at every plan creation: the attributes are per device (and cheap to
// set), so no process-wide flag skips them.
int decode_prepare(const fpsnr_plan_s*) {
    // the decoder reads its stream through cp.async into shared memory, not
    // L1: take the largest shared-memory carveout so that the rings of its
    // resident threads and their blocks' tables fit
    if (!decode_attrs<128>() || !decode_attrs<256>() || !decode_attrs<512>()) return FPSNR_ECUDA;
    // the 3D tile scans stage symbols and column prefixes in shared memory
    if (!vol_attrs<4, 1, false>() || !vol_attrs<4, 1, true>() || !vol_attrs<8, 1, false>() ||
        !vol_attrs<8, 1, true>() || !vol_attrs<16, 1, false>() || !vol_attrs<16, 1, true>() ||
        !vol_attrs<16, 2, false>() || !vol_attrs<16, 2, true>() || !vol_attrs<16, 4, false>() ||
        !vol_attrs<16, 4, true>())
        return FPSNR_ECUDA;
    return FPSNR_OK;
}

// Grid-stride kernels over the outlier / verbatim lists (which can hold a
// tenth of the points at 120 dB): about four blocks per SM over the batch.
static uint32_t small_blocks_d(const fpsnr_plan_s* p, int count) {
    const int g = std::max(1, 4 * p->sm_count / std::max(1, count));
    return (uint32_t)std::min(g, 256);
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

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
    // lossless plans: expand the container (or copy the plain blob) into the
    // plan's scratch; every later kernel reads that copy
    if (launch_zr_unwrap(P, d_blob, bytes, count, st) != FPSNR_OK) return FPSNR_ECUDA;
    const void* blob_of[kMaxBatch];
    for (int f = 0; f < count; f++) blob_of[f] = P[f]->lossless ? (const void*)P[f]->w.zr_scratch : d_blob[f];
    d_blob = blob_of;
    {
        Batch<DsetupArgs> b;
        b.count = (uint32_t)count;
        for (int f = 0; f < count; f++) {
            const fpsnr_plan_s* p = P[f];
            const Workspace& w = p->w;
            b.a[f] = DsetupArgs{w.par, reinterpret_cast<const uint8_t*>(d_blob[f]), bytes[f],
                                p->lossless != 0, p->ndim, p->ld, p->dims[0], p->dims[1],
                                p->dims[2], p->n, (uint32_t)p->chunk, p->nchunks, w.dlut,
                                w.dsyms, w.lb_ctr};
            b.off[f] = (uint32_t)f;
        }
        b.off[count] = (uint32_t)count;
        StageScope sc(prof, kStDsetup, st);
        k_dsetup<<<count, 1024, 0, st>>>(b);
        if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA;
    }
    // decode every field into its plan's symbol buffer
    {
        // 128-thread blocks (a 16 KB table and 128-byte rings: six per SM) start
        // and retire often enough that a batch's last wave stays short
        const int T = P[0]->dec_threads ? P[0]->dec_threads : 128;
        Batch<DecArgs> b;
        b.count = 0;
        for (int f = 0; f < count; f++) {
            const fpsnr_plan_s* p = P[f];
            if (p->n == 0) continue;
            const Workspace& w = p->w;
            blocks[b.count] = (uint32_t)((p->nchunks + T - 1) / T);
            b.a[b.count++] = DecArgs{w.par, p->spin_limit, reinterpret_cast<const uint8_t*>(d_blob[f]),
                                     w.dlut, w.dsyms, w.codes, p->n, (uint32_t)p->chunk, p->nchunks};
        }
        if (b.count) {
            const uint32_t tot = batch_offsets(b, blocks);
            StageScope sc(prof, kStDecode, st);
            if (T == 128) k_decode<128><<<tot, 128, dec_smem(128), st>>>(b);
            else if (T == 256) k_decode<256><<<tot, 256, dec_smem(256), st>>>(b);
            else k_decode<512><<<tot, 512, dec_smem(512), st>>>(b);
            if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA;
            // outlier residuals into the output buffers (checked against the symbols)
            Batch<ScatterArgs> sa;
            sa.count = 0;
            uint32_t sblocks[kMaxBatch];
            for (int f = 0; f < count; f++) {
                const fpsnr_plan_s* p = P[f];
                if (p->n == 0) continue;
                const uint32_t g = small_blocks_d(p, count);
                sblocks[sa.count] = g;
                sa.a[sa.count] = ScatterArgs{p->w.par, reinterpret_cast<const uint8_t*>(d_blob[f]),
                                             p->w.codes, reinterpret_cast<uint32_t*>(d_out[f]), p->n, g};
                sa.count++;
            }
            const uint32_t stot = batch_offsets(sa, sblocks);
            if (stot) {
                k_out_scatter<<<stot, 256, 0, st>>>(sa);
                sc.more(1);
            }
            if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA;
        }
    }
    // 2D fields whose rows fit one block: bands of rows, grouped by kernel variant
    {
        bool done[kMaxBatch] = {};
        for (int f0 = 0; f0 < count; f0++) {
            const fpsnr_plan_s* p0 = P[f0];
            if (done[f0] || p0->n == 0 || !p0->band.on) continue;
            const bool vec0 = p0->band.vec && aligned16(d_out[f0]);
            Batch<BandArgs> b;
            b.count = 0;
            uint32_t nb[kMaxBatch], ncol[kMaxBatch];
            for (int f = f0; f < count; f++) {
                const fpsnr_plan_s* p = P[f];
                if (done[f] || p->n == 0 || !p->band.on) continue;
                const bool vec = p->band.vec && aligned16(d_out[f]);
                if (p->band.g != p0->band.g || vec != vec0) continue;
                done[f] = true;
                const BandGeom& g = p->band;
                nb[b.count] = g.nbands;
                ncol[b.count] = (g.nx + 255u) / 256u;
                b.a[b.count++] = BandArgs{p->w.par, p->w.codes,
                                          reinterpret_cast<const uint8_t*>(d_blob[f]), p->w.bsum,
                                          d_out[f], g.nx, g.rows, g.tr, g.nbands};
            }
            if (vec0) launch_band<true>(b, nb, ncol, p0->band.g, prof, st);
            else launch_band<false>(b, nb, ncol, p0->band.g, prof, st);
            if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA;
        }
    }
    // 3D fields whose rows fit one block: tiles of planes x rows, grouped by kernel variant
    {
        bool done[kMaxBatch] = {};
        for (int f0 = 0; f0 < count; f0++) {
            const fpsnr_plan_s* p0 = P[f0];
            if (done[f0] || p0->n == 0 || !p0->vol.on) continue;
            const bool vec0 = p0->vol.vec && aligned16(d_out[f0]);
            Batch<VolArgs> b;
            b.count = 0;
            uint32_t ntile[kMaxBatch], ncarry[kMaxBatch];
            for (int f = f0; f < count; f++) {
                const fpsnr_plan_s* p = P[f];
                if (done[f] || p->n == 0 || !p->vol.on) continue;
                const bool vec = p->vol.vec && aligned16(d_out[f]);
                if (p->vol.cpl != p0->vol.cpl || p->vol.wpr != p0->vol.wpr || vec != vec0) continue;
                done[f] = true;
                const VolGeom& g = p->vol;
                VolArgs va;
                va.par = p->w.par;
                va.syms = p->w.codes;
                va.out = d_out[f];
                va.cb = p->w.vcb;
                va.ds = p->w.vds;
                va.ts = p->w.vts;
                va.nx = g.nx;
                va.ny = g.ny;
                va.nz = g.nz;
                va.tz = g.tz;
                va.nbands = g.nbands;
                va.nslabs = g.nslabs;
                va.nF = (uint32_t)(((uint64_t)g.nz * g.nx + 255u) / 256u);
                va.nE = (uint32_t)(((uint64_t)g.ny * g.nx + 255u) / 256u);
                va.spin_limit = p->spin_limit;
                ntile[b.count] = g.nslabs * g.nbands;
                ncarry[b.count] = va.nF + va.nE + (g.nx + 31u) / 32u;
                b.a[b.count++] = va;
            }
            if (vec0) launch_vol<true>(b, ntile, ncarry, p0->vol.cpl, p0->vol.wpr, prof, st);
            else launch_vol<false>(b, ntile, ncarry, p0->vol.cpl, p0->vol.wpr, prof, st);
            if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA;
        }
    }
    // other shapes: inverse Lorenzo passes, grouped by pass index and kernel variant
    for (int i = 0; i < 3; i++) {
        bool done[kMaxBatch] = {};
        auto vec_of = [&](const fpsnr_plan_s* p, int f) {
            const ScanPass& sp = p->pass[i];
            return (i == 0 ? sp.vec16 : sp.vec) && aligned16(d_out[f]);
        };
        for (int f0 = 0; f0 < count; f0++) {
            const fpsnr_plan_s* p0 = P[f0];
            if (done[f0] || p0->n == 0 || p0->n_passes <= i) continue;
            const ScanPass& s0 = p0->pass[i];
            const bool vec0 = vec_of(p0, f0);
            Batch<ScanArgs> b;
            b.count = 0;
            for (int f = f0; f < count; f++) {
                const fpsnr_plan_s* p = P[f];
                if (done[f] || p->n == 0 || p->n_passes <= i) continue;
                const ScanPass& sp = p->pass[i];
                if (sp.kind != s0.kind || sp.ipt != s0.ipt || vec_of(p, f) != vec0 ||
                    sp.final_pass != s0.final_pass)
                    continue;
                done[f] = true;
                const Workspace& w = p->w;
                ScanArgs a;
                a.par = w.par;
                a.data = reinterpret_cast<uint32_t*>(d_out[f]);
                a.syms = w.codes;
                a.blob = reinterpret_cast<const uint8_t*>(d_blob[f]);
                a.A = sp.A;
                a.L = sp.L;
                a.B = sp.B;
                a.tiles = sp.tiles;
                a.flags = w.lb_flags + sp.val_off;
                a.agg = w.lb_vals + sp.val_off * p->lb_width;
                a.inc = w.lb_vals + (p->lb_tiles_total + sp.val_off) * p->lb_width;
                a.ctr = w.lb_ctr + 2 * sp.ctr_slot;
                a.spin_limit = p->spin_limit;
                a.skew = p->wait_skew;
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
                // the first pass of every shape is contiguous and reads the symbols
                if (i == 0) {
                    if (s0.final_pass) launch_contig<true, true>(b, tot, s0.ipt, vec0, st);
                    else launch_contig<false, true>(b, tot, s0.ipt, vec0, st);
                } else {
                    if (s0.final_pass) launch_contig<true, false>(b, tot, s0.ipt, vec0, st);
                    else launch_contig<false, false>(b, tot, s0.ipt, vec0, st);
                }
            } else if (vec0) {
                if (s0.final_pass) k_scan_strided<16, 4, true><<<tot, 256, 0, st>>>(b);
                else k_scan_strided<16, 4, false><<<tot, 256, 0, st>>>(b);
            } else {
                if (s0.final_pass) k_scan_strided<16, 1, true><<<tot, 256, 0, st>>>(b);
                else k_scan_strided<16, 1, false><<<tot, 256, 0, st>>>(b);
            }
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
        StageScope sc(prof, kStPatch, st);
        k_patch<<<small_tot, 256, 0, st>>>(sb);
        if (cudaGetLastError() != cudaSuccess) return FPSNR_ECUDA;
    }
    if (d_status) {
        for (int f = 0; f < count; f++) sb.off[f] = (uint32_t)f;
        sb.off[count] = (uint32_t)count;
        k_status<<<count, 32, 0, st>>>(sb);
        prof.launches[kStPatch]++;  // counted with the verbatim patch
    }
    return cudaGetLastError() == cudaSuccess ? FPSNR_OK : FPSNR_ECUDA;
}

}  // namespace fp
