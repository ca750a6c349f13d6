// huffman.cu -- on-device construction of the canonical Huffman code for SZ's
// step 2 (Sec. II-A: "customized Huffman coding" of the quantization codes).
//
// One CTA of 1024 threads.  The code is the one a sequential two-queue
// Huffman construction gives when leaves are taken in ascending (count,
// symbol) order, internal nodes in creation order, and a leaf wins a tie with
// an internal node; while the longest code exceeds lmax every nonzero count c
// becomes max(1, c >> 1) and the code is rebuilt; canonical code values are
// assigned in ascending (length, symbol) order.  The paper leaves these
// choices open; the library fixes them so the bytes are deterministic.
//
// Parallel construction ("bulk rounds" over the two queues): the sequence in
// which the sequential algorithm takes nodes is the merge of the sorted leaf
// queue and the internal-node queue (leaf first on equal weight).  It pairs
// the 1st and 2nd node, the 3rd and 4th, ... for as long as the next node
// does not weigh more than w1 = (1st + 2nd): every new node weighs at least w1
// and queues behind every older node of equal weight.  One round pairs all of
// those at once; w1 grows by at least 1.5x per round, so there are O(log n)
// rounds.  Internal nodes are identified by creation order, so the internal
// queue only stores weights.  Depths follow from one pass over the rounds in
// reverse (a parent is always created in a later round than its children).
//
// Sorting: used symbols are collected in ascending symbol order (each warp a
// contiguous segment of the histogram); a stable sort by count then gives the
// (count, symbol) leaf order (a rank sort for small alphabets, else a stable
// LSD radix sort on 10-bit digits with one warp per contiguous segment).  The canonical order
// (ascending length, then symbol) needs no sort: each warp counts its segment
// of the symbol-ordered list per length, one scan gives its first canonical
// index per length, and equal lengths are ranked by lane.
#include "common.cuh"

namespace fp {

constexpr uint32_t kRankMax = 1024;     // rank sort up to this many items
constexpr uint32_t kSmemQueue = 32768;  // internal-node queue in shared memory up to n leaves
constexpr int kRadixBits = 10;          // digit of the sort by count
static_assert((32u << kRadixBits) <= kSmemQueue, "the radix histograms fit the queue area");
constexpr int kMaxRounds = 128;         // w1 grows 1.5x per round: <= 55 rounds for 2^32 points

struct CBArgs {
    DevParams* par;
    const uint32_t* hist;
    uint32_t* enc;
    uint8_t* len_sym;
    uint32_t nsym;
    int lmax;
    const double* sse_part;
    uint32_t n_sse;
    uint32_t* bpre;
    uint32_t nbmblk;
    unsigned long long* list;
    unsigned long long* buf1;
    unsigned long long* buf2;
    uint32_t* parent;
    uint8_t* out;
};

// dynamic shared memory: internal queue (u32 weights) | internal-node depths (u8)
int codebook_smem_bytes() { return (int)(kSmemQueue * 4 + kMaxSym); }

__device__ __forceinline__ uint32_t key_w(unsigned long long k) { return (uint32_t)(k >> 16); }

// Rank sort of n <= kRankMax distinct keys: out[rank] = key.  kbuf: n u64 of smem.
__device__ void rank_sort(const unsigned long long* in, unsigned long long* out, uint32_t n,
                          unsigned long long* kbuf) {
    const uint32_t tid = threadIdx.x;
    if (tid < n) kbuf[tid] = in[tid];
    __syncthreads();
    if (tid < n) {
        const unsigned long long k = kbuf[tid];
        uint32_t r = 0;
        for (uint32_t j = 0; j < n; j++) r += kbuf[j] < k;
        out[r] = k;
    }
    __syncthreads();
}

// One stable LSD radix pass on the DB-bit digit (key >> shift) & (2^DB - 1):
// each warp owns a contiguous segment; per-warp digit counts are scanned in
// (digit, warp) order; within a group of 32 keys, equal digits are ranked by
// lane.  whist: 32 x 2^DB u32 of smem.  Block of 1024 threads.
template <int DB>
__device__ void radix_pass(const unsigned long long* in, unsigned long long* out, uint32_t n,
                           int shift, uint32_t* whist, uint32_t* sh) {
    constexpr uint32_t NB = 1u << DB;
    constexpr uint32_t mask = NB - 1u;
    constexpr int EPT = (int)(NB * 32u / 1024u);  // (digit, warp) entries per thread in the scan
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint32_t S = (n + 31) / 32;
    const uint32_t b0 = min(n, w * S), b1 = min(n, b0 + S);
    for (uint32_t d = lane; d < NB; d += 32) whist[w * NB + d] = 0;
    __syncwarp();
    for (uint32_t i0 = b0 + lane; i0 < b1; i0 += 128) {
        unsigned long long kk[4];
#pragma unroll
        for (int u = 0; u < 4; u++) kk[u] = i0 + 32u * u < b1 ? in[i0 + 32u * u] : 0ull;
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (i0 + 32u * u < b1) atomicAdd(&whist[w * NB + (uint32_t)((kk[u] >> shift) & mask)], 1u);
    }
    __syncthreads();
    uint32_t v[EPT], sum = 0;
#pragma unroll
    for (int k = 0; k < EPT; k++) {
        const uint32_t e = EPT * threadIdx.x + k;  // e = digit * 32 + warp
        v[k] = whist[(e & 31u) * NB + (e >> 5)];
        sum += v[k];
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan(sum, sh, &tot);
#pragma unroll
    for (int k = 0; k < EPT; k++) {
        const uint32_t e = EPT * threadIdx.x + k;
        whist[(e & 31u) * NB + (e >> 5)] = ex;
        ex += v[k];
    }
    __syncthreads();
    for (uint32_t b4 = b0; b4 < b1; b4 += 128) {
        // the keys of four groups of 32 are loaded before the first is placed
        unsigned long long kk[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t i = b4 + 32u * u + lane;
            kk[u] = i < b1 ? in[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t i = b4 + 32u * u + lane;
            const bool valid = i < b1;
            const unsigned long long key = kk[u];
            const uint32_t d = valid ? (uint32_t)((key >> shift) & mask) : 0xffffu;
            // lanes holding the same digit: one ballot per digit bit
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
            for (int b = 0; b < DB; b++) {
                const bool bit = (d >> b) & 1u;
                const uint32_t bb = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? bb : ~bb;
            }
            const uint32_t rank = __popc(peers & lanemask_lt());
            uint32_t pos = 0;
            if (valid) pos = whist[w * NB + d] + rank;
            __syncwarp();
            if (valid) {
                out[pos] = key;
                if ((uint32_t)(__ffs(peers) - 1) == lane) whist[w * NB + d] += __popc(peers);
            }
            __syncwarp();
        }
    }
    __syncthreads();
}

// Warp-cooperative search: first index in [lo, hi) where pred(index) is false,
// pred monotone (true ... true false ... false).  The whole warp calls it.
template <class P>
__device__ __forceinline__ uint32_t warp_first_false(uint32_t lo, uint32_t hi, P pred) {
    const uint32_t lane = threadIdx.x & 31u;
    while (hi - lo > 32) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t probe = lo + (lane + 1) * step - 1;
        const bool t = probe < hi && pred(probe);
        const uint32_t k = __popc(__ballot_sync(0xffffffffu, t));
        const uint32_t nlo = lo + k * step;
        hi = min(hi, nlo + step);
        lo = nlo;
    }
    const uint32_t idx = lo + lane;
    const bool t = idx < hi && pred(idx);
    return lo + __popc(__ballot_sync(0xffffffffu, t));
}

// Two independent warp_first_false searches advanced in lockstep, so that the
// probes of both are in flight together.
template <class P1, class P2>
__device__ __forceinline__ void warp_first_false2(uint32_t lo1, uint32_t hi1, P1 pred1, uint32_t lo2,
                                                  uint32_t hi2, P2 pred2, uint32_t& r1, uint32_t& r2) {
    const uint32_t lane = threadIdx.x & 31u;
    while (hi1 - lo1 > 32 || hi2 - lo2 > 32) {
        const bool a1 = hi1 - lo1 > 32, a2 = hi2 - lo2 > 32;  // warp-uniform
        const uint32_t step1 = (hi1 - lo1 + 31) / 32, step2 = (hi2 - lo2 + 31) / 32;
        const uint32_t q1 = lo1 + (lane + 1) * step1 - 1, q2 = lo2 + (lane + 1) * step2 - 1;
        const bool t1 = a1 && q1 < hi1 && pred1(q1);
        const bool t2 = a2 && q2 < hi2 && pred2(q2);
        const uint32_t k1 = __popc(__ballot_sync(0xffffffffu, t1));
        const uint32_t k2 = __popc(__ballot_sync(0xffffffffu, t2));
        if (a1) {
            const uint32_t nlo = lo1 + k1 * step1;
            hi1 = min(hi1, nlo + step1);
            lo1 = nlo;
        }
        if (a2) {
            const uint32_t nlo = lo2 + k2 * step2;
            hi2 = min(hi2, nlo + step2);
            lo2 = nlo;
        }
    }
    const uint32_t i1 = lo1 + lane, i2 = lo2 + lane;
    const bool t1 = i1 < hi1 && pred1(i1);
    const bool t2 = i2 < hi2 && pred2(i2);
    r1 = lo1 + __popc(__ballot_sync(0xffffffffu, t1));
    r2 = lo2 + __popc(__ballot_sync(0xffffffffu, t2));
}

__global__ void __launch_bounds__(1024, 1) k_codebook(const __grid_constant__ Batch<CBArgs> B) {
    const CBArgs& a = B.a[blockIdx.x];  // one block per field
    extern __shared__ uint32_t dsm[];
    uint32_t* sq = dsm;                                              // internal queue (n <= 32768)
    uint8_t* depth8 = reinterpret_cast<uint8_t*>(dsm + kSmemQueue);  // internal-node depths
    uint32_t* whist = dsm;                                           // radix histograms (alias)
    unsigned long long* kbuf = reinterpret_cast<unsigned long long*>(dsm + 8192);  // rank sort (alias)
    __shared__ uint32_t sh[33];
    __shared__ double sdbl[32];
    __shared__ uint32_t s_m, s_a, s_err, s_max;
    __shared__ uint32_t s_cnt[32], s_fc[32], s_fi[32];
    __shared__ uint32_t s_wn[32], s_wb[32], s_ntot;  // symbol collection: per-warp counts, offsets
    __shared__ uint32_t s_wc[32][33];                // canonical order: [warp][length] counts, then offsets
    __shared__ uint32_t s_round[kMaxRounds + 2];
    DevParams* par = a.par;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;  // 32 warps
    const uint32_t flags = par->flags;

    // ---- squared-error total, fixed order ----
    {
        double v = 0.0;
        for (uint32_t i = tid; i < a.n_sse; i += blockDim.x) v += a.sse_part[i];
        double t = block_sum_double(v, sdbl);
        if (tid == 0) par->sse = (flags & (kFlagConstant | kFlagError)) ? 0.0 : t;
    }
    if (flags & (kFlagConstant | kFlagError)) {
        if (tid == 0) par->n_sym = 0;
        return;
    }
    // ---- exclusive prefix of bitmap block totals (order-preserving ranks) ----
    for (int list = 0; list < 2; list++) {
        const uint32_t cnt = list == 0 ? par->n_out : par->n_vb;
        if (cnt == 0) continue;
        uint32_t* bp = a.bpre + list * a.nbmblk;
        uint32_t carry = 0;
        for (uint32_t base = 0; base < a.nbmblk; base += blockDim.x) {
            uint32_t i = base + tid;
            uint32_t v = i < a.nbmblk ? bp[i] : 0u;
            uint32_t tot;
            uint32_t ex = block_excl_scan(v, sh, &tot);
            if (i < a.nbmblk) bp[i] = ex + carry;
            carry += tot;
        }
    }

    // ---- used symbols in ascending order (only the range the predictor saw) ----
    const uint32_t c0 = a.hist[0];
    uint32_t n = c0 > 0 ? 1u : 0u;
    uint32_t maxc = c0;
    if (tid == 0 && c0 > 0) a.list[0] = (unsigned long long)c0 << 16;
    const uint32_t lo = par->sym_lo, hi = min(par->sym_hi, a.nsym - 1);
    if (lo <= hi) {
        // each warp collects a contiguous segment of the bins, a multiple of 32
        // of them: coalesced loads, ranks within the warp by ballot, one scan of
        // the warps' counts; the second pass reloads the bins (L1 / L2)
        const uint32_t S = ((hi - lo + 1u + 31u) / 32u + 31u) & ~31u;
        const uint32_t wb0 = lo + wid * S;  // the warp's first bin (may lie past hi)
        auto load8 = [&](uint32_t k, uint32_t (&c)[8]) {
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const uint32_t i = wb0 + k + 32u * u + lane;
                c[u] = (k + 32u * u < S && i <= hi) ? a.hist[i] : 0u;
            }
        };
        uint32_t wcnt = 0;
        for (uint32_t k = 0; k < S; k += 256u) {
            uint32_t c[8];
            load8(k, c);
#pragma unroll
            for (int u = 0; u < 8; u++) {
                wcnt += __popc(__ballot_sync(0xffffffffu, c[u] > 0u));
                maxc = max(maxc, c[u]);
            }
        }
        if (lane == 0) s_wn[wid] = wcnt;
        __syncthreads();
        if (wid == 0) {
            const uint32_t v = s_wn[lane];
            uint32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (uint32_t)o) incl += y;
            }
            s_wb[lane] = incl - v;
            if (lane == 31) s_ntot = incl;
        }
        __syncthreads();
        uint32_t pos = n + s_wb[wid];
        for (uint32_t k = 0; k < S; k += 256u) {
            uint32_t c[8];
            load8(k, c);
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const uint32_t m = __ballot_sync(0xffffffffu, c[u] > 0u);
                if (c[u]) a.list[pos + __popc(m & lanemask_lt())] = ((unsigned long long)c[u] << 16) | (wb0 + k + 32u * u + lane);
                pos += __popc(m);
            }
        }
        n += s_ntot;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxc = max(maxc, __shfl_xor_sync(0xffffffffu, maxc, o));
    if (tid == 0) { s_max = 0; s_err = 0; }
    __syncthreads();
    if ((tid & 31) == 0) atomicMax(&s_max, maxc);
    __syncthreads();
    maxc = s_max;

    if (n == 1) {
        if (tid == 0) a.len_sym[(uint32_t)(a.list[0] & 0xffffu)] = 1;
    } else if (n > 1) {
        const bool smallq = n <= kSmemQueue;
        for (int rebuild = 0;; rebuild++) {
            if (rebuild > 40) {  // 33 halvings leave every count at 1, which always fits
                if (tid == 0) set_error(par, FPSNR_ETIMEOUT);
                return;
            }
            // ---- leaves sorted by (count, symbol) ----
            const unsigned long long* leaves;
            unsigned long long* spare;
            if (n <= kRankMax) {
                rank_sort(a.list, a.buf1, n, kbuf);
                leaves = a.buf1;
                spare = a.buf2;
            } else {
                // 10-bit digits: the per-warp histograms (128 KB) fill the queue area
                const int bits = 32 - __clz(maxc);
                const int passes = (bits + kRadixBits - 1) / kRadixBits;
                const unsigned long long* src = a.list;
                unsigned long long* dst = a.buf1;
                for (int pss = 0; pss < passes; pss++) {
                    radix_pass<kRadixBits>(src, dst, n, 16 + kRadixBits * pss, whist, sh);
                    src = dst;
                    dst = (dst == a.buf1) ? a.buf2 : a.buf1;
                }
                leaves = src;
                spare = dst;
            }
            // internal queue, indexed by creation order (capacity >= n - 1)
            uint32_t* iq = smallq ? sq : reinterpret_cast<uint32_t*>(spare);
            // ---- bulk rounds over the two queues ----
            uint32_t lh = 0, ih = 0, it = 0, next = n, L = n;
            int rounds = 0;
            while (L > 1) {
                if (rounds >= kMaxRounds) {
                    if (tid == 0) s_err = 1;
                    break;
                }
                if (tid < 32) {
                    const uint32_t nl = n - lh, ni = it - ih;
                    uint32_t w[2];
                    {
                        uint32_t i = lh, j = ih;
                        for (int t = 0; t < 2; t++) {
                            const bool tl = i < n && (j >= it || key_w(leaves[i]) <= iq[j]);
                            w[t] = tl ? key_w(leaves[i++]) : iq[j++];
                        }
                    }
                    const uint32_t w1 = w[0] + w[1];
                    uint32_t el, ei;
                    warp_first_false2(
                        lh, n, [&](uint32_t x) { return key_w(leaves[x]) <= w1; }, ih, it,
                        [&](uint32_t x) { return iq[x] <= w1; }, el, ei);
                    const uint32_t kl = el - lh, ki = ei - ih;
                    const uint32_t m = (kl + ki) >> 1;
                    // leaves among the first 2m nodes (merge path, leaf first on ties)
                    const uint32_t d = 2 * m;
                    const uint32_t plo = d > ni ? d - ni : 0, phi = min(d, nl);
                    const uint32_t na = warp_first_false(plo, phi, [&](uint32_t x) {
                        return key_w(leaves[lh + x]) <= iq[ih + d - x - 1];
                    });
                    if (tid == 0) {
                        s_m = m;
                        s_a = na;
                        s_round[rounds] = next;
                    }
                }
                __syncthreads();
                const uint32_t m = s_m, na = s_a, nb = 2 * m - na;
                const uint32_t E = (m + blockDim.x - 1) / blockDim.x;
                const uint32_t p0 = tid * E, p1 = min(p0 + E, m);
                if (p0 < p1) {
                    // position of node 2*p0 within the merged prefix (na leaves, nb internal)
                    const uint32_t d = 2 * p0;
                    uint32_t lo2 = d > nb ? d - nb : 0, hi2 = min(d, na);
                    while (lo2 < hi2) {
                        const uint32_t mid = (lo2 + hi2) >> 1;
                        if (key_w(leaves[lh + mid]) <= iq[ih + d - mid - 1]) lo2 = mid + 1;
                        else hi2 = mid;
                    }
                    uint32_t i = lo2, j = d - lo2;
                    for (uint32_t p = p0; p < p1; p++) {
                        uint32_t id[2], w[2];
                        for (int t = 0; t < 2; t++) {
                            const bool tl = i < na && (j >= nb || key_w(leaves[lh + i]) <= iq[ih + j]);
                            if (tl) { id[t] = lh + i; w[t] = key_w(leaves[lh + i]); i++; }
                            else { id[t] = n + ih + j; w[t] = iq[ih + j]; j++; }
                        }
                        a.parent[id[0]] = next + p;
                        a.parent[id[1]] = next + p;
                        // new nodes go behind every live one: [it, it + m) is never read this round
                        iq[it + p] = w[0] + w[1];
                    }
                }
                __syncthreads();
                lh += na;
                ih += nb;
                it += m;
                next += m;
                L -= m;
                rounds++;
            }
            if (s_err) {
                if (tid == 0) set_error(par, FPSNR_ETIMEOUT);
                return;
            }
            if (tid == 0) s_round[rounds] = next;
            __syncthreads();
            // ---- depths: internal nodes round by round from the root down ----
            const uint32_t root = 2 * n - 2;
            for (int r = rounds - 1; r >= 0; r--) {
                const uint32_t r0 = s_round[r], r1 = s_round[r + 1];
                for (uint32_t id = r0 + tid; id < r1; id += blockDim.x)
                    depth8[id - n] = (id == root) ? 0 : (uint8_t)(depth8[a.parent[id] - n] + 1);
                __syncthreads();
            }
            uint32_t mx = 0;
            for (uint32_t i0 = tid; i0 < n; i0 += 4 * blockDim.x) {
                uint32_t pp[4];
#pragma unroll
                for (int u = 0; u < 4; u++) pp[u] = i0 + u * blockDim.x < n ? a.parent[i0 + u * blockDim.x] : 0u;
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (i0 + u * blockDim.x < n) mx = max(mx, (uint32_t)depth8[pp[u] - n] + 1);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (tid == 0) s_max = 0;
            __syncthreads();
            if ((tid & 31) == 0) atomicMax(&s_max, mx);
            __syncthreads();
            if (s_max <= (uint32_t)a.lmax) {
                for (uint32_t i0 = tid; i0 < n; i0 += 4 * blockDim.x) {
                    uint32_t pp[4], ss[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const uint32_t i = i0 + u * blockDim.x;
                        pp[u] = i < n ? a.parent[i] : 0u;
                        ss[u] = i < n ? (uint32_t)(leaves[i] & 0xffffu) : 0u;
                    }
#pragma unroll
                    for (int u = 0; u < 4; u++)
                        if (i0 + u * blockDim.x < n) a.len_sym[ss[u]] = (uint8_t)(depth8[pp[u] - n] + 1);
                }
                break;
            }
            // too long: halve every count (in the symbol-ordered list) and rebuild
            for (uint32_t i = tid; i < n; i += blockDim.x) {
                const unsigned long long k = a.list[i];
                const uint32_t h = key_w(k) >> 1;
                a.list[i] = ((unsigned long long)(h ? h : 1u) << 16) | (k & 0xffffu);
            }
            maxc = (maxc >> 1) ? (maxc >> 1) : 1u;
            __syncthreads();
        }
    }
    __syncthreads();

    // ---- canonical order: ascending (length, symbol) ----
    // The list holds the used symbols in ascending order.  Each warp takes a
    // contiguous segment of it and counts its symbols per code length; a scan
    // over (length, warp) gives every warp its first canonical index for each
    // length, and the warp walks its segment again, ranking equal lengths by
    // lane, and writes the encoder table and the codebook.
    const uint32_t S = (n + 31u) / 32u;  // list entries per warp
    const uint32_t e0 = min(n, wid * S), e1 = min(n, e0 + S);
    s_wc[wid][lane] = 0u;
    __syncwarp();
    // a warp's entries 256 at a time: the symbols, then their lengths, loaded
    // together before they are ranked
    auto load8 = [&](uint32_t i0, uint32_t (&sym)[8], uint32_t (&len)[8]) {
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const uint32_t i = i0 + 32u * u + lane;
            sym[u] = i < e1 ? (uint32_t)(a.list[i] & 0xffffu) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; u++) len[u] = i0 + 32u * u + lane < e1 ? (uint32_t)a.len_sym[sym[u]] : 0u;
    };
    for (uint32_t i0 = e0; i0 < e1; i0 += 256u) {
        uint32_t sym[8], len[8];
        load8(i0, sym, len);
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const bool v = i0 + 32u * u + lane < e1;
            const uint32_t l = len[u];  // 1..lmax for a used symbol
            const uint32_t peers = __match_any_sync(0xffffffffu, l);
            if (v && lane == (uint32_t)(__ffs(peers) - 1)) s_wc[wid][l] += __popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
    uint32_t wex;  // thread (length wid, warp lane): that warp's symbols of this length before it
    {
        const uint32_t v = s_wc[lane][wid];
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        wex = incl - v;
        if (lane == 31) s_cnt[wid] = incl;
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t code = 0, idx = 0;
        for (uint32_t l = 1; l <= (uint32_t)kMaxLmax; l++) {
            if (l > 1) code = (code + s_cnt[l - 1]) << 1;
            s_fc[l] = code;
            s_fi[l] = idx;
            idx += s_cnt[l];
        }
        par->n_sym = n;
        par->off_ct = kHeaderBytes + ((4ull * n + 15u) & ~15ull);
    }
    __syncthreads();
    if (wid >= 1u && wid <= (uint32_t)kMaxLmax) s_wc[lane][wid] = s_fi[wid] + wex;
    __syncthreads();
    const bool write_cb = kHeaderBytes + 4ull * n <= par->cap;
    uint32_t* cb = reinterpret_cast<uint32_t*>(a.out + kHeaderBytes);
    for (uint32_t i0 = e0; i0 < e1; i0 += 256u) {
        uint32_t sym[8], len[8];
        load8(i0, sym, len);
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const bool v = i0 + 32u * u + lane < e1;
            const uint32_t l = len[u];
            const uint32_t peers = __match_any_sync(0xffffffffu, l);
            if (v) {
                const uint32_t idx = s_wc[wid][l] + __popc(peers & lanemask_lt());  // canonical index
                a.enc[sym[u]] = ((s_fc[l] + (idx - s_fi[l])) << 5) | l;
                if (write_cb) cb[idx] = (l << 16) | sym[u];
            }
            __syncwarp();
            if (v && lane == (uint32_t)(__ffs(peers) - 1)) s_wc[wid][l] += __popc(peers);
            __syncwarp();
        }
    }
}

int launch_codebook_batch(fpsnr_plan_s* const* P, void* const* d_out, int count,
                          cudaStream_t st) {
    Batch<CBArgs> b;
    b.count = (uint32_t)count;
    for (int f = 0; f < count; f++) {
        const fpsnr_plan_s* p = P[f];
        const Workspace& w = p->w;
        CBArgs& a = b.a[f];
        a.par = w.par;
        a.hist = w.hist;
        a.enc = w.enc;
        a.len_sym = w.len_sym;
        a.nsym = p->nsym;
        a.lmax = p->lmax;
        a.sse_part = w.sse_part;
        a.n_sse = p->n ? p->pq.nblocks : 0;
        a.bpre = w.bpre;
        a.nbmblk = (uint32_t)p->nbmblk;
        a.list = w.hlist;
        a.buf1 = w.hbuf1;
        a.buf2 = w.hbuf2;
        a.parent = w.hpar;
        a.out = reinterpret_cast<uint8_t*>(d_out[f]);
        b.off[f] = (uint32_t)f;
    }
    b.off[count] = (uint32_t)count;
    StageScope sc(P[0]->prof, kStCodebook, st);
    k_codebook<<<count, 1024, P[0]->cb_smem, st>>>(b);
    return cudaGetLastError() == cudaSuccess ? FPSNR_OK : FPSNR_ECUDA;
}

int codebook_prepare() {
    return cudaFuncSetAttribute(k_codebook, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                codebook_smem_bytes()) == cudaSuccess
               ? FPSNR_OK
               : FPSNR_ECUDA;
}

}  // namespace fp
