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
// Parallel construction ("bulk merge"): with the available nodes kept in one
// sequence ordered as the two-queue algorithm would take them, the sequential
// algorithm pairs (a0,a1), (a2,a3), ... for as long as the next pair's second
// node does not weigh more than a0 + a1 (every new node weighs at least that
// and is queued behind every older node of equal weight).  All those pairs are
// merged at once, and the new nodes are merged back into the sequence with a
// merge path (old node first on equal weight).  The smallest pair sum grows by
// at least 1.5x per round, so there are O(log n) rounds.  Depths come from
// pointer jumping on the parent links.
#include "common.cuh"

namespace fp {

constexpr int kSmemLeaves = 4096;  // alphabets up to this many used symbols stay in shared memory

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
    unsigned long long* gkeys;
    unsigned long long* gA;
    unsigned long long* gB;
    unsigned long long* gN;
    unsigned long long* gnode;
    uint32_t* gpar;
    uint32_t* glw;
    uint16_t* glsym;
    uint8_t* out;
};

int codebook_smem_bytes() {
    // keys | A (node aliases keys+A) | B | N | par | lw | lsym
    return kSmemLeaves * 8 * 2 + kSmemLeaves * 8 + kSmemLeaves * 4 + kSmemLeaves * 2 * 4 +
           kSmemLeaves * 4 + kSmemLeaves * 2;
}

__device__ __forceinline__ uint32_t wgt(unsigned long long v) { return (uint32_t)(v >> 32); }

__device__ void bitonic_sort(unsigned long long* K, uint32_t P) {
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
                uint32_t ixj = i ^ j;
                if (ixj > i) {
                    unsigned long long x = K[i], y = K[ixj];
                    bool up = (i & k) == 0;
                    if ((x > y) == up) { K[i] = y; K[ixj] = x; }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(1024, 1) k_codebook(CBArgs a) {
    extern __shared__ unsigned long long dsm[];
    __shared__ uint32_t sh[33];
    __shared__ double sdbl[32];
    __shared__ uint32_t s_val, s_any;
    __shared__ uint32_t s_cnt[32], s_fc[32], s_fi[32], s_carry[32];
    __shared__ uint32_t s_wcnt[32][28];
    DevParams* par = a.par;
    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31u, warp = tid >> 5;
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

    // ---- used symbols, ascending symbol order ----
    for (uint32_t s = tid; s < a.nsym; s += blockDim.x) a.len_sym[s] = 0;
    uint32_t n = 0;
    for (uint32_t base = 0; base < a.nsym; base += blockDim.x) {
        const uint32_t s = base + tid;
        const uint32_t c = s < a.nsym ? a.hist[s] : 0u;
        uint32_t tot;
        uint32_t ex = block_excl_scan(c > 0 ? 1u : 0u, sh, &tot);
        if (c > 0) a.gkeys[n + ex] = ((unsigned long long)c << 16) | s;
        n += tot;
    }
    __syncthreads();

    if (n == 1) {
        if (tid == 0) a.len_sym[(uint32_t)(a.gkeys[0] & 0xffffu)] = 1;
    } else if (n > 1) {
        const bool small = n <= (uint32_t)kSmemLeaves;
        unsigned long long* keys = small ? dsm : a.gkeys;
        unsigned long long* A = small ? dsm + kSmemLeaves : a.gA;
        unsigned long long* B = small ? dsm + 2 * kSmemLeaves : a.gB;
        unsigned long long* Nn = small ? dsm + 3 * kSmemLeaves : a.gN;
        unsigned long long* node = small ? dsm : a.gnode;  // aliases keys + A when small
        uint32_t* par_ = small ? reinterpret_cast<uint32_t*>(dsm + 3 * kSmemLeaves + kSmemLeaves / 2)
                               : a.gpar;
        uint32_t* lw = small ? par_ + 2 * kSmemLeaves : a.glw;
        uint16_t* lsym = small ? reinterpret_cast<uint16_t*>(lw + kSmemLeaves) : a.glsym;
        if (small)
            for (uint32_t i = tid; i < n; i += blockDim.x) keys[i] = a.gkeys[i];
        uint32_t P = 2;
        while (P < n) P <<= 1;
        __syncthreads();
        // each rebuild halves every count > 1, so 33 rebuilds leave all counts at 1,
        // whose code fits 2^lmax >= 2R symbols; the cap only guards against a fault
        for (int rebuild = 0;; rebuild++) {
            if (rebuild > 40) {
                if (tid == 0) set_error(par, FPSNR_ETIMEOUT);
                return;
            }
            for (uint32_t i = n + tid; i < P; i += blockDim.x) keys[i] = ~0ull;
            __syncthreads();
            bitonic_sort(keys, P);
            for (uint32_t i = tid; i < n; i += blockDim.x) {
                const unsigned long long k = keys[i];
                lsym[i] = (uint16_t)(k & 0xffffu);
                lw[i] = (uint32_t)(k >> 16);
                A[i] = ((k >> 16) << 32) | i;
            }
            __syncthreads();
            // bulk merge rounds
            uint32_t L = n, next = n;
            unsigned long long* cur = A;
            unsigned long long* oth = B;
            while (L > 1) {
                if (tid == 0) {
                    const uint32_t w1 = wgt(cur[0]) + wgt(cur[1]);
                    uint32_t lo = 2, hi = L;  // first index with weight > w1
                    while (lo < hi) {
                        uint32_t mid = (lo + hi) >> 1;
                        if (wgt(cur[mid]) <= w1) lo = mid + 1;
                        else hi = mid;
                    }
                    s_val = lo >> 1;
                }
                __syncthreads();
                const uint32_t m = s_val;
                for (uint32_t i = tid; i < m; i += blockDim.x) {
                    const unsigned long long x0 = cur[2 * i], x1 = cur[2 * i + 1];
                    const uint32_t id = next + i;
                    par_[(uint32_t)x0] = id;
                    par_[(uint32_t)x1] = id;
                    Nn[i] = ((unsigned long long)(wgt(x0) + wgt(x1)) << 32) | id;
                }
                __syncthreads();
                const unsigned long long* O = cur + 2 * m;
                const uint32_t no = L - 2 * m, tot = L - m;
                const uint32_t E = (tot + blockDim.x - 1) / blockDim.x;
                const uint32_t t0 = tid * E;
                if (t0 < tot) {
                    uint32_t lo = t0 > m ? t0 - m : 0, hi = min(t0, no);
                    while (lo < hi) {
                        uint32_t mid = (lo + hi) >> 1;
                        if (wgt(O[mid]) <= wgt(Nn[t0 - mid - 1])) lo = mid + 1;
                        else hi = mid;
                    }
                    uint32_t i = lo, j = t0 - lo;
                    const uint32_t t1 = min(t0 + E, tot);
                    for (uint32_t t = t0; t < t1; t++) {
                        if (j >= m || (i < no && wgt(O[i]) <= wgt(Nn[j]))) oth[t] = O[i++];
                        else oth[t] = Nn[j++];
                    }
                }
                __syncthreads();
                unsigned long long* tmp = cur;
                cur = oth;
                oth = tmp;
                L = tot;
                next += m;
            }
            // depths by pointer jumping: node[v] = (distance << 32) | ancestor
            const uint32_t total = 2 * n - 1, root = total - 1;
            for (uint32_t v = tid; v < total; v += blockDim.x)
                node[v] = (v == root) ? (unsigned long long)root
                                      : ((1ull << 32) | par_[v]);
            __syncthreads();
            // pointer jumping halves every remaining distance: 18 rounds reach the root
            // of a 2^17-node tree; 64 rounds can only be exceeded by a broken tree
            for (int round = 0;; round++) {
                if (round > 64) {
                    if (tid == 0) set_error(par, FPSNR_ETIMEOUT);
                    return;
                }
                uint32_t changed = 0;
                for (uint32_t v = tid; v < total; v += blockDim.x) {
                    const unsigned long long e = node[v];
                    const uint32_t anc = (uint32_t)e;
                    if (anc != root) {
                        const unsigned long long f = node[anc];
                        node[v] = (((e >> 32) + (f >> 32)) << 32) | (uint32_t)f;
                        changed = 1;
                    }
                }
                if (!__syncthreads_or(changed)) break;
            }
            uint32_t mx = 0;
            for (uint32_t i = tid; i < n; i += blockDim.x) mx = max(mx, (uint32_t)(node[i] >> 32));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (tid == 0) s_any = 0;
            __syncthreads();
            if (lane == 0) atomicMax(&s_any, mx);
            __syncthreads();
            if (s_any <= (uint32_t)a.lmax) {
                for (uint32_t i = tid; i < n; i += blockDim.x)
                    a.len_sym[lsym[i]] = (uint8_t)(node[i] >> 32);
                break;
            }
            // too long: halve the counts and rebuild (keys alias node when small)
            __syncthreads();
            for (uint32_t i = tid; i < n; i += blockDim.x) {
                uint32_t h = lw[i] >> 1;
                keys[i] = ((unsigned long long)(h ? h : 1u) << 16) | lsym[i];
            }
            __syncthreads();
        }
    }
    __syncthreads();

    // ---- canonical codes ----
    if (tid < 32) { s_cnt[tid] = 0; s_carry[tid] = 0; }
    __syncthreads();
    for (uint32_t s = tid; s < a.nsym; s += blockDim.x) {
        uint32_t l = a.len_sym[s];
        if (l) atomicAdd(&s_cnt[l], 1u);
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
    const bool write_cb = kHeaderBytes + 4ull * n <= par->cap;
    uint32_t* cb = reinterpret_cast<uint32_t*>(a.out + kHeaderBytes);
    for (uint32_t base = 0; base < a.nsym; base += blockDim.x) {
        const uint32_t s = base + tid;
        const uint32_t l = s < a.nsym ? a.len_sym[s] : 0u;
        const uint32_t peers = __match_any_sync(0xffffffffu, l);
        const uint32_t rank = __popc(peers & lanemask_lt());
        if (lane < 28) s_wcnt[warp][lane] = 0;
        __syncwarp();
        if ((uint32_t)(__ffs(peers) - 1) == lane) s_wcnt[warp][l] = __popc(peers);
        __syncthreads();
        if (tid < 28) {
            uint32_t run = s_carry[tid];
            for (uint32_t wv = 0; wv < 32; wv++) {
                uint32_t c = s_wcnt[wv][tid];
                s_wcnt[wv][tid] = run;
                run += c;
            }
            s_carry[tid] = run;
        }
        __syncthreads();
        if (s < a.nsym) {
            if (l) {
                const uint32_t pos = s_wcnt[warp][l] + rank;  // rank among length-l symbols
                const uint32_t code = s_fc[l] + pos;
                a.enc[s] = (code << 5) | l;
                if (write_cb) cb[s_fi[l] + pos] = (l << 16) | s;
            } else {
                a.enc[s] = 0u;
            }
        }
        __syncthreads();
    }
}

int launch_codebook(fpsnr_plan_s* p, void* d_out, cudaStream_t st) {
    const Workspace& w = p->w;
    CBArgs a;
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
    a.gkeys = w.hkeys;
    a.gA = w.hseqA;
    a.gB = w.hseqB;
    a.gN = w.hnew;
    a.gnode = w.hnode;
    a.gpar = w.hpar;
    a.glw = w.hlw;
    a.glsym = w.hlsym;
    a.out = reinterpret_cast<uint8_t*>(d_out);
    StageScope sc(p->prof, kStCodebook, st);
    k_codebook<<<1, 1024, p->cb_smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? FPSNR_OK : FPSNR_ECUDA;
}

int codebook_prepare() {
    return cudaFuncSetAttribute(k_codebook, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                codebook_smem_bytes()) == cudaSuccess
               ? FPSNR_OK
               : FPSNR_ECUDA;
}

}  // namespace fp
