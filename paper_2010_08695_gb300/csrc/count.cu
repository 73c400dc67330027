// Per-vertex butterfly counting, Algorithm 1 (pvBcnt).
//
// For every start point sp (both sides), every middle point mp in N_sp and
// every end point ep in N_mp with label(ep) < label(mp) and label(ep) <
// label(sp), wdg[ep] counts the wedges sp-mp-ep. Then C(wdg[ep], 2) goes to
// ep and to sp, and wdg[ep] - 1 goes to mp once per wedge (Algorithm 1,
// "same side" and "opposite side" contributions).
//
// Because neighbour lists are sorted by label, the admissible end points of
// (sp, mp) are a PREFIX of N_mp: those with local id < min(sp, below[mp]).
// A first kernel finds every prefix length by binary search, a scan gives
// each start point's exact wedge count W(sp), and start points are split into
// tiers: W <= 256 -> warp per start point; larger -> CTA per start point with
// the hybrid shared-memory engine; hubs (degree >= 2^16) and anchors whose
// repeat table overflowed -> CTA with global dense counters.
#include "engine.cuh"
#include "internal.cuh"

#include <algorithm>
#include <mutex>
#include <string>

namespace receipt {

namespace {

// plen[q] for every CSR position q of side A (edge sp -> mp)
__global__ void k_prefix_len(const int64_t *__restrict__ offA, const int32_t *__restrict__ adjA,
                             int32_t nA, const int64_t *__restrict__ offB,
                             const int32_t *__restrict__ adjB, const int32_t *__restrict__ belowB,
                             int64_t m, int32_t *__restrict__ plen) {
    // one thread per position; find owner sp by binary search on offA
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m) return;
    int32_t lo = 0, hi = nA - 1;
    while (lo < hi) {
        int32_t mid = (lo + hi + 1) >> 1;
        if (offA[mid] <= q)
            lo = mid;
        else
            hi = mid - 1;
    }
    int32_t sp = lo;
    int32_t mp = adjA[q];
    int32_t lim = min(sp, belowB[mp]);
    int64_t b = offB[mp], e = offB[mp + 1];
    plen[q] = (int32_t)lower_bound_i32(adjB + b, e - b, lim);
}

__global__ void k_plen_i64(const int32_t *__restrict__ plen, int64_t m, int64_t *__restrict__ out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < m) out[q] = plen[q];
}

// Start points with at most HASH_W wedges (and more than WARP_MAX_W) take the
// shared hash tier: small CTAs, any key space, any degree.
constexpr int HASH_SLOTS = 4096;
constexpr int HASH_W = HASH_SLOTS / 2;
constexpr int HASH_THREADS = 256;
using CountHash = CtaHashT<HASH_SLOTS>;

// Splits start points into tiers by their exact wedge count (lh: the hash
// tier, null to leave it out).
__global__ void k_count_tiers(const int64_t *__restrict__ offA, const int64_t *__restrict__ pscan,
                              int32_t nA, int64_t m, int64_t cta_keyspace_max,
                              int32_t *__restrict__ lw, int32_t *__restrict__ lc,
                              int32_t *__restrict__ lg, int32_t *__restrict__ lh,
                              int32_t *__restrict__ nl, unsigned long long *wedges) {
    int32_t sp = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long wsum = 0;
    if (sp < nA) {
        int64_t b = offA[sp], e = offA[sp + 1];
        int64_t pb = pscan[b];
        int64_t pe = e < m ? pscan[e] : pscan[m];
        int64_t W = pe - pb;
        wsum = (unsigned long long)W;
        if (W > 0) {
            int64_t deg = e - b;
            if (W <= WARP_MAX_W)
                lw[atomicAdd(&nl[0], 1)] = sp;
            else if (lh && W <= HASH_W)
                lh[atomicAdd(&nl[8], 1)] = sp;
            else if (deg < 65535 && sp <= cta_keyspace_max)
                lc[atomicAdd(&nl[1], 1)] = sp;
            else
                lg[atomicAdd(&nl[2], 1)] = sp;
        }
    }
    wsum = warp_sum(wsum);
    if ((threadIdx.x & 31) == 0 && wsum) atomicAdd(wedges, wsum);
}

struct CountMids {
    const int32_t *adjA;
    const int64_t *offB;
    const int32_t *plen;
    __device__ __forceinline__ void seg(int64_t q, int64_t &beg, int32_t &len) const {
        int32_t mp = adjA[q];
        beg = offB[mp];
        len = plen[q];
    }
};

struct CountArgs {
    const int64_t *offA;
    const int32_t *adjA;
    const int64_t *offB;
    const int32_t *adjB;
    const int32_t *plen;
    unsigned long long *cntA;
    unsigned long long *cntB;
    const int32_t *list;
    const int32_t *nlist;  // device count
    int32_t *work;         // device work counter
};

// ---------------- warp tier ----------------
__global__ void __launch_bounds__(256) k_count_warp(CountArgs a) {
    __shared__ int32_t skey[8][WARP_SLOTS];
    __shared__ uint32_t sval[8][WARP_SLOTS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    WarpHash H{skey[w], sval[w]};
    H.clear(lane);
    __syncwarp();
    const int32_t n = *a.nlist;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(a.work, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= n) break;
        const int32_t sp = a.list[idx];
        const int64_t q0 = a.offA[sp], q1 = a.offA[sp + 1];
        for (int64_t qb = q0; qb < q1; qb += 32) {
            int64_t q = qb + lane;
            int64_t beg = 0;
            int32_t len = 0;
            if (q < q1) {
                beg = a.offB[a.adjA[q]];
                len = a.plen[q];
            }
            int cnt = (int)imin64(32, q1 - qb);
            for (int t = 0; t < cnt; t++) {
                int64_t b = __shfl_sync(0xffffffffu, beg, t);
                int32_t l = __shfl_sync(0xffffffffu, len, t);
                for (int p = lane; p < l; p += 32) H.add(a.adjB[b + p]);
            }
        }
        __syncwarp();
        // same side: C(c,2) to ep and (summed) to sp
        unsigned long long acc = 0;
        for (int i = lane; i < WARP_SLOTS; i += 32) {
            int32_t k = skey[w][i];
            if (k != EMPTY_KEY) {
                uint32_t c = sval[w][i];
                if (c >= 2) {
                    unsigned long long b = choose2(c);
                    atomicAdd(&a.cntA[k], b);
                    acc += b;
                }
            }
        }
        acc = warp_sum(acc);
        if (lane == 0 && acc) atomicAdd(&a.cntA[sp], acc);
        // opposite side: sum over the prefix of mp of (c - 1)
        for (int64_t q = q0; q < q1; q++) {
            int32_t l = a.plen[q];
            if (l == 0) continue;
            int32_t mp = a.adjA[q];
            int64_t b = a.offB[mp];
            unsigned long long s = 0;
            for (int p = lane; p < l; p += 32) s += H.lookup(a.adjB[b + p]) - 1u;
            s = warp_sum(s);
            if (lane == 0 && s) atomicAdd(&a.cntB[mp], s);
        }
        __syncwarp();
        H.clear(lane);
        __syncwarp();
    }
}

// ---------------- CTA tiers ----------------
template <class Eng>
struct CountSameEmit {
    unsigned long long *cntA;
    unsigned long long acc;
    __device__ void operator()(int32_t k, uint32_t c) {
        unsigned long long b = choose2(c);
        atomicAdd(&cntA[k], b);
        acc += b;
    }
};

template <class Eng>
struct CountOppVisit {
    Eng *eng;
    unsigned long long *sacc;  // per-mid accumulator (shared)
    __device__ void operator()(int k, int32_t key) {
        uint32_t c = eng->count(key);
        if (c > 1) atomicAdd(&sacc[k], (unsigned long long)(c - 1));
    }
    // One walk step: where all the warp's wedges of a group share one middle
    // vertex (long lists), the warp sums its contributions first and makes
    // one shared-memory atomic instead of 32 to the same word.
    template <int N>
    __device__ __forceinline__ void many(const int (&kk)[N], const int32_t (&key)[N]) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int u = 0; u < N; u++) {
            uint32_t v = 0;
            if (key[u] >= 0) {
                const uint32_t c = eng->count(key[u]);
                v = c > 1 ? c - 1 : 0;
            }
            const int k = key[u] >= 0 ? kk[u] : -1;
            const unsigned valid = __ballot_sync(0xffffffffu, k >= 0);
            if (!valid) continue;
            const int kl = __shfl_sync(0xffffffffu, k, __ffs(valid) - 1);
            if (__all_sync(0xffffffffu, k < 0 || k == kl)) {
                const uint32_t sum = __reduce_add_sync(0xffffffffu, v);
                if (lane == 0 && sum) atomicAdd(&sacc[kl], (unsigned long long)sum);
            } else if (v) {
                atomicAdd(&sacc[k], (unsigned long long)v);
            }
        }
    }
};

struct CountOppHook {
    const int32_t *adjA;
    unsigned long long *cntB;
    unsigned long long *sacc;
    __device__ void operator()(int64_t c0, int nm) {
        if ((int)threadIdx.x < nm) {
            unsigned long long s = sacc[threadIdx.x];
            if (s) atomicAdd(&cntB[adjA[c0 + threadIdx.x]], s);
            sacc[threadIdx.x] = 0;
        }
    }
};

template <class Eng>
struct AddVisit {
    Eng *eng;
    __device__ __forceinline__ void operator()(int, int32_t key) { eng->add(key); }
};

__device__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long *tmp) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) tmp[w] = v;
    __syncthreads();
    unsigned long long r = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) r += tmp[i];
    __syncthreads();
    return r;
}

__global__ void __maxnreg__(64) k_count_cta(CountArgs a, int32_t head_cap,
                                                        int32_t bm_cap, int32_t *over_list,
                                                        int32_t *n_over) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_idx, s_used, s_over;
    __shared__ unsigned long long s_red[32];
    CtaHybrid H;
    unsigned char *p = H.bind(smem, head_cap, bm_cap, &s_used, &s_over);
    Chunk ch;
    ch.beg = (int64_t *)p;
    unsigned long long *sacc = (unsigned long long *)(ch.beg + MID_CHUNK);
    ch.pre = (int32_t *)(sacc + MID_CHUNK);
    ch.tmp = ch.pre + MID_CHUNK + 1;
    ch.len = chunk_len_ptr(ch.tmp);
    H.clear_all();
    for (int i = threadIdx.x; i < MID_CHUNK; i += blockDim.x) sacc[i] = 0;
    __syncthreads();
    const int32_t n = *a.nlist;
    CountMids M{a.adjA, a.offB, a.plen};
    NoEmit ne;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(a.work, 1);
        __syncthreads();
        int idx = s_idx;
        if (idx >= n) break;
        const int32_t sp = a.list[idx];
        const int64_t q0 = a.offA[sp], q1 = a.offA[sp + 1];
        H.set_range((int32_t)imin64(head_cap, sp), sp);
        AddVisit<CtaHybrid> add{&H};
        cta_walk(M, q0, q1, a.adjB, ch, add);
        const bool over = s_over;
        if (!over) {
            CountSameEmit<CtaHybrid> em{a.cntA, 0};
            H.sweep<true, false>(em);
            unsigned long long tot = block_sum_u64(em.acc, s_red);
            if (threadIdx.x == 0 && tot) atomicAdd(&a.cntA[sp], tot);
            CountOppVisit<CtaHybrid> ov{&H, sacc};
            CountOppHook hook{a.adjA, a.cntB, sacc};
            cta_walk(M, q0, q1, a.adjB, ch, ov, &hook);
        } else if (threadIdx.x == 0) {
            over_list[atomicAdd(n_over, 1)] = sp;
        }
        __syncthreads();
        H.sweep<false, true>(ne);
        __syncthreads();
        H.reset_scalars();
    }
}

__global__ void __maxnreg__(64) k_count_global(CountArgs a, const int32_t *over_list,
                                                           const int32_t *n_over, uint32_t *gcnt,
                                                           int32_t *gtouch, int64_t keyspace) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_idx, s_nt;
    __shared__ unsigned long long s_red[32];
    Chunk ch;
    ch.beg = (int64_t *)smem;
    unsigned long long *sacc = (unsigned long long *)(ch.beg + MID_CHUNK);
    ch.pre = (int32_t *)(sacc + MID_CHUNK);
    ch.tmp = ch.pre + MID_CHUNK + 1;
    ch.len = chunk_len_ptr(ch.tmp);
    GlobalDense G{gcnt + (size_t)blockIdx.x * keyspace, gtouch + (size_t)blockIdx.x * keyspace, &s_nt};
    for (int i = threadIdx.x; i < MID_CHUNK; i += blockDim.x) sacc[i] = 0;
    const int32_t n1 = *a.nlist, n2 = *n_over;
    CountMids M{a.adjA, a.offB, a.plen};
    for (;;) {
        if (threadIdx.x == 0) {
            s_idx = atomicAdd(a.work, 1);
            s_nt = 0;
        }
        __syncthreads();
        int idx = s_idx;
        if (idx >= n1 + n2) break;
        const int32_t sp = idx < n1 ? a.list[idx] : over_list[idx - n1];
        const int64_t q0 = a.offA[sp], q1 = a.offA[sp + 1];
        AddVisit<GlobalDense> add{&G};
        cta_walk(M, q0, q1, a.adjB, ch, add);
        CountSameEmit<GlobalDense> em{a.cntA, 0};
        G.flush(em);
        unsigned long long tot = block_sum_u64(em.acc, s_red);
        if (threadIdx.x == 0 && tot) atomicAdd(&a.cntA[sp], tot);
        CountOppVisit<GlobalDense> ov{&G, sacc};
        CountOppHook hook{a.adjA, a.cntB, sacc};
        cta_walk(M, q0, q1, a.adjB, ch, ov, &hook);
        G.clear();
        __syncthreads();
    }
}

// Start points with at most HASH_W wedges: one 256-thread CTA each (several
// per SM) with a shared hash table; the same two walks as the CTA tier.
__global__ void __launch_bounds__(HASH_THREADS, 4) k_count_hash(CountArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_idx, s_nt;
    __shared__ unsigned long long s_red[32];
    CountHash H;
    unsigned char *p = H.bind(smem, &s_nt);
    Chunk ch;
    ch.beg = (int64_t *)p;
    unsigned long long *sacc = (unsigned long long *)(ch.beg + HASH_THREADS);
    ch.pre = (int32_t *)(sacc + HASH_THREADS);
    ch.tmp = ch.pre + HASH_THREADS + 1;
    ch.len = chunk_len_ptr(ch.tmp);
    H.clear_all();
    for (int i = threadIdx.x; i < HASH_THREADS; i += blockDim.x) sacc[i] = 0;
    __syncthreads();
    const int32_t n = *a.nlist;
    CountMids M{a.adjA, a.offB, a.plen};
    NoEmit ne;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(a.work, 1);
        __syncthreads();
        const int idx = s_idx;
        if (idx >= n) break;
        const int32_t sp = a.list[idx];
        const int64_t q0 = a.offA[sp], q1 = a.offA[sp + 1];
        AddVisit<CountHash> add{&H};
        cta_walk(M, q0, q1, a.adjB, ch, add);
        CountSameEmit<CountHash> em{a.cntA, 0};
        H.sweep<true, false>(em);
        const unsigned long long tot = block_sum_u64(em.acc, s_red);
        if (threadIdx.x == 0 && tot) atomicAdd(&a.cntA[sp], tot);
        CountOppVisit<CountHash> ov{&H, sacc};
        CountOppHook hook{a.adjA, a.cntB, sacc};
        cta_walk(M, q0, q1, a.adjB, ch, ov, &hook);
        H.sweep<false, true>(ne);
        __syncthreads();
        H.reset_scalars();
    }
}

size_t count_hash_smem() { return CountHash::bytes() + HASH_THREADS * 8 + chunk_bytes(HASH_THREADS); }

__global__ void k_scatter_counts(const unsigned long long *__restrict__ cnt,
                                 const int32_t *__restrict__ new2old, int32_t n,
                                 unsigned long long *__restrict__ out) {
    int32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n) out[new2old[x]] = cnt[x];
}

}  // namespace

size_t count_cta_smem(int64_t keyspace, int32_t *head_cap, int32_t *bm_cap) {
    return hybrid_bytes(keyspace, head_cap, bm_cap) + MID_CHUNK * 8 /*sacc*/ + CHUNK_BYTES;
}

// Counts butterflies of both sides into cnt_local[side] (local ids, zeroed
// here). Returns wedges traversed.
uint64_t count_local(const receipt_graph *g, unsigned long long *cnt_u,
                     unsigned long long *cnt_v, cudaStream_t s, int64_t *points) {
    const int64_t m = g->m;
    RC_CUDA(cudaMemsetAsync(cnt_u, 0, sizeof(unsigned long long) * (g->nu > 0 ? g->nu : 1), s));
    RC_CUDA(cudaMemsetAsync(cnt_v, 0, sizeof(unsigned long long) * (g->nv > 0 ? g->nv : 1), s));
    if (m == 0) return 0;
    const int sms = num_sms();
    DevBuf<int32_t> ctr(16, s);
    DevBuf<unsigned long long> wedges(1, s);
    wedges.zero();
    for (int A = 0; A < 2; A++) {
        const Side &SA = g->side[A];
        const Side &SB = g->side[1 - A];
        const int32_t nA = SA.n;
        if (nA == 0) continue;
        ctr.zero();
        DevBuf<int32_t> plen(m, s);
        DevBuf<int64_t> p64(m + 1, s), pscan(m + 1, s);
        k_prefix_len<<<ceil_div(m, 256), 256, 0, s>>>(SA.off, SA.adj, nA, SB.off, SB.adj, SB.below,
                                                      m, plen.get());
        RC_LAUNCH();
        k_plen_i64<<<ceil_div(m, 256), 256, 0, s>>>(plen.get(), m, p64.get());
        RC_LAUNCH();
        RC_CUDA(cudaMemsetAsync(p64.get() + m, 0, sizeof(int64_t), s));
        scan_exclusive<int64_t>(p64.get(), pscan.get(), m + 1, s);
        p64.release();
        // key space of a CTA-tier start point is [0, sp): start points up to
        // the largest key space that fits in shared memory use the CTA tier
        const int64_t cta_ks_max = max_cta_keyspace(nA, MID_CHUNK * 8 + CHUNK_BYTES);
        int32_t headn = 0, bmw = 0;
        size_t smem = cta_ks_max > 0 ? count_cta_smem(cta_ks_max, &headn, &bmw) : 0;
        DevBuf<int32_t> lw(nA, s), lc(nA, s), lg(nA, s), lo(nA, s), lh(nA, s);
        // [0] warp [1] cta [2] global [3] overflow, [4..7] work, [8] hash, [9] its work
        int32_t *nl = ctr.get();
        k_count_tiers<<<ceil_div(nA, 256), 256, 0, s>>>(SA.off, pscan.get(), nA, m, cta_ks_max,
                                                       lw.get(), lc.get(), lg.get(), lh.get(), nl,
                                                       wedges.get());
        RC_LAUNCH();
        unsigned long long *cA = A ? cnt_v : cnt_u;
        unsigned long long *cB = A ? cnt_u : cnt_v;
        CountArgs a{SA.off, SA.adj, SB.off, SB.adj, plen.get(), cA, cB, lw.get(), nl + 0, nl + 4};
        k_count_warp<<<sms * 8, 256, 0, s>>>(a);
        RC_LAUNCH();
        {
            const size_t hsm = count_hash_smem();
            allow_max_smem((const void *)k_count_hash);
            int occ = 1;
            RC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_count_hash, HASH_THREADS,
                                                                  hsm));
            CountArgs c = a;
            c.list = lh.get();
            c.nlist = nl + 8;
            c.work = nl + 9;
            k_count_hash<<<sms * std::max(1, occ), HASH_THREADS, hsm, s>>>(c);
            RC_LAUNCH();
        }
        if (cta_ks_max > 0) {
            allow_max_smem((const void *)k_count_cta);
            CountArgs c = a;
            c.list = lc.get();
            c.nlist = nl + 1;
            c.work = nl + 5;
            k_count_cta<<<sms, CTA_THREADS, smem, s>>>(c, headn, bmw, lo.get(), nl + 3);
            RC_LAUNCH();
        }
        // global tier: hubs + overflowed anchors; key space [0, nA)
        int32_t hn[10];
        RC_CUDA(cudaMemcpyAsync(hn, nl, sizeof(hn), cudaMemcpyDeviceToHost, s));
        RC_CUDA(cudaStreamSynchronize(s));
        if (points) {
            points[0] += hn[0];
            points[1] += hn[8];
            points[2] += hn[1];
            points[3] += hn[2];
            points[4] += hn[3];
        }
        if (hn[2] + hn[3] > 0) {
            const int gblocks = std::min(sms, hn[2] + hn[3]);
            DevBuf<uint32_t> gcnt((size_t)gblocks * nA, s);
            DevBuf<int32_t> gtouch((size_t)gblocks * nA, s);
            gcnt.zero();
            CountArgs c = a;
            c.list = lg.get();
            c.nlist = nl + 2;
            c.work = nl + 6;
            size_t gsm = MID_CHUNK * 8 + CHUNK_BYTES;
            allow_max_smem((const void *)k_count_global);
            k_count_global<<<gblocks, CTA_THREADS, gsm, s>>>(c, lo.get(), nl + 3, gcnt.get(),
                                                             gtouch.get(), nA);
            RC_LAUNCH();
        }
    }
    unsigned long long h = 0;
    RC_CUDA(cudaMemcpyAsync(&h, wedges.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaStreamSynchronize(s));
    return h;
}

void scatter_to_original(const unsigned long long *local, const int32_t *new2old, int32_t n,
                         unsigned long long *out, cudaStream_t s) {
    if (n <= 0) return;
    k_scatter_counts<<<ceil_div(n, 256), 256, 0, s>>>(local, new2old, n, out);
    RC_LAUNCH();
}

}  // namespace receipt

// ---------------------------------------------------------------------
// Butterfly counting that allocates no device memory
// ---------------------------------------------------------------------
// Every temporary of the counting pass (local counts, prefix lengths, tier
// lists, work counters and the global-tier counter slots) is carved out of
// one statically sized array in this library's device image, so the call
// makes no cudaMalloc/cudaFree and no allocating library call. The array's
// size fixes the largest graph it accepts.
namespace receipt {

namespace {

constexpr int32_t NOALLOC_MAX_SIDE = 65536;   // vertices per side
constexpr int64_t NOALLOC_MAX_M = 1 << 20;    // edges (after duplicate removal)
constexpr int NOALLOC_GSLOTS = 8;             // CTAs of the global-counter tier

constexpr size_t na_round(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t NA_CNT = na_round(8 * (size_t)NOALLOC_MAX_SIDE);
constexpr size_t NA_PLEN = na_round(4 * (size_t)NOALLOC_MAX_M);
constexpr size_t NA_LIST = na_round(4 * (size_t)NOALLOC_MAX_SIDE);
constexpr size_t NA_GLOB = na_round(4 * (size_t)NOALLOC_GSLOTS * NOALLOC_MAX_SIDE);
constexpr size_t NA_MISC = 256;
constexpr size_t NOALLOC_BYTES = 2 * NA_CNT + NA_PLEN + 4 * NA_LIST + 2 * NA_GLOB + NA_MISC;

// ~11 MB per device, held from module load until the process exits.
static __device__ __align__(256) unsigned char g_count_scratch[NOALLOC_BYTES];

std::mutex g_na_mu;
void *g_na_ptr[64] = {nullptr};

// Device address of the scratch array for the current device; looked up once
// per device (host code may not use the symbol itself as an address).
unsigned char *noalloc_scratch() {
    int d = 0;
    RC_CUDA(cudaGetDevice(&d));
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[d & 63]) {
        void *p = nullptr;
        RC_CUDA(cudaGetSymbolAddress(&p, g_count_scratch));
        g_na_ptr[d & 63] = p;
    }
    return (unsigned char *)g_na_ptr[d & 63];
}

// Wedge count W(sp) of every start point summed directly from its prefix
// lengths (one warp per start point), then the same tier split as above.
__global__ void k_count_tiers_direct(const int64_t *__restrict__ offA, const int32_t *__restrict__ plen,
                                     int32_t nA, int64_t cta_keyspace_max, int32_t *__restrict__ lw,
                                     int32_t *__restrict__ lc, int32_t *__restrict__ lg,
                                     int32_t *__restrict__ nl) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sp = warp; sp < nA; sp += nwarps) {
        const int64_t b = offA[sp], e = offA[sp + 1];
        int64_t W = 0;
        for (int64_t q = b + lane; q < e; q += 32) W += plen[q];
        W = warp_sum(W);
        if (lane == 0 && W > 0) {
            const int64_t deg = e - b;
            if (W <= WARP_MAX_W)
                lw[atomicAdd(&nl[0], 1)] = (int32_t)sp;
            else if (deg < 65535 && sp <= cta_keyspace_max)
                lc[atomicAdd(&nl[1], 1)] = (int32_t)sp;
            else
                lg[atomicAdd(&nl[2], 1)] = (int32_t)sp;
        }
    }
}

}  // namespace

void count_noalloc(const receipt_graph *g, unsigned long long *d_cnt_u,
                   unsigned long long *d_cnt_v, cudaStream_t s) {
    if (g->nu > NOALLOC_MAX_SIDE || g->nv > NOALLOC_MAX_SIDE || g->m > NOALLOC_MAX_M)
        fail(RECEIPT_ERR_INVALID,
             "graph exceeds the limits of receipt_count_butterflies_noalloc (at most " +
                 std::to_string(NOALLOC_MAX_SIDE) + " vertices per side and " +
                 std::to_string(NOALLOC_MAX_M) + " edges; got " + std::to_string(g->nu) + " x " +
                 std::to_string(g->nv) + " with " + std::to_string(g->m) + " edges)");
    unsigned char *base = noalloc_scratch();
    unsigned long long *cnt[2] = {(unsigned long long *)base,
                                  (unsigned long long *)(base + NA_CNT)};
    unsigned char *p = base + 2 * NA_CNT;
    int32_t *plen = (int32_t *)p;
    p += NA_PLEN;
    int32_t *lw = (int32_t *)p, *lc = (int32_t *)(p + NA_LIST), *lg = (int32_t *)(p + 2 * NA_LIST),
            *lo = (int32_t *)(p + 3 * NA_LIST);
    p += 4 * NA_LIST;
    uint32_t *gcnt = (uint32_t *)p;
    int32_t *gtouch = (int32_t *)(p + NA_GLOB);
    p += 2 * NA_GLOB;
    int32_t *ctr = (int32_t *)p;  // [8 * side + 0..7]
    // the array keeps the previous call's contents: zero what must start at 0
    RC_CUDA(cudaMemsetAsync(cnt[0], 0, 8 * (size_t)(g->nu > 0 ? g->nu : 1), s));
    RC_CUDA(cudaMemsetAsync(cnt[1], 0, 8 * (size_t)(g->nv > 0 ? g->nv : 1), s));
    RC_CUDA(cudaMemsetAsync(ctr, 0, 16 * sizeof(int32_t), s));
    RC_CUDA(cudaMemsetAsync(gcnt, 0, NA_GLOB, s));
    const int64_t m = g->m;
    const int sms = num_sms();
    if (m > 0) {
        for (int A = 0; A < 2; A++) {
            const Side &SA = g->side[A];
            const Side &SB = g->side[1 - A];
            const int32_t nA = SA.n;
            if (nA == 0) continue;
            int32_t *nl = ctr + 8 * A;  // [0] warp [1] cta [2] global [3] overflow, [4..7] work
            k_prefix_len<<<ceil_div(m, 256), 256, 0, s>>>(SA.off, SA.adj, nA, SB.off, SB.adj,
                                                          SB.below, m, plen);
            RC_LAUNCH();
            const int64_t cta_ks_max = max_cta_keyspace(nA, MID_CHUNK * 8 + CHUNK_BYTES);
            int32_t head_cap = 0, bm_cap = 0;
            size_t smem = cta_ks_max > 0 ? count_cta_smem(cta_ks_max, &head_cap, &bm_cap) : 0;
            k_count_tiers_direct<<<std::min(ceil_div((int64_t)nA * 32, 256), sms * 16), 256, 0, s>>>(
                SA.off, plen, nA, cta_ks_max, lw, lc, lg, nl);
            RC_LAUNCH();
            unsigned long long *cA = cnt[A], *cB = cnt[1 - A];
            CountArgs a{SA.off, SA.adj, SB.off, SB.adj, plen, cA, cB, lw, nl + 0, nl + 4};
            k_count_warp<<<sms * 8, 256, 0, s>>>(a);
            RC_LAUNCH();
            if (cta_ks_max > 0) {
                allow_max_smem((const void *)k_count_cta);
                CountArgs c = a;
                c.list = lc;
                c.nlist = nl + 1;
                c.work = nl + 5;
                k_count_cta<<<sms, CTA_THREADS, smem, s>>>(c, head_cap, bm_cap, lo, nl + 3);
                RC_LAUNCH();
            }
            CountArgs c = a;
            c.list = lg;
            c.nlist = nl + 2;
            c.work = nl + 6;
            const size_t gsm = MID_CHUNK * 8 + CHUNK_BYTES;
            allow_max_smem((const void *)k_count_global);
            k_count_global<<<NOALLOC_GSLOTS, CTA_THREADS, gsm, s>>>(c, lo, nl + 3, gcnt, gtouch, nA);
            RC_LAUNCH();
        }
    }
    if (d_cnt_u) scatter_to_original(cnt[0], g->side[0].new2old, g->nu, d_cnt_u, s);
    if (d_cnt_v) scatter_to_original(cnt[1], g->side[1].new2old, g->nv, d_cnt_v, s);
}

}  // namespace receipt
