// Coarse-grained decomposition, Algorithm 3 (RECEIPT CD).
//
// Per range i (1 <= i <= P):
//  1. init <- support of every remaining vertex (Algorithm 3, support init);
//  2. theta(i+1) from the weighted support histogram of the remaining
//     vertices (findHi) with the adaptive target of Sec. 3.1.1;
//  3. repeat { activeSet <- remaining vertices with support < theta(i+1);
//     peel them concurrently with the update of Algorithm 2 } until the
//     activeSet is empty.
// Vertices left after P ranges form one more subset (Sec. 3.1.1, last
// paragraph).
//
// Reading of the support update on the GPU: the raw support sup[x] is kept
// unclamped. It always equals the butterflies x shares with vertices not yet
// peeled, so it never underflows (Lemma 2: each shared butterfly is removed
// once), and "support in [theta(i), theta(i+1))" is "sup < theta(i+1)" for
// every remaining vertex; the clamp of Algorithm 2 only matters for the
// value recorded, which the fine-grained step applies.
//
// The next activeSet is built without any scan: a vertex enters it exactly
// when one 64-bit atomic subtraction takes its support from >= theta(i+1) to
// < theta(i+1), and that atomic's return value tells the thread that did it.
// A peeled vertex whose raw support is 0 shares no butterfly with any
// remaining vertex, so its update is skipped.
#include <algorithm>
#include <cstddef>
#include <vector>

#include "engine.cuh"
#include "internal.cuh"

namespace receipt {

namespace {

constexpr int NBUCKET = LOG_BUCKETS;
constexpr int NTIER = 5;  // warp, hybrid, global, sliced, dense window
constexpr double DGM_FRAC = 0.125;  // stale share of live entries that triggers a compaction

__device__ __forceinline__ int bucket_of(unsigned long long k) { return log_bucket_of(k); }
__device__ __forceinline__ unsigned long long bucket_top(int b) { return log_bucket_top(b); }

struct CdDev {
    unsigned long long hi;
    int32_t nF, nNext, nLw, nLc, nLg, nLo, nLs, nLb, nLd;
    int32_t par;      // device-driven rounds: which of two buffers holds the activeSet
    int32_t burst_k;  // device-driven rounds: rounds run by the current graph launch
    int32_t pad2;
    int32_t work[6];
    unsigned long long work64;  // item counter of the sliced tier
    unsigned long long peeled_edges;  // adjacency entries of assigned vertices (for DGM)
    int32_t n_remaining;
    int32_t range;  // 0-based index of the range being peeled
    unsigned long long wrem_prev;
    double tgt_prev;
    unsigned long long wedges;
    // per tier: wedges, mids, anchors, nonzero pairs (support atomics)
    unsigned long long tier_w[NTIER], tier_m[NTIER], tier_a[NTIER], tier_p[NTIER];
    unsigned long long front_w;  // sum of wfull over a full-scan activeSet (C_peel)
    unsigned long long hist_w[NBUCKET];
    uint32_t hist_c[NBUCKET];
};

// wfull[x] = sum over y in N_x of d_y (wedges walked when x is peeled)
__global__ void k_deg_of_nbr(const int32_t *__restrict__ adj, int64_t m,
                             const int64_t *__restrict__ offO, int64_t *__restrict__ out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < m) {
        int32_t y = adj[q];
        out[q] = offO[y + 1] - offO[y];
    }
}

__global__ void k_wfull(const int64_t *__restrict__ off, int32_t n, const int64_t *__restrict__ pscan,
                        unsigned long long *__restrict__ wfull) {
    int32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n) wfull[x] = (unsigned long long)(pscan[off[x + 1]] - pscan[off[x]]);
}

__global__ void k_init_state(int32_t *sub, int32_t n) {
    int32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n) sub[x] = -1;
}

// Histogram of remaining vertices' supports weighted by w[x] = wfull - d_x,
// and init <- sup for every remaining vertex.
__global__ void k_cd_hist(int32_t n, const int32_t *__restrict__ sub,
                          const unsigned long long *__restrict__ sup,
                          const unsigned long long *__restrict__ wfull,
                          const int64_t *__restrict__ off, unsigned long long *__restrict__ init,
                          CdDev *st) {
    __shared__ unsigned long long hw[NBUCKET];
    __shared__ uint32_t hc[NBUCKET];
    for (int b = threadIdx.x; b < NBUCKET; b += blockDim.x) {
        hw[b] = 0;
        hc[b] = 0;
    }
    __syncthreads();
    for (int32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        if (sub[x] < 0) {
            unsigned long long v = sup[x];
            init[x] = v;
            int b = bucket_of(v);
            atomicAdd(&hc[b], 1u);
            unsigned long long w = wfull[x] - (unsigned long long)(off[x + 1] - off[x]);
            if (w) atomicAdd(&hw[b], w);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < NBUCKET; b += blockDim.x) {
        if (hc[b]) {
            atomicAdd(&st->hist_c[b], hc[b]);
            if (hw[b]) atomicAdd(&st->hist_w[b], hw[b]);
        }
    }
}

// findHi with the adaptive target (one block). range = 0-based index i-1,
// P = subsets requested. With cap > 0 the bound also stops at the first
// bucket where the remaining vertices below it reach cap: a range of many
// vertices with small walks would hold few wedges but as many peeling levels
// as distinct supports, all peeled one after another by one fine-grained
// task.
__global__ void __launch_bounds__(1024) k_cd_select(CdDev *st, int range, int P, int32_t cap) {
    __shared__ unsigned long long tmpw[33];
    __shared__ uint32_t tmpc[33];
    __shared__ int s_pick, s_first, s_last;
    constexpr int PER = (NBUCKET + 1023) / 1024;
    unsigned long long w[PER];
    uint32_t c[PER];
    unsigned long long wsum = 0;
    uint32_t csum = 0;
    for (int j = 0; j < PER; j++) {
        int b = threadIdx.x * PER + j;
        w[j] = b < NBUCKET ? st->hist_w[b] : 0;
        c[j] = b < NBUCKET ? st->hist_c[b] : 0;
        wsum += w[j];
        csum += c[j];
    }
    if (threadIdx.x == 0) {
        s_pick = NBUCKET;
        s_first = NBUCKET;
        s_last = -1;
    }
    unsigned long long wtot;
    uint32_t ctot;
    unsigned long long wpre = block_exclusive_scan<unsigned long long>(wsum, tmpw, &wtot);
    uint32_t cpre = block_exclusive_scan<uint32_t>(csum, tmpc, &ctot);
    // adaptive target: tgt_i = s_{i-1} * W_rem / (P - i + 1)
    double s_prev = 1.0;
    if (range > 0) {
        unsigned long long covered = st->wrem_prev - wtot;
        if (covered > 0) s_prev = fmin(1.0, st->tgt_prev / (double)covered);
    }
    int left = P - range;
    if (left < 1) left = 1;
    double tgt = s_prev * (double)wtot / (double)left;
    unsigned long long run = wpre;
    uint32_t crun = cpre;
    for (int j = 0; j < PER; j++) {
        int b = threadIdx.x * PER + j;
        run += w[j];
        crun += c[j];
        if (c[j]) {
            atomicMin(&s_first, b);
            atomicMax(&s_last, b);
            if ((double)run >= tgt || (cap > 0 && crun >= (uint32_t)cap)) atomicMin(&s_pick, b);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st->n_remaining = (int32_t)ctot;
        if (ctot > 0) {
            int b = s_pick;
            if (tgt <= 0.0) b = s_first;
            if (b >= NBUCKET) b = s_last;
            unsigned long long top = bucket_top(b);
            st->hi = top == ~0ull ? ~0ull : top + 1ull;
        }
        st->wrem_prev = wtot;
        st->tgt_prev = tgt;
    }
}

__global__ void k_set_hi(CdDev *st, unsigned long long hi) {
    st->hi = hi;
    st->n_remaining = 1;
}

// ActiveSet by a full scan (a range's first round, and the round after a
// recount): remaining vertices with sup < hi, compacted with a warp ballot
// and one atomic per warp on *count; their wedge total (the C_peel of
// Sec. 4.1) is added to st->front_w.
// With F1 != nullptr (device-driven rounds) the round's activeSet is in
// {F, F1}[st->par], the next one goes to the other buffer, and a round with
// an empty activeSet changed nothing, so its scan is skipped.
__global__ void k_cd_frontier(int32_t n, const int32_t *__restrict__ sub,
                              const unsigned long long *__restrict__ sup,
                              const unsigned long long *__restrict__ wfull, CdDev *st,
                              int32_t *count, int32_t *__restrict__ F,
                              int32_t *__restrict__ F1 = nullptr) {
    if (F1 != nullptr) {
        if (st->nF == 0) return;
        if (st->par == 0) F = F1;
    }
    const unsigned long long hi = st->hi;
    const int lane = threadIdx.x & 31;
    unsigned long long wsum = 0;
    for (int32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        int32_t x = base + threadIdx.x;
        bool take = x < n && sub[x] < 0 && sup[x] < hi;
        if (take) wsum += wfull[x];
        unsigned bal = __ballot_sync(0xffffffffu, take);
        if (bal) {
            int pos = 0;
            if (lane == 0) pos = atomicAdd(count, __popc(bal));
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (take) F[pos + __popc(bal & lanemask_lt())] = x;
        }
    }
    wsum = warp_sum(wsum);
    if (lane == 0 && wsum) atomicAdd(&st->front_w, wsum);
}

// Assigns the activeSet to subset `range` and splits the vertices that have
// updates to make into the three engine tiers.
// With F1 != nullptr (device-driven rounds) the activeSet is {F, F1}[st->par].
__global__ void k_cd_prepare(const int32_t *__restrict__ F, CdDev *st,
                             int32_t *__restrict__ sub, const unsigned long long *__restrict__ sup,
                             const unsigned long long *__restrict__ wfull,
                             const int64_t *__restrict__ off_s, int32_t *__restrict__ Lw,
                             int32_t *__restrict__ Lb, int32_t warp_max_w,
                             const int32_t *__restrict__ F1 = nullptr) {
    if (F1 != nullptr && st->par != 0) F = F1;
    const int32_t nF = st->nF;
    const int32_t range = st->range;
    unsigned long long wsum = 0, esum = 0;
    for (int32_t base = blockIdx.x * blockDim.x; base < nF; base += gridDim.x * blockDim.x) {
        int32_t i = base + threadIdx.x;
        int32_t x = -1;
        int tier = -1;
        if (i < nF) {
            x = F[i];
            sub[x] = range;
            esum += (unsigned long long)(off_s[x + 1] - off_s[x]);
            if (sup[x] > 0) {
                unsigned long long W = wfull[x];
                wsum += W;
                tier = W <= (unsigned long long)warp_max_w ? 0 : 1;
            }
        }
        warp_append(tier == 0, x, &st->nLw, Lw);
        warp_append(tier == 1, x, &st->nLb, Lb);
    }
    wsum = warp_sum(wsum);
    esum = warp_sum(esum);
    if ((threadIdx.x & 31) == 0) {
        if (wsum) atomicAdd(&st->wedges, wsum);
        if (esum) atomicAdd(&st->peeled_edges, esum);
    }
}

// Routes the anchors with more than warp_max_w wedges (one warp each): the
// keys their wedges can reach lie in the window [kmin, kmax] spanned by the
// first and last entries of their middle vertices' lists (in a disjoint union
// that is the anchor's own graph). Window of at most DENSE_KEYS keys -> one
// dense-counter item over the window; degree >= 65535 -> global counters;
// window within the hybrid's key space and at most slice_min_w wedges ->
// hybrid; otherwise -> key slices that meet the window.
__global__ void k_cd_route(CdDev *st, const int32_t *__restrict__ Lb,
                           const int64_t *__restrict__ off_s, const int32_t *__restrict__ adj_s,
                           const int2 *__restrict__ kwin,
                           const unsigned long long *__restrict__ wfull, int64_t cta_keys,
                           int32_t slice_min_w, int32_t SW, int32_t *__restrict__ Lc,
                           int32_t *__restrict__ Lc_k, int32_t *__restrict__ Lc_w,
                           int32_t *__restrict__ Ld,
                           int32_t *__restrict__ Ld_k, int32_t *__restrict__ Ld_w,
                           int32_t *__restrict__ Lg,
                           int32_t *__restrict__ Ls, int32_t *__restrict__ Ls_lo,
                           int32_t *__restrict__ Ls_hi) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nb = st->nLb;
    for (int64_t i = warp; i < nb; i += nwarps) {
        const int32_t x = Lb[i];
        const int64_t q0 = off_s[x], q1 = off_s[x + 1];
        int32_t kmin = INT32_MAX, kmax = -1;
        // four middle vertices per lane and step, loads independent; the
        // first and last key of every list are kept in kwin
        for (int64_t qb = q0; qb < q1; qb += 128) {
            int32_t y[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int64_t q = qb + 32 * u + lane;
                y[u] = q < q1 ? adj_s[q] : -1;
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (y[u] >= 0) {
                    const int2 w = kwin[y[u]];
                    kmin = min(kmin, w.x);
                    kmax = max(kmax, w.y);
                }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        }
        if (lane == 0) {
            const int64_t ww = (int64_t)kmax - kmin + 1;
            int p;
            if (q1 - q0 >= 65535) {
                Lg[atomicAdd(&st->nLg, 1)] = x;
            } else if (ww <= DENSE_KEYS) {
                p = atomicAdd(&st->nLd, 1);
                Ld[p] = x;
                Ld_k[p] = kmin;
                Ld_w[p] = (int32_t)ww;
            } else if (ww <= cta_keys && wfull[x] <= (unsigned long long)slice_min_w) {
                p = atomicAdd(&st->nLc, 1);
                Lc[p] = x;
                Lc_k[p] = kmin;
                Lc_w[p] = (int32_t)ww;
            } else {
                p = atomicAdd(&st->nLs, 1);
                Ls[p] = x;
                Ls_lo[p] = kmin / SW;
                Ls_hi[p] = kmax / SW;
            }
        }
    }
}

// Support decrement of one (x, x') pair; `pairs` counts this thread's
// support atomics. With crossing detection (next != null) the atomic's
// returned old value tells whether this decrement took the support below hi
// (the vertex joins the next activeSet); without it the decrement needs no
// returned value and the next activeSet comes from a scan after the round.
struct CdEmit {
    unsigned long long *sup;
    const int32_t *sub;
    unsigned long long hi;
    int32_t *next;
    int32_t *n_next;
    unsigned long long pairs;
    __device__ __forceinline__ void operator()(int32_t k, uint32_t c) {
        if (sub[k] >= 0) return;
        unsigned long long d = choose2(c);
        pairs++;
        if (next) {
            unsigned long long old = atomicAdd(&sup[k], 0ull - d);
            if (old >= hi && old - d < hi) next[atomicAdd(n_next, 1)] = k;
        } else {
            atomicAdd(&sup[k], 0ull - d);
        }
    }
    // N pairs at once (k < 0: none): the `sub` loads, then the support
    // atomics, then the crossing checks, so their latencies overlap.
    template <int N>
    __device__ __forceinline__ void many(const int32_t (&k)[N], const uint32_t (&c)[N]) {
        bool live[N];
#pragma unroll
        for (int u = 0; u < N; u++) live[u] = k[u] >= 0 && sub[k[u]] < 0;
        unsigned long long old[N], d[N];
#pragma unroll
        for (int u = 0; u < N; u++) {
            d[u] = choose2(c[u]);
            old[u] = 0;
            if (live[u]) {
                pairs++;
                if (next)
                    old[u] = atomicAdd(&sup[k[u]], 0ull - d[u]);
                else
                    atomicAdd(&sup[k[u]], 0ull - d[u]);
            }
        }
        if (next) {
#pragma unroll
            for (int u = 0; u < N; u++)
                if (live[u] && old[u] >= hi && old[u] - d[u] < hi) next[atomicAdd(n_next, 1)] = k[u];
        }
    }
};

// Adds the support atomics of every thread of the calling warp to tier t's
// counter (all lanes of the warp must call it).
__device__ __forceinline__ void add_pairs(CdDev *st, int t, unsigned long long p) {
    p = warp_sum(p);
    if ((threadIdx.x & 31) == 0 && p) atomicAdd(&st->tier_p[t], p);
}

// Middle vertex y's list as it stands: the first len_o[y] entries from
// off_o[y] (dynamic graph maintenance drops peeled vertices from the lists).
struct PeelMids {
    const int32_t *adj_s;
    const int64_t *off_o;
    const int32_t *len_o;
    __device__ __forceinline__ void seg(int64_t q, int64_t &beg, int32_t &len) const {
        int32_t y = adj_s[q];
        beg = off_o[y];
        len = len_o[y];
    }
};

// Segment of a middle vertex restricted to key slice j.
// With a slice table, two loads give the bounds; without one (many slices),
// two binary searches in the sorted list do.
struct SlicedMids {
    const int32_t *adj_s;
    const int64_t *off_o;
    const int32_t *soff;   // null: search the list
    const int32_t *len_o;
    const int32_t *adj_o;
    int32_t C1;  // C + 1
    int32_t j;
    int32_t SW;
    __device__ __forceinline__ void seg(int64_t q, int64_t &beg, int32_t &len) const {
        int32_t y = adj_s[q];
        int32_t b, e;
        if (soff) {
            const int32_t *so = soff + (size_t)y * C1 + j;
            b = so[0];
            e = so[1];
        } else {
            const int32_t *L = adj_o + off_o[y];
            const int32_t l = len_o[y];
            b = (int32_t)lower_bound_i32(L, l, j * SW);
            e = b + (int32_t)lower_bound_i32(L + b, l - b, (j + 1) * SW);
        }
        beg = off_o[y] + b;
        len = e - b;
    }
};

// Keys of slice j shifted to the slice's local key space.
template <class Eng>
struct SliceVisit {
    Eng *eng;
    int32_t self_local;  // anchor's own key in this slice's frame (or -1)
    int32_t base;
    __device__ __forceinline__ void operator()(int, int32_t key) {
        int32_t k = key - base;
        if (k != self_local) eng->add(k);
    }
};

struct SliceEmit {
    CdEmit *e;
    int32_t base;
    __device__ __forceinline__ void operator()(int32_t k, uint32_t c) { (*e)(k + base, c); }
    template <int N>
    __device__ __forceinline__ void many(const int32_t (&k)[N], const uint32_t (&c)[N]) {
        int32_t kk[N];
#pragma unroll
        for (int u = 0; u < N; u++) kk[u] = k[u] >= 0 ? k[u] + base : -1;
        e->template many<N>(kk, c);
    }
};

struct PeelArgs {
    const int64_t *off_s;
    const int32_t *adj_s;
    const int64_t *off_o;
    const int32_t *len_o;  // current list lengths (dynamic graph maintenance)
    const int32_t *adj_o;  // working copy of the other side's lists
    unsigned long long *sup;
    const int32_t *sub;
    CdDev *st;
    const int32_t *Lw, *Lc, *Lg;
    int32_t *Ls;           // sliced anchors (the hybrid tier appends its overflows)
    int32_t *next;
    int32_t *Lc_k;         // hybrid anchors: first key and width of their window
    int32_t *Lc_w;
    int32_t *Ls_lo;        // sliced anchors: first and last key slice of their window
    int32_t *Ls_hi;
    const int32_t *Ld;     // dense-window anchors, their first key and window width
    const int32_t *Ld_k;
    const int32_t *Ld_w;
    const int32_t *soff;   // per other-side vertex: C + 1 slice starts within its list
    int32_t C;             // key slices
    int32_t SW;            // keys per slice
    int32_t n_keys;        // keys of the side
    int32_t scan;          // next activeSet by a scan after the round (no crossing detection)
    int32_t fetch;         // sliced tier: candidate items per work-counter atomic (1..32)
};

__global__ void __launch_bounds__(256) k_cd_update_warp(PeelArgs a) {
    __shared__ int32_t skey[8][WARP_SLOTS];
    __shared__ uint32_t sval[8][WARP_SLOTS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // blocks past the round's anchors leave at once (rounds are often empty)
    const int32_t n = a.st->nLw;
    if ((int64_t)blockIdx.x * (blockDim.x >> 5) >= n) return;
    WarpHash H{skey[w], sval[w]};
    H.clear(lane);
    __syncwarp();
    CdEmit emit{a.sup, a.sub, a.st->hi, a.scan ? nullptr : a.next, &a.st->nNext, 0};
    unsigned long long cw = 0, cm = 0, ca = 0;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(&a.st->work[0], 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= n) break;
        const int32_t x = a.Lw[idx];
        const int64_t q0 = a.off_s[x], q1 = a.off_s[x + 1];
        cm += (unsigned long long)(q1 - q0);
        ca++;
        for (int64_t qb = q0; qb < q1; qb += 32) {
            int64_t q = qb + lane;
            int64_t beg = 0;
            int32_t len = 0;
            if (q < q1) {
                int32_t y = a.adj_s[q];
                beg = a.off_o[y];
                len = a.len_o[y];
            }
            int cnt = (int)imin64(32, q1 - qb);
            for (int t = 0; t < cnt; t++) {
                int64_t b = __shfl_sync(0xffffffffu, beg, t);
                int32_t l = __shfl_sync(0xffffffffu, len, t);
                cw += (unsigned long long)l;
                for (int p = lane; p < l; p += 32) {
                    int32_t k = a.adj_o[b + p];
                    if (k != x) H.add(k);
                }
            }
        }
        __syncwarp();
        for (int i = lane; i < WARP_SLOTS; i += 32) {
            int32_t k = skey[w][i];
            if (k != EMPTY_KEY) {
                uint32_t c = sval[w][i];
                if (c >= 2) emit(k, c);
                skey[w][i] = EMPTY_KEY;
                sval[w][i] = 0;
            }
        }
        __syncwarp();
    }
    add_pairs(a.st, 0, emit.pairs);
    if (lane == 0 && ca) {
        atomicAdd(&a.st->tier_w[0], cw);
        atomicAdd(&a.st->tier_m[0], cm);
        atomicAdd(&a.st->tier_a[0], ca);
    }
}

template <class Eng>
struct PeelVisit {
    Eng *eng;
    int32_t self;
    __device__ __forceinline__ void operator()(int, int32_t key) {
        if (key != self) eng->add(key);
    }
};

__global__ void __maxnreg__(64) k_cd_update_cta(PeelArgs a, int32_t head_cap,
                                                            int32_t bm_cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_idx, s_used, s_over;
    const int32_t n = a.st->nLc;
    if ((int32_t)blockIdx.x >= n) return;
    CtaHybrid H;
    unsigned char *p = H.bind(smem, head_cap, bm_cap, &s_used, &s_over);
    Chunk ch;
    ch.beg = (int64_t *)p;
    ch.pre = (int32_t *)(ch.beg + MID_CHUNK);
    ch.tmp = ch.pre + MID_CHUNK + 1;
    ch.len = chunk_len_ptr(ch.tmp);
    H.clear_all();
    __syncthreads();
    CdEmit emit{a.sup, a.sub, a.st->hi, a.scan ? nullptr : a.next, &a.st->nNext, 0};
    PeelMids M{a.adj_s, a.off_o, a.len_o};
    unsigned long long cw = 0, cm = 0, ca = 0;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(&a.st->work[1], 1);
        __syncthreads();
        int idx = s_idx;
        if (idx >= n) break;
        const int32_t x = a.Lc[idx];
        const int32_t kb = a.Lc_k[idx];
        const int32_t kw = a.Lc_w[idx];
        H.set_range((int32_t)imin64(H.head_cap, kw), kw);
        SliceVisit<CtaHybrid> v{&H, x - kb, kb};
        cw += cta_walk<false>(M, a.off_s[x], a.off_s[x + 1], a.adj_o, ch, v);
        cm += (unsigned long long)(a.off_s[x + 1] - a.off_s[x]);
        ca++;
        SliceEmit em{&emit, kb};
        if (!s_over) {
            H.flush_clear<true>(em);
        } else {
            H.flush_clear<false>(em);
            if (threadIdx.x == 0) {
                // redo through the key slices that meet the window
                const int p = atomicAdd(&a.st->nLs, 1);
                a.Ls[p] = x;
                a.Ls_lo[p] = kb / a.SW;
                a.Ls_hi[p] = (kb + kw - 1) / a.SW;
            }
        }
        __syncthreads();
        H.reset_scalars();
    }
    add_pairs(a.st, 1, emit.pairs);
    if (threadIdx.x == 0 && ca) {
        atomicAdd(&a.st->tier_w[1], cw);
        atomicAdd(&a.st->tier_m[1], cm);
        atomicAdd(&a.st->tier_a[1], ca);
    }
}

__global__ void __maxnreg__(64) k_cd_update_global(PeelArgs a, uint32_t *gcnt,
                                                               int32_t *gtouch, int64_t keyspace) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_idx, s_nt;
    Chunk ch;
    ch.beg = (int64_t *)smem;
    ch.pre = (int32_t *)(ch.beg + MID_CHUNK);
    ch.tmp = ch.pre + MID_CHUNK + 1;
    ch.len = chunk_len_ptr(ch.tmp);
    GlobalDense G{gcnt + (size_t)blockIdx.x * keyspace, gtouch + (size_t)blockIdx.x * keyspace, &s_nt};
    const int32_t n1 = a.st->nLg, n2 = 0;
    if ((int32_t)blockIdx.x >= n1 + n2) return;
    CdEmit emit{a.sup, a.sub, a.st->hi, a.scan ? nullptr : a.next, &a.st->nNext, 0};
    PeelMids M{a.adj_s, a.off_o, a.len_o};
    unsigned long long cw = 0, cm = 0, ca = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            s_idx = atomicAdd(&a.st->work[2], 1);
            s_nt = 0;
        }
        __syncthreads();
        int idx = s_idx;
        if (idx >= n1 + n2) break;
        const int32_t x = a.Lg[idx];
        PeelVisit<GlobalDense> v{&G, x};
        cw += cta_walk(M, a.off_s[x], a.off_s[x + 1], a.adj_o, ch, v);
        cm += (unsigned long long)(a.off_s[x + 1] - a.off_s[x]);
        ca++;
        G.flush(emit);
        __syncthreads();
        G.clear();
        __syncthreads();
    }
    add_pairs(a.st, 2, emit.pairs);
    if (threadIdx.x == 0 && ca) {
        atomicAdd(&a.st->tier_w[2], cw);
        atomicAdd(&a.st->tier_m[2], cm);
        atomicAdd(&a.st->tier_a[2], ca);
    }
}

// Anchors with many wedges: the key space is cut into C slices of SW keys and
// every (anchor, slice) pair is one work item, so the slices of a heavy
// anchor run on different CTAs. Each item aggregates its slice with dense
// 16-bit counters in shared memory, listing the keys whose count reaches 2
// (most keys of a wide slice are touched once and emit nothing). Three
// shapes: one 1,024-thread CTA per SM with 98,304-key slices, or two
// 512-thread (49,152 keys) or four 256-thread (22,016 keys) CTAs per SM,
// whose items' barrier-separated phases (staging, walk, sweep) overlap on the
// SM. Each shape's counters, key list and staging fill the SM's shared
// memory.
template <int THREADS, int WORDS>
struct SliceShape {
    static constexpr int threads = THREADS;
    static constexpr int keys = 2 * WORDS;
    using Engine = DenseSliceT<WORDS, TOUCH_PAIRS>;
    static constexpr size_t smem() { return Engine::bytes() + chunk_bytes(THREADS); }
};
using Slice1 = SliceShape<SLICE_THREADS, 49152>;
using Slice2 = SliceShape<512, 24576>;
using Slice4 = SliceShape<256, 11008>;

constexpr int SLICE_FETCH_MAX = 32;  // candidate items per work-counter atomic, at most

template <class Shape>
__global__ void __launch_bounds__(Shape::threads, 1024 / Shape::threads)
    k_cd_update_slice(PeelArgs a, int32_t n) {
    using Engine = typename Shape::Engine;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_items[SLICE_FETCH_MAX];
    __shared__ int s_nitems, s_pos, s_nt;
    if (a.st->nLs == 0) return;
    Engine H;
    unsigned char *p = H.bind(smem, &s_nt);
    Chunk ch;
    ch.beg = (int64_t *)p;
    ch.pre = (int32_t *)(ch.beg + Shape::threads);
    ch.tmp = ch.pre + Shape::threads + 1;
    ch.len = chunk_len_ptr(ch.tmp);
    H.clear_all();
    if (threadIdx.x == 0) s_nitems = s_pos = 0;
    __syncthreads();
    CdEmit emit{a.sup, a.sub, a.st->hi, a.scan ? nullptr : a.next, &a.st->nNext, 0};
    unsigned long long cw = 0, cm = 0, ca = 0;
    const int64_t items = (int64_t)a.st->nLs * a.C;
    const int lane = threadIdx.x & 31;
    for (;;) {
        // warp 0 refills the CTA's batch of (anchor, slice) items whose slice
        // meets the anchor's window: a.fetch consecutive item numbers per
        // atomic, checked by as many lanes at once. Items are numbered anchor
        // by anchor (item = anchor * C + j): consecutive slices of one anchor
        // share its middle vertices' table rows and list positions.
        if (threadIdx.x < 32) {
            __syncwarp();
            if (s_pos >= s_nitems) {
                const int fetch = a.fetch;
                int nvalid = 0;
                bool done = false;
                while (nvalid == 0 && !done) {
                    unsigned long long b = 0;
                    if (lane == 0)
                        b = atomicAdd((unsigned long long *)&a.st->work64, (unsigned long long)fetch);
                    b = __shfl_sync(0xffffffffu, b, 0);
                    const int64_t it = (int64_t)b + lane;
                    bool ok = false;
                    if (lane < fetch && it < items) {
                        const int64_t ai = it / a.C;
                        const int32_t jj = (int32_t)(it % a.C);
                        ok = jj >= a.Ls_lo[ai] && jj <= a.Ls_hi[ai];
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, ok);
                    if (ok) s_items[__popc(bal & lanemask_lt())] = it;
                    nvalid = __popc(bal);
                    done = (int64_t)b + fetch >= items;
                }
                __syncwarp();
                if (lane == 0) {
                    s_nitems = nvalid;
                    s_pos = 0;
                }
            }
        }
        __syncthreads();
        if (s_pos >= s_nitems) break;  // no item left
        const int64_t idx = s_items[s_pos];
        __syncthreads();
        if (threadIdx.x == 0) s_pos++;
        const int64_t ai = idx / a.C;
        const int32_t x = a.Ls[ai];
        const int32_t j = (int32_t)(idx % a.C);
        const int64_t q0 = a.off_s[x], q1 = a.off_s[x + 1];
        if (j == a.Ls_lo[ai]) {
            cm += (unsigned long long)(q1 - q0);
            ca++;
        }
        const int32_t base = j * a.SW;
        const int32_t w = (int32_t)imin64(a.SW, (int64_t)n - base);
        H.set_width(w);
        SlicedMids M{a.adj_s, a.off_o, a.soff, a.len_o, a.adj_o, a.C + 1, j, a.SW};
        const int32_t self = (x >= base && x < base + w) ? x - base : -1;
        SliceVisit<Engine> v{&H, self, base};
        int64_t walked = cta_walk(M, q0, q1, a.adj_o, ch, v);
        cw += walked;
        if (walked == 0) continue;
        SliceEmit em{&emit, base};
        H.template sweep<true, true>(em);
        __syncthreads();
        H.reset_scalars();
    }
    add_pairs(a.st, 3, emit.pairs);
    if (threadIdx.x == 0) {
        if (cw) atomicAdd(&a.st->tier_w[3], cw);
        if (ca) {
            atomicAdd(&a.st->tier_m[3], cm);
            atomicAdd(&a.st->tier_a[3], ca);
        }
    }
}

// Anchors whose keys fit one window of at most DENSE_KEYS keys: dense 16-bit
// counters over the window, exact (no overflow path). A CTA takes DENSE_GROUP
// anchors at a time and aggregates as many of them per pass as their windows
// fit side by side in the counters (anchor a's window at offset off[a]); the
// pass's edges form one virtual list of middle vertices, and the thread that
// stages a middle vertex records its anchor for the visits.
constexpr int DENSE_GROUP = 8;

struct DenseBatchMids {
    const int32_t *adj_s;
    const int64_t *off_o;
    const int32_t *len_o;
    const int64_t *q0;    // first edge of each anchor (shared)
    const int32_t *pre;   // prefix of the anchors' degrees (shared)
    int nb;
    uint8_t *slot;
    __device__ __forceinline__ void seg(int64_t q, int64_t &beg, int32_t &len) const {
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= q)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int32_t y = adj_s[q0[lo] + (q - pre[lo])];
        beg = off_o[y];
        len = len_o[y];
        slot[threadIdx.x] = (uint8_t)lo;
    }
};

struct DenseBatchVisit {
    DenseSlice *eng;
    const uint8_t *slot;
    const int32_t *x;    // anchors (shared)
    const int32_t *kb;   // first key of each window (shared)
    const int32_t *off;  // offset of each window in the counters (shared)
    __device__ __forceinline__ void operator()(int k, int32_t key) {
        const int a = slot[k];
        if (key != x[a]) eng->add(off[a] + key - kb[a]);
    }
};

struct DenseBatchEmit {
    CdEmit *e;
    const int32_t *kb;
    const int32_t *off;
    int nb;
    __device__ __forceinline__ void operator()(int32_t w, uint32_t c) {
        int a = 0;
        while (a + 1 < nb && off[a + 1] <= w) a++;
        (*e)(kb[a] + w - off[a], c);
    }
};

__global__ void __maxnreg__(64) k_cd_update_dense(PeelArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_idx, s_nt, s_nb;
    __shared__ int64_t s_q0[DENSE_GROUP];
    __shared__ int32_t s_x[DENSE_GROUP], s_kb[DENSE_GROUP], s_off[DENSE_GROUP + 1],
        s_pre[DENSE_GROUP + 1];
    __shared__ uint8_t s_slot[DENSE_THREADS];
    const int32_t n = a.st->nLd;
    // anchors per fetch: more than one only when the round has more anchors
    // than CTAs
    const int G = max(1, min(DENSE_GROUP, n / (int)gridDim.x));
    if ((int32_t)blockIdx.x * G >= n) return;
    DenseSlice H;
    unsigned char *p = H.bind(smem, &s_nt);
    Chunk ch;
    ch.beg = (int64_t *)p;
    ch.pre = (int32_t *)(ch.beg + MID_CHUNK);
    ch.tmp = ch.pre + MID_CHUNK + 1;
    ch.len = chunk_len_ptr(ch.tmp);
    H.clear_all();
    __syncthreads();
    CdEmit emit{a.sup, a.sub, a.st->hi, a.scan ? nullptr : a.next, &a.st->nNext, 0};
    const int lane = threadIdx.x & 31;
    unsigned long long cw = 0, cm = 0, ca = 0;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(&a.st->work[4], G);
        __syncthreads();
        const int base = s_idx;
        if (base >= n) break;
        const int gcount = min(G, n - base);
        for (int i0 = 0; i0 < gcount;) {
            if (threadIdx.x < 32) {
                // the leading anchors whose windows fit side by side
                const int i = i0 + lane;
                int32_t w = 0, deg = 0, x = 0, kb = 0;
                int64_t q0 = 0;
                if (i < gcount) {
                    x = a.Ld[base + i];
                    kb = a.Ld_k[base + i];
                    w = a.Ld_w[base + i];
                    q0 = a.off_s[x];
                    deg = (int32_t)(a.off_s[x + 1] - q0);
                }
                int32_t wi = w, di = deg;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t yw = __shfl_up_sync(0xffffffffu, wi, o);
                    const int32_t yd = __shfl_up_sync(0xffffffffu, di, o);
                    if (lane >= o) {
                        wi += yw;
                        di += yd;
                    }
                }
                const bool fits = i < gcount && (lane == 0 || wi <= DENSE_KEYS);
                const int nb = __popc(__ballot_sync(0xffffffffu, fits));
                if (lane < nb) {
                    s_x[lane] = x;
                    s_kb[lane] = kb;
                    s_q0[lane] = q0;
                    s_off[lane + 1] = wi;
                    s_pre[lane + 1] = di;
                }
                if (lane == 0) {
                    s_off[0] = 0;
                    s_pre[0] = 0;
                    s_nb = nb;
                }
            }
            __syncthreads();
            const int nb = s_nb;
            H.set_width(s_off[nb]);
            DenseBatchMids M{a.adj_s, a.off_o, a.len_o, s_q0, s_pre, nb, s_slot};
            DenseBatchVisit v{&H, s_slot, s_x, s_kb, s_off};
            cw += cta_walk(M, 0, s_pre[nb], a.adj_o, ch, v);
            cm += (unsigned long long)s_pre[nb];
            ca += nb;
            DenseBatchEmit em{&emit, s_kb, s_off, nb};
            H.sweep<true, true>(em);
            __syncthreads();
            H.reset_scalars();
            i0 += nb;
            __syncthreads();
        }
    }
    add_pairs(a.st, 4, emit.pairs);
    if (threadIdx.x == 0 && ca) {
        atomicAdd(&a.st->tier_w[4], cw);
        atomicAdd(&a.st->tier_m[4], cm);
        atomicAdd(&a.st->tier_a[4], ca);
    }
}

// Dynamic graph maintenance (Sec. 4.2): drops the vertices already assigned
// to a subset from every list of the working copy, keeping each list sorted
// (one warp per list, ballot compaction in place; the write position never
// passes the read position).
__global__ void k_dgm_compact(const int64_t *__restrict__ off_o, int32_t *__restrict__ len_o,
                              int32_t *__restrict__ adj_w, int32_t n_o,
                              const int32_t *__restrict__ sub) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t y = warp; y < n_o; y += nwarps) {
        const int64_t b = off_o[y];
        const int32_t l = len_o[y];
        int32_t w = 0;
        // 128 entries per step: all loads first, then the ordered writes
        for (int32_t r0 = 0; r0 < l; r0 += 128) {
            int32_t x[4];
            bool keep[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int32_t r = r0 + 32 * u + lane;
                x[u] = r < l ? adj_w[b + r] : -1;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) keep[u] = x[u] >= 0 && sub[x[u]] < 0;
            __syncwarp();
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const unsigned bal = __ballot_sync(0xffffffffu, keep[u]);
                if (keep[u]) adj_w[b + w + __popc(bal & lanemask_lt())] = x[u];
                w += __popc(bal);
            }
            __syncwarp();
        }
        if (lane == 0) len_o[y] = w;
    }
}

__global__ void k_list_lengths(const int64_t *__restrict__ off, int32_t n, int32_t *__restrict__ len) {
    int32_t y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y < n) len[y] = (int32_t)(off[y + 1] - off[y]);
}

// kwin[y] = (first, last) key of the working list y ((INT32_MAX, -1) when
// empty): the window the route of an anchor takes over its middle vertices.
__global__ void k_list_window(const int64_t *__restrict__ off, const int32_t *__restrict__ len,
                              const int32_t *__restrict__ adj, int32_t n, int2 *__restrict__ kwin) {
    int32_t y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= n) return;
    const int32_t l = len[y];
    kwin[y] = l > 0 ? make_int2(adj[off[y]], adj[off[y] + l - 1]) : make_int2(INT32_MAX, -1);
}

// soff[y * (C + 1) + j] = number of entries of N_y below j * SW (j = 0..C).
__global__ void k_slice_table(const int64_t *__restrict__ off_o, const int32_t *__restrict__ len_o,
                              const int32_t *__restrict__ adj_o, int32_t n_o, int32_t C, int32_t SW,
                              int32_t *__restrict__ soff) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t tot = (int64_t)n_o * (C + 1);
    if (i >= tot) return;
    int32_t y = (int32_t)(i / (C + 1)), j = (int32_t)(i % (C + 1));
    int64_t b = off_o[y], e = b + len_o[y];
    soff[i] = j == C ? (int32_t)(e - b) : (int32_t)lower_bound_i32(adj_o + b, e - b, j * SW);
}

// Next round: the vertices that crossed below hi become the activeSet.
__global__ void k_cd_advance(CdDev *st) {
    st->nF = st->nNext;
    st->nNext = 0;
    st->nLw = st->nLc = st->nLg = st->nLo = st->nLs = st->nLb = st->nLd = 0;
    for (int i = 0; i < 6; i++) st->work[i] = 0;
    st->work64 = 0;
}

// Device-driven rounds: the end of a round. The round's header (everything
// before the histogram, as the host loop copies it) goes to record
// st->burst_k, the activeSet advances (the next one is in the other buffer),
// and the graph's while-condition stays set while there is a next activeSet
// and fewer than `burst` rounds ran in this launch.
__global__ void k_cd_round_end(CdDev *st, unsigned long long *__restrict__ rec, int32_t words,
                               int32_t burst, cudaGraphConditionalHandle cond) {
    const int32_t k = st->burst_k;
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(st);
    for (int i = threadIdx.x; i < words; i += blockDim.x) rec[(size_t)k * words + i] = src[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int32_t nn = st->nNext;
        if (nn > 0) st->par ^= 1;
        st->nF = nn;
        st->nNext = 0;
        st->nLw = st->nLc = st->nLg = st->nLo = st->nLs = st->nLb = st->nLd = 0;
        for (int i = 0; i < 6; i++) st->work[i] = 0;
        st->work64 = 0;
        st->burst_k = k + 1;
        cudaGraphSetConditional(cond, (nn > 0 && k + 1 < burst) ? 1u : 0u);
    }
}

__global__ void k_cd_burst_begin(CdDev *st, int32_t par) {
    st->par = par;
    st->burst_k = 0;
}

__global__ void k_cd_new_range(CdDev *st, int32_t range) {
    if (threadIdx.x == 0) {
        st->range = range;
        st->front_w = 0;
        st->nF = st->nNext = 0;
        st->nLw = st->nLc = st->nLg = st->nLo = st->nLs = st->nLb = st->nLd = 0;
        for (int i = 0; i < 6; i++) st->work[i] = 0;
        st->work64 = 0;
    }
    for (int b = threadIdx.x; b < NBUCKET; b += blockDim.x) {
        st->hist_w[b] = 0;
        st->hist_c[b] = 0;
    }
}

// Vertices left after the last range form one more subset; their init is
// their current support.
__global__ void k_cd_leftover(int32_t n, int32_t *__restrict__ sub,
                              const unsigned long long *__restrict__ sup,
                              unsigned long long *__restrict__ init, int32_t range, int *any) {
    for (int32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        if (sub[x] < 0) {
            init[x] = sup[x];
            sub[x] = range;
            *any = 1;
        }
    }
}

}  // namespace

int64_t max_cta_keyspace(int64_t want, size_t extra) {
    const size_t cap = (size_t)max_smem_optin();
    if (hybrid_bytes(want, nullptr, nullptr) + extra <= cap) return want;
    int64_t lo = 0, hi = want;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (hybrid_bytes(mid, nullptr, nullptr) + extra <= cap)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

void cd_run(Decomp &D, const receipt_options &opt, cudaStream_t s) {
    const int32_t n = D.n;
    const int sms = num_sms();
    const Side &S = *D.S;
    const Side &O = *D.O;
    const int P = opt.P > 0 ? opt.P : 150;
    D.bounds.clear();
    D.bounds.push_back(0);
    if (n == 0) {
        D.p_eff = 0;
        return;
    }
    DevBuf<CdDev> st(1, s);
    st.zero();
    DevBuf<int32_t> F(n, s), Nx(n, s), Lw(n, s), Lc(n, s), Lg(n, s), Ls(n, s), Lb(n, s), Ld(n, s);
    DevBuf<int32_t> Lc_k(n, s), Lc_w(n, s), Ld_k(n, s), Ld_w(n, s), Ls_lo(n, s), Ls_hi(n, s);
    const int32_t warp_max_w =
        opt.warp_max_w > 0 ? std::min(opt.warp_max_w, WARP_MAX_W) : WARP_MAX_W;
    const int32_t slice_min_w = opt.slice_min_w > 0 ? opt.slice_min_w : SLICE_MIN_W;
    // key slices for anchors with many wedges; the sliced tier's shape
    const int slice_ctas = opt.slice_ctas == 1 || opt.slice_ctas == 2 ? opt.slice_ctas : 4;
    const void *slice_fn = slice_ctas == 4   ? (const void *)k_cd_update_slice<Slice4>
                           : slice_ctas == 2 ? (const void *)k_cd_update_slice<Slice2>
                                             : (const void *)k_cd_update_slice<Slice1>;
    const int slice_threads = slice_ctas == 4 ? Slice4::threads
                              : slice_ctas == 2 ? Slice2::threads : Slice1::threads;
    const size_t smem_slice = slice_ctas == 4   ? Slice4::smem()
                              : slice_ctas == 2 ? Slice2::smem() : Slice1::smem();
    const int32_t SW = slice_ctas == 4 ? Slice4::keys : slice_ctas == 2 ? Slice2::keys : Slice1::keys;
    const bool scan_next = opt.scan_frontier >= 0;
    const int32_t slice_fetch = opt.slice_fetch > 0 ? std::min(opt.slice_fetch, SLICE_FETCH_MAX) : 1;
    // vertices per range: at most range_max_n (0: 2 n / P, -1: no bound)
    const int32_t range_cap =
        opt.range_max_n < 0 ? 0
                            : (opt.range_max_n > 0 ? opt.range_max_n
                                                   : (int32_t)std::max<int64_t>(1, 2 * (int64_t)n / P));
    const int32_t C = std::max(1, ceil_div(n, SW));
    // slice table (C + 1 starts per list) only while slices are few
    const bool table = C <= 64;
    DevBuf<int32_t> soff(table ? (size_t)O.n * (C + 1) : 1, s);
    // working copy of the other side's lists, compacted between ranges
    DevBuf<int32_t> adj_w(D.m, s), len_w(O.n, s);
    DevBuf<int2> kwin(O.n, s);
    if (D.m > 0)
        RC_CUDA(cudaMemcpyAsync(adj_w.get(), O.adj, sizeof(int32_t) * D.m, cudaMemcpyDeviceToDevice, s));
    const bool dgm = !opt.no_dgm;
    const double dgm_frac = opt.dgm_frac_1024 > 0 ? opt.dgm_frac_1024 / 1024.0 : DGM_FRAC;
    uint64_t peeled_at_dgm = 0;
    // hybrid update computation: C_rcnt once per call when the rule is on
    const int huc = opt.huc;
    const double huc_factor = D.huc_factor;
    DevBuf<unsigned long long> rcost(1, s);
    if (huc == 0)
        launch_recount_cost(S, O, D.m, rcost.get(), s);
    else
        rcost.zero();
    if (O.n > 0) {
        k_list_lengths<<<ceil_div(O.n, 256), 256, 0, s>>>(O.off, O.n, len_w.get());
        RC_LAUNCH();
        k_list_window<<<ceil_div(O.n, 256), 256, 0, s>>>(O.off, len_w.get(), adj_w.get(), O.n,
                                                        kwin.get());
        RC_LAUNCH();
        if (table) {
            k_slice_table<<<ceil_div((int64_t)O.n * (C + 1), 256), 256, 0, s>>>(
                O.off, len_w.get(), adj_w.get(), O.n, C, SW, soff.get());
            RC_LAUNCH();
        }
    }
    allow_max_smem(slice_fn);
    int occ_s = 1;
    RC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, slice_fn, slice_threads,
                                                          smem_slice));
    const int sblocks = sms * std::max(1, occ_s);
    // tiers available for peel anchors (key space = whole side)
    const size_t chunk_extra = CHUNK_BYTES;
    int32_t head_cap = 0, bm_cap = 0;
    // the hybrid engine covers windows of up to cta_keys keys
    const int64_t cta_keys = max_cta_keyspace(n, chunk_extra);
    const bool cta_ok = cta_keys > DENSE_KEYS;
    size_t smem_cta = cta_ok ? hybrid_bytes(cta_keys, &head_cap, &bm_cap) + chunk_extra : 0;
    if (cta_ok) allow_max_smem((const void *)k_cd_update_cta);
    allow_max_smem((const void *)k_cd_update_dense);
    int occ_d = 1;
    RC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_d, k_cd_update_dense, DENSE_THREADS,
                                                          DenseSlice::bytes() + CHUNK_BYTES));
    const int dblocks = sms * std::max(1, occ_d);
    // global-counter slots only exist if the side has a hub whose counts can
    // exceed 16 bits (degree >= 65535)
    const bool hubs = D.max_deg_s >= 65535;
    const int gblocks = hubs ? std::max(1, sms / 2) : 1;
    DevBuf<uint32_t> gcnt((size_t)gblocks * (hubs ? n : 1), s);
    DevBuf<int32_t> gtouch((size_t)gblocks * (hubs ? n : 1), s);
    gcnt.zero();
    const size_t smem_glob = chunk_extra;
    allow_max_smem((const void *)k_cd_update_global);
    const size_t hdr = offsetof(CdDev, hist_w);
    // pinned: C_rcnt, the state's header, the device-driven rounds' records
    constexpr int ROUND_BURST = 64;
    unsigned long long *hpin =
        (unsigned long long *)pinned_scratch(64 + sizeof(CdDev) + ROUND_BURST * hdr);
    CdDev *hst = reinterpret_cast<CdDev *>(hpin + 8);
    unsigned long long *hrec = hpin + 8 + (sizeof(CdDev) + 7) / 8;
    unsigned long long prev_w[NTIER] = {}, prev_a[NTIER] = {};

    // fork/join of the tier streams (no timing)
    cudaEvent_t fork_ev[1 + NUM_TIER_STREAMS] = {};
    struct ForkGuard {
        cudaEvent_t *e;
        ~ForkGuard() {
            for (int i = 0; i < 1 + NUM_TIER_STREAMS; i++)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } fg{fork_ev};
    for (int i = 0; i < 1 + NUM_TIER_STREAMS; i++)
        RC_CUDA(cudaEventCreateWithFlags(&fork_ev[i], cudaEventDisableTiming));
    // ev[0..NTIER]: peel tiers; ev[NTIER + 1..NTIER + 2]: a recount
    cudaEvent_t ev[NTIER + 3] = {};
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int i = 0; i < NTIER + 3; i++)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } eg{ev};
    if (D.timing)
        for (int i = 0; i < NTIER + 3; i++) RC_CUDA(cudaEventCreate(&ev[i]));
    k_init_state<<<ceil_div(n, 256), 256, 0, s>>>(D.sub, n);
    RC_LAUNCH();
    const int nb = std::min(ceil_div(n, 512), sms * 4);
    int range = 0;
    const int nranges = opt.n_bounds > 0 ? std::min(opt.n_bounds, P) : P;
    // activeSet buffers of the two round parities; the range index comes
    // from device memory, so a round's launches do not depend on the range
    int32_t *abuf[2] = {F.get(), Nx.get()};
    cudaGraph_t round_graph[2] = {};
    cudaGraphExec_t round_exec[2] = {};
    struct GraphGuard {
        cudaGraph_t *g;
        cudaGraphExec_t *e;
        ~GraphGuard() {
            for (int k = 0; k < 2; k++) {
                if (e[k]) cudaGraphExecDestroy(e[k]);
                if (g[k]) cudaGraphDestroy(g[k]);
            }
        }
    } gg{round_graph, round_exec};
    uint64_t round_kernels = 0;
    // Device-driven rounds: one graph whose while-node repeats the round
    // body until a round leaves no next activeSet or ROUND_BURST rounds ran;
    // the rounds' headers go to device records that the host reads after the
    // launch, so a range's rounds need no host round trip between them.
    const bool dloop = opt.round_graphs == 0 && scan_next && !D.timing;
    const int32_t hdr_words = (int32_t)(offsetof(CdDev, hist_w) / 8);
    DevBuf<unsigned long long> rec(dloop ? (size_t)ROUND_BURST * hdr_words : 1, s);
    cudaGraphConditionalHandle loop_cond = 0;
    // The round body on stream `q`: split the activeSet `cur` into tiers,
    // route, apply the updates of every tier (their crossings form the next
    // activeSet in `nxt`), copy the round's header to the host, advance.
    // With `loop` the activeSet buffer is chosen on the device ({cur,
    // nxt}[st->par]) and the header goes to the device records instead.
    auto round_body = [&](cudaStream_t q, int32_t *cur, int32_t *nxt, bool external_events,
                          bool loop) {
        auto mark = [&](int i) {
            if (!D.timing) return;
            if (external_events)
                RC_CUDA(cudaEventRecordWithFlags(ev[i], q, cudaEventRecordExternal));
            else
                RC_CUDA(cudaEventRecord(ev[i], q));
        };
        k_cd_prepare<<<nb, 512, 0, q>>>(cur, st.get(), D.sub, D.sup, D.wfull, S.off, Lw.get(),
                                        Lb.get(), warp_max_w, loop ? nxt : nullptr);
        RC_LAUNCH();
        k_cd_route<<<sms * 8, 256, 0, q>>>(st.get(), Lb.get(), S.off, S.adj, kwin.get(),
                                           D.wfull, cta_ok ? cta_keys : 0, slice_min_w,
                                           SW, Lc.get(), Lc_k.get(), Lc_w.get(), Ld.get(),
                                           Ld_k.get(), Ld_w.get(), Lg.get(), Ls.get(), Ls_lo.get(),
                                           Ls_hi.get());
        RC_LAUNCH();
        PeelArgs a{S.off,     S.adj,      O.off,       len_w.get(), adj_w.get(), D.sup, D.sub,
                   st.get(),  Lw.get(),   Lc.get(),    Lg.get(),    Ls.get(), nxt,
                   Lc_k.get(), Lc_w.get(), Ls_lo.get(), Ls_hi.get(), Ld.get(), Ld_k.get(),
                   Ld_w.get(), table ? soff.get() : nullptr, C, SW, n, scan_next ? 1 : 0,
                   slice_fetch};
        // The tiers' anchors are disjoint and their support decrements are
        // atomic, so without per-tier timing the warp, dense-window and
        // global tiers run on their own streams beside the hybrid and sliced
        // tiers (the sliced tier takes the hybrid's overflows: same stream),
        // and the tiers a round leaves empty cost no serial launch gaps.
        const bool fork = !D.timing;
        cudaStream_t qs[NUM_TIER_STREAMS] = {q, q, q};
        if (fork) {
            RC_CUDA(cudaEventRecord(fork_ev[0], q));
            for (int k = 0; k < NUM_TIER_STREAMS; k++) {
                qs[k] = tier_stream(k);
                RC_CUDA(cudaStreamWaitEvent(qs[k], fork_ev[0], 0));
            }
        }
        mark(0);
        k_cd_update_warp<<<sms * 8, 256, 0, qs[0]>>>(a);
        RC_LAUNCH();
        mark(1);
        k_cd_update_dense<<<dblocks, DENSE_THREADS, DenseSlice::bytes() + CHUNK_BYTES, qs[1]>>>(a);
        RC_LAUNCH();
        mark(2);
        if (cta_ok) {
            k_cd_update_cta<<<sms, CTA_THREADS, smem_cta, q>>>(a, head_cap, bm_cap);
            RC_LAUNCH();
        }
        mark(3);
        if (hubs) {
            k_cd_update_global<<<gblocks, CTA_THREADS, smem_glob, qs[2]>>>(a, gcnt.get(),
                                                                          gtouch.get(), n);
            RC_LAUNCH();
        }
        mark(4);
        {
            void *args[] = {&a, (void *)&n};
            RC_CUDA(cudaLaunchKernel(slice_fn, dim3(sblocks), dim3(slice_threads), args, smem_slice,
                                     q));
            RC_LAUNCH();
        }
        mark(5);
        if (fork)
            for (int k = 0; k < NUM_TIER_STREAMS; k++) {
                RC_CUDA(cudaEventRecord(fork_ev[1 + k], qs[k]));
                RC_CUDA(cudaStreamWaitEvent(q, fork_ev[1 + k], 0));
            }
        if (scan_next) {
            // next activeSet: remaining vertices whose support is now below hi
            if (loop)
                k_cd_frontier<<<nb, 512, 0, q>>>(n, D.sub, D.sup, D.wfull, st.get(),
                                                 &st.get()->nNext, cur, nxt);
            else
                k_cd_frontier<<<nb, 512, 0, q>>>(n, D.sub, D.sup, D.wfull, st.get(),
                                                 &st.get()->nNext, nxt);
            RC_LAUNCH();
        }
        if (loop) {
            k_cd_round_end<<<1, 64, 0, q>>>(st.get(), rec.get(), hdr_words, ROUND_BURST,
                                            loop_cond);
            RC_LAUNCH();
            return;
        }
        RC_CUDA(cudaMemcpyAsync(hst, st.get(), hdr, cudaMemcpyDeviceToHost, q));
        k_cd_advance<<<1, 1, 0, q>>>(st.get());
        RC_LAUNCH();
    };
    // A round whose updates are a recount (Sec. 4.1): assign the activeSet
    // `cur`, drop every assigned vertex from the other side's lists (the
    // working copy itself with DGM on, else a copy of it), recount the
    // remaining subgraph into sup and take the next activeSet `nxt` by a
    // full scan.
    DevBuf<int32_t> tadj, tlen;
    auto huc_round = [&](int32_t *cur, int32_t *nxt) {
        k_cd_prepare<<<nb, 512, 0, s>>>(cur, st.get(), D.sub, D.sup, D.wfull, S.off, Lw.get(),
                                        Lb.get(), warp_max_w);
        RC_LAUNCH();
        int32_t *la = adj_w.get(), *ll = len_w.get();
        if (!dgm) {
            if (!tadj.get()) {
                tadj.alloc(D.m, s);
                tlen.alloc(O.n, s);
            }
            RC_CUDA(cudaMemcpyAsync(tadj.get(), adj_w.get(), sizeof(int32_t) * D.m,
                                    cudaMemcpyDeviceToDevice, s));
            RC_CUDA(cudaMemcpyAsync(tlen.get(), len_w.get(), sizeof(int32_t) * O.n,
                                    cudaMemcpyDeviceToDevice, s));
            la = tadj.get();
            ll = tlen.get();
        }
        if (O.n > 0) {
            k_dgm_compact<<<std::min(ceil_div((int64_t)O.n * 32, 256), sms * 32), 256, 0, s>>>(
                O.off, ll, la, O.n, D.sub);
            RC_LAUNCH();
            if (dgm) {
                k_list_window<<<ceil_div(O.n, 256), 256, 0, s>>>(O.off, len_w.get(), adj_w.get(),
                                                                O.n, kwin.get());
                RC_LAUNCH();
            }
            if (dgm && table) {
                k_slice_table<<<ceil_div((int64_t)O.n * (C + 1), 256), 256, 0, s>>>(
                    O.off, len_w.get(), adj_w.get(), O.n, C, SW, soff.get());
                RC_LAUNCH();
            }
        }
        if (D.timing) RC_CUDA(cudaEventRecord(ev[NTIER + 1], s));
        D.wedges_recount += recount_remaining(D, ll, la, s);
        if (D.timing) RC_CUDA(cudaEventRecord(ev[NTIER + 2], s));
        k_cd_frontier<<<nb, 512, 0, s>>>(n, D.sub, D.sup, D.wfull, st.get(), &st.get()->nNext,
                                         nxt);
        RC_LAUNCH();
        RC_CUDA(cudaMemcpyAsync(hst, st.get(), hdr, cudaMemcpyDeviceToHost, s));
        k_cd_advance<<<1, 1, 0, s>>>(st.get());
        RC_LAUNCH();
        D.huc_recounts++;
        if (dgm) D.dgm_passes++;
    };
    // With round_graphs the body is captured once per activeSet parity (on a
    // private stream: the caller's may be the legacy default stream, which
    // cannot capture) and each round is one graph launch.
    const bool graphs = opt.round_graphs > 0;
    cudaGraph_t loop_graph = nullptr;
    cudaGraphExec_t loop_exec = nullptr;
    struct LoopGuard {
        cudaGraph_t *g;
        cudaGraphExec_t *e;
        ~LoopGuard() {
            if (*e) cudaGraphExecDestroy(*e);
            if (*g) cudaGraphDestroy(*g);
        }
    } lg{&loop_graph, &loop_exec};
    if (dloop) {
        // while-node (condition 1 at launch) around the round body, captured
        // into the node's body graph on a private stream
        RC_CUDA(cudaGraphCreate(&loop_graph, 0));
        RC_CUDA(cudaGraphConditionalHandleCreate(&loop_cond, loop_graph, 1,
                                                 cudaGraphCondAssignDefault));
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = loop_cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t wnode;
        RC_CUDA(cudaGraphAddNode(&wnode, loop_graph, nullptr, nullptr, 0, &np));
        cudaGraph_t body = np.conditional.phGraph_out[0];
        cudaStream_t cs = aux_stream();
        RC_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
        round_body(cs, abuf[0], abuf[1], false, true);
        RC_CUDA(cudaStreamEndCapture(cs, &body));
        RC_CUDA(cudaGraphInstantiate(&loop_exec, loop_graph, 0));
        size_t nn = 0;
        RC_CUDA(cudaGraphGetNodes(body, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        RC_CUDA(cudaGraphGetNodes(body, nodes.data(), &nn));
        round_kernels = 0;
        for (size_t k = 0; k < nn; k++) {
            cudaGraphNodeType t;
            RC_CUDA(cudaGraphNodeGetType(nodes[k], &t));
            if (t == cudaGraphNodeTypeKernel) round_kernels++;
        }
        uncount_launches(round_kernels);
    }
    if (graphs) {
        cudaStream_t cs = aux_stream();
        for (int par = 0; par < 2; par++) {
            RC_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            round_body(cs, abuf[par], abuf[par ^ 1], true, false);
            RC_CUDA(cudaStreamEndCapture(cs, &round_graph[par]));
            RC_CUDA(cudaGraphInstantiate(&round_exec[par], round_graph[par], 0));
            // the captured launches are counted per graph launch instead
            size_t nn = 0;
            RC_CUDA(cudaGraphGetNodes(round_graph[par], nullptr, &nn));
            std::vector<cudaGraphNode_t> nodes(nn);
            RC_CUDA(cudaGraphGetNodes(round_graph[par], nodes.data(), &nn));
            round_kernels = 0;
            for (size_t k = 0; k < nn; k++) {
                cudaGraphNodeType t;
                RC_CUDA(cudaGraphNodeGetType(nodes[k], &t));
                if (t == cudaGraphNodeTypeKernel) round_kernels++;
            }
            uncount_launches(round_kernels);
        }
    }
    int parity = 0;
    int32_t *cur = abuf[0];
    uint64_t crcnt = 0;  // C_rcnt (rule on) or 0
    for (range = 0; range < nranges; range++) {
        k_cd_new_range<<<1, 256, 0, s>>>(st.get(), range);
        RC_LAUNCH();
        k_cd_hist<<<nb, 512, 0, s>>>(n, D.sub, D.sup, D.wfull, S.off, D.init, st.get());
        RC_LAUNCH();
        if (opt.n_bounds > 0) {
            k_set_hi<<<1, 1, 0, s>>>(st.get(), opt.h_bounds[range]);
        } else {
            k_cd_select<<<1, 1024, 0, s>>>(st.get(), range, P, range_cap);
        }
        RC_LAUNCH();
        cur = abuf[parity];
        k_cd_frontier<<<nb, 512, 0, s>>>(n, D.sub, D.sup, D.wfull, st.get(), &st.get()->nF, cur);
        RC_LAUNCH();
        // the state's header (hi, n_remaining, the activeSet's C_peel) and,
        // once, C_rcnt back to the host
        RC_CUDA(cudaMemcpyAsync(hst, st.get(), hdr, cudaMemcpyDeviceToHost, s));
        if (range == 0) RC_CUDA(cudaMemcpyAsync(hpin, rcost.get(), 8, cudaMemcpyDeviceToHost, s));
        RC_CUDA(cudaStreamSynchronize(s));
        const uint64_t hi = hst->hi;
        if (hst->n_remaining == 0) break;  // nothing remains
        if (range == 0) crcnt = hpin[0];
        D.cost_recount = crcnt;
        // the rule also skips a recount whose temporaries would not fit
        bool recount = huc == 1 || (huc == 0 && crcnt > 0 &&
                                    (double)hst->front_w > huc_factor * (double)crcnt &&
                                    recount_fits(D));
        // one trace record per round from a copy of the state's header
        auto record_round = [&](const CdDev *h, bool rc) {
            if (!rc)
                for (int t = 0; t < NTIER; t++) D.tier_launches[t]++;
            D.rounds++;
            receipt_round rr{};
            rr.range = range;
            rr.frontier = h->nF;
            rr.hi = hi;
            rr.recount = rc ? 1 : 0;
            for (int t = 0; t < NTIER; t++) {
                rr.anchors[t] = h->tier_a[t] - prev_a[t];
                rr.wedges[t] = h->tier_w[t] - prev_w[t];
                prev_a[t] = h->tier_a[t];
                prev_w[t] = h->tier_w[t];
            }
            if (rc) {
                if (dgm) peeled_at_dgm = h->peeled_edges;  // the lists were just compacted
                if (D.timing) {
                    float ms = 0;
                    RC_CUDA(cudaEventElapsedTime(&ms, ev[NTIER + 1], ev[NTIER + 2]));
                    D.ms_recount += ms;
                }
            } else if (D.timing) {
                // launch order: warp, dense window, hybrid, global, sliced
                static const int tier_of_gap[NTIER] = {0, 4, 1, 2, 3};
                for (int gp = 0; gp < NTIER; gp++) {
                    float ms = 0;
                    RC_CUDA(cudaEventElapsedTime(&ms, ev[gp], ev[gp + 1]));
                    D.tier_ms[tier_of_gap[gp]] += ms;
                    rr.ms[tier_of_gap[gp]] = ms;
                }
            }
            D.trace.push_back(rr);
        };
        for (;;) {
            if (!recount && dloop) {
                // a burst of up to ROUND_BURST rounds in one graph launch
                k_cd_burst_begin<<<1, 1, 0, s>>>(st.get(), parity);
                RC_LAUNCH();
                RC_CUDA(cudaGraphLaunch(loop_exec, s));
                RC_CUDA(cudaMemcpyAsync(hrec, rec.get(), (size_t)ROUND_BURST * hdr,
                                        cudaMemcpyDeviceToHost, s));
                RC_CUDA(cudaMemcpyAsync(hst, st.get(), hdr, cudaMemcpyDeviceToHost, s));
                RC_CUDA(cudaStreamSynchronize(s));
                const int32_t kk = hst->burst_k;
                if (kk < 1 || kk > ROUND_BURST)
                    fail(RECEIPT_ERR_INTERNAL, "device-driven rounds: bad round count");
                count_launches((uint64_t)kk * round_kernels);
                for (int32_t r = 0; r < kk; r++)
                    record_round(reinterpret_cast<const CdDev *>(hrec + (size_t)r * hdr_words),
                                 false);
                parity = hst->par;
                if (hst->nF == 0) break;  // the last round left no next activeSet
                continue;
            }
            if (recount) {
                huc_round(abuf[parity], abuf[parity ^ 1]);
            } else if (graphs) {
                RC_CUDA(cudaGraphLaunch(round_exec[parity], s));
                count_launches(round_kernels);
            } else {
                round_body(s, abuf[parity], abuf[parity ^ 1], false, false);
            }
            RC_CUDA(cudaStreamSynchronize(s));
            record_round(hst, recount);
            if (hst->nNext == 0) break;
            parity ^= 1;  // the next round reads the activeSet this one wrote
            recount = false;
        }
        D.bounds.push_back(hi);
        // dynamic graph maintenance: once the vertices assigned since the last
        // compaction hold DGM_FRAC of the live adjacency entries, drop them
        // from the lists
        const uint64_t peeled_now = hst->peeled_edges;
        if (dgm && O.n > 0 && range + 1 < nranges &&
            (double)(peeled_now - peeled_at_dgm) >= dgm_frac * (double)(D.m - peeled_at_dgm)) {
            k_dgm_compact<<<std::min(ceil_div((int64_t)O.n * 32, 256), sms * 32), 256, 0, s>>>(
                O.off, len_w.get(), adj_w.get(), O.n, D.sub);
            RC_LAUNCH();
            k_list_window<<<ceil_div(O.n, 256), 256, 0, s>>>(O.off, len_w.get(), adj_w.get(), O.n,
                                                            kwin.get());
            RC_LAUNCH();
            if (table) {
                k_slice_table<<<ceil_div((int64_t)O.n * (C + 1), 256), 256, 0, s>>>(
                    O.off, len_w.get(), adj_w.get(), O.n, C, SW, soff.get());
                RC_LAUNCH();
            }
            peeled_at_dgm = peeled_now;
            D.dgm_passes++;
        }
    }
    // leftover subset with an open range
    DevBuf<int> any(1, s);
    any.zero();
    k_cd_leftover<<<nb, 512, 0, s>>>(n, D.sub, D.sup, D.init, range, any.get());
    RC_LAUNCH();
    int hany = 0;
    RC_CUDA(cudaMemcpyAsync(&hany, any.get(), 4, cudaMemcpyDeviceToHost, s));
    unsigned long long hw = 0, ht[4 * NTIER];
    RC_CUDA(cudaMemcpyAsync(&hw, &st.get()->wedges, 8, cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaMemcpyAsync(ht, st.get()->tier_w, sizeof(ht), cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaStreamSynchronize(s));
    D.p_eff = range + (hany ? 1 : 0);
    if (hany) D.bounds.push_back(~0ull);
    D.wedges_cd = hw;
    for (int t = 0; t < NTIER; t++) {
        D.tier_wedges[t] = ht[t];
        D.tier_mids[t] = ht[NTIER + t];
        D.tier_anchors[t] = ht[2 * NTIER + t];
        D.tier_pairs[t] = ht[3 * NTIER + t];
    }
}

void compact_lists(const int64_t *off_o, int32_t *len_w, int32_t *adj_w, int32_t n_o,
                   const int32_t *sub, cudaStream_t s) {
    if (n_o <= 0) return;
    k_dgm_compact<<<std::min(ceil_div((int64_t)n_o * 32, 256), num_sms() * 32), 256, 0, s>>>(
        off_o, len_w, adj_w, n_o, sub);
    RC_LAUNCH();
}

void list_lengths(const int64_t *off, int32_t n, int32_t *len, cudaStream_t s) {
    if (n <= 0) return;
    k_list_lengths<<<ceil_div(n, 256), 256, 0, s>>>(off, n, len);
    RC_LAUNCH();
}

// wfull for side s
void compute_wfull(const Side &S, const Side &O, int64_t m, unsigned long long *wfull,
                   cudaStream_t s) {
    if (S.n == 0) return;
    if (m == 0) {
        RC_CUDA(cudaMemsetAsync(wfull, 0, sizeof(unsigned long long) * S.n, s));
        return;
    }
    DevBuf<int64_t> dn(m + 1, s), ps(m + 1, s);
    k_deg_of_nbr<<<ceil_div(m, 256), 256, 0, s>>>(S.adj, m, O.off, dn.get());
    RC_LAUNCH();
    RC_CUDA(cudaMemsetAsync(dn.get() + m, 0, sizeof(int64_t), s));
    scan_exclusive<int64_t>(dn.get(), ps.get(), m + 1, s);
    k_wfull<<<ceil_div(S.n, 256), 256, 0, s>>>(S.off, S.n, ps.get(), wfull);
    RC_LAUNCH();
}

}  // namespace receipt
