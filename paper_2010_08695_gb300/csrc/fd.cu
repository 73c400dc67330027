// Fine-grained decomposition, Algorithm 4 (RECEIPT FD), with the
// workload-aware scheduling of Sec. 3.2.1.
//
// Setup (all on the device):
//  * members of every subset U_i, ordered by local id; rank[x] = position of
//    x inside its subset (the key space of G_i's aggregation);
//  * the induced subgraphs G_i = (U_i, V, E_i) all at once: the other side's
//    adjacency (sorted by (y, x)) is stably sorted by sub(x), so the block of
//    subset i lists, for every y, the ranks of y's neighbours inside U_i as
//    one contiguous run; every edge (x, y) of side s records where its run
//    (sub(x), y) starts and how long it is;
//  * a task queue of subset ids in decreasing order of their wedge count
//    (Longest Processing Time first).
//
// Peeling: persistent CTAs pop subsets from the queue with one atomic each.
// Inside a subset the CTA runs bottom-up peeling level by level: the level
// mu = max(previous level, min support over the remaining vertices); every
// vertex whose raw support is <= mu is peeled with tip number mu, and the
// updates of Algorithm 2 restricted to G_i are applied. Peeling all
// minimum-support vertices together gives the same tip numbers as peeling
// them one at a time: max(mu, max(mu, a) - b) = max(mu, a - b) for b >= 0,
// and supports are order independent (Lemma 1).
#include <algorithm>

#include "engine.cuh"
#include "internal.cuh"

namespace receipt {

namespace {

constexpr int FD_THREADS = 512;
// dense counters of the fine-grained step: 30,720 words (61,440 16-bit keys)
constexpr int FD_WORDS = 30720;
constexpr int FD_KEYS = 2 * FD_WORDS;
// the touched-word list doubles as the window histogram between passes
using FdEngine = DenseSliceT<FD_WORDS, TOUCH_LIST>;
static_assert(TOUCH_CAP * 2 >= LOG_BUCKETS * 4, "histogram in the touched-word list");
// walk-size flag: the vertex's degree is >= 65535 (counts may need 32 bits)
constexpr unsigned long long WIDE_BIT = 1ull << 63;
// heavy subsets: automatic threshold
constexpr unsigned long long HEAVY_MIN_W = 1ull << 23;
constexpr unsigned long long HEAVY_SHARE = 8;
// a level of a heavy task with at most this many members with big walks
// (and at least two CTAs for each) splits each one's walk over the CTAs
// (partial counts summed in global counters) instead of giving each member
// one CTA
constexpr int FDH_SPLIT_NB = 32;
// a task whose walk wedges reach this many times LEVEL_WEDGES per member is
// walk-bound (see the heavy rule)
constexpr unsigned long long HEAVY_WALK_LEVELS = 4;
// parts of one subset are merged into tasks of at least this many members
constexpr int32_t TASK_MIN = 8192;
// LPT weight of one member of a task in wedges: a level of the one-CTA peel
// costs ~20-40 us (measured on Chung-Lu graphs of 10M-100M edges), the time
// a CTA needs for ~2^15 wedges of updates
constexpr unsigned long long LEVEL_WEDGES = 1ull << 15;

__global__ void k_sub_keys(const int32_t *__restrict__ sub, int32_t n, uint64_t *__restrict__ key,
                           uint32_t *__restrict__ val, int32_t *__restrict__ cnt) {
    int32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n) {
        key[x] = (uint64_t)sub[x];
        val[x] = (uint32_t)x;
        atomicAdd(&cnt[sub[x]], 1);
    }
}

__global__ void k_members(const uint32_t *__restrict__ sorted_x, int32_t n,
                          const int32_t *__restrict__ sub, const int32_t *__restrict__ mstart,
                          int32_t *__restrict__ members, int32_t *__restrict__ rank) {
    int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) {
        int32_t x = (int32_t)sorted_x[p];
        members[p] = x;
        rank[x] = p - mstart[sub[x]];
    }
}

__global__ void k_edge_sub_keys(const int32_t *__restrict__ adj_o, int64_t m,
                                const int32_t *__restrict__ sub, uint64_t *__restrict__ key,
                                uint32_t *__restrict__ val) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) {
        key[k] = (uint64_t)sub[adj_o[k]];
        val[k] = (uint32_t)k;
    }
}

__device__ __forceinline__ int32_t owner_of(const int64_t *off, int32_t n, int64_t q) {
    int32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int32_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= q)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// For sorted position p: y, sub, rank, and run head flag.
__global__ void k_fd_fill(const uint32_t *__restrict__ perm, int64_t m, const int32_t *__restrict__ adj_o,
                          const int64_t *__restrict__ off_o, int32_t n_o,
                          const int32_t *__restrict__ sub, const int32_t *__restrict__ rank,
                          int32_t *__restrict__ fd_adj, int32_t *__restrict__ fd_y,
                          uint32_t *__restrict__ head) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    int64_t k = perm[p];
    int32_t x = adj_o[k];
    int32_t y = owner_of(off_o, n_o, k);
    fd_adj[p] = rank[x];
    fd_y[p] = y;
    uint32_t h = 1;
    if (p > 0) {
        int64_t k2 = perm[p - 1];
        int32_t x2 = adj_o[k2];
        int32_t y2 = owner_of(off_o, n_o, k2);
        h = (sub[x2] != sub[x] || y2 != y) ? 1u : 0u;
    }
    head[p] = h;
}

__global__ void k_run_starts(const uint32_t *__restrict__ head, const uint32_t *__restrict__ hpos,
                             int64_t m, int64_t *__restrict__ run_start) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < m && head[p]) run_start[hpos[p]] = p;
}

// Run of every side-s edge (x, y), and each subset's wedge count.
__global__ void k_fd_edges(const uint32_t *__restrict__ perm, int64_t m,
                           const int32_t *__restrict__ adj_o, const int32_t *__restrict__ fd_y,
                           const uint32_t *__restrict__ head, const uint32_t *__restrict__ hpos,
                           const int64_t *__restrict__ run_start, int64_t nruns,
                           const int64_t *__restrict__ off_s, const int32_t *__restrict__ adj_s,
                           const int32_t *__restrict__ sub, int64_t *__restrict__ fd_beg,
                           int32_t *__restrict__ fd_len, unsigned long long *__restrict__ wsub) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    int64_t r = (int64_t)hpos[p] + head[p] - 1;  // run id
    int64_t rs = run_start[r];
    int64_t re = r + 1 < nruns ? run_start[r + 1] : m;
    int32_t x = adj_o[perm[p]];
    int32_t y = fd_y[p];
    int64_t b = off_s[x];
    int64_t ps = b + lower_bound_i32(adj_s + b, off_s[x + 1] - b, y);
    fd_beg[ps] = rs;
    fd_len[ps] = (int32_t)(re - rs);
    if (head[p]) {
        unsigned long long L = (unsigned long long)(re - rs);
        if (L > 1) atomicAdd(&wsub[sub[x]], L * (L - 1));
    }
}

__global__ void k_i32_to_i64(const int32_t *__restrict__ v, int64_t m, int64_t *__restrict__ out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < m) out[q] = v[q];
}

// Walk size inside G_i of every vertex (sum of its edges' run lengths, from
// the prefix sums `pre`), stored at its member position; WIDE_BIT marks a
// degree >= 65535 (counts may need 32 bits).
__global__ void k_fd_walk_sizes(const int64_t *__restrict__ off_s, int32_t n,
                                const int64_t *__restrict__ pre, const int32_t *__restrict__ sub,
                                const int32_t *__restrict__ mstart, const int32_t *__restrict__ rank,
                                unsigned long long *__restrict__ wr) {
    int32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const int64_t q0 = off_s[x], q1 = off_s[x + 1];
    const unsigned long long W = (unsigned long long)(pre[q1] - pre[q0]);
    wr[mstart[sub[x]] + rank[x]] = W | (q1 - q0 >= 65535 ? WIDE_BIT : 0ull);
}

// Task boundaries: the first member of every subset and, when the side is a
// union of packed graphs (parts = first vertex of each graph), every member
// whose graph differs from the previous member's.
__global__ void k_task_flags(const int32_t *__restrict__ members, int32_t n,
                             const int32_t *__restrict__ sub, const int32_t *__restrict__ mstart,
                             const int64_t *__restrict__ parts, int ng,
                             uint32_t *__restrict__ flag) {
    const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t x = members[p];
    uint32_t f = p == mstart[sub[x]] ? 1u : 0u;
    if (!f && ng > 0) {
        auto graph_of = [&](int64_t v) {
            int lo = 0, hi = ng - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (parts[mid] <= v)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            return lo;
        };
        f = graph_of(x) != graph_of(members[p - 1]) ? 1u : 0u;
    }
    flag[p] = f;
}

__global__ void k_flag_positions(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pos,
                                 int32_t n, int32_t *__restrict__ out) {
    const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n && flag[p]) out[pos[p]] = p;
}

__global__ void k_walk_plain(const unsigned long long *__restrict__ wr, int32_t n,
                             int64_t *__restrict__ out) {
    const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) out[p] = (int64_t)(wr[p] & ~WIDE_BIT);
}

__global__ void k_task_weights(const int32_t *__restrict__ tstart, const int32_t *__restrict__ tlen,
                               const int64_t *__restrict__ cw, int32_t T,
                               unsigned long long *__restrict__ w) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) w[t] = (unsigned long long)(cw[tstart[t] + tlen[t]] - cw[tstart[t]]);
}

struct FdArgs {
    const int32_t *queue;      // task ids, LPT order
    int32_t P;                 // tasks
    int32_t *qhead;
    const int32_t *tstart;     // per task: first member position
    const int32_t *tlen;       // per task: members
    const int32_t *tkb;        // per task: rank of its first member inside its subset
    const int32_t *members;
    const int64_t *off_s;
    const int64_t *fd_beg;
    const int32_t *fd_len;
    const int32_t *fd_adj;
    const int32_t *new2old;
    const unsigned long long *init;
    unsigned long long *fsup;  // by member position
    uint8_t *alive;            // by member position
    int32_t *alist;            // by member position: alive members outside the window (two buffers)
    int32_t *alist2;
    int32_t *clist;            // by member position: members inside the window (two buffers)
    int32_t *clist2;
    int32_t *plist;            // by member position
    int32_t *blist;            // by member position: peeled vertices with big updates
    unsigned long long *tip;   // output, original ids
    unsigned long long *stats; // [0] wedges, [1] levels
    unsigned long long *sub_ns;     // per task: nanoseconds spent
    unsigned long long *sub_levels; // per task: peeling levels
    unsigned long long *wr;    // by member position: walk size inside G_i (WIDE_BIT: degree >= 65535)
};

struct FdMids {
    const int64_t *fd_beg;
    const int32_t *fd_len;
    __device__ __forceinline__ void seg(int64_t q, int64_t &beg, int32_t &len) const {
        beg = fd_beg[q];
        len = fd_len[q];
    }
};

// Support decrement of an alive member. Values below the window bound T
// also lower *mn, so that after a level's updates *mn holds the minimum
// support of the window's survivors (together with the minimum of the
// untouched ones, taken when the level's peeled vertices are selected); a
// member whose support falls below T here joins the window's list.
struct FdEmit {
    unsigned long long *fsup;  // subset base
    const uint8_t *alive;      // subset base
    unsigned long long *mn;    // next level's minimum (shared or global)
    unsigned long long T;      // window bound (~0: everything is inside)
    int32_t *cand;             // window list (null without a window)
    int *n_cand;
    __device__ __forceinline__ void operator()(int32_t k, uint32_t c) {
        if (alive[k]) {
            const unsigned long long d = choose2(c);
            const unsigned long long old = atomicAdd(&fsup[k], 0ull - d);
            const unsigned long long nv = old - d;
            if (nv < T) {
                atomicMin(mn, nv);
                if (old >= T) cand[atomicAdd(n_cand, 1)] = k;
            }
        }
    }
    // N pairs at once (k < 0: none): all `alive` loads, then all support
    // atomics, then the bookkeeping, so their latencies overlap.
    template <int N>
    __device__ __forceinline__ void many(const int32_t (&k)[N], const uint32_t (&c)[N]) {
        bool al[N];
#pragma unroll
        for (int u = 0; u < N; u++) al[u] = k[u] >= 0 && alive[k[u]];
        unsigned long long old[N], d[N];
#pragma unroll
        for (int u = 0; u < N; u++) {
            d[u] = choose2(c[u]);
            old[u] = al[u] ? atomicAdd(&fsup[k[u]], 0ull - d[u]) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < N; u++) {
            if (!al[u]) continue;
            const unsigned long long nv = old[u] - d[u];
            if (nv < T) {
                atomicMin(mn, nv);
                if (old[u] >= T) cand[atomicAdd(n_cand, 1)] = k[u];
            }
        }
    }
};

// Ranks of one slice [base, end) of the subset's rank space: the run of a
// middle vertex is sorted by rank, so the slice is a sub-run found by two
// binary searches.
struct FdSliceMids {
    const int64_t *fd_beg;
    const int32_t *fd_len;
    const int32_t *fd_adj;
    int32_t base, end;
    __device__ __forceinline__ void seg(int64_t q, int64_t &beg, int32_t &len) const {
        const int64_t b = fd_beg[q];
        const int32_t l = fd_len[q];
        const int64_t lo = lower_bound_i32(fd_adj + b, l, base);
        const int64_t hi = lo + lower_bound_i32(fd_adj + b + lo, l - lo, end);
        beg = b + lo;
        len = (int32_t)(hi - lo);
    }
};

// Keys of a run are ranks inside the subset; a task covering the subset's
// ranks [kb, kb + ni) sees them shifted by kb.
struct FdSliceVisit {
    FdEngine *eng;
    int32_t base;  // first rank of the slice (subset ranks)
    int32_t self;  // the anchor's own rank (subset ranks)
    __device__ __forceinline__ void operator()(int, int32_t key) {
        if (key != self) eng->add(key - base);
    }
};

struct FdSliceEmit {
    FdEmit *e;
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

// Several anchors of one level aggregated in one pass: anchor slot a of the
// batch owns keys [a * ni, (a + 1) * ni) of the dense counters. The batch's
// edges form one virtual list of middle vertices; the thread that stages a
// middle vertex records its anchor slot for the visits.
constexpr int FD_BATCH = 32;
// window of the level loop: about max(MIN, min(MAX, alive / 32)) members
constexpr int FD_WINDOW_MIN = 512;
constexpr int FD_WINDOW_MAX = 4096;

struct FdBatchMids {
    const int64_t *fd_beg;
    const int32_t *fd_len;
    const int64_t *bq0;   // first edge of each anchor (shared memory)
    const int32_t *bpre;  // prefix of the anchors' degrees (nb + 1 entries)
    int32_t nb;
    uint8_t *slot;        // anchor slot of the middle vertex staged by each thread
    __device__ __forceinline__ void seg(int64_t q, int64_t &beg, int32_t &len) const {
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bpre[mid] <= q)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int64_t e = bq0[lo] + (q - bpre[lo]);
        beg = fd_beg[e];
        len = fd_len[e];
        slot[threadIdx.x] = (uint8_t)lo;
    }
};

struct FdBatchVisit {
    FdEngine *eng;
    const uint8_t *slot;
    const int32_t *bself;  // rank of each anchor (task ranks)
    int32_t ni;
    int32_t kb;            // first subset rank of the task
    __device__ __forceinline__ void operator()(int k, int32_t key) {
        const int a = slot[k];
        key -= kb;
        if (key != bself[a]) eng->add(a * ni + key);
    }
};

struct FdBatchEmit {
    FdEmit *e;
    int32_t ni;
    __device__ __forceinline__ void operator()(int32_t w, uint32_t c) { (*e)(w % ni, c); }
    template <int N>
    __device__ __forceinline__ void many(const int32_t (&k)[N], const uint32_t (&c)[N]) {
        int32_t kk[N];
#pragma unroll
        for (int u = 0; u < N; u++) kk[u] = k[u] >= 0 ? k[u] % ni : -1;
        e->template many<N>(kk, c);
    }
};

// Update of one peeled member r (anchor x, edges [q0, q1) of side s) whose
// walk has at most WARP_MAX_W wedges: one warp with its private table.
__device__ __forceinline__ void fd_update_warp(WarpHash &WH, const FdMids &M,
                                               const int32_t *__restrict__ fd_adj, int64_t q0,
                                               int64_t q1, int32_t r, int32_t kb, int lane,
                                               FdEmit &emit) {
    auto add = [&](int32_t key) {
        const int32_t k = key - kb;
        if (k != r) WH.add(k);
    };
    warp_walk<4>(M, q0, q1, fd_adj, add);
    __syncwarp();
    WH.flush_clear(emit, lane);
    __syncwarp();
}

// Update of one peeled member r with a bigger walk: the whole CTA aggregates
// slice by slice of the subset's rank space (ni ranks) with dense counters,
// 32-bit ones when the anchor's degree lets a count reach 2^16. Returns the
// wedges walked (the same value in every thread). All threads must call it.
// What a CTA does with one aggregated slice: apply the member's updates
// (count c of a key -> support decrement C(c, 2)) ...
struct FdSweepOut {
    FdEmit *emit;
    __device__ __forceinline__ void slice(FdEngine &H, int32_t base) {
        FdSliceEmit em{emit, base};
        H.sweep<true, true>(em);
    }
};

// ... or add its partial counts (the walk of part of the member's middle
// vertices) to global counters over the task's ranks, listing each key the
// first time its counter leaves 0; the slice is cleared either way.
struct FdPartialOut {
    uint32_t *gcnt;  // ni counters of this member
    int32_t *gtl;    // keys with a non-zero counter
    int32_t *gnt;    // their number
    __device__ __forceinline__ void add(int32_t z, uint32_t c) {
        if (atomicAdd(&gcnt[z], c) == 0u) gtl[atomicAdd(gnt, 1)] = z;
    }
    __device__ __forceinline__ void slice(FdEngine &H, int32_t base) {
        const int nt = *(volatile int *)H.s_nt;
        const bool listed = nt <= FdEngine::TCAP;
        const int n = listed ? nt : H.hw;  // touched words, or every word of the slice
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int w = listed ? (int)H.tl[i] : i;
            const uint32_t v = H.cnt[w];
            if (v == 0u) continue;
            H.cnt[w] = 0u;
            if (H.wide) {
                add(base + w, v);
            } else {
                if (v & 0xffffu) add(base + w, v & 0xffffu);
                if (v >> 16) add(base + w + H.hw, v >> 16);
            }
        }
    }
};

// Part of a member's walk: the runs of its edges [q0, q1) with the first run
// taken from position `skip` on and the last one up to position `keep`
// (split heavy levels cut a walk into equal wedge shares), optionally only
// the ranks of one slice [base, end) of each.
struct FdClipMids {
    const int64_t *fd_beg;
    const int32_t *fd_len;
    const int32_t *fd_adj;
    int64_t qa, ql;       // first and last edge
    int32_t skip, keep;
    int32_t base, end;
    bool sliced;
    __device__ __forceinline__ void seg(int64_t q, int64_t &beg, int32_t &len) const {
        const int64_t b = fd_beg[q];
        const int32_t s0 = q == qa ? skip : 0;
        const int32_t e0 = q == ql ? keep : fd_len[q];
        if (sliced) {
            const int64_t lo = s0 + lower_bound_i32(fd_adj + b + s0, e0 - s0, base);
            const int64_t hi = lo + lower_bound_i32(fd_adj + b + lo, e0 - lo, end);
            beg = b + lo;
            len = (int32_t)(hi - lo);
        } else {
            beg = b + s0;
            len = e0 - s0;
        }
    }
};

// keep < 0: the last run whole (no cut).
template <class Out>
__device__ int64_t fd_update_cta(FdEngine &H, Chunk &ch, const int64_t *__restrict__ fd_beg,
                                 const int32_t *__restrict__ fd_len,
                                 const int32_t *__restrict__ fd_adj, int64_t q0, int64_t q1,
                                 int32_t r, int32_t ni, int32_t kb, Out &out, int32_t skip = 0,
                                 int32_t keep = -1) {
    const bool clip = skip != 0 || keep >= 0;
    if (clip && keep < 0) keep = fd_len[q1 - 1];
    const bool wide = q1 - q0 >= 65535;
    const int32_t SWk = wide ? FD_WORDS : FD_KEYS;
    const int32_t C = (ni + SWk - 1) / SWk;
    // only the slices that meet the anchor's rank window (first and last
    // entries of its runs, which are sorted by rank)
    int32_t j0 = 0, j1 = C - 1;
    if (C > 1) {
        int32_t *win = ch.tmp;  // scan scratch, idle here
        if (threadIdx.x == 0) {
            win[0] = INT32_MAX;
            win[1] = -1;
        }
        __syncthreads();
        int32_t lo = INT32_MAX, hi = -1;
        for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
            const int32_t l = fd_len[q];
            if (l > 0) {
                const int64_t b = fd_beg[q];
                lo = min(lo, fd_adj[b]);
                hi = max(hi, fd_adj[b + l - 1]);
            }
        }
        lo = warp_min(lo);
        hi = -warp_min(-hi);
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&win[0], lo);
            atomicMax(&win[1], hi);
        }
        __syncthreads();
        const int32_t wlo = win[0], whi = win[1];
        __syncthreads();  // win is rewritten by the next call
        if (whi < 0) return 0;  // no runs
        j0 = (wlo - kb) / SWk;
        j1 = (whi - kb) / SWk;
    }
    int64_t wedges = 0;
    for (int32_t j = j0; j <= j1; j++) {
        const int32_t base = j * SWk;
        const int32_t w = (int32_t)imin64(SWk, (int64_t)ni - base);
        H.set_width(w, wide);
        FdSliceVisit v{&H, base + kb, r + kb};
        int64_t walked;
        if (clip) {
            FdClipMids MC{fd_beg, fd_len, fd_adj, q0,       q1 - 1,  skip,
                          keep,   base + kb, base + kb + w, j0 != j1};
            walked = cta_walk(MC, q0, q1, fd_adj, ch, v);
        } else if (j0 == j1) {
            FdMids M{fd_beg, fd_len};
            walked = cta_walk(M, q0, q1, fd_adj, ch, v);
        } else {
            FdSliceMids MS{fd_beg, fd_len, fd_adj, base + kb, base + kb + w};
            walked = cta_walk(MS, q0, q1, fd_adj, ch, v);
        }
        wedges += walked;
        if (walked == 0) continue;
        out.slice(H, base);
        __syncthreads();
        H.reset_scalars();
    }
    return wedges;
}

__device__ __forceinline__ int64_t fd_update_cta(FdEngine &H, Chunk &ch,
                                                 const int64_t *__restrict__ fd_beg,
                                                 const int32_t *__restrict__ fd_len,
                                                 const int32_t *__restrict__ fd_adj, int64_t q0,
                                                 int64_t q1, int32_t r, int32_t ni, int32_t kb,
                                                 FdEmit &emit) {
    FdSweepOut o{&emit};
    return fd_update_cta(H, ch, fd_beg, fd_len, fd_adj, q0, q1, r, ni, kb, o);
}

__device__ __forceinline__ unsigned char *fd_bind_smem(unsigned char *smem, int *s_dn, FdEngine &H,
                                                       Chunk &ch) {
    unsigned char *p = H.bind(smem, s_dn);
    ch.beg = (int64_t *)p;
    ch.pre = (int32_t *)(ch.beg + MID_CHUNK);
    ch.tmp = ch.pre + MID_CHUNK + 1;
    ch.len = chunk_len_ptr(ch.tmp);
    return (unsigned char *)(((uintptr_t)(ch.len + MID_CHUNK) + 15) & ~(uintptr_t)15);
}

__global__ void __launch_bounds__(FD_THREADS, 1) k_fd_peel(FdArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_t, s_dn, s_np, s_nbig, s_nwide, s_nf, s_pick, s_peel, s_rk;
    // window list count and next level's minimum, by level parity: level L
    // fills set L & 1 while stragglers of level L - 1 may still read the other
    __shared__ int s_nk[2];
    __shared__ unsigned long long s_mn[2];
    __shared__ unsigned long long s_rmn;  // minimum of a refilled window
    __shared__ unsigned long long s_T;   // window bound
    __shared__ int32_t s_scan[33];
    __shared__ int64_t s_bq0[FD_BATCH];
    __shared__ int32_t s_bpre[FD_BATCH + 1], s_bself[FD_BATCH];
    __shared__ uint8_t s_slot[FD_THREADS];
    FdEngine H;
    Chunk ch;
    // warp-private tables after the chunk staging
    int32_t *wkey = (int32_t *)fd_bind_smem(smem, &s_dn, H, ch);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    WarpHash WH{wkey + warp * WARP_SLOTS, (uint32_t *)(wkey + nwarps * WARP_SLOTS) + warp * WARP_SLOTS};
    WH.clear(lane);
    H.clear_all();
    FdMids M{a.fd_beg, a.fd_len};
    // per warp (lane 0): wedges walked; thread 0 also counts levels
    unsigned long long wedges = 0, levels = 0;
    __syncthreads();
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_t = atomicAdd(a.qhead, 1);
        __syncthreads();
        const int t = s_t;
        if (t >= a.P) break;
        const int32_t i = a.queue[t];
        const int32_t mb = a.tstart[i];
        const int32_t ni = a.tlen[i];
        const int32_t kb = a.tkb[i];
        if (ni == 0) continue;
        unsigned long long t_start = 0;
        if (threadIdx.x == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
        const unsigned long long levels0 = levels;
        unsigned long long *fsup = a.fsup + mb;
        uint8_t *alive = a.alive + mb;
        // members outside the window (far) and inside it (cand), each
        // double-buffered for compaction
        int32_t *flist = a.alist + mb;
        int32_t *flist_next = a.alist2 + mb;
        int32_t *clist = a.clist + mb;
        int32_t *clist_next = a.clist2 + mb;
        int32_t *plist = a.plist + mb;
        int32_t *blist = a.blist + mb;
        const int32_t *mem = a.members + mb;
        unsigned long long *wr = a.wr + mb;
        for (int r = threadIdx.x; r < ni; r += blockDim.x) {
            fsup[r] = a.init[mem[r]];
            alive[r] = 1;
            flist[r] = r;
        }
        int32_t nalive = ni, nfar = ni, ncand = 0;
        unsigned long long level = 0, mn = ~0ull;
        int par = 0;
        // anchors aggregated per pass of the batched update
        const int32_t bk = ni <= FD_KEYS / 2 ? min(FD_BATCH, FD_KEYS / ni) : 1;
        __syncthreads();
        while (nalive > 0) {
            if (ncand == 0) {
                // Window refill: the smallest supports among the far members,
                // about `target` of them, become the window [.., T); a level
                // then scans the window only, and members whose support
                // falls below T during updates join it.
                uint32_t *hist = (uint32_t *)H.tl;  // idle between passes
                for (int b = threadIdx.x; b < LOG_BUCKETS; b += blockDim.x) hist[b] = 0;
                if (threadIdx.x == 0) {
                    s_pick = LOG_BUCKETS - 1;
                    s_nf = 0;
                    s_rk = 0;
                    s_rmn = ~0ull;
                }
                __syncthreads();
                for (int j = threadIdx.x; j < nfar; j += blockDim.x) {
                    const int32_t r = flist[j];
                    if (alive[r]) atomicAdd(&hist[log_bucket_of(fsup[r])], 1u);
                }
                __syncthreads();
                {
                    constexpr int PER = (LOG_BUCKETS + FD_THREADS - 1) / FD_THREADS;
                    const int target = max(FD_WINDOW_MIN, min(FD_WINDOW_MAX, nalive / 32));
                    int32_t c[PER], sum = 0;
#pragma unroll
                    for (int e = 0; e < PER; e++) {
                        const int b = threadIdx.x * PER + e;
                        c[e] = b < LOG_BUCKETS ? (int32_t)hist[b] : 0;
                        sum += c[e];
                    }
                    int32_t run = block_exclusive_scan<int32_t>(sum, s_scan, nullptr);
#pragma unroll
                    for (int e = 0; e < PER; e++) {
                        run += c[e];
                        if (run >= target && c[e] > 0) atomicMin(&s_pick, threadIdx.x * PER + e);
                    }
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    const unsigned long long top = log_bucket_top(s_pick);
                    s_T = top == ~0ull ? ~0ull : top + 1ull;
                }
                __syncthreads();
                const unsigned long long T = s_T;
                for (int base = 0; base < nfar; base += blockDim.x) {
                    const int j = base + threadIdx.x;
                    int32_t r = -1;
                    unsigned long long v = ~0ull;
                    if (j < nfar) {
                        r = flist[j];
                        if (alive[r])
                            v = fsup[r];
                        else
                            r = -1;
                    }
                    const bool in = r >= 0 && v < T;
                    warp_append(in, r, &s_rk, clist);
                    warp_append(r >= 0 && !in, r, &s_nf, flist_next);
                    const unsigned long long kv = warp_min(in ? v : ~0ull);
                    if (lane == 0 && kv != ~0ull) atomicMin(&s_rmn, kv);
                }
                __syncthreads();
                ncand = s_rk;
                nfar = s_nf;
                mn = s_rmn;
                {
                    int32_t *tmp = flist;
                    flist = flist_next;
                    flist_next = tmp;
                }
                if (ncand == 0) break;  // cannot happen while members are alive
            }
            // mu from the minimum left by the previous level (or the refill);
            // this level's counters: the per-level ones and set `par`
            const unsigned long long mu = mn > level ? mn : level;
            const unsigned long long T = s_T;
            level = mu;
            levels++;
            if (threadIdx.x == 0) {
                s_np = 0;
                s_nk[par] = 0;
                s_nbig = 0;
                s_nwide = 0;
                s_peel = 0;
                s_mn[par] = ~0ull;
            }
            __syncthreads();
            // peel every window member with support <= mu; the rest go to
            // the other window buffer (ballot compaction, order irrelevant)
            int peeled = 0;
            constexpr int SCAN_U = 4;  // window entries per thread with their loads in flight
            for (int base0 = 0; base0 < ncand; base0 += SCAN_U * blockDim.x) {
                int32_t rr[SCAN_U];
                unsigned long long vv[SCAN_U];
#pragma unroll
                for (int u = 0; u < SCAN_U; u++) {
                    const int j = base0 + u * blockDim.x + threadIdx.x;
                    rr[u] = j < ncand ? clist[j] : -1;
                }
#pragma unroll
                for (int u = 0; u < SCAN_U; u++) vv[u] = rr[u] >= 0 ? fsup[rr[u]] : 0ull;
#pragma unroll
                for (int u = 0; u < SCAN_U; u++) {
                    const int32_t r = rr[u];
                    const unsigned long long v = vv[u];
                    const bool keep = r >= 0 && v > mu;
                    const bool peel = r >= 0 && !keep;
                    unsigned long long w = 0;
                    if (peel) {
                        alive[r] = 0;
                        a.tip[a.new2old[mem[r]]] = mu;
                        w = wr[r];
                        peeled++;
                    }
                    // updates: small walks -> one warp each; bigger ones -> the
                    // batched pass; degree >= 65535 (32-bit counts) or a subset
                    // too large to batch -> one anchor per pass (end of blist)
                    const bool upd = peel && v > 0;
                    const bool small = upd && w <= (unsigned long long)WARP_MAX_W;
                    const bool single = upd && !small && ((w & WIDE_BIT) || bk == 1);
                    warp_append(keep, r, &s_nk[par], clist_next);
                    warp_append(small, r, &s_np, plist);
                    warp_append(upd && !small && !single, r, &s_nbig, blist);
                    if (single) blist[ni - 1 - atomicAdd(&s_nwide, 1)] = r;
                    // minimum of the survivors before this level's updates
                    const unsigned long long kv = warp_min(keep ? v : ~0ull);
                    if (lane == 0 && kv != ~0ull) atomicMin(&s_mn[par], kv);
                }
            }
            peeled = warp_sum(peeled);
            if (lane == 0 && peeled) atomicAdd(&s_peel, peeled);
            __syncthreads();
            nalive -= s_peel;
            {
                int32_t *tmp = clist;
                clist = clist_next;
                clist_next = tmp;
            }
            int np = s_np;
            // a level with few updates makes them all in one batched pass
            // (one pass costs less than a warp phase followed by a pass): the
            // pass takes blist's nbig0 anchors, then plist's np
            const int nbig0 = s_nbig;
            int nmerged = 0;
            if (bk > 1 && np > 0 && np + nbig0 <= bk) {
                nmerged = np;
                np = 0;
            }
            // updates of the peeled vertices inside G_i. Phase A: one warp per
            // peeled vertex whose update walks at most WARP_MAX_W wedges.
            FdEmit emit{fsup, alive, &s_mn[par], T, clist, &s_nk[par]};
            for (int pi = warp; pi < np; pi += nwarps) {
                const int32_t r = plist[pi];
                const int32_t x = mem[r];
                fd_update_warp(WH, M, a.fd_adj, a.off_s[x], a.off_s[x + 1], r, kb, lane, emit);
                if (lane == 0) wedges += wr[r];
            }
            if (np > 0) __syncthreads();
            const int nbig = nbig0 + nmerged, nwide = s_nwide;
            // Phase B: bk anchors per pass of the whole CTA over one dense key
            // space of bk * ni keys
            for (int p0 = 0; p0 < nbig; p0 += bk) {
                const int nb = min(bk, nbig - p0);
                if (warp == 0) {
                    int32_t deg = 0;
                    if (lane < nb) {
                        const int i = p0 + lane;
                        const int32_t r = i < nbig0 ? blist[i] : plist[i - nbig0];
                        const int32_t x = mem[r];
                        const int64_t q0 = a.off_s[x];
                        deg = (int32_t)(a.off_s[x + 1] - q0);
                        s_bq0[lane] = q0;
                        s_bself[lane] = r;
                    }
                    int32_t inc = deg;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += y;
                    }
                    if (lane < nb) s_bpre[lane + 1] = inc;
                    if (lane == 0) s_bpre[0] = 0;
                }
                __syncthreads();
                H.set_width(nb * ni, false);
                FdBatchMids BM{a.fd_beg, a.fd_len, s_bq0, s_bpre, nb, s_slot};
                FdBatchVisit v{&H, s_slot, s_bself, ni, kb};
                const int64_t walked = cta_walk(BM, 0, s_bpre[nb], a.fd_adj, ch, v);
                if (threadIdx.x == 0) wedges += (unsigned long long)walked;
                if (walked > 0) {
                    FdBatchEmit em{&emit, ni};
                    H.sweep<true, true>(em);
                    __syncthreads();
                    // the next use of the touched-word count is after the next
                    // pass's set-up barrier (or the level's last barrier)
                    H.reset_scalars();
                }
            }
            // one anchor at a time: degree >= 65535, or a subset too large
            // to batch (rank slices)
            for (int pi = 0; pi < nwide; pi++) {
                const int32_t r = blist[ni - 1 - pi];
                const int32_t x = mem[r];
                const int64_t walked = fd_update_cta(H, ch, a.fd_beg, a.fd_len, a.fd_adj,
                                                     a.off_s[x], a.off_s[x + 1], r, ni, kb, emit);
                if (threadIdx.x == 0) wedges += (unsigned long long)walked;
            }
            __syncthreads();
            // window survivors plus the members that fell below T
            ncand = s_nk[par];
            mn = s_mn[par];
            par ^= 1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t_end;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
            a.sub_ns[i] = t_end - t_start;
            a.sub_levels[i] = levels - levels0;
        }
    }
    if (lane == 0 && wedges) atomicAdd(&a.stats[0], wedges);
    if (threadIdx.x == 0) atomicAdd(&a.stats[1], levels);
}

// ------------------------------------------------------------------------
// Heavy subsets: one subset peeled by all CTAs, level by level. A subset
// whose wedge count dwarfs the others' would otherwise keep one CTA busy
// long after the rest of the queue is done. Per level: mu from the minimum
// support of the alive members; every alive member with support <= mu is
// peeled (tip mu) and listed by the size of its walk; the warp kernel and the
// CTA kernel apply the updates of the listed members, one warp or one CTA per
// member, and the survivors' minimum for the next level is gathered on the
// way. Same levels, same tip numbers as the one-CTA peel.
// ------------------------------------------------------------------------
struct FdhDev {
    unsigned long long mn;       // minimum support of the alive members
    unsigned long long mn_next;  // the same after this level (survivors, updates)
    unsigned long long level;    // mu of the last level
    unsigned long long wedges, levels;
    unsigned long long t0, t1;   // globaltimer at the start and at the end
    unsigned long long cpeel;    // walk sizes of this level's peeled members with updates
    unsigned long long rcnt;     // C_rcnt of the task's induced subgraph
    int32_t nalive, nkeep, nw, nb;
    int32_t gnt[FDH_SPLIT_NB];   // split levels: keys listed per member
    unsigned long long splits;   // split levels so far
};

struct FdhArgs {
    const int32_t *mem;  // task members (local ids), rank order
    int32_t ni;
    int32_t kb;          // rank of the task's first member inside its subset
    const int64_t *off_s;
    const int64_t *fd_beg;
    const int32_t *fd_len;
    const int32_t *fd_adj;
    const int32_t *new2old;
    const unsigned long long *init;
    unsigned long long *fsup;  // by rank
    uint8_t *alive;            // by rank
    unsigned long long *wr;    // by rank: wedges of the member's walk inside G_i
    int32_t *Lw, *Lb;          // peeled members with small / big walks
    unsigned long long *tip;   // output, original ids
    FdhDev *st;
    uint32_t *gcnt;            // split levels: FDH_SPLIT_NB x ni counters, zero between levels
    int32_t *gtl;              // split levels: FDH_SPLIT_NB x ni listed keys
    const int64_t *wpre;       // side-s edges: exclusive prefix of the run lengths
};

// A level splits its big-walk members' middle vertices over the CTAs when it
// has few of them (the same test in the update and the sweep kernel).
__device__ __forceinline__ bool fdh_split(int32_t nb, int32_t grid) {
    return nb > 0 && nb <= FDH_SPLIT_NB && grid >= 2 * nb;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void k_fdh_reset(FdhDev *st, int32_t ni) {
    st->mn = st->mn_next = ~0ull;
    st->cpeel = st->rcnt = 0;
    st->level = 0;
    st->wedges = st->levels = 0;
    st->t0 = globaltimer_ns();
    st->t1 = 0;
    st->nalive = ni;
    st->nkeep = st->nw = st->nb = 0;
    for (int i = 0; i < FDH_SPLIT_NB; i++) st->gnt[i] = 0;
    st->splits = 0;
}

__global__ void k_fdh_init(FdhArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long mn = ~0ull;
    for (int64_t r = w0; r < a.ni; r += nw) {
        if (lane == 0) {
            const unsigned long long v = a.init[a.mem[r]];
            a.fsup[r] = v;
            a.alive[r] = 1;
            mn = v < mn ? v : mn;
        }
    }
    if (lane == 0 && mn != ~0ull) atomicMin(&a.st->mn, mn);
}

__global__ void k_fdh_select(FdhArgs a) {
    const unsigned long long lv = a.st->level, mn = a.st->mn;
    const unsigned long long mu = mn > lv ? mn : lv;
    int32_t keep = 0;
    unsigned long long kmin = ~0ull, cpeel = 0;
    for (int32_t base = blockIdx.x * blockDim.x; base < a.ni; base += gridDim.x * blockDim.x) {
        const int32_t r = base + threadIdx.x;
        const bool al = r < a.ni && a.alive[r];
        const unsigned long long v = al ? a.fsup[r] : 0;
        const bool peel = al && v <= mu;
        if (peel) {
            a.alive[r] = 0;
            a.tip[a.new2old[a.mem[r]]] = mu;
        }
        const bool upd = peel && v > 0;
        const bool small = upd && a.wr[r] <= (unsigned long long)WARP_MAX_W;
        if (upd) cpeel += a.wr[r] & ~WIDE_BIT;
        warp_append(small, r, &a.st->nw, a.Lw);
        warp_append(upd && !small, r, &a.st->nb, a.Lb);
        if (al && !peel) {
            keep++;
            kmin = v < kmin ? v : kmin;
        }
    }
    keep = warp_sum(keep);
    kmin = warp_min(kmin);
    cpeel = warp_sum(cpeel);
    if ((threadIdx.x & 31) == 0) {
        if (keep) atomicAdd(&a.st->nkeep, keep);
        if (kmin != ~0ull) atomicMin(&a.st->mn_next, kmin);
        if (cpeel) atomicAdd(&a.st->cpeel, cpeel);
    }
}

// Hybrid update computation inside the fine-grained step (Sec. 4.1): a
// member's support is the butterflies it shares with the vertices of higher
// subsets (constant while its task is peeled: init minus its count inside
// G_i) plus those it shares with the task's members still alive (its count
// inside the alive part of G_i). A level of a heavy task may therefore
// replace its updates by a recount of the alive part.
//
// C_rcnt of the task's induced subgraph: sum over its members' edges (x, y)
// of min(d_x, d_y inside G_i).
__global__ void k_fdh_rcnt(FdhArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long sum = 0;
    for (int64_t r = w0; r < a.ni; r += nw) {
        const int32_t x = a.mem[r];
        const int64_t q0 = a.off_s[x], q1 = a.off_s[x + 1];
        for (int64_t q = q0 + lane; q < q1; q += 32)
            sum += (unsigned long long)imin64(q1 - q0, a.fd_len[q]);
    }
    sum = warp_sum(sum);
    if (lane == 0 && sum) atomicAdd(&a.st->rcnt, sum);
}

// keep[mem[r]] = -1 for the task's members (alive ones only with alive_only),
// the others of the side stay excluded (0).
__global__ void k_fdh_keep(FdhArgs a, int32_t *__restrict__ keep, int alive_only) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < a.ni && (!alive_only || a.alive[r])) keep[a.mem[r]] = -1;
}

// Supports of the alive members after a recount: init - (count inside G_i)
// + (count inside the alive part of G_i); the next level's minimum follows.
__global__ void k_fdh_apply(FdhArgs a, const unsigned long long *__restrict__ cnt0,
                            const unsigned long long *__restrict__ cntr) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = ~0ull;
    if (r < a.ni && a.alive[r]) {
        const int32_t x = a.mem[r];
        v = a.init[x] - cnt0[x] + cntr[x];
        a.fsup[r] = v;
    }
    v = warp_min(v);
    if ((threadIdx.x & 31) == 0 && v != ~0ull) atomicMin(&a.st->mn_next, v);
}

__global__ void __launch_bounds__(256) k_fdh_warp(FdhArgs a) {
    __shared__ int32_t skey[8][WARP_SLOTS];
    __shared__ uint32_t sval[8][WARP_SLOTS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    WarpHash WH{skey[w], sval[w]};
    WH.clear(lane);
    __syncwarp();
    FdEmit emit{a.fsup, a.alive, &a.st->mn_next, ~0ull, nullptr, nullptr};
    FdMids M{a.fd_beg, a.fd_len};
    const int32_t nw = a.st->nw;
    unsigned long long wedges = 0;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t ngw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gw; i < nw; i += ngw) {
        const int32_t r = a.Lw[i];
        const int32_t x = a.mem[r];
        fd_update_warp(WH, M, a.fd_adj, a.off_s[x], a.off_s[x + 1], r, a.kb, lane, emit);
        wedges += a.wr[r];
    }
    if (lane == 0 && wedges) atomicAdd(&a.st->wedges, wedges);
}

__global__ void __launch_bounds__(FD_THREADS, 1) k_fdh_cta(FdhArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_dn;
    FdEngine H;
    Chunk ch;
    fd_bind_smem(smem, &s_dn, H, ch);
    H.clear_all();
    __syncthreads();
    FdEmit emit{a.fsup, a.alive, &a.st->mn_next, ~0ull, nullptr, nullptr};
    const int32_t nb = a.st->nb;
    unsigned long long wedges = 0;
    if (fdh_split(nb, gridDim.x)) {
        // K CTAs per member, each over an equal share of its walk's wedges
        // (runs cut at the share's ends); k_fdh_sweep applies the summed
        // counts
        const int32_t K = gridDim.x / nb;
        for (int32_t it = blockIdx.x; it < nb * K; it += gridDim.x) {
            const int32_t i = it / K, k = it % K;
            const int32_t r = a.Lb[i];
            const int32_t x = a.mem[r];
            const int64_t q0 = a.off_s[x], q1 = a.off_s[x + 1];
            const int64_t w0 = a.wpre[q0], W = a.wpre[q1] - w0;
            const int64_t lo = w0 + W * k / K, hi = w0 + W * (k + 1) / K;
            if (lo == hi) continue;
            // edge whose run holds wedge position p: the last q in [q0, q1)
            // with wpre[q] <= p (runs of length 0 are passed over)
            auto run_of = [&](int64_t p) {
                int64_t l = q0, h = q1 - 1;
                while (l < h) {
                    const int64_t md = (l + h + 1) >> 1;
                    if (a.wpre[md] <= p)
                        l = md;
                    else
                        h = md - 1;
                }
                return l;
            };
            const int64_t qa = run_of(lo), ql = run_of(hi - 1);
            const int32_t skip = (int32_t)(lo - a.wpre[qa]);
            const int32_t keep = (int32_t)(hi - a.wpre[ql]);
            FdPartialOut o{a.gcnt + (size_t)i * a.ni, a.gtl + (size_t)i * a.ni, &a.st->gnt[i]};
            wedges += (unsigned long long)fd_update_cta(H, ch, a.fd_beg, a.fd_len, a.fd_adj, qa,
                                                        ql + 1, r, a.ni, a.kb, o, skip, keep);
        }
    } else {
        for (int32_t i = blockIdx.x; i < nb; i += gridDim.x) {
            const int32_t r = a.Lb[i];
            const int32_t x = a.mem[r];
            wedges += (unsigned long long)fd_update_cta(H, ch, a.fd_beg, a.fd_len, a.fd_adj,
                                                        a.off_s[x], a.off_s[x + 1], r, a.ni, a.kb,
                                                        emit);
        }
    }
    if (threadIdx.x == 0 && wedges) atomicAdd(&a.st->wedges, wedges);
}

// Split levels: the summed count c of every listed key becomes the support
// decrement C(c, 2) of that member (alive ones only), and the counters return
// to zero. `grid` is the update kernel's grid.
__global__ void k_fdh_sweep(FdhArgs a, int32_t grid) {
    const int32_t nb = a.st->nb;
    if (!fdh_split(nb, grid)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.st->splits++;
    FdEmit emit{a.fsup, a.alive, &a.st->mn_next, ~0ull, nullptr, nullptr};
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    for (int32_t i = 0; i < nb; i++) {
        uint32_t *gc = a.gcnt + (size_t)i * a.ni;
        const int32_t *gl = a.gtl + (size_t)i * a.ni;
        const int32_t n = a.st->gnt[i];
        for (int64_t t = t0; t < n; t += nt) {
            const int32_t z = gl[t];
            const uint32_t c = gc[z];
            gc[z] = 0u;
            if (c >= 2u) emit(z, c);
        }
    }
}

// Closes a level. Launched again after the subset is empty, it changes
// nothing that is read later (the host enqueues levels ahead of its check).
__device__ void fdh_close_level(FdhDev *st) {
    for (int i = 0; i < FDH_SPLIT_NB; i++) st->gnt[i] = 0;
    if (st->nalive == 0) return;
    const unsigned long long mu = st->mn > st->level ? st->mn : st->level;
    st->level = mu;
    st->mn = st->mn_next;
    st->mn_next = ~0ull;
    st->nalive = st->nkeep;
    st->nkeep = st->nw = st->nb = 0;
    st->cpeel = 0;
    st->levels++;
    if (st->nalive == 0) st->t1 = globaltimer_ns();
}

__global__ void k_fdh_next(FdhDev *st) { fdh_close_level(st); }

// The same inside a graph's while-node: the loop goes on while members are
// alive (at most ni levels: every level peels at least one member).
__global__ void k_fdh_next_loop(FdhDev *st, int32_t ni, cudaGraphConditionalHandle cond) {
    fdh_close_level(st);
    cudaGraphSetConditional(cond, (st->nalive > 0 && st->levels < (unsigned long long)ni) ? 1u : 0u);
}

}  // namespace

// A graph and its executable, destroyed together.
struct GraphOwner {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t e = nullptr;
    ~GraphOwner() {
        if (e) cudaGraphExecDestroy(e);
        if (g) cudaGraphDestroy(g);
    }
};

// Levels of one heavy task one at a time, each deciding on the host between
// its updates and a recount of the task's alive members (hybrid update
// computation, Sec. 4.1): with D.fd_huc == 1 every level with updates
// recounts (test hook), otherwise a level whose peeled members' walks exceed
// D.huc_factor * rcnt does. Exact either way.
static void fdh_levels_with_recount(Decomp &D, const FdhArgs &ha, FdhDev *dst, FdhDev *hst_out,
                             uint64_t rcnt, int grid_h, size_t smem_h, int gm, cudaStream_t s) {
    const Side &S = *D.S;
    const Side &O = *D.O;
    const int32_t n = S.n;
    const int sms = num_sms();
    FdhDev *h = (FdhDev *)pinned_scratch(sizeof(FdhDev));
    DevBuf<int32_t> keep, adjc, lenc;
    DevBuf<unsigned long long> cnt0, cntr;
    bool have0 = false;
    // counts of the task's members (all, or the alive ones) inside G_i
    auto count_members = [&](int alive_only, unsigned long long *out) {
        if (!keep.get()) {
            keep.alloc(n, s);
            adjc.alloc(D.m, s);
            lenc.alloc(O.n, s);
        }
        keep.zero();
        k_fdh_keep<<<ceil_div(ha.ni, 256), 256, 0, s>>>(ha, keep.get(), alive_only);
        RC_LAUNCH();
        RC_CUDA(cudaMemcpyAsync(adjc.get(), O.adj, sizeof(int32_t) * D.m, cudaMemcpyDeviceToDevice, s));
        list_lengths(O.off, O.n, lenc.get(), s);
        compact_lists(O.off, lenc.get(), adjc.get(), O.n, keep.get(), s);
        return recount_masked(S, O, D.s, D.m, keep.get(), out, lenc.get(), adjc.get(), s);
    };
    for (;;) {
        k_fdh_select<<<gm, 256, 0, s>>>(ha);
        RC_LAUNCH();
        RC_CUDA(cudaMemcpyAsync(h, dst, sizeof(FdhDev), cudaMemcpyDeviceToHost, s));
        RC_CUDA(cudaStreamSynchronize(s));
        const bool updates = h->nw + h->nb > 0;
        const bool recount =
            updates && (D.fd_huc == 1 || (double)h->cpeel > D.huc_factor * (double)rcnt);
        if (recount) {
            if (!have0) {
                cnt0.alloc(n, s);
                cntr.alloc(n, s);
                D.wedges_fd_recount += count_members(0, cnt0.get());
                have0 = true;
            }
            D.wedges_fd_recount += count_members(1, cntr.get());
            k_fdh_apply<<<ceil_div(ha.ni, 256), 256, 0, s>>>(ha, cnt0.get(), cntr.get());
            RC_LAUNCH();
            D.fd_recounts++;
        } else {
            k_fdh_warp<<<sms * 8, 256, 0, s>>>(ha);
            RC_LAUNCH();
            k_fdh_cta<<<grid_h, FD_THREADS, smem_h, s>>>(ha);
            RC_LAUNCH();
            k_fdh_sweep<<<sms * 4, 256, 0, s>>>(ha, grid_h);
            RC_LAUNCH();
        }
        k_fdh_next<<<1, 1, 0, s>>>(dst);
        RC_LAUNCH();
        if (h->nkeep == 0) break;
    }
    RC_CUDA(cudaMemcpyAsync(hst_out, dst, sizeof(FdhDev), cudaMemcpyDeviceToHost, s));
}

void fd_run(Decomp &D, uint64_t *d_tip, cudaStream_t s) {
    const int32_t n = D.n;
    const int64_t m = D.m;
    const int32_t P = D.p_eff;
    if (n == 0 || P == 0) return;
    const Side &S = *D.S;
    const Side &O = *D.O;
    // members and ranks
    DevBuf<int32_t> cnt(P + 1, s), mstart(P + 1, s), members(n, s), rank(n, s);
    cnt.zero();
    {
        DevBuf<uint64_t> key(n, s);
        DevBuf<uint32_t> val(n, s);
        k_sub_keys<<<ceil_div(n, 256), 256, 0, s>>>(D.sub, n, key.get(), val.get(), cnt.get());
        RC_LAUNCH();
        radix_sort_pairs(key.get(), val.get(), n, 0, bits_for((uint64_t)P), s);
        scan_exclusive<int32_t>(cnt.get(), mstart.get(), P + 1, s);
        k_members<<<ceil_div(n, 256), 256, 0, s>>>(val.get(), n, D.sub, mstart.get(), members.get(),
                                                   rank.get());
        RC_LAUNCH();
    }
    // induced subgraphs
    DevBuf<int32_t> fd_adj(m, s), fd_len(m, s);
    DevBuf<int64_t> fd_beg(m, s), wpre;
    DevBuf<unsigned long long> wr(n, s);
    DevBuf<unsigned long long> wsub(P, s);
    wsub.zero();
    if (m > 0) {
        DevBuf<uint64_t> key(m, s);
        DevBuf<uint32_t> perm(m, s);
        k_edge_sub_keys<<<ceil_div(m, 256), 256, 0, s>>>(O.adj, m, D.sub, key.get(), perm.get());
        RC_LAUNCH();
        radix_sort_pairs(key.get(), perm.get(), m, 0, bits_for((uint64_t)P), s);
        key.release();
        DevBuf<int32_t> fd_y(m, s);
        DevBuf<uint32_t> head(m + 1, s), hpos(m + 1, s);
        k_fd_fill<<<ceil_div(m, 256), 256, 0, s>>>(perm.get(), m, O.adj, O.off, O.n, D.sub,
                                                   rank.get(), fd_adj.get(), fd_y.get(), head.get());
        RC_LAUNCH();
        RC_CUDA(cudaMemsetAsync(head.get() + m, 0, 4, s));
        scan_exclusive<uint32_t>(head.get(), hpos.get(), m + 1, s);
        uint32_t nruns = 0;
        RC_CUDA(cudaMemcpyAsync(&nruns, hpos.get() + m, 4, cudaMemcpyDeviceToHost, s));
        RC_CUDA(cudaStreamSynchronize(s));
        DevBuf<int64_t> run_start(nruns + 1, s);
        k_run_starts<<<ceil_div(m, 256), 256, 0, s>>>(head.get(), hpos.get(), m, run_start.get());
        RC_LAUNCH();
        k_fd_edges<<<ceil_div(m, 256), 256, 0, s>>>(perm.get(), m, O.adj, fd_y.get(), head.get(),
                                                    hpos.get(), run_start.get(), nruns, S.off, S.adj,
                                                    D.sub, fd_beg.get(), fd_len.get(), wsub.get());
        RC_LAUNCH();
        // walk sizes of all vertices: prefix sums of the run lengths (kept
        // for the split levels of heavy tasks)
        DevBuf<int64_t> l64(m + 1, s);
        wpre.alloc(m + 1, s);
        k_i32_to_i64<<<ceil_div(m, 256), 256, 0, s>>>(fd_len.get(), m, l64.get());
        RC_LAUNCH();
        RC_CUDA(cudaMemsetAsync(l64.get() + m, 0, sizeof(int64_t), s));
        scan_exclusive<int64_t>(l64.get(), wpre.get(), m + 1, s);
        k_fd_walk_sizes<<<ceil_div(n, 256), 256, 0, s>>>(S.off, n, wpre.get(), D.sub, mstart.get(),
                                                         rank.get(), wr.get());
        RC_LAUNCH();
    } else {
        wr.zero();
    }
    // subset sizes and wedge counts
    std::vector<int32_t> hms(P + 1);
    std::vector<unsigned long long> hw(P);
    RC_CUDA(cudaMemcpyAsync(hms.data(), mstart.get(), sizeof(int32_t) * (P + 1),
                            cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaMemcpyAsync(hw.data(), wsub.get(), 8 * P, cudaMemcpyDeviceToHost, s));
    // Tasks: a subset, or, in a batch's disjoint union, each packed graph's
    // part of a subset (parts share no butterfly, so each is peeled on its
    // own; consecutive small parts of one subset are merged up to TASK_MIN
    // members). A task covers consecutive member positions, which are
    // consecutive ranks of its subset.
    std::vector<int32_t> tstart, tlen, tkb, tsub;
    {
        const int ng = D.parts ? (int)D.parts->size() - 1 : 0;
        DevBuf<int64_t> dparts(ng > 0 ? ng + 1 : 1, s);
        if (ng > 0)
            RC_CUDA(cudaMemcpyAsync(dparts.get(), D.parts->data(), 8 * (ng + 1),
                                    cudaMemcpyHostToDevice, s));
        DevBuf<uint32_t> flag(n + 1, s), fpos(n + 1, s);
        k_task_flags<<<ceil_div(n, 256), 256, 0, s>>>(members.get(), n, D.sub, mstart.get(),
                                                      dparts.get(), ng, flag.get());
        RC_LAUNCH();
        RC_CUDA(cudaMemsetAsync(flag.get() + n, 0, 4, s));
        scan_exclusive<uint32_t>(flag.get(), fpos.get(), n + 1, s);
        uint32_t nseg = 0;
        RC_CUDA(cudaMemcpyAsync(&nseg, fpos.get() + n, 4, cudaMemcpyDeviceToHost, s));
        RC_CUDA(cudaStreamSynchronize(s));
        DevBuf<int32_t> segs(nseg > 0 ? nseg : 1, s);
        k_flag_positions<<<ceil_div(n, 256), 256, 0, s>>>(flag.get(), fpos.get(), n, segs.get());
        RC_LAUNCH();
        std::vector<int32_t> hseg(nseg);
        if (nseg > 0)
            RC_CUDA(cudaMemcpyAsync(hseg.data(), segs.get(), 4 * (size_t)nseg,
                                    cudaMemcpyDeviceToHost, s));
        RC_CUDA(cudaStreamSynchronize(s));
        int sub_i = 0;
        for (uint32_t k = 0; k < nseg; k++) {
            const int32_t b = hseg[k];
            while (sub_i + 1 <= P && hms[sub_i + 1] <= b) sub_i++;  // subset holding b
            const bool new_sub = tsub.empty() || tsub.back() != sub_i;
            if (new_sub || tlen.back() >= TASK_MIN) {
                tstart.push_back(b);
                tlen.push_back(0);
                tkb.push_back(b - hms[sub_i]);
                tsub.push_back(sub_i);
            }
            const int32_t e = k + 1 < nseg ? hseg[k + 1] : n;
            tlen.back() += e - b;
        }
    }
    const int T = (int)tstart.size();
    // task weights: walk sizes summed over the task's members (LPT key)
    std::vector<unsigned long long> tw(T);
    DevBuf<int32_t> d_tstart(T > 0 ? T : 1, s), d_tlen(T > 0 ? T : 1, s), d_tkb(T > 0 ? T : 1, s);
    if (T > 0) {
        RC_CUDA(cudaMemcpyAsync(d_tstart.get(), tstart.data(), 4 * (size_t)T, cudaMemcpyHostToDevice, s));
        RC_CUDA(cudaMemcpyAsync(d_tlen.get(), tlen.data(), 4 * (size_t)T, cudaMemcpyHostToDevice, s));
        RC_CUDA(cudaMemcpyAsync(d_tkb.get(), tkb.data(), 4 * (size_t)T, cudaMemcpyHostToDevice, s));
        DevBuf<int64_t> w64(n + 1, s), cw(n + 1, s);
        DevBuf<unsigned long long> dtw(T, s);
        k_walk_plain<<<ceil_div(n, 256), 256, 0, s>>>(wr.get(), n, w64.get());
        RC_LAUNCH();
        RC_CUDA(cudaMemsetAsync(w64.get() + n, 0, 8, s));
        scan_exclusive<int64_t>(w64.get(), cw.get(), n + 1, s);
        k_task_weights<<<ceil_div(T, 256), 256, 0, s>>>(d_tstart.get(), d_tlen.get(), cw.get(), T,
                                                        dtw.get());
        RC_LAUNCH();
        RC_CUDA(cudaMemcpyAsync(tw.data(), dtw.get(), 8 * (size_t)T, cudaMemcpyDeviceToHost, s));
        RC_CUDA(cudaStreamSynchronize(s));
    }
    // LPT order (ties by task id). A task's time is its walks plus its
    // levels, each level a chain of dependent steps inside one CTA; levels
    // are at most its members, so a member counts as LEVEL_WEDGES wedges.
    std::vector<int32_t> hq(T);
    for (int k = 0; k < T; k++) hq[k] = k;
    std::stable_sort(hq.begin(), hq.end(), [&](int32_t x, int32_t y) {
        const unsigned long long kx = tw[x] + LEVEL_WEDGES * (unsigned long long)tlen[x];
        const unsigned long long ky = tw[y] + LEVEL_WEDGES * (unsigned long long)tlen[y];
        return kx > ky;
    });
    const size_t warp_tables = (size_t)(FD_THREADS / 32) * WARP_SLOTS * 8 + 16;
    const size_t smem = FdEngine::bytes() + CHUNK_BYTES + warp_tables;
    allow_max_smem((const void *)k_fd_peel);
    int occ = 0;
    RC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fd_peel, FD_THREADS, smem));
    const int sms = num_sms();
    const int grid_all = sms * std::max(occ, 1);
    // Heavy tasks (peeled first by all CTAs): task weight at least the
    // threshold. Automatic: HEAVY_SHARE times the total weight divided by
    // min(CTAs, tasks), and at least HEAVY_MIN_W; with at most half as many
    // tasks as CTAs (most CTAs would idle) the divisor is the CTA count.
    int nheavy = 0;
    if (D.fd_heavy_w >= 0 && T > 0) {
        unsigned long long thr = (unsigned long long)D.fd_heavy_w;
        if (D.fd_heavy_w == 0) {
            unsigned long long tot = 0;
            for (int k = 0; k < T; k++) tot += tw[k];
            const int div = 2 * T <= grid_all ? grid_all : std::min(grid_all, T);
            thr = std::max<unsigned long long>(HEAVY_MIN_W,
                                               tot / (unsigned long long)div * HEAVY_SHARE);
        }
        // Automatic rule, second part: a task above one CTA's share of the
        // LPT weight whose walks outweigh its levels several times over (its
        // one-CTA peel is walk-bound, and split levels spread the walks over
        // every CTA)
        unsigned long long share = ~0ull;
        if (D.fd_heavy_w == 0) {
            unsigned long long totk = 0;
            for (int k = 0; k < T; k++) totk += tw[k] + LEVEL_WEDGES * (unsigned long long)tlen[k];
            share = totk / (unsigned long long)grid_all;
        }
        std::vector<int32_t> front, back;
        for (int k = 0; k < T; k++) {
            const int32_t t = hq[k];
            const unsigned long long lw = LEVEL_WEDGES * (unsigned long long)tlen[t];
            const bool walk_bound = tw[t] + lw >= share && tw[t] >= HEAVY_WALK_LEVELS * lw;
            ((tw[t] >= thr || walk_bound) && tlen[t] > 0 ? front : back).push_back(t);
        }
        nheavy = (int)front.size();
        int pos = 0;
        for (int32_t t : front) hq[pos++] = t;
        for (int32_t t : back) hq[pos++] = t;
    }
    DevBuf<int32_t> queue(T > 0 ? T : 1, s);
    if (T > 0)
        RC_CUDA(cudaMemcpyAsync(queue.get(), hq.data(), 4 * (size_t)T, cudaMemcpyHostToDevice, s));
    DevBuf<unsigned long long> fsup(n, s);
    DevBuf<uint8_t> alive(n, s);
    DevBuf<int32_t> alist(n, s), alist2(n, s), clist(n, s), clist2(n, s), plist(n, s), blist(n, s),
        qhead(1, s);
    DevBuf<unsigned long long> stats(2, s), sub_ns(T > 0 ? T : 1, s), sub_lv(T > 0 ? T : 1, s);
    qhead.zero();
    stats.zero();
    sub_ns.zero();
    sub_lv.zero();
    D.fd_heavy = nheavy;
    D.fd_heavy_ms = 0;
    D.fd_heavy_levels = 0;
    D.fd_split_levels = 0;
    std::vector<FdhDev> hh(nheavy);
    if (nheavy > 0) {
        DevBuf<FdhDev> hst(1, s);
        const size_t smem_h = FdEngine::bytes() + CHUNK_BYTES;
        allow_max_smem((const void *)k_fdh_cta);
        int occ_h = 0;
        RC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_h, k_fdh_cta, FD_THREADS, smem_h));
        const int grid_h = sms * std::max(occ_h, 1);
        // global counters of split levels, sized for the largest heavy task
        int32_t ni_max = 1;
        for (int h = 0; h < nheavy; h++) ni_max = std::max(ni_max, tlen[hq[h]]);
        DevBuf<uint32_t> gcnt((size_t)FDH_SPLIT_NB * ni_max, s);
        DevBuf<int32_t> gtl((size_t)FDH_SPLIT_NB * ni_max, s);
        gcnt.zero();
        for (int h = 0; h < nheavy; h++) {
            const int32_t i = hq[h];
            const int32_t mb = tstart[i], ni = tlen[i];
            FdhArgs ha{members.get() + mb, ni,           tkb[i],         S.off,
                       fd_beg.get(),       fd_len.get(), fd_adj.get(),   S.new2old,
                       D.init,             fsup.get() + mb, alive.get() + mb, wr.get() + mb,
                       plist.get() + mb,   blist.get() + mb, (unsigned long long *)d_tip,
                       hst.get(),          gcnt.get(),   gtl.get(),      wpre.get()};
            const int gm = std::max(1, std::min(ceil_div(ni, 256), sms * 4));
            const int gi = std::max(1, std::min(ceil_div((int64_t)ni * 32, 256), sms * 16));
            k_fdh_reset<<<1, 1, 0, s>>>(hst.get(), ni);
            RC_LAUNCH();
            k_fdh_init<<<gi, 256, 0, s>>>(ha);
            RC_LAUNCH();
            // Recount rule (Sec. 4.1) of this task: a level recounts when its
            // peeled members' walks exceed factor * C_rcnt of the task; no
            // level can when the task's whole walk weight does not.
            bool may_recount = D.fd_huc == 1;
            uint64_t rcnt = 0;
            if (D.fd_huc == 0) {
                k_fdh_rcnt<<<gi, 256, 0, s>>>(ha);
                RC_LAUNCH();
                RC_CUDA(cudaMemcpyAsync(&hh[h], hst.get(), sizeof(FdhDev), cudaMemcpyDeviceToHost, s));
                RC_CUDA(cudaStreamSynchronize(s));
                rcnt = hh[h].rcnt;
                may_recount = rcnt > 0 && (double)tw[i] > D.huc_factor * (double)rcnt;
            }
            // the levels in one graph launch: a while-node repeats select,
            // updates, sweep and close while members are alive
            GraphOwner lg;
            if (!may_recount) {
                RC_CUDA(cudaGraphCreate(&lg.g, 0));
                cudaGraphConditionalHandle cond;
                RC_CUDA(cudaGraphConditionalHandleCreate(&cond, lg.g, 1, cudaGraphCondAssignDefault));
                cudaGraphNodeParams np{};
                np.type = cudaGraphNodeTypeConditional;
                np.conditional.handle = cond;
                np.conditional.type = cudaGraphCondTypeWhile;
                np.conditional.size = 1;
                cudaGraphNode_t wnode;
                RC_CUDA(cudaGraphAddNode(&wnode, lg.g, nullptr, nullptr, 0, &np));
                cudaGraph_t body = np.conditional.phGraph_out[0];
                cudaStream_t cs = aux_stream();
                RC_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeThreadLocal));
                k_fdh_select<<<gm, 256, 0, cs>>>(ha);
                RC_LAUNCH();
                k_fdh_warp<<<sms * 8, 256, 0, cs>>>(ha);
                RC_LAUNCH();
                k_fdh_cta<<<grid_h, FD_THREADS, smem_h, cs>>>(ha);
                RC_LAUNCH();
                k_fdh_sweep<<<sms * 4, 256, 0, cs>>>(ha, grid_h);
                RC_LAUNCH();
                k_fdh_next_loop<<<1, 1, 0, cs>>>(hst.get(), ni, cond);
                RC_LAUNCH();
                RC_CUDA(cudaStreamEndCapture(cs, &body));
                uncount_launches(5);  // counted per level below
                RC_CUDA(cudaGraphInstantiate(&lg.e, lg.g, 0));
                RC_CUDA(cudaGraphLaunch(lg.e, s));
            } else {
                fdh_levels_with_recount(D, ha, hst.get(), &hh[h], rcnt, grid_h, smem_h, gm, s);
            }
            RC_CUDA(cudaMemcpyAsync(&hh[h], hst.get(), sizeof(FdhDev), cudaMemcpyDeviceToHost, s));
            RC_CUDA(cudaStreamSynchronize(s));
            if (!may_recount) count_launches(5 * (uint64_t)hh[h].levels);
            D.fd_heavy_ms += (float)((hh[h].t1 - hh[h].t0) * 1e-6);
            D.fd_heavy_levels += (int64_t)hh[h].levels;
            D.fd_split_levels += (int64_t)hh[h].splits;
        }
        RC_CUDA(cudaMemcpyAsync(qhead.get(), &nheavy, 4, cudaMemcpyHostToDevice, s));
    }
    if (nheavy < T) {
        const int grid = std::max(1, std::min(grid_all, T - nheavy));
        FdArgs a{queue.get(),   T,           qhead.get(),     d_tstart.get(), d_tlen.get(),
                 d_tkb.get(),   members.get(),
                 S.off,         fd_beg.get(), fd_len.get(),   fd_adj.get(), S.new2old,
                 D.init,        fsup.get(),  alive.get(),     alist.get(),  alist2.get(),
                 clist.get(),   clist2.get(),
                 plist.get(),   blist.get(),
                 (unsigned long long *)d_tip, stats.get(),    sub_ns.get(), sub_lv.get(),
                 wr.get()};
        k_fd_peel<<<grid, FD_THREADS, smem, s>>>(a);
        RC_LAUNCH();
    }
    unsigned long long hs[2] = {0, 0};
    RC_CUDA(cudaMemcpyAsync(hs, stats.get(), sizeof(hs), cudaMemcpyDeviceToHost, s));
    std::vector<unsigned long long> hns(T), hlv(T);
    if (T > 0) {
        RC_CUDA(cudaMemcpyAsync(hns.data(), sub_ns.get(), 8 * (size_t)T, cudaMemcpyDeviceToHost, s));
        RC_CUDA(cudaMemcpyAsync(hlv.data(), sub_lv.get(), 8 * (size_t)T, cudaMemcpyDeviceToHost, s));
    }
    RC_CUDA(cudaStreamSynchronize(s));
    D.wedges_fd = hs[0];
    D.levels = (int64_t)hs[1];
    std::vector<bool> heavy(T, false);
    for (int h = 0; h < nheavy; h++) {
        const int32_t t = hq[h];
        heavy[t] = true;
        hns[t] = hh[h].t1 - hh[h].t0;
        hlv[t] = hh[h].levels;
        D.wedges_fd += hh[h].wedges;
        D.levels += (int64_t)hh[h].levels;
    }
    // per subset: its tasks' levels and device time summed
    D.subsets.assign(P, receipt_subset{});
    for (int i = 0; i < P; i++) {
        D.subsets[i].n = hms[i + 1] - hms[i];
        D.subsets[i].wedges_est = hw[i];
    }
    int worst = -1;
    for (int t = 0; t < T; t++) {
        receipt_subset &r = D.subsets[tsub[t]];
        r.levels += (int64_t)hlv[t];
        r.ms += (float)(hns[t] * 1e-6);
        if (heavy[t]) r.heavy = 1;
        if (!heavy[t] && (worst < 0 || hns[t] > hns[worst])) worst = t;
    }
    // slowest task peeled by one CTA
    D.fd_max_ms = worst >= 0 ? (float)(hns[worst] * 1e-6) : 0.f;
    D.fd_max_n = worst >= 0 ? tlen[worst] : 0;
    D.fd_max_levels = worst >= 0 ? (int64_t)hlv[worst] : 0;
    D.fd_tasks = T;
}

}  // namespace receipt
