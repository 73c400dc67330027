// Wedge aggregation engines shared by counting (Algorithm 1), the batched
// peel update of the coarse-grained pass (Algorithm 3 calling the update of
// Algorithm 2) and the fine-grained peel (Algorithm 4).
//
// All three walk, for one anchor vertex a, a list of "middle" vertices and
// for each of them a segment of end points, and need c(e) = the number of
// wedges from a to every distinct end point e. The paper keeps a per-thread
// dense array of |W| counters (Algorithm 1, wdg_arr) or a hashmap
// (Algorithm 2). On GB300 the aggregation lives in shared memory:
//
//  * WarpHash   -- one warp per anchor, a warp-private open-addressing table
//                  (anchors with at most WARP_MAX_W wedges);
//  * CtaHybrid  -- one CTA per anchor. End points below `head` (low labels =
//                  high degree, where repeated end points concentrate) get
//                  dense 16-bit counters; the rest first set a bit in a
//                  bitmap and only a repeat goes to a small hash table of
//                  (key, extra count). Overflow of that table aborts the
//                  anchor before anything is emitted, and the anchor is redone
//                  by the global engine;
//  * GlobalDense -- one CTA per anchor with a dense counter array and a
//                  touched list in global memory (per-CTA slot), for hubs
//                  and for key spaces too large for shared memory.
#pragma once

#include "common.cuh"

namespace receipt {

constexpr int32_t EMPTY_KEY = -1;
constexpr int WARP_MAX_W = 256;     // wedges of a warp-tier anchor
constexpr int WARP_SLOTS = 512;     // per-warp table (load factor <= 1/2)
constexpr int CTA_THREADS = 1024;
constexpr int SLICE_THREADS = 1024; // CTAs of the key-sliced tier (one per SM)
constexpr int DENSE_THREADS = 512;  // CTAs of the dense-window tier (two per SM)
constexpr int MID_CHUNK = CTA_THREADS;
constexpr int REPEAT_SLOTS = 4096;  // CtaHybrid repeat table
constexpr int REPEAT_LIMIT = REPEAT_SLOTS / 2;
constexpr int HEAD_MAX = 16384;     // dense 16-bit counters for keys < head
constexpr int HEAD_SLICE = 2048;    // head of the key slices after the first
constexpr int SLICE_MIN_W = 49152;  // anchors with more wedges use the sliced tier
constexpr int MAX_PROBE = 64;
constexpr int WALK_UNROLL = 8;     // independent loads in flight per warp in cta_walk

__device__ __forceinline__ uint32_t hash_key(int32_t k) {
    return (uint32_t)k * 2654435761u;
}

// Log-spaced buckets of 64-bit values: 32 exact values, then 32 mantissa
// steps per power of two (58 octaves); a bucket's top is within 3% of its
// bottom.
constexpr int LOG_BUCKETS = 1920;
__device__ __forceinline__ int log_bucket_of(unsigned long long k) {
    if (k < 32) return (int)k;
    const int e = 63 - __clzll((long long)k);
    const int mant = (int)((k >> (e - 5)) & 31);
    return 32 + (e - 5) * 32 + mant;
}
__device__ __forceinline__ unsigned long long log_bucket_top(int b) {
    if (b < 32) return (unsigned long long)b;
    const int e = (b - 32) / 32 + 5, mant = (b - 32) % 32;
    if (e == 63 && mant == 31) return ~0ull;
    return ((unsigned long long)(33 + mant) << (e - 5)) - 1ull;
}

// Visits of one walk step (key < 0: no wedge). A visitor with a many<N>()
// member gets the whole step with all 32 lanes (for warp-level aggregation);
// others get one call per key.
template <int N, class V>
__device__ __forceinline__ auto visit_many_impl(V &v, const int (&kk)[N], const int32_t (&key)[N],
                                                int) -> decltype(v.template many<N>(kk, key), void()) {
    v.template many<N>(kk, key);
}
template <int N, class V>
__device__ __forceinline__ void visit_many_impl(V &v, const int (&kk)[N], const int32_t (&key)[N],
                                                long) {
#pragma unroll
    for (int u = 0; u < N; u++)
        if (key[u] >= 0) v(kk[u], key[u]);
}
template <int N, class V>
__device__ __forceinline__ void visit_many(V &v, const int (&kk)[N], const int32_t (&key)[N]) {
    visit_many_impl<N>(v, kk, key, 0);
}

// Emits of up to N (key, count) pairs (key < 0: none). An emitter with a
// many<N>() member gets them together (to overlap their memory operations);
// others get one call per pair.
template <int N, class E>
__device__ __forceinline__ auto emit_many_impl(E &e, const int32_t (&k)[N], const uint32_t (&c)[N],
                                               int) -> decltype(e.template many<N>(k, c), void()) {
    e.template many<N>(k, c);
}
template <int N, class E>
__device__ __forceinline__ void emit_many_impl(E &e, const int32_t (&k)[N], const uint32_t (&c)[N],
                                               long) {
#pragma unroll
    for (int u = 0; u < N; u++)
        if (k[u] >= 0) e(k[u], c[u]);
}
template <int N, class E>
__device__ __forceinline__ void emit_many(E &e, const int32_t (&k)[N], const uint32_t (&c)[N]) {
    emit_many_impl<N>(e, k, c, 0);
}

// Walks the segments of the middle vertices q in [q0, q1) with one warp, 32
// middle vertices at a time: lane i fetches segment i, a warp scan of the
// lengths numbers their wedges, and each lane takes wedges lane, lane + 32,
// ..., finding its segment by a binary search over the lanes' starts, so all
// key loads of a step are independent (U per lane in flight). visit(key).
template <int U, class Mids, class Visit>
__device__ __forceinline__ void warp_walk(const Mids &M, int64_t q0, int64_t q1,
                                          const int32_t *__restrict__ keys, Visit &visit) {
    const int lane = threadIdx.x & 31;
    for (int64_t qb = q0; qb < q1; qb += 32) {
        int64_t beg = 0;
        int32_t len = 0;
        if (qb + lane < q1) M.seg(qb + lane, beg, len);
        int32_t inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const int32_t total = __shfl_sync(0xffffffffu, inc, 31);
        const int32_t ex = inc - len;
        for (int32_t j0 = 0; j0 < total; j0 += 32 * U) {
            int32_t key[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int32_t j = j0 + u * 32 + lane;
                // last lane whose segment starts at or before j (all lanes
                // take part in the shuffles)
                int lo = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int32_t e = __shfl_sync(0xffffffffu, ex, lo + step);
                    if (e <= j) lo += step;
                }
                const int64_t b = __shfl_sync(0xffffffffu, beg, lo);
                const int32_t e0 = __shfl_sync(0xffffffffu, ex, lo);
                key[u] = j < total ? __ldg(keys + b + (j - e0)) : -1;
            }
#pragma unroll
            for (int u = 0; u < U; u++)
                if (key[u] >= 0) visit(key[u]);
        }
    }
}

// ------------------------------------------------------------------
// Warp-private table
// ------------------------------------------------------------------
struct WarpHash {
    int32_t *key;   // WARP_SLOTS
    uint32_t *val;  // WARP_SLOTS

    __device__ void clear(int lane) {
        for (int i = lane; i < WARP_SLOTS; i += 32) {
            key[i] = EMPTY_KEY;
            val[i] = 0;
        }
    }
    // Returns false if the probe ran out (cannot happen at load <= 1/2).
    __device__ bool add(int32_t k) {
        uint32_t h = hash_key(k) & (WARP_SLOTS - 1);
        for (int p = 0; p < WARP_SLOTS; p++) {
            int32_t cur = ((volatile int32_t *)key)[h];
            if (cur == k) {
                atomicAdd(&val[h], 1u);
                return true;
            }
            if (cur == EMPTY_KEY) {
                int32_t prev = atomicCAS(&key[h], EMPTY_KEY, k);
                if (prev == EMPTY_KEY || prev == k) {
                    atomicAdd(&val[h], 1u);
                    return true;
                }
            }
            h = (h + 1) & (WARP_SLOTS - 1);
        }
        return false;
    }
    // emit(key, count) for every key with count >= 2, 8 slots per lane at a
    // time (emits overlapped), and clears the table. One warp.
    template <class Emit>
    __device__ __forceinline__ void flush_clear(Emit &emit, int lane) {
        for (int s0 = 0; s0 < WARP_SLOTS; s0 += 32 * 8) {
            int32_t kk[8];
            uint32_t cc[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int sl = s0 + u * 32 + lane;
                const int32_t k = key[sl];
                const uint32_t c = val[sl];
                kk[u] = (k != EMPTY_KEY && c >= 2) ? k : -1;
                cc[u] = c;
                if (k != EMPTY_KEY) {
                    key[sl] = EMPTY_KEY;
                    val[sl] = 0;
                }
            }
            emit_many<8>(emit, kk, cc);
        }
    }
    __device__ uint32_t lookup(int32_t k) const {
        uint32_t h = hash_key(k) & (WARP_SLOTS - 1);
        for (int p = 0; p < WARP_SLOTS; p++) {
            int32_t cur = key[h];
            if (cur == k) return val[h];
            if (cur == EMPTY_KEY) return 0;
            h = (h + 1) & (WARP_SLOTS - 1);
        }
        return 0;
    }
};

// ------------------------------------------------------------------
// CTA hash: open addressing over any key space, for anchors with few wedges
// ------------------------------------------------------------------
// SLOTS (key, count) pairs at load <= 1/2: an anchor with at most SLOTS / 2
// wedges always finds room (it cannot touch more distinct keys). Every slot
// taken is listed, so flushing and clearing cost what the anchor touched.
template <int SLOTS>
struct CtaHashT {
    static_assert((SLOTS & (SLOTS - 1)) == 0 && SLOTS <= 65536, "slots");
    int32_t *key;   // SLOTS
    uint32_t *val;  // SLOTS
    uint16_t *tl;   // SLOTS / 2: slots taken
    int *s_nt;      // shared scalar: slots taken

    static constexpr size_t bytes() { return (size_t)SLOTS * 8 + (size_t)SLOTS; }
    __device__ unsigned char *bind(unsigned char *base, int *nt) {
        key = (int32_t *)base;
        val = (uint32_t *)(key + SLOTS);
        tl = (uint16_t *)(val + SLOTS);
        s_nt = nt;
        return base + bytes();
    }
    __device__ void clear_all() {
        for (int i = threadIdx.x; i < SLOTS; i += blockDim.x) {
            key[i] = EMPTY_KEY;
            val[i] = 0;
        }
        if (threadIdx.x == 0) *s_nt = 0;
    }
    __device__ __forceinline__ void add(int32_t k) {
        uint32_t h = hash_key(k) & (SLOTS - 1);
        for (int p = 0; p < SLOTS; p++) {
            const int32_t cur = ((volatile int32_t *)key)[h];
            if (cur == k) {
                atomicAdd(&val[h], 1u);
                return;
            }
            if (cur == EMPTY_KEY) {
                const int32_t prev = atomicCAS(&key[h], EMPTY_KEY, k);
                if (prev == EMPTY_KEY) {
                    atomicAdd(&val[h], 1u);
                    tl[atomicAdd(s_nt, 1)] = (uint16_t)h;
                    return;
                }
                if (prev == k) {
                    atomicAdd(&val[h], 1u);
                    return;
                }
            }
            h = (h + 1) & (SLOTS - 1);
        }
    }
    __device__ __forceinline__ uint32_t count(int32_t k) const {
        uint32_t h = hash_key(k) & (SLOTS - 1);
        for (int p = 0; p < SLOTS; p++) {
            const int32_t cur = key[h];
            if (cur == k) return val[h];
            if (cur == EMPTY_KEY) return 0;
            h = (h + 1) & (SLOTS - 1);
        }
        return 0;
    }
    // EMIT: emit(key, count) for every key with count >= 2; CLEAR: empty the
    // slots taken. The caller synchronises afterwards, then reset_scalars().
    template <bool EMIT, bool CLEAR, class Emit>
    __device__ void sweep(Emit &emit) {
        const int nt = *(volatile int *)s_nt;
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
            const int h = tl[i];
            if (EMIT) {
                const uint32_t c = val[h];
                if (c >= 2) emit(key[h], c);
            }
            if (CLEAR) {
                key[h] = EMPTY_KEY;
                val[h] = 0;
            }
        }
    }
    __device__ void reset_scalars() {
        if (threadIdx.x == 0) *s_nt = 0;
    }
};

// ------------------------------------------------------------------
// CTA hybrid: dense head counters + tail bitmap + repeat table
// ------------------------------------------------------------------
// Keys below `headn` (low labels = high degree, where repeated end points
// concentrate) have 16-bit counters, two per word: key k < hw sits in the low
// half of word k, key k >= hw in the high half of word k - hw, so consecutive
// keys land in different words (no same-address atomics within a warp).
// Keys from headn on set a bit in a bitmap; a bit found already set sends the
// key to a small open-addressing table of extra occurrences; every repeat slot
// taken is listed, so the table is flushed and cleared in time proportional
// to its use. The head is swept one word per thread and step; the bitmap is
// cleared with 16-byte stores over the key range in use.
struct CtaHybrid {
    uint32_t *head;   // head_cap/2 words
    uint32_t *hsum;   // reserved (keeps the layout 16-byte aligned)
    uint32_t *bm;     // bm_cap words over keys [headn, headn + 32 * bm_cap)
    uint32_t *tsum;   // reserved
    int32_t *rkey;    // REPEAT_SLOTS
    uint32_t *rval;   // REPEAT_SLOTS: extra occurrences (count - 1)
    int32_t *rlist;   // REPEAT_LIMIT + 1: slots taken, in order
    int *s_used;      // shared scalar: repeat slots taken
    int *s_over;      // shared scalar: repeat table overflowed
    int32_t headn;    // keys with dense counters (<= head_cap)
    int32_t hw;       // (headn + 1) / 2
    int32_t act_bw;   // bitmap words the current key range can touch
    int32_t head_cap; // capacity in keys
    int32_t bm_cap;   // capacity in bitmap words

    __host__ __device__ static int32_t pad4(int64_t w) { return (int32_t)((w + 3) & ~3ll); }
    __host__ __device__ static size_t bytes(int32_t head_cap, int32_t bm_cap) {
        int32_t hwc = pad4((head_cap + 1) / 2), hs = pad4((hwc + 31) / 32);
        int32_t bmc = pad4(bm_cap), ts = pad4((bmc + 31) / 32);
        return (size_t)4 * (hwc + hs + bmc + ts) + (size_t)REPEAT_SLOTS * 8 +
               (size_t)(REPEAT_LIMIT + 4) * 4;
    }
    // Lays the engine out from `base` (16-byte aligned); returns the end.
    __device__ unsigned char *bind(unsigned char *base, int32_t hcap, int32_t bcap, int *used,
                                   int *over) {
        head_cap = hcap;
        bm_cap = pad4(bcap);
        int32_t hwc = pad4((hcap + 1) / 2), hs = pad4((hwc + 31) / 32);
        int32_t ts = pad4((bm_cap + 31) / 32);
        head = (uint32_t *)base;
        hsum = head + hwc;
        bm = hsum + hs;
        tsum = bm + bm_cap;
        rkey = (int32_t *)(tsum + ts);
        rval = (uint32_t *)(rkey + REPEAT_SLOTS);
        rlist = (int32_t *)(rval + REPEAT_SLOTS);
        s_used = used;
        s_over = over;
        set_range(hcap, (int64_t)hcap + 32 * (int64_t)bm_cap);
        return (unsigned char *)(rlist + REPEAT_LIMIT + 4);
    }
    // Current key range [0, keys) with dense counters for the first h keys.
    __device__ void set_range(int32_t h, int64_t keys) {
        headn = h;
        hw = (h + 1) >> 1;
        int64_t t = keys - h;
        act_bw = t > 0 ? (int32_t)imin64((t + 31) >> 5, bm_cap) : 0;
    }
    // Zeroes everything (once per kernel).
    __device__ void clear_all() {
        int32_t hwc = pad4((head_cap + 1) / 2), hs = pad4((hwc + 31) / 32);
        int32_t ts = pad4((bm_cap + 31) / 32);
        uint32_t *w0 = head;
        int32_t nw = hwc + hs + bm_cap + ts;
        for (int i = threadIdx.x; i < nw; i += blockDim.x) w0[i] = 0;
        for (int i = threadIdx.x; i < REPEAT_SLOTS; i += blockDim.x) {
            rkey[i] = EMPTY_KEY;
            rval[i] = 0;
        }
        if (threadIdx.x == 0) {
            *s_used = 0;
            *s_over = 0;
        }
    }
    __device__ __forceinline__ void add(int32_t k) {
        if (k < headn) {
            const bool hi = k >= hw;
            const int32_t w = hi ? k - hw : k;
            atomicAdd(&head[w], hi ? 0x10000u : 1u);
            return;
        }
        const int32_t t = k - headn;
        const uint32_t bit = 1u << (t & 31);
        uint32_t old = atomicOr(&bm[t >> 5], bit);
        if (old & bit) add_repeat(k);
    }
    __device__ void add_repeat(int32_t k) {
        if (*(volatile int *)s_over) return;
        uint32_t h = hash_key(k) & (REPEAT_SLOTS - 1);
        for (int p = 0; p < MAX_PROBE; p++) {
            int32_t cur = ((volatile int32_t *)rkey)[h];
            if (cur == k) {
                atomicAdd(&rval[h], 1u);
                return;
            }
            if (cur == EMPTY_KEY) {
                int32_t prev = atomicCAS(&rkey[h], EMPTY_KEY, k);
                if (prev == EMPTY_KEY) {
                    atomicAdd(&rval[h], 1u);
                    int pos = atomicAdd(s_used, 1);
                    if (pos < REPEAT_LIMIT)
                        rlist[pos] = (int32_t)h;
                    else
                        *(volatile int *)s_over = 1;
                    return;
                }
                if (prev == k) {
                    atomicAdd(&rval[h], 1u);
                    return;
                }
            }
            h = (h + 1) & (REPEAT_SLOTS - 1);
        }
        *(volatile int *)s_over = 1;
    }
    // Count of key k after aggregation (a key >= headn must have been added).
    __device__ __forceinline__ uint32_t count(int32_t k) const {
        if (k < headn) {
            const bool hi = k >= hw;
            return (head[hi ? k - hw : k] >> (hi ? 16 : 0)) & 0xffffu;
        }
        uint32_t h = hash_key(k) & (REPEAT_SLOTS - 1);
        for (int p = 0; p < MAX_PROBE; p++) {
            int32_t cur = rkey[h];
            if (cur == k) return 1u + rval[h];
            if (cur == EMPTY_KEY) return 1u;
            h = (h + 1) & (REPEAT_SLOTS - 1);
        }
        return 1u;
    }
    // Visits what the anchor touched: EMIT calls emit(key, count) for every
    // key with count >= 2 (only valid without overflow); CLEAR returns the
    // touched words and slots to zero. All threads call it; the caller
    // synchronises afterwards, and after a CLEAR calls reset_scalars().
    template <bool EMIT, bool CLEAR, class Emit>
    __device__ void sweep(Emit &emit) {
        const int used = *(volatile int *)s_used;
        const int over = *(volatile int *)s_over;
        // head: words [0, hw), one per thread and step, so that the hot low
        // keys (the window's highest-degree vertices) and their emits are
        // spread over all threads
        for (int w = threadIdx.x; w < hw; w += blockDim.x) {
            const uint32_t v = head[w];
            if (v == 0) continue;
            if (CLEAR) head[w] = 0;
            if (EMIT) {
                const uint32_t c0 = v & 0xffffu, c1 = v >> 16;
                if (c0 >= 2) emit(w, c0);
                if (c1 >= 2) emit(w + hw, c1);
            }
        }
        // tail bitmap: the words the current key range can use
        if (CLEAR) {
            const int bw4 = (act_bw + 3) >> 2;
            for (int i = threadIdx.x; i < bw4; i += blockDim.x)
                ((uint4 *)bm)[i] = make_uint4(0, 0, 0, 0);
        }
        if (over) {
            if (CLEAR)
                for (int i = threadIdx.x; i < REPEAT_SLOTS; i += blockDim.x) {
                    rkey[i] = EMPTY_KEY;
                    rval[i] = 0;
                }
        } else {
            const int nl = used < REPEAT_LIMIT ? used : REPEAT_LIMIT;
            for (int i = threadIdx.x; i < nl; i += blockDim.x) {
                const int32_t h = rlist[i];
                if (EMIT) emit(rkey[h], 1u + rval[h]);
                if (CLEAR) {
                    rkey[h] = EMPTY_KEY;
                    rval[h] = 0;
                }
            }
        }
    }
    template <bool EMIT, class Emit>
    __device__ void flush_clear(Emit &emit) {
        sweep<EMIT, true>(emit);
    }
    __device__ void reset_scalars() {
        if (threadIdx.x == 0) {
            *s_used = 0;
            *s_over = 0;
        }
    }
};

struct NoEmit {
    __device__ void operator()(int32_t, uint32_t) {}
};

// Head and bitmap capacities for a key space (head = the first
// min(keyspace, HEAD_MAX) keys).
inline void hybrid_caps(int64_t keyspace, int32_t *head_cap, int32_t *bm_cap) {
    int64_t h = keyspace < HEAD_MAX ? keyspace : HEAD_MAX;
    int64_t tail = keyspace - h;
    *head_cap = (int32_t)h;
    *bm_cap = (int32_t)((tail + 31) / 32);
}

// shared-memory bytes of a CtaHybrid for a key space
inline size_t hybrid_bytes(int64_t keyspace, int32_t *head_cap_out = nullptr,
                           int32_t *bm_cap_out = nullptr) {
    int32_t hc, bc;
    hybrid_caps(keyspace, &hc, &bc);
    if (head_cap_out) *head_cap_out = hc;
    if (bm_cap_out) *bm_cap_out = bc;
    return CtaHybrid::bytes(hc, bc);
}

// ------------------------------------------------------------------
// Dense slice: 16-bit counters for every key of one key slice
// ------------------------------------------------------------------
// Key k < hw sits in the low half of word k, key k >= hw in the high half of
// word k - hw (hw = half the slice), so consecutive keys of a sorted list hit
// different words. Flushing and clearing visit only the words the slice
// touched, found one of two ways (TRACK):
//  * TOUCH_LIST -- the first increment of a word appends it to a list (one
//    shared atomic per warp and step); past the list's capacity (TCAP) the
//    sweep scans the slice. Suits narrow key ranges (consecutive keys).
//  * TOUCH_BITMAP -- the first increment of a word sets its bit in a bitmap
//    (one bit per counter word, no capacity). Suits wide slices where a
//    warp's keys are far apart (its bitmap words differ).
//  * TOUCH_PAIRS -- only a key whose count goes from 1 to 2 is listed (the
//    keys that will emit); the sweep visits the list and the slice is
//    cleared whole with 16-byte stores; past the list's capacity (PCAP) the
//    sweep scans the slice. Suits wide slices where most keys are touched
//    once (no emit): the sweep costs the emitting keys, not the touched ones.
// Counts must stay below 2^16 (the caller routes anchors of degree >= 65535
// elsewhere) unless the slice is set up with 32-bit counters. SCRATCH extra
// bytes after the tracking structure are free for the caller between passes.
constexpr int DENSE_KEYS = 36864;               // keys per dense slice
constexpr int DENSE_WORDS = DENSE_KEYS / 2;     // 18432 words (72 KB)
constexpr int TOUCH_CAP = 8192;                 // touched-word list capacity
enum { TOUCH_LIST = 0, TOUCH_BITMAP = 1, TOUCH_PAIRS = 2 };

template <int WORDS, int TRACK = TOUCH_LIST, int SCRATCH = 0, int PAIRS_CAP = 4096>
struct DenseSliceT {
    static_assert(WORDS % 128 == 0 && WORDS <= 65536, "counter words");
    static constexpr int BM_WORDS = WORDS / 32;
    static constexpr int TCAP = TOUCH_CAP;
    // listed keys fit 16 bits while a slice has at most 65,536 keys
    static constexpr bool P16 = 2 * WORDS <= 65536;
    static constexpr size_t track_bytes() {
        return TRACK == TOUCH_BITMAP  ? (size_t)BM_WORDS * 4
               : TRACK == TOUCH_PAIRS ? (size_t)PAIRS_CAP * (P16 ? 2 : 4)
                                      : (size_t)TCAP * 2;
    }
    uint32_t *cnt;     // WORDS
    uint32_t *tbm;     // BM_WORDS: touched counter words (bitmap tracking)
    uint16_t *tl;      // TCAP: touched counter words (list tracking)
    uint32_t *pl;      // PAIRS_CAP: keys that reached count 2 (pairs tracking)
    int *s_nt;         // shared scalar: list entries (list tracking)
    int32_t hw;        // half of the current slice width (<= WORDS)
    bool wide;         // 32-bit counters, one key per word (slices of WORDS keys)

    static constexpr size_t bytes() {
        return (size_t)WORDS * 4 + track_bytes() + (size_t)((SCRATCH + 15) & ~15);
    }
    __device__ unsigned char *bind(unsigned char *base, int *nt = nullptr) {
        cnt = (uint32_t *)base;
        tbm = cnt + WORDS;
        tl = (uint16_t *)(cnt + WORDS);
        pl = cnt + WORDS;
        s_nt = nt;
        hw = WORDS;
        wide = false;
        return (unsigned char *)base + bytes();
    }
    __device__ void *scratch() const { return (void *)((unsigned char *)(cnt + WORDS) + track_bytes()); }
    __device__ void clear_all() {
        const int n4 = TRACK == TOUCH_BITMAP ? (WORDS + BM_WORDS) / 4 : WORDS / 4;
        for (int i = threadIdx.x; i < n4; i += blockDim.x) ((uint4 *)cnt)[i] = make_uint4(0, 0, 0, 0);
        if (TRACK != TOUCH_BITMAP && threadIdx.x == 0) *s_nt = 0;
    }
    // Slice of w keys: 16-bit counters (w <= 2 * WORDS), or 32-bit counters
    // when counts may reach 2^16 (w <= WORDS).
    __device__ void set_width(int32_t w, bool wide_counts = false) {
        wide = wide_counts;
        hw = wide ? w : (w + 1) >> 1;
    }
    __device__ __forceinline__ void add(int32_t k) {
        const bool hi = !wide && k >= hw;
        const int32_t w = hi ? k - hw : k;
        const uint32_t old = atomicAdd(&cnt[w], hi ? 0x10000u : 1u);
        if (TRACK == TOUCH_BITMAP) {
            if (old == 0) atomicOr(&tbm[w >> 5], 1u << (w & 31));
        } else if (TRACK == TOUCH_PAIRS) {
            const uint32_t prev = wide ? old : (hi ? old >> 16 : old & 0xffffu);
            const unsigned m = __activemask();
            const unsigned b = __ballot_sync(m, prev == 1);
            if (b) {
                const int lane = threadIdx.x & 31;
                const int leader = __ffs(b) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(s_nt, __popc(b));
                base = __shfl_sync(m, base, leader);
                if (prev == 1) {
                    const int pos = base + __popc(b & lanemask_lt());
                    if (pos < PAIRS_CAP) {
                        if (P16)
                            tl[pos] = (uint16_t)k;
                        else
                            pl[pos] = (uint32_t)k;
                    }
                }
            }
        } else {
            const unsigned m = __activemask();
            const unsigned b = __ballot_sync(m, old == 0);
            if (b) {
                const int lane = threadIdx.x & 31;
                const int leader = __ffs(b) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(s_nt, __popc(b));
                base = __shfl_sync(m, base, leader);
                if (old == 0) {
                    const int pos = base + __popc(b & lanemask_lt());
                    if (pos < TCAP) tl[pos] = (uint16_t)w;
                }
            }
        }
    }
    __device__ __forceinline__ uint32_t count(int32_t k) const {
        if (wide) return cnt[k];
        const bool hi = k >= hw;
        return (cnt[hi ? k - hw : k] >> (hi ? 16 : 0)) & 0xffffu;
    }
    // (key, count) pairs of up to four counter words, for emit_many.
    __device__ __forceinline__ void pairs4(const int (&w)[4], const uint32_t (&v)[4], int32_t (&kk)[8],
                                           uint32_t (&cc)[8]) const {
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (wide) {
                kk[2 * u] = w[u] >= 0 && v[u] >= 2 ? w[u] : -1;
                cc[2 * u] = v[u];
                kk[2 * u + 1] = -1;
                cc[2 * u + 1] = 0;
            } else {
                const uint32_t c0 = v[u] & 0xffffu, c1 = v[u] >> 16;
                kk[2 * u] = w[u] >= 0 && c0 >= 2 ? w[u] : -1;
                cc[2 * u] = c0;
                kk[2 * u + 1] = w[u] >= 0 && c1 >= 2 ? w[u] + hw : -1;
                cc[2 * u + 1] = c1;
            }
        }
    }
    // EMIT: emit(key, count) for every key with count >= 2; CLEAR: zero the
    // touched words (and their bits). Four words at a time per thread, so up
    // to 8 emits are issued together. The caller synchronises afterwards,
    // then reset_scalars().
    template <bool EMIT, bool CLEAR, class Emit>
    __device__ void sweep(Emit &emit) {
        int32_t kk[8];
        uint32_t cc[8];
        int w[4];
        uint32_t v[4];
        if (TRACK == TOUCH_BITMAP) {
            const int nbw = (hw + 31) >> 5;
            for (int b = threadIdx.x; b < nbw; b += blockDim.x) {
                uint32_t m = tbm[b];
                if (m == 0) continue;
                if (CLEAR) tbm[b] = 0;
                do {
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        w[u] = -1;
                        if (m) {
                            w[u] = (b << 5) + __ffs(m) - 1;
                            m &= m - 1;
                        }
                        v[u] = w[u] >= 0 ? cnt[w[u]] : 0u;
                        if (CLEAR && w[u] >= 0) cnt[w[u]] = 0;
                    }
                    pairs4(w, v, kk, cc);
                    if (EMIT) emit_many<8>(emit, kk, cc);
                } while (m);
            }
            return;
        }
        if (TRACK == TOUCH_PAIRS) {
            const int np = *(volatile int *)s_nt;
            if (np <= PAIRS_CAP) {
                // the listed keys, 8 per thread at a time
                for (int i0 = threadIdx.x; i0 < np; i0 += 8 * blockDim.x) {
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int i = i0 + u * blockDim.x;
                        kk[u] = i < np ? (int32_t)(P16 ? (uint32_t)tl[i] : pl[i]) : -1;
                        cc[u] = kk[u] >= 0 ? count(kk[u]) : 0u;
                    }
                    if (EMIT) emit_many<8>(emit, kk, cc);
                }
            } else {
                // too many to list: every word of the slice
                for (int i0 = threadIdx.x; i0 < hw; i0 += 4 * blockDim.x) {
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int i = i0 + u * blockDim.x;
                        w[u] = i < hw ? i : -1;
                        v[u] = w[u] >= 0 ? cnt[w[u]] : 0u;
                        if (v[u] == 0) w[u] = -1;
                    }
                    pairs4(w, v, kk, cc);
                    if (EMIT) emit_many<8>(emit, kk, cc);
                }
            }
            if (CLEAR) {
                __syncthreads();  // every count read before the slice is cleared
                for (int i = threadIdx.x; i < (hw + 3) / 4; i += blockDim.x)
                    ((uint4 *)cnt)[i] = make_uint4(0, 0, 0, 0);
            }
            return;
        }
        const int nt = *(volatile int *)s_nt;
        const bool listed = nt <= TCAP;
        const int n = listed ? nt : hw;  // list entries, or every word of the slice
        for (int i0 = threadIdx.x; i0 < n; i0 += 4 * blockDim.x) {
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int i = i0 + u * blockDim.x;
                w[u] = i < n ? (listed ? (int)tl[i] : i) : -1;
                v[u] = w[u] >= 0 ? cnt[w[u]] : 0u;
                if (v[u] == 0) w[u] = -1;
                if (CLEAR && w[u] >= 0) cnt[w[u]] = 0;
            }
            pairs4(w, v, kk, cc);
            if (EMIT) emit_many<8>(emit, kk, cc);
        }
    }
    __device__ void reset_scalars() {
        if (TRACK != TOUCH_BITMAP && threadIdx.x == 0) *s_nt = 0;
    }
};

using DenseSlice = DenseSliceT<DENSE_WORDS>;

// ------------------------------------------------------------------
// Global dense counters + touched list (one slot per CTA)
// ------------------------------------------------------------------
struct GlobalDense {
    uint32_t *cnt;    // keyspace, all zero between anchors
    int32_t *touch;   // keyspace
    int *s_nt;        // shared scalar: touched entries

    __device__ __forceinline__ void add(int32_t k) {
        uint32_t old = atomicAdd(&cnt[k], 1u);
        if (old == 0) touch[atomicAdd(s_nt, 1)] = k;
    }
    __device__ __forceinline__ uint32_t count(int32_t k) const { return cnt[k]; }
    template <class Emit>
    __device__ void flush(Emit &emit) {
        int nt = *s_nt;
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
            int32_t k = touch[i];
            uint32_t c = cnt[k];
            if (c >= 2) emit(k, c);
        }
    }
    __device__ void clear() {
        int nt = *s_nt;
        for (int i = threadIdx.x; i < nt; i += blockDim.x) cnt[touch[i]] = 0;
    }
};

// ------------------------------------------------------------------
// CTA traversal of one anchor's wedges
// ------------------------------------------------------------------
// Chunk staging in shared memory: up to MID_CHUNK middle vertices with
// non-empty segments, compacted: segment start, exclusive prefix of segment
// lengths, and the mid's index within the chunk.
struct Chunk {
    int64_t *beg;    // MID_CHUNK
    int32_t *pre;    // MID_CHUNK + 1
    int32_t *tmp;    // 36 (scan scratch)
    int32_t *len;    // MID_CHUNK: chunk-local mid index of compacted segment k
};

// staging of up to T middle vertices (a CTA of T threads)
__host__ __device__ constexpr size_t chunk_bytes(int T) {
    return (size_t)T * 8 + (size_t)(T + 1) * 4 + 33 * 4 + (size_t)T * 4 + 16;
}
constexpr size_t CHUNK_BYTES = chunk_bytes(MID_CHUNK);

__device__ __forceinline__ int32_t *chunk_len_ptr(int32_t *tmp) { return tmp + 36; }

struct NoChunkHook {
    __device__ void operator()(int64_t, int) {}
};

// Walks every wedge of one anchor: for q in [q0, q1) (middle vertices), the
// segment M.seg(q) of `keys`. The non-empty segments of up to blockDim.x
// middle vertices are staged at a time; the flat list of their wedges is cut
// into 32-wedge groups. BALANCED: every warp takes an equal contiguous share
// of the groups, WALK_UNROLL per step; otherwise warps take WALK_UNROLL
// consecutive groups in turn (fewer warps busy on small chunks, which suits
// the hybrid engine's shared-memory traffic). In a group, lane i fetches the start of the i-th segment after the
// group's first one; one OR-reduction of those starts gives every lane the
// segment its wedge falls in (a population count), so every lane loads a key
// even when segments are short, and all loads of a step are issued before any
// key is visited.
// Mids source contract:
//   __device__ void seg(int64_t q, int64_t &beg, int32_t &len) const;
// visit(k, key): k = mid index within the chunk, key = end point.
// Returns the number of wedges walked. All threads of the CTA must call it.
template <bool BALANCED = true, class Mids, class Visit, class Hook = NoChunkHook>
__device__ int64_t cta_walk(const Mids &M, int64_t q0, int64_t q1, const int32_t *__restrict__ keys,
                            Chunk &ch, Visit &visit, Hook *hook = nullptr) {
    // one scan of (segment length | non-empty flag << 40) gives both the
    // wedge offsets and the compacted slots (a chunk holds < 2^40 wedges)
    __shared__ long long s_scan[33];
    int64_t walked = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const unsigned lanes_le = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    for (int64_t c0 = q0; c0 < q1; c0 += blockDim.x) {
        const int nm = (int)imin64(blockDim.x, q1 - c0);
        long long tot2;
        if (nm <= 32) {
            // at most 32 middle vertices: warp 0 stages them with a warp scan
            // (one barrier instead of the block scan's three)
            if (warp == 0) {
                int64_t beg = 0;
                int32_t len = 0;
                if (lane < nm) M.seg(c0 + lane, beg, len);
                const long long packed = (long long)len | (len > 0 ? (1ll << 40) : 0ll);
                long long inc = packed;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const long long y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += y;
                }
                const long long ex2 = inc - packed;
                if (len > 0) {
                    const int32_t slot = (int32_t)(ex2 >> 40);
                    ch.beg[slot] = beg;
                    ch.pre[slot] = (int32_t)(ex2 & ((1ll << 40) - 1));
                    ch.len[slot] = lane;
                }
                if (lane == 31) {
                    s_scan[32] = inc;
                    ch.pre[inc >> 40] = (int32_t)(inc & ((1ll << 40) - 1));
                }
            }
            __syncthreads();
            tot2 = s_scan[32];
        } else {
            int64_t beg = 0;
            int32_t len = 0;
            if ((int)threadIdx.x < nm) M.seg(c0 + threadIdx.x, beg, len);
            const long long packed = (long long)len | (len > 0 ? (1ll << 40) : 0ll);
            const long long ex2 = block_exclusive_scan<long long, false>(packed, s_scan, &tot2);
            const int32_t ex = (int32_t)(ex2 & ((1ll << 40) - 1));
            const int32_t slot = (int32_t)(ex2 >> 40);
            if (len > 0) {
                ch.beg[slot] = beg;
                ch.pre[slot] = ex;
                ch.len[slot] = threadIdx.x;
            }
            if (threadIdx.x == 0) ch.pre[tot2 >> 40] = (int32_t)(tot2 & ((1ll << 40) - 1));
            __syncthreads();
        }
        const int32_t total = (int32_t)(tot2 & ((1ll << 40) - 1));
        const int32_t nnz = (int32_t)(tot2 >> 40);
        const int32_t groups = (total + 31) >> 5;
        const int32_t g_lo = BALANCED ? (int32_t)(((int64_t)groups * warp) / nwarps) : warp * WALK_UNROLL;
        const int32_t g_hi = BALANCED ? (int32_t)(((int64_t)groups * (warp + 1)) / nwarps) : groups;
        const int32_t g_step = BALANCED ? WALK_UNROLL : nwarps * WALK_UNROLL;
        for (int32_t gb = g_lo; gb < g_hi; gb += g_step) {
            // segment of the first wedge of group gb (warp-uniform search)
            int lo = 0, hi = nnz - 1;
            const int32_t b0 = gb << 5;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (ch.pre[mid] <= b0)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            int k0 = lo;
            // segment k0 in registers: wedges [p0, p1), first key, mid index
            int32_t p0 = ch.pre[k0], p1 = ch.pre[k0 + 1];
            int64_t bg0 = ch.beg[k0];
            int kl0 = ch.len[k0];
            int kk[WALK_UNROLL];
            int32_t key[WALK_UNROLL];
#pragma unroll
            for (int u = 0; u < WALK_UNROLL; u++) {
                const int32_t base = (gb + u) << 5;
                kk[u] = 0;
                key[u] = -1;
                if (BALANCED ? gb + u < g_hi : base < total) {
                    const int32_t j = base + lane;
                    if (base >= p0 && base + 32 <= p1) {
                        // the whole group lies in segment k0 (long lists: the
                        // common case), no shared-memory lookups
                        kk[u] = kl0;
                        key[u] = __ldg(keys + bg0 + (j - p0));
                    } else {
                        while (ch.pre[k0 + 1] <= base) k0++;
                        const int kn = k0 + 1 + lane;
                        const int32_t bnd = kn < nnz ? ch.pre[kn] - base : 32;
                        const unsigned m =
                            __reduce_or_sync(0xffffffffu, bnd < 32 ? (1u << bnd) : 0u);
                        const int k = k0 + __popc(m & lanes_le);
                        if (j < total) {
                            kk[u] = ch.len[k];
                            key[u] = __ldg(keys + ch.beg[k] + (j - ch.pre[k]));
                        }
                        // continue from the segment of the group's last wedge
                        k0 = min(k0 + __popc(m), nnz - 1);
                        p0 = ch.pre[k0];
                        p1 = ch.pre[k0 + 1];
                        bg0 = ch.beg[k0];
                        kl0 = ch.len[k0];
                    }
                }
            }
            visit_many<WALK_UNROLL>(visit, kk, key);
        }
        walked += total;
        __syncthreads();
        if (hook) {
            (*hook)(c0, nm);
            __syncthreads();
        }
    }
    return walked;
}

}  // namespace receipt
