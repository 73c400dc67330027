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
constexpr int MID_CHUNK = CTA_THREADS;
constexpr int REPEAT_SLOTS = 4096;  // CtaHybrid repeat table
constexpr int REPEAT_LIMIT = REPEAT_SLOTS / 2;
constexpr int HEAD_MAX = 16384;     // dense 16-bit counters for keys < head
constexpr int HEAD_SLICE = 2048;    // head of the key slices after the first
constexpr int SLICE_KEYS = 65536;   // keys per slice of the sliced tier
constexpr int SLICE_MIN_W = 49152;  // anchors with more wedges use the sliced tier
constexpr int MAX_PROBE = 64;
constexpr int WALK_UNROLL = 8;     // independent loads in flight per warp in cta_walk

__device__ __forceinline__ uint32_t hash_key(int32_t k) {
    return (uint32_t)k * 2654435761u;
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
// CTA hybrid: dense head counters + tail bitmap + repeat table
// ------------------------------------------------------------------
struct CtaHybrid {
    uint32_t *head;   // head/2 words, two 16-bit counters each
    uint32_t *bm;     // bitmap over keys [head, keyspace)
    int32_t *rkey;    // REPEAT_SLOTS
    uint32_t *rval;   // REPEAT_SLOTS: extra occurrences (count - 1)
    int *s_used;      // shared scalar: repeat slots in use
    int *s_over;      // shared scalar: repeat table overflowed
    int32_t headn;    // number of head keys (even)
    int32_t bm_words; // bitmap words
    int32_t act_hw;   // head words in use for the current anchor
    int32_t act_bw;   // bitmap words in use for the current anchor

    // Restricts clear/flush to keys below ks (counting: end points < sp).
    __device__ void set_active(int64_t ks) {
        int64_t h = ks < headn ? ks : headn;
        act_hw = (int32_t)((h + 1) >> 1);
        int64_t t = ks - headn;
        act_bw = t > 0 ? (int32_t)imin64((t + 31) >> 5, bm_words) : 0;
    }
    __device__ void clear_active() {
        for (int i = threadIdx.x; i < act_hw; i += blockDim.x) head[i] = 0;
        uint4 z = make_uint4(0, 0, 0, 0);
        for (int i = threadIdx.x; i < (act_bw >> 2); i += blockDim.x) ((uint4 *)bm)[i] = z;
        for (int i = (act_bw & ~3) + threadIdx.x; i < act_bw; i += blockDim.x) bm[i] = 0;
        for (int i = threadIdx.x; i < REPEAT_SLOTS; i += blockDim.x) {
            rkey[i] = EMPTY_KEY;
            rval[i] = 0;
        }
        if (threadIdx.x == 0) {
            *s_used = 0;
            *s_over = 0;
        }
    }

    __device__ void clear_all() {
        uint4 z = make_uint4(0, 0, 0, 0);
        int hw = headn >> 1;
        for (int i = threadIdx.x; i < (hw >> 2); i += blockDim.x) ((uint4 *)head)[i] = z;
        for (int i = (hw & ~3) + threadIdx.x; i < hw; i += blockDim.x) head[i] = 0;
        for (int i = threadIdx.x; i < (bm_words >> 2); i += blockDim.x) ((uint4 *)bm)[i] = z;
        for (int i = (bm_words & ~3) + threadIdx.x; i < bm_words; i += blockDim.x) bm[i] = 0;
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
            atomicAdd(&head[k >> 1], 1u << ((k & 1) << 4));
            return;
        }
        int32_t t = k - headn;
        uint32_t bit = 1u << (t & 31);
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
                if (atomicAdd(s_used, 1) >= REPEAT_LIMIT) {
                    *(volatile int *)s_over = 1;
                    return;
                }
                int32_t prev = atomicCAS(&rkey[h], EMPTY_KEY, k);
                if (prev == EMPTY_KEY) {
                    atomicAdd(&rval[h], 1u);
                    return;
                }
                atomicSub(s_used, 1);
                if (prev == k) {
                    atomicAdd(&rval[h], 1u);
                    return;
                }
            }
            h = (h + 1) & (REPEAT_SLOTS - 1);
        }
        *(volatile int *)s_over = 1;
    }
    // count of key k after aggregation (k must have been added at least once
    // if k >= head; head keys may be 0)
    __device__ __forceinline__ uint32_t count(int32_t k) const {
        if (k < headn) return (head[k >> 1] >> ((k & 1) << 4)) & 0xffffu;
        uint32_t h = hash_key(k) & (REPEAT_SLOTS - 1);
        for (int p = 0; p < MAX_PROBE; p++) {
            int32_t cur = rkey[h];
            if (cur == k) return 1u + rval[h];
            if (cur == EMPTY_KEY) return 1u;
            h = (h + 1) & (REPEAT_SLOTS - 1);
        }
        return 1u;
    }
    // Emits (EMIT) every key with count >= 2 and returns the engine to all
    // zeros for the active key range, reading each structure once. The
    // caller synchronises afterwards and then calls reset_scalars().
    template <bool EMIT, class Emit>
    __device__ void flush_clear(Emit &emit) {
        const int used = *(volatile int *)s_used;
        const int hw = act_hw;
        for (int w = threadIdx.x; w < hw; w += blockDim.x) {
            uint32_t v = head[w];
            if (v) {
                head[w] = 0;
                if (EMIT) {
                    uint32_t c0 = v & 0xffffu, c1 = v >> 16;
                    if (c0 >= 2) emit(2 * w, c0);
                    if (c1 >= 2) emit(2 * w + 1, c1);
                }
            }
        }
        if (used > 0) {
            for (int i = threadIdx.x; i < REPEAT_SLOTS; i += blockDim.x) {
                int32_t k = rkey[i];
                if (k != EMPTY_KEY) {
                    if (EMIT) emit(k, 1u + rval[i]);
                    rkey[i] = EMPTY_KEY;
                    rval[i] = 0;
                }
            }
        }
        uint4 z = make_uint4(0, 0, 0, 0);
        for (int i = threadIdx.x; i < (act_bw >> 2); i += blockDim.x) ((uint4 *)bm)[i] = z;
        for (int i = (act_bw & ~3) + threadIdx.x; i < act_bw; i += blockDim.x) bm[i] = 0;
    }
    __device__ void reset_scalars() {
        if (threadIdx.x == 0) {
            *s_used = 0;
            *s_over = 0;
        }
    }

    // calls emit(key, count) for every key with count >= 2
    template <class Emit>
    __device__ void flush(Emit &emit) {
        int hw = act_hw;
        for (int w = threadIdx.x; w < hw; w += blockDim.x) {
            uint32_t v = head[w];
            if (v) {
                uint32_t c0 = v & 0xffffu, c1 = v >> 16;
                if (c0 >= 2) emit(2 * w, c0);
                if (c1 >= 2) emit(2 * w + 1, c1);
            }
        }
        for (int i = threadIdx.x; i < REPEAT_SLOTS; i += blockDim.x) {
            int32_t k = rkey[i];
            if (k != EMPTY_KEY) emit(k, 1u + rval[i]);
        }
    }
};

// smem bytes of a CtaHybrid for a key space (excluding the chunk arrays)
inline size_t hybrid_bytes(int64_t keyspace, int32_t *headn_out, int32_t *bm_words_out) {
    int64_t headn = keyspace < HEAD_MAX ? keyspace : HEAD_MAX;
    headn = (headn + 1) & ~1ll;
    int64_t tail = keyspace - headn;
    if (tail < 0) tail = 0;
    int64_t bmw = (tail + 31) / 32;
    bmw = (bmw + 3) & ~3ll;
    int64_t hw = ((headn >> 1) + 3) & ~3ll;
    if (headn_out) *headn_out = (int32_t)headn;
    if (bm_words_out) *bm_words_out = (int32_t)bmw;
    return (size_t)(hw * 4 + bmw * 4 + (int64_t)REPEAT_SLOTS * 8);
}

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
// Chunk staging in shared memory: up to MID_CHUNK middle vertices, their
// segment starts and the exclusive prefix of segment lengths.
struct Chunk {
    int64_t *beg;    // MID_CHUNK
    int32_t *pre;    // MID_CHUNK + 1
    int32_t *tmp;    // 33 (scan scratch)
};

constexpr size_t CHUNK_BYTES = MID_CHUNK * 8 + (MID_CHUNK + 1) * 4 + 33 * 4 + 12;

// Mids source contract:
//   __device__ void seg(int64_t q, int64_t &beg, int32_t &len) const;
// visit(k, key): k = mid index within the chunk, key = end point.
// Returns the number of wedges walked. All threads of the CTA must call it.
struct NoChunkHook {
    __device__ void operator()(int64_t, int) {}
};

template <class Mids, class Visit, class Hook = NoChunkHook>
__device__ int64_t cta_walk(const Mids &M, int64_t q0, int64_t q1, const int32_t *__restrict__ keys,
                            Chunk &ch, Visit &visit, Hook *hook = nullptr) {
    int64_t walked = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int64_t c0 = q0; c0 < q1; c0 += blockDim.x) {
        int nm = (int)imin64(blockDim.x, q1 - c0);
        int64_t beg = 0;
        int32_t len = 0;
        if ((int)threadIdx.x < nm) M.seg(c0 + threadIdx.x, beg, len);
        int32_t total;
        int32_t ex = block_exclusive_scan<int32_t>(len, ch.tmp, &total);
        ch.beg[threadIdx.x] = beg;
        ch.pre[threadIdx.x] = ex;
        if (threadIdx.x == 0) ch.pre[blockDim.x] = total;
        __syncthreads();
        // Each warp takes WALK_UNROLL consecutive 32-wide slabs of the flat
        // wedge index per step and issues all their loads before using any,
        // so WALK_UNROLL independent L2 reads are in flight per warp.
        for (int32_t base = warp * 32 * WALK_UNROLL; base < total;
             base += nwarps * 32 * WALK_UNROLL) {
            // largest k with pre[k] <= base (binary search, broadcast reads)
            int lo = 0, hi = nm - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (ch.pre[mid] <= base)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            int kk[WALK_UNROLL];
            int32_t key[WALK_UNROLL];
            int k = lo;
#pragma unroll
            for (int u = 0; u < WALK_UNROLL; u++) {
                int32_t j = base + u * 32 + lane;
                kk[u] = -1;
                if (j < total) {
                    while (k + 1 < nm && ch.pre[k + 1] <= j) k++;
                    kk[u] = k;
                    key[u] = __ldg(keys + ch.beg[k] + (j - ch.pre[k]));
                }
            }
#pragma unroll
            for (int u = 0; u < WALK_UNROLL; u++)
                if (kk[u] >= 0) visit(kk[u], key[u]);
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
