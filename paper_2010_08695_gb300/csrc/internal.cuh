// Cross-translation-unit declarations of libreceipt.so (host side).
#pragma once

#include "common.cuh"

namespace receipt {

receipt_graph *build_graph(const int32_t *d_eu, const int32_t *d_ev, int64_t m, int32_t nu,
                           int32_t nv, int dedup, cudaStream_t s);
void destroy_graph(receipt_graph *g);

// Butterfly counts of both sides by local id; returns wedges traversed.
// points (optional, 5 entries) accumulates the start points per tier: warp,
// shared hash, CTA hybrid, global (by degree or key space), global after a
// repeat-table overflow.
uint64_t count_local(const receipt_graph *g, unsigned long long *cnt_u, unsigned long long *cnt_v,
                     cudaStream_t s, int64_t *points = nullptr);
void scatter_to_original(const unsigned long long *local, const int32_t *new2old, int32_t n,
                         unsigned long long *out, cudaStream_t s);
// Counting with every temporary in a static device array (no allocation).
void count_noalloc(const receipt_graph *g, unsigned long long *d_cnt_u,
                   unsigned long long *d_cnt_v, cudaStream_t s);

// Page-locked host buffer of at least `bytes`, owned by the calling thread
// and reused across calls (no allocation per call).
void *pinned_scratch(size_t bytes);

// Non-blocking auxiliary stream of the calling thread on the current device:
// CUDA graphs are captured on it, and counting runs its second pass on it.
cudaStream_t aux_stream();
// Non-blocking streams of the calling thread on the current device on which
// the independent peel tiers of one round run side by side.
constexpr int NUM_TIER_STREAMS = 3;
cudaStream_t tier_stream(int k);

// Largest key space whose CtaHybrid engine plus `extra` bytes fits in the
// opt-in shared memory of one CTA (capped at `want`); 0 if none.
int64_t max_cta_keyspace(int64_t want, size_t extra);

// Full tip decomposition of side `side` of g into d_tip (original ids).
void tip_decompose_impl(receipt_graph *g, int side, uint64_t *d_tip, const receipt_options *opt,
                        cudaStream_t s);

}  // namespace receipt

namespace receipt {

// Working state of one decomposition of side `s` (device pointers, local ids).
struct Decomp {
    int s = 0;
    const Side *S = nullptr;  // side being decomposed
    const Side *O = nullptr;  // other side
    int32_t n = 0;
    int64_t m = 0;
    int32_t max_deg_s = 0;                // largest degree on side s
    unsigned long long *sup = nullptr;    // raw supports
    unsigned long long *init = nullptr;   // support when the vertex's range began
    int32_t *sub = nullptr;               // subset index, -1 while remaining
    unsigned long long *wfull = nullptr;  // sum of d_y over y in N_x
    int32_t p_eff = 0;
    std::vector<uint64_t> bounds;         // theta(1..p_eff+1)
    uint64_t wedges_cd = 0, wedges_fd = 0;
    int64_t rounds = 0, levels = 0;
    int32_t dgm_passes = 0;
    bool timing = false;
    uint64_t tier_wedges[5] = {}, tier_mids[5] = {};
    uint64_t tier_anchors[5] = {};
    uint64_t tier_pairs[5] = {};  // support atomics (nonzero pairs) per tier
    int64_t tier_launches[5] = {};
    float tier_ms[5] = {};
    std::vector<receipt_round> trace;
    float fd_max_ms = 0;         // slowest subset of the fine-grained step
    int32_t fd_max_n = 0;        // its size
    int64_t fd_max_levels = 0;   // its peeling levels
    int64_t fd_heavy_w = 0;      // heavy-subset threshold (0 automatic, -1 never)
    int32_t fd_heavy = 0;        // subsets peeled by all CTAs
    float fd_heavy_ms = 0;
    int64_t fd_heavy_levels = 0;
    int64_t fd_split_levels = 0; // heavy levels whose big walks were split over the CTAs
    int32_t fd_tasks = 0;        // tasks of the fine-grained step
    // first vertex of every packed graph when the side is a batch's
    // disjoint union (null otherwise)
    const std::vector<int64_t> *parts = nullptr;
    std::vector<receipt_subset> subsets;
    int32_t fd_huc = 0;              // recount rule of the fine-grained step's heavy tasks
    // factor of the recount rules (a range's first round of Algorithm 3, a
    // heavy task's level of Algorithm 4, recounts when its walks exceed
    // huc_factor * C_rcnt): per unit of the two cost measures the peel tiers
    // run 4-10 times faster than the counting kernels (measured on Chung-Lu
    // graphs of 10M and 100M edges), hence 8 by default
    double huc_factor = 8.0;
    int32_t fd_recounts = 0;         // levels of heavy tasks whose updates were a recount
    uint64_t wedges_fd_recount = 0;  // wedges traversed by those recounts
    int32_t huc_recounts = 0;        // rounds whose updates were a recount (Sec. 4.1)
    uint64_t wedges_recount = 0;     // wedges traversed by those recounts
    uint64_t cost_recount = 0;       // C_rcnt = sum over edges of min(d_u, d_v)
    float ms_recount = 0;
};

void cd_run(Decomp &D, const receipt_options &opt, cudaStream_t s);

// Hybrid update computation (Sec. 4.1). Enqueues *d_out = C_rcnt, the sum
// over the edges (x, y) of min(d_x, d_y).
void launch_recount_cost(const Side &S, const Side &O, int64_t m, unsigned long long *d_out,
                         cudaStream_t s);
// Whether free device memory holds a recount's temporaries (upper estimate).
bool recount_fits(const Decomp &D);
// Recounts the butterflies of the subgraph left after removing every vertex
// with D.sub >= 0 and stores each remaining vertex's count in D.sup.
// len_w/adj_w: the other side's lists (original offsets) already compacted
// to remaining vertices. Returns the wedges traversed; synchronises s.
uint64_t recount_remaining(const Decomp &D, const int32_t *len_w, const int32_t *adj_w,
                           cudaStream_t s);
// The same for any kept set: counts, in the subgraph of the side-s vertices
// x with sub[x] < 0 and all of the other side, of every kept vertex into
// sup[x]. len_w/adj_w: the other side's lists (original offsets) already
// compacted to kept vertices. Returns the wedges traversed; synchronises s.
uint64_t recount_masked(const Side &S, const Side &O, int side_s, int64_t m, const int32_t *sub,
                        unsigned long long *sup, const int32_t *len_w, const int32_t *adj_w,
                        cudaStream_t s);
// Drops from every list y of the other side (working copy adj_w with
// lengths len_w, original offsets off_o) the entries x with sub[x] >= 0.
void compact_lists(const int64_t *off_o, int32_t *len_w, int32_t *adj_w, int32_t n_o,
                   const int32_t *sub, cudaStream_t s);
// len[y] = off[y + 1] - off[y]
void list_lengths(const int64_t *off, int32_t n, int32_t *len, cudaStream_t s);
void fd_run(Decomp &D, uint64_t *d_tip, cudaStream_t s);

}  // namespace receipt
