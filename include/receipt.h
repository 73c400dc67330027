/*
 * receipt.h -- C ABI of the GB300 (sm_103a) RECEIPT tip-decomposition library.
 *
 * The method is RECEIPT (Lakhotia, Kannan, Prasanna, De Rose): per-vertex
 * butterfly counting (Algorithm 1), a coarse-grained decomposition that
 * splits one side's vertices into tip-number ranges by concurrent range
 * peeling (Algorithm 3), and a fine-grained decomposition that peels every
 * range's vertex subset independently and exactly (Algorithm 4), with the
 * support update of Algorithm 2.
 *
 * Conventions shared by every entry point
 *  - A bipartite graph G(W = (U, V), E) is given by |U| = nu, |V| = nv and m
 *    edges (eu[i], ev[i]) with 0 <= eu[i] < nu and 0 <= ev[i] < nv (original
 *    ids). Vertex ids are int32; counts and tip numbers are exact uint64.
 *  - Pointers named d_* are device pointers on the current CUDA device and
 *    h_* are host pointers. The caller owns every buffer it passes in; the
 *    library never frees or keeps them past the call.
 *  - Results are indexed by ORIGINAL vertex id.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is
 *    enqueued on it; entry points that need a decision from the device
 *    (the range loop of tip_decompose, validation in build_csr) synchronise
 *    that stream before they return, so outputs are ready on return unless
 *    stated otherwise.
 *  - No C++ exception crosses this boundary. Every entry point returns a
 *    receipt_status; receipt_last_error() gives a thread-local message for the
 *    most recent failure on the calling thread.
 *  - No kernel waits on a flag or on another CTA, and every bounded
 *    structure either is sized from exact counts or has an exact fallback
 *    (an anchor whose repeat table overflows is redone through key slices),
 *    so the decomposition calls have no device-side error path.
 *    RECEIPT_ERR_TIMEOUT and RECEIPT_ERR_INTERNAL come from the serving
 *    engine (a wait that ran out of time; a request whose decomposition
 *    failed in a worker); RECEIPT_ERR_INTERNAL also reports a failed
 *    internal consistency check (not expected to happen).
 */
#ifndef RECEIPT_H
#define RECEIPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RECEIPT_OK = 0,
    RECEIPT_ERR_INVALID = 1,  /* bad argument: id out of range, null pointer, bad side */
    RECEIPT_ERR_OOM = 2,      /* device allocation failed                           */
    RECEIPT_ERR_CUDA = 3,     /* a CUDA runtime call failed                          */
    RECEIPT_ERR_TIMEOUT = 4,  /* a wait for a served request ran out of time         */
    RECEIPT_ERR_OVERFLOW = 5, /* a count would exceed 2^63 or m exceeds the id space */
    RECEIPT_ERR_BUSY = 6,     /* the serving engine has no free slot or memory       */
    RECEIPT_ERR_INTERNAL = 7  /* unexpected failure inside the library               */
} receipt_status;

typedef enum { RECEIPT_SIDE_U = 0, RECEIPT_SIDE_V = 1 } receipt_side;

/* Opaque, library-owned graph: the relabelled two-sided CSR on the device. */
typedef struct receipt_graph receipt_graph;

/*
 * Options of a tip decomposition. Zero-initialise, then set what you need;
 * receipt_options_default() fills the defaults.
 */
typedef struct {
    /* P, the number of vertex subsets the coarse-grained decomposition
     * creates (Algorithm 3, input P; Sec. 5 uses 150). 0 means 150. */
    int32_t P;
    /* Optional injected range bounds theta(2) < theta(3) < ... (host array
     * of n_bounds values, strictly increasing and > 0). When given they
     * replace the adaptive range determination of Sec. 3.1.1; the last
     * subset collects all vertices left after the given ranges. Tip numbers
     * do not depend on the ranges (Theorem 2), so this is a test hook. */
    const uint64_t *h_bounds;
    int32_t n_bounds;
    /* Optional device output: subset index (0-based) of every vertex of the
     * decomposed side, by original id. */
    int32_t *d_subset;
    /* Optional host output of the range lower bounds theta(1..P_eff) and of
     * theta(P_eff + 1) (UINT64_MAX for the last, open range): room for
     * h_bounds_cap values; *h_p_eff receives the number of subsets made. */
    uint64_t *h_bounds_out;
    int32_t h_bounds_cap;
    int32_t *h_p_eff;
    /* Non-zero: record per-phase CUDA-event timings in the graph's stats. */
    int32_t timing;
    /* Tier thresholds of the peel update (0 = built-in defaults): anchors
     * with at most warp_max_w wedges (<= 256) use one warp each; anchors with
     * more than slice_min_w wedges aggregate key slice by key slice. They
     * change speed only, never results. */
    int32_t warp_max_w;
    int32_t slice_min_w;
    /* Non-zero turns off dynamic graph maintenance (Sec. 4.2: between ranges
     * the coarse-grained step drops peeled vertices from a working copy of
     * the adjacency lists). Speed only; results are the same. */
    int32_t no_dgm;
    /* Share of the live adjacency entries that must belong to assigned
     * vertices before the lists are compacted again, in 1/1024 units
     * (0 = 128, i.e. 1/8). Speed only. */
    int32_t dgm_frac_1024;
    /* Fine-grained step (Algorithm 4): subsets whose wedge count (the LPT key
     * of Sec. 3.2.1, sum of L(L-1) over the runs L of G_i) is at least this
     * are peeled by all CTAs level by level instead of by one CTA of the
     * persistent queue. 0 = automatic: 8 times the total weight divided by
     * the smaller of the CTA count and the task count, or by the CTA count
     * when there are at most half as many tasks as CTAs; at least 2^23; and
     * also every task whose weight plus 2^15 per member exceeds the CTA
     * count's share of the total of those sums while its wedges are at
     * least 4 x 2^15 per member (walk-bound). A level of such a task with at
     * most 32 members with big walks spreads each one's walk over the CTAs
     * in equal wedge shares. -1 = never. Speed only. */
    int64_t fd_heavy_w;
    /* How the synchronisation rounds of Algorithm 3 are launched.
     * 0 (default): device-driven; the rounds of a range run inside one
     * launch of a CUDA graph whose while-node repeats the round body until
     * a round leaves no next activeSet (at most 64 rounds a launch), each
     * round's counters going to a device record that the host reads after
     * the launch; with timing on or the activeSet found by crossings the
     * rounds run as with -1. 1: every round is one launch of a CUDA graph
     * captured once per call (the round's kernels, the copy of its counters
     * to the host and the advance), with a host round trip per round.
     * -1: every round's kernels are launched separately, with a host round
     * trip per round. Speed only. */
    int32_t round_graphs;
    /* Hybrid update computation (Sec. 4.1). When the first activeSet of a
     * range of Algorithm 3 carries C_peel wedges (sum over its vertices x
     * of sum_{y in N_x} d_y) and C_peel > factor * C_rcnt, where C_rcnt
     * is the sum over all edges (u, v) of min(d_u, d_v), the round
     * recounts the butterflies of the remaining subgraph (Algorithm 1 with
     * every assigned vertex removed) instead of applying the activeSet's
     * updates (when free device memory holds the recount's temporaries).
     * huc: 0 = that rule, -1 = never, 1 = recount the first round of every
     * range (test hook). huc_factor_1024: the factor in
     * 1/1024 units (0 = 8192, i.e. 8; 1024 is the paper's rule C_peel >
     * C_rcnt). Speed only; results are the same. */
    int32_t huc;
    int32_t huc_factor_1024;
    /* Shape of the key-sliced tier of the peel update (anchors with many
     * wedges, aggregated one key slice at a time): 1 = one 1,024-thread CTA
     * per SM over 98,304-key slices, 2 = two 512-thread CTAs per SM over
     * 49,152-key slices, 4 (or 0) = four 256-thread CTAs per SM over
     * 22,016-key slices. Speed only. */
    int32_t slice_ctas;
    /* How the activeSet of a range's later rounds is found: >= 0 (default)
     * by a scan of the remaining vertices after each round (support <
     * theta(i+1)), so the support decrements need no returned value; -1 from
     * the support atomics' returned values (a vertex joins when its own
     * decrement crosses theta(i+1)). Speed only. */
    int32_t scan_frontier;
    /* Hybrid update computation inside the fine-grained step (Sec. 4.1, its
     * last paragraph), for the tasks peeled by all CTAs (see fd_heavy_w): a
     * member's support is the butterflies it shares with higher subsets
     * (init minus its count inside G_i) plus its count among the task's
     * members still alive, so a level may recount those instead of
     * applying its updates. 0 = a level recounts when its peeled members'
     * walks inside G_i exceed factor * C_rcnt(G_i) (the factor of huc),
     * -1 = never, 1 = every level with updates recounts (test hook). Speed
     * only; results are the same. */
    int32_t fd_huc;
    /* At most this many vertices per range of Algorithm 3 (the range bound
     * stops early when the remaining vertices below it reach the cap):
     * 0 = 2 n / P, -1 = no cap (wedges alone decide, Sec. 3.1.1). A range of
     * many vertices with small walks holds few wedges but as many levels of
     * Algorithm 4 as distinct supports. Speed only (Theorem 2). */
    int32_t range_max_n;
    /* Key-sliced tier: (anchor, slice) items a CTA takes per work-counter
     * atomic, consecutive slices of one anchor (1..32; 0 = 1). Speed only. */
    int32_t slice_fetch;
} receipt_options;

/* Counters of the last call on a graph (Sec. 5: wedges and rounds). */
typedef struct {
    uint64_t wedges_count;   /* wedges traversed by Algorithm 1              */
    uint64_t wedges_cd;      /* wedges of the coarse-grained step's peeled
                                vertices on the whole graph (their walks
                                before dynamic graph maintenance shortens
                                the lists; peel_wedges has what was walked) */
    uint64_t wedges_fd;      /* wedges traversed by fine-grained peeling     */
    uint64_t wedges_bup;     /* sum over the other side of d(d-1): the wedge
                                count of bottom-up peeling, a graph property */
    int64_t rounds_cd;       /* synchronisation rounds of Algorithm 3 (rho)  */
    int64_t levels_fd;       /* peeling levels summed over all subsets       */
    int32_t p_eff;           /* subsets actually created                     */
    int32_t reserved;
    /* Phase device times (CUDA events around each phase, recorded on every
     * call; ms_csr is not measured here and stays 0). */
    float ms_csr, ms_count, ms_cd, ms_fd, ms_total;
    /* Batched peel update of the coarse-grained step, per aggregation tier
     * (0 = warp table, 1 = shared-memory hybrid over the anchor's key window,
     * 2 = global dense counters for hubs, 3 = dense counters over key slices,
     * 4 = dense counters over a key window of at most 36,864 keys):
     * wedges walked, middle vertices (edge visits), anchors (peeled vertices
     * with updates), kernel launches and device time (only if timing != 0). */
    uint64_t peel_wedges[5];
    uint64_t peel_mids[5];
    uint64_t peel_anchors[5];
    int64_t peel_launches[5];
    float ms_peel[5];
    /* Slowest task of the fine-grained step peeled by one CTA: device time,
     * size, levels. */
    float ms_fd_max_subset;
    int32_t fd_max_subset_n;
    int64_t fd_max_subset_levels;
    /* Tasks peeled by all CTAs level by level (see fd_heavy_w), their
     * summed device time (globaltimer) and levels. */
    int32_t fd_heavy_subsets;
    float ms_fd_heavy;
    int64_t levels_fd_heavy;
    /* Tasks of the fine-grained step: one per subset, or, for a batch, one
     * per packed graph's part of a subset (small parts merged). */
    int32_t fd_tasks;
    /* Hybrid update computation (see receipt_options.huc): rounds whose
     * updates were a recount, wedges those recounts traversed, C_rcnt of
     * the graph (0 when the rule was not evaluated) and the recounts'
     * device time (only if timing != 0). */
    int32_t huc_recounts;
    uint64_t wedges_recount;
    uint64_t cost_recount;
    float ms_recount;
    /* Levels of heavy tasks whose big-walk members were each spread over
     * the CTAs (see fd_heavy_w). */
    int32_t fd_split_levels;
    /* Support atomics of the coarse-grained peel update per tier (the same
     * tiers as peel_wedges): one per pair (x, x') of a peeled vertex x and a
     * remaining vertex x' that share at least two neighbours (the pairs whose
     * support changes). */
    uint64_t peel_pairs[5];
    /* Start points of Algorithm 1 per aggregation tier, both sides: warp
     * table, shared hash table (at most 2,048 wedges), shared-memory hybrid,
     * global counters (degree >= 65535 or a key space beyond shared memory),
     * global counters after the hybrid's repeat table overflowed. */
    int64_t count_points[5];
    /* Levels of the fine-grained step's heavy tasks whose updates were a
     * recount (see receipt_options.fd_huc), and the wedges those recounts
     * traversed. */
    int64_t fd_recounts;
    uint64_t wedges_fd_recount;
} receipt_stats;

/* One synchronisation round of the coarse-grained step (Algorithm 3). */
typedef struct {
    int32_t range;        /* 0-based subset index the round belongs to        */
    int32_t frontier;     /* activeSet size (vertices peeled this round)      */
    uint64_t hi;          /* upper bound theta(range + 2) of the range        */
    uint64_t anchors[5];  /* peeled vertices with updates, per peel tier      */
    uint64_t wedges[5];   /* wedges walked, per peel tier                     */
    float ms[5];          /* device time per peel tier (only if timing != 0)  */
    int32_t recount;      /* 1: the round's updates were a recount (HUC)      */
} receipt_round;

/* One subset of the fine-grained step (Algorithm 4, Sec. 3.2.1). */
typedef struct {
    int32_t n;             /* vertices in U_i                                  */
    int32_t heavy;         /* 1: peeled by all CTAs level by level             */
    int64_t levels;        /* peeling levels                                   */
    uint64_t wedges_est;   /* LPT key: sum of L(L-1) over the runs L of G_i    */
    float ms;              /* device time (globaltimer)                        */
    int32_t pad;
} receipt_subset;

/* Fills `opt` with the defaults (P = 150, nothing optional). */
void receipt_options_default(receipt_options *opt);

/*
 * Builds the graph (Algorithm 1, step 1, and the adjacency of Sec. 4.2):
 * removes duplicate edges (dedup != 0; with dedup == 0 a duplicate is an
 * error), relabels each side in descending order of degree (ties by
 * original id; one label space over U u V with U before V on equal degree),
 * and builds the CSR of both sides with every neighbour list sorted by the
 * new labels.
 *   d_eu, d_ev : device int32[m], read only.
 *   m          : number of input edges, 0 <= m < 2^31 (m == 0 is allowed).
 *   nu, nv     : side sizes, >= 0.
 *   out        : receives the new graph; release it with receipt_graph_destroy.
 * Errors: RECEIPT_ERR_INVALID (id out of range, duplicate with dedup == 0,
 * negative sizes), RECEIPT_ERR_OOM, RECEIPT_ERR_CUDA. Synchronises `stream`.
 */
receipt_status receipt_build_csr(const int32_t *d_eu, const int32_t *d_ev, int64_t m,
                                 int32_t nu, int32_t nv, int dedup, void *stream,
                                 receipt_graph **out);

/* Frees a graph and all its device memory (NULL is a no-op). */
receipt_status receipt_graph_destroy(receipt_graph *g);

/* Sizes of a built graph (m after duplicate removal). Any pointer may be NULL. */
receipt_status receipt_graph_info(const receipt_graph *g, int32_t *nu, int32_t *nv,
                                  int64_t *m);

/* Largest degree on each side of a built graph. Any pointer may be NULL. */
receipt_status receipt_graph_max_degree(const receipt_graph *g, int32_t *max_deg_u,
                                        int32_t *max_deg_v);

/*
 * Per-vertex butterfly counts of both sides (Algorithm 1, pvBcnt).
 *   d_cnt_u : device uint64[nu] or NULL; d_cnt_v : device uint64[nv] or NULL.
 * Counts are indexed by original id. Enqueued on `stream`; ready when the
 * stream reaches this point (no host synchronisation).
 */
receipt_status receipt_count_butterflies(receipt_graph *g, uint64_t *d_cnt_u,
                                         uint64_t *d_cnt_v, void *stream);

/*
 * receipt_count_butterflies without any device allocation. The paper has no
 * counterpart: this entry point exists for callers that must not allocate
 * device memory while they run -- for example a serving loop that reserved
 * all of its memory at start-up, or a host framework whose own allocator owns
 * the device -- because cudaMalloc/cudaFree can synchronise the device and
 * fail under a fixed memory budget.
 *   Same arguments, layout and results as receipt_count_butterflies; the
 *   graph must have at most 65,536 vertices on each side and at most
 *   1,048,576 edges (after duplicate removal), else RECEIPT_ERR_INVALID with
 *   a message naming the limits.
 *   Every temporary lives in one fixed array of about 11 MB inside the
 *   library's device image, held on every GPU that loads the library until
 *   the process exits. The first call on a device looks up that array's
 *   device address; make that first call before any stream capture.
 *   All calls share the array and it keeps the previous call's contents
 *   (the call re-zeroes what must start at zero): calls that can overlap on
 *   the GPU -- on different streams or from different threads -- race and
 *   must be serialised by the caller. Enqueued on `stream` with no host
 *   synchronisation; the graph's stats are not updated.
 */
receipt_status receipt_count_butterflies_noalloc(receipt_graph *g, uint64_t *d_cnt_u,
                                                 uint64_t *d_cnt_v, void *stream);

/*
 * Tip decomposition of one side (Algorithms 3 and 4): tip number theta_x of
 * every vertex x of `side`, i.e. the largest k such that x lies in a k-tip
 * (Definition 1).
 *   d_tip : device uint64[n_side], by original id.
 *   opt   : NULL for defaults.
 * Synchronises `stream` once per range and once per peeling round.
 */
receipt_status receipt_tip_decompose(receipt_graph *g, receipt_side side, uint64_t *d_tip,
                                     const receipt_options *opt, void *stream);

/*
 * Tip decomposition of n independent graphs in one pass: the graphs are
 * packed into one disjoint union (tip numbers of a disjoint union are those
 * of its parts), so all of them share the peeling rounds of Algorithm 3 and
 * the persistent task queue of Algorithm 4.
 *   gs[i]     : built graphs (unchanged by the call).
 *   sides[i]  : side to decompose in graph i.
 *   d_tips[i] : device uint64[n_side(i)] outputs by original id.
 */
receipt_status receipt_decompose_batch(receipt_graph *const *gs, const receipt_side *sides,
                                       int32_t n, uint64_t *const *d_tips,
                                       const receipt_options *opt, void *stream);

/*
 * End-to-end convenience over HOST buffers: copies the edge list to the
 * device, builds the graph, decomposes `side`, copies the tip numbers back
 * to h_tip (host uint64[n_side], by original id) and frees everything.
 * Synchronous.
 */
receipt_status receipt_tip_decompose_host(const int32_t *h_eu, const int32_t *h_ev, int64_t m,
                                          int32_t nu, int32_t nv, receipt_side side,
                                          uint64_t *h_tip, const receipt_options *opt,
                                          void *stream);

/* ---------------------------------------------------------------------
 * Serving engine (continuous batching). Not in the paper: it serves many
 * independent decompositions as they arrive. Requests are admitted in
 * arrival order while the device-memory estimate of what is running fits the
 * budget (the oldest request is always admitted when nothing runs); each
 * admitted unit runs on one of `max_inflight` worker streams, so requests
 * that arrive while others are on the GPU overlap with them; requests with at
 * most `batch_max_edges` edges that are waiting together are packed into one
 * disjoint-union decomposition (receipt_decompose_batch). A request's graph
 * and supports stay resident on the device only while it runs.
 * --------------------------------------------------------------------- */
typedef struct receipt_server receipt_server;

typedef struct {
    int32_t max_inflight;     /* worker streams (units running at once); 0 = 4        */
    int32_t P;                /* subsets per decomposition; 0 = 150                   */
    int64_t mem_budget_bytes; /* device bytes admitted units may hold; 0 = 80% of the
                                 free memory when the server is created              */
    int32_t batch_max_edges;  /* requests with at most this many edges may be packed;
                                 0 = never pack (default 200,000)                      */
    int32_t batch_max_graphs; /* at most this many requests per packed unit (64)      */
} receipt_server_config;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t batches;          /* packed units of more than one request                */
    int64_t packed_requests;  /* requests that ran inside such units                  */
    int32_t peak_inflight;    /* most units running at once                           */
    int32_t reserved;
    int64_t peak_inflight_bytes, budget_bytes;
    double p50_ms, p99_ms, mean_ms, max_ms; /* submit -> tips in the caller's buffer  */
    double graphs_per_s;      /* completed / (last completion - first submit)         */
} receipt_server_stats;

/* Fills the defaults (max_inflight 4, P 150, budget 0 = 80% of free memory,
 * batch_max_edges 200,000, batch_max_graphs 64). */
void receipt_server_config_default(receipt_server_config *cfg);

/* Creates a server on the current device and starts its worker threads. */
receipt_status receipt_server_create(const receipt_server_config *cfg, receipt_server **out);

/*
 * Queues one decomposition and returns at once with its id. h_eu/h_ev (m
 * int32 edges, original ids) and h_tip (uint64[n_side] output by original id)
 * are the caller's host buffers and must stay valid until receipt_server_wait
 * returns for this id. RECEIPT_ERR_BUSY once the server is shutting down.
 */
receipt_status receipt_server_submit(receipt_server *sv, const int32_t *h_eu, const int32_t *h_ev,
                                     int64_t m, int32_t nu, int32_t nv, receipt_side side,
                                     uint64_t *h_tip, int64_t *request_id);

/*
 * Waits for a request (timeout_s <= 0: no limit; on timeout returns
 * RECEIPT_ERR_TIMEOUT and the request keeps running), then reports its own
 * status and its latency from submit to completion and forgets the id.
 */
receipt_status receipt_server_wait(receipt_server *sv, int64_t request_id, double timeout_s,
                                   int32_t *request_status, double *latency_ms);

/* Latency percentiles, throughput and admission counters so far. */
receipt_status receipt_server_get_stats(receipt_server *sv, receipt_server_stats *out);

/* Stops the workers after the units they are running; unstarted requests are
 * dropped. */
receipt_status receipt_server_destroy(receipt_server *sv);

/*
 * Upper bound of the butterfly count of any vertex on a side with n_side
 * vertices of degree at most max_deg_side, whose neighbours have degree at
 * most max_deg_other, in a graph of m edges (the count of x is the sum over
 * x' != x of C(|N_x n N_x'|, 2), Sec. 2; every support of Algorithms 2-4
 * starts at the count and only falls). *bound receives the minimum of
 * (n_side - 1) C(max_deg_side, 2), max_deg_side (max_deg_other - 1)
 * (max_deg_side - 1) / 2 and m (max_deg_side - 1) / 2 (UINT64_MAX if above
 * it). Host arithmetic only; no device is needed.
 * Errors: RECEIPT_ERR_OVERFLOW when the bound reaches 2^63 (then counting and
 * decomposition refuse the graph with the same status; with the library's
 * limit m < 2^31 the third term stays below 2^61, so a built graph never
 * does), RECEIPT_ERR_INVALID for negative arguments.
 */
receipt_status receipt_support_bound(int64_t n_side, int32_t max_deg_side,
                                     int32_t max_deg_other, int64_t m, uint64_t *bound);

/* Counters of the last count/decompose call on g. */
receipt_status receipt_get_stats(const receipt_graph *g, receipt_stats *out);

/* Per-round trace of the last tip decomposition on g: copies up to `cap`
 * records to `out` (host array) and the number of rounds to *n_rounds. */
receipt_status receipt_get_trace(const receipt_graph *g, receipt_round *out, int32_t cap,
                                 int32_t *n_rounds);

/* Subsets of the last tip decomposition on g (one record per subset, in
 * subset order): copies up to `cap` records to `out` (host array) and the
 * number of subsets to *n_subsets. */
receipt_status receipt_get_subsets(const receipt_graph *g, receipt_subset *out, int32_t cap,
                                   int32_t *n_subsets);

/* Thread-local text of the last error on the calling thread ("" if none). */
const char *receipt_last_error(void);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t receipt_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* RECEIPT_H */
