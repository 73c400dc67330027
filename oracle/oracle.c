/*
 * CPU oracle for RECEIPT tip decomposition -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, sequential reference implementations written from the paper
 * (Lakhotia, Kannan, Prasanna, De Rose, "RECEIPT: REfine CoarsE-grained
 * IndePendent Tasks for Parallel Tip decomposition of Bipartite Graphs").
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * call it; the CUDA library never does, and the two share no code.
 *
 * Functions:
 *   oracle_count_2hop     -- per-vertex butterfly counts by their definition
 *                            (Sec. 2.1, Table 1: support = # butterflies of u),
 *                            i.e. sum over same-side x' of C(|N_x n N_x'|, 2).
 *   oracle_count_vp       -- Algorithm 1 (pvBcnt), the vertex-priority counter,
 *                            written independently as a cross-check.
 *   oracle_count_vertex   -- listed vertices' counts by the definition (used
 *                            to sample outputs of graphs too large for the
 *                            full oracle); oracle_graph_* keep the adjacency
 *                            built between such calls.
 *   oracle_bup            -- Algorithm 2 (BUP): sequential bottom-up peeling
 *                            with the update of Algorithm 2 (support of every
 *                            2-hop neighbour u' drops by C(wdg[u'],2), clamped
 *                            at the tip number just assigned), with a
 *                            monotone radix heap as the min-support structure.
 *
 * Graph input everywhere: nu, nv, m and two int32 arrays eu[m], ev[m] of
 * original ids. Duplicate edges are removed. Results are indexed by original
 * id. Exact unsigned 64-bit integer arithmetic throughout.
 *
 * Parity pins (see tests/test_oracle.py): brute-force enumeration of pairs
 * and of vertex subsets on tiny graphs, closed forms on K_{a,b}, the
 * 2x-butterflies sum invariant, zero counts on forests, disjoint unions and
 * side transposition.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* ------------------------------------------------------------------ */
/* Adjacency lists (both sides), neighbour lists sorted by original id */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n;      /* vertices on this side */
    int64_t *off;   /* n + 1 */
    int32_t *adj;   /* ids of the other side */
} side_adj;

static void free_side(side_adj *s) {
    free(s->off);
    free(s->adj);
    s->off = NULL;
    s->adj = NULL;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* CSR of side "a" from the (a, b) pairs: place every b in its a's list
 * (counting by a), sort each list, drop repeated entries. */
static int build_side(int64_t na, int64_t nb, int64_t m, const int32_t *ea,
                      const int32_t *eb, side_adj *out) {
    for (int64_t i = 0; i < m; i++)
        if (ea[i] < 0 || ea[i] >= na || eb[i] < 0 || eb[i] >= nb) return ORC_EINVAL;
    out->n = na;
    out->off = (int64_t *)calloc((size_t)na + 1, sizeof(int64_t));
    out->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(na > 0 ? na : 1));
    if (!out->off || !out->adj || !pos) {
        free(pos);
        free_side(out);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < m; i++) out->off[ea[i] + 1]++;
    for (int64_t a = 0; a < na; a++) out->off[a + 1] += out->off[a];
    for (int64_t a = 0; a < na; a++) pos[a] = out->off[a];
    for (int64_t i = 0; i < m; i++) out->adj[pos[ea[i]]++] = eb[i];
    free(pos);
    /* sort every list and keep one copy of each entry, compacting in place */
    int64_t k = 0;
    for (int64_t a = 0; a < na; a++) {
        const int64_t b0 = out->off[a], b1 = out->off[a + 1];
        qsort(out->adj + b0, (size_t)(b1 - b0), sizeof(int32_t), cmp_i32);
        out->off[a] = k;
        for (int64_t i = b0; i < b1; i++)
            if (i == b0 || out->adj[i] != out->adj[i - 1]) out->adj[k++] = out->adj[i];
    }
    out->off[na] = k;
    return ORC_OK;
}

static int build_both(int32_t nu, int32_t nv, int64_t m, const int32_t *eu,
                      const int32_t *ev, side_adj *U, side_adj *V) {
    if (nu < 0 || nv < 0 || m < 0) return ORC_EINVAL;
    int rc = build_side(nu, nv, m, eu, ev, U);
    if (rc) return rc;
    rc = build_side(nv, nu, m, ev, eu, V);
    if (rc) {
        free_side(U);
        return rc;
    }
    return ORC_OK;
}

static inline uint64_t choose2(uint64_t c) { return c * (c - 1) / 2; }

/* ------------------------------------------------------------------ */
/* Counting by definition: butterflies of x = sum_{x' != x} C(c(x,x'),2) */
/* where c(x,x') = |N_x n N_x'|, found by walking the 2-hop neighbourhood */
/* ------------------------------------------------------------------ */

static int count_side_2hop(const side_adj *S, const side_adj *O, uint64_t *cnt) {
    int64_t n = S->n;
    int err = 0;
#pragma omp parallel
    {
        uint32_t *c = (uint32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(uint32_t));
        int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        if (!c || !touched) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t x = 0; x < n; x++) {
                int64_t nt = 0;
                for (int64_t i = S->off[x]; i < S->off[x + 1]; i++) {
                    int32_t y = S->adj[i];
                    for (int64_t j = O->off[y]; j < O->off[y + 1]; j++) {
                        int32_t xp = O->adj[j];
                        if (xp == x) continue;
                        if (c[xp]++ == 0) touched[nt++] = xp;
                    }
                }
                uint64_t s = 0;
                for (int64_t t = 0; t < nt; t++) {
                    s += choose2(c[touched[t]]);
                    c[touched[t]] = 0;
                }
                cnt[x] = s;
            }
        }
        free(c);
        free(touched);
    }
    return err ? ORC_ENOMEM : ORC_OK;
}

int oracle_count_2hop(int32_t nu, int32_t nv, int64_t m, const int32_t *eu,
                      const int32_t *ev, uint64_t *cnt_u, uint64_t *cnt_v) {
    side_adj U, V;
    int rc = build_both(nu, nv, m, eu, ev, &U, &V);
    if (rc) return rc;
    if (cnt_u) rc = count_side_2hop(&U, &V, cnt_u);
    if (!rc && cnt_v) rc = count_side_2hop(&V, &U, cnt_v);
    free_side(&U);
    free_side(&V);
    return rc;
}

/* The listed vertices xs[0..nx) of side S, by the same definition;
 * *walked receives the 2-hop entries visited (sum over y in N_x of d_y). */
static int count_listed(const side_adj *S, const side_adj *O, const int32_t *xs, int64_t nx,
                        uint64_t *out, uint64_t *walked) {
    int rc = ORC_OK;
    uint64_t w = 0;
    uint32_t *c = (uint32_t *)calloc((size_t)(S->n > 0 ? S->n : 1), sizeof(uint32_t));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S->n > 0 ? S->n : 1));
    if (!c || !touched) rc = ORC_ENOMEM;
    for (int64_t q = 0; q < nx && !rc; q++) {
        int32_t x = xs[q];
        if (x < 0 || x >= S->n) {
            rc = ORC_EINVAL;
            break;
        }
        int64_t nt = 0;
        for (int64_t i = S->off[x]; i < S->off[x + 1]; i++) {
            int32_t y = S->adj[i];
            w += (uint64_t)(O->off[y + 1] - O->off[y]);
            for (int64_t j = O->off[y]; j < O->off[y + 1]; j++) {
                int32_t xp = O->adj[j];
                if (xp == x) continue;
                if (c[xp]++ == 0) touched[nt++] = xp;
            }
        }
        uint64_t s = 0;
        for (int64_t t = 0; t < nt; t++) {
            s += choose2(c[touched[t]]);
            c[touched[t]] = 0;
        }
        out[q] = s;
    }
    free(c);
    free(touched);
    if (walked) *walked = w;
    return rc;
}

/* Vertices x of side `side` (0 = U, 1 = V), by the same definition. */
int oracle_count_vertex(int32_t nu, int32_t nv, int64_t m, const int32_t *eu,
                        const int32_t *ev, int side, const int32_t *xs, int64_t nx,
                        uint64_t *out) {
    side_adj U, V;
    int rc = build_both(nu, nv, m, eu, ev, &U, &V);
    if (rc) return rc;
    rc = count_listed(side ? &V : &U, side ? &U : &V, xs, nx, out, NULL);
    free_side(&U);
    free_side(&V);
    return rc;
}

/* The same count on a graph whose adjacency is built once and kept, so that
 * repeated calls (a timed sample of vertices) do not rebuild it. */
typedef struct {
    side_adj U, V;
} oracle_graph;

void *oracle_graph_new(int32_t nu, int32_t nv, int64_t m, const int32_t *eu, const int32_t *ev,
                       int *rc) {
    oracle_graph *g = (oracle_graph *)calloc(1, sizeof(oracle_graph));
    if (!g) {
        *rc = ORC_ENOMEM;
        return NULL;
    }
    *rc = build_both(nu, nv, m, eu, ev, &g->U, &g->V);
    if (*rc) {
        free(g);
        return NULL;
    }
    return g;
}

int oracle_graph_count_vertex(void *h, int side, const int32_t *xs, int64_t nx, uint64_t *out,
                              uint64_t *walked) {
    oracle_graph *g = (oracle_graph *)h;
    if (!g) return ORC_EINVAL;
    return count_listed(side ? &g->V : &g->U, side ? &g->U : &g->V, xs, nx, out, walked);
}

void oracle_graph_free(void *h) {
    oracle_graph *g = (oracle_graph *)h;
    if (!g) return;
    free_side(&g->U);
    free_side(&g->V);
    free(g);
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 (pvBcnt): vertex-priority per-vertex counting           */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t deg;
    int32_t side;
    int32_t id;
} vkey;

static int cmp_vkey(const void *a, const void *b) {
    const vkey *x = (const vkey *)a, *y = (const vkey *)b;
    if (x->deg != y->deg) return x->deg > y->deg ? -1 : 1; /* descending degree */
    if (x->side != y->side) return x->side < y->side ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

int oracle_count_vp(int32_t nu, int32_t nv, int64_t m, const int32_t *eu,
                    const int32_t *ev, uint64_t *cnt_u, uint64_t *cnt_v) {
    side_adj U, V;
    int rc = build_both(nu, nv, m, eu, ev, &U, &V);
    if (rc) return rc;
    int64_t n = (int64_t)nu + nv;
    /* Step 1: one label space over W = U u V in descending order of degree. */
    vkey *order = (vkey *)malloc(sizeof(vkey) * (size_t)(n > 0 ? n : 1));
    int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *old = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t mm = U.off[nu];
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * mm + 1));
    uint32_t *wdg = (uint32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(uint32_t));
    int32_t *nze = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    uint64_t *bc = (uint64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(uint64_t));
    if (!order || !lab || !old || !off || !adj || !wdg || !nze || !bc) {
        rc = ORC_ENOMEM;
        goto done;
    }
    for (int32_t u = 0; u < nu; u++) {
        order[u].deg = U.off[u + 1] - U.off[u];
        order[u].side = 0;
        order[u].id = u;
    }
    for (int32_t v = 0; v < nv; v++) {
        order[nu + v].deg = V.off[v + 1] - V.off[v];
        order[nu + v].side = 1;
        order[nu + v].id = v;
    }
    qsort(order, (size_t)n, sizeof(vkey), cmp_vkey);
    for (int64_t l = 0; l < n; l++) {
        int64_t w = order[l].side ? (int64_t)nu + order[l].id : order[l].id;
        lab[w] = (int32_t)l;
        old[l] = (int32_t)w;
    }
    /* Relabelled adjacency of every vertex, sorted ascending by new label. */
    for (int64_t l = 0; l < n; l++) {
        int64_t w = old[l];
        const side_adj *S = w < nu ? &U : &V;
        int64_t x = w < nu ? w : w - nu;
        off[l + 1] = off[l] + (S->off[x + 1] - S->off[x]);
    }
    for (int64_t l = 0; l < n; l++) {
        int64_t w = old[l];
        int is_v = w >= nu;
        const side_adj *S = is_v ? &V : &U;
        int64_t x = is_v ? w - nu : w;
        int64_t p = off[l];
        for (int64_t i = S->off[x]; i < S->off[x + 1]; i++) {
            int64_t nb = is_v ? S->adj[i] : (int64_t)nu + S->adj[i];
            adj[p++] = lab[nb];
        }
        qsort(adj + off[l], (size_t)(off[l + 1] - off[l]), sizeof(int32_t), cmp_i32);
    }
    /* Wedges sp -> mp -> ep with ep the lowest label of the three. */
    for (int64_t sp = 0; sp < n; sp++) {
        int64_t nz = 0;
        for (int64_t i = off[sp]; i < off[sp + 1]; i++) {
            int32_t mp = adj[i];
            for (int64_t j = off[mp]; j < off[mp + 1]; j++) {
                int32_t ep = adj[j];
                if (ep >= mp || ep >= sp) break;
                if (wdg[ep]++ == 0) nze[nz++] = ep;
            }
        }
        /* same-side contribution: C(wdg,2) to ep and to sp */
        for (int64_t t = 0; t < nz; t++) {
            uint64_t b = choose2(wdg[nze[t]]);
            bc[nze[t]] += b;
            bc[sp] += b;
        }
        /* opposite-side contribution: wdg[ep]-1 to mp for every wedge */
        for (int64_t i = off[sp]; i < off[sp + 1]; i++) {
            int32_t mp = adj[i];
            for (int64_t j = off[mp]; j < off[mp + 1]; j++) {
                int32_t ep = adj[j];
                if (ep >= mp || ep >= sp) break;
                bc[mp] += (uint64_t)wdg[ep] - 1;
            }
        }
        for (int64_t t = 0; t < nz; t++) wdg[nze[t]] = 0;
    }
    for (int64_t l = 0; l < n; l++) {
        int64_t w = old[l];
        if (w < nu) {
            if (cnt_u) cnt_u[w] = bc[l];
        } else if (cnt_v) {
            cnt_v[w - nu] = bc[l];
        }
    }
done:
    free(order);
    free(lab);
    free(old);
    free(off);
    free(adj);
    free(wdg);
    free(nze);
    free(bc);
    free_side(&U);
    free_side(&V);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Monotone radix heap over vertices keyed by their current support    */
/* Keys never drop below the last key popped (the clamp of Algorithm   */
/* 2 guarantees it). Bucket b holds vertices whose key's highest bit    */
/* differing from `last` is bit b-1 (bucket 0: key == last). A vertex   */
/* is filed again only when its bucket changes, and where[v] names the  */
/* bucket of its live entry, so older entries are recognised as stale  */
/* and a vertex has at most 66 entries over the whole peel.             */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t *b[65];
    size_t n[65], cap[65];
    uint64_t last;
    const uint64_t *key; /* current key of every vertex (its support) */
    int8_t *where;       /* bucket of the vertex's live entry, -1: none */
} radix_heap;

static int rh_bucket(uint64_t key, uint64_t last) {
    return key == last ? 0 : 64 - __builtin_clzll(key ^ last);
}

static int rh_append(radix_heap *h, int b, int32_t v) {
    if (h->n[b] == h->cap[b]) {
        size_t nc = h->cap[b] ? 2 * h->cap[b] : 16;
        int32_t *p = (int32_t *)realloc(h->b[b], nc * sizeof(int32_t));
        if (!p) return ORC_ENOMEM;
        h->b[b] = p;
        h->cap[b] = nc;
    }
    h->b[b][h->n[b]++] = v;
    return ORC_OK;
}

/* Files v under its current key (after it was set or lowered). */
static int rh_put(radix_heap *h, int32_t v) {
    if (h->key[v] < h->last) return ORC_EINVAL; /* monotonicity violated */
    int b = rh_bucket(h->key[v], h->last);
    if (h->where[v] == b) return ORC_OK; /* its live entry is in the right bucket */
    h->where[v] = (int8_t)b;
    return rh_append(h, b, v);
}

/* Pops a vertex with the minimum key into *v; returns 1, 0 if no vertex is
 * filed, or minus an ORC_ code on failure. */
static int rh_pop(radix_heap *h, int32_t *v) {
    for (;;) {
        while (h->n[0] > 0) {
            int32_t u = h->b[0][--h->n[0]];
            if (h->where[u] == 0) {
                h->where[u] = -1;
                *v = u;
                return 1;
            }
        }
        int b = 1;
        while (b < 65 && h->n[b] == 0) b++;
        if (b == 65) return 0;
        /* the smallest key among the live entries of bucket b is the new
         * `last`; they all move to lower buckets */
        int32_t *items = h->b[b];
        size_t cnt = h->n[b];
        h->b[b] = NULL;
        h->n[b] = 0;
        h->cap[b] = 0;
        uint64_t mn = UINT64_MAX;
        for (size_t i = 0; i < cnt; i++)
            if (h->where[items[i]] == b && h->key[items[i]] < mn) mn = h->key[items[i]];
        if (mn != UINT64_MAX) {
            h->last = mn;
            for (size_t i = 0; i < cnt; i++) {
                int32_t u = items[i];
                if (h->where[u] != b) continue; /* stale entry */
                h->where[u] = -1;
                int rc = rh_put(h, u);
                if (rc) {
                    free(items);
                    return -rc;
                }
            }
        }
        free(items);
    }
}

static void rh_free(radix_heap *h) {
    for (int b = 0; b < 65; b++) free(h->b[b]);
}

/* ------------------------------------------------------------------ */
/* Algorithm 2 (BUP)                                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t wedges;       /* wedges traversed by the update calls          */
    int64_t peeled;        /* vertices peeled                               */
    double seconds_count;  /* wall time of the initial count                */
    double seconds_peel;   /* wall time of the peeling loop                 */
    int64_t complete;      /* 1 if every vertex was peeled                  */
} oracle_bup_stats;

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/*
 * Tip numbers of side `side` (0 = U, 1 = V) by sequential bottom-up peeling.
 * `max_wedges` > 0 stops the peel once that many wedges were traversed (the
 * CPU-baseline sample); tips of unpeeled vertices are then left untouched.
 */
static int bup_impl(int32_t nu, int32_t nv, int64_t m, const int32_t *eu, const int32_t *ev,
                    int side, const uint64_t *sup0, uint64_t *tip, uint64_t max_wedges,
                    oracle_bup_stats *st);

int oracle_bup(int32_t nu, int32_t nv, int64_t m, const int32_t *eu, const int32_t *ev,
               int side, uint64_t *tip, uint64_t max_wedges, oracle_bup_stats *st) {
    return bup_impl(nu, nv, m, eu, ev, side, NULL, tip, max_wedges, st);
}

/* Same peel, started from given initial supports sup0 (the butterfly counts
 * of the decomposed side, e.g. from oracle_count_2hop) instead of counting
 * them again; used to time bounded peel samples. */
int oracle_bup_from_counts(int32_t nu, int32_t nv, int64_t m, const int32_t *eu,
                           const int32_t *ev, int side, const uint64_t *sup0, uint64_t *tip,
                           uint64_t max_wedges, oracle_bup_stats *st) {
    if (!sup0) return ORC_EINVAL;
    return bup_impl(nu, nv, m, eu, ev, side, sup0, tip, max_wedges, st);
}

static int bup_impl(int32_t nu, int32_t nv, int64_t m, const int32_t *eu, const int32_t *ev,
                    int side, const uint64_t *sup0, uint64_t *tip, uint64_t max_wedges,
                    oracle_bup_stats *st) {
    side_adj U, V;
    int rc = build_both(nu, nv, m, eu, ev, &U, &V);
    if (rc) return rc;
    const side_adj *S = side ? &V : &U, *O = side ? &U : &V;
    int64_t n = S->n;
    uint64_t *sup = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *peeled = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    uint32_t *c = (uint32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(uint32_t));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int8_t *where = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
    radix_heap h;
    memset(&h, 0, sizeof(h));
    h.key = sup;
    h.where = where;
    oracle_bup_stats s;
    memset(&s, 0, sizeof(s));
    if (!sup || !peeled || !c || !touched || !where) {
        rc = ORC_ENOMEM;
        goto done;
    }
    double t0 = now_s();
    if (sup0)
        memcpy(sup, sup0, sizeof(uint64_t) * (size_t)n);
    else
        rc = count_side_2hop(S, O, sup); /* initial supports: butterflies of x in G */
    if (rc) goto done;
    double t1 = now_s();
    s.seconds_count = t1 - t0;
    memset(where, -1, (size_t)n);
    for (int64_t x = 0; x < n; x++)
        if ((rc = rh_put(&h, (int32_t)x))) goto done;
    int32_t x;
    int got;
    while ((got = rh_pop(&h, &x)) != 0) {
        if (got < 0) {
            rc = -got;
            goto done;
        }
        if (max_wedges && s.wedges >= max_wedges) break;
        uint64_t theta = sup[x]; /* minimum support: x's tip number */
        tip[x] = theta;
        peeled[x] = 1;
        s.peeled++;
        /* update(x, theta): common-neighbour counts over the 2-hop walk */
        int64_t nt = 0;
        for (int64_t i = S->off[x]; i < S->off[x + 1]; i++) {
            int32_t y = S->adj[i];
            s.wedges += (uint64_t)(O->off[y + 1] - O->off[y]);
            for (int64_t j = O->off[y]; j < O->off[y + 1]; j++) {
                int32_t xp = O->adj[j];
                if (xp == x || peeled[xp]) continue;
                if (c[xp]++ == 0) touched[nt++] = xp;
            }
        }
        for (int64_t t = 0; t < nt; t++) {
            int32_t xp = touched[t];
            uint64_t b = choose2(c[xp]);
            c[xp] = 0;
            if (b == 0) continue;
            /* support of x' <- max(theta, support of x' - shared butterflies) */
            uint64_t nv2 = (sup[xp] >= b && sup[xp] - b >= theta) ? sup[xp] - b : theta;
            if (nv2 != sup[xp]) {
                sup[xp] = nv2;
                if ((rc = rh_put(&h, xp))) goto done;
            }
        }
    }
    s.seconds_peel = now_s() - t1;
    s.complete = (s.peeled == n);
done:
    if (st) *st = s;
    rh_free(&h);
    free(where);
    free(sup);
    free(peeled);
    free(c);
    free(touched);
    free_side(&U);
    free_side(&V);
    return rc;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
