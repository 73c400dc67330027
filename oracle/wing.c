/*
 * CPU oracle for wing decomposition (edge peeling) -- TEST INFRASTRUCTURE ONLY.
 *
 * The paper's extensions section (Sec. 7, parallel edge peeling) carries
 * RECEIPT over from vertices to edges: the support of an edge is the number
 * of butterflies that contain it, a k-wing is a subgraph in which every edge
 * lies in at least k of the subgraph's butterflies, and the wing number of an
 * edge is the largest k such that some k-wing contains it (the edge analogue
 * of Definition 1). Only the tests may call these functions; the CUDA
 * library never does, and the two share no code.
 *
 * Functions:
 *   oracle_edge_count -- butterflies of every edge by their definition:
 *                        for edge (u, v), the sum over u' in N_v, u' != u,
 *                        of |N_u n N_u'| - 1 (the common neighbours of u and
 *                        u' other than v close one butterfly each).
 *   oracle_wing_bup   -- sequential bottom-up edge peeling, the edge analogue
 *                        of Algorithm 2: repeatedly remove an edge of minimum
 *                        support, record its support as its wing number, and
 *                        take one from the support of the other three edges
 *                        of every butterfly it still closes, clamped at the
 *                        wing number just recorded.
 *
 * Edges are reported in the order of the U side's sorted lists: by u, then
 * by v (duplicates removed). Exact unsigned 64-bit arithmetic throughout.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

typedef struct {
    int64_t nu, nv, m;
    int64_t *uoff; /* nu + 1: edges of u are uoff[u] .. uoff[u+1]-1 (edge ids) */
    int32_t *uadj; /* m: v of edge e */
    int64_t *voff; /* nv + 1 */
    int32_t *vadj; /* m: u of the v-side entry */
    int64_t *veid; /* m: edge id of the v-side entry */
} egraph;

static void eg_free(egraph *g) {
    free(g->uoff);
    free(g->uadj);
    free(g->voff);
    free(g->vadj);
    free(g->veid);
    memset(g, 0, sizeof(*g));
}

static int cmp_key(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Sorted, duplicate-free edge list with both sides' lists and the edge id of
 * every V-side entry. */
static int eg_build(int32_t nu, int32_t nv, int64_t m, const int32_t *eu, const int32_t *ev,
                    egraph *g) {
    memset(g, 0, sizeof(*g));
    if (nu < 0 || nv < 0 || m < 0) return ORC_EINVAL;
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
    if (!key) return ORC_ENOMEM;
    for (int64_t i = 0; i < m; i++) {
        if (eu[i] < 0 || eu[i] >= nu || ev[i] < 0 || ev[i] >= nv) {
            free(key);
            return ORC_EINVAL;
        }
        key[i] = ((uint64_t)(uint32_t)eu[i] << 32) | (uint32_t)ev[i];
    }
    qsort(key, (size_t)m, sizeof(uint64_t), cmp_key);
    int64_t k = 0;
    for (int64_t i = 0; i < m; i++)
        if (i == 0 || key[i] != key[i - 1]) key[k++] = key[i];
    g->nu = nu;
    g->nv = nv;
    g->m = k;
    size_t mk = (size_t)(k > 0 ? k : 1);
    g->uoff = (int64_t *)calloc((size_t)nu + 1, sizeof(int64_t));
    g->uadj = (int32_t *)malloc(sizeof(int32_t) * mk);
    g->voff = (int64_t *)calloc((size_t)nv + 1, sizeof(int64_t));
    g->vadj = (int32_t *)malloc(sizeof(int32_t) * mk);
    g->veid = (int64_t *)malloc(sizeof(int64_t) * mk);
    int64_t *fill = (int64_t *)calloc((size_t)nv + 1, sizeof(int64_t));
    if (!g->uoff || !g->uadj || !g->voff || !g->vadj || !g->veid || !fill) {
        free(key);
        free(fill);
        eg_free(g);
        return ORC_ENOMEM;
    }
    for (int64_t e = 0; e < k; e++) {
        int32_t u = (int32_t)(key[e] >> 32), v = (int32_t)(key[e] & 0xffffffffu);
        g->uoff[u + 1]++;
        g->voff[v + 1]++;
        g->uadj[e] = v;
    }
    for (int64_t u = 0; u < nu; u++) g->uoff[u + 1] += g->uoff[u];
    for (int64_t v = 0; v < nv; v++) g->voff[v + 1] += g->voff[v];
    /* edges in ascending (u, v) order: each v's list comes out ascending in u */
    for (int64_t e = 0; e < k; e++) {
        int32_t u = (int32_t)(key[e] >> 32), v = (int32_t)(key[e] & 0xffffffffu);
        int64_t p = g->voff[v] + fill[v]++;
        g->vadj[p] = u;
        g->veid[p] = e;
    }
    free(fill);
    free(key);
    return ORC_OK;
}

/* Butterflies of every edge by the definition in the header comment. */
static int edge_count(const egraph *g, uint64_t *cnt) {
    uint32_t *c = (uint32_t *)calloc((size_t)(g->nu > 0 ? g->nu : 1), sizeof(uint32_t));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->nu > 0 ? g->nu : 1));
    if (!c || !touched) {
        free(c);
        free(touched);
        return ORC_ENOMEM;
    }
    for (int64_t u = 0; u < g->nu; u++) {
        /* c[u'] = |N_u n N_u'| for every u' != u two hops away */
        int64_t nt = 0;
        for (int64_t e = g->uoff[u]; e < g->uoff[u + 1]; e++) {
            int32_t v = g->uadj[e];
            for (int64_t j = g->voff[v]; j < g->voff[v + 1]; j++) {
                int32_t up = g->vadj[j];
                if (up == u) continue;
                if (c[up]++ == 0) touched[nt++] = up;
            }
        }
        for (int64_t e = g->uoff[u]; e < g->uoff[u + 1]; e++) {
            int32_t v = g->uadj[e];
            uint64_t s = 0;
            for (int64_t j = g->voff[v]; j < g->voff[v + 1]; j++) {
                int32_t up = g->vadj[j];
                if (up != u) s += (uint64_t)c[up] - 1; /* v itself is common */
            }
            cnt[e] = s;
        }
        for (int64_t t = 0; t < nt; t++) c[touched[t]] = 0;
    }
    free(c);
    free(touched);
    return ORC_OK;
}

int oracle_edge_count(int32_t nu, int32_t nv, int64_t m, const int32_t *eu, const int32_t *ev,
                      int32_t *out_u, int32_t *out_v, uint64_t *cnt, int64_t *m_out) {
    egraph g;
    int rc = eg_build(nu, nv, m, eu, ev, &g);
    if (rc) return rc;
    rc = edge_count(&g, cnt);
    for (int64_t u = 0; u < g.nu && !rc; u++)
        for (int64_t e = g.uoff[u]; e < g.uoff[u + 1]; e++) {
            out_u[e] = (int32_t)u;
            out_v[e] = g.uadj[e];
        }
    *m_out = g.m;
    eg_free(&g);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Indexed binary min-heap over edge ids, keyed by (support, edge id);  */
/* supports only decrease while an edge is in the heap.                 */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    int64_t *heap; /* edge ids */
    int64_t *pos;  /* position of each edge in heap, -1 once popped */
    const uint64_t *key;
} eheap;

static int eh_less(const eheap *h, int64_t a, int64_t b) {
    return h->key[a] < h->key[b] || (h->key[a] == h->key[b] && a < b);
}

static void eh_swap(eheap *h, int64_t i, int64_t j) {
    int64_t a = h->heap[i], b = h->heap[j];
    h->heap[i] = b;
    h->heap[j] = a;
    h->pos[b] = i;
    h->pos[a] = j;
}

static void eh_up(eheap *h, int64_t i) {
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!eh_less(h, h->heap[i], h->heap[p])) break;
        eh_swap(h, i, p);
        i = p;
    }
}

static void eh_down(eheap *h, int64_t i) {
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < h->n && eh_less(h, h->heap[l], h->heap[s])) s = l;
        if (r < h->n && eh_less(h, h->heap[r], h->heap[s])) s = r;
        if (s == i) break;
        eh_swap(h, i, s);
        i = s;
    }
}

static int64_t eh_pop(eheap *h) {
    int64_t top = h->heap[0];
    h->n--;
    if (h->n > 0) {
        h->heap[0] = h->heap[h->n];
        h->pos[h->heap[0]] = 0;
        eh_down(h, 0);
    }
    h->pos[top] = -1;
    return top;
}

typedef struct {
    uint64_t butterflies_visited; /* butterflies whose supports were updated */
    uint64_t edges_scanned;       /* adjacency entries read by the peel      */
    int64_t peeled;               /* edges peeled                            */
    int64_t complete;             /* 1 if every edge was peeled              */
} wing_stats;

int oracle_wing_bup(int32_t nu, int32_t nv, int64_t m, const int32_t *eu, const int32_t *ev,
                    int32_t *out_u, int32_t *out_v, uint64_t *wing, int64_t *m_out,
                    wing_stats *st) {
    egraph g;
    int rc = eg_build(nu, nv, m, eu, ev, &g);
    if (rc) return rc;
    const int64_t k = g.m;
    size_t mk = (size_t)(k > 0 ? k : 1);
    uint64_t *sup = (uint64_t *)malloc(sizeof(uint64_t) * mk);
    uint8_t *gone = (uint8_t *)calloc(mk, 1);
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(g.nv > 0 ? g.nv : 1));
    int32_t *eu_of = (int32_t *)malloc(sizeof(int32_t) * mk); /* edge id -> its u */
    eheap h = {k, (int64_t *)malloc(sizeof(int64_t) * mk), (int64_t *)malloc(sizeof(int64_t) * mk),
               sup};
    wing_stats s = {0, 0, 0, 0};
    if (!sup || !gone || !mark || !eu_of || !h.heap || !h.pos) {
        rc = ORC_ENOMEM;
        goto done;
    }
    rc = edge_count(&g, sup);
    if (rc) goto done;
    for (int64_t v = 0; v < g.nv; v++) mark[v] = -1;
    for (int64_t e = 0; e < k; e++) {
        h.heap[e] = e;
        h.pos[e] = e;
    }
    for (int64_t i = k / 2 - 1; i >= 0; i--) eh_down(&h, i);
    uint64_t level = 0;
    for (int64_t u = 0; u < g.nu; u++)
        for (int64_t e = g.uoff[u]; e < g.uoff[u + 1]; e++) eu_of[e] = (int32_t)u;
    while (h.n > 0) {
        const int64_t e = eh_pop(&h);
        const uint64_t th = sup[e] > level ? sup[e] : level;
        wing[e] = th;
        level = th;
        gone[e] = 1;
        s.peeled++;
        const int32_t u = eu_of[e], v = g.uadj[e];
        /* mark[v'] = id of the live edge (u, v'), v' != v */
        for (int64_t f = g.uoff[u]; f < g.uoff[u + 1]; f++)
            if (!gone[f]) mark[g.uadj[f]] = f;
        s.edges_scanned += (uint64_t)(g.uoff[u + 1] - g.uoff[u]);
        /* every live (u', v) with u' != u, and every live (u', v') with
         * (u, v') live: the butterfly {u, u'} x {v, v'} loses edge e */
        for (int64_t j = g.voff[v]; j < g.voff[v + 1]; j++) {
            const int64_t f1 = g.veid[j]; /* (u', v) */
            const int32_t up = g.vadj[j];
            if (up == u || gone[f1]) continue;
            s.edges_scanned += (uint64_t)(g.uoff[up + 1] - g.uoff[up]);
            for (int64_t f3 = g.uoff[up]; f3 < g.uoff[up + 1]; f3++) { /* (u', v') */
                const int32_t vp = g.uadj[f3];
                if (vp == v || gone[f3]) continue;
                const int64_t f2 = mark[vp]; /* (u, v') */
                if (f2 < 0) continue;
                s.butterflies_visited++;
                const int64_t others[3] = {f1, f2, f3};
                for (int t = 0; t < 3; t++) {
                    /* sup <- max(th, sup - 1), the clamp of Algorithm 2
                     * (a live edge's support is never below th) */
                    const int64_t o = others[t];
                    if (sup[o] > th) {
                        sup[o]--;
                        eh_up(&h, h.pos[o]);
                    }
                }
            }
        }
        for (int64_t f = g.uoff[u]; f < g.uoff[u + 1]; f++) mark[g.uadj[f]] = -1;
    }
    s.complete = 1;
    for (int64_t u = 0; u < g.nu; u++)
        for (int64_t e = g.uoff[u]; e < g.uoff[u + 1]; e++) {
            out_u[e] = (int32_t)u;
            out_v[e] = g.uadj[e];
        }
done:
    *m_out = g.m;
    if (st) *st = s;
    free(sup);
    free(gone);
    free(mark);
    free(eu_of);
    free(h.heap);
    free(h.pos);
    eg_free(&g);
    return rc;
}
