// Hybrid update computation, Sec. 4.1 (HUC).
//
// When the vertices a round of Algorithm 3 is about to peel carry many more
// wedges than a butterfly count of the graph traverses, the supports of the
// remaining vertices are recomputed instead of updated: Algorithm 1 runs on
// the subgraph left after removing every vertex already assigned to a subset
// (the round's activeSet included). A remaining vertex's count in that
// subgraph is the number of butterflies it shares with remaining vertices,
// which is exactly the raw support the peel update would have left it with
// (each shared butterfly removed once, Lemma 2), so tip numbers do not change.
//
// The subgraph keeps the local ids and the global vertex order of the full
// graph: an assigned vertex keeps its id with an empty list, and the other
// side's lists keep their entries that are still remaining, in order. The
// counting kernels only need a total order in which every list is ascending
// and `below` places each vertex among the other side's (Sec. 2.2: any total
// order gives the same counts), so they run on the subgraph unchanged.
//
// Cost model of the rule (Sec. 4.1): peeling an activeSet walks the sum over
// its vertices x of sum_{y in N_x} d_y wedges; a count walks at most
// C_rcnt = sum over edges (x, y) of min(d_x, d_y).
#include <algorithm>

#include "internal.cuh"

namespace receipt {

namespace {

constexpr int OWN_CHUNK = 16;  // consecutive CSR positions per thread

// Last list v in [0, n) with off[v] <= q (the owner of position q < off[n]).
__device__ __forceinline__ int32_t owner_of(const int64_t *__restrict__ off, int32_t n, int64_t q) {
    int32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= q)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// C_rcnt = sum over the positions q of side s's lists (edge x -> y) of
// min(d_x, d_y), OWN_CHUNK positions per thread.
__global__ void k_rcnt_cost(const int64_t *__restrict__ off_s, int32_t n_s,
                            const int32_t *__restrict__ adj_s, const int64_t *__restrict__ off_o,
                            int64_t m, unsigned long long *__restrict__ out) {
    const int64_t q0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * OWN_CHUNK;
    unsigned long long sum = 0;
    if (q0 < m) {
        int32_t x = owner_of(off_s, n_s, q0);
        const int64_t e = imin64(q0 + OWN_CHUNK, m);
        for (int64_t q = q0; q < e; q++) {
            while (off_s[x + 1] <= q) x++;
            const int64_t dx = off_s[x + 1] - off_s[x];
            const int32_t y = adj_s[q];
            const int64_t dy = off_o[y + 1] - off_o[y];
            sum += (unsigned long long)imin64(dx, dy);
        }
    }
    sum = warp_sum(sum);
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd(out, sum);
}

// len[x] = d_x for remaining vertices of side s, 0 for assigned ones; len[n] = 0.
__global__ void k_len_remaining(const int64_t *__restrict__ off, const int32_t *__restrict__ sub,
                                int32_t n, int64_t *__restrict__ len) {
    const int32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n) len[x] = sub[x] < 0 ? off[x + 1] - off[x] : 0;
    if (x == n) len[n] = 0;
}

// len[y] = live entries of the other side's compacted list y; len[n] = 0.
__global__ void k_len_live(const int32_t *__restrict__ len_w, int32_t n, int64_t *__restrict__ len) {
    const int32_t y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y < n) len[y] = len_w[y];
    if (y == n) len[n] = 0;
}

// Copies the lists of remaining vertices of side s to their new offsets.
__global__ void k_gather_remaining(const int64_t *__restrict__ off, int32_t n,
                                   const int32_t *__restrict__ adj, const int32_t *__restrict__ sub,
                                   int64_t m, const int64_t *__restrict__ noff,
                                   int32_t *__restrict__ out) {
    const int64_t q0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * OWN_CHUNK;
    if (q0 >= m) return;
    int32_t x = owner_of(off, n, q0);
    const int64_t e = imin64(q0 + OWN_CHUNK, m);
    for (int64_t q = q0; q < e; q++) {
        while (off[x + 1] <= q) x++;
        if (sub[x] < 0) out[noff[x] + (q - off[x])] = adj[q];
    }
}

// Copies the first len_w[y] entries of every list y of the compacted working
// copy (original offsets) to their new offsets.
__global__ void k_gather_live(const int64_t *__restrict__ off, int32_t n,
                              const int32_t *__restrict__ adj_w, const int32_t *__restrict__ len_w,
                              int64_t m, const int64_t *__restrict__ noff,
                              int32_t *__restrict__ out) {
    const int64_t q0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * OWN_CHUNK;
    if (q0 >= m) return;
    int32_t y = owner_of(off, n, q0);
    const int64_t e = imin64(q0 + OWN_CHUNK, m);
    for (int64_t q = q0; q < e; q++) {
        while (off[y + 1] <= q) y++;
        const int64_t r = q - off[y];
        if (r < len_w[y]) out[noff[y] + r] = adj_w[q];
    }
}

// sup[x] <- the recount for every remaining vertex.
__global__ void k_apply_recount(int32_t n, const int32_t *__restrict__ sub,
                                const unsigned long long *__restrict__ cnt,
                                unsigned long long *__restrict__ sup) {
    const int32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n && sub[x] < 0) sup[x] = cnt[x];
}

int chunk_blocks(int64_t m) { return ceil_div(ceil_div(m, OWN_CHUNK), 256); }

}  // namespace

void launch_recount_cost(const Side &S, const Side &O, int64_t m, unsigned long long *d_out,
                         cudaStream_t s) {
    RC_CUDA(cudaMemsetAsync(d_out, 0, sizeof(unsigned long long), s));
    if (m == 0 || S.n == 0) return;
    k_rcnt_cost<<<chunk_blocks(m), 256, 0, s>>>(S.off, S.n, S.adj, O.off, m, d_out);
    RC_LAUNCH();
}

bool recount_fits(const Decomp &D) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    // the subgraph's lists and offsets, the counts, the counting pass's
    // temporaries (prefix lengths and scans, tier lists, the global tier's
    // per-CTA counters) and a copy of the other side's lists
    const size_t n_all = (size_t)D.S->n + (size_t)D.O->n;
    const size_t n_max = (size_t)std::max(D.S->n, D.O->n);
    const size_t need = 40 * (size_t)D.m + 48 * n_all + 8 * (size_t)num_sms() * n_max +
                        ((size_t)64 << 20);
    return need <= fr;
}

uint64_t recount_remaining(const Decomp &D, const int32_t *len_w, const int32_t *adj_w,
                           cudaStream_t s) {
    return recount_masked(*D.S, *D.O, D.s, D.m, D.sub, D.sup, len_w, adj_w, s);
}

uint64_t recount_masked(const Side &S, const Side &O, int side_s, int64_t m, const int32_t *sub,
                        unsigned long long *sup, const int32_t *len_w, const int32_t *adj_w,
                        cudaStream_t s) {
    const int32_t n = S.n, no = O.n;
    if (n == 0 || no == 0 || m == 0) return 0;
    DevBuf<int64_t> ls(n + 1, s), offs(n + 1, s), lo(no + 1, s), offo(no + 1, s);
    k_len_remaining<<<ceil_div(n + 1, 256), 256, 0, s>>>(S.off, sub, n, ls.get());
    RC_LAUNCH();
    k_len_live<<<ceil_div(no + 1, 256), 256, 0, s>>>(len_w, no, lo.get());
    RC_LAUNCH();
    scan_exclusive<int64_t>(ls.get(), offs.get(), n + 1, s);
    scan_exclusive<int64_t>(lo.get(), offo.get(), no + 1, s);
    int64_t h[2] = {0, 0};
    RC_CUDA(cudaMemcpyAsync(&h[0], offs.get() + n, 8, cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaMemcpyAsync(&h[1], offo.get() + no, 8, cudaMemcpyDeviceToHost, s));
    RC_CUDA(cudaStreamSynchronize(s));
    // both sides list the same remaining edges
    if (h[0] != h[1])
        fail(RECEIPT_ERR_INTERNAL, "recount: the two sides of the remaining subgraph disagree");
    const int64_t mr = h[0];
    ls.release();
    lo.release();
    DevBuf<int32_t> adjs(mr, s), adjo(mr, s);
    if (mr > 0) {
        k_gather_remaining<<<chunk_blocks(m), 256, 0, s>>>(S.off, n, S.adj, sub, m, offs.get(),
                                                            adjs.get());
        RC_LAUNCH();
        k_gather_live<<<chunk_blocks(m), 256, 0, s>>>(O.off, no, adj_w, len_w, m, offo.get(),
                                                       adjo.get());
        RC_LAUNCH();
    }
    receipt_graph sg;
    sg.side[side_s] = Side{n, offs.get(), adjs.get(), S.new2old, S.below, nullptr};
    sg.side[1 - side_s] = Side{no, offo.get(), adjo.get(), O.new2old, O.below, nullptr};
    sg.nu = sg.side[0].n;
    sg.nv = sg.side[1].n;
    sg.m = mr;
    DevBuf<unsigned long long> cu(sg.nu, s), cv(sg.nv, s);
    const uint64_t w = count_local(&sg, cu.get(), cv.get(), s);
    k_apply_recount<<<ceil_div(n, 256), 256, 0, s>>>(n, sub, side_s ? cv.get() : cu.get(), sup);
    RC_LAUNCH();
    return w;
}

}  // namespace receipt
