// Graph build (Algorithm 1, steps 1-3): duplicate removal, relabelling of
// each side in descending order of degree, and the CSR of both sides with
// neighbour lists sorted ascending by the new labels.
//
// The paper relabels all of W = U u V in one label space. Here each side
// keeps its own dense local ids (rank by descending degree, ties by original
// id), and `below[x]` records how many vertices of the OTHER side come
// before x in the single global order (descending degree, U before V on a
// tie, then id). For an end point ep on side A and a middle vertex mp on
// side B, "label(ep) < label(mp)" is then exactly "ep < below_B[mp]".
#include "common.cuh"

namespace receipt {

namespace {

__global__ void k_validate_pack(const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                                int64_t m, int32_t nu, int32_t nv, int bits_v,
                                uint64_t *__restrict__ keys, unsigned long long *bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long nbad = 0;
    for (; i < m; i += stride) {
        int32_t u = eu[i], v = ev[i];
        if (u < 0 || u >= nu || v < 0 || v >= nv) {
            nbad++;
            u = 0;
            v = 0;
        }
        keys[i] = ((uint64_t)u << bits_v) | (uint64_t)v;
    }
    nbad = warp_sum(nbad);
    if ((threadIdx.x & 31) == 0 && nbad) atomicAdd(bad, nbad);
}

__global__ void k_head_flags(const uint64_t *__restrict__ keys, int64_t m,
                             uint32_t *__restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

// Compacts unique keys and counts degrees of both sides (original ids).
__global__ void k_compact_degrees(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ flag,
                                  const uint32_t *__restrict__ pos, int64_t m, int bits_v,
                                  uint64_t mask_v, uint64_t *__restrict__ ukeys,
                                  uint32_t *__restrict__ deg_u, uint32_t *__restrict__ deg_v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m && flag[i]) {
        uint64_t k = keys[i];
        ukeys[pos[i]] = k;
        atomicAdd(&deg_u[k >> bits_v], 1u);
        atomicAdd(&deg_v[k & mask_v], 1u);
    }
}

// key = (maxdeg - deg) so an ascending stable sort gives descending degree,
// ties in ascending original id (the input order).
__global__ void k_degree_keys(const uint32_t *__restrict__ deg, int32_t n, uint32_t maxdeg,
                              uint64_t *__restrict__ key, uint32_t *__restrict__ id) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        key[i] = (uint64_t)(maxdeg - deg[i]);
        id[i] = (uint32_t)i;
    }
}

__global__ void k_relabel_maps(const uint32_t *__restrict__ sorted_id, int32_t n,
                               const uint32_t *__restrict__ deg, int32_t *__restrict__ new2old,
                               int32_t *__restrict__ old2new, int64_t *__restrict__ deg_new) {
    int32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n) {
        int32_t o = (int32_t)sorted_id[x];
        new2old[x] = o;
        old2new[o] = x;
        deg_new[x] = deg[o];
    }
}

// below[x] = number of other-side vertices ahead of x in the global order.
// On side U (U wins ties): #{v : deg_v > deg_x}. On side V: #{u : deg_u >= deg_y}.
// deg_other_new is the other side's degree array in its (descending) order.
__global__ void k_below(const int64_t *__restrict__ deg_new, int32_t n,
                        const int64_t *__restrict__ deg_other_new, int32_t n_other, int strict,
                        int32_t *__restrict__ below) {
    int32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    int64_t d = deg_new[x];
    // first index whose degree is <= d (strict) or < d (non-strict)
    int32_t lo = 0, hi = n_other;
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        bool ahead = strict ? (deg_other_new[mid] > d) : (deg_other_new[mid] >= d);
        if (ahead)
            lo = mid + 1;
        else
            hi = mid;
    }
    below[x] = lo;
}

// Relabelled keys for both sides' CSR sorts.
__global__ void k_relabel_edges(const uint64_t *__restrict__ ukeys, int64_t m, int bits_v,
                                uint64_t mask_v, const int32_t *__restrict__ o2n_u,
                                const int32_t *__restrict__ o2n_v, int bu, int bv,
                                uint64_t *__restrict__ key_u, uint64_t *__restrict__ key_v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) {
        uint64_t k = ukeys[i];
        uint64_t u = (uint64_t)o2n_u[k >> bits_v];
        uint64_t v = (uint64_t)o2n_v[k & mask_v];
        key_u[i] = (u << bv) | v;
        key_v[i] = (v << bu) | u;
    }
}

__global__ void k_low_bits(const uint64_t *__restrict__ key, int64_t m, uint64_t mask,
                           int32_t *__restrict__ adj) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) adj[i] = (int32_t)(key[i] & mask);
}

__global__ void k_set_last(int64_t *off, int32_t n, int64_t m) {
    if (threadIdx.x == 0 && blockIdx.x == 0) off[n] = m;
}

__global__ void k_u32_max(const uint32_t *__restrict__ a, int32_t n, unsigned *out) {
    unsigned mx = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        mx = max(mx, a[i]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// Builds a graph; the device arrays live in one allocation owned by g.
receipt_graph *build_graph(const int32_t *d_eu, const int32_t *d_ev, int64_t m, int32_t nu,
                           int32_t nv, int dedup, cudaStream_t s) {
    if (nu < 0 || nv < 0 || m < 0) fail(RECEIPT_ERR_INVALID, "negative size");
    if (m >= (int64_t)INT32_MAX) fail(RECEIPT_ERR_OVERFLOW, "m must be below 2^31");
    if (m > 0 && (!d_eu || !d_ev)) fail(RECEIPT_ERR_INVALID, "null edge pointer");
    if (m > 0 && ((int64_t)nu == 0 || nv == 0)) fail(RECEIPT_ERR_INVALID, "edges on an empty side");
    const int bu = bits_for(nu > 0 ? (uint64_t)(nu - 1) : 0);
    const int bv = bits_for(nv > 0 ? (uint64_t)(nv - 1) : 0);
    const uint64_t mask_v = bv ? ((1ull << bv) - 1) : 0;
    const uint64_t mask_u = bu ? ((1ull << bu) - 1) : 0;

    // scalars read back at the end: [0] bad ids, [1] max deg U, [2] max deg V
    DevBuf<unsigned long long> scal(4, s);
    scal.zero();
    DevBuf<uint64_t> keys(m, s);
    if (m > 0) {
        k_validate_pack<<<std::min<unsigned>(blocks_for(m), 4096), 256, 0, s>>>(
            d_eu, d_ev, m, nu, nv, bv, keys.get(), scal.get());
        RC_LAUNCH();
    }
    radix_sort_pairs(keys.get(), nullptr, m, 0, bu + bv, s);
    DevBuf<uint32_t> flag(m, s), pos(m + 1, s);
    DevBuf<uint64_t> ukeys(m, s);
    DevBuf<uint32_t> deg_u(nu, s), deg_v(nv, s);
    deg_u.zero();
    deg_v.zero();
    if (m > 0) {
        k_head_flags<<<blocks_for(m), 256, 0, s>>>(keys.get(), m, flag.get());
        RC_LAUNCH();
        scan_exclusive<uint32_t>(flag.get(), pos.get(), m, s);
        k_compact_degrees<<<blocks_for(m), 256, 0, s>>>(keys.get(), flag.get(), pos.get(), m, bv,
                                                        mask_v, ukeys.get(), deg_u.get(),
                                                        deg_v.get());
        RC_LAUNCH();
    }
    keys.release();
    // number of unique edges = pos[m-1] + flag[m-1]; read together with the checks
    unsigned long long h[4] = {0, 0, 0, 0};
    uint32_t last_pos = 0, last_flag = 0;
    unsigned *dmax = reinterpret_cast<unsigned *>(scal.get() + 1);
    if (nu > 0) {
        k_u32_max<<<std::min<unsigned>(blocks_for(nu), 1024), 256, 0, s>>>(deg_u.get(), nu, dmax);
        RC_LAUNCH();
    }
    if (nv > 0) {
        k_u32_max<<<std::min<unsigned>(blocks_for(nv), 1024), 256, 0, s>>>(deg_v.get(), nv,
                                                                          dmax + 2);
        RC_LAUNCH();
    }
    RC_CUDA(cudaMemcpyAsync(h, scal.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
    if (m > 0) {
        RC_CUDA(cudaMemcpyAsync(&last_pos, pos.get() + (m - 1), 4, cudaMemcpyDeviceToHost, s));
        RC_CUDA(cudaMemcpyAsync(&last_flag, flag.get() + (m - 1), 4, cudaMemcpyDeviceToHost, s));
    }
    RC_CUDA(cudaStreamSynchronize(s));
    if (h[0]) fail(RECEIPT_ERR_INVALID, std::to_string(h[0]) + " edge ids out of range");
    const int64_t mu = m > 0 ? (int64_t)last_pos + last_flag : 0;
    if (!dedup && mu != m) fail(RECEIPT_ERR_INVALID, "duplicate edges with dedup == 0");
    const uint32_t maxdeg_u = (uint32_t)(h[1] & 0xffffffffu);
    const uint32_t maxdeg_v = (uint32_t)(h[2] & 0xffffffffu);
    flag.release();
    pos.release();

    // one allocation for every array the graph keeps
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t sz_off_u = al(8 * ((size_t)nu + 1)), sz_off_v = al(8 * ((size_t)nv + 1));
    size_t sz_adj = al(4 * (size_t)(mu > 0 ? mu : 1));
    size_t sz_id_u = al(4 * (size_t)(nu > 0 ? nu : 1)), sz_id_v = al(4 * (size_t)(nv > 0 ? nv : 1));
    size_t total = sz_off_u + sz_off_v + 2 * sz_adj + 2 * sz_id_u + 2 * sz_id_v;
    receipt_graph *g = new receipt_graph();
    g->nu = nu;
    g->nv = nv;
    g->m = mu;
    RC_CUDA(cudaGetDevice(&g->device));
    char *base = nullptr;
    if (cudaMallocAsync((void **)&base, total, s) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        fail(RECEIPT_ERR_OOM, "graph allocation failed");
    }
    g->owned = base;
    char *p = base;
    auto take = [&](size_t b) {
        char *r = p;
        p += b;
        return r;
    };
    Side &SU = g->side[0];
    Side &SV = g->side[1];
    SU.n = nu;
    SV.n = nv;
    SU.off = (int64_t *)take(sz_off_u);
    SV.off = (int64_t *)take(sz_off_v);
    SU.adj = (int32_t *)take(sz_adj);
    SV.adj = (int32_t *)take(sz_adj);
    SU.new2old = (int32_t *)take(sz_id_u);
    SV.new2old = (int32_t *)take(sz_id_v);
    SU.below = (int32_t *)take(sz_id_u);
    SV.below = (int32_t *)take(sz_id_v);
    g->max_deg[0] = (int32_t)maxdeg_u;
    g->max_deg[1] = (int32_t)maxdeg_v;

    try {
        // relabel each side: stable sort by (maxdeg - deg)
        DevBuf<int32_t> o2n_u(nu, s), o2n_v(nv, s);
        DevBuf<int64_t> dn_u(nu + 1, s), dn_v(nv + 1, s);
        for (int sd = 0; sd < 2; sd++) {
            int32_t n = sd ? nv : nu;
            if (n == 0) continue;
            uint32_t mx = sd ? maxdeg_v : maxdeg_u;
            DevBuf<uint64_t> dk(n, s);
            DevBuf<uint32_t> id(n, s);
            k_degree_keys<<<blocks_for(n), 256, 0, s>>>(sd ? deg_v.get() : deg_u.get(), n, mx,
                                                        dk.get(), id.get());
            RC_LAUNCH();
            radix_sort_pairs(dk.get(), id.get(), n, 0, bits_for(mx), s);
            k_relabel_maps<<<blocks_for(n), 256, 0, s>>>(
                id.get(), n, sd ? deg_v.get() : deg_u.get(), sd ? SV.new2old : SU.new2old,
                sd ? o2n_v.get() : o2n_u.get(), sd ? dn_v.get() : dn_u.get());
            RC_LAUNCH();
        }
        if (nu > 0) {
            k_below<<<blocks_for(nu), 256, 0, s>>>(dn_u.get(), nu, dn_v.get(), nv, 1, SU.below);
            RC_LAUNCH();
        }
        if (nv > 0) {
            k_below<<<blocks_for(nv), 256, 0, s>>>(dn_v.get(), nv, dn_u.get(), nu, 0, SV.below);
            RC_LAUNCH();
        }
        // offsets from the relabelled degree arrays
        if (nu > 0) scan_exclusive<int64_t>(dn_u.get(), SU.off, nu, s);
        if (nv > 0) scan_exclusive<int64_t>(dn_v.get(), SV.off, nv, s);
        k_set_last<<<1, 32, 0, s>>>(SU.off, nu, mu);
        k_set_last<<<1, 32, 0, s>>>(SV.off, nv, mu);
        RC_LAUNCH();
        deg_u.release();
        deg_v.release();
        if (mu > 0) {
            DevBuf<uint64_t> ku(mu, s), kv(mu, s);
            k_relabel_edges<<<blocks_for(mu), 256, 0, s>>>(ukeys.get(), mu, bv, mask_v,
                                                           o2n_u.get(), o2n_v.get(), bu, bv,
                                                           ku.get(), kv.get());
            RC_LAUNCH();
            ukeys.release();
            radix_sort_pairs(ku.get(), nullptr, mu, 0, bu + bv, s);
            k_low_bits<<<blocks_for(mu), 256, 0, s>>>(ku.get(), mu, mask_v, SU.adj);
            RC_LAUNCH();
            ku.release();
            radix_sort_pairs(kv.get(), nullptr, mu, 0, bu + bv, s);
            k_low_bits<<<blocks_for(mu), 256, 0, s>>>(kv.get(), mu, mask_u, SV.adj);
            RC_LAUNCH();
        }
        RC_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        cudaStreamSynchronize(s);
        cudaFreeAsync(g->owned, s);
        delete g;
        throw;
    }
    return g;
}

// The graph's memory goes back to the stream-ordered pool without a device
// synchronisation. Every entry point has finished its work on the graph when
// it returns, so ordering the free on the legacy stream is safe.
void destroy_graph(receipt_graph *g) {
    if (!g) return;
    if (g->owned) {
        int prev = -1;
        cudaGetDevice(&prev);
        if (prev != g->device) cudaSetDevice(g->device);
        cudaFreeAsync(g->owned, 0);
        if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
    }
    delete g;
}

}  // namespace receipt
