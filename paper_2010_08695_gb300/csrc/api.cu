// extern "C" entry points of libreceipt.so (declared in include/receipt.h),
// the decomposition driver, and the batch packer.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <utility>

#include "internal.cuh"

namespace receipt {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launches(uint64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }

void set_last_error(const std::string &msg) { g_last_error = msg; }

void fail(receipt_status st, const std::string &msg) { throw ReceiptError{st, msg}; }

void check_cuda(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    cudaGetLastError();
    std::string msg = std::string(cudaGetErrorName(e)) + " (" + cudaGetErrorString(e) + ") in " +
                      what + " at " + file + ":" + std::to_string(line);
    fail(e == cudaErrorMemoryAllocation ? RECEIPT_ERR_OOM : RECEIPT_ERR_CUDA, msg);
}

namespace {
struct DevInfo {
    int sms = 0;
    int smem_optin = 0;
    bool pool_set = false;
};
std::mutex g_info_mu;
DevInfo g_info[64];

DevInfo &dev_info() {
    int d = 0;
    RC_CUDA(cudaGetDevice(&d));
    std::lock_guard<std::mutex> lk(g_info_mu);
    DevInfo &I = g_info[d & 63];
    if (!I.sms) {
        RC_CUDA(cudaDeviceGetAttribute(&I.sms, cudaDevAttrMultiProcessorCount, d));
        RC_CUDA(cudaDeviceGetAttribute(&I.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d));
    }
    if (!I.pool_set) {
        // keep freed temporaries in the stream-ordered pool between calls
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
        I.pool_set = true;
    }
    return I;
}
}  // namespace

namespace {
struct PinnedTLS {
    void *p = nullptr;
    size_t n = 0;
    ~PinnedTLS() {
        if (p) cudaFreeHost(p);
    }
};
thread_local PinnedTLS g_pinned;
}  // namespace

void *pinned_scratch(size_t bytes) {
    if (g_pinned.n < bytes) {
        if (g_pinned.p) cudaFreeHost(g_pinned.p);
        g_pinned.p = nullptr;
        g_pinned.n = 0;
        size_t want = bytes < 4096 ? 4096 : bytes;
        RC_CUDA(cudaMallocHost(&g_pinned.p, want));
        g_pinned.n = want;
    }
    return g_pinned.p;
}

namespace {
// per device: [0] the capture stream, [1..NUM_TIER_STREAMS] the tier streams
struct CaptureTLS {
    cudaStream_t s[64][1 + NUM_TIER_STREAMS] = {};
    ~CaptureTLS() {
        for (auto &d : s)
            for (auto &x : d)
                if (x) cudaStreamDestroy(x);
    }
};
thread_local CaptureTLS g_capture;

cudaStream_t device_stream(int k) {
    int d = 0;
    RC_CUDA(cudaGetDevice(&d));
    if (d < 0 || d >= 64) fail(RECEIPT_ERR_INTERNAL, "device index out of range");
    if (!g_capture.s[d][k])
        RC_CUDA(cudaStreamCreateWithFlags(&g_capture.s[d][k], cudaStreamNonBlocking));
    return g_capture.s[d][k];
}
}  // namespace

cudaStream_t aux_stream() { return device_stream(0); }

cudaStream_t tier_stream(int k) {
    if (k < 0 || k >= NUM_TIER_STREAMS) fail(RECEIPT_ERR_INTERNAL, "tier stream index");
    return device_stream(1 + k);
}

int num_sms() { return dev_info().sms; }
int max_smem_optin() { return dev_info().smem_optin - 1024; }
void allow_max_smem(const void *kernel) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    const int optin = dev_info().smem_optin;
    int d = 0;
    RC_CUDA(cudaGetDevice(&d));
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({d, kernel})) return;
    cudaFuncAttributes fa;
    RC_CUDA(cudaFuncGetAttributes(&fa, kernel));
    RC_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes));
    done.insert({d, kernel});
}

void compute_wfull(const Side &S, const Side &O, int64_t m, unsigned long long *wfull,
                   cudaStream_t s);

// Upper bound of the butterfly count (Sec. 2: sum over x' != x of
// C(|N_x n N_x'|, 2)) of any vertex of a side with n_s vertices of degree at
// most ds, whose neighbours have degree at most d_o, in a graph of m edges.
// Every support of Algorithms 2-4 starts at such a count and only falls, so
// the bound covers every 64-bit support and count the library keeps:
//  (a) at most n_s - 1 partners x', each sharing c <= ds neighbours;
//  (b) the partners' c add up to the wedges leaving x, sum over y in N_x of
//      (d_y - 1) <= ds (d_o - 1), and C(c, 2) <= c (ds - 1) / 2;
//  (c) those wedges are also at most m.
unsigned __int128 count_bound(int64_t n_s, int64_t ds, int64_t d_o, int64_t m) {
    typedef unsigned __int128 u128;
    if (n_s < 2 || ds < 2) return 0;
    const u128 c2 = (u128)ds * (u128)(ds - 1) / 2;
    const u128 a = (u128)(n_s - 1) * c2;
    const u128 b = (u128)ds * (u128)(d_o > 0 ? d_o - 1 : 0) * (u128)(ds - 1) / 2;
    const u128 c = (u128)(m > 0 ? m : 0) * (u128)(ds - 1) / 2;
    u128 r = a < b ? a : b;
    return r < c ? r : c;
}

// Fails with RECEIPT_ERR_OVERFLOW when a count of either side of g could
// reach 2^63 (never with m < 2^31, where bound (c) stays below 2^61).
void check_count_bound(const receipt_graph *g) {
    for (int t = 0; t < 2; t++) {
        const unsigned __int128 b =
            count_bound(g->side[t].n, g->max_deg[t], g->max_deg[1 - t], g->m);
        if (b >> 63)
            fail(RECEIPT_ERR_OVERFLOW, std::string("butterfly counts of side ") + "UV"[t] +
                                           " could exceed 2^63");
    }
}

namespace {

__global__ void k_scatter_i32(const int32_t *__restrict__ v, const int32_t *__restrict__ new2old,
                              int32_t n, int32_t *__restrict__ out) {
    int32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n) out[new2old[x]] = v[x];
}

// sum over the other side of d(d - 1): wedges bottom-up peeling walks
__global__ void k_bup_wedges(const int64_t *__restrict__ off, int32_t n, unsigned long long *out) {
    unsigned long long acc = 0;
    for (int32_t y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
        unsigned long long d = (unsigned long long)(off[y + 1] - off[y]);
        acc += d * (d ? d - 1 : 0);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

struct Timer {
    bool on;
    cudaStream_t s;
    cudaEvent_t ev[8];
    int n = 0;
    Timer(bool on_, cudaStream_t s_) : on(on_), s(s_) {
        if (on)
            for (auto &e : ev) RC_CUDA(cudaEventCreate(&e));
    }
    ~Timer() {
        if (on)
            for (auto &e : ev) cudaEventDestroy(e);
    }
    void mark() {
        if (on && n < 8) RC_CUDA(cudaEventRecord(ev[n++], s));
    }
    float ms(int a, int b) {
        if (!on || b >= n) return 0.f;
        RC_CUDA(cudaEventSynchronize(ev[b]));
        float r = 0;
        RC_CUDA(cudaEventElapsedTime(&r, ev[a], ev[b]));
        return r;
    }
};

}  // namespace

void tip_decompose_impl(receipt_graph *g, int side, uint64_t *d_tip, const receipt_options *optp,
                        cudaStream_t s) {
    if (!g) fail(RECEIPT_ERR_INVALID, "null graph");
    if (side != 0 && side != 1) fail(RECEIPT_ERR_INVALID, "side must be 0 (U) or 1 (V)");
    receipt_options opt;
    receipt_options_default(&opt);
    if (optp) opt = *optp;
    if (opt.P <= 0) opt.P = 150;
    if (opt.n_bounds > 0) {
        if (!opt.h_bounds) fail(RECEIPT_ERR_INVALID, "n_bounds > 0 with null h_bounds");
        for (int i = 0; i < opt.n_bounds; i++)
            if (opt.h_bounds[i] == 0 || (i && opt.h_bounds[i] <= opt.h_bounds[i - 1]))
                fail(RECEIPT_ERR_INVALID, "h_bounds must be positive and strictly increasing");
    }
    if (opt.huc < -1 || opt.huc > 1) fail(RECEIPT_ERR_INVALID, "huc must be -1, 0 or 1");
    if (opt.huc_factor_1024 < 0) fail(RECEIPT_ERR_INVALID, "huc_factor_1024 must be >= 0");
    if (opt.fd_huc < -1 || opt.fd_huc > 1) fail(RECEIPT_ERR_INVALID, "fd_huc must be -1, 0 or 1");
    const Side &S = g->side[side];
    const int32_t n = S.n;
    if (n > 0 && !d_tip) fail(RECEIPT_ERR_INVALID, "null d_tip");
    check_count_bound(g);
    Timer T(true, s);  // phase times on every call (four events)
    T.mark();
    Decomp D;
    D.s = side;
    D.S = &g->side[side];
    D.O = &g->side[1 - side];
    D.n = n;
    D.m = g->m;
    D.timing = opt.timing != 0;
    D.max_deg_s = g->max_deg[side];
    D.fd_heavy_w = opt.fd_heavy_w;
    D.fd_huc = opt.fd_huc;
    D.huc_factor = opt.huc_factor_1024 > 0 ? opt.huc_factor_1024 / 1024.0 : 8.0;
    D.parts = (side == 0 && !g->parts.empty()) ? &g->parts : nullptr;
    DevBuf<unsigned long long> cu(g->nu, s), cv(g->nv, s), init(n, s), wfull(n, s);
    DevBuf<int32_t> sub(n, s);
    DevBuf<unsigned long long> wbup(1, s);
    wbup.zero();
    if (D.O->n > 0) {
        k_bup_wedges<<<std::min(ceil_div(D.O->n, 256), 1024), 256, 0, s>>>(D.O->off, D.O->n,
                                                                           wbup.get());
        RC_LAUNCH();
    }
    unsigned long long h_wbup = 0;
    RC_CUDA(cudaMemcpyAsync(&h_wbup, wbup.get(), 8, cudaMemcpyDeviceToHost, s));
    int64_t cpoints[5] = {0, 0, 0, 0, 0};
    uint64_t wc = count_local(g, cu.get(), cv.get(), s, cpoints);
    T.mark();
    D.sup = side ? cv.get() : cu.get();
    D.init = init.get();
    D.sub = sub.get();
    D.wfull = wfull.get();
    compute_wfull(S, *D.O, g->m, D.wfull, s);
    cd_run(D, opt, s);
    T.mark();
    fd_run(D, d_tip, s);
    T.mark();
    if (opt.d_subset && n > 0) {
        k_scatter_i32<<<ceil_div(n, 256), 256, 0, s>>>(D.sub, S.new2old, n, opt.d_subset);
        RC_LAUNCH();
    }
    if (opt.h_p_eff) *opt.h_p_eff = D.p_eff;
    if (opt.h_bounds_out)
        for (int i = 0; i < opt.h_bounds_cap && i < (int)D.bounds.size(); i++)
            opt.h_bounds_out[i] = D.bounds[i];
    RC_CUDA(cudaStreamSynchronize(s));
    receipt_stats &st = g->stats;
    st = receipt_stats{};
    st.wedges_count = wc;
    for (int t = 0; t < 5; t++) st.count_points[t] = cpoints[t];
    st.wedges_bup = h_wbup;
    st.wedges_cd = D.wedges_cd;
    st.wedges_fd = D.wedges_fd;
    st.rounds_cd = D.rounds;
    st.levels_fd = D.levels;
    st.p_eff = D.p_eff;
    g->trace = std::move(D.trace);
    st.ms_fd_max_subset = D.fd_max_ms;
    st.fd_max_subset_n = D.fd_max_n;
    st.fd_max_subset_levels = D.fd_max_levels;
    st.fd_heavy_subsets = D.fd_heavy;
    st.ms_fd_heavy = D.fd_heavy_ms;
    st.levels_fd_heavy = D.fd_heavy_levels;
    st.fd_split_levels = (int32_t)std::min<int64_t>(D.fd_split_levels, INT32_MAX);
    st.fd_tasks = D.fd_tasks;
    st.huc_recounts = D.huc_recounts;
    st.fd_recounts = D.fd_recounts;
    st.wedges_fd_recount = D.wedges_fd_recount;
    st.wedges_recount = D.wedges_recount;
    st.cost_recount = D.cost_recount;
    st.ms_recount = D.ms_recount;
    g->subsets = std::move(D.subsets);
    for (int t = 0; t < 5; t++) {
        st.peel_wedges[t] = D.tier_wedges[t];
        st.peel_mids[t] = D.tier_mids[t];
        st.peel_anchors[t] = D.tier_anchors[t];
        st.peel_pairs[t] = D.tier_pairs[t];
        st.peel_launches[t] = D.tier_launches[t];
        st.ms_peel[t] = D.tier_ms[t];
    }
    st.ms_count = T.ms(0, 1);
    st.ms_cd = T.ms(1, 2);
    st.ms_fd = T.ms(2, 3);
    st.ms_total = T.ms(0, 3);
}

// ---------------------------------------------------------------------
// Batch: pack graphs into one disjoint union (graph-major global order)
// ---------------------------------------------------------------------
namespace {

struct PackSrc {
    const int64_t *off[2];  // [0] decomposed side A, [1] other side B
    const int32_t *adj[2];
    const int32_t *n2o[2];
    const int32_t *below[2];
    int32_t n[2];
    int64_t m;
};

__device__ __forceinline__ int find_graph(const int64_t *base, int ng, int64_t x) {
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// vertices of side t (0 = A, 1 = B): offsets, new2old (as positions in the
// concatenated output), below.
__global__ void k_pack_vertices(const PackSrc *__restrict__ src, int ng, int t,
                                const int64_t *__restrict__ vbase, const int64_t *__restrict__ obase,
                                const int64_t *__restrict__ ebase, int64_t ntot,
                                int64_t *__restrict__ off, int32_t *__restrict__ n2o,
                                int32_t *__restrict__ below) {
    int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ntot) return;
    int gi = find_graph(vbase, ng, x);
    int64_t lx = x - vbase[gi];
    const PackSrc &p = src[gi];
    off[x] = p.off[t][lx] + ebase[gi];
    n2o[x] = (int32_t)(vbase[gi] + p.n2o[t][lx]);
    below[x] = (int32_t)(p.below[t][lx] + obase[gi]);
}

__global__ void k_pack_adj(const PackSrc *__restrict__ src, int ng, int t,
                           const int64_t *__restrict__ ebase, const int64_t *__restrict__ obase,
                           int64_t mtot, int32_t *__restrict__ adj) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mtot) return;
    int gi = find_graph(ebase, ng, e);
    adj[e] = (int32_t)(src[gi].adj[t][e - ebase[gi]] + obase[gi]);
}

__global__ void k_set_off_end(int64_t *off, int64_t n, int64_t m) { off[n] = m; }

__global__ void k_split_tips(const unsigned long long *__restrict__ cat, const int64_t *__restrict__ abase,
                             int ng, int64_t ntot, unsigned long long *const *__restrict__ outs) {
    int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ntot) return;
    int gi = find_graph(abase, ng, x);
    outs[gi][x - abase[gi]] = cat[x];
}

}  // namespace

void decompose_batch_impl(receipt_graph *const *gs, const receipt_side *sides, int32_t n,
                          uint64_t *const *d_tips, const receipt_options *opt, cudaStream_t s) {
    if (n < 0 || (n > 0 && (!gs || !sides || !d_tips))) fail(RECEIPT_ERR_INVALID, "bad batch");
    if (n == 0) return;
    std::vector<PackSrc> src(n);
    std::vector<int64_t> abase(n + 1, 0), bbase(n + 1, 0), ebase(n + 1, 0);
    int dev = -1;
    int32_t maxdeg[2] = {0, 0};
    for (int i = 0; i < n; i++) {
        const receipt_graph *g = gs[i];
        if (!g) fail(RECEIPT_ERR_INVALID, "null graph in batch");
        if (sides[i] != 0 && sides[i] != 1) fail(RECEIPT_ERR_INVALID, "bad side in batch");
        if (dev < 0) dev = g->device;
        if (g->device != dev) fail(RECEIPT_ERR_INVALID, "batch graphs on different devices");
        int a = sides[i], b = 1 - sides[i];
        PackSrc &p = src[i];
        for (int t = 0; t < 2; t++) {
            const Side &S = g->side[t ? b : a];
            p.off[t] = S.off;
            p.adj[t] = S.adj;
            p.n2o[t] = S.new2old;
            p.below[t] = S.below;
            p.n[t] = S.n;
        }
        p.m = g->m;
        if (g->side[a].n > 0 && !d_tips[i]) fail(RECEIPT_ERR_INVALID, "null output in batch");
        abase[i + 1] = abase[i] + p.n[0];
        bbase[i + 1] = bbase[i] + p.n[1];
        ebase[i + 1] = ebase[i] + p.m;
        maxdeg[0] = std::max(maxdeg[0], g->max_deg[a]);
        maxdeg[1] = std::max(maxdeg[1], g->max_deg[b]);
    }
    const int64_t NA = abase[n], NB = bbase[n], M = ebase[n];
    if (NA >= INT32_MAX || NB >= INT32_MAX || M >= INT32_MAX)
        fail(RECEIPT_ERR_OVERFLOW, "batch exceeds the int32 id space");
    // union graph (side 0 = A)
    receipt_graph U;
    U.nu = (int32_t)NA;
    U.nv = (int32_t)NB;
    U.m = M;
    U.device = dev;
    U.max_deg[0] = maxdeg[0];
    U.max_deg[1] = maxdeg[1];
    U.parts = abase;
    DevBuf<int64_t> offA(NA + 1, s), offB(NB + 1, s);
    DevBuf<int32_t> adjA(M, s), adjB(M, s), n2oA(NA, s), n2oB(NB, s), belA(NA, s), belB(NB, s);
    DevBuf<PackSrc> dsrc(n, s);
    DevBuf<int64_t> dab(n + 1, s), dbb(n + 1, s), deb(n + 1, s);
    RC_CUDA(cudaMemcpyAsync(dsrc.get(), src.data(), sizeof(PackSrc) * n, cudaMemcpyHostToDevice, s));
    RC_CUDA(cudaMemcpyAsync(dab.get(), abase.data(), 8 * (n + 1), cudaMemcpyHostToDevice, s));
    RC_CUDA(cudaMemcpyAsync(dbb.get(), bbase.data(), 8 * (n + 1), cudaMemcpyHostToDevice, s));
    RC_CUDA(cudaMemcpyAsync(deb.get(), ebase.data(), 8 * (n + 1), cudaMemcpyHostToDevice, s));
    if (NA > 0) {
        k_pack_vertices<<<ceil_div(NA, 256), 256, 0, s>>>(dsrc.get(), n, 0, dab.get(), dbb.get(),
                                                          deb.get(), NA, offA.get(), n2oA.get(),
                                                          belA.get());
        RC_LAUNCH();
    }
    if (NB > 0) {
        k_pack_vertices<<<ceil_div(NB, 256), 256, 0, s>>>(dsrc.get(), n, 1, dbb.get(), dab.get(),
                                                          deb.get(), NB, offB.get(), n2oB.get(),
                                                          belB.get());
        RC_LAUNCH();
    }
    k_set_off_end<<<1, 1, 0, s>>>(offA.get(), NA, M);
    k_set_off_end<<<1, 1, 0, s>>>(offB.get(), NB, M);
    RC_LAUNCH();
    if (M > 0) {
        k_pack_adj<<<ceil_div(M, 256), 256, 0, s>>>(dsrc.get(), n, 0, deb.get(), dbb.get(), M,
                                                     adjA.get());
        RC_LAUNCH();
        k_pack_adj<<<ceil_div(M, 256), 256, 0, s>>>(dsrc.get(), n, 1, deb.get(), dab.get(), M,
                                                     adjB.get());
        RC_LAUNCH();
    }
    U.side[0] = Side{(int32_t)NA, offA.get(), adjA.get(), n2oA.get(), belA.get(), nullptr};
    U.side[1] = Side{(int32_t)NB, offB.get(), adjB.get(), n2oB.get(), belB.get(), nullptr};
    DevBuf<unsigned long long> cat(NA, s);
    tip_decompose_impl(&U, 0, (uint64_t *)cat.get(), opt, s);
    if (NA > 0) {
        DevBuf<unsigned long long *> outs(n, s);
        RC_CUDA(cudaMemcpyAsync(outs.get(), d_tips, sizeof(void *) * n, cudaMemcpyHostToDevice, s));
        k_split_tips<<<ceil_div(NA, 256), 256, 0, s>>>(cat.get(), dab.get(), n, NA, outs.get());
        RC_LAUNCH();
        RC_CUDA(cudaStreamSynchronize(s));
    }
    gs[0]->stats = U.stats;
    gs[0]->trace = std::move(U.trace);
    gs[0]->subsets = std::move(U.subsets);
}

}  // namespace receipt

using namespace receipt;

namespace {

template <class F>
receipt_status guarded(F &&f) {
    try {
        f();
        set_last_error("");
        return RECEIPT_OK;
    } catch (const ReceiptError &e) {
        set_last_error(e.msg);
        return e.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return RECEIPT_ERR_OOM;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return RECEIPT_ERR_INTERNAL;
    } catch (...) {
        set_last_error("unknown internal error");
        return RECEIPT_ERR_INTERNAL;
    }
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            prev = -1;
            cudaGetLastError();
        }
        if (prev != dev) RC_CUDA(cudaSetDevice(dev));
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

void receipt_options_default(receipt_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->P = 150;
}

receipt_status receipt_build_csr(const int32_t *d_eu, const int32_t *d_ev, int64_t m, int32_t nu,
                                 int32_t nv, int dedup, void *stream, receipt_graph **out) {
    return guarded([&] {
        if (!out) fail(RECEIPT_ERR_INVALID, "null output handle");
        *out = nullptr;
        *out = build_graph(d_eu, d_ev, m, nu, nv, dedup, (cudaStream_t)stream);
    });
}

receipt_status receipt_graph_destroy(receipt_graph *g) {
    return guarded([&] { destroy_graph(g); });
}

receipt_status receipt_graph_info(const receipt_graph *g, int32_t *nu, int32_t *nv, int64_t *m) {
    return guarded([&] {
        if (!g) fail(RECEIPT_ERR_INVALID, "null graph");
        if (nu) *nu = g->nu;
        if (nv) *nv = g->nv;
        if (m) *m = g->m;
    });
}

receipt_status receipt_graph_max_degree(const receipt_graph *g, int32_t *max_deg_u,
                                        int32_t *max_deg_v) {
    return guarded([&] {
        if (!g) fail(RECEIPT_ERR_INVALID, "null graph");
        if (max_deg_u) *max_deg_u = g->max_deg[0];
        if (max_deg_v) *max_deg_v = g->max_deg[1];
    });
}

receipt_status receipt_count_butterflies(receipt_graph *g, uint64_t *d_cnt_u, uint64_t *d_cnt_v,
                                         void *stream) {
    return guarded([&] {
        if (!g) fail(RECEIPT_ERR_INVALID, "null graph");
        DeviceGuard dg(g->device);
        check_count_bound(g);
        cudaStream_t s = (cudaStream_t)stream;
        DevBuf<unsigned long long> cu(g->nu, s), cv(g->nv, s);
        int64_t cpoints[5] = {0, 0, 0, 0, 0};
        uint64_t w = count_local(g, cu.get(), cv.get(), s, cpoints);
        if (d_cnt_u)
            scatter_to_original(cu.get(), g->side[0].new2old, g->nu, (unsigned long long *)d_cnt_u, s);
        if (d_cnt_v)
            scatter_to_original(cv.get(), g->side[1].new2old, g->nv, (unsigned long long *)d_cnt_v, s);
        g->stats = receipt_stats{};
        g->stats.wedges_count = w;
        for (int t = 0; t < 5; t++) g->stats.count_points[t] = cpoints[t];
    });
}

receipt_status receipt_count_butterflies_noalloc(receipt_graph *g, uint64_t *d_cnt_u,
                                                 uint64_t *d_cnt_v, void *stream) {
    return guarded([&] {
        if (!g) fail(RECEIPT_ERR_INVALID, "null graph");
        DeviceGuard dg(g->device);
        check_count_bound(g);
        count_noalloc(g, (unsigned long long *)d_cnt_u, (unsigned long long *)d_cnt_v,
                      (cudaStream_t)stream);
    });
}

receipt_status receipt_tip_decompose(receipt_graph *g, receipt_side side, uint64_t *d_tip,
                                     const receipt_options *opt, void *stream) {
    return guarded([&] {
        if (!g) fail(RECEIPT_ERR_INVALID, "null graph");
        DeviceGuard dg(g->device);
        tip_decompose_impl(g, (int)side, d_tip, opt, (cudaStream_t)stream);
    });
}

receipt_status receipt_decompose_batch(receipt_graph *const *gs, const receipt_side *sides,
                                       int32_t n, uint64_t *const *d_tips,
                                       const receipt_options *opt, void *stream) {
    return guarded([&] {
        if (n > 0 && gs && gs[0]) {
            DeviceGuard dg(gs[0]->device);
            decompose_batch_impl(gs, sides, n, d_tips, opt, (cudaStream_t)stream);
        } else {
            decompose_batch_impl(gs, sides, n, d_tips, opt, (cudaStream_t)stream);
        }
    });
}

receipt_status receipt_tip_decompose_host(const int32_t *h_eu, const int32_t *h_ev, int64_t m,
                                          int32_t nu, int32_t nv, receipt_side side,
                                          uint64_t *h_tip, const receipt_options *opt,
                                          void *stream) {
    return guarded([&] {
        if (m > 0 && (!h_eu || !h_ev)) fail(RECEIPT_ERR_INVALID, "null edge pointer");
        if (side != 0 && side != 1) fail(RECEIPT_ERR_INVALID, "side must be 0 (U) or 1 (V)");
        int32_t n = side ? nv : nu;
        if (n > 0 && !h_tip) fail(RECEIPT_ERR_INVALID, "null h_tip");
        cudaStream_t s = (cudaStream_t)stream;
        DevBuf<int32_t> eu(m, s), ev(m, s);
        if (m > 0) {
            RC_CUDA(cudaMemcpyAsync(eu.get(), h_eu, 4 * m, cudaMemcpyHostToDevice, s));
            RC_CUDA(cudaMemcpyAsync(ev.get(), h_ev, 4 * m, cudaMemcpyHostToDevice, s));
        }
        receipt_graph *g = build_graph(eu.get(), ev.get(), m, nu, nv, 1, s);
        struct G {
            receipt_graph *g;
            ~G() { destroy_graph(g); }
        } gg{g};
        eu.release();
        ev.release();
        DevBuf<unsigned long long> tip(n, s);
        tip_decompose_impl(g, (int)side, (uint64_t *)tip.get(), opt, s);
        if (n > 0) RC_CUDA(cudaMemcpyAsync(h_tip, tip.get(), 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
        RC_CUDA(cudaStreamSynchronize(s));
    });
}

receipt_status receipt_support_bound(int64_t n_side, int32_t max_deg_side,
                                     int32_t max_deg_other, int64_t m, uint64_t *bound) {
    return guarded([&] {
        if (n_side < 0 || max_deg_side < 0 || max_deg_other < 0 || m < 0)
            fail(RECEIPT_ERR_INVALID, "negative size");
        const unsigned __int128 b = count_bound(n_side, max_deg_side, max_deg_other, m);
        if (bound) *bound = (b >> 64) ? ~0ull : (uint64_t)b;
        if (b >> 63) fail(RECEIPT_ERR_OVERFLOW, "the bound reaches 2^63");
    });
}

receipt_status receipt_get_stats(const receipt_graph *g, receipt_stats *out) {
    return guarded([&] {
        if (!g || !out) fail(RECEIPT_ERR_INVALID, "null argument");
        *out = g->stats;
    });
}

receipt_status receipt_get_trace(const receipt_graph *g, receipt_round *out, int32_t cap,
                                 int32_t *n_rounds) {
    return guarded([&] {
        if (!g) fail(RECEIPT_ERR_INVALID, "null graph");
        if (cap > 0 && !out) fail(RECEIPT_ERR_INVALID, "null output with cap > 0");
        const int32_t n = (int32_t)g->trace.size();
        for (int32_t i = 0; i < n && i < cap; i++) out[i] = g->trace[i];
        if (n_rounds) *n_rounds = n;
    });
}

receipt_status receipt_get_subsets(const receipt_graph *g, receipt_subset *out, int32_t cap,
                                   int32_t *n_subsets) {
    return guarded([&] {
        if (!g) fail(RECEIPT_ERR_INVALID, "null graph");
        if (cap > 0 && !out) fail(RECEIPT_ERR_INVALID, "null output with cap > 0");
        const int32_t n = (int32_t)g->subsets.size();
        for (int32_t i = 0; i < n && i < cap; i++) out[i] = g->subsets[i];
        if (n_subsets) *n_subsets = n;
    });
}

const char *receipt_last_error(void) { return g_last_error.c_str(); }

uint64_t receipt_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
