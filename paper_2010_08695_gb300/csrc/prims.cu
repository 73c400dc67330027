// Device primitives used by the CSR build and the fine-grained setup:
// an exclusive prefix scan (reduce, scan of tile totals, scan-and-add) and a
// stable LSD radix sort with 8-bit digits (tile histogram, scan, stable
// scatter ranked by warp match).
#include <cstdio>

#include "common.cuh"

namespace receipt {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__global__ void k_tile_sums(const T *__restrict__ in, int64_t n, T *__restrict__ sums) {
    __shared__ T tmp[33];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T s = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t g = base + i;
        if (g < n) s += in[g];
    }
    T tot;
    block_exclusive_scan<T>(s, tmp, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_tile_scan(const T *__restrict__ in, T *__restrict__ out, int64_t n,
                            const T *__restrict__ offsets) {
    __shared__ T tile[SCAN_TILE];
    __shared__ T tmp[33];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t g = base + i;
        tile[i] = g < n ? in[g] : T(0);
    }
    __syncthreads();
    T loc[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        loc[j] = s;
        s += tile[threadIdx.x * SCAN_ITEMS + j];
    }
    T tot;
    T pre = block_exclusive_scan<T>(s, tmp, &tot);
    T off = (offsets ? offsets[blockIdx.x] : T(0)) + pre;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) tile[threadIdx.x * SCAN_ITEMS + j] = loc[j] + off;
    __syncthreads();
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t g = base + i;
        if (g < n) out[g] = tile[i];
    }
}

}  // namespace

template <typename T>
void scan_exclusive(const T *d_in, T *d_out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        k_tile_scan<T><<<1, SCAN_THREADS, 0, s>>>(d_in, d_out, n, nullptr);
        RC_LAUNCH();
        return;
    }
    DevBuf<T> sums(tiles, s), offs(tiles, s);
    k_tile_sums<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(d_in, n, sums.get());
    RC_LAUNCH();
    scan_exclusive<T>(sums.get(), offs.get(), tiles, s);
    k_tile_scan<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(d_in, d_out, n, offs.get());
    RC_LAUNCH();
}

template void scan_exclusive<int64_t>(const int64_t *, int64_t *, int64_t, cudaStream_t);
template void scan_exclusive<uint64_t>(const uint64_t *, uint64_t *, int64_t, cudaStream_t);
template void scan_exclusive<uint32_t>(const uint32_t *, uint32_t *, int64_t, cudaStream_t);
template void scan_exclusive<int32_t>(const int32_t *, int32_t *, int64_t, cudaStream_t);

// ---------------------------------------------------------------------
// Radix sort
// ---------------------------------------------------------------------
namespace {

constexpr int RS_WARPS = 8;
constexpr int RS_THREADS = RS_WARPS * 32;
constexpr int RS_ITEMS = 16;                         // per lane
constexpr int RS_WARP_CHUNK = 32 * RS_ITEMS;         // 512 consecutive keys per warp
constexpr int RS_TILE = RS_WARPS * RS_WARP_CHUNK;    // 4096 keys per block

__global__ void k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                          uint32_t *__restrict__ hist, int64_t ntiles) {
    __shared__ uint32_t h[256];
    for (int i = threadIdx.x; i < 256; i += RS_THREADS) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
        int64_t g = base + i;
        if (g < n) atomicAdd(&h[(keys[g] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += RS_THREADS) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

template <typename V>
__global__ void k_rs_scatter(const uint64_t *__restrict__ kin, const V *__restrict__ vin,
                             uint64_t *__restrict__ kout, V *__restrict__ vout, int64_t n,
                             int shift, const uint32_t *__restrict__ offs, int64_t ntiles) {
    __shared__ uint32_t wcnt[RS_WARPS][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * RS_WARP_CHUNK;
    uint64_t k[RS_ITEMS];
    V v[RS_ITEMS];
    int dg[RS_ITEMS];
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        int64_t g = wbase + j * 32 + lane;
        if (g < n) {
            k[j] = kin[g];
            if (vin) v[j] = vin[g];
            dg[j] = (int)((k[j] >> shift) & 0xff);
        } else {
            dg[j] = 256 + lane;  // distinct sentinel per lane, never stored
        }
    }
    // per-warp digit counts
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        unsigned peers = __match_any_sync(0xffffffffu, dg[j]);
        if (dg[j] < 256 && (__ffs(peers) - 1) == lane) wcnt[warp][dg[j]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per-warp starting offsets: tile offset + counts of earlier warps
    for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
        uint32_t run = offs[(int64_t)d * ntiles + blockIdx.x];
        for (int w = 0; w < RS_WARPS; w++) {
            uint32_t c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        unsigned peers = __match_any_sync(0xffffffffu, dg[j]);
        if (dg[j] < 256) {
            uint32_t pos = wcnt[warp][dg[j]] + __popc(peers & lanemask_lt());
            kout[pos] = k[j];
            if (vin) vout[pos] = v[j];
        }
        __syncwarp();
        if (dg[j] < 256 && (__ffs(peers) - 1) == lane) wcnt[warp][dg[j]] += __popc(peers);
        __syncwarp();
    }
}

template <typename V>
void radix_sort_impl(uint64_t *keys, V *vals, int64_t n, int begin_bit, int end_bit,
                     cudaStream_t s) {
    if (n <= 1 || end_bit <= begin_bit) return;
    if (n >= (int64_t)UINT32_MAX) fail(RECEIPT_ERR_OVERFLOW, "radix sort of more than 2^32 keys");
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    DevBuf<uint64_t> k2(n, s);
    DevBuf<V> v2;
    if (vals) v2.alloc(n, s);
    DevBuf<uint32_t> hist(ntiles * 256, s);
    uint64_t *ka = keys, *kb = k2.get();
    V *va = vals, *vb = vals ? v2.get() : nullptr;
    int passes = 0;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        k_rs_hist<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, n, shift, hist.get(), ntiles);
        RC_LAUNCH();
        scan_exclusive<uint32_t>(hist.get(), hist.get(), ntiles * 256, s);
        k_rs_scatter<V><<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift,
                                                                hist.get(), ntiles);
        RC_LAUNCH();
        std::swap(ka, kb);
        std::swap(va, vb);
        passes++;
    }
    if (passes & 1) {
        RC_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        if (vals) RC_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(V), cudaMemcpyDeviceToDevice, s));
    }
}

}  // namespace

void radix_sort_pairs(uint64_t *keys, uint32_t *vals, int64_t n, int begin_bit, int end_bit,
                      cudaStream_t s) {
    radix_sort_impl<uint32_t>(keys, vals, n, begin_bit, end_bit, s);
}

void radix_sort_pairs64(uint64_t *keys, uint64_t *vals, int64_t n, int begin_bit, int end_bit,
                        cudaStream_t s) {
    radix_sort_impl<uint64_t>(keys, vals, n, begin_bit, end_bit, s);
}

}  // namespace receipt
