// Internal declarations shared by the translation units of libreceipt.so.
// Host code throws ReceiptError internally; every extern "C" entry point
// catches it and turns it into a receipt_status plus a thread-local message.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "receipt.h"

namespace receipt {

struct ReceiptError {
    receipt_status status;
    std::string msg;
};

[[noreturn]] void fail(receipt_status st, const std::string &msg);
void check_cuda(cudaError_t e, const char *what, const char *file, int line);
void set_last_error(const std::string &msg);

#define RC_CUDA(call) ::receipt::check_cuda((call), #call, __FILE__, __LINE__)
void count_launch();
#define RC_LAUNCH()                                                                  \
    do {                                                                             \
        ::receipt::check_cuda(cudaGetLastError(), "kernel launch", __FILE__, __LINE__); \
        ::receipt::count_launch();                                                   \
    } while (0)

int num_sms();
// Kernel launch counter of the library (graph launches add their kernels).
void count_launches(uint64_t n);
void uncount_launches(uint64_t n);
int max_smem_optin();
// Sets a kernel's MaxDynamicSharedMemorySize to all the shared memory the
// device allows it (opt-in limit minus its static shared memory), once per
// device and kernel. The value never depends on a call's sizes, so
// concurrent callers cannot lower it under one another's launches.
void allow_max_smem(const void *kernel);

// Stream-ordered device buffer (cudaMallocAsync / cudaFreeAsync on one stream).
template <typename T>
class DevBuf {
  public:
    DevBuf() = default;
    DevBuf(size_t n, cudaStream_t s) { alloc(n, s); }
    ~DevBuf() { release(); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept { *this = std::move(o); }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            release();
            p_ = o.p_;
            n_ = o.n_;
            s_ = o.s_;
            o.p_ = nullptr;
            o.n_ = 0;
        }
        return *this;
    }
    void alloc(size_t n, cudaStream_t s) {
        release();
        s_ = s;
        n_ = n;
        size_t bytes = (n ? n : 1) * sizeof(T);
        cudaError_t e = cudaMallocAsync((void **)&p_, bytes, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p_ = nullptr;
            fail(RECEIPT_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
        }
    }
    void zero() {
        if (p_) RC_CUDA(cudaMemsetAsync(p_, 0, (n_ ? n_ : 1) * sizeof(T), s_));
    }
    void release() {
        if (p_) cudaFreeAsync(p_, s_);
        p_ = nullptr;
        n_ = 0;
    }
    T *get() const { return p_; }
    size_t size() const { return n_; }

  private:
    T *p_ = nullptr;
    size_t n_ = 0;
    cudaStream_t s_ = 0;
};

// One side of the relabelled two-sided CSR. Local ids are ranks in
// descending order of degree (ties by original id). adj holds local ids of
// the other side, ascending within each list.
struct Side {
    int32_t n = 0;
    int64_t *off = nullptr;      // n + 1
    int32_t *adj = nullptr;      // m
    int32_t *new2old = nullptr;  // n
    int32_t *below = nullptr;    // n: other-side vertices ahead in the global order
    int64_t *row = nullptr;      // unused (reserved)
};

}  // namespace receipt

struct receipt_graph {
    int32_t nu = 0, nv = 0;
    int64_t m = 0;
    int device = 0;
    int32_t max_deg[2] = {0, 0};
    receipt::Side side[2];
    receipt_stats stats{};
    std::vector<receipt_round> trace;  // rounds of the last decomposition
    std::vector<receipt_subset> subsets;  // fine-grained subsets of the last decomposition
    std::vector<int64_t> parts;  // batch union: first side-0 vertex of every packed graph
    void *owned = nullptr;  // device allocation holding every array above
};

namespace receipt {

// ---------------------------------------------------------------------
// Primitives (prims.cu)
// ---------------------------------------------------------------------
template <typename T>
void scan_exclusive(const T *d_in, T *d_out, int64_t n, cudaStream_t s);
// Stable LSD radix sort of keys in [begin_bit, end_bit); vals may be null.
void radix_sort_pairs(uint64_t *keys, uint32_t *vals, int64_t n, int begin_bit, int end_bit,
                      cudaStream_t s);
void radix_sort_pairs64(uint64_t *keys, uint64_t *vals, int64_t n, int begin_bit, int end_bit,
                        cudaStream_t s);

inline int bits_for(uint64_t maxval) {  // bits needed to hold values 0..maxval
    int b = 0;
    while (b < 64 && (maxval >> b)) b++;
    return b;
}

// ---------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Appends x to list[] for every lane with take set: one atomic per warp on
// *cnt, positions in lane order. All lanes of the warp must call it.
__device__ __forceinline__ void warp_append(bool take, int32_t x, int32_t *cnt, int32_t *list) {
    unsigned bal = __ballot_sync(0xffffffffu, take);
    if (!bal) return;
    const int lane = threadIdx.x & 31;
    int leader = __ffs(bal) - 1;
    int pos = 0;
    if (lane == leader) pos = atomicAdd(cnt, __popc(bal));
    pos = __shfl_sync(0xffffffffu, pos, leader);
    if (take) list[pos + __popc(bal & lanemask_lt())] = x;
}

// Number of entries of the ascending list a[0..n) that are < key.
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *a, int64_t n, int32_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ unsigned long long choose2(unsigned long long c) {
    return c * (c - 1ull) / 2ull;
}

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024,
// multiple of 32). `tmp` is __shared__ storage of 33 elements. TAIL_SYNC =
// false leaves out the closing barrier: the caller must pass a barrier
// before `tmp` is written again.
template <typename T, bool TAIL_SYNC = true>
__device__ __forceinline__ T block_exclusive_scan(T v, T *tmp, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nwarps ? tmp[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nwarps) tmp[lane] = w;  // inclusive warp totals
        if (lane == nwarps - 1) tmp[32] = w;
    }
    __syncthreads();
    T base = warp ? tmp[warp - 1] : T(0);
    T r = base + x - v;
    if (total) *total = tmp[32];
    if (TAIL_SYNC) __syncthreads();
    return r;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T y = __shfl_xor_sync(0xffffffffu, v, o);
        v = y < v ? y : v;
    }
    return v;
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace receipt
