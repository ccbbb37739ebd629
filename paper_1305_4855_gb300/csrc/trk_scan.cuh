// Device-wide exclusive scan (three kernels: block scans, a scan of the block sums, the
// carry-in), values produced by a functor; shared by the pipelines of the library.
// Kernels are static: each translation unit that includes this has its own copies.
#pragma once

#include "trk_common.cuh"

namespace trk {

// ---------------------------------------------------------------------------------------
// device-wide exclusive scan (3 kernels), values produced by a functor
// ---------------------------------------------------------------------------------------

constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 4;
constexpr int kScanBlock = kScanThreads * kScanPerThread;

template <class V>
__device__ __forceinline__ int64_t block_exclusive_scan(V val, int64_t start, int64_t n,
                                                        int64_t out_vals[kScanPerThread],
                                                        int64_t *warp_tot)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int64_t loc[kScanPerThread];
    int64_t s = 0;
#pragma unroll
    for (int q = 0; q < kScanPerThread; ++q) {
        const int64_t i = start + (int64_t)tid * kScanPerThread + q;
        loc[q] = i < n ? val(i) : 0;
        s += loc[q];
    }
    int64_t v = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(kFull, v, o);
        if (lane >= o)
            v += u;
    }
    if (lane == 31)
        warp_tot[w] = v;
    __syncthreads();
    if (w == 0) {
        int64_t t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(kFull, t, o);
            if (lane >= o)
                t += u;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    int64_t run = (w > 0 ? warp_tot[w - 1] : 0) + v - s;
#pragma unroll
    for (int q = 0; q < kScanPerThread; ++q) {
        out_vals[q] = run;
        run += loc[q];
    }
    const int64_t total = warp_tot[31];
    __syncthreads();
    return total;
}

template <class V, class OutT>
static __global__ void __launch_bounds__(kScanThreads) k_scan_local(V val, const unsigned long long *n_dev,
                                                             int64_t n_host, int64_t n_cap,
                                                             OutT *out, int64_t *bsum)
{
    __shared__ int64_t warp_tot[32];
    int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    n = n < n_cap ? n : n_cap;
    const int64_t start = (int64_t)blockIdx.x * kScanBlock;
    if (start >= n) {
        if (threadIdx.x == 0)
            bsum[blockIdx.x] = 0;
        return;
    }
    int64_t ex[kScanPerThread];
    const int64_t tot = block_exclusive_scan(val, start, n, ex, warp_tot);
#pragma unroll
    for (int q = 0; q < kScanPerThread; ++q) {
        const int64_t i = start + (int64_t)threadIdx.x * kScanPerThread + q;
        if (i < n)
            out[i] = (OutT)ex[q];
    }
    if (threadIdx.x == 0)
        bsum[blockIdx.x] = tot;
}

struct ArrayVal {
    const int64_t *a;
    __device__ int64_t operator()(int64_t i) const { return a[i]; }
};

static __global__ void __launch_bounds__(kScanThreads) k_scan_bsum(int64_t *bsum, int nb,
                                                            unsigned long long *total_out)
{
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0)
        carry = 0;
    __syncthreads();
    for (int s0 = 0; s0 < nb; s0 += kScanBlock) {
        int64_t ex[kScanPerThread];
        const int64_t tot = block_exclusive_scan(ArrayVal{bsum}, s0, nb, ex, warp_tot);
        const int64_t c = carry;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kScanPerThread; ++q) {
            const int64_t i = s0 + (int64_t)threadIdx.x * kScanPerThread + q;
            if (i < nb)
                bsum[i] = ex[q] + c;
        }
        __syncthreads();
        if (threadIdx.x == 0)
            carry = c + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total_out)
        *total_out = (unsigned long long)carry;
}

template <class OutT>
static __global__ void __launch_bounds__(kScanThreads) k_scan_add(OutT *out, const int64_t *bsum,
                                                           const unsigned long long *n_dev,
                                                           int64_t n_host, int64_t n_cap)
{
    int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    n = n < n_cap ? n : n_cap;
    const int64_t start = (int64_t)blockIdx.x * kScanBlock;
    if (start >= n || blockIdx.x == 0)
        return;
    const int64_t add = bsum[blockIdx.x];
#pragma unroll
    for (int q = 0; q < kScanPerThread; ++q) {
        const int64_t i = start + (int64_t)threadIdx.x * kScanPerThread + q;
        if (i < n)
            out[i] = (OutT)((int64_t)out[i] + add);
    }
}

template <class V, class OutT>
static cudaError_t scan_exclusive(V val, const unsigned long long *n_dev, int64_t n_host,
                                  int64_t n_cap, OutT *out, int64_t *bsum,
                                  unsigned long long *total_out, cudaStream_t s)
{
    const int64_t nb64 = (n_cap + kScanBlock - 1) / kScanBlock;
    const int nb = (int)(nb64 > 0 ? nb64 : 1);
    k_scan_local<V, OutT><<<nb, kScanThreads, 0, s>>>(val, n_dev, n_host, n_cap, out, bsum);
    k_scan_bsum<<<1, kScanThreads, 0, s>>>(bsum, nb, total_out);
    k_scan_add<OutT><<<nb, kScanThreads, 0, s>>>(out, bsum, n_dev, n_host, n_cap);
    return cudaGetLastError();
}

struct PopcVal {
    const uint32_t *w;
    __device__ int64_t operator()(int64_t i) const { return __popc(w[i]); }
};
}  // namespace trk
