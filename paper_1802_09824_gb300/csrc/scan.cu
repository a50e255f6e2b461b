// Device-wide exclusive prefix sums (reduce, scan of block sums, scan).
//
// The element count can be read from device memory so that a scan over a
// count produced by an earlier kernel needs no host round trip; the grid is
// fixed, each block owns one contiguous chunk of the input.
#include "phpp_internal.cuh"

namespace phpp {
namespace {

constexpr int kScanBlocks = 512;
constexpr int kScanThreads = 256;
constexpr int kItems = 4;
constexpr int kTile = kScanThreads * kItems;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total
// through `total`.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T &total)
{
    __shared__ T warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[w] = inc;
    __syncthreads();
    if (w == 0) {
        T s = lane < kScanThreads / 32 ? warp_sums[lane] : T(0);
        s = warp_incl_scan(s);
        if (lane < kScanThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    T base = w > 0 ? warp_sums[w - 1] : T(0);
    total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return base + inc - v;
}

__device__ __forceinline__ int64_t load_n(int64_t n, const int32_t *d_n)
{
    return d_n ? (int64_t)(*d_n) : n;
}

__device__ __forceinline__ int64_t chunk_of(int64_t n)
{
    int64_t tiles = (n + kTile - 1) / kTile;
    int64_t per = (tiles + gridDim.x - 1) / gridDim.x;
    return per * kTile;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_reduce(const T *in, int64_t n_host, const int32_t *d_n, T *partial)
{
    const int64_t n = load_n(n_host, d_n);
    const int64_t chunk = chunk_of(n);
    const int64_t lo = (int64_t)blockIdx.x * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    T s = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kScanThreads) s += in[i];
    T tot;
    block_excl_scan<T>(s, tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_partials(T *partial, int nb)
{
    // nb <= kScanBlocks = 2 * kScanThreads: two items per thread
    T a = 2 * threadIdx.x < nb ? partial[2 * threadIdx.x] : T(0);
    T b = 2 * threadIdx.x + 1 < nb ? partial[2 * threadIdx.x + 1] : T(0);
    T tot;
    T ex = block_excl_scan<T>(a + b, tot);
    if (2 * threadIdx.x < nb) partial[2 * threadIdx.x] = ex;
    if (2 * threadIdx.x + 1 < nb) partial[2 * threadIdx.x + 1] = ex + a;
    if (threadIdx.x == 0) partial[kScanBlocks] = tot;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan(const T *in, T *out, int64_t n_host, const int32_t *d_n,
                                                        const T *partial)
{
    const int64_t n = load_n(n_host, d_n);
    const int64_t chunk = chunk_of(n);
    const int64_t lo = (int64_t)blockIdx.x * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    T run = partial[blockIdx.x];
    for (int64_t base = lo; base < hi; base += kTile) {
        T v[kItems];
        T s = 0;
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            int64_t i = base + threadIdx.x * kItems + k;
            v[k] = i < hi ? in[i] : T(0);
            s += v[k];
        }
        T tot;
        T ex = block_excl_scan<T>(s, tot) + run;
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            int64_t i = base + threadIdx.x * kItems + k;
            if (i < hi) out[i] = ex;
            ex += v[k];
        }
        run += tot;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = partial[kScanBlocks];
}

template <typename T>
int scan_impl(const T *in, T *out, int64_t n, const int32_t *d_n, void *temp, cudaStream_t s)
{
    T *partial = static_cast<T *>(temp);
    int nb = kScanBlocks;
    k_reduce<T><<<nb, kScanThreads, 0, s>>>(in, n, d_n, partial);
    count_launch();
    k_scan_partials<T><<<1, kScanThreads, 0, s>>>(partial, nb);
    count_launch();
    k_scan<T><<<nb, kScanThreads, 0, s>>>(in, out, n, d_n, partial);
    count_launch();
    return cuda_check(cudaGetLastError(), "scan launch");
}

}  // namespace

size_t scan_temp_bytes(int64_t) { return (kScanBlocks + 1) * sizeof(int64_t); }

int scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, const int32_t *d_n, void *temp, cudaStream_t s)
{
    return scan_impl<int32_t>(in, out, n, d_n, temp, s);
}

int scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, const int32_t *d_n, void *temp, cudaStream_t s)
{
    return scan_impl<int64_t>(in, out, n, d_n, temp, s);
}

}  // namespace phpp
