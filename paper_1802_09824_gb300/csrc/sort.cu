// Stable LSD radix sort of (64-bit key, 32-bit value) pairs, 8-bit digits.
//
// Each pass: per-tile digit histograms (digit-major layout), one exclusive
// scan over all (digit, tile) counts, then a scatter in which every tile
// ranks its keys stably (warp by warp, 32 keys at a time, with
// __match_any_sync), reorders them by digit in shared memory and writes each
// digit's run after the keys of earlier tiles with consecutive threads on
// consecutive positions.
#include <utility>

#include "checks.cuh"
#include "phpp_internal.cuh"

namespace phpp {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;                  // rounds of 32 keys per warp
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kBins = 1 << kSortBits;

__global__ void __launch_bounds__(kSortThreads) k_hist(const uint64_t *keys, int64_t n, int shift, int32_t *hist,
                                                        int ntiles)
{
    __shared__ int32_t h[kBins];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        int64_t i = base + k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kBins - 1)], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_scatter(const uint64_t *keys, const int32_t *vals, uint64_t *keys_out,
                                                           int32_t *vals_out, int64_t n, int shift,
                                                           const int32_t *offsets, int ntiles)
{
    __shared__ int32_t cnt[kSortWarps][kBins];
    __shared__ int32_t s_off[kBins];
    __shared__ int32_t s_start[kBins];          // first slot of each digit in the tile
    __shared__ int32_t s_wsum[kSortWarps];
    __shared__ uint64_t s_key[kSortTile];
    __shared__ int32_t s_val[kSortTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < kBins; d += 32) cnt[w][d] = 0;
    s_off[threadIdx.x] = offsets[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncwarp();
    // warp w owns keys [base + w*256, base + (w+1)*256), 32 per round, in order
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const int64_t base = tile0 + (int64_t)w * 32 * kSortItems;
    const unsigned lt = (1u << lane) - 1u;
    uint64_t k_[kSortItems];
    int32_t v_[kSortItems];
    int32_t d_[kSortItems];
    int32_t r_[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        int64_t i = base + r * 32 + lane;
        bool ok = i < n;
        uint64_t key = ok ? keys[i] : 0ull;
        int digit = ok ? (int)((key >> shift) & (kBins - 1)) : kBins;   // kBins = no key
        unsigned peers = __match_any_sync(0xffffffffu, digit);
        int leader = __ffs(peers) - 1;
        int old = 0;
        if (ok && lane == leader) old = cnt[w][digit];
        old = __shfl_sync(0xffffffffu, old, leader);
        __syncwarp();
        if (ok && lane == leader) cnt[w][digit] = old + __popc(peers);
        __syncwarp();
        k_[r] = key;
        v_[r] = ok ? vals[i] : 0;
        d_[r] = digit;
        r_[r] = old + __popc(peers & lt);
    }
    __syncthreads();
    {   // per digit: exclusive prefix of the per-warp counts over warps, and
        // the digit's total in the tile
        const int d = threadIdx.x;
        int run = 0;
#pragma unroll
        for (int ww = 0; ww < kSortWarps; ww++) {
            const int c = cnt[ww][d];
            cnt[ww][d] = run;
            run += c;
        }
        // exclusive scan of the totals over digits (block-wide)
        int incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) s_wsum[w] = incl;
        __syncthreads();
        int wbase = 0;
#pragma unroll
        for (int ww = 0; ww < kSortWarps; ww++) wbase += ww < w ? s_wsum[ww] : 0;
        s_start[d] = wbase + incl - run;
    }
    __syncthreads();
    // the tile in digit order in shared memory ...
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        if (d_[r] < kBins) {
            const int slot = s_start[d_[r]] + cnt[w][d_[r]] + r_[r];
            s_key[slot] = k_[r];
            s_val[slot] = v_[r];
        }
    }
    __syncthreads();
    // ... then written out slot by slot: consecutive threads write consecutive
    // positions of a digit's run
    const int tile_n = n - tile0 < kSortTile ? (int)(n - tile0) : kSortTile;
    for (int slot = threadIdx.x; slot < tile_n; slot += kSortThreads) {
        const uint64_t key = s_key[slot];
        const int d = (int)((key >> shift) & (kBins - 1));
        const int64_t pos = (int64_t)s_off[d] + (slot - s_start[d]);
        if (in_bounds(pos, n, BS_SORT_OUT)) {
            keys_out[pos] = key;
            vals_out[pos] = s_val[slot];
        }
    }
}

}  // namespace

size_t sort_temp_bytes(int64_t n)
{
    int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    if (ntiles < 1) ntiles = 1;
    size_t counts = (size_t)(kBins * ntiles + 1) * sizeof(int32_t);
    counts = (counts + 255) & ~(size_t)255;
    return 2 * counts + scan_temp_bytes(kBins * ntiles) + 256;
}

int radix_sort_pairs(uint64_t *keys, int32_t *vals, uint64_t *keys_alt, int32_t *vals_alt, int64_t n, int bits,
                     void *temp, cudaStream_t s, bool *result_in_alt)
{
    *result_in_alt = false;
    if (n <= 1) return PH_OK;
    const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    size_t counts = (size_t)(kBins * ntiles + 1) * sizeof(int32_t);
    counts = (counts + 255) & ~(size_t)255;
    int32_t *hist = static_cast<int32_t *>(temp);
    int32_t *offs = reinterpret_cast<int32_t *>(static_cast<char *>(temp) + counts);
    void *scan_tmp = static_cast<char *>(temp) + 2 * counts;
    uint64_t *kin = keys, *kout = keys_alt;
    int32_t *vin = vals, *vout = vals_alt;
    bool alt = false;
    for (int shift = 0; shift < bits; shift += kSortBits) {
        k_hist<<<ntiles, kSortThreads, 0, s>>>(kin, n, shift, hist, ntiles);
        count_launch();
        int rc = scan_exclusive_i32(hist, offs, (int64_t)kBins * ntiles, nullptr, scan_tmp, s);
        if (rc) return rc;
        k_scatter<<<ntiles, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, shift, offs, ntiles);
        count_launch();
        std::swap(kin, kout);
        std::swap(vin, vout);
        alt = !alt;
    }
    *result_in_alt = alt;
    return cuda_check(cudaGetLastError(), "radix sort launch");
}

}  // namespace phpp
