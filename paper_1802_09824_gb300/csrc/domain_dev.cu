// Device side of the domain decomposition's particle exchange (Sec. 4.1):
// for ranks that keep their particles on the GPU, the ground cell of every
// particle and the cell counts, the send buffer grouped by destination rank,
// and the local set made from a received buffer are computed here, so the
// only host traffic of an exchange is the cell counts (for the cut, which
// ph_domain_partition makes on the host), the owner table back, and the
// per-rank row counts.  The rows between ranks are moved by the caller's
// collective (all_to_all of NCCL on device memory).
//
// A row is PH_DOMAIN_ROW doubles: x, y, z (as given, wrapped by the build
// later), mass, the flag the row has at its destination (1 own, 2 ghost) and
// the caller's int64 identifier (its bits).  Within a destination the rows
// keep the sender's particle order; the local set keeps the received order,
// own rows first: the exchange is deterministic.
#include <algorithm>
#include <cmath>
#include <vector>

#include "checks.cuh"
#include "handles.cuh"

using namespace phpp;

namespace {

constexpr int kDomThreads = 256;

int grid_of(int64_t n)
{
    const int64_t b = (n + kDomThreads - 1) / kDomThreads;
    return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

// The host's wrap and cell arithmetic (ph_domain_cells), with every rounding
// spelt out so that the device decides each cell exactly as the host does.
__device__ __forceinline__ double wrap64_dev(double x, double L)
{
    if (x >= 0.0 && x < L) return x;
    return __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
}

__device__ __forceinline__ int cell_coord_dev(double xw, double invL, int g, int nside)
{
    const double u = scalbn(__dmul_rn(xw, invL), g);
    const int c = (int)floor(u);
    return c < 0 ? 0 : (c >= nside ? nside - 1 : c);
}

// Cell counts: with at most kSmemCells cells each block counts into shared
// memory and adds its counts to the global ones at the end (few global
// atomics instead of one per particle on a few thousand addresses).
constexpr int kSmemCells = 4096;

template <int kPosType, bool kSmem>
__global__ void k_domain_cells(const void *pos, int64_t n, double L, float L_up, double invL, int g,
                               int32_t *cell, unsigned long long *count, uint32_t *status)
{
    __shared__ unsigned int s_count[kSmem ? kSmemCells : 1];
    const int nside = 1 << g;
    const int cells = nside * nside * nside;
    if (kSmem) {
        for (int c = threadIdx.x; c < cells; c += blockDim.x) s_count[c] = 0;
        __syncthreads();
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int c[3];
        bool bad = false;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            double xw;
            if (kPosType == PH_F32) {
                const float x = static_cast<const float *>(pos)[3 * i + a];
                bad |= !isfinite(x);
                xw = (x >= 0.f && x < L_up) ? (double)x : wrap64_dev((double)x, L);
            } else {
                const double x = static_cast<const double *>(pos)[3 * i + a];
                bad |= !isfinite(x);
                xw = wrap64_dev(x, L);
            }
            c[a] = bad ? 0 : cell_coord_dev(xw, invL, g, nside);
        }
        if (bad) atomicOr(status, ST_NONFINITE);
        const int id = (c[0] * nside + c[1]) * nside + c[2];
        cell[i] = id;
        if (kSmem)
            atomicAdd(s_count + id, 1u);
        else
            atomicAdd(count + id, 1ull);
    }
    if (kSmem) {
        __syncthreads();
        for (int c = threadIdx.x; c < cells; c += blockDim.x)
            if (s_count[c]) atomicAdd(count + c, (unsigned long long)s_count[c]);
    }
}

// 1 where particle i goes to rank r: r owns its cell, or holds the cell as
// a ghost (bit r of the cell's ghost mask).
__global__ void k_dest_flag(const int32_t *cell, int64_t n, const int32_t *owner, const unsigned long long *ghost,
                            int r, int32_t *flag)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = cell[i];
        flag[i] = (owner[c] == r || ((ghost[c] >> r) & 1ull)) ? 1 : 0;
    }
}

// Rank r's rows at base + position; base and the count follow on the
// device (base[r + 1] = base[r] + count of r).
template <int kPosType>
__global__ void k_dest_scatter(const void *pos, const float *mass, const int64_t *ids, const int32_t *cell,
                               int64_t n, const int32_t *owner, int r, const int32_t *flag, const int32_t *excl,
                               int64_t *base, int64_t cap, double *send, uint32_t *status)
{
    const int64_t b = base[r];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        const int64_t row = b + excl[i];
        if (row >= cap) {
            atomicOr(status, ST_CAPACITY);
            continue;
        }
        double *o = send + PH_DOMAIN_ROW * row;
        if (kPosType == PH_F32) {
            const float *p = static_cast<const float *>(pos) + 3 * i;
            o[0] = p[0];
            o[1] = p[1];
            o[2] = p[2];
        } else {
            const double *p = static_cast<const double *>(pos) + 3 * i;
            o[0] = p[0];
            o[1] = p[1];
            o[2] = p[2];
        }
        o[3] = mass ? (double)mass[i] : 0.0;
        o[4] = owner[cell[i]] == r ? 1.0 : 2.0;
        o[5] = __longlong_as_double(ids ? (long long)ids[i] : (long long)i);
    }
    // the last thread that sees the end of the scan advances the base
    if (blockIdx.x == 0 && threadIdx.x == 0) base[r + 1] = b + (n > 0 ? (int64_t)excl[n - 1] + flag[n - 1] : 0);
}

__global__ void k_own_flag(const double *recv, int64_t n, int32_t *own)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        own[i] = recv[PH_DOMAIN_ROW * i + 4] == 1.0 ? 1 : 0;
}

template <int kPosType>
__global__ void k_unpack(const double *recv, int64_t n, const int32_t *own, const int32_t *excl, void *pos,
                         float *mass, int64_t *ids)
{
    const int64_t n_own = n > 0 ? (int64_t)excl[n - 1] + own[n - 1] : 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        // own rows keep their order at the front, ghosts theirs behind them
        const int64_t o = own[i] ? (int64_t)excl[i] : n_own + (i - (int64_t)excl[i]);
        if (!in_bounds(o, n, BS_DOM_ROW)) continue;
        const double *r = recv + PH_DOMAIN_ROW * i;
        if (kPosType == PH_F32) {
            float *p = static_cast<float *>(pos) + 3 * o;
            p[0] = (float)r[0];
            p[1] = (float)r[1];
            p[2] = (float)r[2];
        } else {
            double *p = static_cast<double *>(pos) + 3 * o;
            p[0] = r[0];
            p[1] = r[1];
            p[2] = r[2];
        }
        mass[o] = (float)r[3];
        ids[o] = (int64_t)__double_as_longlong(r[5]);
    }
}

// Scratch of the exchange kernels, kept from call to call (grown as needed)
// on the device it was made on.
struct DomScratch {
    int device = -1;
    DevBuf flag, excl, owner, ghost, base, temp, status;
};
DomScratch g_scratch;

// Drops the scratch if it lives on another device than the current one.
int scratch_on_current_device()
{
    int dev = 0;
    int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (g_scratch.device != dev) {
        DevBuf *b[] = {&g_scratch.flag, &g_scratch.excl, &g_scratch.owner, &g_scratch.ghost, &g_scratch.base,
                       &g_scratch.temp, &g_scratch.status};
        for (DevBuf *x : b) {
            x->p = nullptr;     // the old device's buffers are left to that device (freed at exit)
            x->bytes = 0;
        }
        g_scratch.device = dev;
    }
    return PH_OK;
}

}  // namespace

extern "C" {

int ph_domain_cells_device(const void *d_pos, int pos_type, int64_t n, const ph_params *params, int32_t *nside,
                           int32_t *d_cell, int64_t *d_counts, void *stream)
{
    TraceRange trace_("ph_domain_cells_device");
    if (!params || !nside || !d_counts || (n > 0 && (!d_pos || !d_cell))) return fail(PH_ERR_ARG, "NULL argument");
    if (pos_type != PH_F32 && pos_type != PH_F64) return fail(PH_ERR_ARG, "pos_type must be PH_F32 or PH_F64");
    if (n < 0) return fail(PH_ERR_ARG, "n must be >= 0");
    if (n > 0 && (!is_device_ptr(d_pos) || !is_device_ptr(d_cell))) return fail(PH_ERR_ARG, "device buffers only");
    if (!is_device_ptr(d_counts)) return fail(PH_ERR_ARG, "device buffers only");
    const double L = params->L, rcut = params->rcut;
    if (!(std::isfinite(L) && L > 0 && std::isfinite(rcut) && rcut > 0 && rcut < 0.5 * L))
        return fail(PH_ERR_ARG, "need 0 < rcut < L/2");
    const int g = ground_level(L, rcut);
    *nside = 1 << g;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t cells = (size_t)1 << (3 * g);
    int rc = scratch_on_current_device();
    if (!rc) rc = ensure(g_scratch.status, 16);
    if (!rc) rc = cuda_check(cudaMemsetAsync(g_scratch.status.p, 0, 4, s), "clear status");
    if (!rc) rc = cuda_check(cudaMemsetAsync(d_counts, 0, 8 * cells, s), "clear counts");
    if (rc) return rc;
    uint32_t *st = static_cast<uint32_t *>(g_scratch.status.p);
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(d_counts);
    if (n > 0) {
        // a grid of at most 2 blocks per SM when the counts go through shared memory
        const bool smem = cells <= (size_t)kSmemCells;
        const int grid = smem ? std::min(grid_of(n), 2 * sm_count()) : grid_of(n);
        const float Lu = float_at_or_above(L);
        if (pos_type == PH_F32)
            smem ? k_domain_cells<PH_F32, true><<<grid, kDomThreads, 0, s>>>(d_pos, n, L, Lu, 1.0 / L, g, d_cell, cnt, st)
                 : k_domain_cells<PH_F32, false><<<grid, kDomThreads, 0, s>>>(d_pos, n, L, Lu, 1.0 / L, g, d_cell, cnt, st);
        else
            smem ? k_domain_cells<PH_F64, true><<<grid, kDomThreads, 0, s>>>(d_pos, n, L, Lu, 1.0 / L, g, d_cell, cnt, st)
                 : k_domain_cells<PH_F64, false><<<grid, kDomThreads, 0, s>>>(d_pos, n, L, Lu, 1.0 / L, g, d_cell, cnt, st);
        count_launch();
        rc = cuda_check(cudaGetLastError(), "cells kernel");
    }
    uint32_t h = 0;
    if (!rc) rc = cuda_check(cudaMemcpyAsync(&h, st, 4, cudaMemcpyDeviceToHost, s), "read status");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "cells sync");
    if (rc) return rc;
    if (h & ST_NONFINITE) return fail(PH_ERR_NONFINITE, "non-finite position");
    return PH_OK;
}

int ph_domain_pack(const void *d_pos, int pos_type, const float *d_mass, const int64_t *d_ids, const int32_t *d_cell,
                   int64_t n, const int32_t *h_owner, int32_t nside, int32_t n_ranks, double *d_send,
                   int64_t send_capacity, int64_t *h_send_counts, void *stream)
{
    TraceRange trace_("ph_domain_pack");
    if (!h_owner || !h_send_counts || (n > 0 && (!d_pos || !d_cell))) return fail(PH_ERR_ARG, "NULL argument");
    if (pos_type != PH_F32 && pos_type != PH_F64) return fail(PH_ERR_ARG, "pos_type must be PH_F32 or PH_F64");
    if (n < 0 || n >= ((int64_t)1 << 31) || send_capacity < 0) return fail(PH_ERR_ARG, "bad n or capacity");
    if (n_ranks < 1 || n_ranks > 64) return fail(PH_ERR_ARG, "n_ranks must be 1..64");
    int g = 0;
    while (g <= kGroundMax && (1 << g) != nside) g++;
    if (g > kGroundMax) return fail(PH_ERR_ARG, "nside must be a power of two up to %d", 1 << kGroundMax);
    if (n > 0 && (!is_device_ptr(d_pos) || !is_device_ptr(d_cell) || (d_mass && !is_device_ptr(d_mass)) ||
                  (d_ids && !is_device_ptr(d_ids)) || (send_capacity > 0 && !is_device_ptr(d_send))))
        return fail(PH_ERR_ARG, "device buffers only");
    const int64_t cells = (int64_t)nside * nside * nside;
    // owner and ghost mask of every cell (host): the ghost cells of rank r
    // are the periodic 26-neighbours of its own cells it does not own
    std::vector<unsigned long long> ghost(cells, 0ull);
    for (int64_t id = 0; id < cells; id++) {
        if (h_owner[id] < 0 || h_owner[id] >= n_ranks) return fail(PH_ERR_ARG, "owner out of range at cell %lld", (long long)id);
    }
    for (int i = 0; i < nside; i++)
        for (int j = 0; j < nside; j++)
            for (int k = 0; k < nside; k++) {
                const int r = h_owner[((int64_t)i * nside + j) * nside + k];
                for (int di = -1; di <= 1; di++)
                    for (int dj = -1; dj <= 1; dj++)
                        for (int dk = -1; dk <= 1; dk++) {
                            const int a = (i + di + nside) % nside, b = (j + dj + nside) % nside,
                                      c = (k + dk + nside) % nside;
                            const int64_t nb = ((int64_t)a * nside + b) * nside + c;
                            if (h_owner[nb] != r) ghost[nb] |= 1ull << r;
                        }
            }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t N = (size_t)(n > 0 ? n : 1);
    int rc = scratch_on_current_device();
    if (!rc) rc = ensure(g_scratch.flag, 4 * N);
    if (!rc) rc = ensure(g_scratch.excl, 4 * (N + 1));   // the scan writes its total at [n]
    if (!rc) rc = ensure(g_scratch.owner, 4 * (size_t)cells);
    if (!rc) rc = ensure(g_scratch.ghost, 8 * (size_t)cells);
    if (!rc) rc = ensure(g_scratch.base, 8 * 72);
    if (!rc) rc = ensure(g_scratch.temp, scan_temp_bytes(n));
    if (!rc) rc = ensure(g_scratch.status, 16);
    if (rc) return rc;
    int32_t *flag = static_cast<int32_t *>(g_scratch.flag.p), *excl = static_cast<int32_t *>(g_scratch.excl.p);
    int32_t *own = static_cast<int32_t *>(g_scratch.owner.p);
    unsigned long long *gm = static_cast<unsigned long long *>(g_scratch.ghost.p);
    int64_t *base = static_cast<int64_t *>(g_scratch.base.p);
    uint32_t *st = static_cast<uint32_t *>(g_scratch.status.p);
    rc = cuda_check(cudaMemcpyAsync(own, h_owner, 4 * (size_t)cells, cudaMemcpyHostToDevice, s), "copy owner");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(gm, ghost.data(), 8 * (size_t)cells, cudaMemcpyHostToDevice, s),
                             "copy ghost masks");
    if (!rc) rc = cuda_check(cudaMemsetAsync(base, 0, 8 * 72, s), "clear bases");
    if (!rc) rc = cuda_check(cudaMemsetAsync(st, 0, 4, s), "clear status");
    for (int r = 0; !rc && r < n_ranks; r++) {
        if (n > 0) {
            k_dest_flag<<<grid_of(n), kDomThreads, 0, s>>>(d_cell, n, own, gm, r, flag);
            rc = scan_exclusive_i32(flag, excl, n, nullptr, g_scratch.temp.p, s);
            if (rc) break;
        }
        if (pos_type == PH_F32)
            k_dest_scatter<PH_F32><<<grid_of(n), kDomThreads, 0, s>>>(d_pos, d_mass, d_ids, d_cell, n, own, r, flag,
                                                                      excl, base, send_capacity, d_send, st);
        else
            k_dest_scatter<PH_F64><<<grid_of(n), kDomThreads, 0, s>>>(d_pos, d_mass, d_ids, d_cell, n, own, r, flag,
                                                                      excl, base, send_capacity, d_send, st);
        count_launch(n > 0 ? 2 : 1);
        rc = cuda_check(cudaGetLastError(), "pack kernels");
    }
    int64_t hb[65];
    uint32_t hs = 0;
    if (!rc) rc = cuda_check(cudaMemcpyAsync(hb, base, 8 * (size_t)(n_ranks + 1), cudaMemcpyDeviceToHost, s), "read bases");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(&hs, st, 4, cudaMemcpyDeviceToHost, s), "read status");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "pack sync");
    if (rc) return rc;
    for (int r = 0; r < n_ranks; r++) h_send_counts[r] = hb[r + 1] - hb[r];
    if (hs & ST_CAPACITY)
        return fail(PH_ERR_CAPACITY, "send buffer of %lld rows, %lld needed", (long long)send_capacity,
                    (long long)hb[n_ranks]);
    return PH_OK;
}

int ph_domain_unpack(const double *d_recv, int64_t n_recv, int pos_type, void *d_pos, float *d_mass, int64_t *d_ids,
                     int64_t *h_n_own, void *stream)
{
    TraceRange trace_("ph_domain_unpack");
    if (!h_n_own || (n_recv > 0 && (!d_recv || !d_pos || !d_mass || !d_ids))) return fail(PH_ERR_ARG, "NULL argument");
    if (pos_type != PH_F32 && pos_type != PH_F64) return fail(PH_ERR_ARG, "pos_type must be PH_F32 or PH_F64");
    if (n_recv < 0 || n_recv >= ((int64_t)1 << 31)) return fail(PH_ERR_ARG, "bad n_recv");
    *h_n_own = 0;
    if (n_recv == 0) return PH_OK;
    if (!is_device_ptr(d_recv) || !is_device_ptr(d_pos) || !is_device_ptr(d_mass) || !is_device_ptr(d_ids))
        return fail(PH_ERR_ARG, "device buffers only");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t N = (size_t)n_recv;
    int rc = scratch_on_current_device();
    if (!rc) rc = ensure(g_scratch.flag, 4 * N);
    if (!rc) rc = ensure(g_scratch.excl, 4 * (N + 1));   // the scan writes its total at [n]
    if (!rc) rc = ensure(g_scratch.temp, scan_temp_bytes(n_recv));
    if (rc) return rc;
    int32_t *own = static_cast<int32_t *>(g_scratch.flag.p), *excl = static_cast<int32_t *>(g_scratch.excl.p);
    k_own_flag<<<grid_of(n_recv), kDomThreads, 0, s>>>(d_recv, n_recv, own);
    rc = scan_exclusive_i32(own, excl, n_recv, nullptr, g_scratch.temp.p, s);
    if (rc) return rc;
    if (pos_type == PH_F32)
        k_unpack<PH_F32><<<grid_of(n_recv), kDomThreads, 0, s>>>(d_recv, n_recv, own, excl, d_pos, d_mass, d_ids);
    else
        k_unpack<PH_F64><<<grid_of(n_recv), kDomThreads, 0, s>>>(d_recv, n_recv, own, excl, d_pos, d_mass, d_ids);
    count_launch(2);
    rc = cuda_check(cudaGetLastError(), "unpack kernels");
    int32_t last[2] = {0, 0};
    if (!rc) rc = cuda_check(cudaMemcpyAsync(&last[0], excl + n_recv - 1, 4, cudaMemcpyDeviceToHost, s), "read scan");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(&last[1], own + n_recv - 1, 4, cudaMemcpyDeviceToHost, s), "read flag");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "unpack sync");
    if (rc) return rc;
    *h_n_own = (int64_t)last[0] + last[1];
    return PH_OK;
}

}  // extern "C"
