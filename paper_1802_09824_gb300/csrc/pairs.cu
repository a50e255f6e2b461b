// Cutoff leaf-pair list (CSR by target group).
//
// Sec. 4.3: each ground cell is one task that sums over itself and its 26
// neighbours (the cells are at least R_cut wide, Sec. 3.1, so no pair within
// R_cut is further away).  Sec. 3.3: leaf-leaf pairs go to the PP kernel.
// Here the unit on the target side is a group of consecutive particles of one
// ground cell; for every group the leaves of the 27 cells around it are
// tested box against box, each neighbour cell with the periodic image its
// offset implies (with N_side < 3 the same cell appears through several
// images; at most one of them can be within R_cut < L/2 of any particle).
//
// The test runs in FP32 on cell-relative centres with a relative margin on
// R_cut, so no pair the PP kernel could accept is ever dropped.
//
// The count pass also gives each group its cost, the source particles its
// list holds (a warp's time on a group is proportional to them: it runs all
// 32 lanes whatever the group's size), and the groups are then ordered by
// decreasing cost for the PP kernel's queue (Sec. 4.4 weighs work by
// particle counts): the heaviest groups start first, so that the last ones
// to finish are short.  The order is a stable counting sort on the cost's
// quarter-octave (8-bit key), so it is deterministic, and the forces do not
// depend on it (each group is summed by one warp on its own).  The stored
// offset of an accepted pair is the difference of the reference points
// rounded once to FP32: in FP32 directly when no periodic image is involved
// (the reference points are FP32 numbers), from the FP64 points otherwise.
#include "checks.cuh"
#include "handles.cuh"

namespace phpp {
namespace {

struct PairArgs {
    const BoxDev *boxes;
    const int32_t *n_groups;
    const int32_t *group_cell;
    const int32_t *group_box;
    const float4 *group_c4, *group_h4;
    const double *group_ref;
    const int32_t *cell_leaf_first;
    const float4 *leaf_c4, *leaf_h4;
    const double *leaf_ref;
    const float4 *leaf_r4, *group_r4;   // the reference points as (exact) FP32
    int64_t *cnt;            // count pass output [n_groups]
    uint8_t *gkey;           // count pass output [n_groups]: queue key (255 - cost bucket), or NULL
    const int64_t *off;      // fill pass input   [n_groups + 1]
    float4 *ent;             // fill pass output: offset x, y, z, first source particle (bits)
    uint8_t *ecnt;           // fill pass output: particles in the leaf - 1
    const int32_t *leaf_first;
    const int32_t *group_list;   // active-particle mode: the groups to list (n_groups points at their count)
    int64_t n_particles;     // mass-centre particle of leaf l: pos_leaf[n_particles + l]
    int64_t cap;
    uint32_t *status;
    int64_t n_leaf_rows;     // rows of the leaf arrays (bounds checks)
};

__device__ __forceinline__ int warp_incl_scan_i(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// One warp per target group.  Lane t < 27 takes neighbour cell t (offset
// (t/9-1, t/3%3-1, t%3-1)), skips it when the whole cell is beyond rcut of
// the group's box, and contributes its leaf count; the warp then walks the
// concatenated candidate leaves 32 at a time.  The neighbour that owns a
// candidate follows from the runs that start inside the current 32: their
// start bits are OR-ed across the warp, and the owner of position q0 + t is
// the number of runs started before q0 plus the start bits at or below t,
// minus one (lanes with no leaves start no run).  Candidates keep the order
// (neighbour, leaf), so the list is deterministic.
// Quarter-octave bucket of a cost: 0 for 0, else 1 + 4 e + f with e the
// position of the leading bit and f the next two bits (1 .. 128).
__device__ __forceinline__ int cost_bucket(unsigned c)
{
    if (c == 0) return 0;
    const int e = 31 - __clz(c);
    const unsigned f = e >= 2 ? (c >> (e - 2)) & 3u : (c << (2 - e)) & 3u;
    return 1 + 4 * e + (int)f;
}

template <bool kFill>
__global__ void __launch_bounds__(kThreads) k_pairs(PairArgs a)
{
    __shared__ int2 s_run[kThreads / 32][32];   // per warp: (image code, first leaf - excl) of each run
    __shared__ float4 s_sh[kThreads / 32][32];  // per warp: the run's cell offset (dx h, dy h, dz h) in the group's frame
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int ng = *a.n_groups;
    for (int gi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; gi < ng; gi += warps) {
        const int g = a.group_list ? a.group_list[gi] : gi;
        const BoxDev &bx = a.boxes[a.group_box[g]];
        const int ns = bx.nside;
        const int ground = a.group_cell[g] - bx.cell_base;
        const int gx = ground / (ns * ns), gy = (ground / ns) % ns, gz = ground % ns;
        const float4 gc = a.group_c4[g], gh = a.group_h4[g];
        const float hc = (float)bx.h;
        const float rf2 = bx.rfilt2;
        // this lane's neighbour cell
        const int dx = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dz = lane % 3 - 1;
        int l0 = 0, cnt = 0, img = 13;
        if (lane < 27) {
            const int ax = gx + dx, ay = gy + dy, az = gz + dz;
            const int sx = ax < 0 ? -1 : (ax >= ns ? 1 : 0);
            const int sy = ay < 0 ? -1 : (ay >= ns ? 1 : 0);
            const int sz = az < 0 ? -1 : (az >= ns ? 1 : 0);
            const int nc = bx.cell_base + ((ax - sx * ns) * ns + (ay - sy * ns)) * ns + (az - sz * ns);
            // the neighbour cell spans [d h, (d+1) h) in the group's cell frame
            const float qx = fmaxf(fmaxf(dx * hc - (gc.x + gh.x), (gc.x - gh.x) - (dx + 1) * hc), 0.f);
            const float qy = fmaxf(fmaxf(dy * hc - (gc.y + gh.y), (gc.y - gh.y) - (dy + 1) * hc), 0.f);
            const float qz = fmaxf(fmaxf(dz * hc - (gc.z + gh.z), (gc.z - gh.z) - (dz + 1) * hc), 0.f);
            if (qx * qx + qy * qy + qz * qz < rf2 * 1.0001f) {
                l0 = a.cell_leaf_first[nc];
                cnt = a.cell_leaf_first[nc + 1] - l0;
            }
            img = (sx + 1) * 9 + (sy + 1) * 3 + (sz + 1);
        }
        const int incl = warp_incl_scan_i(cnt, lane);
        const int excl = incl - cnt;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        float4 gr4 = make_float4(0.f, 0.f, 0.f, 0.f);
        int64_t base = 0;
        if (kFill) {
            gr4 = a.group_r4[g];
            base = a.off[g];
        }
        // the lanes with leaves, in lane order, as runs (lane, first leaf - excl):
        // candidate q of run k is leaf (first - excl) + q
        const unsigned nonempty = __ballot_sync(0xffffffffu, cnt > 0);
        if (cnt > 0) {
            const int rk = __popc(nonempty & lt);
            s_run[w][rk] = make_int2(img, l0 - excl);
            s_sh[w][rk] = make_float4((lane / 9 - 1) * hc, ((lane / 3) % 3 - 1) * hc, (lane % 3 - 1) * hc, 0.f);
        }
        __syncwarp();
        int64_t count = 0;
        unsigned src = 0;  // source particles of this lane's accepted candidates (count pass)
        int before = 0;   // runs started before q0
        for (int q0 = 0; q0 < total; q0 += 32) {
            const int q = q0 + lane;
            const unsigned sq = (unsigned)(excl - q0);
            const unsigned starts = __reduce_or_sync(0xffffffffu, (cnt > 0 && sq < 32u) ? 1u << sq : 0u);
            int r = before + __popc(starts & (0xffffffffu >> (31 - lane))) - 1;   // owner run
            if (!in_bounds(r, 32, BS_PAIR_RUN)) r = 0;
            before += __popc(starts);
            const int2 ru = s_run[w][r];
            const int im = ru.x, lb = ru.y;
            const float4 sh = s_sh[w][r];
            bool acc = false, mono = false;
            int l = 0;
            float4 lc = make_float4(0.f, 0.f, 0.f, 0.f), lh = lc;   // w: first particle, particles (bits)
            if (q < total && in_bounds(lb + q, a.n_leaf_rows, BS_PAIR_LEAF)) {
                l = lb + q;
                lc = a.leaf_c4[l];
                lh = a.leaf_h4[l];
                const float px = fmaxf(fabsf((lc.x + sh.x) - gc.x) - (gh.x + lh.x), 0.f);
                const float py = fmaxf(fabsf((lc.y + sh.y) - gc.y) - (gh.y + lh.y), 0.f);
                const float pz = fmaxf(fabsf((lc.z + sh.z) - gc.z) - (gh.z + lh.z), 0.f);
                acc = px * px + py * py + pz * pz < rf2;
                // tree part (Sec. 3.3): accepted as one mass-centre particle
                // when both opening angles are below theta, theta_1 = (A + B)/R
                // and theta_2 = B/(R - A) (A the group's largest box width, B
                // the leaf's, R the distance of the box centres), i.e. R >
                // (A + B)/theta and R > A + B/theta, compared as squares
                if (acc && bx.c_acc < INFINITY) {
                    const float ex = (lc.x + sh.x) - gc.x;
                    const float ey = (lc.y + sh.y) - gc.y;
                    const float ez = (lc.z + sh.z) - gc.z;
                    const float R2 = ex * ex + ey * ey + ez * ez;
                    const float A = 2.f * fmaxf(fmaxf(gh.x, gh.y), gh.z);
                    const float Bw = 2.f * fmaxf(fmaxf(lh.x, lh.y), lh.z);
                    const float D1 = (A + Bw) * bx.c_acc;
                    const float D2 = A + Bw * bx.c_acc;
                    mono = R2 > D1 * D1 && R2 > D2 * D2;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, acc);
            if (!kFill && acc) src += mono ? 1u : (unsigned)__float_as_int(lh.w);
            if (kFill && acc) {
                const int64_t pos = base + count + __popc(bal & lt);
                if (pos < a.cap) {
                    const int sx = im / 9 - 1, sy = (im / 3) % 3 - 1, sz = im % 3 - 1;   // periodic image
                    float4 e;
                    if ((sx | sy | sz) == 0) {
                        // the rounded difference of two FP32 numbers, exactly the
                        // shift the target frame was built with (pos_group)
                        const float4 lr4 = a.leaf_r4[l];
                        e.x = __fsub_rn(lr4.x, gr4.x);
                        e.y = __fsub_rn(lr4.y, gr4.y);
                        e.z = __fsub_rn(lr4.z, gr4.z);
                    } else {
                        // a periodic image: the FP64 difference rounded once
                        const double *lr = a.leaf_ref + 3 * (int64_t)l;
                        const double *gr = a.group_ref + 3 * (int64_t)g;
                        const double L = bx.L;
                        e.x = __double2float_rn((lr[0] + sx * L) - gr[0]);
                        e.y = __double2float_rn((lr[1] + sy * L) - gr[1]);
                        e.z = __double2float_rn((lr[2] + sz * L) - gr[2]);
                    }
                    if (mono) {
                        e.w = __int_as_float((int)(a.n_particles + l));  // the leaf's mass-centre particle
                        a.ent[pos] = e;
                        a.ecnt[pos] = 0;
                    } else {
                        e.w = lc.w;                                        // first particle (bits)
                        a.ent[pos] = e;
                        a.ecnt[pos] = (uint8_t)(__float_as_int(lh.w) - 1); // particles - 1
                    }
                } else {
                    atomicOr(a.status, ST_CAPACITY);
                }
            }
            count += __popc(bal);
        }
        if (!kFill) {
            const unsigned cost = __reduce_add_sync(0xffffffffu, src);
            if (lane == 0) {
                a.cnt[g] = count;
                if (a.gkey) a.gkey[g] = (uint8_t)(255 - cost_bucket(cost));
            }
        }
        __syncwarp();   // s_run is rewritten for the next group
    }
}

// Stable counting sort of the groups by their 8-bit queue key.  The groups
// are cut into kOrdChunks equal chunks (sized from the device-side group
// count, so the launches do not depend on it): per-chunk histograms
// (key-major), one exclusive scan over them, then each chunk ranks its keys
// in order -- 2048 at a time, warp by warp, 32 per round -- and writes each
// group's index after the same keys of earlier chunks and earlier rounds.
constexpr int kOrdItems = 8;
constexpr int kOrdWarps = kThreads / 32;
constexpr int kOrdSub = kThreads * kOrdItems;   // groups ranked per pass of a chunk
constexpr int kOrdBins = 256;
constexpr int kOrdChunks = 128;
static_assert(kThreads == kOrdBins, "one thread per key value");

__device__ __forceinline__ void order_chunk(int ng, int &c0, int &c1)
{
    const int chunk = (ng + kOrdChunks - 1) / kOrdChunks;
    c0 = min(ng, (int)blockIdx.x * chunk);
    c1 = min(ng, c0 + chunk);
}

__global__ void __launch_bounds__(kThreads) k_order_hist(const uint8_t *key, const int32_t *n_groups, int32_t *hist)
{
    __shared__ int32_t h[kOrdBins];
    h[threadIdx.x] = 0;
    __syncthreads();
    int c0, c1;
    order_chunk(*n_groups, c0, c1);
    for (int i = c0 + threadIdx.x; i < c1; i += kThreads) atomicAdd(&h[key[i]], 1);
    __syncthreads();
    hist[threadIdx.x * kOrdChunks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) k_order_scatter(const uint8_t *key, const int32_t *n_groups,
                                                             const int32_t *offsets, int32_t *order)
{
    __shared__ int32_t cnt[kOrdWarps][kOrdBins];
    __shared__ int32_t next[kOrdBins];   // next slot of each key for this chunk
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int ng = *n_groups;
    int c0, c1;
    order_chunk(ng, c0, c1);
    next[threadIdx.x] = offsets[threadIdx.x * kOrdChunks + blockIdx.x];
    for (int sub = c0; sub < c1; sub += kOrdSub) {
        for (int d = lane; d < kOrdBins; d += 32) cnt[w][d] = 0;
        __syncwarp();
        // warp w ranks groups [base, base + 256) of this pass, 32 per round, in order
        const int base = sub + w * 32 * kOrdItems;
        int d_[kOrdItems], r_[kOrdItems];
#pragma unroll
        for (int r = 0; r < kOrdItems; r++) {
            const int i = base + r * 32 + lane;
            const bool ok = i < c1;
            const int d = ok ? (int)key[i] : kOrdBins;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int leader = __ffs(peers) - 1;
            int old = 0;
            if (ok && lane == leader) old = cnt[w][d];
            old = __shfl_sync(0xffffffffu, old, leader);
            __syncwarp();
            if (ok && lane == leader) cnt[w][d] = old + __popc(peers);
            __syncwarp();
            d_[r] = d;
            r_[r] = old + __popc(peers & lt);
        }
        __syncthreads();
        int total;
        {   // per key value: exclusive prefix of the per-warp counts over warps
            const int d = threadIdx.x;
            int run = 0;
#pragma unroll
            for (int ww = 0; ww < kOrdWarps; ww++) {
                const int c = cnt[ww][d];
                cnt[ww][d] = run;
                run += c;
            }
            total = run;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kOrdItems; r++) {
            if (d_[r] < kOrdBins) {
                const int pos = next[d_[r]] + cnt[w][d_[r]] + r_[r];
                if (in_bounds(pos, ng, BS_ORDER)) order[pos] = base + r * 32 + lane;
            }
        }
        __syncthreads();
        next[threadIdx.x] += total;
        __syncthreads();
    }
}

}  // namespace

// Scratch of the group order: the per-chunk histograms and their scan, and
// the scan's own scratch (the same for any number of groups).
size_t order_temp_bytes(int64_t)
{
    size_t counts = (size_t)(kOrdBins * kOrdChunks + 1) * sizeof(int32_t);   // the scan also writes out[n]
    counts = (counts + 255) & ~(size_t)255;
    return 2 * counts + scan_temp_bytes(kOrdBins * kOrdChunks);
}

// The sizing (with `sizing_sync`: read the total, grow the entry buffers)
// and the fill pass, on stream s.
static int fill_pairs(ph_pairs *pr, PairArgs &a, const int32_t *n_all, int grid, cudaStream_t s, bool sizing_sync)
{
    int rc = 0;
    if (sizing_sync) {
        // total = group_off[n_groups]; read the count then the total
        int32_t ng = 0;
        rc = cuda_check(cudaMemcpyAsync(&ng, n_all, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "copy n_groups");
        if (rc) return rc;
        rc = cuda_check(cudaStreamSynchronize(s), "sync n_groups");
        if (rc) return rc;
        int64_t total = 0;
        rc = cuda_check(cudaMemcpyAsync(&total, static_cast<const int64_t *>(pr->group_off.p) + ng, sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, s),
                        "copy pair total");
        if (rc) return rc;
        rc = cuda_check(cudaStreamSynchronize(s), "sync pair total");
        if (rc) return rc;
        pr->n_pairs = total;
        if (total > pr->capacity) {
            int64_t cap = total + total / 8 + 1024;
            rc = ensure(pr->entries, (size_t)cap * sizeof(float4));
            if (!rc) rc = ensure(pr->ecount, (size_t)cap);
            if (rc) return rc;
            pr->capacity = cap;
        }
    }
    a.ent = static_cast<float4 *>(pr->entries.p);
    a.ecnt = static_cast<uint8_t *>(pr->ecount.p);
    a.cap = pr->capacity;
    k_pairs<true><<<grid, kThreads, 0, s>>>(a);
    count_launch();
    return PH_OK;
}

int build_pairs_device(const ph_leaves *lv, ph_pairs *pr, cudaStream_t s, bool sizing_sync)
{
    PairArgs a;
    a.boxes = static_cast<const BoxDev *>(lv->boxes.p);
    a.n_groups = static_cast<const int32_t *>(lv->counts.p) + 1;
    a.group_cell = static_cast<const int32_t *>(lv->group_cell.p);
    a.group_box = static_cast<const int32_t *>(lv->group_box.p);
    a.group_c4 = static_cast<const float4 *>(lv->group_c4.p);
    a.group_h4 = static_cast<const float4 *>(lv->group_h4.p);
    a.group_ref = static_cast<const double *>(lv->group_ref.p);
    a.cell_leaf_first = static_cast<const int32_t *>(lv->cell_leaf_first.p);
    a.leaf_c4 = static_cast<const float4 *>(lv->leaf_c4.p);
    a.leaf_h4 = static_cast<const float4 *>(lv->leaf_h4.p);
    a.n_leaf_rows = (int64_t)(lv->leaf_h4.bytes / sizeof(float4));
    a.leaf_ref = static_cast<const double *>(lv->leaf_ref.p);
    a.leaf_r4 = static_cast<const float4 *>(lv->leaf_r4.p);
    a.group_r4 = static_cast<const float4 *>(lv->group_r4.p);
    a.leaf_first = static_cast<const int32_t *>(lv->leaf_first.p);
    a.group_list = nullptr;
    if (lv->active) {
        // only the active groups get entries; the others keep an empty range
        a.group_list = static_cast<const int32_t *>(lv->active_list.p);
        a.n_groups = static_cast<const int32_t *>(lv->counts.p) + 2;
    }
    a.n_particles = lv->n;
    a.cnt = static_cast<int64_t *>(pr->group_cnt.p);
    // the cost order (queue_order 0) where the handle has its buffers
    const bool ordered = lv->queue_order == 0 && pr->group_key.p && pr->group_order.p && pr->order_temp.p;
    a.gkey = ordered ? static_cast<uint8_t *>(pr->group_key.p) : nullptr;
    pr->ordered = ordered;
    a.off = static_cast<const int64_t *>(pr->group_off.p);
    a.status = static_cast<uint32_t *>(pr->status.p);
    const int64_t n = lv->n;
    const int grid = 152 * 8;
    const int32_t *n_all = static_cast<const int32_t *>(lv->counts.p) + 1;
    if (lv->active) {
        int rz = cuda_check(cudaMemsetAsync(a.cnt, 0, 8 * (size_t)(n > 0 ? n : 1), s), "clear counts");
        if (!rz && a.gkey) rz = cuda_check(cudaMemsetAsync(a.gkey, 0xFF, (size_t)(n > 0 ? n : 1), s), "clear keys");
        if (rz) return rz;
    }
    k_pairs<false><<<grid, kThreads, 0, s>>>(a);
    count_launch();
    int rc = scan_exclusive_i64(a.cnt, static_cast<int64_t *>(pr->group_off.p), n, n_all, pr->temp.p, s);
    if (rc) return rc;
    // the PP queue's order: all groups (the inactive ones of the
    // active-particle mode last, with cost 0), on the side stream while the
    // sizing and the fill pass run on `s`; every path after the fork joins
    // it back, so a capture never ends with the side stream forked
    cudaStream_t os = s;
    if (ordered && pr->side && pr->ev_fork && pr->ev_join) {
        rc = cuda_check(cudaEventRecord(pr->ev_fork, s), "order fork");
        if (!rc) rc = cuda_check(cudaStreamWaitEvent(pr->side, pr->ev_fork, 0), "order fork wait");
        if (rc) return rc;
        os = pr->side;
    }
    if (ordered) {
        size_t counts = (size_t)(kOrdBins * kOrdChunks + 1) * sizeof(int32_t);
        counts = (counts + 255) & ~(size_t)255;
        int32_t *hist = static_cast<int32_t *>(pr->order_temp.p);
        int32_t *offs = reinterpret_cast<int32_t *>(static_cast<char *>(pr->order_temp.p) + counts);
        void *scan_tmp = static_cast<char *>(pr->order_temp.p) + 2 * counts;
        k_order_hist<<<kOrdChunks, kThreads, 0, os>>>(a.gkey, n_all, hist);
        count_launch();
        rc = scan_exclusive_i32(hist, offs, (int64_t)kOrdBins * kOrdChunks, nullptr, scan_tmp, os);
        if (!rc) {
            k_order_scatter<<<kOrdChunks, kThreads, 0, os>>>(a.gkey, n_all, offs,
                                                             static_cast<int32_t *>(pr->group_order.p));
            count_launch();
        }
    }
    if (!rc) rc = fill_pairs(pr, a, n_all, grid, s, sizing_sync);
    if (os != s) {
        const int rj = cuda_check(cudaEventRecord(pr->ev_join, os), "order join");
        if (!rc) rc = rj;
        if (!rj) {
            const int rw = cuda_check(cudaStreamWaitEvent(s, pr->ev_join, 0), "order join wait");
            if (!rc) rc = rw;
        }
    }
    if (rc) return rc;
    return cuda_check(cudaGetLastError(), "pair kernels");
}

}  // namespace phpp
