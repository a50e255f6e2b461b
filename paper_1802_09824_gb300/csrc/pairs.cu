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
// R_cut, so no pair the PP kernel could accept is ever dropped.  The stored
// offset of an accepted pair is the difference of the reference points
// rounded once to FP32: in FP32 directly when no periodic image is involved
// (the reference points are FP32 numbers), from the FP64 points otherwise.
//
// The count pass also gives each group its cost, the source particles its
// list holds (a warp's time on a group is proportional to them: it runs all
// 32 lanes whatever the group's size), and the groups are ordered by
// decreasing cost for the PP kernel's queue (Sec. 4.4 weighs work by
// particle counts): the heaviest groups start first, so that the last ones
// to finish are short.  The order is a counting sort on the cost's
// quarter-octave class (an 8-bit key) folded into the two passes: the count
// pass counts the groups of each key, and the fill pass, which has the
// counts, places each group after the keys below its own with an atomic
// cursor per key.  Groups of one key land in the order the fill pass meets
// them; the forces do not depend on the order (each group is summed by one
// warp on its own).
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
    int32_t *ohist;          // [256] groups per key (count pass), then [256] cursors (fill pass)
    int32_t *order;          // fill pass output [n_groups]: the queue's order
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
constexpr int kOrdKeys = 256;   // queue keys (8 bits)

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
    __shared__ int32_t s_start[kOrdKeys];   // fill pass with an order: first slot of each key
    if (kFill && a.order) {
        // exclusive scan of the per-key counts (one thread per key)
        static_assert(kThreads == kOrdKeys, "one thread per key");
        const int c = a.ohist[threadIdx.x];
        int incl = warp_incl_scan_i(c, lane);
        __shared__ int32_t s_wsum[kThreads / 32];
        if (lane == 31) s_wsum[w] = incl;
        __syncthreads();
        for (int ww = 0; ww < w; ww++) incl += s_wsum[ww];
        s_start[threadIdx.x] = incl - c;
        __syncthreads();
    }
    for (int gi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; gi < ng; gi += warps) {
        const int g = a.group_list ? a.group_list[gi] : gi;
        if (kFill && a.order && lane == 0) {
            // this group's place in the queue: after every group of a lower key
            const int k = a.gkey[g];
            const int pos = s_start[k] + atomicAdd(&a.ohist[kOrdKeys + k], 1);
            if (in_bounds(pos, ng, BS_ORDER)) a.order[pos] = g;
        }
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
                if (a.gkey) {
                    const int k = 255 - cost_bucket(cost);
                    a.gkey[g] = (uint8_t)k;
                    atomicAdd(&a.ohist[k], 1);
                }
            }
        }
        __syncwarp();   // s_run is rewritten for the next group
    }
}

}  // namespace

// Scratch of the group order: the per-key counts and cursors.
size_t order_temp_bytes(int64_t) { return 2 * kOrdKeys * sizeof(int32_t); }

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
    // the cost order (queue_order 0) where the handle has its buffers; not in
    // the active-particle mode, whose inactive groups get no list (the PP
    // kernel takes them in group order there)
    const bool ordered =
        lv->queue_order == 0 && !lv->active && pr->group_key.p && pr->group_order.p && pr->order_temp.p;
    a.gkey = ordered ? static_cast<uint8_t *>(pr->group_key.p) : nullptr;
    a.ohist = ordered ? static_cast<int32_t *>(pr->order_temp.p) : nullptr;
    a.order = ordered ? static_cast<int32_t *>(pr->group_order.p) : nullptr;
    pr->ordered = ordered;
    a.off = static_cast<const int64_t *>(pr->group_off.p);
    a.status = static_cast<uint32_t *>(pr->status.p);
    const int64_t n = lv->n;
    const int grid = 152 * 8;
    const int32_t *n_all = static_cast<const int32_t *>(lv->counts.p) + 1;
    if (lv->active) {
        const int rz = cuda_check(cudaMemsetAsync(a.cnt, 0, 8 * (size_t)(n > 0 ? n : 1), s), "clear counts");
        if (rz) return rz;
    }
    if (ordered) {
        const int rz = cuda_check(cudaMemsetAsync(a.ohist, 0, order_temp_bytes(0), s), "clear key counts");
        if (rz) return rz;
    }
    k_pairs<false><<<grid, kThreads, 0, s>>>(a);
    count_launch();
    int rc = scan_exclusive_i64(a.cnt, static_cast<int64_t *>(pr->group_off.p), n, n_all, pr->temp.p, s);
    if (rc) return rc;
    rc = fill_pairs(pr, a, n_all, grid, s, sizing_sync);
    if (rc) return rc;
    return cuda_check(cudaGetLastError(), "pair kernels");
}

}  // namespace phpp
