// Tree build on the GPU: keys, sort, leaves, target groups, frames.
//
// Sec. 3.2 ("Tree building"): each particle is labelled with its ground cell
// index (i N_side + j) N_side + k, particles are ordered by that index and,
// inside a ground cell, by a Morton (or Peano-Hilbert, Sec. 4.1) key, so that
// every octree node is one contiguous run of particles.  Leaves are the
// largest cells holding at most leaf_max particles (the N_pp of Sec. 3.1, the
// leaf size of Sec. 4.4); a level of the hierarchy is level_bits key bits:
// 3 gives the octree cells, 1 splits every octree level into its three
// binary sub-levels (half, quarter cell), which are key prefixes too.
//
// Leaf rule, evaluated independently for every particle k: k starts a leaf
// iff k is the first particle of a ground cell, or the smallest cell that
// holds both k-1 and k (their common key prefix) has more than leaf_max
// particles -- then k-1 and k lie in different children of a cell that had
// to be split.  Particles with identical keys (a finest cell) that number
// more than leaf_max are cut into runs of leaf_max from the run's start.
//
// Positions are stored relative to a reference point of their leaf in FP32
// (the FP64 wrap and the reference points are the only FP64 data on the
// device), and a second copy relative to the reference point of their target
// group, derived from the first by one FP32 add of the FP64-computed offset,
// exactly as the PP kernel shifts source particles, so that a particle seen
// as target and as source has bitwise the same coordinates.
#include <climits>
#include <cmath>

#include "checks.cuh"
#include "curve.cuh"
#include "handles.cuh"

namespace phpp {
namespace {

__device__ __forceinline__ int find_box(const int32_t *box_first, int nb, int64_t i)
{
    int lo = 0, hi = nb - 1;          // largest b with box_first[b] <= i
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (box_first[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ double wrap_coord(double x, double L)
{
    // x - L floor(x / L), each operation rounded once (no contraction); a
    // coordinate already in [0, L) is returned as is, which is what the
    // formula gives for it (floor = 0), without the FP64 divide
    if (x >= 0.0 && x < L) return x;
    double f = floor(__ddiv_rn(x, L));
    return __dsub_rn(x, __dmul_rn(L, f));
}

__device__ __forceinline__ uint32_t quant_coord(double xw, double S, int T)
{
    // floor(xw S) of a wrapped (finite, non-negative) coordinate, clamped
    const int q = __double2int_rd(__dmul_rn(xw, S));
    const int top = (1 << T) - 1;
    return (uint32_t)(q < 0 ? 0 : (q > top ? top : q));
}

// Wrapped coordinate of an FP32 input: the in-box test runs in FP32 (x < L
// exactly when x < L_up), so only the multiply of the key and the widening
// to FP64 remain on the FP64 pipe for particles already in the box.
__device__ __forceinline__ double wrap_f32(float x, const BoxDev &bx)
{
    if (x >= 0.f && x < bx.L_up) return (double)x;
    return wrap_coord((double)x, bx.L);
}

// Particle i's coordinates wrapped into [0, L) in FP64 (non-finite input
// counts as 0 and is reported once per particle through `bad`).
template <int kPosType>
__device__ __forceinline__ void wrapped_pos(const void *pos, int64_t i, const BoxDev &bx, double &x, double &y,
                                            double &z, bool &bad)
{
    if (kPosType == PH_F64) {
        const double *p = static_cast<const double *>(pos) + 3 * i;
        x = p[0]; y = p[1]; z = p[2];
        bad = !(isfinite(x) && isfinite(y) && isfinite(z));
        if (bad) x = y = z = 0.0;
        x = wrap_coord(x, bx.L);
        y = wrap_coord(y, bx.L);
        z = wrap_coord(z, bx.L);
    } else {
        const float *p = static_cast<const float *>(pos) + 3 * i;
        float fx = p[0], fy = p[1], fz = p[2];
        bad = !(isfinite(fx) && isfinite(fy) && isfinite(fz));
        if (bad) fx = fy = fz = 0.f;
        x = wrap_f32(fx, bx);
        y = wrap_f32(fy, bx);
        z = wrap_f32(fz, bx);
    }
}

template <int kPosType>
__global__ void k_keys(const void *pos, int64_t n, const int32_t *box_first, int nb, const BoxDev *boxes, int T,
                       int key_kind, uint64_t *keys, int32_t *vals, uint32_t *status)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int bi = nb > 1 ? find_box(box_first, nb, i) : 0;
        const BoxDev &bx = boxes[bi];
        double x, y, z;
        bool bad;
        wrapped_pos<kPosType>(pos, i, bx, x, y, z, bad);
        if (bad) atomicOr(status, ST_NONFINITE);
        const uint32_t qx = quant_coord(x, bx.S, T);
        const uint32_t qy = quant_coord(y, bx.S, T);
        const uint32_t qz = quant_coord(z, bx.S, T);
        const int b = bx.b;
        const uint32_t lm = (1u << b) - 1u;
        uint64_t ground = ((uint64_t)(qx >> b) * bx.nside + (qy >> b)) * bx.nside + (qz >> b);
        uint64_t local = key_kind == PH_KEY_HILBERT ? hilbert3(qx & lm, qy & lm, qz & lm, b)
                                                    : interleave3(qx & lm, qy & lm, qz & lm);
        uint64_t boxbits = 3 * T < 64 ? ((uint64_t)bi << (3 * T)) : 0ull;
        keys[i] = boxbits | (ground << (3 * b)) | local;
        vals[i] = (int32_t)i;
    }
}

template <int kPosType>
__global__ void k_gather(const void *pos, const float *mass, int64_t n, const uint64_t *keys, const int32_t *perm,
                         const BoxDev *boxes, int T, double *xw, float *mass_sorted, uint32_t *status)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = perm[k];
        if (!in_bounds(i, n, BS_BUILD_ROW)) i = 0;
        const int bi = 3 * T < 64 ? (int)(keys[k] >> (3 * T)) : 0;
        const BoxDev &bx = boxes[bi];
        double x, y, z;
        bool bad;
        wrapped_pos<kPosType>(pos, i, bx, x, y, z, bad);
        xw[3 * k + 0] = x;
        xw[3 * k + 1] = y;
        xw[3 * k + 2] = z;
        float m = mass ? mass[i] : bx.mass_default;
        if (!isfinite(m)) {
            atomicOr(status, ST_NONFINITE);
            m = 0.f;
        }
        mass_sorted[k] = m;
    }
}

__device__ __forceinline__ int box_of_cell(const BoxDev *boxes, int nb, int c)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (boxes[mid].cell_base <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t *a, int64_t lo, int64_t hi, uint64_t v)
{
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_cell_first(const uint64_t *keys, int64_t n, const BoxDev *boxes, int nb, int n_cells, int T,
                             int32_t *cell_first)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= n_cells; c += gridDim.x * blockDim.x) {
        if (c == n_cells) {
            cell_first[c] = (int32_t)n;
            continue;
        }
        const int bi = box_of_cell(boxes, nb, c);
        const BoxDev &bx = boxes[bi];
        const uint64_t boxbits = 3 * T < 64 ? ((uint64_t)bi << (3 * T)) : 0ull;
        const uint64_t pre = boxbits | ((uint64_t)(c - bx.cell_base) << (3 * bx.b));
        cell_first[c] = (int32_t)lower_bound_u64(keys, bx.first, (int64_t)bx.first + bx.n, pre);
    }
}

// Leaf and group start flags (see the leaf rule in the file comment).
__global__ void k_flags(const uint64_t *keys, int64_t n, const BoxDev *boxes, int T, int leaf_max, int level_bits,
                        const int32_t *cell_first, int32_t *leaf_flag, int32_t *group_flag)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t Bk = keys[k];
        const int bi = 3 * T < 64 ? (int)(Bk >> (3 * T)) : 0;
        const BoxDev &bx = boxes[bi];
        const int b = bx.b;
        const uint64_t cellpre = Bk >> (3 * b);
        const int cell = bx.cell_base + (int)(cellpre & ((1ull << (3 * bx.g)) - 1ull));
        // target groups: runs of group_size inside each ground cell
        const int64_t cf = cell_first[cell];
        group_flag[k] = ((k - cf) % bx.group_size) == 0 ? 1 : 0;
        int lf;
        if (k == 0) {
            lf = 1;
        } else {
            const uint64_t A = keys[k - 1];
            if ((A >> (3 * b)) != cellpre || (3 * T < 64 && (A >> (3 * T)) != (Bk >> (3 * T)))) {
                lf = 1;   // new box or new ground cell
            } else {
                const uint64_t x = A ^ Bk;
                if (x == 0) {
                    // identical keys: a finest cell; cut into runs of leaf_max
                    // from its first particle if it is too full
                    int64_t lo = k - 1, step = 1;
                    while (lo - step >= 0 && keys[lo - step] == Bk) { lo -= step; step <<= 1; }
                    int64_t a = lo - step < 0 ? 0 : lo - step;  // keys[a] may or may not equal Bk
                    lo = lower_bound_u64(keys, a, lo + 1, Bk);
                    int64_t hi = k, st2 = 1;
                    while (hi + st2 < n && keys[hi + st2] == Bk) { hi += st2; st2 <<= 1; }
                    int64_t e = hi + st2 < n ? hi + st2 : n;
                    hi = lower_bound_u64(keys, hi, e, Bk + 1);   // first index > Bk
                    lf = (hi - lo > leaf_max && ((k - lo) % leaf_max) == 0) ? 1 : 0;
                } else {
                    const int hb = 63 - __clzll((long long)x);
                    const int sh = level_bits * (hb / level_bits + 1);   // prefix shift of the common cell
                    const uint64_t P = Bk >> sh;
                    // is the common cell (holding k-1 and k) larger than leaf_max?
                    bool big;
                    const int64_t far = k - 1 - leaf_max;
                    if (far >= 0 && (keys[far] >> sh) == P) {
                        big = true;
                    } else {
                        int64_t lo = far < 0 ? 0 : far + 1, hi = k - 1;   // first index with prefix P
                        while (lo < hi) {
                            int64_t mid = (lo + hi) >> 1;
                            if ((keys[mid] >> sh) < P) lo = mid + 1; else hi = mid;
                        }
                        const int64_t q = lo + leaf_max;
                        big = q < n && (keys[q] >> sh) == P;
                    }
                    lf = big ? 1 : 0;
                }
            }
        }
        leaf_flag[k] = lf;
    }
}

// First particle of every leaf and every group; also resets the boxes'
// extent accumulators (ordered-integer min and max per axis) for k_extents.
__global__ void k_firsts(const int32_t *lflag, const int32_t *lscan, const int32_t *gflag, const int32_t *gscan,
                         int64_t n, int32_t *lfirst, int32_t *gfirst, long long *lext, long long *gext)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        if (lflag[k] && in_bounds(lscan[k], n, BS_BUILD_ROW)) {
            const int64_t l = lscan[k];
            lfirst[l] = (int32_t)k;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                lext[6 * l + d] = LLONG_MAX;
                lext[6 * l + 3 + d] = LLONG_MIN;
            }
        }
        if (gflag[k] && in_bounds(gscan[k], n, BS_BUILD_ROW)) {
            const int64_t l = gscan[k];
            gfirst[l] = (int32_t)k;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                gext[6 * l + d] = LLONG_MAX;
                gext[6 * l + 3 + d] = LLONG_MIN;
            }
        }
        if (k == n - 1) {
            lfirst[lscan[n]] = (int32_t)n;
            gfirst[gscan[n]] = (int32_t)n;
        }
    }
}

// Orders doubles like their values when compared as signed 64-bit integers.
__device__ __forceinline__ long long dkey(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}

__device__ __forceinline__ double dkey_inv(long long k)
{
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffll));
}

// Per-axis extents of every leaf and every group, one thread per particle:
// the particles of a box are consecutive, so a warp combines each box's part
// of its 32 particles by a segmented reduction (shuffle down within runs of
// the same box), and the first lane of each run folds that into the box's
// accumulators with 64-bit atomic min/max (boxes may straddle warps).
// Coordinates enter as ordered integers (dkey), so the integer order is the
// FP64 order.
__device__ __forceinline__ void segment_extent(const long long v[3], int l, int lane, long long *ext)
{
    long long lo[3] = {v[0], v[1], v[2]}, hi[3] = {v[0], v[1], v[2]};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int lo_l = __shfl_down_sync(0xffffffffu, l, o);
        const bool same = lane + o < 32 && lo_l == l;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const long long vl = __shfl_down_sync(0xffffffffu, lo[d], o);
            const long long vh = __shfl_down_sync(0xffffffffu, hi[d], o);
            if (same) {
                lo[d] = vl < lo[d] ? vl : lo[d];
                hi[d] = vh > hi[d] ? vh : hi[d];
            }
        }
    }
    const int prev = __shfl_up_sync(0xffffffffu, l, 1);
    if (l >= 0 && (lane == 0 || prev != l)) {
#pragma unroll
        for (int d = 0; d < 3; d++) {
            atomicMin(ext + 6 * (int64_t)l + d, lo[d]);
            atomicMax(ext + 6 * (int64_t)l + 3 + d, hi[d]);
        }
    }
}

__global__ void k_extents(const double *xw, int64_t n, const int32_t *lscan, const int32_t *gscan, long long *lext,
                          long long *gext)
{
    const int lane = threadIdx.x & 31;
    const int64_t k0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    for (int64_t base = k0; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = base + lane;
        const bool in = k < n;
        long long v[3];
#pragma unroll
        for (int d = 0; d < 3; d++) v[d] = in ? dkey(xw[3 * k + d]) : 0;
        segment_extent(v, in ? lscan[k + 1] - 1 : -1, lane, lext);
        segment_extent(v, in ? gscan[k + 1] - 1 : -1, lane, gext);
    }
}

// Bounding box of each leaf (or group) from its extents, one thread per box:
// FP64 reference point near the box centre, FP32 half extents around it
// rounded up, FP32 reference point relative to the ground cell's lower
// corner.
//
// The reference point is the centre rounded to a multiple of U = 2^(e-24),
// the FP32 spacing of the box's largest |coordinate| (2^(e-1) <= m < 2^e),
// so that an FP32 coordinate minus it is exact; rounding to a multiple of U
// is done as (c + 1.5 2^52 U) - 1.5 2^52 U (round half to even).  Being a
// multiple of U below 2^e in magnitude, it is itself an FP32 number: r4
// holds that exact FP32 copy.
__global__ void k_boxes(const int32_t *first, const int32_t *scan_total, const long long *ext, const uint64_t *keys,
                        const BoxDev *boxes, int T, double *ref, float4 *r4, float4 *c4, float4 *h4,
                        int32_t *cell_of, int32_t *box_of)
{
    const int count = *scan_total;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < count; l += gridDim.x * blockDim.x) {
        long long lo[3], hi[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            lo[d] = ext[6 * (int64_t)l + d];
            hi[d] = ext[6 * (int64_t)l + 3 + d];
        }
        const uint64_t key = keys[first[l]];
        const int bi = 3 * T < 64 ? (int)(key >> (3 * T)) : 0;
        const BoxDev &bx = boxes[bi];
        const uint32_t ground = (uint32_t)((key >> (3 * bx.b)) & ((1ull << (3 * bx.g)) - 1ull));
        const uint32_t gz = ground % bx.nside, gy = (ground / bx.nside) % bx.nside, gx = ground / (bx.nside * bx.nside);
        const uint32_t gc[3] = {gx, gy, gz};
        float c[3], hh[3], rf[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double vlo = dkey_inv(lo[d]), vhi = dkey_inv(hi[d]);
            const double m = fmax(fabs(vlo), fabs(vhi));
            const int ex = (int)((__double_as_longlong(m) >> 52) & 0x7ff) - 1022;   // m = f 2^ex, f in [0.5, 1)
            const double C = __longlong_as_double(((long long)(ex + 28 + 1023) << 52) | (1ll << 51));
            const double cen = __dmul_rn(0.5, __dadd_rn(vlo, vhi));
            const double r = __dsub_rn(__dadd_rn(cen, C), C);
            const double half = fmax(__dsub_rn(vhi, r), __dsub_rn(r, vlo));
            ref[3 * (int64_t)l + d] = r;
            rf[d] = __double2float_rn(r);   // exact
            c[d] = __double2float_rn(__dsub_rn(r, __dmul_rn((double)gc[d], bx.h)));
            hh[d] = __double2float_ru(half);
        }
        r4[l] = make_float4(rf[0], rf[1], rf[2], 0.f);
        const int f0 = first[l];
        c4[l] = make_float4(c[0], c[1], c[2], __int_as_float(f0));              // w: first particle
        h4[l] = make_float4(hh[0], hh[1], hh[2], __int_as_float(first[l + 1] - f0));   // w: particles
        if (cell_of) cell_of[l] = bx.cell_base + (int)ground;
        if (box_of) box_of[l] = bi;
    }
}

// Tree part (theta > 0): one particle per leaf carrying the leaf's mass at
// its mass centre, sum(m x) / sum(m) over the leaf's wrapped positions in
// FP64 (summed in particle order), stored after the N particles of pos_leaf
// relative to the leaf's reference point like the leaf's own particles.  A
// massless leaf keeps its reference point.
__global__ void k_leaf_mass(const int32_t *first, const int32_t *scan_total, const double *xw, const float *mass,
                            const double *ref, int64_t n, float4 *pos_leaf)
{
    const int count = *scan_total;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < count; l += gridDim.x * blockDim.x) {
        const int a = first[l], e = first[l + 1];
        double M = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        for (int k = a; k < e; k++) {
            const double m = mass[k];
            M = __dadd_rn(M, m);
            sx = __dadd_rn(sx, __dmul_rn(m, xw[3 * (int64_t)k]));
            sy = __dadd_rn(sy, __dmul_rn(m, xw[3 * (int64_t)k + 1]));
            sz = __dadd_rn(sz, __dmul_rn(m, xw[3 * (int64_t)k + 2]));
        }
        const double *r = ref + 3 * (int64_t)l;
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (M > 0.0) {
            q.x = __double2float_rn(__dsub_rn(__ddiv_rn(sx, M), r[0]));
            q.y = __double2float_rn(__dsub_rn(__ddiv_rn(sy, M), r[1]));
            q.z = __double2float_rn(__dsub_rn(__ddiv_rn(sz, M), r[2]));
            q.w = __double2float_rn(M);
        }
        pos_leaf[n + l] = q;
    }
}

__global__ void k_pos(int64_t n, const double *xw, const float *mass_sorted, const int32_t *leaf_scan,
                      const int32_t *group_scan, const double *leaf_ref, const float4 *leaf_r4, const float4 *group_r4,
                      float4 *pos_leaf, float4 *pos_group)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t l = leaf_scan[k + 1] - 1;
        int64_t g = group_scan[k + 1] - 1;
        if (!in_bounds(l, n, BS_BUILD_ROW)) l = 0;
        if (!in_bounds(g, n, BS_BUILD_ROW)) g = 0;
        const float4 lr4 = leaf_r4[l], gr4 = group_r4[g];
        const float lrf[3] = {lr4.x, lr4.y, lr4.z}, grf[3] = {gr4.x, gr4.y, gr4.z};
        float p[3], q[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            p[d] = __double2float_rn(__dsub_rn(xw[3 * k + d], leaf_ref[3 * l + d]));
            // the same FP32 offset (the rounded difference of the two exact FP32
            // reference points) and FP32 add as the PP kernel's source shift
            const float off = __fsub_rn(lrf[d], grf[d]);
            q[d] = __fadd_rn(p[d], off);
        }
        const float m = mass_sorted[k];
        pos_leaf[k] = make_float4(p[0], p[1], p[2], m);
        pos_group[k] = make_float4(q[0], q[1], q[2], m);
    }
}

__global__ void k_cell_leaf_first(const int32_t *cell_first, const int32_t *leaf_scan, int n_cells,
                                  int32_t *cell_leaf_first)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= n_cells; c += gridDim.x * blockDim.x)
        cell_leaf_first[c] = leaf_scan[cell_first[c]];
}

inline int grid_for(int64_t n, int threads = kThreads, int cap = 152 * 16)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

// Active-particle mode: flag the groups that hold at least one particle
// flagged active (flags in caller order, perm maps sorted -> caller row).
__global__ void k_group_active(const int32_t *gfirst, const int32_t *n_groups, const int32_t *perm,
                               const uint8_t *active, int32_t *gflag)
{
    const int ng = *n_groups;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        int f = 0;
        for (int j = gfirst[g]; j < gfirst[g + 1] && !f; j++) f = active[perm[j]] ? 1 : 0;
        gflag[g] = f;
    }
}

// The flagged groups in order, and their number into *n_active.
__global__ void k_active_list(const int32_t *gflag, const int32_t *gscan, const int32_t *n_groups, int32_t *list,
                              int32_t *n_active)
{
    const int ng = *n_groups;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x)
        if (gflag[g]) list[gscan[g]] = g;
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_active = gscan[ng];
}

}  // namespace

// h(u) = exp(u^2) erfc(u) + 2u/sqrt(pi), so that Eq. (split) is f = exp(-u^2) h(u)
// with u = s / 2R_s.  Chebyshev interpolation of h on [0, U] at deg+1 nodes,
// returned as monomial coefficients in t = 2u/U - 1.
void fit_factor_poly(double U, int deg, float *coef)
{
    const int n = deg + 1;
    double f[kMaxPoly + 1], c[kMaxPoly + 1];
    for (int k = 0; k < n; k++) {
        double t = std::cos(M_PI * (k + 0.5) / n);
        double u = 0.5 * (t + 1.0) * U;
        f[k] = std::exp(u * u) * std::erfc(u) + 2.0 * u / std::sqrt(M_PI);
    }
    for (int j = 0; j < n; j++) {
        double s = 0.0;
        for (int k = 0; k < n; k++) s += f[k] * std::cos(j * M_PI * (k + 0.5) / n);
        c[j] = 2.0 * s / n;
    }
    c[0] *= 0.5;
    // monomial coefficients: sum_j c_j T_j(t), T_{j+1} = 2t T_j - T_{j-1}
    double m[kMaxPoly + 1] = {0}, Tm1[kMaxPoly + 2] = {0}, T0[kMaxPoly + 2] = {0}, T1[kMaxPoly + 2] = {0};
    T0[0] = 1.0;                    // T_0
    for (int j = 0; j < n; j++) {
        const double *Tj = j == 0 ? T0 : T1;
        for (int k = 0; k <= j; k++) m[k] += c[j] * Tj[k];
        if (j == 0) {
            T1[1] = 1.0;            // T_1 = t
            for (int k = 0; k <= kMaxPoly; k++) Tm1[k] = T0[k];
        } else {
            double Tn[kMaxPoly + 2] = {0};
            for (int k = 0; k <= j; k++) Tn[k + 1] += 2.0 * T1[k];
            for (int k = 0; k <= j; k++) Tn[k] -= Tm1[k];
            for (int k = 0; k <= kMaxPoly; k++) { Tm1[k] = T1[k]; T1[k] = Tn[k]; }
        }
    }
    for (int k = 0; k <= kMaxPoly; k++) coef[k] = k < n ? (float)m[k] : 0.f;
}

// Enqueue the whole leaf/group build for the particles already in device
// memory (pos, mass).  The handle's box table and buffers are set up.
int build_leaves_device(ph_leaves *h, const void *pos, int pos_type, const float *mass, cudaStream_t s)
{
    const int64_t n = h->n;
    const int nb = h->n_boxes;
    const int T = h->key_bits;
    const BoxDev *boxes = static_cast<const BoxDev *>(h->boxes.p);
    const int32_t *box_first = static_cast<const int32_t *>(h->box_first.p);
    uint32_t *status = static_cast<uint32_t *>(h->status.p);
    uint64_t *keys = static_cast<uint64_t *>(h->keys.p);
    int32_t *vals = static_cast<int32_t *>(h->vals.p);
    if (n > 0) {
        if (pos_type == PH_F64)
            k_keys<PH_F64><<<grid_for(n), kThreads, 0, s>>>(pos, n, box_first, nb, boxes, T, h->key_kind, keys, vals,
                                                            status);
        else
            k_keys<PH_F32><<<grid_for(n), kThreads, 0, s>>>(pos, n, box_first, nb, boxes, T, h->key_kind, keys, vals,
                                                            status);
        count_launch();
        bool alt = false;
        int box_bits = 0;
        while ((1 << box_bits) < nb) box_bits++;
        int bits = 3 * T + box_bits;
        bits = (bits + kSortBits - 1) / kSortBits * kSortBits;
        int rc = radix_sort_pairs(keys, vals, static_cast<uint64_t *>(h->keys_alt.p),
                                  static_cast<int32_t *>(h->vals_alt.p), n, bits, h->temp.p, s, &alt);
        if (rc) return rc;
        h->keys_in_alt = alt;
    } else {
        h->keys_in_alt = false;
    }
    const uint64_t *sk = static_cast<const uint64_t *>(h->keys_in_alt ? h->keys_alt.p : h->keys.p);
    const int32_t *perm = static_cast<const int32_t *>(h->keys_in_alt ? h->vals_alt.p : h->vals.p);
    double *xw = static_cast<double *>(h->xw.p);
    float *ms = static_cast<float *>(h->mass_sorted.p);
    int32_t *cell_first = static_cast<int32_t *>(h->cell_first.p);
    int32_t *lflag = static_cast<int32_t *>(h->leaf_flag.p), *gflag = static_cast<int32_t *>(h->group_flag.p);
    int32_t *lscan = static_cast<int32_t *>(h->leaf_scan.p), *gscan = static_cast<int32_t *>(h->group_scan.p);
    if (n > 0)
        if (pos_type == PH_F64)
            k_gather<PH_F64><<<grid_for(n), kThreads, 0, s>>>(pos, mass, n, sk, perm, boxes, T, xw, ms, status);
        else
            k_gather<PH_F32><<<grid_for(n), kThreads, 0, s>>>(pos, mass, n, sk, perm, boxes, T, xw, ms, status);
        count_launch();
    k_cell_first<<<grid_for(h->n_cells + 1), kThreads, 0, s>>>(sk, n, boxes, nb, h->n_cells, T, cell_first);
    count_launch();
    if (n > 0)
        k_flags<<<grid_for(n), kThreads, 0, s>>>(sk, n, boxes, T, h->max_leaf, h->level_bits, cell_first, lflag,
                                                 gflag);
        count_launch();
    int rc = scan_exclusive_i32(lflag, lscan, n, nullptr, h->temp.p, s);
    if (rc) return rc;
    rc = scan_exclusive_i32(gflag, gscan, n, nullptr, h->temp.p, s);
    if (rc) return rc;
    int32_t *lfirst = static_cast<int32_t *>(h->leaf_first.p), *gfirst = static_cast<int32_t *>(h->group_first.p);
    long long *lext = static_cast<long long *>(h->box_ext.p), *gext = lext + 6 * (size_t)n;
    // first particles (and extent reset), extents, then the boxes of leaves and groups
    if (n > 0) {
        k_firsts<<<grid_for(n), kThreads, 0, s>>>(lflag, lscan, gflag, gscan, n, lfirst, gfirst, lext, gext);
        count_launch();
        k_extents<<<grid_for(n), kThreads, 0, s>>>(xw, n, lscan, gscan, lext, gext);
        count_launch();
    } else {
        cudaMemsetAsync(lfirst, 0, sizeof(int32_t), s);
        cudaMemsetAsync(gfirst, 0, sizeof(int32_t), s);
    }
    k_boxes<<<grid_for(n), kThreads, 0, s>>>(lfirst, lscan + n, lext, sk, boxes, T, static_cast<double *>(h->leaf_ref.p),
                                             static_cast<float4 *>(h->leaf_r4.p), static_cast<float4 *>(h->leaf_c4.p),
                                             static_cast<float4 *>(h->leaf_h4.p), nullptr, nullptr);
    count_launch();
    k_boxes<<<grid_for(n), kThreads, 0, s>>>(gfirst, gscan + n, gext, sk, boxes, T,
                                             static_cast<double *>(h->group_ref.p),
                                             static_cast<float4 *>(h->group_r4.p),
                                             static_cast<float4 *>(h->group_c4.p),
                                             static_cast<float4 *>(h->group_h4.p),
                                             static_cast<int32_t *>(h->group_cell.p),
                                             static_cast<int32_t *>(h->group_box.p));
    count_launch();
    if (n > 0 && h->tree_leaves) {
        k_leaf_mass<<<grid_for(n), kThreads, 0, s>>>(lfirst, lscan + n, xw, ms, static_cast<const double *>(h->leaf_ref.p),
                                                     n, static_cast<float4 *>(h->pos_leaf.p));
        count_launch();
    }
    if (n > 0)
        k_pos<<<grid_for(n), kThreads, 0, s>>>(n, xw, ms, lscan, gscan, static_cast<const double *>(h->leaf_ref.p),
                                               static_cast<const float4 *>(h->leaf_r4.p),
                                               static_cast<const float4 *>(h->group_r4.p),
                                               static_cast<float4 *>(h->pos_leaf.p),
                                               static_cast<float4 *>(h->pos_group.p));
        count_launch();
    k_cell_leaf_first<<<grid_for(h->n_cells + 1), kThreads, 0, s>>>(cell_first, lscan, h->n_cells,
                                                                    static_cast<int32_t *>(h->cell_leaf_first.p));
    count_launch();
    // device copies of the counts
    int32_t *cnt = static_cast<int32_t *>(h->counts.p);
    cudaMemcpyAsync(cnt + 0, lscan + n, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(cnt + 1, gscan + n, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (h->active && n > 0) {
        // the groups to sum in active-particle mode (buffers sized by the caller)
        int32_t *gact = static_cast<int32_t *>(h->group_act.p), *gacts = static_cast<int32_t *>(h->group_act_scan.p);
        const int32_t *perm = static_cast<const int32_t *>(h->keys_in_alt ? h->vals_alt.p : h->vals.p);
        k_group_active<<<grid_for(n), kThreads, 0, s>>>(gfirst, cnt + 1, perm, h->active, gact);
        count_launch();
        rc = scan_exclusive_i32(gact, gacts, n, cnt + 1, h->temp.p, s);
        if (rc) return rc;
        k_active_list<<<grid_for(n), kThreads, 0, s>>>(gact, gacts, cnt + 1,
                                                       static_cast<int32_t *>(h->active_list.p), cnt + 2);
        count_launch();
    }
    return cuda_check(cudaGetLastError(), "build kernels");
}

}  // namespace phpp
