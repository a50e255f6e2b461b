// PP direct summation over the cutoff leaf-pair list.
//
// One warp takes one target group at a time from a global queue (the task
// queue of Sec. 4.3, ground cells rolled in ascending order) and holds one
// target particle per lane in registers.  The source leaves of the group's
// list are streamed through shared memory: lanes load a leaf's particles with
// coalesced float4 loads, shift them into the group frame (one FP32 add of
// the pair's offset), drop those farther than R_cut from the group's bounding
// box, and append the rest to a per-warp buffer; a full buffer is summed with
// every lane reading the same source (shared-memory broadcast).
//
// Per pair (Eq. (split), Plummer factor, hard cutoff):
//   r2 = |d|^2,  w = m_j f(r) / (r2 + eps^2)^{3/2}  if r2 < rcut^2 else 0
//   f(r) = 2^(r2 c_e) h(t),  t = r / (R_s U) - 1,  h a degree-NPOLY polynomial
// with rsqrt (plus one Newton correction), sqrt and ex2 on the SFU.  Partial
// sums over runs of 16 sources are added to the total with Kahan compensation.
#include "handles.cuh"

namespace phpp {
namespace {

constexpr int kPPWarps = 8;
constexpr int kPPThreads = kPPWarps * 32;
constexpr int kJBuf = 256;

__device__ __forceinline__ float rsqrt_sfu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_sfu(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ex2_sfu(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct PPArgs {
    const BoxDev *boxes;
    const int32_t *n_groups;
    const int32_t *group_first;
    const int32_t *group_box;
    const float4 *group_h4;
    const float4 *pos_group;
    const float4 *pos_leaf;
    const int32_t *leaf_first;
    const int32_t *perm;
    const int64_t *group_off;
    const float4 *entries;
    int64_t cap;             // entries written (reads stop there)
    int32_t *queue;
    unsigned long long *n_inter;
    unsigned long long *n_staged;
    float *acc;
};

struct Kahan3 {
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    __device__ __forceinline__ void add(float px, float py, float pz)
    {
        float y, t;
        y = px - cx; t = sx + y; cx = (t - sx) - y; sx = t;
        y = py - cy; t = sy + y; cy = (t - sy) - y; sy = t;
        y = pz - cz; t = sz + y; cz = (t - sz) - y; sz = t;
    }
};

// One pair: accumulate m_j f(r) d / (r^2 + eps^2)^{3/2} into (px, py, pz).
template <int NPOLY>
__device__ __forceinline__ void interact(const float4 pj, const float4 xi, const float *poly, float eps2, float rcut2,
                                         float c_v, float c_e, float &px, float &py, float &pz)
{
    const float dx = pj.x - xi.x, dy = pj.y - xi.y, dz = pj.z - xi.z;
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    // (r2 + eps2)^(-3/2): SFU rsqrt y, then the first-order Newton
    // correction y^3 (1 + 3/2 (1 - x y^2)), which removes the SFU error
    const float x = r2 + eps2;
    const float y = rsqrt_sfu(x);
    const float y2 = y * y;
    const float y3 = y2 * y;
    const float e15 = fmaf(x * -1.5f, y2, 1.5f);
    const float inv3 = fmaf(y3, e15, y3);
    const float t = sqrt_sfu(r2 * c_v) - 1.f;
    float hp = poly[NPOLY];
#pragma unroll
    for (int q = NPOLY - 1; q >= 0; q--) hp = fmaf(hp, t, poly[q]);
    const float f = ex2_sfu(r2 * c_e) * hp;
    float w = (pj.w * f) * inv3;
    w = r2 < rcut2 ? w : 0.f;
    px = fmaf(w, dx, px);
    py = fmaf(w, dy, py);
    pz = fmaf(w, dz, pz);
}

// Sum a staged buffer: plain FP32 partial sums over runs of kChunk sources,
// each run added to the total with Kahan compensation.
constexpr int kChunk = 16;

template <int NPOLY>
__device__ __forceinline__ void sum_buffer(const float4 *buf, int nbuf, const float4 xi, const float *poly,
                                           float eps2, float rcut2, float c_v, float c_e, Kahan3 &k)
{
    int jj = 0;
    for (; jj + kChunk <= nbuf; jj += kChunk) {
        float px = 0.f, py = 0.f, pz = 0.f;
#pragma unroll 4
        for (int u = 0; u < kChunk; u++)
            interact<NPOLY>(buf[jj + u], xi, poly, eps2, rcut2, c_v, c_e, px, py, pz);
        k.add(px, py, pz);
    }
    if (jj < nbuf) {
        float px = 0.f, py = 0.f, pz = 0.f;
        for (; jj < nbuf; jj++) interact<NPOLY>(buf[jj], xi, poly, eps2, rcut2, c_v, c_e, px, py, pz);
        k.add(px, py, pz);
    }
}

template <int NPOLY>
__global__ void __launch_bounds__(kPPThreads, 4) k_pp_exact(PPArgs a)
{
    __shared__ float4 sbuf[kPPWarps][kJBuf];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    float4 *buf = sbuf[w];
    const int ng = *a.n_groups;
    unsigned long long inter = 0, staged = 0;
    for (;;) {
        int g = 0;
        if (lane == 0) g = atomicAdd(a.queue, 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ng) break;
        const int i0 = a.group_first[g], ni = a.group_first[g + 1] - i0;
        const BoxDev &bx = a.boxes[a.group_box[g]];
        float poly[NPOLY + 1];
#pragma unroll
        for (int q = 0; q <= NPOLY; q++) poly[q] = bx.poly[q];
        const float eps2 = bx.eps2, rcut2 = bx.rcut2, c_v = bx.c_v, c_e = bx.c_e, rf2 = bx.rfilt2;
        const float4 gh = a.group_h4[g];
        const float4 xi = lane < ni ? a.pos_group[i0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        Kahan3 k;
        int nbuf = 0;
        const int64_t e1 = a.group_off[g + 1] < a.cap ? a.group_off[g + 1] : a.cap;
        for (int64_t e = a.group_off[g]; e < e1; e++) {
            const float4 ent = a.entries[e];
            const int leaf = __float_as_int(ent.w);
            const int j1 = a.leaf_first[leaf + 1];
            for (int jb = a.leaf_first[leaf]; jb < j1; jb += 32) {
                const int j = jb + lane;
                float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
                bool keep = false;
                if (j < j1) {
                    p = a.pos_leaf[j];
                    p.x = __fadd_rn(p.x, ent.x);
                    p.y = __fadd_rn(p.y, ent.y);
                    p.z = __fadd_rn(p.z, ent.z);
                    const float qx = fmaxf(fabsf(p.x) - gh.x, 0.f);
                    const float qy = fmaxf(fabsf(p.y) - gh.y, 0.f);
                    const float qz = fmaxf(fabsf(p.z) - gh.z, 0.f);
                    keep = qx * qx + qy * qy + qz * qz < rf2;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                const int cnt = __popc(bal);
                if (nbuf + cnt > kJBuf) {
                    __syncwarp();
                    sum_buffer<NPOLY>(buf, nbuf, xi, poly, eps2, rcut2, c_v, c_e, k);
                    inter += (unsigned long long)nbuf * ni;
                    staged += nbuf;
                    nbuf = 0;
                    __syncwarp();
                }
                if (keep) buf[nbuf + __popc(bal & lt)] = p;
                nbuf += cnt;
            }
        }
        __syncwarp();
        sum_buffer<NPOLY>(buf, nbuf, xi, poly, eps2, rcut2, c_v, c_e, k);
        inter += (unsigned long long)nbuf * ni;
        staged += nbuf;
        __syncwarp();
        if (lane < ni) {
            const int64_t o = a.perm[i0 + lane];
            const float G = bx.G;
            a.acc[3 * o + 0] = G * (k.sx - k.cx);
            a.acc[3 * o + 1] = G * (k.sy - k.cy);
            a.acc[3 * o + 2] = G * (k.sz - k.cz);
        }
    }
    if (lane == 0 && inter) {
        atomicAdd(a.n_inter, inter);
        atomicAdd(a.n_staged, staged);
    }
}

// Number of (i, j) pairs with r^2 < rcut^2 in the lists, self pairs
// included (each target meets itself once, at d = 0): the work the cutoff
// keeps, counted with the PP kernel's own FP32 decision.
__global__ void __launch_bounds__(kPPThreads) k_count_within(PPArgs a)
{
    __shared__ float4 sbuf[kPPWarps][kJBuf];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    float4 *buf = sbuf[w];
    const int ng = *a.n_groups;
    unsigned long long cnt_within = 0;
    for (;;) {
        int g = 0;
        if (lane == 0) g = atomicAdd(a.queue, 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ng) break;
        const int i0 = a.group_first[g], ni = a.group_first[g + 1] - i0;
        const BoxDev &bx = a.boxes[a.group_box[g]];
        const float rcut2 = bx.rcut2;
        const float4 xi = lane < ni ? a.pos_group[i0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int64_t e1 = a.group_off[g + 1] < a.cap ? a.group_off[g + 1] : a.cap;
        for (int64_t e = a.group_off[g]; e < e1; e++) {
            const float4 ent = a.entries[e];
            const int leaf = __float_as_int(ent.w);
            const int j1 = a.leaf_first[leaf + 1];
            for (int jb = a.leaf_first[leaf]; jb < j1; jb += 32) {
                const int j = jb + lane;
                const bool ok = j < j1;
                float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
                if (ok) {
                    p = a.pos_leaf[j];
                    p.x = __fadd_rn(p.x, ent.x);
                    p.y = __fadd_rn(p.y, ent.y);
                    p.z = __fadd_rn(p.z, ent.z);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                __syncwarp();
                if (ok) buf[__popc(bal & lt)] = p;
                __syncwarp();
                const int nb = __popc(bal);
                for (int jj = 0; jj < nb; jj++) {
                    const float4 pj = buf[jj];
                    const float dx = pj.x - xi.x, dy = pj.y - xi.y, dz = pj.z - xi.z;
                    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    if (lane < ni && r2 < rcut2) cnt_within++;
                }
            }
        }
    }
    if (cnt_within) atomicAdd(a.n_inter, cnt_within);
}

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

static void pp_args(const ph_leaves *lv, const ph_pairs *pr, float *d_acc, PPArgs &a);

int count_within_device(const ph_leaves *lv, const ph_pairs *pr, cudaStream_t s)
{
    PPArgs a;
    pp_args(lv, pr, nullptr, a);
    int rc = cuda_check(cudaMemsetAsync(pr->work.p, 0, 24, s), "reset work queue");
    if (rc) return rc;
    k_count_within<<<sm_count() * 4, kPPThreads, 0, s>>>(a);
    count_launch();
    return cuda_check(cudaGetLastError(), "count kernel");
}

static void pp_args(const ph_leaves *lv, const ph_pairs *pr, float *d_acc, PPArgs &a)
{
    a.boxes = static_cast<const BoxDev *>(lv->boxes.p);
    a.n_groups = static_cast<const int32_t *>(lv->counts.p) + 1;
    a.group_first = static_cast<const int32_t *>(lv->group_first.p);
    a.group_box = static_cast<const int32_t *>(lv->group_box.p);
    a.group_h4 = static_cast<const float4 *>(lv->group_h4.p);
    a.pos_group = static_cast<const float4 *>(lv->pos_group.p);
    a.pos_leaf = static_cast<const float4 *>(lv->pos_leaf.p);
    a.leaf_first = static_cast<const int32_t *>(lv->leaf_first.p);
    a.perm = static_cast<const int32_t *>(lv->keys_in_alt ? lv->vals_alt.p : lv->vals.p);
    a.group_off = static_cast<const int64_t *>(pr->group_off.p);
    a.entries = static_cast<const float4 *>(pr->entries.p);
    a.cap = pr->capacity;
    char *work = static_cast<char *>(pr->work.p);
    a.queue = reinterpret_cast<int32_t *>(work);
    a.n_inter = reinterpret_cast<unsigned long long *>(work + 8);
    a.n_staged = reinterpret_cast<unsigned long long *>(work + 16);
    a.acc = d_acc;
}

int pp_exact_device(const ph_leaves *lv, const ph_pairs *pr, float *d_acc, cudaStream_t s)
{
    PPArgs a;
    pp_args(lv, pr, d_acc, a);
    int rc = cuda_check(cudaMemsetAsync(pr->work.p, 0, 24, s), "reset work queue");
    if (rc) return rc;
    const int grid = sm_count() * 4;
    switch (lv->poly_degree) {
    case 10: k_pp_exact<10><<<grid, kPPThreads, 0, s>>>(a); count_launch(); break;
    case 12: k_pp_exact<12><<<grid, kPPThreads, 0, s>>>(a); count_launch(); break;
    case 14: k_pp_exact<14><<<grid, kPPThreads, 0, s>>>(a); count_launch(); break;
    case 16: k_pp_exact<16><<<grid, kPPThreads, 0, s>>>(a); count_launch(); break;
    default: return fail(PH_ERR_STATE, "unsupported polynomial degree %d", lv->poly_degree);
    }
    return cuda_check(cudaGetLastError(), "pp kernel");
}

}  // namespace phpp
