// PP direct summation over the cutoff leaf-pair list.
//
// One warp takes one target group at a time from a global queue (the task
// queue of Sec. 4.3; in the pair builder's order of decreasing cost, or in
// ground-cell order along the curve) and holds one
// target particle per lane in registers.  The source leaves of the group's
// list are streamed through shared memory: lanes load the leaves' particles
// with float4 loads (32 useful loads per round whatever the leaf sizes),
// shift them into the group frame (one FP32 add of the pair's offset), drop
// those farther than R_cut from the group's bounding box, and append the rest
// to a per-warp buffer as pairs; a full buffer is summed with every lane
// reading the same two sources (shared-memory broadcast) and evaluating both
// with packed FP32x2 instructions.
//
// Per pair (Eq. (split), Plummer factor, hard cutoff):
//   r2 = |d|^2,  w = m_j f(r) / (r2 + eps^2)^{3/2}  if r2 < rcut^2 else 0
//   f(r) = 2^(r2 c_e) h(t),  t = r / (R_s U) - 1,  h a degree-NPOLY polynomial
// with rsqrt (plus one Newton correction), sqrt and ex2 on the SFU.  Partial
// sums over runs of 16 sources are added to the total with Kahan compensation.
#include <cstring>

#include "factor.cuh"
#include "handles.cuh"

namespace phpp {
namespace {

#ifndef PHPP_PP_WARPS
#define PHPP_PP_WARPS 8
#endif
#ifndef PHPP_PP_BLOCKS0
#define PHPP_PP_BLOCKS0 2
#endif
#ifndef PHPP_PP_BLOCKS1
#define PHPP_PP_BLOCKS1 3
#endif
constexpr int kPPWarps = PHPP_PP_WARPS;
constexpr int kPPThreads = kPPWarps * 32;
// resident blocks per SM of the two kernel shapes (pp_variant 0 and 1): the
// register budget each instantiation is compiled for, and the persistent
// grid (SMs x blocks)
constexpr int kBlocks0 = PHPP_PP_BLOCKS0;
constexpr int kBlocks1 = PHPP_PP_BLOCKS1;
constexpr int kJBuf = 256;      // staged sources per warp (even)


// Constants of one box, each duplicated into both halves of a pair.
struct PairConsts {
    f2_t poly[kMaxPoly + 1];
    f2_t s2, eps2s, c_t, c_e, m1;
    float rcut2, rfilt2;
};

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
    const float4 *entries;   // offset xyz, first source particle (bits)
    const uint8_t *ecount;   // particles in the entry's leaf - 1
    int64_t cap;             // entries written (reads stop there)
    int32_t *queue;
    unsigned long long *n_inter;
    unsigned long long *n_staged;
    float *acc;
    const float *mlp_w;      // learned factor weights [321] (learned kernel)
    // constants shared by every box (the uniform kernels read them straight
    // from the parameter bank instead of holding them in registers)
    PairConsts uc;
    // the leaf-pair walk of the direct mode (no stored list)
    const int32_t *group_cell;       // global ground cell of each group
    const float4 *group_c4;          // group box centre in its cell frame
    const float4 *group_r4, *leaf_r4;   // reference points in FP32 (exact)
    const double *group_ref, *leaf_ref; // the same in FP64 (periodic images)
    const float4 *leaf_c4, *leaf_h4; // leaf boxes; w: first particle, particles (int bits)
    const int32_t *cell_leaf_first;  // first leaf of each ground cell
    // tabulated factor (PH_G_TABLE): kTabN + 1 nodes (f(r_i), f'(r_i) dr)
    const float2 *table;
    float tab_scale2;                // (kTabN / rcut)^2
    int64_t n_pos;                   // rows of pos_leaf (bounds checks)
    const int32_t *order;            // queue slot -> group (groups by decreasing cost), or NULL
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

// Two sources (A = x0 x1 y0 y1, B = z0 z1 m0 m1) against one target: add
// m_j f(r) d / (r^2 + eps^2)^{3/2} into the pair accumulators.
template <int NPOLY>
__device__ __forceinline__ void interact2(const float4 a, const float4 b, const f2_t xi, const f2_t yi, const f2_t zi,
                                          const PairConsts &c, f2_t &px, f2_t &py, f2_t &pz)
{
    const f2_t dx = sub2(pk(a.x, a.y), xi), dy = sub2(pk(a.z, a.w), yi), dz = sub2(pk(b.x, b.y), zi);
    f2_t r2 = mul2(dx, dx);
    r2 = fma2(dy, dy, r2);
    r2 = fma2(dz, dz, r2);
    // (r^2 + eps^2)^(-3/2) up to the box's power-of-two scale: one SFU
    // rsqrt of x^3 with x = r^2 s2 + eps2s = O(1), so the SFU's relative
    // error enters once (not tripled, as it would be in rsqrt(x)^3)
    const f2_t x = fma2(r2, c.s2, c.eps2s);
    const f2_t x3 = mul2(mul2(x, x), x);
    const f2_t inv3 = pk(rsqrt_sfu(lo_of(x3)), rsqrt_sfu(hi_of(x3)));
    const f2_t t = fma2(pk(sqrt_sfu(lo_of(r2)), sqrt_sfu(hi_of(r2))), c.c_t, c.m1);   // 2 r / rcut - 1
    f2_t h = c.poly[NPOLY];
#pragma unroll
    for (int q = NPOLY - 1; q >= 0; q--) h = fma2(h, t, c.poly[q]);
    const f2_t ea = mul2(r2, c.c_e);
    const f2_t f = mul2(pk(ex2_sfu(lo_of(ea)), ex2_sfu(hi_of(ea))), h);
    const f2_t w = mul2(mul2(pk(b.z, b.w), f), inv3);
    const float w0 = lo_of(r2) < c.rcut2 ? lo_of(w) : 0.f;
    const float w1 = hi_of(r2) < c.rcut2 ? hi_of(w) : 0.f;
    const f2_t wm = pk(w0, w1);
    px = fma2(wm, dx, px);
    py = fma2(wm, dy, py);
    pz = fma2(wm, dz, pz);
}

// Sum a staged buffer of npair source pairs.  With kSplit lanes per target
// (target groups of 32 / kSplit particles) lane slot h takes the pairs
// h, h + kSplit, h + 2 kSplit, ...; the buffer is padded with massless
// sources to a whole number of pairs per slot.  Plain FP32 partial sums over
// runs of kRun pairs, each run added to the lane's total with Kahan
// compensation.
#ifndef PHPP_PP_RUN
#define PHPP_PP_RUN 8
#endif
#ifndef PHPP_PP_UNROLL
#define PHPP_PP_UNROLL 8
#endif
constexpr int kRun = PHPP_PP_RUN;
constexpr int kUnroll = PHPP_PP_UNROLL;

template <int NPOLY, int kSplit>
__device__ __forceinline__ void sum_buffer(const float4 *A, const float4 *B, int npair, int h, const f2_t xi,
                                           const f2_t yi, const f2_t zi, const PairConsts &c, Kahan3 &k)
{
    const int nstep = npair / kSplit;
    int s = 0;
    for (; s + kRun <= nstep; s += kRun) {
        f2_t px = 0ull, py = 0ull, pz = 0ull;
#pragma unroll kUnroll
        for (int u = 0; u < kRun; u++) {
            const int m = (s + u) * kSplit + h;
            interact2<NPOLY>(A[m], B[m], xi, yi, zi, c, px, py, pz);
        }
        k.add(lo_of(px) + hi_of(px), lo_of(py) + hi_of(py), lo_of(pz) + hi_of(pz));
    }
    if (s < nstep) {
        f2_t px = 0ull, py = 0ull, pz = 0ull;
        for (; s < nstep; s++) {
            const int m = s * kSplit + h;
            interact2<NPOLY>(A[m], B[m], xi, yi, zi, c, px, py, pz);
        }
        k.add(lo_of(px) + hi_of(px), lo_of(py) + hi_of(py), lo_of(pz) + hi_of(pz));
    }
}

// Tabulated factor (PH_G_TABLE, the pre-computed table of Sec. 3.1): f at
// kTabN + 1 nodes r_i = i rcut / kTabN with its derivative times the node
// spacing; a pair takes the node nearest to r and its slope,
// f = f_i + (r / dr - i) f'_i dr.  The node index comes from the FP32
// round-to-nearest of r / dr + 1.5 2^23 (exact for r / dr < 2^22), clamped
// to the last node (pairs beyond rcut are removed by the cutoff select).
constexpr int kTabN = 4096;
constexpr float kMagic = 12582912.f;   // 1.5 2^23
__device__ __forceinline__ void interact2_table(const float4 a, const float4 b, const f2_t xi, const f2_t yi,
                                                const f2_t zi, const PairConsts &c, const float2 *tab,
                                                const f2_t scale2, f2_t &px, f2_t &py, f2_t &pz)
{
    const f2_t dx = sub2(pk(a.x, a.y), xi), dy = sub2(pk(a.z, a.w), yi), dz = sub2(pk(b.x, b.y), zi);
    f2_t r2 = mul2(dx, dx);
    r2 = fma2(dy, dy, r2);
    r2 = fma2(dz, dz, r2);
    const f2_t x = fma2(r2, c.s2, c.eps2s);
    const f2_t x3 = mul2(mul2(x, x), x);
    const f2_t inv3 = pk(rsqrt_sfu(lo_of(x3)), rsqrt_sfu(hi_of(x3)));
    const f2_t q = mul2(r2, scale2);
    const f2_t u = pk(sqrt_sfu(lo_of(q)), sqrt_sfu(hi_of(q)));   // r / dr
    const f2_t mg = pk(kMagic, kMagic);
    const f2_t y = add2(u, mg);
    const f2_t fr = sub2(u, sub2(y, mg));                            // r / dr - nearest node
    int i0 = min(__float_as_int(lo_of(y)) - 0x4B400000, kTabN);
    int i1 = min(__float_as_int(hi_of(y)) - 0x4B400000, kTabN);
    if (!in_bounds(i0, kTabN + 1, BS_F_TABLE)) i0 = 0;
    if (!in_bounds(i1, kTabN + 1, BS_F_TABLE)) i1 = 0;
    const float2 t0 = tab[i0], t1 = tab[i1];
    const f2_t f = pk(fmaf(t0.y, lo_of(fr), t0.x), fmaf(t1.y, hi_of(fr), t1.x));
    const f2_t w = mul2(mul2(pk(b.z, b.w), f), inv3);
    const float w0 = lo_of(r2) < c.rcut2 ? lo_of(w) : 0.f;
    const float w1 = hi_of(r2) < c.rcut2 ? hi_of(w) : 0.f;
    const f2_t wm = pk(w0, w1);
    px = fma2(wm, dx, px);
    py = fma2(wm, dy, py);
    pz = fma2(wm, dz, pz);
}

template <int kSplit>
__device__ __forceinline__ void sum_buffer_table(const float4 *A, const float4 *B, int npair, int h, const f2_t xi,
                                                 const f2_t yi, const f2_t zi, const PairConsts &c,
                                                 const float2 *tab, const f2_t scale2, Kahan3 &k)
{
    const int nstep = npair / kSplit;
    int s = 0;
    for (; s + kRun <= nstep; s += kRun) {
        f2_t px = 0ull, py = 0ull, pz = 0ull;
#pragma unroll
        for (int u = 0; u < kRun; u++) {
            const int m = (s + u) * kSplit + h;
            interact2_table(A[m], B[m], xi, yi, zi, c, tab, scale2, px, py, pz);
        }
        k.add(lo_of(px) + hi_of(px), lo_of(py) + hi_of(py), lo_of(pz) + hi_of(pz));
    }
    if (s < nstep) {
        f2_t px = 0ull, py = 0ull, pz = 0ull;
        for (; s < nstep; s++) {
            const int m = s * kSplit + h;
            interact2_table(A[m], B[m], xi, yi, zi, c, tab, scale2, px, py, pz);
        }
        k.add(lo_of(px) + hi_of(px), lo_of(py) + hi_of(py), lo_of(pz) + hi_of(pz));
    }
}

// Learned factor.  The network is evaluated warp-wide (32 pairs per call on
// the tensor cores), and only pairs within R_cut need it: each lane takes
// its next source each step, and the pairs with 0 < r^2 < R_cut^2 are
// appended (ballot order) to a per-warp ring of 64 slots holding their
// separation and mass; whenever 32 pairs are pending, lane k evaluates the
// k-th oldest (softened inverse cube, network, weight) and writes the
// entry's force back into its slot, and every lane adds the forces of the
// entries it owns in slot order (a deterministic order).  The evaluated half
// of the ring is then free and the pending entries stay where they are.
// Pairs beyond R_cut, the self pair and coincident pairs contribute exactly
// zero and are not queued.
constexpr int kLQ = 64;   // ring slots per warp (at most 31 pending + 32 new)
struct LearnedQueue {
    float4 *q;                       // per-warp ring in shared memory: (dx, dy, dz, m_j);
                                     // slot kLQ holds zeros
    const float4 *l1;                // layer 1's table (shared memory)
    int head = 0;                    // slot of the oldest pending entry: 0 or 32 (warp-uniform)
    int n = 0;                       // pending entries (warp-uniform)
    unsigned long long own = 0;      // ring slots this lane's entries occupy
};

// Evaluate the `ne` (<= 32) oldest entries and add their forces to their
// owners' sums (px, py, pz).
__device__ __forceinline__ void learned_flush(LearnedQueue &q, int ne, int lane, float eps2, float c_v,
                                              const MlpLane &L, float &px, float &py, float &pz)
{
    __syncwarp();
    const bool on = lane < ne;
    float4 *win = q.q + q.head;      // the 32 slots being evaluated
    const float4 e = on ? win[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float r2 = fmaf(e.z, e.z, fmaf(e.y, e.y, e.x * e.x));   // as when it was queued
    const float y = rsqrt_sfu(r2 + eps2);
    const float inv3 = y * y * y;
    const float t = sqrt_sfu(r2 * c_v) - 1.f;
    const float gh = mlp_warp_eval(t, L, q.l1);
    const float w = on ? (e.w * gh) * inv3 : 0.f;
    win[lane] = make_float4(w * e.x, w * e.y, w * e.z, 0.f);   // the slot this lane read
    __syncwarp();
    // the lane's entries in slot order, two loads in flight (a missing second
    // one reads the zero slot)
    unsigned m32 = (unsigned)(q.own >> q.head) & (ne == 32 ? 0xffffffffu : ((1u << ne) - 1u));
    while (m32) {
        const int b0 = q.head + __ffs(m32) - 1;
        m32 &= m32 - 1u;
        const int b1 = m32 ? q.head + __ffs(m32) - 1 : kLQ;
        m32 &= m32 - 1u;
        const float4 f0 = q.q[b0], f1 = q.q[b1];
        px += f0.x;
        py += f0.y;
        pz += f0.z;
        px += f1.x;
        py += f1.y;
        pz += f1.z;
    }
    __syncwarp();
    q.own &= q.head ? 0x00000000ffffffffull : 0xffffffff00000000ull;
    q.head ^= 32;
    q.n -= ne;
}

// One step of the learned sum: a source at separation (dx, dy, dz) and r^2
// from the lane's target; a pair within R_cut joins the queue, and 32
// pending pairs are evaluated.
__device__ __forceinline__ void learned_step(float dx, float dy, float dz, float r2, float mj, bool live, unsigned lt,
                                             int lane, float eps2, float rcut2, float c_v, const MlpLane &L,
                                             LearnedQueue &q, float &px, float &py, float &pz)
{
    // (lanes without a target, massless padding and r = 0 contribute nothing)
    const bool use = live && r2 < rcut2 && r2 > 0.f && mj != 0.f;
    const unsigned bal = __ballot_sync(0xffffffffu, use);
    const int slot = (q.head + q.n + __popc(bal & lt)) & (kLQ - 1);
    if (use && in_bounds(slot, kLQ, BS_PP_QUEUE)) {
        q.q[slot] = make_float4(dx, dy, dz, mj);
        q.own |= 1ull << slot;
    }
    q.n += __popc(bal);
    if (q.n >= 32) learned_flush(q, 32, lane, eps2, c_v, L, px, py, pz);
}

// The staged sources against the lane's target; the forces of this buffer
// are summed plainly and added to the compensated total once.
template <int kSplit>
__device__ __forceinline__ void sum_buffer_learned(const float4 *A, const float4 *B, int nbuf, int h, const float4 xi,
                                                   bool live, float eps2, float rcut2, float c_v, const MlpLane &L,
                                                   LearnedQueue &q, Kahan3 &k)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    float px = 0.f, py = 0.f, pz = 0.f;
    if (kSplit == 1) {
        // both sources of a staged pair per iteration: (x, x', y, y') and (z, z', m, m')
        const f2_t xi2 = pk(xi.x, xi.x), yi2 = pk(xi.y, xi.y), zi2 = pk(xi.z, xi.z);
        for (int m = 0; m < nbuf / 2; m++) {
            const float4 a = A[m], b = B[m];
            const f2_t dx = sub2(pk(a.x, a.y), xi2), dy = sub2(pk(a.z, a.w), yi2), dz = sub2(pk(b.x, b.y), zi2);
            const f2_t r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
            learned_step(lo_of(dx), lo_of(dy), lo_of(dz), lo_of(r2), b.z, live, lt, lane, eps2, rcut2, c_v, L, q,
                         px, py, pz);
            learned_step(hi_of(dx), hi_of(dy), hi_of(dz), hi_of(r2), b.w, live, lt, lane, eps2, rcut2, c_v, L, q,
                         px, py, pz);
        }
    } else {
        const float *Af = reinterpret_cast<const float *>(A), *Bf = reinterpret_cast<const float *>(B);
        const int nstep = nbuf / kSplit;
        for (int jj = 0; jj < nstep; jj++) {
            const int j = jj * kSplit + h;
            const int m = j >> 1, sl = j & 1;
            const float dx = Af[m * 4 + sl] - xi.x, dy = Af[m * 4 + 2 + sl] - xi.y, dz = Bf[m * 4 + sl] - xi.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            learned_step(dx, dy, dz, r2, Bf[m * 4 + 2 + sl], live, lt, lane, eps2, rcut2, c_v, L, q, px, py, pz);
        }
    }
    k.add(px, py, pz);
}

template <int kSplit>
__device__ __forceinline__ int pad_sources(float *Af, float *Bf, int nbuf, int lane)
{
    const int padded = (nbuf + 2 * kSplit - 1) / (2 * kSplit) * (2 * kSplit);
    const int j = nbuf + lane;
    if (j < padded) {
        const int m = j >> 1, sl = j & 1;
        Af[m * 4 + sl] = 0.f;
        Af[m * 4 + 2 + sl] = 0.f;
        Bf[m * 4 + sl] = 0.f;
        Bf[m * 4 + 2 + sl] = 0.f;
    }
    return padded;
}

__device__ __forceinline__ int warp_incl_scan_i(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// 32 consecutive pair entries, one per lane, with the exclusive prefix sums
// of their leaf sizes: concatenated particle q of the batch lies in the
// entry whose range [excl, excl + count) holds q, at row base + q of the
// leaf-relative positions (base = first particle - excl).
struct EntryBatch {
    float4 ent;
    int base, excl, total;
    // this lane's entry given directly (cnt = 0: no entry)
    __device__ __forceinline__ void set(float4 e, int cnt, int lane)
    {
        ent = e;
        const int incl = warp_incl_scan_i(cnt, lane);
        excl = incl - cnt;
        base = __float_as_int(ent.w) - excl;
        total = __shfl_sync(0xffffffffu, incl, 31);
    }
    __device__ __forceinline__ void load(const PPArgs &a, int64_t eb, int64_t e1, int lane)
    {
        const int64_t e = eb + lane;
        int cnt = 0;
        ent = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < e1) {
            ent = a.entries[e];
            cnt = (int)a.ecount[e] + 1;
        }
        const int incl = warp_incl_scan_i(cnt, lane);
        excl = incl - cnt;
        base = __float_as_int(ent.w) - excl;
        total = __shfl_sync(0xffffffffu, incl, 31);
    }
};

// One staging round: the particle each lane loads (in flight until used) and
// the offset of its entry.  The entry of lane t's particle q = q0 + t is
// found without a search: the entries starting inside [q0, q0 + 32) set
// their start bit in a warp-wide OR, so the owner is the number of entries
// started before q0 (`before`, carried from round to round) plus the start
// bits at or below t, minus one.
struct Round {
    float4 p;
    float ox, oy, oz;
    bool valid;
    __device__ __forceinline__ void issue(const PPArgs &a, const EntryBatch &b, int q0, int lane, int &before)
    {
        const int q = q0 + lane;
        const unsigned s = (unsigned)(b.excl - q0);
        const unsigned starts = __reduce_or_sync(0xffffffffu, s < 32u ? 1u << s : 0u);
        const int o = before + __popc(starts & (0xffffffffu >> (31 - lane))) - 1;
        before += __popc(starts);
        const int j = __shfl_sync(0xffffffffu, b.base, o) + q;
        ox = __shfl_sync(0xffffffffu, b.ent.x, o);
        oy = __shfl_sync(0xffffffffu, b.ent.y, o);
        oz = __shfl_sync(0xffffffffu, b.ent.z, o);
        valid = q < b.total;
        p = (valid && in_bounds(j, a.n_pos, BS_PP_SOURCE)) ? a.pos_leaf[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
};

// Source staging and summation for one target group.  Entries are taken 32
// at a time, one per lane; the lanes' leaf sizes are prefix-summed and the
// concatenated source particles are loaded 32 per round, each lane finding
// the entry of its particle from the start bits of the round (see Round), so
// that every lane loads a useful particle whatever the leaf sizes.  Kept sources
// are written as pairs into the warp's buffer; a full buffer is summed.
// kMinBlocks: resident 8-warp blocks per SM the register budget must allow
// (2: up to 128 registers, deeper unrolled pair loop; 3: up to 80).
// kSplit: lanes per target (target groups of 32 / kSplit particles).
// kUniform: every box has the same factor constants, read from the kernel's
// parameter bank (no registers); else they are loaded per group.
template <int NPOLY, bool kLearned, int kMinBlocks, int kSplit, bool kUniform, bool kTable = false>
__global__ void __launch_bounds__(kPPThreads, kMinBlocks) k_pp(PPArgs a)
{
    __shared__ float4 sA[kPPWarps][kJBuf / 2];
    __shared__ float4 sB[kPPWarps][kJBuf / 2];
    __shared__ float4 sQ[kLearned ? kPPWarps : 1][kLearned ? kLQ + 1 : 1];   // learned: the pair queue
    extern __shared__ float4 sDyn[];   // dynamic: the factor table (kTable) or layer 1's table (kLearned)
    float2 *const sTab = reinterpret_cast<float2 *>(sDyn);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    float4 *A = sA[w], *Bq = sB[w];
    float *Af = reinterpret_cast<float *>(A), *Bf = reinterpret_cast<float *>(Bq);
    const int ng = *a.n_groups;
    unsigned long long inter = 0, staged = 0;
    MlpLane L;
    if (kLearned) {
        mlp_lane_load(a.mlp_w, L);
        l1_table_fill(a.mlp_w, sDyn);
        __syncthreads();
    }
    if (kTable) {
        for (int i = threadIdx.x; i <= kTabN; i += blockDim.x) sTab[i] = a.table[i];
        __syncthreads();
    }
    for (;;) {
        int g = 0;
        if (lane == 0) {
            g = atomicAdd(a.queue, 1);
            if (a.order && g < ng) g = a.order[g];   // the queue's order (a permutation of the groups)
        }
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ng) break;
        const int i0 = a.group_first[g], ni = a.group_first[g + 1] - i0;
        const BoxDev &bx = a.boxes[a.group_box[g]];
        PairConsts cl;
        if (!kUniform) {
#pragma unroll
            for (int q = 0; q <= NPOLY; q++) cl.poly[q] = pk(bx.poly[q], bx.poly[q]);
            cl.s2 = pk(bx.s2, bx.s2);
            cl.eps2s = pk(bx.eps2s, bx.eps2s);
            cl.c_t = pk(bx.c_t, bx.c_t);
            cl.c_e = pk(bx.c_e, bx.c_e);
            cl.m1 = pk(-1.f, -1.f);
            cl.rcut2 = bx.rcut2;
            cl.rfilt2 = bx.rfilt2;
        }
        const PairConsts &c = kUniform ? a.uc : cl;
        const float rf2 = c.rfilt2;
        const float4 gh = a.group_h4[g];
        constexpr int G = 32 / kSplit;
        const int ti = lane & (G - 1), hs = lane / G;   // target slot, source slot
        const float4 xi4 = ti < ni ? a.pos_group[i0 + ti] : make_float4(0.f, 0.f, 0.f, 0.f);
        const f2_t xi = pk(xi4.x, xi4.x), yi = pk(xi4.y, xi4.y), zi = pk(xi4.z, xi4.z);
        Kahan3 k;
        int nbuf = 0;
        LearnedQueue lq;
        if (kLearned) {
            lq.q = sQ[kLearned ? w : 0];
            lq.l1 = sDyn;
            if (lane == 0) lq.q[kLQ] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int64_t e1 = a.group_off[g + 1] < a.cap ? a.group_off[g + 1] : a.cap;
        // Entries are taken 32 at a time; each round loads 32 concatenated
        // source particles of the batch, one per lane.
        for (int64_t eb = a.group_off[g]; eb < e1; eb += 32) {
            EntryBatch bt;
            bt.load(a, eb, e1, lane);
            int before = 0;
            for (int q0 = 0; q0 < bt.total; q0 += 32) {
                Round cur;
                cur.issue(a, bt, q0, lane, before);
                float4 p = cur.p;
                bool keep = false;
                if (cur.valid) {
                    p.x = __fadd_rn(p.x, cur.ox);
                    p.y = __fadd_rn(p.y, cur.oy);
                    p.z = __fadd_rn(p.z, cur.oz);
                    const float qx = fmaxf(fabsf(p.x) - gh.x, 0.f);
                    const float qy = fmaxf(fabsf(p.y) - gh.y, 0.f);
                    const float qz = fmaxf(fabsf(p.z) - gh.z, 0.f);
                    keep = qx * qx + qy * qy + qz * qz < rf2;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                const int nk = __popc(bal);
                if (nbuf + nk > kJBuf) {
                    const int padded = pad_sources<kSplit>(Af, Bf, nbuf, lane);
                    __syncwarp();
                    if (kLearned)
                        sum_buffer_learned<kSplit>(A, Bq, padded, hs, xi4, ti < ni, bx.eps2, bx.rcut2, bx.c_v, L, lq, k);
                    else if (kTable)
                        sum_buffer_table<kSplit>(A, Bq, padded >> 1, hs, xi, yi, zi, c, sTab,
                                                 pk(a.tab_scale2, a.tab_scale2), k);
                    else
                        sum_buffer<NPOLY, kSplit>(A, Bq, padded >> 1, hs, xi, yi, zi, c, k);
                    inter += (unsigned long long)nbuf * ni;
                    staged += nbuf;
                    nbuf = 0;
                    __syncwarp();
                }
                const int idx = nbuf + __popc(bal & lt);
                if (keep && in_bounds(idx, kJBuf, BS_PP_STAGE)) {
                    const int m = idx >> 1, sl = idx & 1;
                    Af[m * 4 + sl] = p.x;
                    Af[m * 4 + 2 + sl] = p.y;
                    Bf[m * 4 + sl] = p.z;
                    Bf[m * 4 + 2 + sl] = p.w;
                }
                nbuf += nk;
            }
        }
        const int padded = pad_sources<kSplit>(Af, Bf, nbuf, lane);
        __syncwarp();
        if (kLearned)
            sum_buffer_learned<kSplit>(A, Bq, padded, hs, xi4, ti < ni, bx.eps2, bx.rcut2, bx.c_v, L, lq, k);
        else if (kTable)
            sum_buffer_table<kSplit>(A, Bq, padded >> 1, hs, xi, yi, zi, c, sTab, pk(a.tab_scale2, a.tab_scale2), k);
        else
            sum_buffer<NPOLY, kSplit>(A, Bq, padded >> 1, hs, xi, yi, zi, c, k);
        inter += (unsigned long long)nbuf * ni;
        staged += nbuf;
        if (kLearned && lq.n > 0) {
            // the queue's last, partial batch
            float px = 0.f, py = 0.f, pz = 0.f;
            learned_flush(lq, lq.n, lane, bx.eps2, bx.c_v, L, px, py, pz);
            k.add(px, py, pz);
        }
        __syncwarp();
        // the kSplit source slots of a target add up their compensated totals
        float tx = k.sx - k.cx, ty = k.sy - k.cy, tz = k.sz - k.cz;
#pragma unroll
        for (int o = G; o < 32; o <<= 1) {
            tx += __shfl_xor_sync(0xffffffffu, tx, o);
            ty += __shfl_xor_sync(0xffffffffu, ty, o);
            tz += __shfl_xor_sync(0xffffffffu, tz, o);
        }
        if (hs == 0 && ti < ni) {
            const int64_t o = a.perm[i0 + ti];
            const float Gc = kLearned ? bx.G : bx.c_g;
            a.acc[3 * o + 0] = Gc * tx;
            a.acc[3 * o + 1] = Gc * ty;
            a.acc[3 * o + 2] = Gc * tz;
        }
    }
    if (lane == 0 && inter) {
        atomicAdd(a.n_inter, inter);
        atomicAdd(a.n_staged, staged);
    }
}

// Direct mode (exact factor): k_pp without a stored pair list.  Each group's
// leaf pairs are found here as the pair builder finds them -- lane t < 27
// takes neighbour cell t, the candidate leaves are box-tested in the same
// order -- and queued until 32 make a batch, so the batches, the staging and
// the sums are those of k_pp over the list, bit for bit.  The staging loop
// is repeated here rather than shared with k_pp: sharing it (a template
// switch around a common loop) changed the list kernel's register allocation
// and cost it 2.5 %.  For the same reason the walk's arguments sit at the end
// of PPArgs.
template <int NPOLY, int kMinBlocks, int kSplit, bool kUniform>
__global__ void __launch_bounds__(kPPThreads, kMinBlocks) k_pp_walk(PPArgs a)
{
    __shared__ float4 sA[kPPWarps][kJBuf / 2];
    __shared__ float4 sB[kPPWarps][kJBuf / 2];
    // direct mode: cell runs and the queue of found entries
    __shared__ int2 sRun[kPPWarps][32];
    __shared__ float4 sQEnt[kPPWarps][64];
    __shared__ int sQCnt[kPPWarps][64];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    float4 *A = sA[w], *Bq = sB[w];
    float *Af = reinterpret_cast<float *>(A), *Bf = reinterpret_cast<float *>(Bq);
    const int ng = *a.n_groups;
    unsigned long long inter = 0, staged = 0;
    for (;;) {
        int g = 0;
        if (lane == 0) g = atomicAdd(a.queue, 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ng) break;
        const int i0 = a.group_first[g], ni = a.group_first[g + 1] - i0;
        const BoxDev &bx = a.boxes[a.group_box[g]];
        PairConsts cl;
        if (!kUniform) {
#pragma unroll
            for (int q = 0; q <= NPOLY; q++) cl.poly[q] = pk(bx.poly[q], bx.poly[q]);
            cl.s2 = pk(bx.s2, bx.s2);
            cl.eps2s = pk(bx.eps2s, bx.eps2s);
            cl.c_t = pk(bx.c_t, bx.c_t);
            cl.c_e = pk(bx.c_e, bx.c_e);
            cl.m1 = pk(-1.f, -1.f);
            cl.rcut2 = bx.rcut2;
            cl.rfilt2 = bx.rfilt2;
        }
        const PairConsts &c = kUniform ? a.uc : cl;
        const float rf2 = c.rfilt2;
        const float4 gh = a.group_h4[g];
        constexpr int G = 32 / kSplit;
        const int ti = lane & (G - 1), hs = lane / G;   // target slot, source slot
        const float4 xi4 = ti < ni ? a.pos_group[i0 + ti] : make_float4(0.f, 0.f, 0.f, 0.f);
        const f2_t xi = pk(xi4.x, xi4.x), yi = pk(xi4.y, xi4.y), zi = pk(xi4.z, xi4.z);
        Kahan3 k;
        int nbuf = 0;
        // The source particles of a batch of (up to) 32 entries, one per lane:
        // each round loads 32 concatenated particles, one per lane.
        auto stage_batch = [&](const EntryBatch &bt) {
            int before = 0;
            for (int q0 = 0; q0 < bt.total; q0 += 32) {
                Round cur;
                cur.issue(a, bt, q0, lane, before);
                float4 p = cur.p;
                bool keep = false;
                if (cur.valid) {
                    p.x = __fadd_rn(p.x, cur.ox);
                    p.y = __fadd_rn(p.y, cur.oy);
                    p.z = __fadd_rn(p.z, cur.oz);
                    const float qx = fmaxf(fabsf(p.x) - gh.x, 0.f);
                    const float qy = fmaxf(fabsf(p.y) - gh.y, 0.f);
                    const float qz = fmaxf(fabsf(p.z) - gh.z, 0.f);
                    keep = qx * qx + qy * qy + qz * qz < rf2;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                const int nk = __popc(bal);
                if (nbuf + nk > kJBuf) {
                    const int padded = pad_sources<kSplit>(Af, Bf, nbuf, lane);
                    __syncwarp();
                    sum_buffer<NPOLY, kSplit>(A, Bq, padded >> 1, hs, xi, yi, zi, c, k);
                    inter += (unsigned long long)nbuf * ni;
                    staged += nbuf;
                    nbuf = 0;
                    __syncwarp();
                }
                const int idx = nbuf + __popc(bal & lt);
                if (keep && in_bounds(idx, kJBuf, BS_PP_STAGE)) {
                    const int m = idx >> 1, sl = idx & 1;
                    Af[m * 4 + sl] = p.x;
                    Af[m * 4 + 2 + sl] = p.y;
                    Bf[m * 4 + sl] = p.z;
                    Bf[m * 4 + 2 + sl] = p.w;
                }
                nbuf += nk;
            }
        };
        {
            // Direct mode: the leaf pairs of the group are found here, as the
            // pair builder finds them (same test, same order), and queued
            // until 32 make a batch.  Lane t < 27 takes neighbour cell t.
            const int ns = bx.nside;
            const int ground = a.group_cell[g] - bx.cell_base;
            const int gx = ground / (ns * ns), gy = (ground / ns) % ns, gz = ground % ns;
            const float4 gc = a.group_c4[g];
            const float hc = (float)bx.h;
            int l0 = 0, cnt = 0;
            if (lane < 27) {
                const int dx = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dz = lane % 3 - 1;
                const int ax = gx + dx, ay = gy + dy, az = gz + dz;
                const int sx = ax < 0 ? -1 : (ax >= ns ? 1 : 0);
                const int sy = ay < 0 ? -1 : (ay >= ns ? 1 : 0);
                const int sz = az < 0 ? -1 : (az >= ns ? 1 : 0);
                const int nc = bx.cell_base + ((ax - sx * ns) * ns + (ay - sy * ns)) * ns + (az - sz * ns);
                const float qx = fmaxf(fmaxf(dx * hc - (gc.x + gh.x), (gc.x - gh.x) - (dx + 1) * hc), 0.f);
                const float qy = fmaxf(fmaxf(dy * hc - (gc.y + gh.y), (gc.y - gh.y) - (dy + 1) * hc), 0.f);
                const float qz = fmaxf(fmaxf(dz * hc - (gc.z + gh.z), (gc.z - gh.z) - (dz + 1) * hc), 0.f);
                if (qx * qx + qy * qy + qz * qz < rf2 * 1.0001f) {
                    l0 = a.cell_leaf_first[nc];
                    cnt = a.cell_leaf_first[nc + 1] - l0;
                }
            }
            const int cincl = warp_incl_scan_i(cnt, lane);
            const int cexcl = cincl - cnt;
            const int ctotal = __shfl_sync(0xffffffffu, cincl, 31);
            const unsigned nonempty = __ballot_sync(0xffffffffu, cnt > 0);
            if (cnt > 0) sRun[w][__popc(nonempty & lt)] = make_int2(lane, l0 - cexcl);
            __syncwarp();
            const float4 gr4 = a.group_r4[g];
            int qn = 0;        // queued entries
            int runs = 0;      // cell runs started before c0
            for (int c0 = 0; c0 < ctotal; c0 += 32) {
                const int q = c0 + lane;
                const unsigned sq = (unsigned)(cexcl - c0);
                const unsigned starts = __reduce_or_sync(0xffffffffu, (cnt > 0 && sq < 32u) ? 1u << sq : 0u);
                const int r = runs + __popc(starts & (0xffffffffu >> (31 - lane))) - 1;
                runs += __popc(starts);
                const int2 ru = sRun[w][r];
                const int o = ru.x;
                const int odx = o / 9 - 1, ody = (o / 3) % 3 - 1, odz = o % 3 - 1;
                bool acc = false;
                float4 ent = make_float4(0.f, 0.f, 0.f, 0.f);
                int ec = 0;
                if (q < ctotal) {
                    const int l = ru.y + q;
                    const float4 lc = a.leaf_c4[l], lh = a.leaf_h4[l];
                    const float px = fmaxf(fabsf((lc.x + odx * hc) - gc.x) - (gh.x + lh.x), 0.f);
                    const float py = fmaxf(fabsf((lc.y + ody * hc) - gc.y) - (gh.y + lh.y), 0.f);
                    const float pz = fmaxf(fabsf((lc.z + odz * hc) - gc.z) - (gh.z + lh.z), 0.f);
                    acc = px * px + py * py + pz * pz < rf2;
                    if (acc) {
                        const int ax = gx + odx, ay = gy + ody, az = gz + odz;
                        const int sx = ax < 0 ? -1 : (ax >= ns ? 1 : 0);
                        const int sy = ay < 0 ? -1 : (ay >= ns ? 1 : 0);
                        const int sz = az < 0 ? -1 : (az >= ns ? 1 : 0);
                        if ((sx | sy | sz) == 0) {
                            const float4 lr4 = a.leaf_r4[l];
                            ent.x = __fsub_rn(lr4.x, gr4.x);
                            ent.y = __fsub_rn(lr4.y, gr4.y);
                            ent.z = __fsub_rn(lr4.z, gr4.z);
                        } else {
                            const double *lr = a.leaf_ref + 3 * (int64_t)l;
                            const double *gr = a.group_ref + 3 * (int64_t)g;
                            const double L = bx.L;
                            ent.x = __double2float_rn((lr[0] + sx * L) - gr[0]);
                            ent.y = __double2float_rn((lr[1] + sy * L) - gr[1]);
                            ent.z = __double2float_rn((lr[2] + sz * L) - gr[2]);
                        }
                        ent.w = lc.w;
                        ec = __float_as_int(lh.w);
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, acc);
                if (acc) {
                    const int slot = qn + __popc(bal & lt);
                    sQEnt[w][slot] = ent;
                    sQCnt[w][slot] = ec;
                }
                qn += __popc(bal);
                __syncwarp();
                if (qn >= 32) {
                    EntryBatch bt;
                    bt.set(sQEnt[w][lane], sQCnt[w][lane], lane);
                    __syncwarp();
                    if (lane < qn - 32) {
                        sQEnt[w][lane] = sQEnt[w][32 + lane];
                        sQCnt[w][lane] = sQCnt[w][32 + lane];
                    }
                    __syncwarp();
                    qn -= 32;
                    stage_batch(bt);
                }
            }
            if (qn > 0) {
                EntryBatch bt;
                bt.set(lane < qn ? sQEnt[w][lane] : make_float4(0.f, 0.f, 0.f, 0.f), lane < qn ? sQCnt[w][lane] : 0,
                       lane);
                stage_batch(bt);
            }
            __syncwarp();   // sRun and the queue are rewritten for the next group
        }
        const int padded = pad_sources<kSplit>(Af, Bf, nbuf, lane);
        __syncwarp();
        sum_buffer<NPOLY, kSplit>(A, Bq, padded >> 1, hs, xi, yi, zi, c, k);
        inter += (unsigned long long)nbuf * ni;
        staged += nbuf;
        __syncwarp();
        // the kSplit source slots of a target add up their compensated totals
        float tx = k.sx - k.cx, ty = k.sy - k.cy, tz = k.sz - k.cz;
#pragma unroll
        for (int o = G; o < 32; o <<= 1) {
            tx += __shfl_xor_sync(0xffffffffu, tx, o);
            ty += __shfl_xor_sync(0xffffffffu, ty, o);
            tz += __shfl_xor_sync(0xffffffffu, tz, o);
        }
        if (hs == 0 && ti < ni) {
            const int64_t o = a.perm[i0 + ti];
            const float Gc = bx.c_g;
            a.acc[3 * o + 0] = Gc * tx;
            a.acc[3 * o + 1] = Gc * ty;
            a.acc[3 * o + 2] = Gc * tz;
        }
    }
    if (lane == 0 && inter) {
        atomicAdd(a.n_inter, inter);
        atomicAdd(a.n_staged, staged);
    }
}

// Number of (i, j) pairs, j != i, with r^2 < rcut^2 in the lists (the self
// pair is recognised by its index: sources and targets share the sorted
// order): the work the cutoff keeps, counted with the PP kernel's own FP32
// decision.  Groups without a list (active-particle mode) count nothing.
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
            const int j0 = __float_as_int(ent.w);
            const int j1 = j0 + (int)a.ecount[e] + 1;
            for (int jb = j0; jb < j1; jb += 32) {
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
                    if (lane < ni && r2 < rcut2 && jb + jj != i0 + lane) cnt_within++;   // not the self pair
                }
            }
        }
    }
    if (cnt_within) atomicAdd(a.n_inter, cnt_within);
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
    a.n_pos = (int64_t)(lv->pos_leaf.bytes / sizeof(float4));
    a.leaf_first = static_cast<const int32_t *>(lv->leaf_first.p);
    a.perm = static_cast<const int32_t *>(lv->keys_in_alt ? lv->vals_alt.p : lv->vals.p);
    a.group_off = pr ? static_cast<const int64_t *>(pr->group_off.p) : nullptr;
    a.entries = pr ? static_cast<const float4 *>(pr->entries.p) : nullptr;
    a.ecount = pr ? static_cast<const uint8_t *>(pr->ecount.p) : nullptr;
    a.cap = pr ? pr->capacity : 0;
    a.order = pr && pr->ordered ? static_cast<const int32_t *>(pr->group_order.p) : nullptr;
    a.group_cell = static_cast<const int32_t *>(lv->group_cell.p);
    a.group_c4 = static_cast<const float4 *>(lv->group_c4.p);
    a.group_r4 = static_cast<const float4 *>(lv->group_r4.p);
    a.leaf_r4 = static_cast<const float4 *>(lv->leaf_r4.p);
    a.group_ref = static_cast<const double *>(lv->group_ref.p);
    a.leaf_ref = static_cast<const double *>(lv->leaf_ref.p);
    a.leaf_c4 = static_cast<const float4 *>(lv->leaf_c4.p);
    a.leaf_h4 = static_cast<const float4 *>(lv->leaf_h4.p);
    a.cell_leaf_first = static_cast<const int32_t *>(lv->cell_leaf_first.p);
    char *work = static_cast<char *>(pr ? pr->work.p : lv->work.p);
    a.queue = reinterpret_cast<int32_t *>(work);
    a.n_inter = reinterpret_cast<unsigned long long *>(work + 8);
    a.n_staged = reinterpret_cast<unsigned long long *>(work + 16);
    a.acc = d_acc;
}

template <bool kLearned, int kMinBlocks, int kSplit, bool kUniform>
static void launch_pp(int npoly, int grid, cudaStream_t s, const PPArgs &a)
{
    switch (npoly) {
    case 10: k_pp<10, kLearned, kMinBlocks, kSplit, kUniform><<<grid, kPPThreads, 0, s>>>(a); break;
    case 12: k_pp<12, kLearned, kMinBlocks, kSplit, kUniform><<<grid, kPPThreads, 0, s>>>(a); break;
    case 14: k_pp<14, kLearned, kMinBlocks, kSplit, kUniform><<<grid, kPPThreads, 0, s>>>(a); break;
    default: k_pp<16, kLearned, kMinBlocks, kSplit, kUniform><<<grid, kPPThreads, 0, s>>>(a); break;
    }
}

template <int kMinBlocks, int kSplit, bool kUniform>
static void launch_walk_one(int npoly, int grid, cudaStream_t s, const PPArgs &a)
{
    switch (npoly) {
    case 10: k_pp_walk<10, kMinBlocks, kSplit, kUniform><<<grid, kPPThreads, 0, s>>>(a); break;
    case 12: k_pp_walk<12, kMinBlocks, kSplit, kUniform><<<grid, kPPThreads, 0, s>>>(a); break;
    case 14: k_pp_walk<14, kMinBlocks, kSplit, kUniform><<<grid, kPPThreads, 0, s>>>(a); break;
    default: k_pp_walk<16, kMinBlocks, kSplit, kUniform><<<grid, kPPThreads, 0, s>>>(a); break;
    }
}

// The direct-mode kernel for every group size and kernel shape.
static void launch_walk(const ph_leaves *lv, int npoly, bool uni, cudaStream_t s, const PPArgs &a)
{
    const bool three = lv->pp_variant == 1 && uni;
    const int grid = sm_count() * (three ? kBlocks1 : kBlocks0);
    const int gs = lv->group_size;
    if (three) {
        if (gs == 8) launch_walk_one<kBlocks1, 4, true>(npoly, grid, s, a);
        else if (gs == 16) launch_walk_one<kBlocks1, 2, true>(npoly, grid, s, a);
        else launch_walk_one<kBlocks1, 1, true>(npoly, grid, s, a);
    } else if (uni) {
        if (gs == 8) launch_walk_one<kBlocks0, 4, true>(npoly, grid, s, a);
        else if (gs == 16) launch_walk_one<kBlocks0, 2, true>(npoly, grid, s, a);
        else launch_walk_one<kBlocks0, 1, true>(npoly, grid, s, a);
    } else {
        if (gs == 8) launch_walk_one<kBlocks0, 4, false>(npoly, grid, s, a);
        else if (gs == 16) launch_walk_one<kBlocks0, 2, false>(npoly, grid, s, a);
        else launch_walk_one<kBlocks0, 1, false>(npoly, grid, s, a);
    }
}

constexpr int kTabBytes = (kTabN + 1) * (int)sizeof(float2);

template <int kSplit>
static void launch_table_one(int grid, cudaStream_t s, const PPArgs &a)
{
    static bool ready = false;
    if (!ready) {
        cudaFuncSetAttribute(k_pp<10, false, kBlocks0, kSplit, true, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTabBytes);
        ready = true;
    }
    k_pp<10, false, kBlocks0, kSplit, true, true><<<grid, kPPThreads, kTabBytes, s>>>(a);
}

constexpr int kL1Bytes = 4 * kL1Nodes * (int)sizeof(float4);   // layer 1's table (dynamic shared memory)

// The learned kernels' opt-in above 48 KB of shared memory, once per
// process; called when a network handle is made, so that it never runs
// inside a stream capture.
int pp_learned_setup()
{
    static bool done = false;
    if (done) return PH_OK;
    int rc = cuda_check(cudaFuncSetAttribute(k_pp<10, true, kBlocks0, 4, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kL1Bytes), "smem opt-in");
    if (!rc) rc = cuda_check(cudaFuncSetAttribute(k_pp<10, true, kBlocks0, 2, false>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kL1Bytes), "smem opt-in");
    if (!rc) rc = cuda_check(cudaFuncSetAttribute(k_pp<10, true, kBlocks0, 1, false>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kL1Bytes), "smem opt-in");
    if (!rc) done = true;
    return rc;
}

int pp_learned_device(const ph_leaves *lv, const ph_pairs *pr, const float *mlp_w, float *d_acc, cudaStream_t s)
{
    PPArgs a;
    pp_args(lv, pr, d_acc, a);
    a.mlp_w = mlp_w;
    int rc = cuda_check(cudaMemsetAsync(pr->work.p, 0, 24, s), "reset work queue");
    if (rc) return rc;
    const int grid = sm_count() * kBlocks0;
    rc = pp_learned_setup();
    if (rc) return rc;
    if (lv->group_size == 8) k_pp<10, true, kBlocks0, 4, false><<<grid, kPPThreads, kL1Bytes, s>>>(a);
    else if (lv->group_size == 16) k_pp<10, true, kBlocks0, 2, false><<<grid, kPPThreads, kL1Bytes, s>>>(a);
    else k_pp<10, true, kBlocks0, 1, false><<<grid, kPPThreads, kL1Bytes, s>>>(a);
    count_launch();
    return cuda_check(cudaGetLastError(), "learned pp kernel");
}

// true if every box has the same factor constants (then the kernel reads
// them from its parameter bank)
static bool uniform_consts(const ph_leaves *lv, PairConsts &uc)
{
    if ((int)lv->boxes_host.size() < lv->n_boxes || lv->n_boxes < 1) return false;   // no host copy of the boxes
    const BoxDev &b0 = lv->boxes_host[0];
    for (int b = 1; b < lv->n_boxes; b++) {
        const BoxDev &bx = lv->boxes_host[b];
        if (memcmp(bx.poly, b0.poly, sizeof b0.poly) || bx.s2 != b0.s2 || bx.eps2s != b0.eps2s || bx.c_t != b0.c_t ||
            bx.c_e != b0.c_e || bx.rcut2 != b0.rcut2 || bx.rfilt2 != b0.rfilt2)
            return false;
    }
    auto dup = [](float v) {
        uint64_t u;
        uint32_t bits;
        memcpy(&bits, &v, 4);
        u = ((uint64_t)bits << 32) | bits;
        return (f2_t)u;
    };
    for (int q = 0; q <= kMaxPoly; q++) uc.poly[q] = dup(b0.poly[q]);
    uc.s2 = dup(b0.s2);
    uc.eps2s = dup(b0.eps2s);
    uc.c_t = dup(b0.c_t);
    uc.c_e = dup(b0.c_e);
    uc.m1 = dup(-1.f);
    uc.rcut2 = b0.rcut2;
    uc.rfilt2 = b0.rfilt2;
    return true;
}

// PP with the tabulated factor (every box shares one rcut and rs; the table
// is lv->table, filled by the caller for them).
int pp_table_device(const ph_leaves *lv, const ph_pairs *pr, float *d_acc, cudaStream_t s)
{
    PPArgs a;
    pp_args(lv, pr, d_acc, a);
    a.mlp_w = nullptr;
    if (!uniform_consts(lv, a.uc)) return fail(PH_ERR_ARG, "the tabulated factor needs one rcut and rs for all boxes");
    a.table = static_cast<const float2 *>(lv->table.p);
    a.tab_scale2 = (float)((kTabN / lv->table_rcut) * (kTabN / lv->table_rcut));
    int rc2 = cuda_check(cudaMemsetAsync(pr->work.p, 0, 24, s), "reset work queue");
    if (rc2) return rc2;
    const int grid = sm_count() * kBlocks0;
    if (lv->group_size == 8) launch_table_one<4>(grid, s, a);
    else if (lv->group_size == 16) launch_table_one<2>(grid, s, a);
    else launch_table_one<1>(grid, s, a);
    count_launch();
    return cuda_check(cudaGetLastError(), "table pp kernel");
}

int pp_exact_device(const ph_leaves *lv, const ph_pairs *pr, float *d_acc, cudaStream_t s)
{
    PPArgs a;
    pp_args(lv, pr, d_acc, a);
    a.mlp_w = nullptr;
    int rc = cuda_check(cudaMemsetAsync(pr ? pr->work.p : lv->work.p, 0, 24, s), "reset work queue");
    if (rc) return rc;
    const int npoly = lv->poly_degree;
    if (npoly != 10 && npoly != 12 && npoly != 14 && npoly != 16)
        return fail(PH_ERR_STATE, "unsupported polynomial degree %d", npoly);
    const bool uni = uniform_consts(lv, a.uc);
    if (!pr) {
        launch_walk(lv, npoly, uni, s, a);
        count_launch();
        return cuda_check(cudaGetLastError(), "pp kernel");
    }
    const bool three = lv->pp_variant == 1;
    const int grid = sm_count() * (three ? kBlocks1 : kBlocks0);
    const int gs = lv->group_size;
    if (uni) {
        if (three) {
            if (gs == 8) launch_pp<false, kBlocks1, 4, true>(npoly, grid, s, a);
            else if (gs == 16) launch_pp<false, kBlocks1, 2, true>(npoly, grid, s, a);
            else launch_pp<false, kBlocks1, 1, true>(npoly, grid, s, a);
        } else {
            if (gs == 8) launch_pp<false, kBlocks0, 4, true>(npoly, grid, s, a);
            else if (gs == 16) launch_pp<false, kBlocks0, 2, true>(npoly, grid, s, a);
            else launch_pp<false, kBlocks0, 1, true>(npoly, grid, s, a);
        }
    } else {
        // boxes with different constants: the two-block shape only
        const int g2 = sm_count() * kBlocks0;
        if (gs == 8) launch_pp<false, kBlocks0, 4, false>(npoly, g2, s, a);
        else if (gs == 16) launch_pp<false, kBlocks0, 2, false>(npoly, g2, s, a);
        else launch_pp<false, kBlocks0, 1, false>(npoly, g2, s, a);
    }
    count_launch();
    return cuda_check(cudaGetLastError(), "pp kernel");
}

}  // namespace phpp
