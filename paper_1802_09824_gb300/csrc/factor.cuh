// Device evaluation of the short-range factor: the exact form of Eq. (split)
// (SFU + polynomial) and the learned 1-16-16-1 SiLU network (tensor cores).
#pragma once

#include <cuda_bf16.h>

#include "checks.cuh"
#include "phpp_internal.cuh"

namespace phpp {

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

__device__ __forceinline__ float rcp_sfu(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---- packed FP32 pairs (f32x2, sm_100+): two values per instruction

typedef unsigned long long f2_t;   // two FP32 values in one 64-bit register pair

__device__ __forceinline__ f2_t pk(float lo, float hi)
{
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float lo_of(f2_t v)
{
    float lo;
    [[maybe_unused]] float hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return lo;
}
__device__ __forceinline__ float hi_of(f2_t v)
{
    [[maybe_unused]] float lo;
    float hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return hi;
}
__device__ __forceinline__ f2_t add2(f2_t a, f2_t b)
{
    f2_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t sub2(f2_t a, f2_t b)
{
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t mul2(f2_t a, f2_t b)
{
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t fma2(f2_t a, f2_t b, f2_t c)
{
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Exact factor f(r) = 2^(r^2 c_e) h(t), t = 2r/rcut - 1 (scalar form of the
// PP kernel's evaluation).
__device__ __forceinline__ float exact_factor(float r2, float t, const float *poly, int npoly, float c_e)
{
    float h = poly[npoly];
    for (int q = npoly - 1; q >= 0; q--) h = fmaf(h, t, poly[q]);
    return ex2_sfu(r2 * c_e) * h;
}

// Network parameters in the flat order W1[16], b1[16], W2[16][16] (row k =
// weights into unit k), b2[16], W3[16], b3.
constexpr int kMlpParams = 321;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// x = hi + lo with hi = bf16(x), lo = bf16(x - hi): ~16 significant bits.
__device__ __forceinline__ void split_bf16(float x, float &hi, float &lo)
{
    hi = __bfloat162float(__float2bfloat16_rn(x));
    lo = x - hi;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The SiLU of the network in scaled units.  With z = -log2(e) a the SiLU is
// silu(a) = -ln2 * z / (1 + 2^z): the factor -log2(e) is folded into the
// weights and biases that produce z and -ln2 into the weights that consume
// the activation (see mlp_lane_load), so a unit costs an SFU ex2, an add, an
// SFU reciprocal and a multiply.  (A Newton reciprocal on the FMA pipe for
// part of the units, to unload the SFU, measured slower, and so did one
// reciprocal for several units by batch inversion.)
__device__ __forceinline__ float silu_scaled(float z)
{
    return z * rcp_sfu(1.f + ex2_sfu(z));
}

// Two units at once: the add and the multiply as packed FP32.
__device__ __forceinline__ f2_t silu_scaled2(f2_t z)
{
    const f2_t den = add2(pk(ex2_sfu(lo_of(z)), ex2_sfu(hi_of(z))), pk(1.f, 1.f));
    return mul2(z, pk(rcp_sfu(lo_of(den)), rcp_sfu(hi_of(den))));
}

// The same split for a packed pair, as two BF16x2 registers (first value in
// the low half): hi = bf16(x), lo = bf16(x - hi), both rounded to nearest.
__device__ __forceinline__ void split_pack2(f2_t x, uint32_t &hi, uint32_t &lo)
{
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(hi_of(x)), "f"(lo_of(x)));
    const f2_t hf = pk(__uint_as_float(hi << 16), __uint_as_float(hi & 0xFFFF0000u));
    const f2_t l = sub2(x, hf);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(hi_of(l)), "f"(lo_of(l)));
}

// Layer 1 as a table.  Its input is the one scalar t = 2r/rcut - 1 in
// [-1, 1], so each of its 16 activations h(t) = silu(w1 t + b1) is a smooth
// function of t alone: the kernels tabulate them (in FP32, through
// silu_scaled) at kL1Nodes equally spaced nodes t_i = i D - 1,
// D = 2/(kL1Nodes - 1), and interpolate linearly.  The interpolation error of
// a unit is at most (D^2/8) max|h''| = (D^2/8) w1^2 / 2 (|silu''| <= 1/2 at
// 0), 1.4e-5 for |w1| = 3.8 (the trained 128^3 network), which moves g_hat by
// ~1e-6, below what the BF16 hi/lo split of layer 2's operands does (~7e-6);
// each network's validation measures g_hat through this table.  Node i holds,
// for each lane quad q, the units {2q, 2q+1, 2q+8, 2q+9} of the A fragment
// (one float4): the table has kL1Nodes x 4 float4 (32 KB).
constexpr int kL1Nodes = 512;

// Fill the table (all threads of the block; the caller synchronises).
// w: network parameters in the flat order of kMlpParams.
__device__ __forceinline__ void l1_table_fill(const float *w, float4 *tab)
{
    const float kz = -1.4426950408889634f;   // -log2(e)
    const float D = 2.f / (float)(kL1Nodes - 1);
    for (int e = threadIdx.x; e < 4 * kL1Nodes; e += blockDim.x) {
        const int i = e >> 2, q = e & 3;
        const float t = fmaf((float)i, D, -1.f);
        float v[4];
        const int cols[4] = {2 * q, 2 * q + 1, 2 * q + 8, 2 * q + 9};
#pragma unroll
        for (int c = 0; c < 4; c++) v[c] = silu_scaled(fmaf(kz * w[cols[c]], t, kz * w[16 + cols[c]]));
        tab[e] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// Per-lane share of the network for warp-level evaluation with
// mma.sync.m16n8k16 (BF16 in, FP32 accumulate).  Lane = 4 g + q: the lane
// owns rows g and g+8 of each 16-pair tile and hidden columns
// {2q, 2q+1, 2q+8, 2q+9}; the 16x16 second layer is two n8 halves.
// Weights are stored in the scaled units of silu_scaled: W1, b1 and b2
// times -log2(e), W3 times -ln2 (W2 and b3 unchanged); layer 1 is the table.
struct MlpLane {
    uint32_t bhi[2][2], blo[2][2];   // W2^T fragments (hi / lo parts), per n-half
    float b2[2][2];              // bias of output columns 8h + 2q, 8h + 2q + 1
    f2_t w3[2];                  // W3 of the same two columns, per n-half
    float b3;
};

__device__ __forceinline__ void mlp_lane_load(const float *w, MlpLane &L)
{
    const float kz = -1.4426950408889634f;   // -log2(e)
    const float ka = -0.6931471805599453f;   // -ln(2)
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int cols[4] = {2 * q, 2 * q + 1, 2 * q + 8, 2 * q + 9};
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int n = g + 8 * h;             // output unit of this B column
        const float *row = w + 32 + 16 * n;  // W2[n][kk]
        float hi[4], lo[4];
#pragma unroll
        for (int c = 0; c < 4; c++) split_bf16(row[cols[c]], hi[c], lo[c]);
        L.bhi[h][0] = pack_bf16(hi[0], hi[1]);
        L.bhi[h][1] = pack_bf16(hi[2], hi[3]);
        L.blo[h][0] = pack_bf16(lo[0], lo[1]);
        L.blo[h][1] = pack_bf16(lo[2], lo[3]);
        L.b2[h][0] = kz * w[288 + 8 * h + 2 * q];
        L.b2[h][1] = kz * w[288 + 8 * h + 2 * q + 1];
        L.w3[h] = pk(ka * w[304 + 8 * h + 2 * q], ka * w[304 + 8 * h + 2 * q + 1]);
    }
    L.b3 = w[320];
}

// The network's factor for the warp's 32 pairs: lane i passes the input
// z0 = 2r/rcut - 1 of its pair and receives g_hat of its pair.  Layer 1 from
// the table (linear interpolation, two units per packed instruction), layer
// 2 as BF16 tensor-core MMAs with FP32 accumulation, activations and weights
// split into BF16 hi + lo parts (hi*hi + lo*hi + hi*lo), which keeps ~16
// bits, then its SiLUs and layer 3 in FP32 (the lane's two columns 2q, 2q + 1
// of a row share layer 3's accumulator pair).
__device__ __forceinline__ float mlp_warp_eval(float z0, const MlpLane &L, const float4 *tab)
{
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, q = lane & 3;
    const float kInv = 0.5f * (float)(kL1Nodes - 1);   // 1 / D
    const float kMagic = 12582912.f;                   // 1.5 * 2^23: adding it rounds to an integer
    float out = 0.f;
#pragma unroll
    for (int tile = 0; tile < 2; tile++) {
        const float za = __shfl_sync(0xffffffffu, z0, 16 * tile + g);
        const float zb = __shfl_sync(0xffffffffu, z0, 16 * tile + g + 8);
        // node index i = floor(u) (clamped into the table) and fraction u - i of rows g, g + 8
        const f2_t u0 = fma2(pk(za, zb), pk(kInv, kInv), pk(kInv, kInv));
        const f2_t u = pk(fminf(fmaxf(lo_of(u0), 0.f), (float)(kL1Nodes - 1)),
                          fminf(fmaxf(hi_of(u0), 0.f), (float)(kL1Nodes - 1)));
        const f2_t y = add2(add2(u, pk(-0.5f, -0.5f)), pk(kMagic, kMagic));
        const f2_t fr = sub2(u, sub2(y, pk(kMagic, kMagic)));
        int ia = __float_as_int(lo_of(y)) - __float_as_int(kMagic);
        int ib = __float_as_int(hi_of(y)) - __float_as_int(kMagic);
        if (!in_bounds(ia, kL1Nodes - 1, BS_L1_TABLE)) ia = 0;
        if (!in_bounds(ib, kL1Nodes - 1, BS_L1_TABLE)) ib = 0;
        const float4 a0 = tab[4 * ia + q], a1 = tab[4 * ia + 4 + q];
        const float4 b0 = tab[4 * ib + q], b1 = tab[4 * ib + 4 + q];
        const f2_t fa = pk(lo_of(fr), lo_of(fr)), fb = pk(hi_of(fr), hi_of(fr));
        const f2_t va0 = pk(a0.x, a0.y), va1 = pk(a0.z, a0.w), vb0 = pk(b0.x, b0.y), vb1 = pk(b0.z, b0.w);
        uint32_t Ahi[4], Alo[4];
        split_pack2(fma2(fa, sub2(pk(a1.x, a1.y), va0), va0), Ahi[0], Alo[0]);   // row g, cols 2q, 2q+1
        split_pack2(fma2(fb, sub2(pk(b1.x, b1.y), vb0), vb0), Ahi[1], Alo[1]);   // row g+8
        split_pack2(fma2(fa, sub2(pk(a1.z, a1.w), va1), va1), Ahi[2], Alo[2]);   // row g, cols 2q+8, 2q+9
        split_pack2(fma2(fb, sub2(pk(b1.z, b1.w), vb1), vb1), Ahi[3], Alo[3]);   // row g+8
        f2_t s[4];   // per n-half hh: s[2 hh] row g, s[2 hh + 1] row g + 8 (columns 8hh + 2q, + 1)
#pragma unroll
        for (int hh = 0; hh < 2; hh++) {
            float d[4] = {L.b2[hh][0], L.b2[hh][1], L.b2[hh][0], L.b2[hh][1]};
            mma_bf16(d, Alo, L.bhi[hh][0], L.bhi[hh][1]);
            mma_bf16(d, Ahi, L.blo[hh][0], L.blo[hh][1]);
            mma_bf16(d, Ahi, L.bhi[hh][0], L.bhi[hh][1]);
            s[2 * hh] = silu_scaled2(pk(d[0], d[1]));
            s[2 * hh + 1] = silu_scaled2(pk(d[2], d[3]));
        }
        // rows g and g + 8: (even column, odd column) partial sums
        const f2_t ya = fma2(L.w3[1], s[2], mul2(L.w3[0], s[0]));
        const f2_t yb = fma2(L.w3[1], s[3], mul2(L.w3[0], s[1]));
        float sa = lo_of(ya) + hi_of(ya), sb = lo_of(yb) + hi_of(yb);
        sa += __shfl_xor_sync(0xffffffffu, sa, 1);
        sa += __shfl_xor_sync(0xffffffffu, sa, 2);
        sb += __shfl_xor_sync(0xffffffffu, sb, 1);
        sb += __shfl_xor_sync(0xffffffffu, sb, 2);
        // pair p = 16 tile + rho is lane p; rows rho < 8 are held as sa, others
        // as sb, by the quad 4 (rho % 8) .. 4 (rho % 8) + 3
        const int rho = lane & 15;
        const float va = __shfl_sync(0xffffffffu, sa, 4 * (rho & 7));
        const float vb = __shfl_sync(0xffffffffu, sb, 4 * (rho & 7));
        if ((lane >> 4) == tile) out = (rho < 8 ? va : vb) + L.b3;
    }
    return out;
}

}  // namespace phpp
