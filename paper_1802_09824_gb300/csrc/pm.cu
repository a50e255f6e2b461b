// Long-range side of the force split: the particle-mesh (PM) part of
// Sec. 3.1 on one periodic box.
//
//   1. CIC assignment of the masses to an N^3 mesh (k_pm_deposit): the cell
//      and fraction in FP64, the CIC weights in FP32, summed as 64-bit
//      fixed-point atomics, so the node masses do not depend on the order of
//      the additions (replays are bit-identical).
//   2. FFT of the node masses (cuFFT, real to complex, FP32).
//   3. Green's function of the 3-point difference Laplacian (the equation of
//      Sec. 3.1), phi_k = -pi G Delta_g^2 rho_k / (sin^2(pi l/N) +
//      sin^2(pi m/N) + sin^2(pi n/N)), times the long-range filter
//      exp(-k^2 R_s^2) (the k-space complement of Eq. (split)); k = 0
//      dropped (k_pm_green).
//   4. Inverse FFT: the potential on the mesh.
//   5. Mesh acceleration by the 2-point central difference (k_pm_grad), CIC
//      interpolation back to the particles with the assignment weights
//      (k_pm_interp), written or added to the caller's acceleration array.
//
// The cell of a particle is decided in FP64 with fixed roundings: a
// coordinate in [0, L) is kept, any other becomes x_w = x - L floor(x / L)
// (x_w = L maps to 0); u = x_w (N / L), i0 = floor(u) mod N, fraction
// u - floor(u).
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "checks.cuh"
#include "phpp_internal.cuh"

struct ph_pm {
    uint32_t kind = phpp::KIND_PM;
    cudaStream_t last_stream = nullptr;
    int32_t n_mesh = 0;
    int64_t last_n = 0;
    bool plans = false;
    cufftHandle plan_r2c = 0, plan_c2r = 0;
    phpp::DevBuf mesh_q;     // unsigned long long [N^3]: node masses, fixed point
    phpp::DevBuf mesh_r;     // float [N^3]: node masses, then the potential
    phpp::DevBuf mesh_c;     // cufftComplex [N N (N/2+1)]
    phpp::DevBuf mesh_a;     // float4 [N^3]: -grad phi (x, y, z) and phi
    phpp::DevBuf tab;        // float [2N]: sin^2(pi l / N), exp(-k_l^2 R_s^2)
    phpp::DevBuf fft_work;   // cuFFT work area (both plans)
    phpp::DevBuf scale;      // uint32 largest |m| (float bits)
    phpp::DevBuf status;     // uint32 device status word
    phpp::DevBuf in_pos, in_mass, acc_tmp, pot_tmp;
    double tab_L = 0.0, tab_rs = -1.0;
    // active-particle mode (adaptive time steps): when set (caller-order
    // flags, device), only flagged particles are interpolated; the others
    // keep their acceleration (every particle is still deposited)
    const uint8_t *active = nullptr;
};

namespace phpp {

namespace {

constexpr int kPmThreads = 256;

inline int grid_of(int64_t n, int per_block = kPmThreads)
{
    int64_t b = (n + per_block - 1) / per_block;
    const int64_t cap = (int64_t)sm_count() * 16;
    if (b > cap) b = cap;
    return (int)(b > 0 ? b : 1);
}

// Node and fraction of one coordinate (FP64, fixed roundings).  The FP64
// division of the wrap (a long instruction sequence on this GPU's narrow
// FP64 pipe) is only taken for coordinates outside [0, L).
__device__ __forceinline__ int pm_cell(double x, double L, double inv_dg, int N, double &f)
{
    double xw = x;
    if (!(x >= 0.0 && x < L)) {
        const double q = floor(__ddiv_rn(x, L));
        xw = __dsub_rn(x, __dmul_rn(L, q));
        if (xw >= L) xw = 0.0;
    }
    const double u = __dmul_rn(xw, inv_dg);
    const double fl = floor(u);
    f = __dsub_rn(u, fl);
    // fl is in [-1, N]: -1 when x sits just below a multiple of L and x / L
    // rounded up (then x_w is a tiny negative number), N when u rounded up
    int i = (int)fl;
    if (i >= N) i -= N;
    if (i < 0) i += N;
    return i;
}

// The same for an FP32 coordinate without FP64: u = x N/L as a double-float
// product -- x times the double-float (c_hi, c_lo) of N/L, the product's
// rounding error taken exactly by an FMA -- the node from the high part and
// the fraction from the exact difference of the high part and its floor
// plus the low part (error ~2^-48 u in u, one FP32 rounding in f).  For x in
// [0, L); the caller sends other coordinates through pm_cell.
struct CellScale {
    float c_hi, c_lo, L_up;   // N/L as c_hi + c_lo; L_up: an FP32 x is below L iff x < L_up
};

__device__ __forceinline__ int pm_cell32(float x, const CellScale &cs, int N, float &f)
{
    const float p = x * cs.c_hi;
    const float e = fmaf(x, cs.c_hi, -p);   // x c_hi - p exactly
    const float lo = fmaf(x, cs.c_lo, e);   // the rest of x N/L
    float fl = floorf(p);
    float fr = (p - fl) + lo;                // p - fl is exact
    if (fr < 0.f) {
        fr += 1.f;
        fl -= 1.f;
    } else if (fr >= 1.f) {
        fr -= 1.f;
        fl += 1.f;
    }
    int i = (int)fl;
    if (i >= N) i -= N;
    if (i < 0) i += N;
    f = fr;
    return i;
}

// Node and FP32 fraction of coordinate x: the FP32 path for an FP32 x in
// [0, L), the FP64 one otherwise.
template <int PT>
__device__ __forceinline__ int pm_cell_any(const void *pos, int64_t k, double L, double inv_dg, const CellScale &cs,
                                           int N, float &f)
{
    if (PT == PH_F32) {
        const float x = static_cast<const float *>(pos)[k];
        if (x >= 0.f && x < cs.L_up) return pm_cell32(x, cs, N, f);
    }
    double fd;
    const int i = pm_cell(PT == PH_F32 ? (double)static_cast<const float *>(pos)[k] : static_cast<const double *>(pos)[k],
                          L, inv_dg, N, fd);
    f = (float)fd;
    return i;
}

// Round a finite FP32 value to the nearest 64-bit integer (ties to even) with
// integer operations (|v| < 2^63), from the binary32 format: the significand
// shifted by the exponent.
__device__ __forceinline__ long long f2ll_rn(float v)
{
    const unsigned int b = __float_as_uint(v) & 0x7FFFFFFFu;
    const int e = (int)(b >> 23) - 127;   // v = 1.m 2^e
    unsigned long long q = 0;
    if (e >= 23) {
        q = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u) << (e - 23);
    } else if (e >= -1) {
        const unsigned int m = (b & 0x7FFFFFu) | 0x800000u;
        const int sh = 23 - e;            // 1 .. 24
        const unsigned int qq = m >> sh, rem = m & ((1u << sh) - 1u), half = 1u << (sh - 1);
        q = qq + ((rem > half || (rem == half && (qq & 1u))) ? 1u : 0u);
    }
    return (__float_as_uint(v) >> 31) ? -(long long)q : (long long)q;
}

// A 64-bit integer (|q| < 2^63) to the nearest FP32 value (ties to even)
// with integer operations.
__device__ __forceinline__ float ll2f_rn(long long q)
{
    if (q == 0) return 0.f;
    const unsigned int sign = q < 0 ? 0x80000000u : 0u;
    unsigned long long a = q < 0 ? (unsigned long long)(-q) : (unsigned long long)q;
    int e = 63 - __clzll((long long)a);   // a in [2^e, 2^(e+1))
    unsigned long long m;
    if (e <= 23) {
        m = a << (23 - e);
    } else {
        const int sh = e - 23;
        m = a >> sh;
        const unsigned long long rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (m & 1ull))) m++;
        if (m == (1ull << 24)) {
            m >>= 1;
            e++;
        }
    }
    return __uint_as_float(sign | ((unsigned int)(e + 127) << 23) | ((unsigned int)m & 0x7FFFFFu));
}

// Fixed-point scale 2^(62 - e) with n max|m| < 2^e: no node (nor the total)
// can exceed 2^62 in magnitude.
__device__ __forceinline__ double pm_scale(const uint32_t *mmax_bits, int64_t n)
{
    const double b = (double)__uint_as_float(*mmax_bits) * (double)n;
    if (!(b > 0.0)) return 1.0;
    return ldexp(1.0, 62 - (ilogb(b) + 1));
}

// The exponent k of the scale 2^k, computed once per block (its FP64 steps
// are slow on this GPU) and shared; values are scaled with ldexpf (exact).
__device__ __forceinline__ int pm_scale_exp_block(const uint32_t *mmax_bits, int64_t n)
{
    __shared__ int s_k;
    if (threadIdx.x == 0) s_k = ilogb(pm_scale(mmax_bits, n));
    __syncthreads();
    return s_k;
}

__global__ void k_pm_mass_max(const float *mass, int64_t n, float mass_default, uint32_t *mmax_bits,
                              uint32_t *status)
{
    uint32_t best = 0;
    if (!mass) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(mmax_bits, __float_as_uint(fabsf(mass_default)));
        return;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float m = mass[i];
        if (!isfinite(m)) {
            atomicOr(status, ST_NONFINITE);
            continue;
        }
        best = max(best, __float_as_uint(fabsf(m)));
    }
    for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    // one atomic per block (the warps' maxima through shared memory)
    __shared__ uint32_t s_best[kPmThreads / 32];
    if ((threadIdx.x & 31) == 0) s_best[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
        best = threadIdx.x < (blockDim.x >> 5) ? s_best[threadIdx.x] : 0u;
        for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (threadIdx.x == 0 && best) atomicMax(mmax_bits, best);
    }
}

template <int PT>
__global__ void k_pm_deposit(const void *pos, const float *mass, int64_t n, float mass_default, double L,
                             double inv_dg, CellScale cs, int N, const uint32_t *mmax_bits,
                             unsigned long long *mesh_q, uint32_t *status)
{
    const int kS = pm_scale_exp_block(mmax_bits, n);   // S = 2^kS: m S is exact in FP32
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float m = mass ? mass[i] : mass_default;
        bool finite = isfinite(m);
        if (PT == PH_F32) {
            const float *p = static_cast<const float *>(pos) + 3 * i;
            finite = finite && isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]);
        } else {
            const double *p = static_cast<const double *>(pos) + 3 * i;
            finite = finite && isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]);
        }
        if (!finite) {
            atomicOr(status, ST_NONFINITE);
            continue;
        }
        // the node and fraction of each axis; the weights, the shares and
        // their conversion to 64-bit fixed point in FP32 and integer
        // operations (this GPU's FP64 pipe is narrow): a node's share carries
        // ~3 FP32 roundings, the integer sums none
        float gx, gy, gz;
        const int ix = pm_cell_any<PT>(pos, 3 * i, L, inv_dg, cs, N, gx);
        const int iy = pm_cell_any<PT>(pos, 3 * i + 1, L, inv_dg, cs, N, gy);
        const int iz = pm_cell_any<PT>(pos, 3 * i + 2, L, inv_dg, cs, N, gz);
        const float wx[2] = {1.f - gx, gx}, wy[2] = {1.f - gy, gy};
        const float mS = ldexpf(m, kS);
        const float wzm[2] = {(1.f - gz) * mS, gz * mS};
        const int jx[2] = {ix, ix + 1 == N ? 0 : ix + 1};
        const int jy[2] = {iy, iy + 1 == N ? 0 : iy + 1};
        const int jz[2] = {iz, iz + 1 == N ? 0 : iz + 1};
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++) {
                const float wab = wx[a] * wy[b];
                const int64_t row = ((int64_t)jx[a] * N + jy[b]) * N;
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const long long q = f2ll_rn(wab * wzm[c]);
                    if (q && in_bounds(row + jz[c], (int64_t)N * N * N, BS_PM_NODE))
                        atomicAdd(mesh_q + row + jz[c], (unsigned long long)q);
                }
            }
    }
}

// Node masses back to FP32 (the FFT input).
__global__ void k_pm_unfix(const unsigned long long *mesh_q, int64_t cells, int64_t n, const uint32_t *mmax_bits,
                           float *mesh_r)
{
    const int kS = pm_scale_exp_block(mmax_bits, n);   // S = 2^kS
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cells; i += (int64_t)gridDim.x * blockDim.x)
        mesh_r[i] = ldexpf(ll2f_rn((long long)mesh_q[i]), -kS);
}

// Multiply the half spectrum by the filtered Green's function.  c0 folds
// -pi G Delta_g^2, the 1 / Delta_g^3 of the density and the 1 / N^3 of the
// unnormalised inverse transform.
__global__ void k_pm_green(float2 *mc, int N, const float *s2, const float *ek, float c0)
{
    const int nh = N / 2 + 1;
    const int64_t total = (int64_t)N * N * nh;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx % nh);
        const int64_t r = idx / nh;
        const int b = (int)(r % N);
        const int a = (int)(r / N);
        const float den = s2[a] + s2[b] + s2[c];
        const float g = idx == 0 ? 0.f : c0 * (ek[a] * ek[b] * ek[c]) / den;
        float2 v = mc[idx];
        v.x *= g;
        v.y *= g;
        mc[idx] = v;
    }
}

// -grad phi by the 2-point central difference; phi kept in w.
__global__ void k_pm_grad(const float *phi, int N, float c_half, float4 *mesh_a)
{
    const int64_t cells = (int64_t)N * N * N;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < cells;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const int64_t r = idx / N;
        const int j = (int)(r % N);
        const int i = (int)(r / N);
        const int ip = i + 1 == N ? 0 : i + 1, im = i == 0 ? N - 1 : i - 1;
        const int jp = j + 1 == N ? 0 : j + 1, jm = j == 0 ? N - 1 : j - 1;
        const int kp = k + 1 == N ? 0 : k + 1, km = k == 0 ? N - 1 : k - 1;
        const int64_t NN = (int64_t)N * N;
        float4 o;
        o.x = c_half * (phi[ip * NN + (int64_t)j * N + k] - phi[im * NN + (int64_t)j * N + k]);
        o.y = c_half * (phi[i * NN + (int64_t)jp * N + k] - phi[i * NN + (int64_t)jm * N + k]);
        o.z = c_half * (phi[r * N + kp] - phi[r * N + km]);
        o.w = phi[idx];
        mesh_a[idx] = o;
    }
}

template <int PT>
__global__ void k_pm_interp(const void *pos, int64_t n, double L, double inv_dg, CellScale cs, int N,
                            const float4 *mesh_a, float *acc, float *pot, int accumulate, const uint8_t *active)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (active && !active[i]) continue;
        bool finite;
        if (PT == PH_F32) {
            const float *p = static_cast<const float *>(pos) + 3 * i;
            finite = isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]);
        } else {
            const double *p = static_cast<const double *>(pos) + 3 * i;
            finite = isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]);
        }
        if (!finite) continue;   // latched by the deposit
        float gx, gy, gz;
        const int ix = pm_cell_any<PT>(pos, 3 * i, L, inv_dg, cs, N, gx);
        const int iy = pm_cell_any<PT>(pos, 3 * i + 1, L, inv_dg, cs, N, gy);
        const int iz = pm_cell_any<PT>(pos, 3 * i + 2, L, inv_dg, cs, N, gz);
        const float wx[2] = {1.f - gx, gx}, wy[2] = {1.f - gy, gy}, wz[2] = {1.f - gz, gz};
        const int jx[2] = {ix, ix + 1 == N ? 0 : ix + 1};
        const int jy[2] = {iy, iy + 1 == N ? 0 : iy + 1};
        const int jz[2] = {iz, iz + 1 == N ? 0 : iz + 1};
        float ax = 0.f, ay = 0.f, az = 0.f, ph = 0.f;
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++) {
                const float wab = wx[a] * wy[b];
                const int64_t row = ((int64_t)jx[a] * N + jy[b]) * N;
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const float w = wab * wz[c];
                    const float4 v = __ldg(mesh_a + row + jz[c]);
                    ax = fmaf(w, v.x, ax);
                    ay = fmaf(w, v.y, ay);
                    az = fmaf(w, v.z, az);
                    ph = fmaf(w, v.w, ph);
                }
            }
        if (accumulate) {
            acc[3 * i] += ax;
            acc[3 * i + 1] += ay;
            acc[3 * i + 2] += az;
        } else {
            acc[3 * i] = ax;
            acc[3 * i + 1] = ay;
            acc[3 * i + 2] = az;
        }
        if (pot) pot[i] = ph;
    }
}

int cufft_check(cufftResult r, const char *what)
{
    if (r == CUFFT_SUCCESS) return PH_OK;
    if (r == CUFFT_ALLOC_FAILED) return fail(PH_ERR_OOM, "%s: cuFFT allocation failed", what);
    return fail(PH_ERR_CUDA, "%s: cuFFT error %d", what, (int)r);
}

void pm_release(ph_pm *h)
{
    if (h->plans) {
        cufftDestroy(h->plan_r2c);
        cufftDestroy(h->plan_c2r);
        h->plans = false;
    }
    DevBuf *bufs[] = {&h->mesh_q, &h->mesh_r, &h->mesh_c, &h->mesh_a, &h->tab, &h->fft_work, &h->scale,
                      &h->status, &h->in_pos, &h->in_mass, &h->acc_tmp, &h->pot_tmp};
    for (DevBuf *b : bufs) release(*b);
}

// Mesh buffers and FFT plans for an N^3 mesh (kept while N is unchanged).
int pm_setup(ph_pm *h, int N)
{
    if (h->plans && h->n_mesh == N) return PH_OK;
    if (h->plans) {
        cufftDestroy(h->plan_r2c);
        cufftDestroy(h->plan_c2r);
        h->plans = false;
    }
    const size_t cells = (size_t)N * N * N, half = (size_t)N * N * (N / 2 + 1);
    int rc = ensure(h->mesh_q, 8 * cells);
    if (!rc) rc = ensure(h->mesh_r, 4 * cells);
    if (!rc) rc = ensure(h->mesh_c, 8 * half);
    if (!rc) rc = ensure(h->mesh_a, 16 * cells);
    if (!rc) rc = ensure(h->tab, 8 * (size_t)N);
    if (!rc) rc = ensure(h->scale, 16);
    if (rc) return rc;
    size_t w1 = 0, w2 = 0;
    rc = cufft_check(cufftCreate(&h->plan_r2c), "cufftCreate");
    if (rc) return rc;
    if ((rc = cufft_check(cufftCreate(&h->plan_c2r), "cufftCreate"))) {
        cufftDestroy(h->plan_r2c);
        return rc;
    }
    h->plans = true;
    rc = cufft_check(cufftSetAutoAllocation(h->plan_r2c, 0), "cufftSetAutoAllocation");
    if (!rc) rc = cufft_check(cufftSetAutoAllocation(h->plan_c2r, 0), "cufftSetAutoAllocation");
    if (!rc) rc = cufft_check(cufftMakePlan3d(h->plan_r2c, N, N, N, CUFFT_R2C, &w1), "cufftMakePlan3d R2C");
    if (!rc) rc = cufft_check(cufftMakePlan3d(h->plan_c2r, N, N, N, CUFFT_C2R, &w2), "cufftMakePlan3d C2R");
    if (!rc) rc = ensure(h->fft_work, std::max<size_t>(std::max(w1, w2), 16));
    if (!rc) rc = cufft_check(cufftSetWorkArea(h->plan_r2c, h->fft_work.p), "cufftSetWorkArea");
    if (!rc) rc = cufft_check(cufftSetWorkArea(h->plan_c2r, h->fft_work.p), "cufftSetWorkArea");
    if (rc) {
        cufftDestroy(h->plan_r2c);
        cufftDestroy(h->plan_c2r);
        h->plans = false;
        return rc;
    }
    h->n_mesh = N;
    h->tab_rs = -1.0;
    return PH_OK;
}

// The per-axis factors of the Green's function: sin^2(pi l / N) and
// exp(-(2 pi l' / L)^2 R_s^2) with l' the signed frequency, in FP64 on the
// host, rounded to FP32; uploaded when N, L or R_s change.
int pm_tables(ph_pm *h, double L, double rs, cudaStream_t s)
{
    if (h->tab_L == L && h->tab_rs == rs) return PH_OK;
    const int N = h->n_mesh;
    std::vector<float> t(2 * (size_t)N);
    for (int l = 0; l < N; l++) {
        const double sn = std::sin(M_PI * l / N);
        t[l] = (float)(sn * sn);
        const int ls = l > N / 2 ? l - N : l;
        const double k = 2.0 * M_PI * ls / L;
        t[N + l] = (float)std::exp(-k * k * rs * rs);
    }
    int rc = cuda_check(cudaStreamSynchronize(s), "sync before table upload");
    if (!rc) rc = cuda_check(cudaMemcpy(h->tab.p, t.data(), t.size() * 4, cudaMemcpyHostToDevice), "upload PM tables");
    if (rc) return rc;
    h->tab_L = L;
    h->tab_rs = rs;
    return PH_OK;
}

}  // namespace

void pm_set_active(ph_pm *h, const uint8_t *active) { h->active = active; }

void pm_free(ph_pm *h)
{
    pm_release(h);
    delete h;
}

int pm_status(const ph_pm *h)
{
    uint32_t st = 0;
    int rc = cuda_check(cudaMemcpyAsync(&st, h->status.p, 4, cudaMemcpyDeviceToHost, h->last_stream), "read status");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(h->last_stream), "status sync");
    if (rc) return rc;
    if (st & ST_NONFINITE) return fail(PH_ERR_NONFINITE, "non-finite position or mass");
    return PH_OK;
}

}  // namespace phpp

using namespace phpp;

extern "C" {

int ph_pm_accel(const void *pos, int pos_type, const float *mass, int64_t n, const ph_params *params,
                int32_t n_mesh, float *acc, float *pot, int32_t accumulate, void *stream, ph_pm **pm)
{
    TraceRange trace_("ph_pm_accel");
    if (!pm || !params) return fail(PH_ERR_ARG, "pm and params must not be NULL");
    if (pos_type != PH_F32 && pos_type != PH_F64) return fail(PH_ERR_ARG, "pos_type must be PH_F32 or PH_F64");
    if (n < 0 || n >= (int64_t)1 << 31) return fail(PH_ERR_ARG, "n must be 0..2^31-1");
    if (n > 0 && (!pos || !acc)) return fail(PH_ERR_ARG, "pos and acc must not be NULL");
    if (n_mesh < 4 || n_mesh > PH_PM_MAX_MESH || (n_mesh & 1))
        return fail(PH_ERR_ARG, "n_mesh must be even and in 4..%d", PH_PM_MAX_MESH);
    const ph_params &p = *params;
    if (!(std::isfinite(p.L) && p.L > 0)) return fail(PH_ERR_ARG, "L must be finite and > 0");
    if (!(std::isfinite(p.rs) && p.rs >= 0)) return fail(PH_ERR_ARG, "rs must be >= 0");
    if (!std::isfinite(p.G)) return fail(PH_ERR_ARG, "G must be finite");
    ph_pm *h = *pm;
    if (h && h->kind != KIND_PM) return fail(PH_ERR_STATE, "handle is not a ph_pm");
    const bool fresh = !h;
    if (fresh) {
        h = new (std::nothrow) ph_pm();
        if (!h) return fail(PH_ERR_OOM, "host allocation failed");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last_stream = s;
    int rc = ensure(h->status, 16);
    if (!rc && fresh) rc = cuda_check(cudaMemsetAsync(h->status.p, 0, 16, s), "status reset");
    if (!rc) rc = pm_setup(h, n_mesh);
    if (!rc) rc = pm_tables(h, p.L, p.rs, s);
    if (rc) {
        if (fresh) pm_free(h);
        return rc;
    }
    *pm = h;
    h->last_n = n;
    if (n == 0) return PH_OK;

    // inputs and outputs in host memory go through device copies
    const void *dpos = pos;
    const float *dmass = mass;
    float *dacc = acc, *dpot = pot;
    const bool host_acc = !is_device_ptr(acc), host_pot = pot && !is_device_ptr(pot);
    const size_t pbytes = (size_t)n * 3 * (pos_type == PH_F64 ? 8 : 4);
    if (!is_device_ptr(pos)) {
        rc = ensure(h->in_pos, pbytes);
        if (!rc) rc = cuda_check(cudaMemcpyAsync(h->in_pos.p, pos, pbytes, cudaMemcpyHostToDevice, s), "copy positions");
        dpos = h->in_pos.p;
    }
    if (!rc && mass && !is_device_ptr(mass)) {
        rc = ensure(h->in_mass, (size_t)n * 4);
        if (!rc) rc = cuda_check(cudaMemcpyAsync(h->in_mass.p, mass, (size_t)n * 4, cudaMemcpyHostToDevice, s),
                                 "copy masses");
        dmass = static_cast<const float *>(h->in_mass.p);
    }
    if (!rc && host_acc) {
        rc = ensure(h->acc_tmp, (size_t)n * 12);
        dacc = static_cast<float *>(h->acc_tmp.p);
        if (!rc && accumulate)
            rc = cuda_check(cudaMemcpyAsync(dacc, acc, (size_t)n * 12, cudaMemcpyHostToDevice, s), "copy acc in");
    }
    if (!rc && host_pot) {
        rc = ensure(h->pot_tmp, (size_t)n * 4);
        dpot = static_cast<float *>(h->pot_tmp.p);
    }
    if (rc) return rc;

    const int N = n_mesh;
    const int64_t cells = (int64_t)N * N * N;
    const double dg = p.L / N, inv_dg = (double)N / p.L;
    CellScale cs;
    cs.c_hi = (float)inv_dg;
    cs.c_lo = (float)(inv_dg - (double)cs.c_hi);
    cs.L_up = (float)p.L;
    if ((double)cs.L_up < p.L) cs.L_up = std::nextafter(cs.L_up, INFINITY);
    const float mdef = (float)(1.0 / (double)n);
    uint32_t *st = static_cast<uint32_t *>(h->status.p);
    uint32_t *mmax = static_cast<uint32_t *>(h->scale.p);
    unsigned long long *mq = static_cast<unsigned long long *>(h->mesh_q.p);
    rc = cuda_check(cudaMemsetAsync(mmax, 0, 4, s), "clear scale");
    if (!rc) rc = cuda_check(cudaMemsetAsync(mq, 0, 8 * (size_t)cells, s), "clear mesh");
    if (rc) return rc;
    k_pm_mass_max<<<dmass ? grid_of(n) : 1, kPmThreads, 0, s>>>(dmass, n, mdef, mmax, st);
    if (pos_type == PH_F64)
        k_pm_deposit<PH_F64><<<grid_of(n), kPmThreads, 0, s>>>(dpos, dmass, n, mdef, p.L, inv_dg, cs, N, mmax, mq,
                                                               st);
    else
        k_pm_deposit<PH_F32><<<grid_of(n), kPmThreads, 0, s>>>(dpos, dmass, n, mdef, p.L, inv_dg, cs, N, mmax, mq,
                                                               st);
    float *mr = static_cast<float *>(h->mesh_r.p);
    k_pm_unfix<<<grid_of(cells), kPmThreads, 0, s>>>(mq, cells, n, mmax, mr);
    count_launch(3);
    rc = cufft_check(cufftSetStream(h->plan_r2c, s), "cufftSetStream");
    if (!rc) rc = cufft_check(cufftSetStream(h->plan_c2r, s), "cufftSetStream");
    if (!rc) rc = cufft_check(cufftExecR2C(h->plan_r2c, mr, static_cast<cufftComplex *>(h->mesh_c.p)), "R2C");
    if (rc) return rc;
    const float *s2 = static_cast<const float *>(h->tab.p);
    const double c0 = -M_PI * p.G / (dg * (double)cells);
    k_pm_green<<<grid_of((int64_t)N * N * (N / 2 + 1)), kPmThreads, 0, s>>>(static_cast<float2 *>(h->mesh_c.p), N, s2,
                                                                          s2 + N, (float)c0);
    count_launch();
    rc = cufft_check(cufftExecC2R(h->plan_c2r, static_cast<cufftComplex *>(h->mesh_c.p), mr), "C2R");
    if (rc) return rc;
    float4 *ma = static_cast<float4 *>(h->mesh_a.p);
    k_pm_grad<<<grid_of(cells), kPmThreads, 0, s>>>(mr, N, (float)(-0.5 / dg), ma);
    if (pos_type == PH_F64)
        k_pm_interp<PH_F64><<<grid_of(n), kPmThreads, 0, s>>>(dpos, n, p.L, inv_dg, cs, N, ma, dacc, dpot,
                                                              accumulate, h->active);
    else
        k_pm_interp<PH_F32><<<grid_of(n), kPmThreads, 0, s>>>(dpos, n, p.L, inv_dg, cs, N, ma, dacc, dpot,
                                                              accumulate, h->active);
    count_launch(2);
    rc = cuda_check(cudaGetLastError(), "PM kernels");
    if (!rc && host_acc)
        rc = cuda_check(cudaMemcpyAsync(acc, dacc, (size_t)n * 12, cudaMemcpyDeviceToHost, s), "copy acc out");
    if (!rc && host_pot)
        rc = cuda_check(cudaMemcpyAsync(pot, dpot, (size_t)n * 4, cudaMemcpyDeviceToHost, s), "copy pot out");
    if (!rc && (host_acc || host_pot)) rc = cuda_check(cudaStreamSynchronize(s), "PM sync");
    return rc;
}

int ph_pm_get_view(const ph_pm *pm, ph_pm_view *out)
{
    if (!pm || pm->kind != KIND_PM || !out) return fail(PH_ERR_ARG, "bad arguments");
    int rc = cuda_check(cudaStreamSynchronize(pm->last_stream), "view sync");
    if (rc) return rc;
    memset(out, 0, sizeof *out);
    uint32_t bits = 0;
    rc = cuda_check(cudaMemcpy(&bits, pm->scale.p, 4, cudaMemcpyDeviceToHost), "read scale");
    if (rc) return rc;
    float mmax = 0.f;
    memcpy(&mmax, &bits, 4);
    const double b = (double)mmax * (double)pm->last_n;
    out->n_mesh = pm->n_mesh;
    out->mass_unit = b > 0.0 ? std::ldexp(1.0, std::ilogb(b) + 1 - 62) : 1.0;
    out->mass_fixed = static_cast<const int64_t *>(pm->mesh_q.p);
    out->mesh = static_cast<const float *>(pm->mesh_a.p);
    return PH_OK;
}

}  // extern "C"
