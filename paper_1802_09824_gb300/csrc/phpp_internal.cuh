// Internal declarations shared by the translation units of libphpp.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/phpp.h"

namespace phpp {

// An NVTX range around a public call, for profilers that record ranges (ncu
// --nvtx, Nsight Systems); without an attached tool it costs a test of a
// function pointer.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// ---------------------------------------------------------------- limits
constexpr int kMaxPoly = 16;          // highest degree of the factor polynomial
constexpr int kMaxLeaf = 256;         // largest leaf_max accepted
constexpr int kGroundMax = 7;         // N_side <= 2^7 per box
constexpr int kSortBits = 8;          // radix digit width
constexpr int kThreads = 256;
constexpr int kDefaultGroup = 32;   // target group size when ph_params.group_size = 0

// Per-box constants, one record per box in device memory.
struct BoxDev {
    double L;          // box side
    double S;          // 2^T / L: quantisation scale of the key grid
    double h;          // ground cell side L / N_side
    float G;
    float eps2;        // eps^2
    float rcut2;       // rcut^2 (cutoff decision of the PP kernel)
    float rfilt2;      // (rcut (1 + margin))^2 for conservative box tests
    float c_v;         // v = sqrt(r^2 c_v) = r / (R_s U), t = v - 1 in [-1, 1]
    float c_t;         // 2 / rcut: t = sqrt(r^2) c_t - 1 (exact kernel)
    float c_e;         // exp(-r^2 / 4R_s^2) = 2^(r^2 c_e)
    float mass_default;
    int32_t g;         // ground level, N_side = 2^g
    int32_t b;         // local key bits per axis
    int32_t nside;
    int32_t cell_base; // first global ground cell of this box
    int32_t first;     // first particle row of this box
    int32_t n;         // particles in this box
    int32_t group_size;
    int32_t pad;
    float poly[kMaxPoly + 1];   // h(t) = sum poly[k] t^k, f = 2^(r^2 c_e) h
    // Scaled softening for the exact kernel: x = r^2 s2 + eps2s is O(1) at the
    // cutoff (s2 = 4^-k, a power of four near 1 / (rcut^2 + eps^2)), so x^3
    // stays a normal FP32 number and (r^2 + eps^2)^(-3/2) = s2^(3/2) x^(-3/2)
    // with the power of two s2^(3/2) folded into c_g = G s2^(3/2).
    float s2;
    float eps2s;       // max(eps^2 s2, 1e-12)
    float c_g;
    float L_up;        // smallest FP32 number >= L: an FP32 x is below L iff x < L_up
    float c_acc;       // 1 / theta of the tree part (infinite: every leaf pair by PP)
};

// The smallest FP32 number not below L.
inline float float_at_or_above(double L)
{
    float f = (float)L;
    if ((double)f < L) f = std::nextafter(f, INFINITY);
    return f;
}

// Ground level of a box (N_side = 2^g cells of side >= rcut); api.cu.
int ground_level(double L, double rcut);

// Key bits per axis for n_boxes boxes of at most nmax particles whose finest
// ground level is gmax; api.cu.
int key_bits_for(int64_t nmax, int gmax, int n_boxes);

// Degree of the factor polynomial for U = rcut / (2 rs), -1 if unsupported;
// api.cu.
int poly_degree_for(double U);

// The device record of one box (constants of the build, the pair builder and
// the PP kernel) from its parameters; api.cu.
void fill_box(BoxDev &bx, const struct ph_params &p, int key_bits, int poly_degree, int64_t n_box, int cell_base,
              int32_t first, int group_size);

// Active-particle mode of a PM handle (pm.cu): interpolate only the
// particles flagged in `active` (caller order, device; NULL = all).
void pm_set_active(ph_pm *h, const uint8_t *active);

// Streaming multiprocessors of the current device (persistent grids).
inline int sm_count()
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

// Softening and force-scale constants of one box (see BoxDev).
inline void set_softening(BoxDev &bx, double G, double eps, double rcut)
{
    const double e2 = eps * eps;
    bx.G = (float)G;
    bx.eps2 = (float)(e2 > 1e-24 ? e2 : 1e-24);
    const int k = (int)std::lround(0.5 * std::log2(rcut * rcut + e2));
    bx.s2 = (float)std::ldexp(1.0, -2 * k);
    const double es = e2 * std::ldexp(1.0, -2 * k);
    bx.eps2s = (float)(es > 1e-12 ? es : 1e-12);
    bx.c_g = (float)(G * std::ldexp(1.0, -3 * k));
}

// Device-side status word bits.
enum : uint32_t {
    ST_NONFINITE = 1u,
    ST_CAPACITY = 2u,
    ST_TIMEOUT = 4u,
};

// ---------------------------------------------------------------- handles
enum HandleKind : uint32_t {
    KIND_LEAVES = 0x4c454146u,
    KIND_PAIRS = 0x50414952u,
    KIND_MLP = 0x4d4c5021u,
    KIND_GRAPH = 0x47524150u,
    KIND_PM = 0x504d2121u,
    KIND_SIM = 0x53494d21u,
};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct ph_leaves_impl;
struct ph_pairs_impl;

// Thread-local error message.
void set_error(const char *fmt, ...);
int fail(int code, const char *fmt, ...);

// Grow a device buffer to at least `bytes` (contents not preserved).
int ensure(DevBuf &b, size_t bytes);
void release(DevBuf &b);

// true if `p` is device-accessible memory (device or managed).
bool is_device_ptr(const void *p);

int cuda_check(cudaError_t e, const char *what);

// Host-side count of kernel launches issued by the library (all threads).
void count_launch(int n = 1);

// Debug bounds checks (checks.cuh): each translation unit of a checked build
// registers a reader of its device words (hits, first site) at load time.
void register_bounds_reader(int (*read)(unsigned int *hits, unsigned int *site));

// ---------------------------------------------------------------- kernels
// scan.cu: exclusive scans over n elements (n read from device memory when
// d_n != nullptr, else the host value).  out[n] receives the total.
size_t scan_temp_bytes(int64_t max_n);
int scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, const int32_t *d_n, void *temp,
                       cudaStream_t s);
int scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, const int32_t *d_n, void *temp,
                       cudaStream_t s);

// pairs.cu: scratch of the PP queue's group order for up to n groups.
size_t order_temp_bytes(int64_t n);

// sort.cu: stable LSD radix sort of (key, value) pairs on the low `bits` bits.
size_t sort_temp_bytes(int64_t n);
int radix_sort_pairs(uint64_t *keys, int32_t *vals, uint64_t *keys_alt, int32_t *vals_alt, int64_t n, int bits,
                     void *temp, cudaStream_t s, bool *result_in_alt);

}  // namespace phpp
