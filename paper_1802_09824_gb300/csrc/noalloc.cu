// ph_accel_noalloc: the whole short-range step for one small box, with every
// intermediate buffer carved out of one fixed device array that the library
// owns for the life of the process.  No cudaMalloc, no cudaFree, no host heap.
//
// Who needs it: code that may not allocate device memory itself -- a host
// application that hands the library a fixed memory budget through its own
// allocator, or a latency-critical loop that cannot afford the implicit
// device-wide synchronisation cudaMalloc/cudaFree bring.  Such a caller still
// owns the positions, masses and accelerations; only the scratch is ours.
//
// The scratch array is a file-scope __device__ variable, so every GPU that
// loads libphpp.so holds PH_NOALLOC_SCRATCH_BYTES of it until exit.  Host
// code must not use the array's name as a pointer (on the host it is only a
// shadow symbol); its device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device.
#include <cmath>
#include <cstring>
#include <mutex>

#include "handles.cuh"

namespace phpp {
int build_leaves_device(ph_leaves *h, const void *pos, int pos_type, const float *mass, cudaStream_t s);
int build_pairs_device(const ph_leaves *lv, ph_pairs *pr, cudaStream_t s, bool sizing_sync);
int pp_exact_device(const ph_leaves *lv, const ph_pairs *pr, float *d_acc, cudaStream_t s);
}  // namespace phpp

using namespace phpp;

namespace {

constexpr size_t kScratchBytes = (size_t)PH_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

void *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device.
int scratch_address(void **out)
{
    int dev = 0;
    int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev < 0 || dev >= kMaxDevices) return fail(PH_ERR_ARG, "device ordinal %d above %d", dev, kMaxDevices - 1);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        rc = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(scratch)");
        if (rc) return rc;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PH_OK;
}

// Bump carver over the scratch array (256-byte aligned slices); with base
// NULL it only measures.
struct Carver {
    char *base;
    size_t used = 0;
    bool over = false;
    void take(DevBuf &b, size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        size_t at = (used + 255) & ~(size_t)255;
        if (at + bytes > kScratchBytes) {
            over = true;
            b.p = nullptr;
            b.bytes = 0;
            return;
        }
        b.p = base ? base + at : nullptr;
        b.bytes = bytes;
        used = at + bytes;
    }
};

// Carve every buffer of the step for n particles and `cells` ground cells.
void carve(Carver &c, ph_leaves &lv, ph_pairs &pr, int64_t n, int cells)
{
    const size_t N = (size_t)n;
    c.take(lv.boxes, sizeof(BoxDev));
    c.take(lv.box_first, 2 * sizeof(int32_t));
    c.take(lv.keys, 8 * N);
    c.take(lv.keys_alt, 8 * N);
    c.take(lv.vals, 4 * N);
    c.take(lv.vals_alt, 4 * N);
    c.take(lv.xw, 24 * N);
    c.take(lv.mass_sorted, 4 * N);
    c.take(lv.cell_first, 4 * (size_t)(cells + 1));
    c.take(lv.leaf_flag, 4 * N);
    c.take(lv.group_flag, 4 * N);
    c.take(lv.leaf_scan, 4 * (N + 1));
    c.take(lv.group_scan, 4 * (N + 1));
    c.take(lv.leaf_first, 4 * (N + 1));
    c.take(lv.group_first, 4 * (N + 1));
    c.take(lv.leaf_ref, 24 * N);
    c.take(lv.leaf_c4, 16 * N);
    c.take(lv.leaf_h4, 16 * N);
    c.take(lv.group_ref, 24 * N);
    c.take(lv.group_c4, 16 * N);
    c.take(lv.group_h4, 16 * N);
    c.take(lv.leaf_r4, 16 * N);
    c.take(lv.group_r4, 16 * N);
    c.take(lv.box_ext, 96 * N);
    c.take(lv.group_cell, 4 * N);
    c.take(lv.group_box, 4 * N);
    c.take(lv.pos_leaf, 16 * N);
    c.take(lv.pos_group, 16 * N);
    c.take(lv.cell_leaf_first, 4 * (size_t)(cells + 1));
    c.take(lv.counts, 16);
    c.take(lv.status, 16);
    const size_t tsort = sort_temp_bytes(n), tscan = scan_temp_bytes(n);
    c.take(lv.temp, tsort > tscan ? tsort : tscan);
    c.take(pr.group_cnt, 8 * (N + 1));
    c.take(pr.group_off, 8 * (N + 1));
    c.take(pr.work, 64);
    c.take(pr.status, 16);
    c.take(pr.temp, tscan);
    const size_t cap = (size_t)PH_NOALLOC_PAIRS_PER_PARTICLE * N;
    c.take(pr.entries, 16 * cap);
    c.take(pr.ecount, cap);
}

}  // namespace

extern "C" int ph_accel_noalloc(const float *d_pos, const float *d_mass, int64_t n, const ph_params *params,
                                float *d_acc, void *stream)
{
    if (!params) return fail(PH_ERR_ARG, "params must not be NULL");
    if (n < 0 || n > PH_NOALLOC_MAX_N)
        return fail(PH_ERR_ARG, "ph_accel_noalloc: n = %lld outside 0..%d (the fixed scratch holds at most %d particles)",
                    (long long)n, PH_NOALLOC_MAX_N, PH_NOALLOC_MAX_N);
    const ph_params &p = *params;
    if (!(std::isfinite(p.L) && p.L > 0) || !(std::isfinite(p.rs) && p.rs > 0) || !(std::isfinite(p.eps) && p.eps >= 0) ||
        !std::isfinite(p.G) || !(std::isfinite(p.rcut) && p.rcut > 0))
        return fail(PH_ERR_ARG, "ph_accel_noalloc: L, rs, rcut must be finite and > 0, eps >= 0, G finite");
    if (!(p.rcut < 0.5 * p.L)) return fail(PH_ERR_RCUT_GE_HALF_L, "rcut %g >= L/2 %g", p.rcut, 0.5 * p.L);
    if (p.leaf_max < 1 || p.leaf_max > kMaxLeaf) return fail(PH_ERR_ARG, "leaf_max must be 1..%d", kMaxLeaf);
    if (p.theta != 0) return fail(PH_ERR_ARG, "ph_accel_noalloc: theta must be 0 (every leaf pair by PP)");
    if (p.key_kind != PH_KEY_MORTON && p.key_kind != PH_KEY_HILBERT) return fail(PH_ERR_ARG, "unknown key_kind");
    if (p.group_size != 0 && p.group_size != 32) return fail(PH_ERR_ARG, "group_size must be 0 or 32");
    if (p.level_bits != 0 && p.level_bits != 1 && p.level_bits != 3) return fail(PH_ERR_ARG, "level_bits must be 0, 1 or 3");
    if (p.pp_variant != 0 && p.pp_variant != 1) return fail(PH_ERR_ARG, "pp_variant must be 0 or 1");
    const int deg = poly_degree_for(p.rcut / (2.0 * p.rs));
    if (deg < 0) return fail(PH_ERR_ARG, "rcut/rs = %g above the supported 9.2", p.rcut / p.rs);
    const int g = ground_level(p.L, p.rcut);
    const int nside = 1 << g;
    const int cells = nside * nside * nside;
    if (cells > PH_NOALLOC_MAX_CELLS)
        return fail(PH_ERR_ARG, "ph_accel_noalloc: L/rcut gives %d ground cells, above the fixed %d", cells,
                    PH_NOALLOC_MAX_CELLS);
    {
        // the documented maximum must fit the array whatever n this call has,
        // so a buffer that grows breaks every call, not only the largest ones
        ph_leaves lm;
        ph_pairs pm;
        Carver dry{nullptr};
        carve(dry, lm, pm, PH_NOALLOC_MAX_N, PH_NOALLOC_MAX_CELLS);
        if (dry.over)
            return fail(PH_ERR_CAPACITY, "ph_accel_noalloc: the fixed scratch (%u bytes) is smaller than its "
                        "documented maximum of %d particles and %d cells needs", PH_NOALLOC_SCRATCH_BYTES,
                        PH_NOALLOC_MAX_N, PH_NOALLOC_MAX_CELLS);
    }
    if (n == 0) return PH_OK;
    if (!d_pos || !d_acc || !is_device_ptr(d_pos) || !is_device_ptr(d_acc) || (d_mass && !is_device_ptr(d_mass)))
        return fail(PH_ERR_ARG, "ph_accel_noalloc: pos, mass and acc must be device memory");

    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // one box with the constants and key depth ph_build_leaves derives for it
    const int T = key_bits_for(n, g, 1);
    BoxDev bx;
    fill_box(bx, p, T, deg, n, 0, 0, kDefaultGroup);
    const int32_t box_first[2] = {0, (int32_t)n};

    ph_leaves lv;   // host descriptors only; every buffer points into the scratch
    ph_pairs pr;
    lv.n = n;
    lv.n_boxes = 1;
    lv.n_cells = cells;
    lv.key_bits = T;
    lv.group_size = kDefaultGroup;
    lv.poly_degree = deg;
    lv.max_leaf = p.leaf_max;
    lv.key_kind = p.key_kind;
    lv.level_bits = p.level_bits ? p.level_bits : 1;
    lv.pp_variant = p.pp_variant == 1 ? 1 : 0;
    Carver c{static_cast<char *>(base)};
    carve(c, lv, pr, n, cells);
    if (c.over) return fail(PH_ERR_CAPACITY, "ph_accel_noalloc: fixed scratch too small for n = %lld", (long long)n);
    pr.capacity = (int64_t)PH_NOALLOC_PAIRS_PER_PARTICLE * n;
    pr.fixed_capacity = true;

    // the array keeps the previous call's contents: clear what must start at zero
    rc = cuda_check(cudaMemsetAsync(lv.status.p, 0, 16, s), "clear status");
    if (!rc) rc = cuda_check(cudaMemsetAsync(pr.status.p, 0, 16, s), "clear pair status");
    if (!rc) rc = cuda_check(cudaMemsetAsync(lv.counts.p, 0, 16, s), "clear counts");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(lv.boxes.p, &bx, sizeof bx, cudaMemcpyHostToDevice, s), "copy box");
    if (!rc)
        rc = cuda_check(cudaMemcpyAsync(lv.box_first.p, box_first, sizeof box_first, cudaMemcpyHostToDevice, s),
                        "copy box table");
    if (!rc) rc = build_leaves_device(&lv, d_pos, PH_F32, d_mass, s);
    if (!rc) rc = build_pairs_device(&lv, &pr, s, false);
    if (!rc) rc = pp_exact_device(&lv, &pr, d_acc, s);
    // one synchronisation: the box record lives on this stack frame, and the
    // latched device status decides the return code
    uint32_t st[2] = {0, 0};
    if (!rc) rc = cuda_check(cudaMemcpyAsync(&st[0], lv.status.p, 4, cudaMemcpyDeviceToHost, s), "read status");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(&st[1], pr.status.p, 4, cudaMemcpyDeviceToHost, s), "read status");
    int sync_rc = cuda_check(cudaStreamSynchronize(s), "ph_accel_noalloc sync");
    if (!rc) rc = sync_rc;
    if (rc) return rc;
    if ((st[0] | st[1]) & ST_NONFINITE) return fail(PH_ERR_NONFINITE, "non-finite position or mass");
    if ((st[0] | st[1]) & ST_CAPACITY)
        return fail(PH_ERR_CAPACITY, "ph_accel_noalloc: more than %d leaf pairs per particle (fixed list capacity)",
                    PH_NOALLOC_PAIRS_PER_PARTICLE);
    return PH_OK;
}
