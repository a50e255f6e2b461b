// C ABI entry points: argument checks, handle management, host/device
// staging.  Every step of the computation runs in the kernels of build.cu,
// pairs.cu and pp.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "handles.cuh"
#include "mlp_handle.cuh"

namespace phpp {

int build_leaves_device(ph_leaves *h, const void *pos, int pos_type, const float *mass, cudaStream_t s);
int build_pairs_device(const ph_leaves *lv, ph_pairs *pr, cudaStream_t s, bool sizing_sync);
int pp_exact_device(const ph_leaves *lv, const ph_pairs *pr, float *d_acc, cudaStream_t s);
int count_within_device(const ph_leaves *lv, const ph_pairs *pr, cudaStream_t s);
int pp_learned_device(const ph_leaves *lv, const ph_pairs *pr, const float *mlp_w, float *d_acc, cudaStream_t s);
int pp_table_device(const ph_leaves *lv, const ph_pairs *pr, float *d_acc, cudaStream_t s);

// The tabulated factor of PH_G_TABLE for the handle's (single) rs and rcut:
// f(r_i) = erfc(u) + (2u / sqrt(pi)) exp(-u^2), u = r_i / (2 rs), at
// r_i = i rcut / 4096, i = 0..4096, with f'(r_i) dr = -(4 u^2 / sqrt(pi))
// exp(-u^2) / (2 rs) dr, in FP64 then rounded to FP32; uploaded once per
// (rs, rcut) before any launch that reads it.
int ensure_table(ph_leaves *lv, cudaStream_t s)
{
    if (lv->n_boxes < 1 || (int)lv->boxes_host.size() < lv->n_boxes) return fail(PH_ERR_STATE, "no boxes");
    const double rcut = std::sqrt((double)lv->boxes_host[0].rcut2);
    const double rs = std::sqrt(-1.4426950408889634 / (4.0 * (double)lv->boxes_host[0].c_e));
    for (int b = 1; b < lv->n_boxes; b++)
        if (lv->boxes_host[b].rcut2 != lv->boxes_host[0].rcut2 || lv->boxes_host[b].c_e != lv->boxes_host[0].c_e)
            return fail(PH_ERR_ARG, "the tabulated factor needs one rcut and rs for all boxes");
    if (lv->table.p && lv->table_rs == rs && lv->table_rcut == rcut) return PH_OK;
    constexpr int N = 4096;
    std::vector<float> host(2 * (N + 1));
    const double dr = rcut / N, sqpi = std::sqrt(M_PI);
    for (int i = 0; i <= N; i++) {
        const double u = i * dr / (2.0 * rs);
        const double e = std::exp(-u * u);
        host[2 * i] = (float)(std::erfc(u) + 2.0 * u / sqpi * e);
        host[2 * i + 1] = (float)(-4.0 * u * u / sqpi * e / (2.0 * rs) * dr);
    }
    int rc = ensure(lv->table, host.size() * sizeof(float));
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "sync before table upload");
    if (!rc) rc = cuda_check(cudaMemcpy(lv->table.p, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice),
                             "upload factor table");
    if (rc) return rc;
    lv->table_rs = rs;
    lv->table_rcut = rcut;
    return PH_OK;
}
void graph_free(ph_graph *g);
void pm_free(ph_pm *h);
int pm_status(const ph_pm *h);
void sim_free(ph_sim *h);
void fit_factor_poly(double U, int deg, float *coef);

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// The translation units' bounds-word readers (checked builds), filled by
// their static initialisers when the library is loaded.
static std::vector<int (*)(unsigned int *, unsigned int *)> &bounds_readers()
{
    static std::vector<int (*)(unsigned int *, unsigned int *)> v;
    return v;
}

void register_bounds_reader(int (*read)(unsigned int *hits, unsigned int *site)) { bounds_readers().push_back(read); }

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_check(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return PH_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(PH_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(PH_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Testing hook (ph_debug_fail_allocation): the number of device allocations
// still allowed before one fails as if the device were out of memory; -1 off.
static std::atomic<long long> g_fail_after{-1};

int ensure(DevBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return PH_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    long long k = g_fail_after.load();
    while (k >= 0 && !g_fail_after.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 0) return fail(PH_ERR_OOM, "cudaMalloc(%zu bytes) failed: injected allocation failure", bytes);
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return fail(PH_ERR_OOM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return PH_OK;
}

void release(DevBuf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Ground level g of a box: the finest N_side = 2^g (g <= kGroundMax) whose
// cells are at least rcut wide (Sec. 4.3: a cell and its 26 neighbours hold
// every particle within rcut of the cell).
int ground_level(double L, double rcut)
{
    int g = 0;
    while (g < kGroundMax && L / (double)(1 << (g + 1)) >= rcut) g++;
    return g;
}

static int key_bits_per_axis(int n_boxes)
{
    int box_bits = 0;
    while ((1 << box_bits) < n_boxes) box_bits++;
    return (63 - box_bits) / 3;
}

// Key bits per axis: enough for cells ~64 times finer than the mean spacing
// of the most populated box (deeper cells never hold more than leaf_max
// particles outside strong clustering; cells that do are cut into runs),
// capped by the 63-bit key and at least 4 bits below the ground grid.  The
// sort takes ceil((3 T + box bits) / 8) passes: 5 for 2^21 particles in one
// box.
int key_bits_for(int64_t nmax, int gmax, int n_boxes)
{
    int lg = 0;
    while ((int64_t)1 << (3 * lg) < nmax) lg++;     // ceil(log2(cbrt(nmax)))
    return std::min(key_bits_per_axis(n_boxes), std::max(lg + 6, gmax + 4));
}

int poly_degree_for(double U)
{
    if (U <= 2.3) return 10;
    if (U <= 3.05) return 12;
    if (U <= 4.05) return 14;
    if (U <= 4.6) return 16;
    return -1;
}

static int check_params(const ph_params &p, int b)
{
    if (!(std::isfinite(p.L) && p.L > 0)) return fail(PH_ERR_ARG, "box %d: L must be finite and > 0", b);
    if (!(std::isfinite(p.rs) && p.rs > 0)) return fail(PH_ERR_ARG, "box %d: rs must be > 0", b);
    if (!(std::isfinite(p.eps) && p.eps >= 0)) return fail(PH_ERR_ARG, "box %d: eps must be >= 0", b);
    if (!std::isfinite(p.G)) return fail(PH_ERR_ARG, "box %d: G must be finite", b);
    if (!(std::isfinite(p.rcut) && p.rcut > 0)) return fail(PH_ERR_ARG, "box %d: rcut must be > 0", b);
    if (!(p.rcut < 0.5 * p.L)) return fail(PH_ERR_RCUT_GE_HALF_L, "box %d: rcut %g >= L/2 %g", b, p.rcut, 0.5 * p.L);
    if (p.leaf_max < 1 || p.leaf_max > kMaxLeaf) return fail(PH_ERR_ARG, "box %d: leaf_max must be 1..%d", b, kMaxLeaf);
    if (p.key_kind != PH_KEY_MORTON && p.key_kind != PH_KEY_HILBERT)
        return fail(PH_ERR_ARG, "box %d: unknown key_kind %d", b, p.key_kind);
    if (p.group_size != 0 && p.group_size != 8 && p.group_size != 16 && p.group_size != 32)
        return fail(PH_ERR_ARG, "box %d: group_size must be 0, 8, 16 or 32", b);
    if (p.level_bits != 0 && p.level_bits != 1 && p.level_bits != 3)
        return fail(PH_ERR_ARG, "box %d: level_bits must be 0, 1 or 3", b);
    if (p.pp_variant != 0 && p.pp_variant != 1) return fail(PH_ERR_ARG, "box %d: pp_variant must be 0 or 1", b);
    if (p.queue_order != 0 && p.queue_order != 1) return fail(PH_ERR_ARG, "box %d: queue_order must be 0 or 1", b);
    if (!(std::isfinite(p.theta) && p.theta >= 0 && p.theta < 1))
        return fail(PH_ERR_ARG, "box %d: theta must be in [0, 1)", b);
    if (poly_degree_for(p.rcut / (2.0 * p.rs)) < 0)
        return fail(PH_ERR_ARG, "box %d: rcut/rs = %g above the supported 9.2", b, p.rcut / p.rs);
    return PH_OK;
}

void fill_box(BoxDev &bx, const ph_params &p, int key_bits, int poly_degree, int64_t n_box, int cell_base,
              int32_t first, int group_size)
{
    memset(&bx, 0, sizeof bx);
    bx.L = p.L;
    bx.L_up = float_at_or_above(p.L);
    bx.c_acc = p.theta > 0 ? (float)(1.0 / p.theta) : INFINITY;
    bx.g = ground_level(p.L, p.rcut);
    bx.b = key_bits - bx.g;
    bx.nside = 1 << bx.g;
    bx.S = std::ldexp(1.0, key_bits) / p.L;
    bx.h = p.L / bx.nside;
    set_softening(bx, p.G, p.eps, p.rcut);
    bx.rcut2 = (float)(p.rcut * p.rcut);
    const double rf = p.rcut * (1.0 + 3e-5);
    bx.rfilt2 = (float)(rf * rf);
    bx.c_v = (float)(4.0 / (p.rcut * p.rcut));
    bx.c_t = (float)(2.0 / p.rcut);
    bx.c_e = (float)(-1.4426950408889634 / (4.0 * p.rs * p.rs));
    bx.mass_default = n_box > 0 ? (float)(1.0 / (double)n_box) : 0.f;
    bx.cell_base = cell_base;
    bx.first = first;
    bx.n = (int32_t)n_box;
    bx.group_size = group_size;
    fit_factor_poly(p.rcut / (2.0 * p.rs), poly_degree, bx.poly);
}

int check_built(const ph_leaves *lv, const ph_pairs *pr)
{
    if (!lv->valid) return fail(PH_ERR_STATE, "the leaves handle holds no completed build (a build failed)");
    if (pr && !pr->valid) return fail(PH_ERR_STATE, "the pairs handle holds no completed list (ph_leaf_pairs failed)");
    if (pr && pr->leaves_generation != lv->generation)
        return fail(PH_ERR_STATE, "the pair list was made for an earlier build of the leaves: call ph_leaf_pairs");
    return PH_OK;
}

static void fp_mix(uint64_t &h, uint64_t v)
{
    for (int i = 0; i < 8; i++) {
        h ^= (v >> (8 * i)) & 0xffu;
        h *= 1099511628211ull;
    }
}

// (The factor table is left out: it has one fixed size, so once made it
// never moves; the other buffers move when a build needs them larger.)
uint64_t buffers_fingerprint(const ph_leaves *h, const ph_pairs *p)
{
    uint64_t f = 1469598103934665603ull;
    const DevBuf *lb[] = {&h->boxes, &h->box_first, &h->keys, &h->keys_alt, &h->vals, &h->vals_alt, &h->xw,
                          &h->mass_sorted, &h->cell_first, &h->leaf_flag, &h->group_flag, &h->leaf_scan,
                          &h->group_scan, &h->leaf_first, &h->group_first, &h->leaf_ref, &h->leaf_c4, &h->leaf_h4,
                          &h->group_ref, &h->group_c4, &h->group_h4, &h->leaf_r4, &h->group_r4, &h->box_ext,
                          &h->work, &h->group_cell, &h->group_box, &h->pos_leaf, &h->pos_group,
                          &h->cell_leaf_first, &h->counts, &h->status, &h->temp, &h->group_act, &h->group_act_scan,
                          &h->active_list};
    for (const DevBuf *b : lb) {
        fp_mix(f, (uint64_t)(uintptr_t)b->p);
        fp_mix(f, (uint64_t)b->bytes);
    }
    fp_mix(f, (uint64_t)h->n);
    if (p) {
        const DevBuf *pb[] = {&p->group_cnt, &p->group_off, &p->entries, &p->ecount, &p->work, &p->status, &p->temp,
                              &p->group_key, &p->group_order, &p->order_temp};
        for (const DevBuf *b : pb) {
            fp_mix(f, (uint64_t)(uintptr_t)b->p);
            fp_mix(f, (uint64_t)b->bytes);
        }
        fp_mix(f, (uint64_t)p->capacity);
    }
    return f;
}

static void free_leaves(ph_leaves *h)
{
    DevBuf *bufs[] = {&h->boxes, &h->box_first, &h->in_pos, &h->in_mass, &h->keys, &h->keys_alt, &h->vals,
                      &h->vals_alt, &h->xw, &h->mass_sorted, &h->cell_first, &h->leaf_flag, &h->group_flag,
                      &h->leaf_scan, &h->group_scan, &h->leaf_first, &h->group_first, &h->leaf_ref, &h->leaf_c4,
                      &h->leaf_h4, &h->group_ref, &h->group_c4, &h->group_h4, &h->leaf_r4, &h->group_r4, &h->box_ext, &h->work, &h->acc_tmp, &h->table, &h->group_cell, &h->group_box,
                      &h->pos_leaf, &h->pos_group, &h->cell_leaf_first, &h->counts, &h->status, &h->temp,
                      &h->group_act, &h->group_act_scan, &h->active_list};
    for (DevBuf *b : bufs) release(*b);
}

static void free_pairs(ph_pairs *h)
{
    DevBuf *bufs[] = {&h->group_cnt, &h->group_off, &h->entries, &h->ecount, &h->work, &h->status, &h->temp,
                      &h->acc_tmp, &h->group_key, &h->group_order, &h->order_temp};
    for (DevBuf *b : bufs) release(*b);
}

// Set up boxes and buffers for n particles, copy host inputs, launch the build.
static int leaves_common(const void *pos, int pos_type, const float *mass, const int64_t *box_offsets, int32_t nb,
                         const ph_params *params, void *stream, ph_leaves **leaves)
{
    if (!leaves) return fail(PH_ERR_ARG, "leaves must not be NULL");
    if (!params) return fail(PH_ERR_ARG, "params must not be NULL");
    if (pos_type != PH_F32 && pos_type != PH_F64) return fail(PH_ERR_ARG, "pos_type must be PH_F32 or PH_F64");
    if (nb < 1 || nb > 65536) return fail(PH_ERR_ARG, "n_boxes must be 1..65536");
    if (box_offsets[0] != 0) return fail(PH_ERR_ARG, "box_offsets[0] must be 0");
    for (int b = 0; b < nb; b++)
        if (box_offsets[b + 1] < box_offsets[b]) return fail(PH_ERR_ARG, "box_offsets must be non-decreasing");
    const int64_t n = box_offsets[nb];
    if (n < 0 || n >= (int64_t)1 << 31) return fail(PH_ERR_ARG, "n must be 0..2^31-1");
    if (n > 0 && !pos) return fail(PH_ERR_ARG, "pos must not be NULL");
    for (int b = 0; b < nb; b++) {
        int rc = check_params(params[b], b);
        if (rc) return rc;
        if (params[b].leaf_max != params[0].leaf_max || params[b].key_kind != params[0].key_kind ||
            params[b].group_size != params[0].group_size || params[b].level_bits != params[0].level_bits ||
            params[b].pp_variant != params[0].pp_variant || params[b].queue_order != params[0].queue_order)
            return fail(PH_ERR_ARG, "leaf_max, key_kind, group_size, level_bits, pp_variant and queue_order must be "
                                    "the same for all boxes");
    }
    ph_leaves *h = *leaves;
    if (h && h->kind != KIND_LEAVES) return fail(PH_ERR_STATE, "handle is not a ph_leaves");
    bool fresh = false;
    if (!h) {
        h = new (std::nothrow) ph_leaves();
        if (!h) return fail(PH_ERR_OOM, "host allocation failed");
        fresh = true;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->valid = false;   // until this build completes
    h->n = n;
    h->n_boxes = nb;
    {
        int64_t nmax = 1;
        int gmax = 0;
        for (int b = 0; b < nb; b++) {
            nmax = std::max<int64_t>(nmax, box_offsets[b + 1] - box_offsets[b]);
            gmax = std::max(gmax, ground_level(params[b].L, params[b].rcut));
        }
        h->key_bits = key_bits_for(nmax, gmax, nb);
    }
    h->max_leaf = params[0].leaf_max;
    h->key_kind = params[0].key_kind;
    h->group_size = params[0].group_size ? params[0].group_size : kDefaultGroup;
    h->level_bits = params[0].level_bits ? params[0].level_bits : 1;
    h->pp_variant = params[0].pp_variant;
    h->queue_order = params[0].queue_order;
    h->boxes_host.resize(nb);
    int deg = 10;
    for (int b = 0; b < nb; b++) {
        int d = poly_degree_for(params[b].rcut / (2.0 * params[b].rs));
        if (d > deg) deg = d;
    }
    h->poly_degree = deg;
    int cells = 0;
    std::vector<int32_t> bf(nb + 1);
    h->tree_leaves = false;
    for (int b = 0; b < nb; b++) {
        const ph_params &p = params[b];
        BoxDev &bx = h->boxes_host[b];
        if (p.theta > 0) h->tree_leaves = true;
        fill_box(bx, p, h->key_bits, deg, box_offsets[b + 1] - box_offsets[b], cells, (int32_t)box_offsets[b],
                 h->group_size);
        cells += bx.nside * bx.nside * bx.nside;
        bf[b] = (int32_t)box_offsets[b];
    }
    bf[nb] = (int32_t)n;
    h->n_cells = cells;
    const size_t N = (size_t)(n > 0 ? n : 1);
    int rc = 0;
#define ENS(buf, bytes) \
    if (!rc) rc = ensure(buf, bytes)
    ENS(h->boxes, sizeof(BoxDev) * nb);
    ENS(h->box_first, sizeof(int32_t) * (nb + 1));
    ENS(h->keys, 8 * N);
    ENS(h->keys_alt, 8 * N);
    ENS(h->vals, 4 * N);
    ENS(h->vals_alt, 4 * N);
    ENS(h->xw, 24 * N);
    ENS(h->mass_sorted, 4 * N);
    ENS(h->cell_first, 4 * (size_t)(cells + 1));
    ENS(h->leaf_flag, 4 * N);
    ENS(h->group_flag, 4 * N);
    ENS(h->leaf_scan, 4 * (N + 1));
    ENS(h->group_scan, 4 * (N + 1));
    ENS(h->leaf_first, 4 * (N + 1));
    ENS(h->group_first, 4 * (N + 1));
    ENS(h->leaf_ref, 24 * N);
    ENS(h->leaf_c4, 16 * N);
    ENS(h->leaf_h4, 16 * N);
    ENS(h->group_ref, 24 * N);
    ENS(h->group_c4, 16 * N);
    ENS(h->group_h4, 16 * N);
    ENS(h->leaf_r4, 16 * N);
    ENS(h->group_r4, 16 * N);
    ENS(h->box_ext, 96 * N);
    ENS(h->work, 64);
    ENS(h->group_cell, 4 * N);
    ENS(h->group_box, 4 * N);
    ENS(h->pos_leaf, 32 * N);
    ENS(h->pos_group, 16 * N);
    ENS(h->cell_leaf_first, 4 * (size_t)(cells + 1));
    ENS(h->counts, 16);
    ENS(h->status, 16);
    size_t tb = sort_temp_bytes(n);
    size_t ts = scan_temp_bytes(n);
    ENS(h->temp, tb > ts ? tb : ts);
    if (h->active) {
        ENS(h->group_act, 4 * (N + 1));
        ENS(h->group_act_scan, 4 * (N + 1));
        ENS(h->active_list, 4 * N);
    }
#undef ENS
    if (rc) {
        if (fresh) {
            free_leaves(h);
            delete h;
        }
        return rc;
    }
    if (fresh) {
        rc = cuda_check(cudaMemsetAsync(h->status.p, 0, 16, s), "status reset");
        if (rc) {
            free_leaves(h);
            delete h;
            return rc;
        }
    }
    rc = cuda_check(cudaMemcpyAsync(h->boxes.p, h->boxes_host.data(), sizeof(BoxDev) * nb, cudaMemcpyHostToDevice, s),
                    "copy boxes");
    if (!rc)
        rc = cuda_check(cudaMemcpyAsync(h->box_first.p, bf.data(), 4 * (nb + 1), cudaMemcpyHostToDevice, s),
                        "copy box table");
    // the box table copies read host memory that dies with this call
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "box table sync");
    const void *dpos = pos;
    const float *dmass = mass;
    if (!rc && n > 0 && !is_device_ptr(pos)) {
        size_t bytes = (size_t)n * 3 * (pos_type == PH_F64 ? 8 : 4);
        rc = ensure(h->in_pos, bytes);
        if (!rc) rc = cuda_check(cudaMemcpyAsync(h->in_pos.p, pos, bytes, cudaMemcpyHostToDevice, s), "copy positions");
        dpos = h->in_pos.p;
    }
    if (!rc && n > 0 && mass && !is_device_ptr(mass)) {
        rc = ensure(h->in_mass, (size_t)n * 4);
        if (!rc) rc = cuda_check(cudaMemcpyAsync(h->in_mass.p, mass, (size_t)n * 4, cudaMemcpyHostToDevice, s),
                                 "copy masses");
        dmass = static_cast<const float *>(h->in_mass.p);
    }
    if (!rc) rc = build_leaves_device(h, dpos, pos_type, dmass, s);
    h->last_stream = s;
    if (rc) {
        if (fresh) {
            free_leaves(h);
            delete h;
        }
        return rc;
    }
    h->valid = true;
    h->generation++;
    *leaves = h;
    return PH_OK;
}

static int read_status(const DevBuf &b, cudaStream_t s)
{
    uint32_t st = 0;
    int rc = cuda_check(cudaMemcpyAsync(&st, b.p, 4, cudaMemcpyDeviceToHost, s), "read status");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "status sync");
    if (rc) return rc;
    if (st & ST_NONFINITE) return fail(PH_ERR_NONFINITE, "non-finite position or mass");
    if (st & ST_CAPACITY) return fail(PH_ERR_CAPACITY, "pair list capacity exceeded");
    if (st & ST_TIMEOUT) return fail(PH_ERR_TIMEOUT, "bounded device wait gave up");
    return PH_OK;
}

}  // namespace phpp

using namespace phpp;

extern "C" {

int ph_build_leaves(const void *pos, int pos_type, const float *mass, int64_t n, const ph_params *params,
                    void *stream, ph_leaves **leaves)
{
    TraceRange trace_("ph_build_leaves");
    if (n < 0) return fail(PH_ERR_ARG, "n must be >= 0");
    int64_t off[2] = {0, n};
    return leaves_common(pos, pos_type, mass, off, 1, params, stream, leaves);
}

int ph_build_leaves_batched(const void *pos, int pos_type, const float *mass, const int64_t *box_offsets,
                            int32_t n_boxes, const ph_params *params, void *stream, ph_leaves **leaves)
{
    TraceRange trace_("ph_build_leaves_batched");
    if (!box_offsets) return fail(PH_ERR_ARG, "box_offsets must not be NULL");
    return leaves_common(pos, pos_type, mass, box_offsets, n_boxes, params, stream, leaves);
}

int ph_pairs_reserve(ph_pairs **pairs, int64_t capacity)
{
    if (!pairs || capacity < 0) return fail(PH_ERR_ARG, "bad arguments");
    ph_pairs *p = *pairs;
    if (p && p->kind != KIND_PAIRS) return fail(PH_ERR_STATE, "handle is not a ph_pairs");
    bool fresh = !p;
    if (fresh) {
        p = new (std::nothrow) ph_pairs();
        if (!p) return fail(PH_ERR_OOM, "host allocation failed");
    }
    // the entries may move: the list has to be built (again) before use
    p->valid = false;
    int rc = ensure(p->entries, (size_t)(capacity > 0 ? capacity : 1) * sizeof(float4));
    if (!rc) rc = ensure(p->ecount, (size_t)(capacity > 0 ? capacity : 1));
    if (rc) {
        if (fresh) {
            free_pairs(p);
            delete p;
        }
        return rc;
    }
    p->capacity = capacity;
    p->fixed_capacity = true;
    *pairs = p;
    return PH_OK;
}

int ph_leaf_pairs(ph_leaves *leaves, void *stream, ph_pairs **pairs)
{
    TraceRange trace_("ph_leaf_pairs");
    if (!leaves || leaves->kind != KIND_LEAVES) return fail(PH_ERR_STATE, "leaves is not a ph_leaves handle");
    if (!pairs) return fail(PH_ERR_ARG, "pairs must not be NULL");
    ph_pairs *p = *pairs;
    if (p && p->kind != KIND_PAIRS) return fail(PH_ERR_STATE, "handle is not a ph_pairs");
    int rc0 = check_built(leaves, nullptr);
    if (rc0) return rc0;
    bool fresh = !p;
    if (fresh) {
        p = new (std::nothrow) ph_pairs();
        if (!p) return fail(PH_ERR_OOM, "host allocation failed");
    }
    p->valid = false;   // until this list completes
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t N = (size_t)(leaves->n > 0 ? leaves->n : 1);
    int rc = 0;
    if (!rc) rc = ensure(p->group_cnt, 8 * (N + 1));
    if (!rc) rc = ensure(p->group_off, 8 * (N + 1));
    if (!rc) rc = ensure(p->work, 64);
    if (!rc) rc = ensure(p->temp, scan_temp_bytes((int64_t)N));
    if (!rc && leaves->queue_order == 0) {
        rc = ensure(p->group_key, N);
        if (!rc) rc = ensure(p->group_order, 4 * N);
        if (!rc) rc = ensure(p->order_temp, order_temp_bytes((int64_t)N));
    }
    if (!rc && !p->status.p) {
        rc = ensure(p->status, 16);
        if (!rc) rc = cuda_check(cudaMemsetAsync(p->status.p, 0, 16, s), "status reset");
    }
    if (!rc && !p->entries.p) {
        rc = ensure(p->entries, 16 * 1024);
        if (!rc) rc = ensure(p->ecount, 1024);
        if (!rc) p->capacity = 1024;
    }
    if (!rc) rc = build_pairs_device(leaves, p, s, !p->fixed_capacity);
    if (rc) {
        if (fresh) {
            free_pairs(p);
            delete p;
        }
        return rc;
    }
    p->built_from = leaves;
    p->leaves_generation = leaves->generation;
    p->valid = true;
    p->last_stream = s;
    *pairs = p;
    return PH_OK;
}

int ph_pp_accel(const ph_leaves *leaves, const ph_pairs *pairs, int g_mode, const ph_mlp *mlp, float *acc,
                void *stream)
{
    TraceRange trace_("ph_pp_accel");
    if (!leaves || leaves->kind != KIND_LEAVES) return fail(PH_ERR_STATE, "leaves is not a ph_leaves handle");
    if (pairs && pairs->kind != KIND_PAIRS) return fail(PH_ERR_STATE, "pairs is not a ph_pairs handle");
    if (pairs && pairs->built_from != leaves) return fail(PH_ERR_STATE, "pairs were not built from these leaves");
    {
        const int rb = check_built(leaves, pairs);
        if (rb) return rb;
    }
    if (g_mode != PH_G_EXACT && g_mode != PH_G_LEARNED && g_mode != PH_G_TABLE)
        return fail(PH_ERR_ARG, "unknown g_mode %d", g_mode);
    if (g_mode == PH_G_LEARNED && (!mlp || mlp->kind != KIND_MLP))
        return fail(PH_ERR_ARG, "PH_G_LEARNED needs a ph_mlp handle");
    if (g_mode != PH_G_EXACT && !pairs) return fail(PH_ERR_ARG, "the learned and tabulated factors need a pair list");
    if (!pairs && leaves->tree_leaves) return fail(PH_ERR_ARG, "the tree part (theta > 0) needs a pair list");
    if (leaves->n > 0 && !acc) return fail(PH_ERR_ARG, "acc must not be NULL");
    // the exact path judges the network: its validated error and the
    // rcut / rs it was trained for decide whether it may stand in
    bool use_learned = false;
    char why[160] = "";
    if (g_mode == PH_G_LEARNED) {
        use_learned = true;
        const double ratio = mlp->rcut / mlp->rs;
        for (int b = 0; b < leaves->n_boxes && use_learned; b++) {
            const BoxDev &bx = leaves->boxes_host[b];
            const double rb = std::sqrt((double)bx.rcut2) / std::sqrt(-1.4426950408889634 / (4.0 * (double)bx.c_e));
            if (std::fabs(rb / ratio - 1.0) > 1e-5) {
                use_learned = false;
                snprintf(why, sizeof why, "box %d has rcut/rs %.6g, the network was trained for %.6g", b, rb, ratio);
            }
        }
        if (use_learned && !(mlp->max_rel_err <= mlp->tol)) {
            use_learned = false;
            snprintf(why, sizeof why, "validated network error %.3e above its tolerance %.1e", mlp->max_rel_err,
                     mlp->tol);
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ph_pairs *pr = const_cast<ph_pairs *>(pairs);
    ph_leaves *lvm = const_cast<ph_leaves *>(leaves);
    if (leaves->n == 0) return PH_OK;
    const bool dev = is_device_ptr(acc);
    float *dacc = acc;
    int rc = 0;
    if (!dev) {
        DevBuf &tmp = pr ? pr->acc_tmp : lvm->acc_tmp;
        rc = ensure(tmp, (size_t)leaves->n * 12);
        if (rc) return rc;
        dacc = static_cast<float *>(tmp.p);
    }
    if (g_mode == PH_G_TABLE) {
        rc = ensure_table(lvm, s);
        if (!rc) rc = pp_table_device(leaves, pairs, dacc, s);
    } else {
        rc = use_learned ? pp_learned_device(leaves, pairs, static_cast<const float *>(mlp->theta.p), dacc, s)
                         : pp_exact_device(leaves, pairs, dacc, s);
    }
    if (!rc && !dev)
        rc = cuda_check(cudaMemcpyAsync(acc, dacc, (size_t)leaves->n * 12, cudaMemcpyDeviceToHost, s), "copy acc");
    if (pr) pr->last_stream = s;
    else lvm->last_stream = s;
    if (!rc && g_mode == PH_G_LEARNED && !use_learned) return fail(PH_WARN_FALLBACK, "exact factor used: %s", why);
    return rc;
}

int ph_accel(const void *pos, int pos_type, const float *mass, int64_t n, const ph_params *params, int g_mode,
             const ph_mlp *mlp, float *acc, void *stream, ph_leaves **leaves, ph_pairs **pairs)
{
    TraceRange trace_("ph_accel");
    if (!leaves) return fail(PH_ERR_ARG, "leaves must not be NULL");
    int rc = ph_build_leaves(pos, pos_type, mass, n, params, stream, leaves);
    if (rc) return rc;
    if (!pairs) return ph_pp_accel(*leaves, nullptr, g_mode, mlp, acc, stream);   // direct mode
    rc = ph_leaf_pairs(*leaves, stream, pairs);
    if (rc) return rc;
    return ph_pp_accel(*leaves, *pairs, g_mode, mlp, acc, stream);
}

void ph_free(void *handle)
{
    if (!handle) return;
    uint32_t kind = *static_cast<uint32_t *>(handle);
    if (kind == KIND_LEAVES) {
        ph_leaves *h = static_cast<ph_leaves *>(handle);
        free_leaves(h);
        delete h;
    } else if (kind == KIND_PAIRS) {
        ph_pairs *h = static_cast<ph_pairs *>(handle);
        free_pairs(h);
        delete h;
    } else if (kind == KIND_MLP) {
        mlp_free(static_cast<ph_mlp *>(handle));
    } else if (kind == KIND_GRAPH) {
        graph_free(static_cast<ph_graph *>(handle));
    } else if (kind == KIND_PM) {
        pm_free(static_cast<ph_pm *>(handle));
    } else if (kind == KIND_SIM) {
        sim_free(static_cast<ph_sim *>(handle));
    }
}

const char *ph_last_error(void) { return g_err; }

int ph_status(const void *handle)
{
    if (!handle) return fail(PH_ERR_ARG, "NULL handle");
    uint32_t kind = *static_cast<const uint32_t *>(handle);
    if (kind == KIND_LEAVES) {
        const ph_leaves *h = static_cast<const ph_leaves *>(handle);
        return read_status(h->status, h->last_stream);
    }
    if (kind == KIND_PAIRS) {
        const ph_pairs *h = static_cast<const ph_pairs *>(handle);
        return read_status(h->status, h->last_stream);
    }
    if (kind == KIND_PM) return pm_status(static_cast<const ph_pm *>(handle));
    if (kind == KIND_SIM) return ph_sim_get(static_cast<const ph_sim *>(handle), nullptr, nullptr, nullptr, nullptr,
                                            nullptr, nullptr);
    if (kind == KIND_MLP || kind == KIND_GRAPH) return PH_OK;
    return fail(PH_ERR_STATE, "unknown handle");
}

int ph_leaves_get_view(const ph_leaves *h, ph_leaves_view *out)
{
    if (!h || h->kind != KIND_LEAVES || !out) return fail(PH_ERR_ARG, "bad arguments");
    {
        const int rb = check_built(h, nullptr);
        if (rb) return rb;
    }
    int32_t cnt[2] = {0, 0};
    int rc = cuda_check(cudaMemcpyAsync(cnt, h->counts.p, 8, cudaMemcpyDeviceToHost, h->last_stream), "read counts");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(h->last_stream), "view sync");
    if (rc) return rc;
    memset(out, 0, sizeof *out);
    out->n = h->n;
    out->n_boxes = h->n_boxes;
    out->n_leaves = cnt[0];
    out->n_groups = cnt[1];
    out->n_cells = h->n_cells;
    out->keys = static_cast<const uint64_t *>(h->keys_in_alt ? h->keys_alt.p : h->keys.p);
    out->perm = static_cast<const int32_t *>(h->keys_in_alt ? h->vals_alt.p : h->vals.p);
    out->leaf_first = static_cast<const int32_t *>(h->leaf_first.p);
    out->leaf_ref = static_cast<const double *>(h->leaf_ref.p);
    out->leaf_half = static_cast<const float *>(h->leaf_h4.p);
    out->group_first = static_cast<const int32_t *>(h->group_first.p);
    out->group_ref = static_cast<const double *>(h->group_ref.p);
    out->group_half = static_cast<const float *>(h->group_h4.p);
    out->pos_leaf = static_cast<const float *>(h->pos_leaf.p);
    out->pos_group = static_cast<const float *>(h->pos_group.p);
    out->cell_leaf_first = static_cast<const int32_t *>(h->cell_leaf_first.p);
    for (int b = 0; b < 4 && b < h->n_boxes; b++) out->g[b] = h->boxes_host[b].g;
    out->key_bits = h->key_bits;
    out->group_size = h->group_size;
    return PH_OK;
}

int ph_pairs_get_view(const ph_pairs *p, ph_pairs_view *out)
{
    if (!p || p->kind != KIND_PAIRS || !out || !p->built_from) return fail(PH_ERR_ARG, "bad arguments");
    const ph_leaves *lv = p->built_from;
    {
        const int rb = check_built(lv, p);
        if (rb) return rb;
    }
    int32_t ng = 0;
    int rc = cuda_check(cudaMemcpyAsync(&ng, static_cast<const int32_t *>(lv->counts.p) + 1, 4,
                                        cudaMemcpyDeviceToHost, p->last_stream),
                        "read groups");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(p->last_stream), "view sync");
    int64_t total = 0;
    if (!rc)
        rc = cuda_check(cudaMemcpyAsync(&total, static_cast<const int64_t *>(p->group_off.p) + ng, 8,
                                        cudaMemcpyDeviceToHost, p->last_stream),
                        "read total");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(p->last_stream), "view sync");
    if (rc) return rc;
    memset(out, 0, sizeof *out);
    out->n_pairs = total;
    out->n_groups = ng;
    out->group_off = static_cast<const int64_t *>(p->group_off.p);
    out->entries = static_cast<const float *>(p->entries.p);
    out->counts = static_cast<const uint8_t *>(p->ecount.p);
    out->group_order = p->ordered ? static_cast<const int32_t *>(p->group_order.p) : nullptr;
    return PH_OK;
}

int ph_count_within(const ph_leaves *leaves, const ph_pairs *pairs, int64_t *n_within, void *stream)
{
    TraceRange trace_("ph_count_within");
    if (!leaves || leaves->kind != KIND_LEAVES || !pairs || pairs->kind != KIND_PAIRS || !n_within)
        return fail(PH_ERR_ARG, "bad arguments");
    if (pairs->built_from != leaves) return fail(PH_ERR_STATE, "pairs were not built from these leaves");
    {
        const int rb = check_built(leaves, pairs);
        if (rb) return rb;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    *n_within = 0;
    if (leaves->n == 0) return PH_OK;
    ph_pairs *pr = const_cast<ph_pairs *>(pairs);
    int rc = count_within_device(leaves, pairs, s);
    unsigned long long v = 0;
    if (!rc)
        rc = cuda_check(cudaMemcpyAsync(&v, static_cast<char *>(pr->work.p) + 8, 8, cudaMemcpyDeviceToHost, s),
                        "read count");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "count sync");
    if (rc) return rc;
    *n_within = (int64_t)v;
    pr->last_stream = s;
    return PH_OK;
}

int64_t ph_launch_counter(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

void ph_debug_fail_allocation(int64_t k) { g_fail_after.store(k < 0 ? -1 : (long long)k); }

int ph_debug_bounds(int64_t *hits, int32_t *first_site)
{
    if (!hits || !first_site) return fail(PH_ERR_ARG, "ph_debug_bounds: null output");
    *hits = 0;
    *first_site = 0;
#ifndef PHPP_BOUNDS_CHECK
    return fail(PH_ERR_STATE, "library built without bounds checks");
#else
    int rc = cuda_check(cudaDeviceSynchronize(), "bounds sync");
    if (rc) return rc;
    for (auto read : bounds_readers()) {
        unsigned int h = 0, site = 0;
        if (read(&h, &site)) return fail(PH_ERR_CUDA, "reading the bounds words failed");
        *hits += h;
        if (!*first_site && site) *first_site = (int32_t)site;
    }
    return PH_OK;
#endif
}

int ph_leaves_set_active(ph_leaves *leaves, const uint8_t *d_active, int64_t n)
{
    if (!leaves || leaves->kind != KIND_LEAVES) return fail(PH_ERR_STATE, "leaves is not a ph_leaves handle");
    if (!d_active) {
        leaves->active = nullptr;
        return PH_OK;
    }
    if (n < 0 || !is_device_ptr(d_active)) return fail(PH_ERR_ARG, "active flags must be device memory, n >= 0");
    // the group flags, their scan and the list, for builds of up to n particles
    // (a build of more particles grows them)
    const size_t N = (size_t)(n > 0 ? n : 1);
    int rc = ensure(leaves->group_act, 4 * (N + 1));
    if (!rc) rc = ensure(leaves->group_act_scan, 4 * (N + 1));
    if (!rc) rc = ensure(leaves->active_list, 4 * N);
    if (rc) {
        leaves->active = nullptr;
        return rc;
    }
    leaves->active = d_active;
    return PH_OK;
}

int ph_pp_counters(const void *handle, int64_t *interactions, int64_t *staged)
{
    if (!handle) return fail(PH_ERR_ARG, "bad arguments");
    const uint32_t kind = *static_cast<const uint32_t *>(handle);
    const void *work = nullptr;
    cudaStream_t st = nullptr;
    if (kind == KIND_PAIRS) {
        const ph_pairs *p = static_cast<const ph_pairs *>(handle);
        work = p->work.p;
        st = p->last_stream;
    } else if (kind == KIND_LEAVES) {
        const ph_leaves *l = static_cast<const ph_leaves *>(handle);
        work = l->work.p;
        st = l->last_stream;
    } else {
        return fail(PH_ERR_ARG, "not a pairs or leaves handle");
    }
    unsigned long long v[3] = {0, 0, 0};
    if (!work) return fail(PH_ERR_STATE, "no PP work recorded on this handle");
    int rc = cuda_check(cudaMemcpyAsync(v, work, 24, cudaMemcpyDeviceToHost, st), "read counters");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "counter sync");
    if (rc) return rc;
    if (interactions) *interactions = (int64_t)v[1];
    if (staged) *staged = (int64_t)v[2];
    return PH_OK;
}

}  // extern "C"
