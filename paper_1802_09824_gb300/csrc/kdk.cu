// Adaptive Kick-Drift-Kick block steps (Sec. 3.4) driving the force calls.
//
// Drift x += p D(t1; t2), Kick p += a K(t1; t2) with D = int dt / a^2 and
// K = int dt / a (Newtonian clock: both t2 - t1).  One top step of length dt
// is an integer timeline of T = 2^max_level ticks; a particle on level k
// has steps of T / 2^k ticks, its level the smallest k with
// (dt_phys / 2^k)^2 |a| <= 2 eta eps (t_acc = sqrt(2 eta eps / |a|), the
// step halved until it fits).  Per top step: levels and opening half kicks
// for all; then per event (the earliest end of any step): drift all to it,
// one force pass (short-range PP + long-range PM), closing half kicks of the
// particles whose step ends, and (before the top step's end) their new
// levels, refined until aligned with the elapsed ticks, and opening half
// kicks.  State in FP64 (positions kept in [0, L)); the criterion and the
// kicks/drifts use FP64 with fixed roundings (no contraction), the same
// operations as the FP64 oracle's.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "handles.cuh"

struct ph_sim {
    uint32_t kind = phpp::KIND_SIM;
    cudaStream_t last_stream = nullptr;
    int64_t n = 0;
    ph_params prm{};
    ph_kdk_params kp{};
    double t = 0.0;
    int64_t force_passes = 0;
    bool has_mass = false;
    phpp::DevBuf x, p, mass, acc, level, start, next;
    phpp::DevBuf act;             // uint8[n]: particles whose step ends at the next event
    ph_leaves *lv = nullptr;
    ph_pairs *pr = nullptr;
    ph_pm *pm = nullptr;
    ph_graph *graph = nullptr;    // build + pairs + PP captured once (fixed pair capacity)
};

namespace phpp {

namespace {

constexpr int kSimThreads = 256;
constexpr int kMaxLevel = 20;

struct KickArgs {
    double k_open[kMaxLevel + 1];    // K(t_tick; t_tick + dt_k / 2)
    double k_close[kMaxLevel + 1];   // K(t_tick - dt_k / 2; t_tick)
    double dt_crit;                  // top step in physical time units
    double thr;                      // 2 eta eps
    int32_t tick, T, max_level, first, last;
};

inline int grid_of(int64_t n)
{
    int64_t b = (n + kSimThreads - 1) / kSimThreads;
    const int64_t cap = (int64_t)sm_count() * 16;
    if (b > cap) b = cap;
    return (int)(b > 0 ? b : 1);
}

__device__ __forceinline__ int level_of(float ax, float ay, float az, double dt, double thr, int kmax)
{
    const double a0 = ax, a1 = ay, a2 = az;
    const double amag = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(a0, a0), __dmul_rn(a1, a1)), __dmul_rn(a2, a2)));
    double lhs = __dmul_rn(__dmul_rn(dt, dt), amag);
    int k = 0;
    while (k < kmax && lhs > thr) {
        lhs = __dmul_rn(lhs, 0.25);
        k++;
    }
    return k;
}

// guard: the pair list's status word; when the force pass overflowed the
// list (its accelerations are incomplete) the kick does nothing, so the host
// can rebuild the list, redo the force pass and launch the kick again.
__global__ void k_sim_kick(int64_t n, const float *acc, double *p, int32_t *level, int32_t *start, int32_t *next,
                           const uint32_t *guard, KickArgs ka)
{
    if (guard && (*guard & ST_CAPACITY)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float ax = acc[3 * i], ay = acc[3 * i + 1], az = acc[3 * i + 2];
        const double a[3] = {ax, ay, az};
        int k = level[i];
        int s = start[i];
        bool open = false;
        if (ka.first) {
            k = level_of(ax, ay, az, ka.dt_crit, ka.thr, ka.max_level);
            s = 0;
            open = true;
        } else if (s + (ka.T >> k) == ka.tick) {
            const double kc = ka.k_close[k];
#pragma unroll
            for (int c = 0; c < 3; c++) p[3 * i + c] = __dadd_rn(p[3 * i + c], __dmul_rn(a[c], kc));
            if (!ka.last) {
                k = level_of(ax, ay, az, ka.dt_crit, ka.thr, ka.max_level);
                while (ka.tick % (ka.T >> k)) k++;
                s = ka.tick;
                open = true;
            }
        }
        if (open) {
            const double ko = ka.k_open[k];
#pragma unroll
            for (int c = 0; c < 3; c++) p[3 * i + c] = __dadd_rn(p[3 * i + c], __dmul_rn(a[c], ko));
            level[i] = k;
            start[i] = s;
        }
        if (!ka.last) atomicMin(next, s + (ka.T >> k));
    }
}

// The particles whose step ends at the next event (the tick the kick just
// found): the only ones whose forces the next force pass must compute.  Like
// the kick, it does nothing after a pair-list overflow (the flags of the
// event to redo stay as they are).
__global__ void k_sim_active(int64_t n, const int32_t *level, const int32_t *start, const int32_t *next, int T,
                             const uint32_t *guard, uint8_t *act)
{
    if (guard && (*guard & ST_CAPACITY)) return;
    const int t = *next;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        act[i] = start[i] + (T >> level[i]) == t ? 1 : 0;
}

__global__ void k_sim_drift(int64_t n, double *x, const double *p, double D, double L)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = __dadd_rn(x[i], __dmul_rn(p[i], D));
        if (!(v >= 0.0 && v < L)) {
            v = __dsub_rn(v, __dmul_rn(L, floor(__ddiv_rn(v, L))));
            if (v >= L) v = 0.0;
        }
        x[i] = v;
    }
}

// ---------------------------------------------------------------- clocks (host)
// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_m).
struct GaussLegendre {
    static constexpr int M = 24;
    double x[M], w[M];
    GaussLegendre()
    {
        for (int i = 0; i < M; i++) {
            double z = std::cos(M_PI * (i + 0.75) / (M + 0.5)), pp = 0.0;
            for (int it = 0; it < 100; it++) {
                double p1 = 1.0, p2 = 0.0;
                for (int j = 1; j <= M; j++) {
                    const double p3 = p2;
                    p2 = p1;
                    p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
                }
                pp = M * (z * p1 - p2) / (z * z - 1.0);
                const double dz = p1 / pp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) break;
            }
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
        }
    }
};

double hubble(const ph_kdk_params &k, double a) { return k.H0 * std::sqrt(k.omega_m / (a * a * a) + k.omega_l); }

// int_{a1}^{a2} da / (a^power H(a)): composite Gauss-Legendre, 8 panels.
double clock_integral(const ph_kdk_params &k, double a1, double a2, int power)
{
    static const GaussLegendre gl;
    const int panels = 8;
    const double hp = (a2 - a1) / panels;
    double s = 0.0;
    for (int q = 0; q < panels; q++) {
        const double lo = a1 + q * hp, mid = lo + 0.5 * hp;
        for (int i = 0; i < GaussLegendre::M; i++) {
            const double a = mid + 0.5 * hp * gl.x[i];
            s += gl.w[i] * 0.5 * hp / (std::pow(a, power) * hubble(k, a));
        }
    }
    return s;
}

double drift_factor(const ph_kdk_params &k, double t1, double t2)
{
    if (k.clock == PH_CLOCK_NEWTON || t1 == t2) return t2 - t1;
    return clock_integral(k, t1, t2, 3);
}

double kick_factor(const ph_kdk_params &k, double t1, double t2)
{
    if (k.clock == PH_CLOCK_NEWTON || t1 == t2) return t2 - t1;
    return clock_integral(k, t1, t2, 2);
}

double step_scale(const ph_kdk_params &k, double t) { return k.clock == PH_CLOCK_NEWTON ? 1.0 : t * hubble(k, t); }

void sim_release(ph_sim *h)
{
    if (h->graph) ph_free(h->graph);
    h->graph = nullptr;
    if (h->pm) ph_free(h->pm);
    if (h->pr) ph_free(h->pr);
    if (h->lv) ph_free(h->lv);
    h->pm = nullptr;
    h->pr = nullptr;
    h->lv = nullptr;
    DevBuf *bufs[] = {&h->x, &h->p, &h->mass, &h->acc, &h->level, &h->start, &h->next, &h->act};
    for (DevBuf *b : bufs) release(*b);
}

// The long-range part added onto the short-range accelerations.
int add_pm(ph_sim *h, cudaStream_t s)
{
    if (h->kp.n_mesh <= 0) return PH_OK;
    const float *m = h->has_mass ? static_cast<const float *>(h->mass.p) : nullptr;
    const int rc = ph_pm_accel(h->x.p, PH_F64, m, h->n, &h->prm, h->kp.n_mesh, static_cast<float *>(h->acc.p),
                               nullptr, 1, s, &h->pm);
    return rc < 0 ? rc : PH_OK;
}

// From now on the force passes compute forces for the active particles
// only (Sec. 3.4: a particle's force is needed at the end of its own step):
// the build lists the groups holding an active particle, the pair builder
// lists sources for those groups only (the PP kernel passes over the others
// and writes zeros for them), PM interpolates active particles only.  The
// kicks read the accelerations of active particles only; at the end of a
// top step every particle is active.
int enable_active(ph_sim *h)
{
    if (!h->lv) return PH_OK;
    const size_t N = (size_t)h->n;
    int rc = ensure(h->lv->group_act, 4 * (N + 1));
    if (!rc) rc = ensure(h->lv->group_act_scan, 4 * (N + 1));
    if (!rc) rc = ensure(h->lv->active_list, 4 * N);
    if (rc) return rc;
    h->lv->active = static_cast<const uint8_t *>(h->act.p);
    if (h->pm) pm_set_active(h->pm, static_cast<const uint8_t *>(h->act.p));
    return PH_OK;
}

// A full force pass with sizing (host synchronisations): build, a pair list
// sized for the current positions, PP, PM; then the build, pairs and PP are
// captured as one graph with a fixed pair capacity (25 % headroom) for the
// following passes.
int force_pass_sized(ph_sim *h, cudaStream_t s)
{
    const float *m = h->has_mass ? static_cast<const float *>(h->mass.p) : nullptr;
    float *acc = static_cast<float *>(h->acc.p);
    if (h->graph) {
        ph_free(h->graph);
        h->graph = nullptr;
    }
    int rc = PH_OK;
    if (h->pr) {
        h->pr->fixed_capacity = false;           // let the list be sized again
        rc = cuda_check(cudaMemsetAsync(h->pr->status.p, 0, 4, s), "clear the overflow");
        if (rc) return rc;
    }
    rc = ph_accel(h->x.p, PH_F64, m, h->n, &h->prm, h->kp.g_mode, nullptr, acc, s, &h->lv, &h->pr);
    if (rc < 0) return rc;
    rc = add_pm(h, s);
    if (!rc) rc = enable_active(h);
    if (rc) return rc;
    rc = ph_graph_create(h->lv, h->pr, h->x.p, PH_F64, m, h->kp.g_mode, nullptr, acc, 0.25, s, &h->graph);
    return rc < 0 ? rc : PH_OK;
}

// One force pass at the current positions: the captured build + pairs + PP
// (no host synchronisation) then PM added.  A pair list that outgrew its
// capacity is latched in its status word, which the kick checks.
int force_pass(ph_sim *h, cudaStream_t s)
{
    int rc;
    if (h->graph) {
        rc = ph_graph_launch(h->graph, s);
        if (!rc) rc = add_pm(h, s);
    } else {
        rc = force_pass_sized(h, s);
    }
    if (!rc) h->force_passes++;
    return rc;
}

// The kicks of one event, guarded by the pair list's status; reads back the
// next event tick and the status with one synchronisation.  After an
// overflow (the guarded kick did nothing) the force pass is redone with a
// list sized afresh and the kick launched again.
int launch_kick(ph_sim *h, const KickArgs &ka, cudaStream_t s, int32_t *next_host)
{
    int32_t *nx = static_cast<int32_t *>(h->next.p);
    for (int attempt = 0; attempt < 2; attempt++) {
        const uint32_t *guard = h->pr ? static_cast<const uint32_t *>(h->pr->status.p) : nullptr;
        int rc = cuda_check(cudaMemsetAsync(nx, 0x7f, 4, s), "reset event");
        if (rc) return rc;
        k_sim_kick<<<grid_of(h->n), kSimThreads, 0, s>>>(h->n, static_cast<const float *>(h->acc.p),
                                                        static_cast<double *>(h->p.p),
                                                        static_cast<int32_t *>(h->level.p),
                                                        static_cast<int32_t *>(h->start.p), nx, guard, ka);
        count_launch();
        if (!ka.last) {
            k_sim_active<<<grid_of(h->n), kSimThreads, 0, s>>>(h->n, static_cast<const int32_t *>(h->level.p),
                                                              static_cast<const int32_t *>(h->start.p), nx, ka.T,
                                                              guard, static_cast<uint8_t *>(h->act.p));
            count_launch();
        }
        rc = cuda_check(cudaGetLastError(), "kick kernel");
        uint32_t st = 0;
        if (!rc) rc = cuda_check(cudaMemcpyAsync(next_host, nx, 4, cudaMemcpyDeviceToHost, s), "read event");
        if (!rc && guard) rc = cuda_check(cudaMemcpyAsync(&st, guard, 4, cudaMemcpyDeviceToHost, s), "read status");
        if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "event sync");
        if (rc) return rc;
        if (!(st & ST_CAPACITY)) return PH_OK;
        rc = force_pass_sized(h, s);     // the kick above did nothing: redo the pass, then kick
        if (rc) return rc;
    }
    return fail(PH_ERR_CAPACITY, "pair list overflow persisted after resizing");
}

int top_step(ph_sim *h, cudaStream_t s)
{
    const ph_kdk_params &kp = h->kp;
    const int kmax = kp.max_level;
    const int T = 1 << kmax;
    const double h_tick = kp.dt / T;
    const double t0 = h->t;
    auto tt = [&](double tick) { return t0 + tick * h_tick; };
    const double eps = kp.eps_step > 0 ? kp.eps_step : h->prm.eps;
    KickArgs ka;
    memset(&ka, 0, sizeof ka);
    ka.T = T;
    ka.max_level = kmax;
    ka.thr = 2.0 * kp.eta * eps;
    ka.first = 1;
    ka.dt_crit = kp.dt / step_scale(kp, t0);
    for (int k = 0; k <= kmax; k++) ka.k_open[k] = kick_factor(kp, t0, tt((double)(T >> k) / 2.0));
    int32_t nxt = 0;
    int rc = launch_kick(h, ka, s, &nxt);
    int tick = 0;
    while (!rc && tick < T) {
        if (nxt <= tick || nxt > T) return fail(PH_ERR_STATE, "event tick %d after %d out of range", nxt, tick);
        k_sim_drift<<<grid_of(3 * h->n), kSimThreads, 0, s>>>(h->n, static_cast<double *>(h->x.p),
                                                             static_cast<const double *>(h->p.p),
                                                             drift_factor(kp, tt(tick), tt(nxt)), h->prm.L);
        count_launch();
        tick = nxt;
        rc = cuda_check(cudaGetLastError(), "drift kernel");
        if (!rc) rc = force_pass(h, s);
        if (rc) break;
        ka.first = 0;
        ka.tick = tick;
        ka.last = tick == T;
        ka.dt_crit = kp.dt / step_scale(kp, tt(tick));
        for (int k = 0; k <= kmax; k++) {
            const double half = (double)(T >> k) / 2.0;
            ka.k_close[k] = kick_factor(kp, tt((double)tick - half), tt(tick));
            ka.k_open[k] = kick_factor(kp, tt(tick), tt((double)tick + half));
        }
        rc = launch_kick(h, ka, s, &nxt);
    }
    if (!rc) h->t = t0 + kp.dt;
    return rc;
}

}  // namespace

void sim_free(ph_sim *h)
{
    sim_release(h);
    delete h;
}

}  // namespace phpp

using namespace phpp;

extern "C" {

int ph_sim_create(const double *pos, const double *mom, const float *mass, int64_t n, const ph_params *params,
                  const ph_kdk_params *kp, double t0, void *stream, ph_sim **sim)
{
    TraceRange trace_("ph_sim_create");
    if (!sim || !params || !kp || !pos || !mom) return fail(PH_ERR_ARG, "sim, params, kp, pos and mom must not be NULL");
    if (*sim) return fail(PH_ERR_STATE, "*sim must be NULL (a new simulation)");
    if (n < 1 || n >= (int64_t)1 << 31) return fail(PH_ERR_ARG, "n must be 1..2^31-1");
    if (!(std::isfinite(kp->dt) && kp->dt > 0)) return fail(PH_ERR_ARG, "dt must be > 0");
    if (!(std::isfinite(kp->eta) && kp->eta > 0)) return fail(PH_ERR_ARG, "eta must be > 0");
    if (!(std::isfinite(kp->eps_step) && kp->eps_step >= 0)) return fail(PH_ERR_ARG, "eps_step must be >= 0");
    if (kp->eps_step == 0 && !(params->eps > 0)) return fail(PH_ERR_ARG, "the criterion needs eps_step or eps > 0");
    if (kp->max_level < 0 || kp->max_level > kMaxLevel) return fail(PH_ERR_ARG, "max_level must be 0..%d", kMaxLevel);
    if (kp->n_mesh != 0 && (kp->n_mesh < 4 || kp->n_mesh > PH_PM_MAX_MESH || (kp->n_mesh & 1)))
        return fail(PH_ERR_ARG, "n_mesh must be 0 or even in 4..%d", PH_PM_MAX_MESH);
    if (kp->clock != PH_CLOCK_NEWTON && kp->clock != PH_CLOCK_LCDM) return fail(PH_ERR_ARG, "unknown clock");
    if (kp->clock == PH_CLOCK_LCDM &&
        !(kp->H0 > 0 && kp->omega_m > 0 && kp->omega_l >= 0 && t0 > 0 && std::isfinite(t0)))
        return fail(PH_ERR_ARG, "the Lambda-CDM clock needs H0 > 0, omega_m > 0, omega_l >= 0 and a0 > 0");
    if (kp->g_mode != PH_G_EXACT && kp->g_mode != PH_G_TABLE) return fail(PH_ERR_ARG, "g_mode must be exact or table");
    ph_sim *h = new (std::nothrow) ph_sim();
    if (!h) return fail(PH_ERR_OOM, "host allocation failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->n = n;
    h->prm = *params;
    h->kp = *kp;
    h->t = t0;
    h->has_mass = mass != nullptr;
    h->last_stream = s;
    const size_t N = (size_t)n;
    int rc = ensure(h->x, 24 * N);
    if (!rc) rc = ensure(h->p, 24 * N);
    if (!rc && mass) rc = ensure(h->mass, 4 * N);
    if (!rc) rc = ensure(h->acc, 12 * N);
    if (!rc) rc = ensure(h->level, 4 * N);
    if (!rc) rc = ensure(h->start, 4 * N);
    if (!rc) rc = ensure(h->next, 16);
    if (!rc) rc = ensure(h->act, N);
    const cudaMemcpyKind kind = cudaMemcpyDefault;
    if (!rc) rc = cuda_check(cudaMemcpyAsync(h->x.p, pos, 24 * N, kind, s), "copy positions");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(h->p.p, mom, 24 * N, kind, s), "copy momenta");
    if (!rc && mass) rc = cuda_check(cudaMemcpyAsync(h->mass.p, mass, 4 * N, kind, s), "copy masses");
    if (!rc) rc = cuda_check(cudaMemsetAsync(h->level.p, 0, 4 * N, s), "clear levels");
    if (!rc) rc = cuda_check(cudaMemsetAsync(h->start.p, 0, 4 * N, s), "clear starts");
    if (!rc) {
        // positions into [0, L) as the drift keeps them
        k_sim_drift<<<grid_of(3 * h->n), kSimThreads, 0, s>>>(h->n, static_cast<double *>(h->x.p),
                                                             static_cast<const double *>(h->p.p), 0.0, h->prm.L);
        count_launch();
        rc = cuda_check(cudaGetLastError(), "wrap kernel");
    }
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "create sync");
    if (!rc) rc = force_pass_sized(h, s);
    if (!rc) h->force_passes++;
    if (rc) {
        sim_free(h);
        return rc;
    }
    *sim = h;
    return PH_OK;
}

int ph_sim_step(ph_sim *sim, int32_t n_steps, void *stream)
{
    TraceRange trace_("ph_sim_step");
    if (!sim || sim->kind != KIND_SIM || n_steps < 0) return fail(PH_ERR_ARG, "bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    sim->last_stream = s;
    for (int k = 0; k < n_steps; k++) {
        int rc = top_step(sim, s);
        if (rc) return rc;
    }
    return PH_OK;
}

int ph_sim_get(const ph_sim *sim, double *pos, double *mom, float *acc, int32_t *level, double *t,
               int64_t *force_passes)
{
    if (!sim || sim->kind != KIND_SIM) return fail(PH_ERR_ARG, "not a ph_sim handle");
    cudaStream_t s = sim->last_stream;
    const size_t N = (size_t)sim->n;
    int rc = PH_OK;
    if (pos) rc = cuda_check(cudaMemcpyAsync(pos, sim->x.p, 24 * N, cudaMemcpyDefault, s), "read positions");
    if (!rc && mom) rc = cuda_check(cudaMemcpyAsync(mom, sim->p.p, 24 * N, cudaMemcpyDefault, s), "read momenta");
    if (!rc && acc) rc = cuda_check(cudaMemcpyAsync(acc, sim->acc.p, 12 * N, cudaMemcpyDefault, s), "read acc");
    if (!rc && level) rc = cuda_check(cudaMemcpyAsync(level, sim->level.p, 4 * N, cudaMemcpyDefault, s), "read levels");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "get sync");
    if (rc) return rc;
    if (t) *t = sim->t;
    if (force_passes) *force_passes = sim->force_passes;
    if (sim->lv) {
        rc = ph_status(sim->lv);
        if (!rc && sim->pr) rc = ph_status(sim->pr);
        if (!rc && sim->pm) rc = ph_status(sim->pm);
    }
    return rc;
}

}  // extern "C"
