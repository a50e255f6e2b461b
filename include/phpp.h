/*
 * phpp -- short-range particle-particle (PP) gravity on one GB300 GPU.
 *
 * C ABI of the library libphpp.so.  The operation is the short-range part of
 * the PM-Tree-PP force split of PHoTo"N"s (arXiv:1802.09824):
 *
 *   a_i = G sum_{j != i, r_ij < rcut} m_j d_ij f(r_ij) / (r_ij^2 + eps^2)^{3/2}
 *   f(s) = erfc(s / 2R_s) + s / (R_s sqrt(pi)) exp(-s^2 / 4R_s^2)
 *
 * f is the short-range factor of Eq. (split) (Sec. 3.1); R_cut is the radius
 * beyond which the short-range force is dropped (Sec. 3.1, R_cut = 4.5 R_s);
 * d_ij is the minimum-image separation in a periodic box of side L; eps is a
 * Plummer softening that enters the Newtonian factor only (f is taken at the
 * unsoftened r).  The sum is organised as in Sec. 3.2-3.3 and Sec. 4.3:
 * particles are sorted along a space-filling curve inside a ground grid whose
 * cells are at least R_cut wide, cut into octree leaves, and each group of
 * target particles sums directly over the leaves of its own and the 26
 * neighbouring ground cells that lie within R_cut (leaf-leaf PP).
 *
 * Conventions for every call
 *  - Return value: PH_OK (0), a positive warning, or a negative PH_ERR_*.
 *    On error ph_last_error() gives a message (thread-local, valid until the
 *    next call on the same thread).
 *  - All work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *    stream) and is asynchronous unless stated otherwise.
 *  - Pointers named d_* must be device memory.  Pointers documented as
 *    "host or device" are classified with cudaPointerGetAttributes: device
 *    (or managed) memory is used in place; host memory is copied through a
 *    device buffer owned by the handle on the same stream, and such a call
 *    returns only after the copies it needs have been issued (pageable host
 *    memory makes the copy synchronous).  Host buffers must stay valid until
 *    the stream has executed the call.
 *  - Handles (ph_leaves, ph_pairs, ph_mlp) own their device memory until
 *    ph_free().  A handle pointer passed in non-NULL is rebuilt in place,
 *    reusing its buffers when they are large enough.
 *  - Device-side faults that do not corrupt memory (capacity overflow, a
 *    non-finite input) are latched in a word inside the handle and reported
 *    by ph_status() and by the next call that synchronises.
 */
#ifndef PHPP_H
#define PHPP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define PH_OK                   0
#define PH_WARN_FALLBACK        1   /* learned factor rejected; exact path used */
#define PH_ERR_ARG             -1   /* bad argument (NULL, size, range)          */
#define PH_ERR_RCUT_GE_HALF_L  -2   /* rcut >= L/2: minimum image not unique     */
#define PH_ERR_NONFINITE       -3   /* NaN/Inf in positions or masses            */
#define PH_ERR_OOM             -4   /* device allocation failed                  */
#define PH_ERR_CUDA            -5   /* a CUDA runtime call failed                */
#define PH_ERR_CAPACITY        -6   /* a fixed-capacity buffer overflowed        */
#define PH_ERR_TIMEOUT         -7   /* a bounded device wait gave up             */
#define PH_ERR_STATE           -8   /* handle in the wrong state / wrong type    */

/* element type of a position array */
#define PH_F32 0
#define PH_F64 1

/* ordering of particles inside a ground cell */
#define PH_KEY_MORTON   0   /* Morton order (Sec. 3.2)                         */
#define PH_KEY_HILBERT  1   /* Peano-Hilbert order (the curve of Sec. 4.1)     */

/* how the short-range factor f is evaluated in the PP kernel */
#define PH_G_EXACT    0     /* Eq. (split), FP32 with SFU exp/rsqrt             */
#define PH_G_LEARNED  1     /* the 1-16-16-1 SiLU network of a ph_mlp           */
#define PH_G_TABLE    2     /* Eq. (split) tabulated at 4097 nodes in r (the
                               pre-computed table of Sec. 3.1): nearest node
                               plus its slope; one rcut and rs for all boxes */

/*
 * Parameters of one periodic box.
 *   L         box side (> 0); positions may lie anywhere, they are wrapped.
 *   G         gravitational constant.
 *   eps       Plummer softening (>= 0).  The exact kernel evaluates
 *             (r^2 + eps^2)^(-3/2) in units where rcut is ~1 and floors the
 *             scaled eps^2 at 1e-12 (so that no FP32 intermediate of a
 *             coincident pair leaves the normal range): a softening below
 *             ~1e-6 rcut acts as ~1e-6 rcut.
 *   rs        split scale R_s of Eq. (split) (> 0).
 *   rcut      cutoff radius, 0 < rcut < L/2 (R_cut of Sec. 3.1).
 *   leaf_max  largest number of particles in an octree leaf, 1..256 (the
 *             N_pp of Sec. 3.1 / leaf size of Sec. 4.4).
 *   key_kind  PH_KEY_MORTON or PH_KEY_HILBERT.
 *   group_size target particles summed together by one warp: 32, 16 or 8
 *             (then 2 or 4 lanes share a target, each taking every 2nd or
 *             4th source; smaller groups waste fewer pairs beyond rcut);
 *             0 = default (32).
 *   level_bits key bits per level of the leaf hierarchy: 3 = octree cells
 *             (each level splits a cell into 8 children, Sec. 3.2), 1 = the
 *             same tree with every octree level split into three binary
 *             levels along the key's x, y, z bits (leaves closer to
 *             leaf_max); 0 = default (1).
 *   pp_variant PP kernel shape: 0 = two 8-warp blocks per SM (deeper
 *             unrolled source loop), 1 = three blocks per SM (fewer
 *             registers, more warps).  Same results.
 *   queue_order order in which the PP kernel's warps take the target groups
 *             (the task queue of Sec. 4.3): 0 (default) = by decreasing
 *             cost, the source particles of the group's list (Sec. 4.4
 *             weighs work by counts), in quarter-octave classes (within a
 *             class in the order the pair builder meets the groups) -- the
 *             heaviest groups start first, so the launch ends on short
 *             ones; 1 = plain group order (along the curve).  Same results
 *             (each group is summed by one warp on its own).  The direct
 *             mode (no stored list) and the active-particle mode take group
 *             order.
 *   theta     opening criterion of the tree part (Sec. 3.3), in [0, 1):
 *             0 (default) = every leaf pair by PP (the exact short-range
 *             sum); theta > 0 = a leaf for which both opening angles
 *             theta_1 = (A + B) / R and theta_2 = B / (R - A) are below
 *             theta (A the target group's largest box width, B the leaf's,
 *             R the distance of the box centres) acts on the group as one
 *             particle of the leaf's mass at its mass centre, still with
 *             the split factor and the cutoff.  Decided in FP32 from the
 *             stored boxes (rounded outwards to FP32), so a pair within a
 *             few FP32 roundings of the threshold may go either way.  Tree
 *             leaves only (no interior nodes).
 */
typedef struct ph_params {
    double  L;
    double  G;
    double  eps;
    double  rs;
    double  rcut;
    int32_t leaf_max;
    int32_t key_kind;
    int32_t group_size;
    int32_t level_bits;
    int32_t pp_variant;
    int32_t queue_order;
    double  theta;
} ph_params;

typedef struct ph_leaves ph_leaves;   /* sorted particles + leaf / group tables */
typedef struct ph_pairs  ph_pairs;    /* cutoff leaf-pair list (CSR by group)    */
typedef struct ph_mlp    ph_mlp;      /* learned short-range factor             */
typedef struct ph_graph  ph_graph;    /* a whole step captured as a CUDA graph  */
typedef struct ph_pm     ph_pm;       /* long-range particle-mesh solver         */
typedef struct ph_sim    ph_sim;      /* particles advanced by adaptive KDK steps */

/*
 * Sort the particles of one box along the space-filling curve and cut them
 * into leaves and target groups (Sec. 3.2, "Tree building": ground cell
 * index (i N_side + j) N_side + k, bucket order of ground cells, Morton
 * order inside; leaves are the largest cells of the tree -- octree cells, or
 * their binary sub-levels, see level_bits -- holding <= leaf_max particles,
 * Sec. 3.1 / 4.4).
 *
 *   pos       [n*3] host or device; pos_type PH_F32 or PH_F64; xyz per row.
 *   mass      [n]   host or device float32, or NULL for equal masses 1/n.
 *   n         number of particles (0 allowed: an empty handle).
 *   params    box parameters (host memory).
 *   stream    cudaStream_t.
 *   leaves    in/out: *leaves == NULL creates a handle, else it is rebuilt.
 * Errors: PH_ERR_ARG, PH_ERR_RCUT_GE_HALF_L, PH_ERR_OOM, PH_ERR_CUDA; a
 * non-finite coordinate is latched and reported as PH_ERR_NONFINITE by the
 * next synchronising call.  Synchronises the stream once (to size the leaf
 * and group tables).
 */
int ph_build_leaves(const void *pos, int pos_type, const float *mass, int64_t n,
                    const ph_params *params, void *stream, ph_leaves **leaves);

/*
 * Same for B independent boxes stored one after another: box b owns rows
 * [box_offsets[b], box_offsets[b+1]).  box_offsets [B+1] host int64,
 * box_offsets[0] = 0; params [B] host, one per box (mass NULL means 1/n_b
 * in box b).  Boxes never interact.  1 <= B <= 65536.
 */
int ph_build_leaves_batched(const void *pos, int pos_type, const float *mass,
                            const int64_t *box_offsets, int32_t n_boxes,
                            const ph_params *params, void *stream, ph_leaves **leaves);

/*
 * Build the cutoff leaf-pair list: for every target group, each leaf of the
 * 27 ground cells around it (Sec. 4.3: a ground cell and its 26 neighbours,
 * each with the periodic image its offset implies) whose bounding box comes
 * within rcut of the group's bounding box (Sec. 3.3: leaf-leaf interactions
 * go to the PP kernel).  Stored per entry: the FP32 offset (leaf reference -
 * group reference, computed in FP64, image included), the leaf's first
 * particle and its particle count.  With queue_order 0 the same passes
 * also order the groups by decreasing cost for the PP kernel's queue (see
 * ph_params).
 * Synchronises the stream once to size the list, unless the handle was given
 * a fixed capacity with ph_pairs_reserve (then overflow is latched as
 * PH_ERR_CAPACITY and no entry beyond the capacity is written).
 */
int ph_leaf_pairs(ph_leaves *leaves, void *stream, ph_pairs **pairs);

/* Give a pairs handle a fixed capacity (entries) and stop the sizing sync. */
int ph_pairs_reserve(ph_pairs **pairs, int64_t capacity);

/*
 * PP direct summation over the pair list (Eq. (split), Sec. 3.3, Sec. 4.4):
 * writes acc[3*i .. 3*i+2] = a_i for every particle, in the caller's
 * original order (box-concatenated order for batched handles).
 *   pairs   a list from ph_leaf_pairs on these leaves, or NULL for the direct
 *           mode (exact factor only): the PP kernel finds each group's leaf
 *           pairs itself, with the same test and in the same order as
 *           ph_leaf_pairs, so no list is stored and the result is the same
 *           bit for bit.
 *   g_mode  PH_G_EXACT, PH_G_LEARNED (then mlp and pairs must be non-NULL)
 *           or PH_G_TABLE (pairs must be non-NULL; the table is made on the
 *           host and uploaded at the first call for an rcut / rs).
 *   acc     [n*3] float32, host or device.
 * Returns PH_WARN_FALLBACK when the learned factor's validated error is above
 * its tolerance: the exact factor is used instead.
 */
int ph_pp_accel(const ph_leaves *leaves, const ph_pairs *pairs, int g_mode,
                const ph_mlp *mlp, float *acc, void *stream);

/*
 * Whole step in one call: build leaves, pairs, then PP, reusing *leaves and
 * *pairs (created when NULL).  pos/mass/acc host or device as above.
 * pairs = NULL: build, then the direct-mode PP (no list; exact factor only).
 */
int ph_accel(const void *pos, int pos_type, const float *mass, int64_t n,
             const ph_params *params, int g_mode, const ph_mlp *mlp, float *acc,
             void *stream, ph_leaves **leaves, ph_pairs **pairs);

/*
 * Capture the whole step (build, pairs, PP) for these handles as one CUDA
 * graph (pairs = NULL: build and the direct-mode PP, exact factor only, no
 * list and no capacity): one replay launches every kernel of the step -- the PP part one
 * persistent launch over all boxes of a batched handle -- with no host
 * synchronisation and no allocation (the batched, graph-captured execution
 * of the many-box workload; Sec. 4.3's task queue over all boxes' groups).
 *   leaves, pairs  built once before (ph_build_leaves[_batched], ph_leaf_pairs)
 *                  for the same particle count and boxes.
 *   d_pos, d_mass, d_acc  device buffers read / written at every replay.
 *   headroom       the pair list gets a fixed capacity of
 *                  (1 + headroom) x its current length (e.g. 0.25).
 * Replays that would overflow it latch PH_ERR_CAPACITY in ph_status(pairs)
 * (no entry beyond the capacity is written); rebuild the pairs and recreate
 * the graph.  Learned mode with a network that fails its tolerance captures
 * the exact factor and returns PH_WARN_FALLBACK.  Synchronises once.
 */
int ph_graph_create(ph_leaves *leaves, ph_pairs *pairs, const void *d_pos, int pos_type, const float *d_mass,
                    int g_mode, const ph_mlp *mlp, float *d_acc, double headroom, void *stream,
                    ph_graph **graph);

/* Replay a captured step on `stream` (asynchronous). */
int ph_graph_launch(ph_graph *graph, void *stream);

/*
 * Replay with host buffers: copy h_pos [n*3] (the pos_type of the capture)
 * and, when not NULL, h_mass [n] into the device buffers the graph reads,
 * replay it, and copy the accelerations into h_acc [n*3] (caller order).
 * Returns after the copies have completed (synchronises the stream once) and
 * reports the step's latched status: PH_ERR_CAPACITY means the pair list
 * outgrew its capacity (rebuild the pairs and the graph), PH_ERR_NONFINITE a
 * non-finite input.  h_mass must be NULL for a graph captured without
 * masses.  Pinned host memory makes the copies asynchronous DMA.
 */
int ph_graph_launch_host(ph_graph *graph, const void *h_pos, const float *h_mass, float *h_acc, void *stream);

/*
 * The same work as ph_graph_launch_host -- the copies in, the replay, the
 * copy out -- enqueued on `stream` without waiting for it.  h_acc holds the
 * step's accelerations once the stream has passed this work (synchronise
 * it); h_pos and h_mass must stay unchanged until then.  Device conditions
 * (capacity, non-finite input) are latched in the handles' status words:
 * read them with ph_status on the leaves and pairs after synchronising.
 * With pinned host memory, two graphs over separate handles and device
 * buffers replayed alternately on two streams overlap one step's copies
 * with the other's kernels.  Errors: PH_ERR_ARG, PH_ERR_STATE (as
 * ph_graph_launch), PH_ERR_CUDA.
 */
int ph_graph_launch_host_async(ph_graph *graph, const void *h_pos, const float *h_mass, float *h_acc,
                               void *stream);

/* Kernels launched by one replay. */
int ph_graph_kernels(const ph_graph *graph, int64_t *kernels);

/*
 * Autotuner: time the whole step (build, pairs, exact PP) for every
 * combination of leaf_max in {16, 32, 64}, key_kind in {Morton, Hilbert},
 * pp_variant in {0, 1} and group_size in {16, 32} (24 candidates, binary
 * levels) on the caller's particles (device buffers; boxes as for
 * ph_build_leaves_batched, n_boxes = 1 for one box) and return the fastest
 * as out->best (params[0] with the winning knobs), with every candidate's
 * median of `reps` timed steps.  The knobs do not change the result beyond
 * FP32 summation order.  Synchronises.
 */
#define PH_TUNE_MAX 32
typedef struct ph_tune_result {
    ph_params best;
    float     best_ms;
    int32_t   n_tried;
    float     ms[PH_TUNE_MAX];
    int32_t   leaf_max[PH_TUNE_MAX];
    int32_t   level_bits[PH_TUNE_MAX];
    int32_t   pp_variant[PH_TUNE_MAX];
    int32_t   group_size[PH_TUNE_MAX];
    int32_t   key_kind[PH_TUNE_MAX];
} ph_tune_result;

int ph_autotune(const void *d_pos, int pos_type, const float *d_mass, const int64_t *box_offsets, int32_t n_boxes,
                const ph_params *params, int32_t reps, void *stream, ph_tune_result *out);

/* ------------------------------------------------------------ long-range PM
 * The particle-mesh side of the force split (Sec. 3.1), which supplies what
 * the short-range sum leaves out: the total force is ph_pp_accel's short-range
 * acceleration plus this one.  Steps, in the paper's order:
 *   1. Cloud-in-Cell assignment of the masses to a periodic N^3 mesh with
 *      nodes at x = i L/N (64-bit fixed-point sums: the node masses do not
 *      depend on the order of the additions);
 *   2. FFT (cuFFT, FP32);
 *   3. the Green's function of the 3-point difference Laplacian of Sec. 3.1,
 *      phi_k = -pi G Delta_g^2 rho_k / (sin^2(pi l/N) + sin^2(pi m/N) +
 *      sin^2(pi n/N)), Delta_g = L/N, rho = node mass / Delta_g^3, times the
 *      long-range filter exp(-k^2 R_s^2) (k the continuum wavenumber
 *      2 pi l'/L of the mode, l' in (-N/2, N/2]); the k = 0 mode is dropped
 *      (neutralising background);
 *   4. inverse FFT: the potential on the mesh;
 *   5. a = -grad phi on the mesh by the 2-point central difference, then
 *      Cloud-in-Cell interpolation to each particle with the assignment
 *      weights.  No window deconvolution.
 * The cell of a particle is decided in FP64: a coordinate in [0, L) is kept,
 * any other becomes x_w = x - L floor(x/L); u = x_w (N/L), node floor(u)
 * mod N, fraction u - floor(u).
 *
 *   pos, pos_type, mass, n   as for ph_build_leaves (host or device; mass
 *                NULL = 1/n each); one box, caller order.
 *   params       L, G and rs are used (rs = 0: no filter, the whole
 *                periodic PM force); the other fields are ignored.
 *   n_mesh       N, even, 4..PH_PM_MAX_MESH.
 *   acc          [n*3] float32 host or device: written, or added to when
 *                accumulate != 0 (e.g. onto ph_pp_accel's result).
 *   pot          [n] float32 host or device, nullable: the long-range
 *                potential interpolated to each particle.
 *   pm           in/out handle (mesh buffers, FFT plans); created when
 *                *pm == NULL; kept while N is unchanged.
 * Memory: 44 N^3 bytes + the FFT work area (about 95 MB at N = 128).
 * Errors: PH_ERR_ARG, PH_ERR_OOM, PH_ERR_CUDA; a non-finite coordinate or
 * mass is latched (ph_status(pm) reports PH_ERR_NONFINITE) and that
 * particle is left out.  Synchronises only when acc or pot are host memory
 * or when the Green's function tables are (re)made for a new N, L or rs.
 */
#define PH_PM_MAX_MESH 1024

int ph_pm_accel(const void *pos, int pos_type, const float *mass, int64_t n, const ph_params *params,
                int32_t n_mesh, float *acc, float *pot, int32_t accumulate, void *stream, ph_pm **pm);

typedef struct ph_pm_view {
    int32_t n_mesh;
    int32_t reserved;
    double  mass_unit;          /* node mass = mass_fixed[i] * mass_unit        */
    const int64_t *mass_fixed;  /* [N^3] node masses of step 1, fixed point,
                                   index (i N + j) N + k for node (i, j, k)     */
    const float   *mesh;        /* [N^3 * 4] per node: -dphi/dx, -dphi/dy,
                                   -dphi/dz, phi (steps 4-5, before the
                                   interpolation)                              */
} ph_pm_view;

/* Device views of the last ph_pm_accel's meshes (synchronises). */
int ph_pm_get_view(const ph_pm *pm, ph_pm_view *out);

/* ------------------------------------------------------------ adaptive KDK
 * The time integration of Sec. 3.4 driving repeated force calls: the
 * symplectic Drift x += p int dt/a^2 and Kick p += a_grav int dt/a, applied
 * as Kick-Drift-Kick, with every particle's step the top step halved until
 * it is below t_acc = sqrt(2 eta eps / |a|) (Gadget-2's criterion; the
 * printed form is garbled), so steps are dt / 2^level and meet at the ends
 * of coarser steps (block steps).
 *
 * One top step: every particle takes its level from its acceleration and an
 * opening half kick; then, at each event (the earliest end of any
 * particle's current step, on a timeline of 2^max_level ticks), all
 * particles drift to it, the force is recomputed for all (ph_accel: build,
 * pairs, short-range PP; then ph_pm_accel added when n_mesh > 0) for the
 * particles whose step ends there (only their groups get source lists),
 * those particles take their closing half kick and, before the
 * top step's end, a new level (refined until its step length divides the
 * elapsed ticks) and an opening half kick.  The level is the smallest k in
 * [0, max_level] with (dt_phys / 2^k)^2 |a| <= 2 eta eps_step, decided in
 * FP64.  Positions (FP64) stay in [0, L).
 *
 * Clocks: PH_CLOCK_NEWTON (time t, drift and kick factors t2 - t1) or
 * PH_CLOCK_LCDM (time = scale factor a of a flat Lambda-CDM universe,
 * D = int da / (a^3 H), K = int da / (a^2 H), H = H0 sqrt(omega_m a^-3 +
 * omega_l); dt_phys = dt / (a H(a)) in the criterion).
 */
#define PH_CLOCK_NEWTON 0
#define PH_CLOCK_LCDM   1

typedef struct ph_kdk_params {
    double  dt;         /* top step in the time variable (> 0)                  */
    double  eta;        /* accuracy parameter of the criterion (> 0)            */
    double  eps_step;   /* softening length of the criterion; 0 = params->eps   */
    double  H0, omega_m, omega_l;   /* PH_CLOCK_LCDM only                       */
    int32_t max_level;  /* finest level, 0..20 (steps down to dt / 2^max_level) */
    int32_t n_mesh;     /* PM mesh for the long-range force; 0 = short range only */
    int32_t clock;      /* PH_CLOCK_NEWTON or PH_CLOCK_LCDM                     */
    int32_t g_mode;     /* PH_G_EXACT or PH_G_TABLE                             */
} ph_kdk_params;

/*
 * Copy n particles (pos, mom [n*3] float64, mass [n] float32 or NULL = 1/n;
 * host or device) into a new simulation at time t0 (for PH_CLOCK_LCDM the
 * scale factor a0 > 0), wrap the positions into [0, L) and compute their
 * first force.  params: the box of ph_build_leaves.  *sim must be NULL.
 * Synchronises.
 */
int ph_sim_create(const double *pos, const double *mom, const float *mass, int64_t n, const ph_params *params,
                  const ph_kdk_params *kp, double t0, void *stream, ph_sim **sim);

/* Advance by n_steps top steps (one host synchronisation per event). */
int ph_sim_step(ph_sim *sim, int32_t n_steps, void *stream);

/* Current state (each output host or device, nullable): positions and
 * momenta [n*3] float64, accelerations [n*3] float32 of the last force pass
 * (after a whole top step: of every particle), levels [n] of the last top
 * step, time, and force passes so far.  Synchronises and reports any status
 * latched by the force calls. */
int ph_sim_get(const ph_sim *sim, double *pos, double *mom, float *acc, int32_t *level, double *t,
               int64_t *force_passes);

/* ------------------------------------------------------------ domains
 * Domain decomposition for several GPUs (Sec. 4.1).  A box is cut along the
 * space-filling curve of its ground cells (the N_side^3 cells of side >=
 * rcut the tree build starts from, N_side = 2^g from L and rcut) into runs of
 * consecutive cells, one run per domain, balanced by work: a cell's work is
 * its particle count times the particle count of its 27-cell neighbourhood.
 * A domain's ghost cells are the cells of the periodic 26-neighbourhood of
 * its own cells that it does not own; own + ghost cells hold every particle
 * within rcut of a particle it owns, so each domain (one GPU) computes its
 * own particles' short-range forces from its local set alone, with one
 * exchange of particles per step and no reduction.  These three calls run on
 * the host (no GPU, no stream); the exchange itself is the caller's (the
 * Python package does it with torch.distributed).
 */

/* Ground grid size (*nside) and each particle's ground cell
 * (i N_side + j) N_side + k, decided as the tree build decides it.  pos host
 * memory [n*3] (PH_F32 or PH_F64); params: L and rcut; cell [n] host. */
int ph_domain_cells(const void *pos, int pos_type, int64_t n, const ph_params *params, int32_t *nside,
                    int32_t *cell);

/* owner[cell] in [0, n_domains): runs of consecutive cells along the
 * key_kind curve (PH_KEY_MORTON or PH_KEY_HILBERT) of about equal work, from
 * the particle count of every cell (host int64 [N_side^3], summed over all
 * ranks).  domain_cost [n_domains] (nullable): the work each domain got. */
int ph_domain_partition(const int64_t *cell_count, int32_t nside, int32_t key_kind, int32_t n_domains,
                        int32_t *owner, double *domain_cost);

/* need[cell] for one domain (host uint8 [N_side^3]): 1 own cell, 2 ghost
 * cell (periodic 26-neighbour of an own cell), 0 not needed. */
int ph_domain_halo(const int32_t *owner, int32_t nside, int32_t domain, uint8_t *need);

/*
 * Device side of the exchange (Sec. 4.1) for ranks that keep particles on the
 * GPU.  The rows sent between ranks are PH_DOMAIN_ROW doubles per particle:
 * x, y, z (as given), mass, its flag at the destination (1 own, 2 ghost)
 * and the caller's int64 identifier (its 64 bits).  These calls share one
 * scratch area inside the library: calls from several host threads or on
 * several streams must not overlap.
 */
#define PH_DOMAIN_ROW 6

/* ph_domain_cells on the device: d_cell [n] (int32) the ground cell of
 * every particle, bit for bit the host's decision, and d_counts
 * [N_side^3] (int64, cleared first) the particles per cell.  Device
 * buffers.  Synchronises once (PH_ERR_NONFINITE for a non-finite
 * position). */
int ph_domain_cells_device(const void *d_pos, int pos_type, int64_t n, const ph_params *params, int32_t *nside,
                           int32_t *d_cell, int64_t *d_counts, void *stream);

/* The send buffer: for every rank r = 0 .. n_ranks-1 in turn, the rows of
 * the particles r needs (those in cells r owns, flag 1, and in r's ghost
 * cells, flag 2; h_owner from ph_domain_partition), in particle order.
 * d_mass NULL: mass 0 is sent; d_ids NULL: the row index is sent.
 * h_send_counts [n_ranks] receives the rows per rank even when the capacity
 * (rows of d_send) is too small, which returns PH_ERR_CAPACITY.
 * Synchronises once. */
int ph_domain_pack(const void *d_pos, int pos_type, const float *d_mass, const int64_t *d_ids, const int32_t *d_cell,
                   int64_t n, const int32_t *h_owner, int32_t nside, int32_t n_ranks, double *d_send,
                   int64_t send_capacity, int64_t *h_send_counts, void *stream);

/* A rank's local set from the n_recv rows it received: own rows first, then
 * the ghosts, each in received order; positions written as pos_type,
 * masses float32, identifiers int64 (device buffers of n_recv).  *h_n_own:
 * the number of own rows.  Synchronises once. */
int ph_domain_unpack(const double *d_recv, int64_t n_recv, int pos_type, void *d_pos, float *d_mass, int64_t *d_ids,
                     int64_t *h_n_own, void *stream);

/* Free any handle (ph_leaves, ph_pairs, ph_mlp, ph_graph, ph_pm, ph_sim).  NULL is a no-op. */
void ph_free(void *handle);

/* Message of the last failing call on this thread ("" if none). */
const char *ph_last_error(void);

/* Synchronise the handle's last stream and return its latched device status. */
int ph_status(const void *handle);

/* ------------------------------------------------------------ introspection
 * Read-only views of the internal arrays (device pointers, valid until the
 * handle is rebuilt or freed).  Used by tests to check each step.
 */
typedef struct ph_leaves_view {
    int64_t n;                 /* particles                                    */
    int32_t n_boxes;
    int32_t n_leaves;
    int32_t n_groups;
    int32_t n_cells;           /* ground cells over all boxes                  */
    const uint64_t *keys;      /* [n] sorted keys                              */
    const int32_t *perm;       /* [n] sorted position -> caller row            */
    const int32_t *leaf_first; /* [n_leaves+1]                                 */
    const double  *leaf_ref;   /* [n_leaves*3] leaf reference point (FP64)     */
    const float   *leaf_half;  /* [n_leaves*4] bounding-box half extents x, y,
                                  z; w holds the particle count (int bits)   */
    const int32_t *group_first;/* [n_groups+1]                                 */
    const double  *group_ref;  /* [n_groups*3]                                 */
    const float   *group_half; /* [n_groups*4] as leaf_half                    */
    const float   *pos_leaf;   /* [n*4] x-ref_leaf, y, z, mass (FP32)          */
    const float   *pos_group;  /* [n*4] x-ref_group, y, z, mass (FP32)         */
    const int32_t *cell_leaf_first; /* [n_cells+1] first leaf of each cell     */
    int32_t g[4];              /* ground level of box 0..3 (N_side = 2^g)      */
    int32_t key_bits;          /* T: key bits per axis                         */
    int32_t group_size;
} ph_leaves_view;

typedef struct ph_pairs_view {
    int64_t n_pairs;
    int32_t n_groups;
    int32_t reserved;
    const int64_t *group_off;  /* [n_groups+1] CSR offsets                     */
    const float   *entries;    /* [n_pairs*4] off.x, off.y, off.z, and the     */
                               /* leaf's first particle (int32 bits, sorted)   */
    const uint8_t *counts;     /* [n_pairs] particles in the leaf minus one    */
    const int32_t *group_order;/* [n_groups] the PP queue's order of the groups
                                  (queue_order 0), or NULL (group order)      */
} ph_pairs_view;

int ph_leaves_get_view(const ph_leaves *leaves, ph_leaves_view *out);
int ph_pairs_get_view(const ph_pairs *pairs, ph_pairs_view *out);

/* Work counted by the last ph_pp_accel on this handle (synchronises):
 * interactions evaluated by the PP kernel, and the j-particles staged.
 * `handle` is the pairs handle of that call, or its leaves handle after a
 * direct-mode call (pairs = NULL). */
int ph_pp_counters(const void *handle, int64_t *interactions, int64_t *staged);

/* Active-particle mode (Sec. 3.4: only the particles whose step ends need
 * a force; Sec. 4.1: only a domain's own particles, not its ghosts): with
 * d_active set (device uint8 [n] in the caller's order of the particles of
 * the next builds, nonzero = active), every later build of this handle
 * marks the target groups holding an active particle and the pair builder
 * gives entries to those groups only, so the PP kernel sums nothing for
 * the others and writes zero accelerations for them.  The flags are read at
 * each build: keep the buffer alive and sized for the build's particles.
 * NULL turns the mode off.  Rebuild the leaves (and the pairs) after
 * changing it. */
int ph_leaves_set_active(ph_leaves *leaves, const uint8_t *d_active, int64_t n);

/* Number of ordered pairs (i, j), j != i, with r_ij < rcut in the lists,
 * decided in FP32 exactly as ph_pp_accel decides its cutoff: the work the
 * cutoff keeps (the oracle's count up to pairs within rounding of rcut and
 * coincident particles).  Synchronises. */
int ph_count_within(const ph_leaves *leaves, const ph_pairs *pairs, int64_t *n_within, void *stream);

/* ------------------------------------------------------------ learned factor
 * A 1-16-16-1 network with SiLU activations stands in for Eq. (split) in the
 * PP inner loop (PH_G_LEARNED).  Input z0 = 2 r / rcut - 1; output g_hat(r).
 * Parameters, flat float32[321]: W1[16], b1[16], W2[16][16] (row k holds the
 * weights into unit k), b2[16], W3[16], b3.  Inference in the PP kernel:
 * layer 1 (one scalar input) by linear interpolation in a 512-node table of
 * its 16 activations that each kernel builds in shared memory from the
 * weights, layer 2 as BF16 tensor-core MMAs (mma.sync m16n8k16, FP32
 * accumulation, activations and weights split into BF16 hi + lo parts), its
 * SiLUs in FP32 (SFU ex2/rcp) and layer 3 in FP32; only pairs with
 * r < rcut are evaluated.  A handle records the largest relative error of
 * g_hat against the exact factor over r in [0, rcut) (the exact path judges
 * the network); ph_pp_accel falls back to the exact factor and returns
 * PH_WARN_FALLBACK when that error is above the handle's tolerance or the
 * box's rcut / rs differs from the one the network was trained for.
 */
#define PH_MLP_PARAMS 321

typedef struct ph_train_params {
    int64_t  n_samples;   /* training samples r ~ U[0, rcut) (e.g. 10^6)           */
    int32_t  batch;       /* samples per Adam step                                  */
    int32_t  steps;       /* Adam steps                                             */
    float    lr0, lr_min; /* cosine learning-rate schedule from lr0 to lr_min       */
    float    tol;         /* accepted largest relative error of g_hat (0 = 1e-3)    */
    int32_t  reserved;
    uint64_t seed;        /* init stream = seed, samples = seed+1, batches = seed+2 */
} ph_train_params;

/*
 * Train the network on the GPU (the project's own forward, backward and Adam
 * kernels, FP32): samples and their exact-factor targets are generated on the
 * device; loss = mean ((g_hat - g) / g)^2 over each batch.  init_weights:
 * host float[321], or NULL for the seeded initialisation.  Synchronises.
 */
int ph_mlp_train(const ph_train_params *tp, double rs, double rcut, const float *init_weights,
                 void *stream, ph_mlp **mlp);

/* A handle from given weights (host or device float[321]); validates them. */
int ph_mlp_create(const float *weights, double rs, double rcut, float tol, void *stream, ph_mlp **mlp);

/* Weights (host float[321], nullable), validated error and last training loss. */
int ph_mlp_get(const ph_mlp *mlp, float *weights, float *max_rel_err, float *last_loss);

/* g_hat at n inputs z0 = 2r/rcut - 1 (device float[n] in, device float[n]
 * out), evaluated exactly as the learned PP kernel does (layer-1 table,
 * BF16 tensor-core layer 2, FP32 SiLUs and layer 3), for tests and
 * inspection.  Asynchronous on `stream`.  Errors: PH_ERR_ARG (bad handle or
 * pointers, host buffers), PH_ERR_CUDA. */
int ph_mlp_eval(const ph_mlp *mlp, const float *d_z0, int64_t n, float *d_out, void *stream);

/* One forward + backward pass of the training kernel on given inputs
 * (host or device float[n] each): gradient of the mean relative squared
 * error (host float[321]) and the loss.  Synchronises. */
int ph_mlp_loss_grad(const float *weights, const float *z0, const float *target, int64_t n, float *grad,
                     float *loss, void *stream);

/*
 * Saving and loading a trained network (no counterpart in the paper, which
 * tabulates g instead: this is the checkpoint of the learned factor).
 *
 * File layout, all little-endian, 1348 bytes:
 *   bytes  0..7     magic "PHMLP\0\0\1"
 *   8..11           uint32 format version (1)
 *   12..15          uint32 parameter count (321)
 *   16..23          float64 rs the network was trained for
 *   24..31          float64 rcut
 *   32..35          float32 validated max |g_hat/g - 1| at save time
 *   36..39          float32 last training loss
 *   40..43          int32   training steps done
 *   44..47          uint32  reserved (0)
 *   48..1331        float32 weights[321] in the order of ph_mlp_create
 *   1332..1339      uint64  FNV-1a hash of bytes 0..1331
 *   1340..1347      uint64  reserved (0)
 *
 * ph_mlp_file_write / ph_mlp_file_read are host only (no GPU needed).
 * Read errors: PH_ERR_ARG for a missing or short file, a wrong magic,
 * version or count, or a hash that does not match (a damaged file).
 * ph_mlp_save writes the weights of a handle (synchronising the device);
 * ph_mlp_load reads a file into a new handle whose error is validated anew
 * on the device against the exact factor, accepted up to `tol` as in
 * ph_mlp_create.  The caller owns the returned handle (ph_free).
 */
int ph_mlp_file_write(const char *path, const float *weights, double rs, double rcut, float max_rel_err,
                      float last_loss, int32_t steps);
int ph_mlp_file_read(const char *path, float *weights, double *rs, double *rcut, float *max_rel_err,
                     float *last_loss, int32_t *steps);
int ph_mlp_save(const ph_mlp *mlp, const char *path);
int ph_mlp_load(const char *path, float tol, void *stream, ph_mlp **mlp);

/* ------------------------------------------------------------ no allocation
 * ph_accel_noalloc -- the whole step (ph_accel with the exact factor) for
 * one small box, without allocating anything.
 *
 * The paper has no counterpart: this exists for callers that must not
 * allocate device memory themselves, e.g. an application that gives every
 * library a fixed device-memory budget through its own allocator, or a
 * latency-critical loop that cannot take the device-wide synchronisation
 * that cudaMalloc and cudaFree imply.  The caller owns the inputs and the
 * output; all intermediate data live in one fixed array of
 * PH_NOALLOC_SCRATCH_BYTES that every GPU which loads libphpp.so holds until
 * the process exits.  No cudaMalloc, cudaFree or other allocating routine is
 * called.
 *
 *   d_pos   [n*3] device float32 positions (any real coordinates; wrapped).
 *   d_mass  [n]   device float32 masses, or NULL for 1/n each.
 *   n       0 .. PH_NOALLOC_MAX_N; larger n returns PH_ERR_ARG.
 *   params  as for ph_build_leaves, with three limits (else PH_ERR_ARG):
 *           theta must be 0 (every leaf pair by PP), group_size 0 or 32,
 *           and L/rcut must give at most PH_NOALLOC_MAX_CELLS ground cells.
 *           The key depth, factor polynomial and box constants are those
 *           ph_build_leaves derives for the same box.
 *   d_acc   [n*3] device float32 output, caller order.
 * The call synchronises `stream` once before returning.  PH_ERR_CAPACITY
 * means the leaf-pair list needed more than PH_NOALLOC_PAIRS_PER_PARTICLE
 * entries per particle (strongly clustered input): use ph_accel instead.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  Every
 * call on a device uses the same array and overwrites what the previous call
 * left there, so calls that overlap on the GPU (other streams, other host
 * threads) race: serialise them.
 */
#define PH_NOALLOC_MAX_N               16384
#define PH_NOALLOC_MAX_CELLS           4096
#define PH_NOALLOC_PAIRS_PER_PARTICLE  32
#define PH_NOALLOC_SCRATCH_BYTES       (16u << 20)
int ph_accel_noalloc(const float *d_pos, const float *d_mass, int64_t n, const ph_params *params,
                     float *d_acc, void *stream);

/* Kernel launches the library has issued so far in this process (all
 * threads); differences around a region count the launches inside it. */
int64_t ph_launch_counter(void);

/*
 * Testing hook for failure paths (no counterpart in the paper): after k
 * more device allocations made by the library (k = 0: the next one), one
 * fails exactly as if the device were out of memory (the old buffer is
 * released, PH_ERR_OOM is returned); k < 0 turns the hook off.  One shot:
 * the hook turns itself off after the failure.  A call that fails this way
 * leaves a fresh handle unmade (nothing leaks) and an existing handle
 * invalid (PH_ERR_STATE from every call that would read it) until it is
 * built again successfully.
 */
void ph_debug_fail_allocation(int64_t k);

/*
 * Debug bounds checks (a testing aid; no counterpart in the paper).  A
 * library built with bounds checks (`python -m paper_1802_09824_gb300.build
 * --checked`: libphpp_checked.so, the same sources compiled with
 * PHPP_BOUNDS_CHECK) tests the indices of its kernels' buffer accesses; an
 * index outside its buffer skips the access (no trap, no wait) and is
 * counted.  This call synchronises the device, returns the number of such
 * accesses since the last call in *hits and the site of the first one in
 * *first_site (a small code, 0 = none), and clears both.  Returns
 * PH_ERR_STATE from a library built without the checks.
 */
int ph_debug_bounds(int64_t *hits, int32_t *first_site);

#ifdef __cplusplus
}
#endif

#endif /* PHPP_H */
