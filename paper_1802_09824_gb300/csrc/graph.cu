// A whole step captured once as a CUDA graph and replayed.
//
// The capture records every kernel of the step -- keys, radix sort, leaves,
// groups, frames, pair count / scan / fill and the persistent PP kernel over
// all boxes -- with the handles' buffers at fixed addresses and the pair list
// at a fixed capacity, so a replay needs no host round trip and no
// allocation.  Positions and masses are read from the captured device
// pointers at every replay (update them in place between replays).  A replay
// whose pair list would outgrow the capacity writes no entry beyond it and
// latches PH_ERR_CAPACITY in the pairs handle's status (ph_status); rebuild
// with ph_leaf_pairs and create a new graph then.
#include <new>

#include "handles.cuh"
#include "mlp_handle.cuh"

namespace phpp {
int build_leaves_device(ph_leaves *h, const void *pos, int pos_type, const float *mass, cudaStream_t s);
int build_pairs_device(const ph_leaves *lv, ph_pairs *pr, cudaStream_t s, bool sizing_sync);
int pp_exact_device(const ph_leaves *lv, const ph_pairs *pr, float *d_acc, cudaStream_t s);
int pp_learned_device(const ph_leaves *lv, const ph_pairs *pr, const float *mlp_w, float *d_acc, cudaStream_t s);
int pp_table_device(const ph_leaves *lv, const ph_pairs *pr, float *d_acc, cudaStream_t s);
int ensure_table(ph_leaves *lv, cudaStream_t s);
}  // namespace phpp

struct ph_graph {
    uint32_t kind = phpp::KIND_GRAPH;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;        // our kernel launches per replay
    // the buffers the capture reads and writes (for host-buffer replays)
    const void *d_pos = nullptr;
    const float *d_mass = nullptr;
    float *d_acc = nullptr;
    int pos_type = PH_F32;
    int64_t n = 0;
    ph_leaves *leaves = nullptr;
    ph_pairs *pairs = nullptr;
    uint64_t fingerprint = 0;     // the handles' buffers at capture (replays need the same)
};

using namespace phpp;

namespace phpp {
void graph_free(ph_graph *g)
{
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}
}  // namespace phpp

extern "C" {

int ph_graph_create(ph_leaves *leaves, ph_pairs *pairs, const void *d_pos, int pos_type, const float *d_mass,
                    int g_mode, const ph_mlp *mlp, float *d_acc, double headroom, void *stream, ph_graph **out)
{
    TraceRange trace_("ph_graph_create");
    if (!leaves || leaves->kind != KIND_LEAVES || (pairs && pairs->kind != KIND_PAIRS) || !out)
        return fail(PH_ERR_ARG, "ph_graph_create: leaves and out must be valid, pairs valid or NULL");
    if (pairs && pairs->built_from != leaves) return fail(PH_ERR_STATE, "pairs were not built from these leaves");
    {
        const int rb = check_built(leaves, pairs);
        if (rb) return rb;
    }
    if (!pairs && g_mode != PH_G_EXACT) return fail(PH_ERR_ARG, "ph_graph_create: the direct mode is exact only");
    if (!pairs && leaves->tree_leaves) return fail(PH_ERR_ARG, "ph_graph_create: the tree part needs a pair list");
    if (g_mode == PH_G_TABLE) {
        const int rt = ensure_table(leaves, static_cast<cudaStream_t>(stream));   // before the capture
        if (rt) return rt;
    }
    if (leaves->n > 0 && (!d_pos || !d_acc || !is_device_ptr(d_pos) || !is_device_ptr(d_acc) ||
                          (d_mass && !is_device_ptr(d_mass))))
        return fail(PH_ERR_ARG, "ph_graph_create: pos, mass and acc must be device memory");
    if (pos_type != PH_F32 && pos_type != PH_F64) return fail(PH_ERR_ARG, "bad pos_type");
    if (g_mode != PH_G_EXACT && g_mode != PH_G_LEARNED && g_mode != PH_G_TABLE) return fail(PH_ERR_ARG, "bad g_mode");
    if (g_mode == PH_G_LEARNED && (!mlp || mlp->kind != KIND_MLP)) return fail(PH_ERR_ARG, "learned mode needs mlp");
    if (!(headroom >= 0 && headroom < 100)) return fail(PH_ERR_ARG, "headroom must be in [0, 100)");
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    if (pairs) {
        // fixed pair capacity with headroom over the current list
        const int64_t want = (int64_t)((double)pairs->n_pairs * (1.0 + headroom)) + 1024;
        if (want > pairs->capacity) {
            int rc = cuda_check(cudaStreamSynchronize(caller), "sync before growing");
            if (!rc) rc = ensure(pairs->entries, (size_t)want * sizeof(float4));
            if (!rc) rc = ensure(pairs->ecount, (size_t)want);
            if (rc) {
                pairs->valid = false;   // the entries are gone
                return rc;
            }
            pairs->capacity = want;
        }
        pairs->fixed_capacity = true;
    }
    bool learned = false;
    if (g_mode == PH_G_LEARNED) {
        learned = mlp->max_rel_err <= mlp->tol;
    }
    ph_graph *g = new (std::nothrow) ph_graph();
    if (!g) return fail(PH_ERR_OOM, "host allocation failed");
    cudaStream_t s = nullptr;
    int rc = cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "create capture stream");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(caller), "sync before capture");
    const long long k0 = ph_launch_counter();
    if (!rc) rc = cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (!rc) {
        int rc2 = cuda_check(cudaMemsetAsync(leaves->status.p, 0, 4, s), "clear status");
        if (!rc2 && pairs) rc2 = cuda_check(cudaMemsetAsync(pairs->status.p, 0, 4, s), "clear status");
        if (!rc2) rc2 = build_leaves_device(leaves, d_pos, pos_type, d_mass, s);
        if (!rc2 && pairs) rc2 = build_pairs_device(leaves, pairs, s, false);
        if (!rc2 && leaves->n > 0)
            rc2 = g_mode == PH_G_TABLE ? pp_table_device(leaves, pairs, d_acc, s)
                  : learned ? pp_learned_device(leaves, pairs, static_cast<const float *>(mlp->theta.p), d_acc, s)
                            : pp_exact_device(leaves, pairs, d_acc, s);
        cudaGraph_t gr = nullptr;
        rc = cuda_check(cudaStreamEndCapture(s, &gr), "end capture");
        g->graph = gr;
        if (!rc) rc = rc2;
    }
    g->kernels = ph_launch_counter() - k0;
    if (!rc) rc = cuda_check(cudaGraphInstantiate(&g->exec, g->graph, 0), "instantiate");
    if (s) cudaStreamDestroy(s);
    if (rc) {
        graph_free(g);
        return rc;
    }
    // the capture only recorded the launches; do not count them as run
    count_launch((int)-g->kernels);
    g->d_pos = d_pos;
    g->d_mass = d_mass;
    g->d_acc = d_acc;
    g->pos_type = pos_type;
    g->n = leaves->n;
    g->leaves = leaves;
    g->pairs = pairs;
    g->fingerprint = buffers_fingerprint(leaves, pairs);
    leaves->last_stream = caller;
    if (pairs) pairs->last_stream = caller;
    *out = g;
    if (g_mode == PH_G_LEARNED && !learned)
        return fail(PH_WARN_FALLBACK, "exact factor captured: validated network error %.3e above %.1e",
                    mlp->max_rel_err, mlp->tol);
    return PH_OK;
}

int ph_graph_launch(ph_graph *g, void *stream)
{
    TraceRange trace_("ph_graph_launch");
    if (!g || g->kind != KIND_GRAPH) return fail(PH_ERR_ARG, "not a ph_graph handle");
    // the capture holds the handles' buffer addresses: a rebuild that moved
    // or dropped any of them (larger n, a failed build) ends the graph's use
    if (!g->leaves->valid || (g->pairs && !g->pairs->valid) ||
        buffers_fingerprint(g->leaves, g->pairs) != g->fingerprint)
        return fail(PH_ERR_STATE, "the handles' buffers changed since the capture: create a new graph");
    int rc = cuda_check(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)), "graph launch");
    if (!rc) count_launch((int)g->kernels);
    return rc;
}

int ph_graph_launch_host(ph_graph *g, const void *h_pos, const float *h_mass, float *h_acc, void *stream)
{
    TraceRange trace_("ph_graph_launch_host");
    if (!g || g->kind != KIND_GRAPH) return fail(PH_ERR_ARG, "not a ph_graph handle");
    if (g->n > 0 && (!h_pos || !h_acc)) return fail(PH_ERR_ARG, "h_pos and h_acc must not be NULL");
    if (h_mass && !g->d_mass) return fail(PH_ERR_ARG, "the graph was captured without masses");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)g->n;
    const size_t pbytes = n * 3 * (g->pos_type == PH_F64 ? 8 : 4);
    int rc = PH_OK;
    if (n) rc = cuda_check(cudaMemcpyAsync(const_cast<void *>(g->d_pos), h_pos, pbytes, cudaMemcpyDefault, s),
                           "copy positions");
    if (!rc && n && h_mass)
        rc = cuda_check(cudaMemcpyAsync(const_cast<float *>(g->d_mass), h_mass, n * 4, cudaMemcpyDefault, s),
                        "copy masses");
    if (!rc) rc = ph_graph_launch(g, stream);
    if (!rc && n) rc = cuda_check(cudaMemcpyAsync(h_acc, g->d_acc, n * 12, cudaMemcpyDefault, s), "copy acc");
    uint32_t st[2] = {0, 0};
    if (!rc) rc = cuda_check(cudaMemcpyAsync(&st[0], g->leaves->status.p, 4, cudaMemcpyDeviceToHost, s), "status");
    if (!rc && g->pairs)
        rc = cuda_check(cudaMemcpyAsync(&st[1], g->pairs->status.p, 4, cudaMemcpyDeviceToHost, s), "status");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "host replay sync");
    if (rc) return rc;
    const uint32_t any = st[0] | st[1];
    if (any & ST_NONFINITE) return fail(PH_ERR_NONFINITE, "non-finite position or mass");
    if (any & ST_CAPACITY) return fail(PH_ERR_CAPACITY, "pair list capacity exceeded: rebuild the pairs and the graph");
    return PH_OK;
}

int ph_graph_launch_host_async(ph_graph *g, const void *h_pos, const float *h_mass, float *h_acc, void *stream)
{
    TraceRange trace_("ph_graph_launch_host_async");
    if (!g || g->kind != KIND_GRAPH) return fail(PH_ERR_ARG, "not a ph_graph handle");
    if (g->n > 0 && (!h_pos || !h_acc)) return fail(PH_ERR_ARG, "h_pos and h_acc must not be NULL");
    if (h_mass && !g->d_mass) return fail(PH_ERR_ARG, "the graph was captured without masses");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)g->n;
    const size_t pbytes = n * 3 * (g->pos_type == PH_F64 ? 8 : 4);
    int rc = PH_OK;
    if (n) rc = cuda_check(cudaMemcpyAsync(const_cast<void *>(g->d_pos), h_pos, pbytes, cudaMemcpyDefault, s),
                           "copy positions");
    if (!rc && n && h_mass)
        rc = cuda_check(cudaMemcpyAsync(const_cast<float *>(g->d_mass), h_mass, n * 4, cudaMemcpyDefault, s),
                        "copy masses");
    if (!rc) rc = ph_graph_launch(g, stream);
    if (!rc && n) rc = cuda_check(cudaMemcpyAsync(h_acc, g->d_acc, n * 12, cudaMemcpyDefault, s), "copy acc");
    return rc;
}

int ph_graph_kernels(const ph_graph *g, int64_t *kernels)
{
    if (!g || g->kind != KIND_GRAPH || !kernels) return fail(PH_ERR_ARG, "bad arguments");
    *kernels = g->kernels;
    return PH_OK;
}

}  // extern "C"
