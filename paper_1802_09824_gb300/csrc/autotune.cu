// In-project autotuner: leaf size, local key (Morton or Peano-Hilbert),
// target group size and PP kernel shape.
//
// Every candidate (leaf_max x key_kind x pp_variant x group_size) runs the
// whole step on the caller's particles -- build, pairs, PP -- once to warm up and then
// `reps` times under CUDA events; the candidate with the smallest median
// step time wins.  The result does not depend on the knobs (only the FP32
// summation order does), so the choice is free to follow the hardware.
#include <algorithm>
#include <cstring>
#include <vector>

#include "handles.cuh"

using namespace phpp;

extern "C" {

int ph_autotune(const void *d_pos, int pos_type, const float *d_mass, const int64_t *box_offsets, int32_t n_boxes,
                const ph_params *params, int32_t reps, void *stream, ph_tune_result *out)
{
    TraceRange trace_("ph_autotune");
    if (!d_pos || !box_offsets || !params || !out || n_boxes < 1 || reps < 1 || reps > 50)
        return fail(PH_ERR_ARG, "ph_autotune: bad arguments");
    if (!is_device_ptr(d_pos) || (d_mass && !is_device_ptr(d_mass)))
        return fail(PH_ERR_ARG, "ph_autotune: positions and masses must be device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = box_offsets[n_boxes];
    float *acc = nullptr;
    int rc = cuda_check(cudaMalloc(&acc, (size_t)(n > 0 ? n : 1) * 12), "tuner output");
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc) rc = cuda_check(cudaEventCreate(&e0), "event");
    if (!rc) rc = cuda_check(cudaEventCreate(&e1), "event");
    const int leaf_sizes[] = {16, 32, 64};
    const int keys[] = {PH_KEY_MORTON, PH_KEY_HILBERT};
    const int variants[] = {0, 1};
    const int groups[] = {16, 32};
    const int lb = 1;   // binary levels (octree levels never measured faster)
    std::vector<ph_params> prm(params, params + n_boxes);
    memset(out, 0, sizeof *out);
    out->best_ms = 3.0e38f;
    ph_leaves *lv = nullptr;
    ph_pairs *pr = nullptr;
    for (int lm : leaf_sizes)
        for (int kk : keys)
            for (int pv : variants)
            for (int gs : groups) {
                if (rc || out->n_tried >= PH_TUNE_MAX) break;
                for (auto &p : prm) {
                    p.leaf_max = lm;
                    p.key_kind = kk;
                    p.level_bits = lb;
                    p.pp_variant = pv;
                    p.group_size = gs;
                }
                std::vector<float> ms;
                for (int r = 0; !rc && r <= reps; r++) {
                    rc = cuda_check(cudaEventRecord(e0, s), "event");
                    if (!rc) rc = ph_build_leaves_batched(d_pos, pos_type, d_mass, box_offsets, n_boxes, prm.data(), s, &lv);
                    if (!rc) rc = ph_leaf_pairs(lv, s, &pr);
                    if (!rc) rc = ph_pp_accel(lv, pr, PH_G_EXACT, nullptr, acc, s);
                    if (!rc) rc = cuda_check(cudaEventRecord(e1, s), "event");
                    if (!rc) rc = cuda_check(cudaEventSynchronize(e1), "event sync");
                    float t = 0.f;
                    if (!rc) rc = cuda_check(cudaEventElapsedTime(&t, e0, e1), "elapsed");
                    if (!rc && r > 0) ms.push_back(t);    // the first run warms up
                }
                if (rc) break;
                std::sort(ms.begin(), ms.end());
                const float med = ms[ms.size() / 2];
                const int k = out->n_tried++;
                out->ms[k] = med;
                out->leaf_max[k] = lm;
                out->level_bits[k] = lb;
                out->pp_variant[k] = pv;
                out->group_size[k] = gs;
                out->key_kind[k] = kk;
                if (med < out->best_ms) {
                    out->best_ms = med;
                    out->best = prm[0];
                }
            }
    if (pr) ph_free(pr);
    if (lv) ph_free(lv);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(acc);
    return rc;
}

}  // extern "C"
