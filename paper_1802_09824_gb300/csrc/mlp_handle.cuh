// Handle of the learned short-range factor.
#pragma once

#include "phpp_internal.cuh"

struct ph_mlp {
    uint32_t kind = phpp::KIND_MLP;
    double rs = 0, rcut = 0;     // the network was trained for rcut / rs
    float tol = 1e-3f;           // accepted largest relative error of g_hat
    float max_rel_err = 0;       // validated on the tensor-core inference path
    float last_loss = 0;
    int32_t steps_done = 0;
    phpp::DevBuf theta;          // [321] weights
    phpp::DevBuf m, v;           // Adam moments
    phpp::DevBuf z0, tgt;        // training samples
    phpp::DevBuf partial;        // per-block gradient partials
    phpp::DevBuf work;           // step counter, validation word
    phpp::DevBuf loss_hist;      // loss per step
};

namespace phpp {
void mlp_free(ph_mlp *h);
}
