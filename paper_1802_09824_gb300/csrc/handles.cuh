// Handle layouts (host structs owning device buffers).
#pragma once

#include <vector>

#include "phpp_internal.cuh"

struct ph_leaves {
    uint32_t kind = phpp::KIND_LEAVES;
    cudaStream_t last_stream = nullptr;
    // valid: the last build completed, so the buffers hold a tree (a build
    // that fails part-way, e.g. out of memory, leaves the handle invalid
    // until the next successful build); generation counts successful builds
    bool valid = false;
    uint64_t generation = 0;
    int64_t n = 0;
    int32_t n_boxes = 0;
    int32_t n_cells = 0;
    int32_t key_bits = 21;       // T
    int32_t group_size = 32;
    int32_t poly_degree = 10;
    int32_t max_leaf = 32;
    int32_t key_kind = PH_KEY_MORTON;
    int32_t level_bits = 1;      // key bits per level of the leaf hierarchy (1 or 3)
    int32_t pp_variant = 0;      // PP kernel register/occupancy variant (0: 2 blocks/SM, 1: 3)
    int32_t queue_order = 0;     // PP queue: 0 = groups by decreasing cost, 1 = group order
    bool tree_leaves = false;    // some box has theta > 0: leaf mass-centre particles are made
    std::vector<phpp::BoxDev> boxes_host;
    // device buffers
    phpp::DevBuf boxes;          // BoxDev[n_boxes]
    phpp::DevBuf box_first;      // int32[n_boxes + 1]  first particle row of each box
    phpp::DevBuf in_pos;         // staging copy of host positions
    phpp::DevBuf in_mass;        // staging copy of host masses
    phpp::DevBuf keys, keys_alt; // uint64[n]
    phpp::DevBuf vals, vals_alt; // int32[n]
    phpp::DevBuf xw;             // double[3n] wrapped positions in sorted order
    phpp::DevBuf mass_sorted;    // float[n]
    phpp::DevBuf cell_first;     // int32[n_cells + 1]
    phpp::DevBuf leaf_flag, group_flag;   // int32[n]
    phpp::DevBuf leaf_scan, group_scan;   // int32[n + 1]
    phpp::DevBuf leaf_first;     // int32[n + 1]
    phpp::DevBuf group_first;    // int32[n + 1]
    phpp::DevBuf leaf_ref;       // double[3 n]
    phpp::DevBuf leaf_c4, leaf_h4;        // float4[n] (centre in cell frame, half extents)
    phpp::DevBuf group_ref;      // double[3 n]
    phpp::DevBuf group_c4, group_h4;      // float4[n]
    phpp::DevBuf leaf_r4, group_r4;       // float4[n]: the reference points in FP32 (exact; see k_boxes)
    phpp::DevBuf box_ext;                 // long long[12 n]: extent accumulators of leaves, then groups (build scratch)
    phpp::DevBuf work;                    // direct-mode PP: group queue and counters (32 B)
    phpp::DevBuf acc_tmp;                 // direct-mode PP into a host buffer: device copy of acc
    phpp::DevBuf table;                   // PH_G_TABLE: float2[4097] factor nodes (value, slope x spacing)
    double table_rs = 0.0, table_rcut = 0.0;   // the rs, rcut the table was made for
    phpp::DevBuf group_cell;     // int32[n] global ground cell of each group
    phpp::DevBuf group_box;      // int32[n]
    phpp::DevBuf pos_leaf;       // float4[2n]: particles, then one mass-centre particle per leaf (theta > 0)
    phpp::DevBuf pos_group;      // float4[n]
    phpp::DevBuf cell_leaf_first;// int32[n_cells + 1]
    phpp::DevBuf counts;         // int32[4]: n_leaves, n_groups (device copies)
    phpp::DevBuf status;         // uint32 device status word
    phpp::DevBuf temp;           // scan / sort scratch
    bool keys_in_alt = false;
    // active-particle mode (adaptive time steps): when `active` (caller-order
    // flags, device) is set, the build lists the groups holding a flagged
    // particle and the pair builder gives entries to those groups only; the
    // other groups get empty lists, so the PP kernel sums nothing for them
    // (and writes zero accelerations) at almost no cost
    const uint8_t *active = nullptr;
    phpp::DevBuf group_act;      // int32[n + 1]: group flags
    phpp::DevBuf group_act_scan; // int32[n + 1]: their exclusive scan
    phpp::DevBuf active_list;    // int32[n]: the active groups in order; count in counts[2]
};

struct ph_pairs {
    uint32_t kind = phpp::KIND_PAIRS;
    cudaStream_t last_stream = nullptr;
    // valid: the last ph_leaf_pairs completed; leaves_generation: the build
    // of built_from the list was made for (a later build of the leaves makes
    // the list stale)
    bool valid = false;
    uint64_t leaves_generation = 0;
    int64_t capacity = 0;        // entries
    bool fixed_capacity = false;
    int64_t n_pairs = 0;         // host copy (valid after sizing sync)
    int32_t n_groups_cap = 0;
    const ph_leaves *built_from = nullptr;
    phpp::DevBuf group_cnt;      // int64[n + 1]
    phpp::DevBuf group_off;      // int64[n + 1]
    phpp::DevBuf entries;        // float4[capacity]: offset xyz, first source particle
    phpp::DevBuf ecount;         // uint8[capacity]: particles in the entry's leaf - 1
    phpp::DevBuf work;           // int32 queue counter + int64 work counters
    phpp::DevBuf status;         // uint32
    phpp::DevBuf temp;
    phpp::DevBuf acc_tmp;        // float[3n] when the caller passes host memory
    // the PP queue's order (groups by decreasing cost), made by the count
    // pass when these buffers exist; `ordered` says the last list has it
    phpp::DevBuf group_key;      // uint8[n]: 255 - cost bucket
    phpp::DevBuf group_order;    // int32[n]: groups in queue order
    phpp::DevBuf order_temp;     // histograms and scan scratch
    bool ordered = false;
};

namespace phpp {
// Refuses a leaves handle without a completed build and a pairs handle that
// is incomplete or made for another build (PH_ERR_STATE), so no kernel ever
// reads buffers that a failed or newer build left behind.
int check_built(const ph_leaves *lv, const ph_pairs *pr);

// A fingerprint of the device buffers of a leaves (and pairs) handle: their
// addresses and sizes.  A captured graph holds these addresses; it may only
// be replayed while the fingerprint is unchanged.
uint64_t buffers_fingerprint(const ph_leaves *lv, const ph_pairs *pr);
}  // namespace phpp
