// Host-side state of a simulation handle and of its workspace layout,
// shared by the translation units of the C ABI (lbm_api.cu, lbm_batch.cu).
#pragma once

#include <vector>

#include "lbm_internal.cuh"

namespace lbm {

// Byte offsets of the buffers carved from the caller's workspace.
struct Layout {
    int pitch = 0;
    long long ps = 0;
    size_t nslots = 0;
    size_t A[2], own[2], flags, slot_node, slot_q, slot_base, cur, nxt, prev, force, pos4, prc, lsum,
        geo[3], pconst, lorder, status, pack, stage, newborn, near, dsum, cells[2], runs[2], total;
    int newborn_cap = 0;
    int cell_gx = 1, cell_gy = 1; // cell grid of the pair screening
    double cell_side = 1.0;
    int stage_rows = 0;
};

} // namespace lbm

struct lbm_handle {
    lbm_domain d;
    lbm_params prm;
    int np = 0;
    lbm::Layout L;
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    cudaStream_t side = nullptr;           // branch for k_boundary beside k_stream_collide
    cudaStream_t far = nullptr;            // branch for the far-tile pass beside the particle kernels
    cudaEvent_t fork = nullptr, join = nullptr, fork0 = nullptr, join0 = nullptr;
    lbm::Dev D;
    void *A[2]; // planes of D.storage elements
    int *own[2];
    int parity = 0;
    int since_order = 0; // steps since the link order was last computed
    cudaGraphExec_t gexec[4][2] = {};               // 2^l steps (l = 0..3) from each parity
    bool timing = false;
    struct Ev {
        cudaEvent_t a, b;
        int kind;
    };
    std::vector<Ev> ev;
    size_t ev_used = 0;
    double acc_ms[lbm::kNumKernelKinds] = {};
    long long acc_n[lbm::kNumKernelKinds] = {};
    long long launches = 0;
    int sticky = LBM_OK;
};

