// Device copy of a plan: cone descriptors, register-kernel work lists and
// large-state shapes (shared by the C-ABI translation units).
#pragma once

#include <utility>
#include <vector>

#include "big.cuh"
#include "device.cuh"

struct DevWork {
    int32_t *slot_cone = nullptr;   // plan index of every slot's cone; bit 31 set in padding slots
    int32_t *warp_graph = nullptr;  // graph of every warp's slots
    void *rec_hi = nullptr;         // [S][slots] cut words (uint32 or uint64, see RegWork)
    float *rec_wk = nullptr;        // [S][slots] block multiplicities
    uint2 *rec_cw = nullptr;        // depth-1 lists: [kP1Blocks][slots] cut values and multiplicity
    int64_t slots = 0, warps = 0;
    int32_t n = 0;
};

// Cones of one shape (n_in, k_1..k_p) on the large-state path.  Items of a
// call are numbered cone by cone (P * n_blocks each).
struct BigShape {
    int32_t n_in = 0;
    std::vector<int32_t> k;
    std::vector<int32_t> cones;   // plan indices
    std::vector<int64_t> ystart;  // [cones + 1] prefix of the cones' shell-block counts
    int32_t *d_cones = nullptr;
    int64_t *d_ystart = nullptr;
    bool split_e = false, split_g = false;  // core-tile schedule usable (energy, adjoint)
    std::vector<qaoa::BigPass> fwd, grad;   // general schedule
};

struct qaoa_device_plan {
    int device = -1;
    qaoa::DevCone *cones = nullptr;
    int64_t n_cones = 0;
    DevWork reg_e;       // work list of the energy kernels
    DevWork reg_g[2];    // of the adjoint kernels with 4 and 5 register qubits
    DevWork reg_p1;      // of the depth-1 kernel (p = 1 plans whose register cones all mix qubits 0, 1 only)
    std::vector<BigShape> big;
    size_t big_budget = size_t(1) << 30;  // scratch bytes per call for big cones
    double *half_edges = nullptr;
    uint64_t *shell = nullptr;  // shell table (see DevCone)
    int32_t *status = nullptr;
    int32_t cmax1 = 1;
    int64_t n_big = 0;
    int32_t points_per_task = 0;  // 0: default (see qaoa_tuning_t)
    int32_t blocks_per_sm = 0;
    int32_t reg_bits_grad = 0;    // adjoint register qubits (4 or 5; 0: 4)
    int32_t chunk_window = 10;    // largest outer window of a shared-memory chunk pass (6..10)
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    int64_t all_launches = 0;
};

// The register kernels' view of a work list.
inline qaoa::RegWork reg_work(const qaoa_device_plan *d, const DevWork &w) {
    qaoa::RegWork r;
    r.cones = d->cones;
    r.slot_cone = w.slot_cone;
    r.warp_graph = w.warp_graph;
    r.rec_hi = w.rec_hi;
    r.rec_wk = w.rec_wk;
    r.rec_cw = w.rec_cw;
    r.n_cones = w.n;
    r.slots = w.slots;
    r.warps = w.warps;
    return r;
}
