// Large-state cone path (cones with more inner qubits than the register
// kernels hold): launch structures and pass lists.
#pragma once

#include <algorithm>
#include <vector>

#include "device.cuh"

namespace qaoa {

constexpr int kBigRegBits = 5;   // register qubits per lane in a tile
constexpr int kBigMaxOps = 40;

enum BigOpType : uint8_t {
    kOpGenPhase = 1,  // |+> times the layer-1 phase (no load)
    kOpPhase = 2,     // exp(-i gamma_l C)
    kOpMix = 3,       // exp(-i beta_l X_q), q in [q0, q1)
    kOpReduce = 4,    // <Z_0 Z_1> partial into energy / terms
    kOpLamInit = 5,   // lambda = -1/2 Z_0 Z_1 psi
    kOpUnmix = 6,     // d/d beta_l term for q in [q0, q1), then exp(+i beta_l X_q)
    kOpUnphase = 7    // d/d gamma_l term, then (q0 = 1) exp(+i gamma_l C)
};

struct BigOp {
    uint8_t type, layer, q0, q1;
};

struct BigPass {
    int32_t b;  // register window [b, b+5); lanes hold qubits 0..4
    int32_t nops;
    int32_t load_psi, store_psi, load_lam, store_lam;
    BigOp ops[kBigMaxOps];
};

struct BigLaunch {
    const DevCone *cones;
    const int32_t *cone_ids;  // this shape's cones (plan indices)
    int32_t n, n_in;          // qubits, inner qubits (shared by the shape)
    int64_t Y;                // shell blocks per (cone, point)
    const uint64_t *shell;    // shell table
    int64_t P;
    int32_t p, cmax1;
    int64_t item0, n_items;   // items (cone, point, shell) of this wave
    const float2 *lut;        // [G][P][p][cmax1]
    const float2 *cs;         // [G][P][p] (cos beta, sin beta)
    float2 *psi, *lam;        // scratch: n_items blocks of 2^n_in
    double *energy, *grad, *terms;
    int32_t *status;
    BigPass pass;
};

std::vector<BigPass> big_forward_passes(int n_in, int p, const int32_t *k);
std::vector<BigPass> big_grad_passes(int n_in, int p, const int32_t *k);
cudaError_t launch_big_prep(const double *params, int64_t GP, int p, float2 *cs, cudaStream_t s);
cudaError_t launch_big_pass(const BigLaunch &a, bool grad, int grid, cudaStream_t s);
int big_grid(bool grad);

}  // namespace qaoa
