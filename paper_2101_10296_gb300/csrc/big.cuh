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

// Core-tile schedule ("split"): usable when every layer after the first
// mixes only the core qubits [0, RB + 5).  The block is stored with address
// bits 0..4 = qubits RB..RB+4, bits 5..RB+4 = qubits 0..RB-1 and bits from
// RB+5 on = the outer qubits themselves, so that one warp loads a core tile
// (lanes = qubits RB..RB+4, registers = qubits 0..RB-1) with coalesced
// accesses, and an outer pass (lanes = address bits 0..4, registers = five
// address bits [b, b+5)) does too.
constexpr int kSplitRbEnergy = 5;
constexpr int kSplitRbGrad = 4;

enum SplitOuterMode : int32_t { kOuterGen = 0, kOuterMix = 1, kOuterFirst = 2 };

struct BigLaunch {
    const DevCone *cones;
    const int32_t *cone_ids;  // this shape's cones (plan indices)
    const int64_t *ystart;    // [n_shape + 1] prefix of the cones' shell-block counts
    int32_t n_shape;          // cones in the shape
    int32_t n_in;             // inner qubits (shared by the shape)
    const uint64_t *shell;    // shell table
    int64_t P;
    int32_t p, cmax1;
    int64_t item0, n_items;   // items (cone, point, shell block) of this wave
    const float2 *lut;        // [G][P][p][cmax1]
    const float4 *cs;         // [G][P][p] (cos beta, sin beta, and their FP32 rounding errors)
    const float2 *fa;         // [G][P] the first layer's factored coefficient as FP32 hi + lo
                              // (adjoint passes), or null: the hi part alone (see first_mix)
    const float2 *mix;        // [G][P][p] (tau, flip) and
    const float *kpow;        // [G][P][p][kKpow] kappa^(2k): the register kernels' mixer tables
    float2 *psi, *lam;        // scratch: n_items blocks of 2^n_in
    double *energy, *grad, *terms;
    int32_t *status;
    int32_t norm;             // 1: the observable is the identity (terms = sum |psi|^2, energy unused)
    BigPass pass;             // general schedule: the pass to run
    // core-tile schedule
    int32_t rb;               // register qubits of a core tile
    int32_t b, w0, w1;        // outer pass: register window [b, b+5), outer qubits [w0, w1) to mix
    int32_t x0, x1;           // kOuterFirst: outer qubits [x0, x1) outside the window
    int32_t mode, sign;       // SplitOuterMode; +1 mix, -1 un-mix (kOuterMix)
    int32_t load;             // core pass: load the tile (1) or generate layer 1's phase state (0)
};

// Cones of one shape share n_in and k; items of a wave are numbered cone by
// cone, point by point, shell block by shell block.
std::vector<BigPass> big_forward_passes(int n_in, int p, const int32_t *k);
std::vector<BigPass> big_grad_passes(int n_in, int p, const int32_t *k);
cudaError_t launch_big_prep(const double *params, int64_t GP, int p, float4 *cs, float2 *fa, cudaStream_t s);
cudaError_t launch_big_pass(const BigLaunch &a, bool grad, int grid, cudaStream_t s);
int big_grid(bool grad);

// Core-tile schedule: whether a shape can use it, the scratch it needs per
// item (one block; the general adjoint needs two), and one wave's launches.
bool split_ok(int n_in, int p, const int32_t *k, bool grad);
// Per-device kernel attributes (shared memory of the chunk passes), set at
// upload so that no attribute call falls inside a stream capture.
cudaError_t split_prepare();
// chunk_window: largest outer window of a shared-memory chunk pass (6..10)
cudaError_t launch_split_wave(BigLaunch B, bool grad, int chunk_window, int64_t &launches, cudaStream_t s);

}  // namespace qaoa
