// Device-side data layout shared by the kernels and the C-ABI launch code.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/qaoa.h"

namespace qaoa {

// One simulated cone (representative edge), as the kernels read it.
//
// Local qubits: 0 = u, 1 = v, then by (distance, vertex id).  `col[q]` has
// bit e set when cone edge e touches qubit q, so for a basis index z the
// word M(z) = XOR over set bits q of z of col[q] has bit e set exactly when
// edge e is cut, and the cut value is C(z) = popcount(M(z)).  M is linear
// over GF(2): M(hi | lo) = M(hi) ^ M(lo), which the kernels use to split z
// into a per-thread part and a per-register part.
struct alignas(16) DevCone {
    int32_t graph;   // graph index g
    int32_t n;       // qubits
    int32_t n_in;    // inner qubits: the only ones any mixer touches
    int32_t m;       // cut-word bits: cone edges, an edge of weight w counting |w|
    int32_t k[QAOA_MAX_P];  // layer l mixes qubits [0, k[l])
    double weight;   // orbit size
    int64_t rep;     // row of this cone in terms[]
    int64_t n_blocks;  // shell blocks: prod over shell classes of (size + 1)
    int32_t n_cls;     // shell classes
    int32_t cls_off;   // this cone's entries in the shell table
    uint64_t col[QAOA_MAX_CONE_QUBITS];
    uint64_t pw[QAOA_MAX_P];  // M of the qubits layer l mixes, [0, k[l])
    uint64_t neg;             // bits of negative-weight edges (already in the shell table's words)
};

// Shell table, per cone from cls_off.  n_cls < 0: an explicit list of
// n_blocks (shell word, multiplicity as float bits) pairs -- the blocks left
// after merging those related by the cone's symmetries.  Otherwise per
// class c of size s: word 0 = s,
// words 1..s+1 = XOR of col[] over the class's first 0..s qubits, words
// s+2..2s+2 = binomial(s, 0..s) as float bits.  Block beta of a cone is the
// mixed-radix number (n_0, n_1, ...) with 0 <= n_c <= s_c, least significant
// class first: its shell word is the XOR of the classes' prefix words for
// n_c and its multiplicity the product of binomial(s_c, n_c).
__device__ __forceinline__ uint64_t shell_block(const DevCone *__restrict__ C, const uint64_t *__restrict__ tab,
                                                uint32_t beta, float &mult) {
    if (C->n_cls < 0) {  // explicit list: (word, multiplicity bits) per block
        if (int64_t(beta) >= C->n_blocks) {
            mult = 0.f;
            return 0;
        }
        const uint64_t *e = tab + C->cls_off + 2 * size_t(beta);
        mult = __uint_as_float(uint32_t(e[1]));
        return e[0];
    }
    const uint64_t *t = tab + C->cls_off;
    uint64_t m = 0;
    float w = 1.f;
    for (int c = 0; c < C->n_cls; ++c) {
        const uint32_t sz = uint32_t(t[0]);
        const uint32_t q = beta / (sz + 1);
        const uint32_t nc = beta - q * (sz + 1);
        beta = q;
        m ^= t[1 + nc];
        w *= __uint_as_float(uint32_t(t[2 + sz + nc]));
        t += 2 * sz + 3;
    }
    mult = w;
    return m;
}

// Work list of the register-resident kernels.  An inner block of 2^n_in
// amplitudes takes G = 2^max(n_in - R, 0) threads (R register qubits per
// thread); when n_in < R a thread holds S = 2^(R - n_in) blocks.  A (cone,
// point) needs T_c = ceil(B / S) * G threads for its B shell blocks.  Cones
// are sorted by (G descending, graph) and packed back to back, T_c slots
// each; a graph change is padded to the next multiple of 32 slots, so every
// cone's first slot is aligned to min(G, 32) lanes and no warp spans two
// graphs.  A warp task covers 32 consecutive slots for `jpt` consecutive
// parameter points of that graph.
//
// Slot records: everything a thread derives from its slot before the first
// point does not depend on the parameters, so it is computed once at upload.
// For register index i = 4k + r of slot s's thread (r = bits 0-1: qubits u,
// v), rec_hi[k * slots + s] is the part of the cut word M(z_i) that does not
// involve qubits 0 and 1 -- the thread's inner qubits, its shell block's word
// and register bits 2.. -- and rec_wk[k * slots + s] the multiplicity of the
// block index i belongs to (0 past the cone's blocks and in padding slots).
// Words are uint32 when every cone has at most 32 cut bits, else uint64.
struct RegWork {
    const DevCone *cones = nullptr;       // plan order
    const int32_t *slot_cone = nullptr;   // plan index of each slot's cone; bit 31: padding slot
    const int32_t *warp_graph = nullptr;  // the graph of each warp's slots
    const void *rec_hi = nullptr;         // slot records (above)
    const float *rec_wk = nullptr;
    const uint2 *rec_cw = nullptr;        // depth-1 work lists: per block the four cut values and the multiplicity
    int32_t n_cones = 0;
    int64_t slots = 0;                    // slots per point (with padding; a multiple of 32)
    int64_t warps = 0;                    // warps per point
};

// Per-point mixer data.  exp(-i beta X) = kappa (I - i tau X) with
// tau = tan(beta), kappa = cos(beta) when |tan(beta)| <= 1; otherwise the
// kernel applies exp(-i (beta - pi/2) X) (tau = -cot(beta), kappa = sin(beta))
// followed by exp(-i pi/2 X) = -i X, whose bit flip it tracks instead of
// applying (flip = 1).  kpow[k] = kappa^(2k), rounded once from FP64.
constexpr int kKpow = QAOA_MAX_CONE_QUBITS + 1;

struct RegLaunch {
    RegWork work;
    int64_t n_points;
    int32_t jpt;              // parameter points per warp task
    int32_t p;
    int32_t cmax1;            // phase-table row length (max cone edges + 1)
    const float2 *lut;        // [G][P][p][cmax1]  exp(-i gamma_l c)
    const float2 *mix;        // [G][P][p]         (tau_l, flip_l)
    const float *kpow;        // [G][P][p][kKpow]  kappa_l^(2k)
    double *energy;           // [G][P]
    double *grad;             // [G][P][2p] or null
    double *terms;            // [reps][P] or null
    int32_t *status;
    int32_t norm = 0;         // 1: the observable is the identity (terms = sum |psi|^2, energy unused)
};

struct PrepArgs {
    const double *params;     // [G][P][2p]
    int32_t G, p, cmax1;
    int64_t P;
    const double *half_edges; // [G]
    float2 *lut;
    float2 *mix;
    float *kpow;
    double *energy;
    double *grad;             // may be null
    double *terms;            // may be null
    int64_t n_reps;
};

// launchers (kernels.cu)
cudaError_t launch_prep(const PrepArgs &a, cudaStream_t s);
// wide = some cone has more than 32 edges (64-bit cut words).  Dynamic
// shared memory: 4 warps x jpt x p x cmax1 float2 (phase tables).
cudaError_t launch_reg_energy(const RegLaunch &a, bool wide, int grid, cudaStream_t s);
// rg: register qubits per thread of the adjoint kernel (4 or 5)
cudaError_t launch_reg_grad(const RegLaunch &a, bool wide, int rg, int grid, cudaStream_t s);
cudaError_t launch_cut_table(const DevCone *cone, uint8_t *out, int32_t n, int32_t *status, cudaStream_t s);
// occupancy-sized persistent grids for a given dynamic shared memory size
int reg_energy_grid(bool wide, size_t smem);
int sm_count();  // multiprocessors of the current device (cached)
// Dynamic shared memory a block may use when `blocks` blocks share one
// multiprocessor of the current device: the multiprocessor's shared memory
// split evenly, less what the hardware reserves per block (cached).
int smem_per_block(int blocks);
int reg_grad_grid(bool wide, size_t smem, int p, int rg);
cudaError_t reg_grad_prepare();
// Raises the register kernels' dynamic shared memory limit to kRegMaxSmem
// (once per device; called at upload, outside any stream capture).
cudaError_t reg_prepare();
constexpr int kRegBlock = 128;
constexpr int kRegMaxSmem = 96 * 1024;

#ifndef QAOA_REG_BITS_ENERGY
#define QAOA_REG_BITS_ENERGY 5
#endif
#ifndef QAOA_REG_BITS_GRAD
#define QAOA_REG_BITS_GRAD 4
#endif
// register qubits per thread of the energy and the adjoint kernels
constexpr int kRegBitsEnergy = QAOA_REG_BITS_ENERGY;
constexpr int kRegBitsGrad = QAOA_REG_BITS_GRAD;
constexpr int kLaneBits = 5;
// resident 128-thread blocks per SM the register allocation is sized for
// (the adjoint with four register qubits; with five it holds twice the
// amplitudes and is sized for two)
#ifndef QAOA_GRAD_MIN_BLOCKS
#define QAOA_GRAD_MIN_BLOCKS 4
#endif
constexpr int kGradMinBlocks = QAOA_GRAD_MIN_BLOCKS;
constexpr int kGradMinBlocks5 = 2;
constexpr int kEnergyMinBlocks = 3;
// largest inner part the register kernels take (both must fit)
constexpr int kRegMaxInner = (kRegBitsEnergy < kRegBitsGrad ? kRegBitsEnergy : kRegBitsGrad) + kLaneBits;

// The register kernels stage every lane's share of each output of a point
// (the energy, and with the adjoint the 2p derivatives) in shared memory and
// sum it over the warp for a group of points at once: per warp, outputs x
// group points x 32 lanes FP32 partials.
__host__ __device__ constexpr int reg_outputs(int p, bool grad) { return grad ? 1 + 2 * p : 1; }
__host__ __device__ constexpr int reg_group(int p, bool grad) {
    // at most 24 x 32 partials (3 KB) per warp, so that the point tables and
    // this buffer leave room for four blocks per SM
    return reg_outputs(p, grad) * 8 <= 24 ? 8
           : reg_outputs(p, grad) * 4 <= 24 ? 4
           : reg_outputs(p, grad) * 2 <= 24 ? 2 : 1;
}
// kappa powers a register kernel reads: kappa^(2k) for k <= its largest inner part
constexpr int kRegKpow = 10;
// 32-bit words of per-lane cone fields a register kernel keeps in shared
// memory: the layers' k (one byte each, two words), the adjoint's cut-value
// offset, and per layer the flip word M(F_l) as two words
__host__ __device__ constexpr int reg_lane_words(int p) { return 3 + 2 * p; }
// Depth-1 kernel (p1_kernel.cu): shell blocks per thread, and the resident
// blocks per SM its register allocation is sized for.  Its work lists hold
// per graph the shell blocks of all the graph's cones back to back, block k
// of slot s as rec_cw[k * slots + s] = (c_0 | c_1 << 8 | c_2 << 16 | c_3 <<
// 24, bits of W), c_a the cut value of amplitude a = z_u + 2 z_v and W the
// block's multiplicity x orbit size x 2^-n; the amplitudes may be relabelled
// by X_u, X_v or both (a -> a xor f), with W negated for a single flip, so
// that c_0 is the middle one of the four; warp_graph as for the other lists.
constexpr int kP1Blocks = 16;
constexpr int kP1GradMinBlocks = 6;
constexpr int kP1EnergyMinBlocks = 8;
// Dynamic shared memory of a depth-1 block: per warp jpt phase tables, jpt
// (tau, kappa^4) pairs, the records of its 32 slots and the reduction buffer.
// Points per reduction group of the depth-1 kernel (see reg_flush): four for
// the adjoint, whose three outputs would otherwise take 3 KB per warp
__host__ __device__ constexpr int reg_p1_group(bool grad) { return grad ? 4 : 8; }
inline size_t reg_p1_smem_bytes(int jpt, int cmax1, bool grad) {
    return size_t(kRegBlock / 32) *
           (size_t(jpt) * (cmax1 + 1) * sizeof(float2) + size_t(kP1Blocks) * 32 * sizeof(uint2) +
            size_t(reg_outputs(1, grad)) * reg_p1_group(grad) * 32 * sizeof(float));
}
int reg_p1_grid(bool grad, size_t smem);
cudaError_t reg_p1_prepare();
cudaError_t launch_reg_p1(const RegLaunch &a, bool grad, int grid, cudaStream_t s);

// Dynamic shared memory of a register-kernel block: per warp and point the
// phase tables (p x cmax1 float2), the mixer data (p float2) and the kappa
// powers (p x kRegKpow float) of jpt points, the reduction buffer, and the
// lanes' cone fields (reg_lane_words).
inline size_t reg_smem_bytes(int jpt, int p, int cmax1, bool grad) {
    return size_t(kRegBlock / 32) *
           (size_t(jpt) * p * (cmax1 + 1) * sizeof(float2) +
            (size_t(jpt) * p * kRegKpow + size_t(reg_outputs(p, grad)) * reg_group(p, grad) * 32 +
             size_t(reg_lane_words(p)) * 32) * sizeof(float));
}

}  // namespace qaoa
