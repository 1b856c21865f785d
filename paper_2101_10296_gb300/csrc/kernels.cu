// Register-resident cone kernels for sm_103a.
//
// Per (cone, parameter point) the kernel evolves the cone's state vector
// |+>^n through p layers of U_P(gamma_l) = exp(-i gamma_l C) and
// U_B(beta_l) = prod exp(-i beta_l X_q) (Sec. 2.2) and reduces
// <Z_0 Z_1> = sum_z |psi_z|^2 (-1)^(z_0 xor z_1) (Sec. 2.3-2.4).
//
// Gate pruning (Sec. 2.3, reverse causal cone): a mixer of layer l only acts
// on qubits within distance p-l of the edge -- elsewhere it commutes through
// the observable and cancels -- so layer l mixes qubits [0, k_l) and the
// outermost shell (distance p) is never mixed.  Those shell qubits therefore
// stay classical: for each assignment of them the remaining amplitudes
// evolve independently.  A thread holds 2^R amplitudes (the R lowest qubits)
// in registers; qubits R..R+4 live on lane bits of the warp (butterflies via
// shuffles); higher qubits are shell bits that index independent threads.
// This is the full 2^n state vector, computed in 2^(n-R) register-sized
// slices that never leave the SM.
//
// Stored form.  The registers hold s with psi = K X^F s: K is a scalar whose
// |K|^2 = sigma each lane tracks in FP32 from a table rounded once from FP64,
// and F is a set of bit flips.  exp(-i beta X) = kappa (I - i tau X) with
// |tau| <= 1 (tau = tan beta), or, when |tan beta| > 1, the same form for
// beta - pi/2 times exp(-i pi/2 X) = -i X; that X is not applied but added
// to F.  Each butterfly output is then two FMAs.  A phase lookup needs
// C(z xor F), which is popcount(M(z) ^ M(F)) since the cut word M is linear,
// so F costs one XOR into the per-thread part of M per flipped layer.
// Every layer flips qubits 0 and 1 together, so Z_0 Z_1 never changes sign.
//
// Numerics: complex64 amplitudes and FP32 arithmetic; the phase table
// exp(-i gamma c), tan and the kappa powers are computed in FP64 and rounded
// once; lane partial sums are reduced across the warp in FP32 and
// accumulated across warps, cones and orbits in FP64 (atomicAdd).
#include <algorithm>
#include <map>
#include <set>
#include <mutex>
#include <tuple>

#include "cone_kernel.cuh"

namespace qaoa {
namespace {

__global__ void prep_kernel(const PrepArgs a) {
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t GP = int64_t(a.G) * a.P;
    const int p2 = 2 * a.p;
    // one row per (graph, point, layer): exp(-i gamma c) for c = 0 .. cmax1-1 by the
    // recurrence z_(c+1) = z_c exp(-i gamma) in FP64 (one sincos per row; after at most
    // 64 steps its rounding error, ~1e-14, is far below the FP32 table's own)
    for (int64_t r = tid; r < GP * a.p; r += stride) {
        const int64_t l = r % a.p;
        const int64_t gj = r / a.p;
        double sn, cs;
        sincos(a.params[gj * p2 + l], &sn, &cs);
        float2 *row = a.lut + r * a.cmax1;
        double zr = 1.0, zi = 0.0;
        for (int c = 0; c < a.cmax1; ++c) {
            row[c] = make_float2(float(zr), float(zi));
            const double nr = fma(zr, cs, zi * sn);  // (zr + i zi)(cos gamma - i sin gamma)
            zi = fma(zi, cs, -(zr * sn));
            zr = nr;
        }
    }
    for (int64_t i = tid; i < GP * a.p; i += stride) {
        const int64_t gj = i / a.p, l = i % a.p;
        double sn, cs;
        sincos(a.params[gj * p2 + a.p + l], &sn, &cs);
        const bool flip = fabs(sn) > fabs(cs);
        const double tau = flip ? -cs / sn : sn / cs;
        const double k2 = flip ? sn * sn : cs * cs;
        a.mix[i] = make_float2(float(tau), flip ? 1.f : 0.f);
        double pw = 1.0;
        for (int k = 0; k < kKpow; ++k) {
            a.kpow[i * kKpow + k] = float(pw);
            pw *= k2;
        }
    }
    for (int64_t i = tid; i < GP; i += stride) a.energy[i] = a.half_edges[i / a.P];
    if (a.grad)
        for (int64_t i = tid; i < GP * p2; i += stride) a.grad[i] = 0.0;
    if (a.terms)
        for (int64_t i = tid; i < a.n_reps * a.P; i += stride) a.terms[i] = 0.0;
}

// C(z) for every z of one cone, through the same cut-word routine.
template <typename MT>
__global__ void cut_table_kernel(const DevCone *__restrict__ C, uint8_t *__restrict__ out, int32_t n,
                                 int32_t *status) {
    constexpr int R = kRegBitsEnergy;
    const int64_t threads = int64_t(1) << (n > R ? n - R : 0);
    const int nreg = n < R ? n : R;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < threads;
         t += int64_t(gridDim.x) * blockDim.x) {
        CutWords<R, MT> cw;
        cw.init(C, n, t);
        cw.visit([&](int i, int c) {
            if (!(i >> nreg)) out[(t << R) | i] = uint8_t(c);
        });
    }
    if (n != C->n && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, 1);
}

}  // namespace

// Persistent grid size for (kernel, block, dynamic shared memory) on the
// current device, computed once and cached (the runtime query is not free
// and small evaluations are dominated by host overhead).
int occupancy_grid(const void *fn, int block, size_t smem) {
    struct Key {
        const void *fn;
        int block, dev;
        size_t smem;
        bool operator<(const Key &o) const {
            return std::tie(fn, block, dev, smem) < std::tie(o.fn, o.block, o.dev, o.smem);
        }
    };
    static std::mutex mu;
    static std::map<Key, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const Key key{fn, block, dev, smem};
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, block, smem);
    if (per < 1) per = 1;
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = sms * per;
    return sms * per;
}

int sm_count() {
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = sms;
    return sms;
}

int smem_per_block(int blocks) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({dev, blocks});
    if (it != cache.end()) return it->second;
    int per_sm = 0, reserved = 0;
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    const int v = std::max(0, per_sm / std::max(blocks, 1) - reserved);
    cache[{dev, blocks}] = v;
    return v;
}

cudaError_t launch_prep(const PrepArgs &a, cudaStream_t s) {
    // threads for the widest loop: table rows, gradient zeroing or term zeroing
    int64_t work = int64_t(a.G) * a.P * 2 * a.p;
    if (a.terms) work = std::max<int64_t>(work, a.n_reps * a.P);
    int64_t blocks = (work + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    prep_kernel<<<int(blocks), 256, 0, s>>>(a);
    return cudaGetLastError();
}

int reg_energy_grid(bool wide, size_t smem) {
    return wide ? occupancy_grid((const void *)reg_cone_kernel<kRegBitsEnergy, uint64_t, false, 0>, kRegBlock, smem)
                : occupancy_grid((const void *)reg_cone_kernel<kRegBitsEnergy, uint32_t, false, 0>, kRegBlock, smem);
}
cudaError_t reg_prepare() {
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(dev)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute((const void *)reg_cone_kernel<kRegBitsEnergy, uint32_t, false, 0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kRegMaxSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)reg_cone_kernel<kRegBitsEnergy, uint64_t, false, 0>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kRegMaxSmem);
    if (e == cudaSuccess) e = reg_grad_prepare();
    if (e == cudaSuccess) e = reg_p1_prepare();
    if (e == cudaSuccess) done.insert(dev);
    return e;
}

cudaError_t launch_reg_energy(const RegLaunch &a, bool wide, int grid, cudaStream_t s) {
    const size_t sm = reg_smem_bytes(a.jpt, a.p, a.cmax1, false);
    if (wide)
        reg_cone_kernel<kRegBitsEnergy, uint64_t, false, 0><<<grid, kRegBlock, sm, s>>>(a);
    else
        reg_cone_kernel<kRegBitsEnergy, uint32_t, false, 0><<<grid, kRegBlock, sm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cut_table(const DevCone *cone, uint8_t *out, int32_t n, int32_t *status, cudaStream_t s) {
    int64_t threads = int64_t(1) << (n > kRegBitsEnergy ? n - kRegBitsEnergy : 0);
    int64_t blocks = (threads + 127) / 128;
    if (blocks > 65535) blocks = 65535;
    cut_table_kernel<uint64_t><<<int(blocks), 128, 0, s>>>(cone, out, n, status);
    return cudaGetLastError();
}

}  // namespace qaoa
