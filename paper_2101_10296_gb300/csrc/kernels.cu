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
// Numerics: complex64 amplitudes and FP32 arithmetic; the phase table
// exp(-i gamma c) is computed in FP64 and rounded; the amplitude scale 2^-n
// and every sum across threads are applied / accumulated in FP64.
#include "device.cuh"

namespace qaoa {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__host__ __device__ constexpr int ctz_c(int k) {
    int c = 0;
    while (!(k & 1)) {
        k >>= 1;
        ++c;
    }
    return c;
}

// XOR of col[q] over the set bits q >= R of z = (t << R): the thread's share
// of the cut word M(z).
__device__ __forceinline__ uint64_t hi_mask(const DevCone *__restrict__ C, int R, int64_t t, int n) {
    uint64_t m = 0;
    for (int q = R; q < n; ++q)
        if ((t >> (q - R)) & 1) m ^= C->col[q];
    return m;
}

// Visits the 2^R register indices in Gray-code order, keeping the cut word
// M(t << R | idx) = mhi ^ M(idx) up to date with one XOR per step, and calls
// f(idx, C(z)).  Shared by the energy, gradient and cut-table kernels.
template <int R, class F>
__device__ __forceinline__ void gray_visit(const uint64_t (&colr)[R], uint64_t mhi, F &&f) {
    uint64_t m = mhi;
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k > 0) m ^= colr[ctz_c(k)];
        f(k ^ (k >> 1), __popcll(m));
    }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// Im(conj(a) b)
__device__ __forceinline__ float imconj(float2 a, float2 b) { return a.x * b.y - a.y * b.x; }
// exp(-i beta X) on a pair, seen from one side: me' = c me - i s other
__device__ __forceinline__ float2 rot(float2 me, float2 o, float c, float s) {
    return make_float2(c * me.x + s * o.y, c * me.y - s * o.x);
}

// exp(-i beta X_q) for every register qubit q < kl.
template <int R>
__device__ __forceinline__ void rx_reg(float2 (&x)[1 << R], int kl, float c, float s) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
        if (q < kl) {
#pragma unroll
            for (int i = 0; i < (1 << R); ++i) {
                if (i & (1 << q)) continue;
                const int j = i | (1 << q);
                const float2 a = x[i], b = x[j];
                x[i] = rot(a, b, c, s);
                x[j] = rot(b, a, c, s);
            }
        }
    }
}

// exp(-i beta X_q) for lane qubits q = R..R+4 below kl (partner lane = xor).
template <int R>
__device__ __forceinline__ void rx_lane(float2 (&x)[1 << R], int kl, float c, float s) {
#pragma unroll
    for (int L = 0; L < kLaneBits; ++L) {
        const bool mine = (R + L) < kl;
        if (__any_sync(kFull, mine)) {
#pragma unroll
            for (int i = 0; i < (1 << R); ++i) {
                const float ox = __shfl_xor_sync(kFull, x[i].x, 1 << L);
                const float oy = __shfl_xor_sync(kFull, x[i].y, 1 << L);
                if (mine) x[i] = rot(x[i], make_float2(ox, oy), c, s);
            }
        }
    }
}

// sum_i |x_i|^2 (-1)^(i_0 xor i_1)
template <int R>
__device__ __forceinline__ float zz_partial(const float2 (&x)[1 << R]) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < (1 << R); ++i) {
        const float a2 = x[i].x * x[i].x + x[i].y * x[i].y;
        acc[i & 3] += a2;  // i&3 in {0,3}: z0 == z1; {1,2}: differ
    }
    return (acc[0] + acc[3]) - (acc[1] + acc[2]);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Adds v into base[(g*P + j)*stride + comp], one atomic per warp when every
// lane's graph is the same.
__device__ __forceinline__ void add_gp(double v, double *base, int g, int64_t P, int64_t j, int stride,
                                       int comp) {
    const int lane = threadIdx.x & 31;
    const int g0 = __shfl_sync(kFull, g, 0);
    if (__all_sync(kFull, g == g0)) {
        v = warp_sum(v);
        if (lane == 0) atomicAdd(base + (int64_t(g0) * P + j) * stride + comp, v);
    } else if (v != 0.0) {
        atomicAdd(base + (int64_t(g) * P + j) * stride + comp, v);
    }
}

template <int R, bool GRAD>
__global__ void __launch_bounds__(128) reg_cone_kernel(const RegLaunch L) {
    constexpr int NA = 1 << R;
    const int lane = threadIdx.x & 31;
    const RegWork &W = L.work;
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int64_t ntask = W.warps * L.n_points;
    const int p = L.p;
    for (int64_t task = gw; task < ntask; task += nw) {
        const int64_t j = task / W.warps;
        const int64_t w = task - j * W.warps;
        const int64_t slot = w * 32 + lane;
        bool active = slot < W.slots;
        int ci = W.warp_first[w];
        if (active)
            while (W.prefix[ci + 1] <= slot) ++ci;
        const DevCone *__restrict__ C = W.cones + W.order[ci];
        int n = C->n;
        if (n < 2 || n > QAOA_MAX_CONE_QUBITS || C->n_in > R + kLaneBits) {
            if (active) atomicOr(L.status, 1);
            active = false;
            n = 2;
        }
        const int g = C->graph;
        const int64_t t = active ? slot - W.prefix[ci] : 0;
        const int nreg = n < R ? n : R;
        uint64_t colr[R];
#pragma unroll
        for (int q = 0; q < R; ++q) colr[q] = q < n ? C->col[q] : 0ull;
        const uint64_t mhi = hi_mask(C, R, t, n);
        const int64_t gj = int64_t(g) * L.n_points + j;
        const float2 *__restrict__ lut = L.lut + gj * p * L.cmax1;
        const float2 *__restrict__ mix = L.mix + gj * p;

        float2 x[NA];
        // layer 1 phase on |+>: amplitude exp(-i gamma_1 C(z)) (scale 2^-n/2 deferred)
        gray_visit<R>(colr, mhi, [&](int idx, int c) {
            const float2 ph = __ldg(lut + c);
            x[idx] = (idx >> nreg) ? make_float2(0.f, 0.f) : ph;
        });
        for (int l = 0; l < p; ++l) {
            if (l > 0) {
                const float2 *__restrict__ lt = lut + l * L.cmax1;
                gray_visit<R>(colr, mhi, [&](int idx, int c) { x[idx] = cmul(x[idx], __ldg(lt + c)); });
            }
            const float2 cs = __ldg(mix + l);
            const int kl = C->k[l];
            rx_reg<R>(x, kl, cs.x, cs.y);
            rx_lane<R>(x, kl, cs.x, cs.y);
        }
        const double scale = ldexp(1.0, -n);
        const float tl = zz_partial<R>(x);
        const double tsc = active ? double(tl) * scale : 0.0;
        if (active && !isfinite(tsc)) atomicOr(L.status, 2);
        const double w8 = C->weight;
        add_gp(-0.5 * w8 * tsc, L.energy, g, L.n_points, j, 1, 0);
        if (L.terms) {
            const int64_t Tc = int64_t(1) << (n > R ? n - R : 0);
            double tv = tsc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double ov = __shfl_xor_sync(kFull, tv, o);
                if (o < Tc) tv += ov;
            }
            const int64_t grp = Tc < 32 ? Tc : 32;
            if (active && (t & (grp - 1)) == 0) atomicAdd(L.terms + C->rep * L.n_points + j, tv);
        }
        if constexpr (GRAD) {
            // co-state lambda = -1/2 Z_0 Z_1 psi
            float2 lam[NA];
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                const float sg = ((i ^ (i >> 1)) & 1) ? 0.5f : -0.5f;
                lam[i] = make_float2(sg * x[i].x, sg * x[i].y);
            }
            const double gscale = active ? 2.0 * w8 * scale : 0.0;
            for (int l = p - 1; l >= 0; --l) {
                const float2 cs = __ldg(mix + l);
                const float c = cs.x, s = cs.y;
                const int kl = C->k[l];
                float db = 0.f;
                // d/d beta_l: 2 Im <lam| sum_q X_q |psi>; then undo exp(-i beta_l X_q)
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    if (q < kl) {
#pragma unroll
                        for (int i = 0; i < NA; ++i) {
                            if (i & (1 << q)) continue;
                            const int k2 = i | (1 << q);
                            const float2 a = x[i], b = x[k2], la = lam[i], lb = lam[k2];
                            db += imconj(la, b) + imconj(lb, a);
                            x[i] = rot(a, b, c, -s);
                            x[k2] = rot(b, a, c, -s);
                            lam[i] = rot(la, lb, c, -s);
                            lam[k2] = rot(lb, la, c, -s);
                        }
                    }
                }
#pragma unroll
                for (int Lb = 0; Lb < kLaneBits; ++Lb) {
                    const bool mine = (R + Lb) < kl;
                    if (__any_sync(kFull, mine)) {
#pragma unroll
                        for (int i = 0; i < NA; ++i) {
                            float2 xo, lo;
                            xo.x = __shfl_xor_sync(kFull, x[i].x, 1 << Lb);
                            xo.y = __shfl_xor_sync(kFull, x[i].y, 1 << Lb);
                            lo.x = __shfl_xor_sync(kFull, lam[i].x, 1 << Lb);
                            lo.y = __shfl_xor_sync(kFull, lam[i].y, 1 << Lb);
                            if (mine) {
                                db += imconj(lam[i], xo);
                                x[i] = rot(x[i], xo, c, -s);
                                lam[i] = rot(lam[i], lo, c, -s);
                            }
                        }
                    }
                }
                add_gp(gscale * double(db), L.grad, g, L.n_points, j, 2 * p, p + l);
                // d/d gamma_l: 2 Im <lam| C |psi>; then undo exp(-i gamma_l C)
                float dg = 0.f;
                const float2 *__restrict__ lt = lut + l * L.cmax1;
                gray_visit<R>(colr, mhi, [&](int idx, int cv) {
                    dg += float(cv) * imconj(lam[idx], x[idx]);
                    if (l > 0) {
                        const float2 ph = __ldg(lt + cv);
                        x[idx] = cmulc(x[idx], ph);
                        lam[idx] = cmulc(lam[idx], ph);
                    }
                });
                add_gp(gscale * double(dg), L.grad, g, L.n_points, j, 2 * p, l);
            }
        }
    }
}

__global__ void prep_kernel(const PrepArgs a) {
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t GP = int64_t(a.G) * a.P;
    const int64_t nlut = GP * a.p * a.cmax1;
    const int p2 = 2 * a.p;
    for (int64_t i = tid; i < nlut; i += stride) {
        const int64_t c = i % a.cmax1;
        const int64_t r = i / a.cmax1;
        const int64_t l = r % a.p;
        const int64_t gj = r / a.p;
        const double gam = a.params[gj * p2 + l];
        double sn, cs;
        sincos(gam * double(c), &sn, &cs);
        a.lut[i] = make_float2(float(cs), float(-sn));
    }
    for (int64_t i = tid; i < GP * a.p; i += stride) {
        const int64_t gj = i / a.p, l = i % a.p;
        double sn, cs;
        sincos(a.params[gj * p2 + a.p + l], &sn, &cs);
        a.mix[i] = make_float2(float(cs), float(sn));
    }
    for (int64_t i = tid; i < GP; i += stride) a.energy[i] = a.half_edges[i / a.P];
    if (a.grad)
        for (int64_t i = tid; i < GP * p2; i += stride) a.grad[i] = 0.0;
    if (a.terms)
        for (int64_t i = tid; i < a.n_reps * a.P; i += stride) a.terms[i] = 0.0;
}

// C(z) for every z of one cone, through the same Gray-code routine.
__global__ void cut_table_kernel(const DevCone *__restrict__ C, uint8_t *__restrict__ out, int32_t n,
                                 int32_t *status) {
    constexpr int R = kRegBitsEnergy;
    const int64_t threads = int64_t(1) << (n > R ? n - R : 0);
    const int nreg = n < R ? n : R;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < threads;
         t += int64_t(gridDim.x) * blockDim.x) {
        uint64_t colr[R];
#pragma unroll
        for (int q = 0; q < R; ++q) colr[q] = q < n ? C->col[q] : 0ull;
        const uint64_t mhi = hi_mask(C, R, t, n);
        gray_visit<R>(colr, mhi, [&](int idx, int c) {
            if (!(idx >> nreg)) out[(t << R) | idx] = uint8_t(c);
        });
    }
    if (n != C->n && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, 1);
}

int occupancy_grid(const void *fn, int block) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, block, 0);
    if (per < 1) per = 1;
    return sms * per;
}

}  // namespace

cudaError_t launch_prep(const PrepArgs &a, cudaStream_t s) {
    int64_t work = int64_t(a.G) * a.P * a.p * a.cmax1;
    int64_t blocks = (work + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    prep_kernel<<<int(blocks), 256, 0, s>>>(a);
    return cudaGetLastError();
}

int reg_energy_grid() {
    static int grid = occupancy_grid((const void *)reg_cone_kernel<kRegBitsEnergy, false>, 128);
    return grid;
}
int reg_grad_grid() {
    static int grid = occupancy_grid((const void *)reg_cone_kernel<kRegBitsGrad, true>, 128);
    return grid;
}

cudaError_t launch_reg_energy(const RegLaunch &a, int grid, cudaStream_t s) {
    reg_cone_kernel<kRegBitsEnergy, false><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reg_grad(const RegLaunch &a, int grid, cudaStream_t s) {
    reg_cone_kernel<kRegBitsGrad, true><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cut_table(const DevCone *cone, uint8_t *out, int32_t n, int32_t *status, cudaStream_t s) {
    int64_t threads = int64_t(1) << (n > kRegBitsEnergy ? n - kRegBitsEnergy : 0);
    int64_t blocks = (threads + 127) / 128;
    if (blocks > 65535) blocks = 65535;
    cut_table_kernel<<<int(blocks), 128, 0, s>>>(cone, out, n, status);
    return cudaGetLastError();
}

}  // namespace qaoa
