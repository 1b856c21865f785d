// Register-resident cone kernel template, included by kernels.cu (energy
// instantiations, phase tables, cut tables) and kernels_grad.cu (adjoint
// instantiations), which compile in parallel.
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
// once; each lane's partial of an output is summed over the warp with
// compensated FP32 additions (the shell blocks' derivative terms cancel), and
// across warps, cones and orbits in FP64 (atomicAdd).
#pragma once

#include "reg_common.cuh"

namespace qaoa {
namespace {

template <typename MT>
__device__ __forceinline__ int popc_t(MT x);
template <>
__device__ __forceinline__ int popc_t<uint32_t>(uint32_t x) {
    return __popc(x);
}
template <>
__device__ __forceinline__ int popc_t<uint64_t>(uint64_t x) {
    return __popcll(x);
}

// Cut word of basis index z = (t << R) | i, split as lo[i & 3] ^ hi[i >> 2]
// so that every register index's word is one XOR away (no serial chain).
// hi[] also carries the shell part of the thread and the flip word M(F).
template <int R, typename MT>
struct CutWords {
    MT lo[4];
    MT hi[1 << (R - 2)];

    __device__ __forceinline__ void init(const DevCone *__restrict__ C, int n, int64_t t) {
        const MT c0 = MT(C->col[0]), c1 = MT(C->col[1]);
        lo[0] = 0;
        lo[1] = c0;
        lo[2] = c1;
        lo[3] = c0 ^ c1;
        MT base = MT(C->neg);  // negative-weight edges (see DevCone)
        for (int q = R; q < n; ++q)
            if ((t >> (q - R)) & 1) base ^= MT(C->col[q]);
        MT cm[R - 2];
#pragma unroll
        for (int b = 0; b < R - 2; ++b) cm[b] = (2 + b < n) ? MT(C->col[2 + b]) : MT(0);
#pragma unroll
        for (int k = 0; k < (1 << (R - 2)); ++k) {
            MT v = base;
#pragma unroll
            for (int b = 0; b < R - 2; ++b)
                if ((k >> b) & 1) v ^= cm[b];
            hi[k] = v;
        }
    }
    // From the slot records (see RegWork): lo[] from the columns of qubits 0
    // and 1, hi[k] and the multiplicities wk[k] from the slot's record.
    __device__ __forceinline__ void load(const DevCone *__restrict__ C, const RegWork &W, int64_t slot,
                                         float (&wk)[1 << (R - 2)]) {
        const MT c0 = MT(C->col[0]), c1 = MT(C->col[1]);
        lo[0] = 0;
        lo[1] = c0;
        lo[2] = c1;
        lo[3] = c0 ^ c1;
        const MT *__restrict__ rh = static_cast<const MT *>(W.rec_hi);
#pragma unroll
        for (int k = 0; k < (1 << (R - 2)); ++k) {
            hi[k] = __ldg(rh + k * W.slots + slot);
            wk[k] = __ldg(W.rec_wk + k * W.slots + slot);
        }
    }
    __device__ __forceinline__ void flip(MT f) {
#pragma unroll
        for (int k = 0; k < (1 << (R - 2)); ++k) hi[k] ^= f;
    }
    // f(i, C(z_i xor F)) for every register index i
    template <class F>
    __device__ __forceinline__ void visit(F &&f) const {
#pragma unroll
        for (int i = 0; i < (1 << R); ++i) f(i, popc_t<MT>(lo[i & 3] ^ hi[i >> 2]));
    }
    // C(z_i) of every register index, one byte each (a cone has < 256 cut bits)
    __device__ __forceinline__ void pack(uint32_t (&pk)[1 << (R - 2)]) const {
#pragma unroll
        for (int k = 0; k < (1 << (R - 2)); ++k) {
            uint32_t w = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a) w |= uint32_t(popc_t<MT>(lo[a] ^ hi[k])) << (8 * a);
            pk[k] = w;
        }
    }
};

// f(i, c_i) from counts packed by CutWords::pack
template <int R, class F>
__device__ __forceinline__ void visit_packed(const uint32_t (&pk)[1 << (R - 2)], F &&f) {
#pragma unroll
    for (int i = 0; i < (1 << R); ++i) f(i, int((pk[i >> 2] >> (8 * (i & 3))) & 0xffu));
}

// (I - i tau X_q) on register qubits q < KQ (compile-time count)
template <int R, int KQ>
__device__ __forceinline__ void mix_reg_fixed(float2 (&x)[1 << R], float tau) {
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
#pragma unroll
        for (int i = 0; i < (1 << R); ++i) {
            if (i & (1 << q)) continue;
            const int j = i | (1 << q);
            const float2 a = x[i], b = x[j];
            x[i] = bfly(a, b, tau);
            x[j] = bfly(b, a, tau);
        }
    }
}

// (I - i tau X_q) on every register qubit q < k.  A layer mixes either all
// register qubits or only qubits 0 and 1 (the last layer) except in small
// cones, so those two cases are straight-line code.
template <int R>
__device__ __forceinline__ void mix_reg(float2 (&x)[1 << R], int k, float tau) {
    if (__all_sync(kFull, k >= R)) {
        mix_reg_fixed<R, R>(x, tau);
    } else if (__all_sync(kFull, k == 2)) {
        mix_reg_fixed<R, 2>(x, tau);
    } else {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (q < k) {
#pragma unroll
                for (int i = 0; i < (1 << R); ++i) {
                    if (i & (1 << q)) continue;
                    const int j = i | (1 << q);
                    const float2 a = x[i], b = x[j];
                    x[i] = bfly(a, b, tau);
                    x[j] = bfly(b, a, tau);
                }
            }
        }
    }
}

// (I - i tau X_q) on lane qubits q = R..R+4 below k (partner lane = xor).
// Mixed qubits are a prefix, so the loop stops at the first lane bit no lane
// of the warp mixes; it is not unrolled (shuffle distance is a register).
template <int R>
__device__ __forceinline__ void mix_lane(float2 (&x)[1 << R], int k, float tau) {
#pragma unroll 1
    for (int L = 0; L < kLaneBits; ++L) {
        const bool mine = (R + L) < k;
        if (!__any_sync(kFull, mine)) break;
        const int m = 1 << L;
#pragma unroll
        for (int i = 0; i < (1 << R); ++i) {
            float2 o;
            o.x = __shfl_xor_sync(kFull, x[i].x, m);
            o.y = __shfl_xor_sync(kFull, x[i].y, m);
            if (mine) x[i] = bfly(x[i], o, tau);
        }
    }
}

// sum_i w_(i>>2) |x_i|^2 (-1)^(i_0 xor i_1); with ns = +1 instead of -1 the
// identity's sum_i w |x_i|^2 (the norm)
template <int R>
__device__ __forceinline__ float zz_partial(const float2 (&x)[1 << R], const float (&wk)[1 << (R - 2)],
                                            float ns = -1.f) {
    float tot = 0.f;
#pragma unroll
    for (int k = 0; k < (1 << (R - 2)); ++k) {
        const float2 a = x[4 * k], b = x[4 * k + 1], c = x[4 * k + 2], d = x[4 * k + 3];
        const float pos = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(d.x, d.x, d.y * d.y)));
        const float neg = fmaf(b.x, b.x, fmaf(b.y, b.y, fmaf(c.x, c.x, c.y * c.y)));
        tot = fmaf(wk[k], fmaf(ns, neg, pos), tot);
    }
    return tot;
}

// Outputs reduced per unrolled copy of the reduction loop (1 keeps one copy of
// its code: the adjoint body is large enough for instruction fetch to stall).
#ifndef QAOA_FLUSH_UNROLL
#define QAOA_FLUSH_UNROLL 1
#endif
constexpr int kFlushUnroll = QAOA_FLUSH_UNROLL;

// PC > 0: the depth p is the compile-time constant PC (layer loops unrolled);
// PC = 0: p is read from the launch arguments.
template <int R, typename MT, bool GRAD, int PC>
__global__ void __launch_bounds__(kRegBlock, GRAD ? (R <= 4 ? kGradMinBlocks : kGradMinBlocks5) : kEnergyMinBlocks)
    reg_cone_kernel(const RegLaunch L) {
    constexpr int NA = 1 << R;
    extern __shared__ float2 s_tab[];
    const int lane = threadIdx.x & 31;
    const RegWork &W = L.work;
    const int p = PC > 0 ? PC : L.p;
    const int row = p * L.cmax1;  // one point's phase table
    // Per warp: the phase tables, mixer data (tau, flip) and kappa powers of
    // the task's points, and the reduction buffer: this lane's share of output
    // c (0: energy, 1 + i: gradient component i) of point jj sits at
    // [c][jj mod G][(lane + jj) mod 32] (the skew keeps the reads below free
    // of bank conflicts).
    constexpr int NOUT_C = PC > 0 ? reg_outputs(PC, GRAD) : 0;
    constexpr int G_C = PC > 0 ? reg_group(PC, GRAD) : 0;
    const int NOUT = PC > 0 ? NOUT_C : reg_outputs(p, GRAD);
    const int G = PC > 0 ? G_C : reg_group(p, GRAD);
    const int warp = threadIdx.x >> 5;
    float2 *my_tab = s_tab + warp * (L.jpt * row);
    float2 *my_mix = s_tab + (kRegBlock / 32) * (L.jpt * row) + warp * (L.jpt * p);
    float *my_kp = reinterpret_cast<float *>(s_tab + (kRegBlock / 32) * (L.jpt * (row + p))) +
                   warp * (L.jpt * p * kRegKpow);
    float *red_all = reinterpret_cast<float *>(s_tab + (kRegBlock / 32) * (L.jpt * (row + p))) +
                     (kRegBlock / 32) * (L.jpt * p * kRegKpow);
    float *red = red_all + warp * (NOUT * G * 32);
    uint32_t *my_cone =
        reinterpret_cast<uint32_t *>(red_all + (kRegBlock / 32) * (NOUT * G * 32)) + warp * (reg_lane_words(p) * 32);
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int64_t nblk = (L.n_points + L.jpt - 1) / L.jpt;
    const int64_t ntask = W.warps * nblk;
    for (int64_t task = gw; task < ntask; task += nw) {
        const int64_t jb = task / W.warps;
        const int64_t w = task - jb * W.warps;
        const int64_t j0 = jb * L.jpt;
        const int jn = int(L.n_points - j0 < L.jpt ? L.n_points - j0 : L.jpt);
        const int64_t slot = w * 32 + lane;
        // Stage the phase tables, mixer data and kappa powers of points j0 ..
        // j0+jn-1 of the warp's graph first: they depend on nothing else, so
        // their loads overlap the cone descriptor's.
        const int gwarp = __ldg(W.warp_graph + w);
        __syncwarp();  // the previous task's reads of the tables are done
        {
            // asynchronous copies (no register round trip): all of them are in
            // flight while the lanes load their slots' records and cones
            const float2 *__restrict__ src = L.lut + (int64_t(gwarp) * L.n_points + j0) * row;
            for (int e = lane; e < jn * row; e += 32) cp_async8(my_tab + e, src + e);
            const float2 *__restrict__ msrc = L.mix + (int64_t(gwarp) * L.n_points + j0) * p;
            for (int e = lane; e < jn * p; e += 32) cp_async8(my_mix + e, msrc + e);
            const float *__restrict__ ksrc = L.kpow + (int64_t(gwarp) * L.n_points + j0) * p * kKpow;
            for (int e = lane; e < jn * p * kRegKpow; e += 32)
                cp_async4(my_kp + e, ksrc + (e / kRegKpow) * kKpow + (e % kRegKpow));
        }
        // the slot's cone (every lane of a warp below W.warps has a slot) and
        // whether the slot carries work (padding slots have weight 0)
        const int32_t sc = __ldg(W.slot_cone + (slot < W.slots ? slot : W.slots - 1));
        const int ci = sc & 0x7fffffff;
        bool active = sc >= 0 && slot < W.slots;
        const DevCone *__restrict__ C = W.cones + ci;
        CutWords<R, MT> cw;
        float wk[NA / 4];
        cw.load(C, W, slot < W.slots ? slot : W.slots - 1, wk);
        int n = C->n;
        if (n < 2 || n > QAOA_MAX_CONE_QUBITS || C->n_in < 2 || C->n_in > R + kLaneBits) {
            if (active) atomicOr(L.status, 1);
            active = false;
            n = 2;
        }
        const int g = C->graph;  // the warp's graph on every lane (padded work list)
        const bool uni = __all_sync(kFull, g == gwarp);
        if (!uni && lane == 0) atomicOr(L.status, 1);
        const float wgt = float(C->weight);
        // The cone fields the point loop reads go to the lane's slots in shared
        // memory once per task: a warp's lanes read up to 32 different cone
        // structs, which do not stay in L1 from one point to the next.  Word 0
        // (1) holds k of layers 0-3 (4-7), one byte each; words 3 + 2l and
        // 4 + 2l the flip word of layer l; word 2 holds c0 =
        // m/2: Im<lambda|psi> = <psi_end|O|psi_end> is real at every point of
        // the sweep (and within every shell block), so C may be replaced by
        // C - c0 in d/d gamma, which removes the mean cut value and with it most
        // of the cancellation in the FP32 sums.
        {
            uint32_t kw[2] = {0u, 0u};
            for (int l = 0; l < p; ++l)
                kw[l >> 2] |= min(unsigned(C->k[l]), unsigned(kRegKpow - 1)) << (8 * (l & 3));
            my_cone[lane] = kw[0];
            my_cone[32 + lane] = kw[1];
            my_cone[64 + lane] = __float_as_uint(0.5f * float(C->m));
            if (PC != 1) {
                for (int l = 0; l < p; ++l) {
                    const uint64_t f = C->pw[l];
                    my_cone[(3 + 2 * l) * 32 + lane] = uint32_t(f);
                    my_cone[(4 + 2 * l) * 32 + lane] = uint32_t(f >> 32);
                }
            }
        }
        auto k_of = [&](int l) -> int { return int((my_cone[(l >> 2) * 32 + lane] >> (8 * (l & 3))) & 0xffu); };
        auto pw_of = [&](int l) -> MT {
            MT f = MT(my_cone[(3 + 2 * l) * 32 + lane]);
            if constexpr (sizeof(MT) == 8) f |= MT(my_cone[(4 + 2 * l) * 32 + lane]) << 32;
            return f;
        };
        if (!active) {
#pragma unroll
            for (int k = 0; k < NA / 4; ++k) wk[k] = 0.f;
        }
        // At p = 1 every phase lookup (the layer-1 table forward, and again for
        // d/d gamma_1) uses the cut values without flips: count them once per task.
        uint32_t pk[NA / 4];
        if constexpr (PC == 1) cw.pack(pk);
        auto visit = [&](auto &&f) {
            if constexpr (PC == 1)
                visit_packed<R>(pk, f);
            else
                cw.visit(f);
        };
        cp_async_wait_all();
        __syncwarp();  // the point tables staged above are complete and visible to the warp
        // output c of point jj: this lane's share
        auto stash = [&](int c, int jj, float v) {
            if (uni) {
                red[(c * G + (jj & (G - 1))) * 32 + ((lane + jj) & 31)] = v;
            } else {  // a warp over two graphs (never made by the planner): one atomic per lane
                const int64_t gjj = int64_t(g) * L.n_points + j0 + jj;
                atomicAdd(c == 0 ? L.energy + gjj : L.grad + gjj * 2 * p + (c - 1), f2d(v));
            }
        };
        // warp sums of the group of points ending at jj (see reg_flush)
        auto flush = [&](int jj) {
            __syncwarp();
            if (uni)
                reg_flush<kFlushUnroll>(red, NOUT, G, jj, lane, int64_t(g) * L.n_points + j0, 2 * p, L.energy,
                                        L.grad);
            __syncwarp();
        };
        for (int jj = 0; jj < jn; ++jj) {
            const int64_t j = j0 + jj;
            const float2 *lut = my_tab + jj * row;
            const float2 *mix = my_mix + jj * p;
            const float *kp = my_kp + jj * p * kRegKpow;

            float2 x[NA];
            // layer 1 phase on |+>: amplitude exp(-i gamma_1 C(z)) (2^-n/2 kept in sigma)
            visit([&](int i, int c) { x[i] = lut[c]; });
            float sig = __int_as_float((127 - n) << 23);  // 2^-n
            MT fw = 0;                                      // accumulated flip word
#pragma unroll(PC > 0 ? PC : 1)
            for (int l = 0; l < p; ++l) {
                if (l > 0) {
                    const float2 *lt = lut + l * L.cmax1;
                    visit([&](int i, int c) { x[i] = cmul(x[i], lt[c]); });
                }
                const float2 mx = mix[l];
                const int k = k_of(l);
                mix_reg<R>(x, k, mx.x);
                mix_lane<R>(x, k, mx.x);
                sig *= kp[l * kRegKpow + k];
                if (PC != 1 && mx.y != 0.f) {  // (no lookup follows a flip at p = 1)
                    const MT f = pw_of(l);
                    cw.flip(f);
                    fw ^= f;
                }
            }
            const float tl = GRAD ? zz_partial<R>(x, wk) : zz_partial<R>(x, wk, L.norm ? 1.f : -1.f);
            stash(0, jj, -0.5f * wgt * sig * tl);
            if (L.terms) {
                float tv = sig * tl;
                if (seg_sum(tv, active ? ci : -1) && active) atomicAdd(L.terms + C->rep * L.n_points + j, f2d(tv));
            }
            if constexpr (!GRAD) {
                if (PC != 1) cw.flip(fw);  // back to no flips for the next point
            } else {
                // co-state lambda = -1/2 Z_0 Z_1 psi, in the same stored form; r
                // holds Z_0 Z_1 psi (signs only) and the -1/2 goes into the weight
                float2 r[NA];
#pragma unroll
                for (int i = 0; i < NA; ++i) r[i] = ((i ^ (i >> 1)) & 1) ? make_float2(-x[i].x, -x[i].y) : x[i];
                const float gw2 = active ? -wgt : 0.f;  // 2 x (-1/2) x orbit weight
                const float sig_end = sig;
                const float c0 = __uint_as_float(my_cone[64 + lane]);
#pragma unroll(PC > 0 ? PC : 1)
                for (int l = p - 1; l >= 0; --l) {
                    const float2 mx = mix[l];
                    const float tau = mx.x;
                    const int k = k_of(l);
                    const int kr = k < R ? k : R;
                    const float *kpl = kp + l * kRegKpow;
                    float db = 0.f;
                    if (PC > 0 && l == p - 1 && __all_sync(kFull, k == 2)) {
                        // The last layer of a pruned cone mixes qubits 0 and 1 only, and
                        // r = Z_0 Z_1 x here, so the two pair terms of each qubit coincide
                        // (with p a compile-time constant; the run-time-p body stays small):
                        // Im<r|X_0 + X_1|x> = 2 [Im(x0* x1) - Im(x2* x3) + Im(x0* x2) - Im(x1* x3)]
                        // per group of four amplitudes (half the products; the 2 is in the stash).
#pragma unroll
                        for (int kk = 0; kk < NA / 4; ++kk) {
                            const float2 a = x[4 * kk], b = x[4 * kk + 1], c = x[4 * kk + 2], e = x[4 * kk + 3];
                            float d = 0.f;
                            acc_imconj(d, a, b);
                            acc_imconj(d, a, c);
                            d = fmaf(-c.x, e.y, d);
                            d = fmaf(c.y, e.x, d);
                            d = fmaf(-b.x, e.y, d);
                            d = fmaf(b.y, e.x, d);
                            db = fmaf(wk[kk], d, db);
                        }
                        db *= 2.f;
                        if (l > 0) mix_reg_fixed<R, 2>(x, -tau);
                        mix_reg_fixed<R, 2>(r, -tau);
                    } else {
                        // d/d beta_l = 2 sigma Im <r| sum_q X_q |s>, register qubits
                        // on the untouched state first
                        float d[NA / 4];
#pragma unroll
                        for (int kk = 0; kk < NA / 4; ++kk) d[kk] = 0.f;
#pragma unroll
                        for (int q = 0; q < R; ++q) {
                            if (q < k) {
#pragma unroll
                                for (int i = 0; i < NA; ++i) {
                                    if (i & (1 << q)) continue;
                                    const int i2 = i | (1 << q);
                                    acc_imconj(d[i >> 2], r[i], x[i2]);
                                    acc_imconj(d[i >> 2], r[i2], x[i]);
                                }
                            }
                        }
#pragma unroll
                        for (int kk = 0; kk < NA / 4; ++kk) db = fmaf(wk[kk], d[kk], db);
                        // lane qubits: each term is taken after the lane qubits before
                        // it were undone, which scales it by (1 + tau^2) each; kappa^2
                        // per undone qubit takes that back out
#pragma unroll 1
                        for (int Lb = 0; Lb < kLaneBits; ++Lb) {
                            const bool mine = (R + Lb) < k;
                            if (!__any_sync(kFull, mine)) break;
                            const int m = 1 << Lb;
                            float e4[NA / 4];
#pragma unroll
                            for (int kk = 0; kk < NA / 4; ++kk) e4[kk] = 0.f;
#pragma unroll
                            for (int i = 0; i < NA; ++i) {
                                float2 xo, ro;
                                xo.x = __shfl_xor_sync(kFull, x[i].x, m);
                                xo.y = __shfl_xor_sync(kFull, x[i].y, m);
                                ro.x = __shfl_xor_sync(kFull, r[i].x, m);
                                ro.y = __shfl_xor_sync(kFull, r[i].y, m);
                                if (mine) {
                                    acc_imconj(e4[i >> 2], r[i], xo);
                                    x[i] = bfly(x[i], xo, -tau);
                                    r[i] = bfly(r[i], ro, -tau);
                                }
                            }
                            if (mine) {
                                float e = 0.f;
#pragma unroll
                                for (int kk = 0; kk < NA / 4; ++kk) e = fmaf(wk[kk], e4[kk], e);
                                db = fmaf(e, kpl[Lb], db);
                            }
                        }
                        // undo the register-qubit butterflies (psi only above layer 1: below
                        // it psi is the layer-1 phase table itself, read back for d/d gamma_1)
                        if (l > 0) mix_reg<R>(x, kr, -tau);
                        mix_reg<R>(r, kr, -tau);
                    }
                    // the blocks' terms cancel across lanes: the grouped reduction
                    // adds the lanes' shares with compensation
                    stash(1 + p + l, jj, gw2 * sig * db);
                    sig *= kpl[k];
                    if (PC != 1 && mx.y != 0.f) cw.flip(pw_of(l));
                    // d/d gamma_l = 2 sigma Im <r| C |s>; then undo the phase
                    float dg4[NA / 4];
#pragma unroll
                    for (int kk = 0; kk < NA / 4; ++kk) dg4[kk] = 0.f;
                    const float2 *lt = lut + l * L.cmax1;
                    if (l > 0) {
                        visit([&](int i, int cv) {
                            dg4[i >> 2] = fmaf(float(cv) - c0, imconj(r[i], x[i]), dg4[i >> 2]);
                            const float2 ph = lt[cv];
                            x[i] = cmulc(x[i], ph);
                            r[i] = cmulc(r[i], ph);
                        });
                    } else {
                        // The un-mixed psi would be Lambda * exp(-i gamma_1 C) with
                        // Lambda = prod_l (1 + tau_l^2)^k_l from the unnormalised inverse
                        // butterflies, and sigma * Lambda = sigma at the end of the forward
                        // sweep: use the table and that sigma.
                        visit([&](int i, int cv) {
                            dg4[i >> 2] = fmaf(float(cv) - c0, imconj(r[i], lt[cv]), dg4[i >> 2]);
                        });
                    }
                    float dgs = 0.f;
#pragma unroll
                    for (int kk = 0; kk < NA / 4; ++kk) dgs = fmaf(wk[kk], dg4[kk], dgs);
                    stash(1 + l, jj, gw2 * (l > 0 ? sig : sig_end) * dgs);
                }
            }
            if ((jj & (G - 1)) == G - 1 || jj == jn - 1) flush(jj);
        }
    }
}

}  // namespace
}  // namespace qaoa
