// Large-state cones, core-tile schedule.
//
// In a pruned cone, layer l mixes the qubits within distance p - l of the
// edge (Sec. 2.3), so the outer inner qubits -- those at distance p - 1 --
// are mixed by the first layer only.  When every later layer mixes only the
// T = RB + 5 core qubits [0, T) of a warp tile, the state after the first
// layer's mixer decouples into 2^(n_in - T) independent core tiles:
//
//   forward   outer passes build V_U exp(-i gamma_1 C)|+> (V_U: the first
//             mixer on the outer qubits), five outer qubits per pass; the
//             core pass loads one tile, applies the first mixer to the core
//             qubits, runs layers 2..p in registers and reduces <Z_0 Z_1>.
//   adjoint   the core pass continues with lambda = -1/2 Z_0 Z_1 psi, runs
//             both states back through layers p..2 (the derivative terms of
//             those layers), takes the first mixer's terms of the core
//             qubits, un-mixes lambda alone on the core qubits and stores it
//             in place of psi.  Outer passes un-mix lambda on the outer
//             qubits; the last one evaluates the first layer's phase term
//             and the outer qubits' mixer terms against the state before the
//             first mixer, exp(-i gamma_1 C)|+>, which is known in closed
//             form (amplitude = phase-table entry of C(z)).
//
// Both derivative identities rest on the first mixer commuting with every
// X_q it contains: <lambda|X_q|psi> is the same before and after it.  Only
// one state block per item is ever stored (the general schedule stores psi
// and lambda), and psi is never written back after the core pass.
//
// Storage: address bits 0..4 = qubits RB..RB+4, bits 5..RB+4 = qubits
// 0..RB-1, higher bits = the outer qubits themselves.  A core tile is one
// warp: lane = qubits RB..RB+4, register i = qubits 0..RB-1, so the most
// often mixed qubits 0, 1 are register butterflies and <Z_0 Z_1>'s sign is a
// compile-time function of the register.  Every load and store moves 256
// contiguous bytes per warp instruction.
#include <cuda.h>  // CUtensorMap and its enums (the encoder itself is fetched from the driver at run time)

#include <mutex>
#include <set>

#include "big.cuh"
#include "big_common.cuh"

namespace qaoa {
namespace {

// The first layer's mixer in factored form, without bit flips:
// exp(-i beta X) = kappa D with D = I - i a X (a = tan beta, kappa = cos beta)
// when |tan beta| <= 1, else D = a I - i X (a = cot beta, kappa = sin beta);
// its inverse up to the same factor, D' = exp(+i beta X) / kappa, is I + i a X
// or a I + i X.  Two FMAs per output amplitude in both cases (the exact
// rotation takes four).  Only the first layer uses it: every state of the
// schedule then carries one known factor, kappa^(n_in) per amplitude of psi,
// and every derivative term is taken either before any of the first mixer
// is undone or after all of it, so (D'D = 1 / kappa^2 per qubit) nothing else
// changes.
//
// With LO the coefficient is a + alo (FP32 hi and lo parts of the FP64 value),
// one FMA more per output: a single FP32 a is tan or cot of a slightly
// different angle (|delta beta| ~ 1e-8), which moves the gradient by the
// Hessian times that shift -- as large as the whole 1e-4 tolerance at points
// where |grad E| ~ 1e-3 |E|.  The adjoint's passes use it; the energy's need
// not (E moves by grad E . delta beta).
template <bool B, bool INV, bool LO>
__device__ __forceinline__ float2 fmix(float2 me, float2 o, float a, float alo) {
    if (!B) {
        const float ox = LO ? fmaf(INV ? -alo : alo, o.y, me.x) : me.x;
        const float oy = LO ? fmaf(INV ? alo : -alo, o.x, me.y) : me.y;
        return INV ? make_float2(fmaf(-a, o.y, ox), fmaf(a, o.x, oy)) : make_float2(fmaf(a, o.y, ox), fmaf(-a, o.x, oy));
    }
    const float px = LO ? fmaf(alo, me.x, INV ? -o.y : o.y) : (INV ? -o.y : o.y);
    const float py = LO ? fmaf(alo, me.y, INV ? o.x : -o.x) : (INV ? o.x : -o.x);
    return make_float2(fmaf(a, me.x, px), fmaf(a, me.y, py));
}

// D (or D') on register bits [r0, r1).
template <int NR, bool B, bool INV, bool LO>
__device__ __forceinline__ void fmix_regs(float2 (&x)[NR], int r0, int r1, float a, float alo) {
#pragma unroll
    for (int rb = 0; (1 << rb) < NR; ++rb) {
        if (rb >= r0 && rb < r1) {
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                if (i & (1 << rb)) continue;
                const int i2 = i | (1 << rb);
                const float2 u = x[i], v = x[i2];
                x[i] = fmix<B, INV, LO>(u, v, a, alo);
                x[i2] = fmix<B, INV, LO>(v, u, a, alo);
            }
        }
    }
}

// D (or D') on lane bits [0, nb).
template <int NR, bool B, bool INV, bool LO>
__device__ __forceinline__ void fmix_lanes(float2 (&x)[NR], int nb, float a, float alo) {
    for (int lb = 0; lb < nb; ++lb) {
        const int m = 1 << lb;
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            float2 o;
            o.x = __shfl_xor_sync(kFull, x[i].x, m);
            o.y = __shfl_xor_sync(kFull, x[i].y, m);
            x[i] = fmix<B, INV, LO>(x[i], o, a, alo);
        }
    }
}

// The first layer's a (hi and lo), form (b: the a I - i X form) and
// kappa^(2 n_in) of one (graph, point): a and the form from the register
// kernels' mixer tables, the lo part from L.fa where the launch has it.
struct FirstMix {
    float a, alo, k2n;
    bool b;
};
__device__ __forceinline__ FirstMix first_mix(const BigLaunch &L, int64_t gj, int n_in) {
    const float2 m = __ldg(L.mix + gj * L.p);  // (tau, flip) of the factored form with bit flips
    FirstMix f;
    f.b = m.y != 0.f;
    f.a = f.b ? -m.x : m.x;  // flip form: tau = -cot beta
    f.alo = L.fa ? __ldg(L.fa + gj).y : 0.f;
    f.k2n = __ldg(L.kpow + gj * L.p * kKpow + n_in);
    return f;
}

// The same factored form for layer l mixing k qubits (kappa_l^(2k) in k2n).
__device__ __forceinline__ FirstMix layer_mix(const BigLaunch &L, int64_t gj, int l, int k) {
    const float2 m = __ldg(L.mix + gj * L.p + l);
    FirstMix f;
    f.b = m.y != 0.f;
    f.a = f.b ? -m.x : m.x;
    f.alo = 0.f;
    f.k2n = __ldg(L.kpow + (gj * L.p + l) * kKpow + k);
    return f;
}

template <int NR, bool INV>
__device__ __forceinline__ void first_mix_regs(float2 (&x)[NR], int r0, int r1, const FirstMix &f) {
    if (f.alo != 0.f) {
        if (f.b)
            fmix_regs<NR, true, INV, true>(x, r0, r1, f.a, f.alo);
        else
            fmix_regs<NR, false, INV, true>(x, r0, r1, f.a, f.alo);
    } else if (f.b) {
        fmix_regs<NR, true, INV, false>(x, r0, r1, f.a, 0.f);
    } else {
        fmix_regs<NR, false, INV, false>(x, r0, r1, f.a, 0.f);
    }
}

template <int NR, bool INV>
__device__ __forceinline__ void first_mix_lanes(float2 (&x)[NR], int nb, const FirstMix &f) {
    if (f.alo != 0.f) {
        if (f.b)
            fmix_lanes<NR, true, INV, true>(x, nb, f.a, f.alo);
        else
            fmix_lanes<NR, false, INV, true>(x, nb, f.a, f.alo);
    } else if (f.b) {
        fmix_lanes<NR, true, INV, false>(x, nb, f.a, 0.f);
    } else {
        fmix_lanes<NR, false, INV, false>(x, nb, f.a, 0.f);
    }
}

// exp(-i beta X) on register qubits [0, nbits) (nbits <= log2 NR).
template <int NR>
__device__ __forceinline__ void mix_regs(float2 (&x)[NR], int nbits, float4 cs) {
#pragma unroll
    for (int rb = 0; (1 << rb) < NR; ++rb) {
        if (rb < nbits) {
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                if (i & (1 << rb)) continue;
                const int i2 = i | (1 << rb);
                const float2 a = x[i], bb = x[i2];
                x[i] = rot(a, bb, cs);
                x[i2] = rot(bb, a, cs);
            }
        }
    }
}

// exp(-i beta X) on lane bits [0, nb).
template <int NR>
__device__ __forceinline__ void mix_lanes(float2 (&x)[NR], int nb, float4 cs) {
    for (int lb = 0; lb < nb; ++lb) {
        const int m = 1 << lb;
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            float2 o;
            o.x = __shfl_xor_sync(kFull, x[i].x, m);
            o.y = __shfl_xor_sync(kFull, x[i].y, m);
            x[i] = rot(x[i], o, cs);
        }
    }
}

// Adjoint step of a mixer on register qubits [0, nbits): adds
// Im<r|X_q|x> for each (one qubit's terms at a time into the compensated
// sum), then applies exp(+i beta X) to both states.
template <int NR>
__device__ __forceinline__ void unmix_regs_d(float2 (&x)[NR], float2 (&r)[NR], int nbits, float4 cs, Dfl &acc) {
#pragma unroll
    for (int rb = 0; (1 << rb) < NR; ++rb) {
        if (rb < nbits) {
            float d = 0.f;
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                if (i & (1 << rb)) continue;
                const int i2 = i | (1 << rb);
                const float2 a = x[i], bb = x[i2], ra = r[i], rbv = r[i2];
                d += imconj(ra, bb) + imconj(rbv, a);
                x[i] = unrot(a, bb, cs);
                x[i2] = unrot(bb, a, cs);
                r[i] = unrot(ra, rbv, cs);
                r[i2] = unrot(rbv, ra, cs);
            }
            dfl_add(acc, d);
        }
    }
}

template <int NR>
__device__ __forceinline__ void unmix_lanes_d(float2 (&x)[NR], float2 (&r)[NR], int nb, float4 cs, Dfl &acc) {
    for (int lb = 0; lb < nb; ++lb) {
        const int m = 1 << lb;
        float d = 0.f;
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            float2 xo, ro;
            xo.x = __shfl_xor_sync(kFull, x[i].x, m);
            xo.y = __shfl_xor_sync(kFull, x[i].y, m);
            ro.x = __shfl_xor_sync(kFull, r[i].x, m);
            ro.y = __shfl_xor_sync(kFull, r[i].y, m);
            d += imconj(r[i], xo);
            x[i] = unrot(x[i], xo, cs);
            r[i] = unrot(r[i], ro, cs);
        }
        dfl_add(acc, d);
    }
}

// Sum of Im<r|X_q|x> over every register and lane qubit (only qubits 0 and 1
// unless `all`), states unchanged; one qubit's terms at a time into the
// compensated sum.
template <int NR>
__device__ __forceinline__ Dfl xterms(const float2 (&x)[NR], const float2 (&r)[NR], bool all) {
    Dfl acc{0.f, 0.f};
#pragma unroll
    for (int rb = 0; (1 << rb) < NR; ++rb) {
        if (!all && rb >= 2) continue;
        float d = 0.f;
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            if (i & (1 << rb)) continue;
            const int i2 = i | (1 << rb);
            d += imconj(r[i], x[i2]) + imconj(r[i2], x[i]);
        }
        dfl_add(acc, d);
    }
    if (!all) return acc;
#pragma unroll
    for (int lb = 0; lb < 5; ++lb) {
        float d = 0.f;
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            float2 xo;
            xo.x = __shfl_xor_sync(kFull, x[i].x, 1 << lb);
            xo.y = __shfl_xor_sync(kFull, x[i].y, 1 << lb);
            d += imconj(r[i], xo);
        }
        dfl_add(acc, d);
    }
    return acc;
}

// <Z_0 Z_1> sign of register i (qubits 0 and 1 are register bits 0 and 1).
__host__ __device__ constexpr float zz_sign(int i) { return ((i ^ (i >> 1)) & 1) ? -1.f : 1.f; }

#ifndef QAOA_SPLIT_GRAD_BLOCKS
#define QAOA_SPLIT_GRAD_BLOCKS 4  // resident CTAs per SM of the adjoint core kernel
#endif

template <bool GRAD, int RB>
__global__ void __launch_bounds__(128, GRAD ? QAOA_SPLIT_GRAD_BLOCKS : 3) split_core_kernel(const __grid_constant__ BigLaunch L) {
    constexpr int NR = 1 << RB;
    constexpr int T = RB + 5;
    constexpr int NW = NR / 4;  // packed cut counts, 4 registers per word
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int nin = L.n_in;
    const int p = L.p;
    const int64_t tiles = int64_t(1) << (nin - T);
    const int64_t ntask = L.n_items * tiles;
    const int64_t block_amps = int64_t(1) << nin;
    for (int64_t task = gw; task < ntask; task += nw) {
        const int64_t it = task / tiles;
        const int64_t u = task - it * tiles;
        int ci;
        int64_t j, y;
        decode_item(L, L.item0 + it, ci, j, y);
        const DevCone *__restrict__ C = L.cones + L.cone_ids[ci];
        if (C->n_in != nin) {
            if (lane == 0) atomicOr(L.status, 1);
            continue;
        }
        const int64_t gj = int64_t(C->graph) * L.P + j;
        const float2 *__restrict__ lut = L.lut + gj * p * L.cmax1;
        const float4 *__restrict__ cs = L.cs + gj * p;
        // cut word of the tile's fixed bits: shell block, outer qubits, lane qubits
        float mult = 1.f;
        uint64_t base = shell_block(C, L.shell, uint32_t(y), mult);
        for (int q = T; q < nin; ++q)
            if ((u >> (q - T)) & 1) base ^= C->col[q];
#pragma unroll
        for (int lb = 0; lb < 5; ++lb)
            if ((lane >> lb) & 1) base ^= C->col[RB + lb];
        // cut value of every register, one byte each (a cone has < 256 edges)
        uint32_t cnt[NW];
        {
            const uint64_t c0 = C->col[0], c1 = C->col[1];
            const uint64_t lo[4] = {0ull, c0, c1, c0 ^ c1};
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                uint64_t h = base;
#pragma unroll
                for (int t = 0; t < RB - 2; ++t)
                    if ((w >> t) & 1) h ^= C->col[2 + t];
                uint32_t packed = 0;
#pragma unroll
                for (int a = 0; a < 4; ++a) packed |= uint32_t(__popcll(lo[a] ^ h)) << (8 * a);
                cnt[w] = packed;
            }
        }
        auto cut = [&](int i) -> int { return int((cnt[i >> 2] >> (8 * (i & 3))) & 0xffu); };
        float2 *__restrict__ sp = L.psi + it * block_amps + (u << T) + lane;
        float2 x[NR];
        if (L.load) {
#pragma unroll
            for (int i = 0; i < NR; ++i) x[i] = sp[i << 5];
        } else {
#pragma unroll
            for (int i = 0; i < NR; ++i) x[i] = __ldg(lut + cut(i));
        }
        const FirstMix f1 = first_mix(L, gj, nin);
        // |psi|^2 = 2^-n kappa_1^(2 n_in) |x|^2 (the first mixer's factored form)
        float sig = __int_as_float((127 - C->n) << 23) * f1.k2n;
        // first mixer on the core qubits
        first_mix_regs<NR, false>(x, 0, RB, f1);
        first_mix_lanes<NR, false>(x, 5, f1);
        for (int l = 1; l < p; ++l) {
            const float2 *__restrict__ lt = lut + l * L.cmax1;
#pragma unroll
            for (int i = 0; i < NR; ++i) x[i] = cmul(x[i], __ldg(lt + cut(i)));
            const int kl = C->k[l];
            if (GRAD) {  // the adjoint keeps exact rotations (its derivative terms need them)
                const float4 c_s = __ldg(cs + l);
                mix_regs<NR>(x, kl < RB ? kl : RB, c_s);
                if (kl > RB) mix_lanes<NR>(x, kl - RB, c_s);
            } else {  // the energy: the factored form, two FMAs per output, kappa^(2 k_l) into sigma
                const FirstMix fl = layer_mix(L, gj, l, kl);
                first_mix_regs<NR, false>(x, 0, kl < RB ? kl : RB, fl);
                if (kl > RB) first_mix_lanes<NR, false>(x, kl - RB, fl);
                sig *= fl.k2n;
            }
        }
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < NR; ++i) acc += (GRAD || !L.norm ? zz_sign(i) : 1.f) * fmaf(x[i].x, x[i].x, x[i].y * x[i].y);
        const float tv = acc * sig * mult;  // this tile's share of <Z_0 Z_1>
        add_gp(-0.5f * float(C->weight) * tv, L.energy, gj);
        if (L.terms) add_gp(tv, L.terms, C->rep * L.P + j);
        if (GRAD) {
            const float wgt2 = 2.f * float(C->weight) * mult * sig;
            float2 r[NR];
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                const float h = -0.5f * zz_sign(i);
                r[i] = make_float2(h * x[i].x, h * x[i].y);
            }
            // In d/d gamma_l, C may be replaced by C - c0: Im<lambda|psi> =
            // <psi_end|O|psi_end> is zero within every core tile, and c0 = m/2
            // (the mean cut value) removes most of the cancellation in the
            // FP32 sums.
            const float c0 = 0.5f * float(C->m);
            for (int l = p - 1; l >= 1; --l) {
                const float4 c_s = __ldg(cs + l);
                const int kl = C->k[l];
                Dfl d{0.f, 0.f};
                unmix_regs_d<NR>(x, r, kl < RB ? kl : RB, c_s, d);
                if (kl > RB) unmix_lanes_d<NR>(x, r, kl - RB, c_s, d);
                add_gp(d, wgt2, L.grad, gj * 2 * p + p + l);
                const float2 *__restrict__ lt = lut + l * L.cmax1;
                // keep the shifted cut values from being hoisted out of the layer
                // loop into sixteen live registers
#pragma unroll
                for (int w = 0; w < NW; ++w) asm volatile("" : "+r"(cnt[w]));
                float dg = 0.f;
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    const int c = cut(i);
                    dg = fmaf(float(c) - c0, imconj(r[i], x[i]), dg);
                    const float2 ph = __ldg(lt + c);
                    x[i] = cmulc(x[i], ph);
                    r[i] = cmulc(r[i], ph);
                }
                add_gp(Dfl{dg, 0.f}, wgt2, L.grad, gj * 2 * p + l);
            }
            // first mixer: the core qubits' terms, then lambda alone un-mixed
            // At p = 1 the first layer is the last: lambda = O psi with
            // O = -1/2 Z_0 Z_1, and <psi|O X_q|psi> is real for every q other
            // than 0 and 1 (X_q and O commute), so only those two contribute.
            add_gp(xterms<NR>(x, r, p > 1), wgt2, L.grad, gj * 2 * p + p);
            first_mix_regs<NR, true>(r, 0, RB, f1);
            first_mix_lanes<NR, true>(r, 5, f1);
#pragma unroll
            for (int i = 0; i < NR; ++i) sp[i << 5] = r[i];
        }
    }
}

// Qubit held by storage address bit a (see the layout above).
__device__ __forceinline__ int qubit_of(int a, int rb) { return a < 5 ? rb + a : (a < rb + 5 ? a - 5 : a); }

template <int MODE>
__global__ void __launch_bounds__(128, MODE == kOuterGen ? 4 : 3) split_outer_kernel(const __grid_constant__ BigLaunch L) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int nin = L.n_in, b = L.b, RB = L.rb;
    const int r0 = L.w0 - b, r1 = L.w1 - b;  // register bits of the outer qubits to mix
    const int p = L.p;
    const int64_t tiles = int64_t(1) << (nin - 10);
    const int64_t ntask = L.n_items * tiles;
    const int64_t block_amps = int64_t(1) << nin;
    const int64_t lowmask = (int64_t(1) << (b - 5)) - 1;
    for (int64_t task = gw; task < ntask; task += nw) {
        const int64_t it = task / tiles;
        const int64_t tile = task - it * tiles;
        int ci;
        int64_t j, y;
        decode_item(L, L.item0 + it, ci, j, y);
        const DevCone *__restrict__ C = L.cones + L.cone_ids[ci];
        if (C->n_in != nin) {
            if (lane == 0) atomicOr(L.status, 1);
            continue;
        }
        const int64_t gj = int64_t(C->graph) * L.P + j;
        const FirstMix f1 = first_mix(L, gj, nin);
        // address of (lane, register i) = xb | (i << b) | lane
        const int64_t xb = ((tile & lowmask) << 5) | ((tile >> (b - 5)) << (b + 5));
        float2 *__restrict__ sp = L.psi + it * block_amps + xb + lane;
        float2 x[32];
        if (MODE != kOuterGen) {
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] = sp[int64_t(i) << b];
        }
        if (MODE == kOuterMix) {
            if (L.sign > 0)
                first_mix_regs<32, false>(x, r0, r1, f1);
            else
                first_mix_regs<32, true>(x, r0, r1, f1);
        } else {
            const float2 *__restrict__ lut = L.lut + gj * p * L.cmax1;  // first layer's phase table
            float mult = 1.f;
            uint64_t base = shell_block(C, L.shell, uint32_t(y), mult);
#pragma unroll
            for (int lb = 0; lb < 5; ++lb)
                if ((lane >> lb) & 1) base ^= C->col[RB + lb];
            for (int a = 5; a < nin; ++a)
                if ((a < b || a >= b + 5) && ((xb >> a) & 1)) base ^= C->col[qubit_of(a, RB)];
            uint64_t lo[4], hi[8];
            {
                const uint64_t c0 = C->col[qubit_of(b, RB)], c1 = C->col[qubit_of(b + 1, RB)];
                const uint64_t c2 = C->col[qubit_of(b + 2, RB)], c3 = C->col[qubit_of(b + 3, RB)];
                const uint64_t c4 = C->col[qubit_of(b + 4, RB)];
                lo[0] = 0;
                lo[1] = c0;
                lo[2] = c1;
                lo[3] = c0 ^ c1;
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    hi[k] = base ^ ((k & 1) ? c2 : 0ull) ^ ((k & 2) ? c3 : 0ull) ^ ((k & 4) ? c4 : 0ull);
            }
            if (MODE == kOuterGen) {
#pragma unroll
                for (int i = 0; i < 32; ++i) x[i] = __ldg(lut + __popcll(lo[i & 3] ^ hi[i >> 2]));
                first_mix_regs<32, false>(x, r0, r1, f1);
            } else {  // kOuterFirst: x holds lambda
                first_mix_regs<32, true>(x, r0, r1, f1);
                // the outer qubits' mixer terms vanish at p = 1, where the first
                // layer is the last (only qubits 0 and 1 contribute there)
                const bool outer_terms = p > 1;
                const float c0 = 0.5f * float(C->m);  // Im<lambda|psi> = 0: C - c0 in place of C
                float dg = 0.f, dq[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // per window qubit
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int c = __popcll(lo[i & 3] ^ hi[i >> 2]);
                    const float2 ph = __ldg(lut + c);  // state before the first mixer, times 2^(n/2)
                    dg = fmaf(float(c) - c0, imconj(x[i], ph), dg);
                    if (outer_terms) {
#pragma unroll
                        for (int rb = 0; rb < 5; ++rb)
                            if (rb >= r0 && rb < r1) dq[rb] += imconj(x[i ^ (1 << rb)], ph);
                    }
                }
                Dfl db{0.f, 0.f};
#pragma unroll
                for (int rb = 0; rb < 5; ++rb) dfl_add(db, dq[rb]);
                for (int q = L.x0; q < (outer_terms ? L.x1 : L.x0); ++q) {  // outer qubits outside the window
                    const uint64_t cq = C->col[q];
                    float t = 0.f;
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        t += imconj(x[i], __ldg(lut + __popcll(lo[i & 3] ^ hi[i >> 2] ^ cq)));
                    dfl_add(db, t);
                }
                // lambda = 2^(-n/2) kappa_1^(2 n_in) x once the first mixer is undone
                const float wgt2 = 2.f * float(C->weight) * mult * __int_as_float((127 - C->n) << 23) * f1.k2n;
                add_gp(Dfl{dg, 0.f}, wgt2, L.grad, gj * 2 * p);
                if (outer_terms) add_gp(db, wgt2, L.grad, gj * 2 * p + p);
            }
        }
        if (MODE != kOuterFirst) {
#pragma unroll
            for (int i = 0; i < 32; ++i) sp[int64_t(i) << b] = x[i];
        }
    }
}

// ------------------------------------------------------------ chunk passes
// An outer pass over more than five outer qubits stages a chunk of the block
// in shared memory: 2^13 amplitudes made of the lowest lo = 13 - w address
// bits (contiguous runs of at least 64 bytes) and a window of w <=
// kChunkMaxW outer qubits.  The window is mixed five qubits at a time by
// register butterflies over amplitudes gathered from shared memory, so one
// HBM round trip covers all of it.  The chunk moves between HBM and shared
// memory by the tensor memory accelerator: one cp.async.bulk.tensor per
// chunk and direction, described by a tensor map of the block (the run, the
// address bits between run and window, the window in two dimensions of at
// most 256, the bits above it times the wave's items), completion of a load
// tracked by an mbarrier.  The copies use the natural order (element e at
// e); the rounds in between use a bank-swizzled order.
constexpr int kChunkBits = 13;
constexpr int kChunkMaxW = 10;
constexpr int kChunkThreads = 256;

// Bank swizzle for runs of eight amplitudes (a window of ten): bit 3 of the
// shared-memory index (which 64-byte half of a 128-byte row) is flipped by
// the parity of the bits above it, so the four 64-byte runs that a warp
// touches fall two in each half.  With runs of 16 or more the rounds' lanes
// read 16 consecutive amplitudes per half-warp, free of conflicts as they
// are, and no swizzle is applied.
__device__ __forceinline__ int swz(int s) { return s ^ ((__popc(s >> 4) & 1) << 3); }
__device__ __forceinline__ int sidx(int s, bool swizzled) { return swizzled ? swz(s) : s; }

// ---- tensor-memory-accelerator helpers (one thread issues, an mbarrier tracks loads)
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses before later accesses
// of the asynchronous (TMA) proxy.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Load of one box into shared memory, completing on bar (issued by one thread).
__device__ __forceinline__ void tma_load(const CUtensorMap *map, void *dst, uint64_t *bar, uint32_t bytes,
                                         const int (&c)[5]) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(smem_addr(bar))
        : "memory");
}

// Store of one box from shared memory; returns once the box has been read
// (issued by one thread, after every writer's fence_async_smem and a barrier).
__device__ __forceinline__ void tma_store(const CUtensorMap *map, const void *src, const int (&c)[5]) {
    asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];" ::"l"(
                     map),
                 "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(smem_addr(src))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void tma_store_drain() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Waits for phase `phase` of bar to complete, for at most limit_ns; false if
// it has not.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase, uint64_t limit_ns) {
    const uint32_t a = smem_addr(bar);
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(phase)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}
constexpr uint64_t kTmaWaitNs = 2000000000ull;  // 2 s: a load of 64 KB takes microseconds

// slot with gn zero bits inserted at bit position pos
__device__ __forceinline__ int spread_slot(int slot, int pos, int gn) {
    return (slot & ((1 << pos) - 1)) | ((slot >> pos) << (pos + gn));
}

// First-layer cut words of a chunk slot: `base` for the slot's fixed bits,
// lo/hi over the G register qubits w0 .. w0+G-1.
template <int G>
__device__ __forceinline__ void slot_words(const DevCone *__restrict__ C, uint64_t base, int w0, uint64_t (&lo)[4],
                                           uint64_t (&hi)[8]) {
    uint64_t cr[5];
#pragma unroll
    for (int b = 0; b < 5; ++b) cr[b] = b < G ? C->col[w0 + b] : 0ull;
    lo[0] = 0;
    lo[1] = cr[0];
    lo[2] = cr[1];
    lo[3] = cr[0] ^ cr[1];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        hi[k] = base ^ ((k & 1) ? cr[2] : 0ull) ^ ((k & 2) ? cr[3] : 0ull) ^ ((k & 4) ? cr[4] : 0ull);
}

// One round of a chunk pass: every slot gathers the 2^G amplitudes that
// differ in chunk bits [pos, pos+G), applies the mixer to those G qubits and
// writes them back.  GEN in its first round generates the amplitudes instead.
template <int G, bool GEN>
__device__ __forceinline__ void chunk_round(float2 *__restrict__ sm, int n_el, int pos, FirstMix f, bool inv,
                                            const DevCone *__restrict__ C, uint64_t cw, int lo_bits, int RB, int w0,
                                            const float2 *__restrict__ lut, bool rd_swz, bool wr_swz) {
    constexpr int NR = 1 << G;
    for (int slot = threadIdx.x; slot < (n_el >> G); slot += kChunkThreads) {
        const int sb = spread_slot(slot, pos, G);
        float2 x[NR];
        if (GEN) {
            uint64_t base = cw;
            for (int b = 0; b < lo_bits; ++b)  // the window bits of sb are zero in the first round
                if ((sb >> b) & 1) base ^= C->col[qubit_of(b, RB)];
            for (int b = lo_bits + G; b < kChunkBits; ++b)
                if ((sb >> b) & 1) base ^= C->col[w0 + b - lo_bits];
            uint64_t lo[4], hi[8];
            slot_words<G>(C, base, w0, lo, hi);
#pragma unroll
            for (int i = 0; i < NR; ++i) x[i] = __ldg(lut + __popcll(lo[i & 3] ^ hi[i >> 2]));
        } else {
#pragma unroll
            for (int i = 0; i < NR; ++i) x[i] = sm[sidx(sb | (i << pos), rd_swz)];
        }
        if (inv)
            first_mix_regs<NR, true>(x, 0, G, f);
        else
            first_mix_regs<NR, false>(x, 0, G, f);
#pragma unroll
        for (int i = 0; i < NR; ++i) sm[sidx(sb | (i << pos), wr_swz)] = x[i];
    }
}

template <bool GEN>
__device__ __forceinline__ void chunk_round_any(int G, float2 *sm, int n_el, int pos, FirstMix f, bool inv,
                                                const DevCone *C, uint64_t cw, int lo_bits, int RB, int w0,
                                                const float2 *lut, bool rd_swz, bool wr_swz) {
    switch (G) {
        case 1: chunk_round<1, GEN>(sm, n_el, pos, f, inv, C, cw, lo_bits, RB, w0, lut, rd_swz, wr_swz); break;
        case 2: chunk_round<2, GEN>(sm, n_el, pos, f, inv, C, cw, lo_bits, RB, w0, lut, rd_swz, wr_swz); break;
        case 3: chunk_round<3, GEN>(sm, n_el, pos, f, inv, C, cw, lo_bits, RB, w0, lut, rd_swz, wr_swz); break;
        case 4: chunk_round<4, GEN>(sm, n_el, pos, f, inv, C, cw, lo_bits, RB, w0, lut, rd_swz, wr_swz); break;
        default: chunk_round<5, GEN>(sm, n_el, pos, f, inv, C, cw, lo_bits, RB, w0, lut, rd_swz, wr_swz); break;
    }
}

template <int MODE>
__global__ void __launch_bounds__(kChunkThreads, 2)
    split_chunk_kernel(const __grid_constant__ BigLaunch L, const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) float2 sm[];
    __shared__ uint64_t s_bar;  // completion of the chunk's load
    const int tid = threadIdx.x;
    if (tid == 0) mbar_init(&s_bar);
    __syncthreads();
    uint32_t phase = 0;
    const int nin = L.n_in, RB = L.rb, w0 = L.w0, w = L.w1 - L.w0;
    const int lo_bits = kChunkBits - w;  // lowest address bits of the chunk (w0 >= lo_bits)
    const int n_el = 1 << kChunkBits;
    const int p = L.p;
    const int64_t chunks = int64_t(1) << (nin - kChunkBits);
    const int64_t ntask = L.n_items * chunks;
    const int64_t lowmask = (int64_t(1) << (w0 - lo_bits)) - 1;
    for (int64_t task = blockIdx.x; task < ntask; task += gridDim.x) {
        const int64_t it = task / chunks;
        const int64_t ch = task - it * chunks;
        int ci;
        int64_t j, y;
        decode_item(L, L.item0 + it, ci, j, y);
        const DevCone *__restrict__ C = L.cones + L.cone_ids[ci];
        if (C->n_in != nin) {  // uniform over the CTA
            if (tid == 0) atomicOr(L.status, 1);
            continue;
        }
        const int64_t gj = int64_t(C->graph) * L.P + j;
        const FirstMix f1 = first_mix(L, gj, nin);
        const bool inv = MODE == kOuterFirst || (MODE == kOuterMix && L.sign < 0);
        // element e of the chunk <-> address xb + (e & runmask) + ((e >> lo_bits) << w0) of
        // item it; tensor coordinates: run, middle bits, window (two dimensions), high bits x item
        const int64_t xb = ((ch & lowmask) << lo_bits) | ((ch >> (w0 - lo_bits)) << (w0 + w));
        const int crd[5] = {0, int(ch & lowmask), 0, 0,
                            int(it * (int64_t(1) << (nin - w0 - w)) + (ch >> (w0 - lo_bits)))};
        if (MODE != kOuterGen && tid == 0) {
            fence_async_smem();  // the previous task's accesses come before the copy's writes
            tma_load(&tmap, sm, &s_bar, uint32_t(n_el * sizeof(float2)), crd);
        }
        // cut word of the chunk's fixed bits (shell block and address bits outside the chunk)
        float mult = 1.f;
        uint64_t cw = 0;
        const float2 *__restrict__ lut = L.lut + gj * p * L.cmax1;  // first layer's phase table
        if (MODE != kOuterMix) {
            cw = shell_block(C, L.shell, uint32_t(y), mult);
            for (int a = lo_bits; a < nin; ++a)
                if ((a < w0 || a >= w0 + w) && ((xb >> a) & 1)) cw ^= C->col[qubit_of(a, RB)];
        }
        if (MODE != kOuterGen) {
            // bounded wait; should it ever run out (never expected), record it,
            // give the copy the same time again to land, and stop this block
            const bool ok = mbar_wait(&s_bar, phase, kTmaWaitNs);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicOr(L.status, 4);
                mbar_wait(&s_bar, phase, kTmaWaitNs);
                return;
            }
            phase ^= 1u;
        }
        __syncthreads();
        for (int g0 = 0; g0 < w; g0 += 5) {
            const int gn = min(5, w - g0);  // this round's qubits: chunk bits lo_bits + g0 ..
            // the copies use the natural order, the rounds between them the swizzled one
            const bool swz_on = lo_bits < 4;
            const bool rd_swz = swz_on && g0 > 0, wr_swz = swz_on && (g0 + gn < w || MODE == kOuterFirst);
            if (MODE == kOuterGen && g0 == 0)
                chunk_round_any<true>(gn, sm, n_el, lo_bits, f1, false, C, cw, lo_bits, RB, w0, lut, rd_swz, wr_swz);
            else
                chunk_round_any<false>(gn, sm, n_el, lo_bits + g0, f1, inv, C, cw, lo_bits, RB, w0, lut, rd_swz,
                                       wr_swz);
            __syncthreads();
        }
        if (MODE == kOuterFirst) {
            // lambda is now fully un-mixed: the first layer's phase term and the
            // outer qubits' mixer terms against exp(-i gamma_1 C)|+>
            const bool outer_terms = p > 1;
            const float c0 = 0.5f * float(C->m);  // Im<lambda|psi> = 0: C - c0 in place of C
            const int gn = min(5, w);
            const int nreg = 1 << gn;
            Dfl dg{0.f, 0.f}, db{0.f, 0.f};  // this thread's slots, compensated
            for (int slot = tid; slot < (n_el >> gn); slot += kChunkThreads) {
                const int sb = spread_slot(slot, lo_bits, gn);
                float2 x[32];
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    x[i] = i < nreg ? sm[sidx(sb | (i << lo_bits), lo_bits < 4)] : make_float2(0.f, 0.f);
                uint64_t base = cw;
                for (int b = 0; b < lo_bits; ++b)
                    if ((sb >> b) & 1) base ^= C->col[qubit_of(b, RB)];
                for (int b = lo_bits + gn; b < kChunkBits; ++b)
                    if ((sb >> b) & 1) base ^= C->col[w0 + b - lo_bits];
                uint64_t lo[4], hi[8];
                slot_words<5>(C, base, w0, lo, hi);  // w > 5 here: five window qubits in registers
                float dgs = 0.f, dq[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int c = __popcll(lo[i & 3] ^ hi[i >> 2]);
                    const float2 ph = __ldg(lut + c);
                    dgs = fmaf(float(c) - c0, imconj(x[i], ph), dgs);
                    if (outer_terms) {
#pragma unroll
                        for (int rb = 0; rb < 5; ++rb) dq[rb] += imconj(x[i ^ (1 << rb)], ph);
                    }
                }
                dfl_add(dg, dgs);
                if (outer_terms) {
#pragma unroll
                    for (int rb = 0; rb < 5; ++rb) dfl_add(db, dq[rb]);
                    // the other outer qubits: the rest of the window, then beyond it
                    for (int q = w0 + 5; q < L.x1; ++q) {
                        const uint64_t cq = C->col[q];
                        float t = 0.f;
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            t += imconj(x[i], __ldg(lut + __popcll(lo[i & 3] ^ hi[i >> 2] ^ cq)));
                        dfl_add(db, t);
                    }
                }
            }
            // lambda = 2^(-n/2) kappa_1^(2 n_in) x once the first mixer is undone
            const float wgt2 = 2.f * float(C->weight) * mult * __int_as_float((127 - C->n) << 23) * f1.k2n;
            add_gp(dg, wgt2, L.grad, gj * 2 * p);
            if (outer_terms) add_gp(db, wgt2, L.grad, gj * 2 * p + p);
        } else {
            fence_async_smem();  // every thread's writes, before the copy reads them
            __syncthreads();
            if (tid == 0) tma_store(&tmap, sm, crd);
        }
        __syncthreads();  // the next task reuses the shared chunk
    }
    if (tid == 0) tma_store_drain();
}

// Tensor map of a wave's blocks as the chunk passes of window [w0, w0 + w) see
// them (8-byte elements): the run of the lo = 13 - w lowest address bits,
// the bits between run and window, the window in two dimensions of at most 2^8,
// the bits above it times the items.  Dense: every stride is the previous one
// times the previous extent.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    });
    return fn;
}

cudaError_t chunk_map(const BigLaunch &B, int w0, int w, CUtensorMap *map) {
    EncodeTiledFn enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    const int nin = B.n_in, lo = kChunkBits - w, wa = w < 8 ? w : 8;
    const cuuint64_t dim[5] = {cuuint64_t(1) << lo, cuuint64_t(1) << (w0 - lo), cuuint64_t(1) << wa,
                               cuuint64_t(1) << (w - wa), cuuint64_t(B.n_items) << (nin - w0 - w)};
    const cuuint64_t stride[4] = {cuuint64_t(8) << lo, cuuint64_t(8) << w0, cuuint64_t(8) << (w0 + wa),
                                  cuuint64_t(8) << (w0 + w)};
    const cuuint32_t box[5] = {1u << lo, 1u, 1u << wa, 1u << (w - wa), 1u};
    const cuuint32_t estride[5] = {1u, 1u, 1u, 1u, 1u};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, B.psi, dim, stride, box, estride,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

int occupancy_grid(const void *fn, int block, size_t smem);

bool split_ok(int n_in, int p, const int32_t *k, bool grad) {
    const int T = (grad ? kSplitRbGrad : kSplitRbEnergy) + 5;
    if (n_in < 10 || n_in < T || n_in > QAOA_MAX_CONE_QUBITS || k[0] != n_in) return false;
    if (grad && n_in == T) return false;
    for (int l = 1; l < p; ++l)
        if (k[l] > T) return false;
    return true;
}

// Chunk kernels need more than the default 48 KB of dynamic shared memory:
// raised once per kernel and device.
static cudaError_t allow_chunk_smem(const void *fn, int mode) {
    static std::mutex mu;
    static std::set<std::pair<int, int>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, mode})) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(sizeof(float2) << kChunkBits));
    if (e == cudaSuccess) done.insert({dev, mode});
    return e;
}

cudaError_t split_prepare() {
    cudaError_t e = allow_chunk_smem((const void *)split_chunk_kernel<kOuterGen>, kOuterGen);
    if (e == cudaSuccess) e = allow_chunk_smem((const void *)split_chunk_kernel<kOuterMix>, kOuterMix);
    if (e == cudaSuccess) e = allow_chunk_smem((const void *)split_chunk_kernel<kOuterFirst>, kOuterFirst);
    return e;
}

cudaError_t launch_split_wave(BigLaunch B, bool grad, int chunk_window, int64_t &launches, cudaStream_t s) {
    const int cw_max = chunk_window < 6 ? 6 : (chunk_window > kChunkMaxW ? kChunkMaxW : chunk_window);
    const int RB = grad ? kSplitRbGrad : kSplitRbEnergy, T = RB + 5;
    const int nin = B.n_in;
    B.rb = RB;
    // Outer qubit windows: shared-memory chunks of up to kChunkMaxW qubits
    // while more than five remain, then one register window of at most five.
    struct Win {
        int w0, w1;
        bool chunk;
    };
    std::vector<Win> win;
    for (int w0 = T; w0 < nin;) {
        const int left = nin - w0;
        const int n = left > 5 ? std::min(left, cw_max) : left;
        win.push_back({w0, w0 + n, left > 5});
        w0 += n;
    }
    auto grid_for = [](const void *fn, int64_t tasks) {
        const int64_t need = std::max<int64_t>(1, (tasks + 3) / 4);
        return int(std::min<int64_t>(occupancy_grid(fn, 128, 0), need));
    };
    auto outer = [&](int mode, size_t w, int sign) -> cudaError_t {
        B.mode = mode;
        B.w0 = win[w].w0;
        B.w1 = win[w].w1;
        B.b = std::min(B.w0, nin - 5);
        B.x0 = win[w].w1;
        B.x1 = nin;
        B.sign = sign;
        if (win[w].chunk) {
            const size_t smem = size_t(sizeof(float2)) << kChunkBits;
            CUtensorMap map;
            if (cudaError_t e = chunk_map(B, B.w0, B.w1 - B.w0, &map); e != cudaSuccess) return e;
            const int64_t tasks = B.n_items << (nin - kChunkBits);
            const void *fn = mode == kOuterGen   ? (const void *)split_chunk_kernel<kOuterGen>
                             : mode == kOuterMix ? (const void *)split_chunk_kernel<kOuterMix>
                                                 : (const void *)split_chunk_kernel<kOuterFirst>;
            if (cudaError_t e = allow_chunk_smem(fn, mode); e != cudaSuccess) return e;
            const int grid = int(std::min<int64_t>(occupancy_grid(fn, kChunkThreads, smem), std::max<int64_t>(tasks, 1)));
            if (mode == kOuterGen)
                split_chunk_kernel<kOuterGen><<<grid, kChunkThreads, smem, s>>>(B, map);
            else if (mode == kOuterMix)
                split_chunk_kernel<kOuterMix><<<grid, kChunkThreads, smem, s>>>(B, map);
            else
                split_chunk_kernel<kOuterFirst><<<grid, kChunkThreads, smem, s>>>(B, map);
        } else {
            const int64_t tasks = B.n_items << (nin - 10);
            if (mode == kOuterGen) {
                const void *fn = (const void *)split_outer_kernel<kOuterGen>;
                split_outer_kernel<kOuterGen><<<grid_for(fn, tasks), 128, 0, s>>>(B);
            } else if (mode == kOuterMix) {
                const void *fn = (const void *)split_outer_kernel<kOuterMix>;
                split_outer_kernel<kOuterMix><<<grid_for(fn, tasks), 128, 0, s>>>(B);
            } else {
                const void *fn = (const void *)split_outer_kernel<kOuterFirst>;
                split_outer_kernel<kOuterFirst><<<grid_for(fn, tasks), 128, 0, s>>>(B);
            }
        }
        ++launches;
        return cudaGetLastError();
    };
    if (grad && win.empty()) return cudaErrorInvalidValue;  // excluded by split_ok
    cudaError_t e = cudaSuccess;
    for (size_t w = 0; w < win.size() && e == cudaSuccess; ++w) e = outer(w == 0 ? kOuterGen : kOuterMix, w, 1);
    if (e != cudaSuccess) return e;
    B.load = win.empty() ? 0 : 1;
    const int64_t core_tasks = B.n_items << (nin - T);
    if (grad) {
        const void *fn = (const void *)split_core_kernel<true, kSplitRbGrad>;
        split_core_kernel<true, kSplitRbGrad><<<grid_for(fn, core_tasks), 128, 0, s>>>(B);
    } else {
        const void *fn = (const void *)split_core_kernel<false, kSplitRbEnergy>;
        split_core_kernel<false, kSplitRbEnergy><<<grid_for(fn, core_tasks), 128, 0, s>>>(B);
    }
    ++launches;
    if ((e = cudaGetLastError()) != cudaSuccess || !grad) return e;
    for (size_t w = win.size(); w-- > 1 && e == cudaSuccess;) e = outer(kOuterMix, w, -1);
    if (e != cudaSuccess) return e;
    return outer(kOuterFirst, 0, -1);
}

}  // namespace qaoa
