// Large-state cone path: cones whose inner part (the qubits any mixer
// touches, within distance p-1 of the edge) is too large for registers.
//
// Every (cone, point, shell assignment) owns a block of 2^n_in complex64
// amplitudes in scratch memory.  A pass streams a block once through
// registers: a warp tile covers 10 qubits -- qubits 0..4 on the lanes, so
// that each load or store instruction of the warp touches 256 contiguous
// bytes, and qubits b..b+4 in registers -- and applies a short list of
// operations (phase, mixer on the tile's qubits, reduction, and in the
// adjoint their inverses with the derivative terms).  Gates are the exact
// unitaries exp(-i gamma C) and exp(-i beta X) (Sec. 2.2); the adjoint uses
// exp(+i beta X) and exp(+i gamma C), which keep <lambda|X_q|psi> invariant
// under the un-mixing of any qubit of the same layer.
#include "big.cuh"
#include "big_common.cuh"

namespace qaoa {
namespace {

constexpr int NR = 1 << kBigRegBits;

template <bool GRAD>
__global__ void __launch_bounds__(128) big_pass_kernel(const __grid_constant__ BigLaunch L) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const BigPass &ps = L.pass;
    const int b = ps.b;
    const int nin = L.n_in;
    const int64_t tiles = int64_t(1) << (nin - 10);
    const int64_t ntask = L.n_items * tiles;
    const int64_t block_amps = int64_t(1) << nin;
    const int p = L.p;
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
        const int g = C->graph;
        const int64_t gj = int64_t(g) * L.P + j;
        const float2 *__restrict__ lut = L.lut + gj * p * L.cmax1;
        const float4 *__restrict__ cs = L.cs + gj * p;
        // inner index of (lane, register i): xb | (i << b) | lane
        const int64_t lowmask = (int64_t(1) << (b - 5)) - 1;
        const int64_t xb = ((tile & lowmask) << 5) | ((tile >> (b - 5)) << (b + 5));
        // cut word: shell part ^ fixed inner part ^ lane part, then per register index
        float mult = 1.f;
        uint64_t base = shell_block(C, L.shell, uint32_t(y), mult);
        for (int q = 5; q < nin; ++q)
            if ((xb >> q) & 1) base ^= C->col[q];
#pragma unroll
        for (int q = 0; q < 5; ++q)
            if ((lane >> q) & 1) base ^= C->col[q];
        uint64_t lo[4], hi[8];
        {
            const uint64_t c0 = C->col[b], c1 = C->col[b + 1];
            lo[0] = 0;
            lo[1] = c0;
            lo[2] = c1;
            lo[3] = c0 ^ c1;
            const uint64_t c2 = C->col[b + 2], c3 = C->col[b + 3], c4 = C->col[b + 4];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                hi[k] = base ^ ((k & 1) ? c2 : 0ull) ^ ((k & 2) ? c3 : 0ull) ^ ((k & 4) ? c4 : 0ull);
        }
        float2 *__restrict__ sp = L.psi + it * block_amps + xb + lane;
        float2 *__restrict__ lp = GRAD ? L.lam + it * block_amps + xb + lane : nullptr;
        float2 x[NR], r[NR];
        if (ps.load_psi) {
#pragma unroll
            for (int i = 0; i < NR; ++i) x[i] = sp[int64_t(i) << b];
        }
        if (GRAD && ps.load_lam) {
#pragma unroll
            for (int i = 0; i < NR; ++i) r[i] = lp[int64_t(i) << b];
        }
        const float wgt = float(C->weight) * mult;  // orbit size x shell multiplicity
        const float sig = __int_as_float((127 - C->n) << 23);  // 2^-n
        for (int o = 0; o < ps.nops; ++o) {
            const BigOp op = ps.ops[o];
            const int l = op.layer;
            switch (op.type) {
                case kOpGenPhase: {  // |+> (amplitude 1) times exp(-i gamma_1 C)
#pragma unroll
                    for (int i = 0; i < NR; ++i) x[i] = __ldg(lut + __popcll(lo[i & 3] ^ hi[i >> 2]));
                    break;
                }
                case kOpPhase: {
                    const float2 *__restrict__ lt = lut + l * L.cmax1;
#pragma unroll
                    for (int i = 0; i < NR; ++i) x[i] = cmul(x[i], __ldg(lt + __popcll(lo[i & 3] ^ hi[i >> 2])));
                    break;
                }
                case kOpMix: {
                    const float4 c_s = __ldg(cs + l);
                    for (int q = op.q0; q < op.q1; ++q) {
                        if (q < 5) {
                            const int m = 1 << q;
#pragma unroll
                            for (int i = 0; i < NR; ++i) {
                                float2 ot;
                                ot.x = __shfl_xor_sync(kFull, x[i].x, m);
                                ot.y = __shfl_xor_sync(kFull, x[i].y, m);
                                x[i] = rot(x[i], ot, c_s);
                            }
                        } else {
                            const int rq = q - b;
#pragma unroll
                            for (int rb = 0; rb < kBigRegBits; ++rb) {
                                if (rb != rq) continue;
#pragma unroll
                                for (int i = 0; i < NR; ++i) {
                                    if (i & (1 << rb)) continue;
                                    const int i2 = i | (1 << rb);
                                    const float2 a = x[i], bb = x[i2];
                                    x[i] = rot(a, bb, c_s);
                                    x[i2] = rot(bb, a, c_s);
                                }
                            }
                        }
                    }
                    break;
                }
                case kOpReduce: {
                    const float sg = ((lane ^ (lane >> 1)) & 1) && !L.norm ? -1.f : 1.f;
                    float acc = 0.f;
#pragma unroll
                    for (int i = 0; i < NR; ++i) acc = fmaf(x[i].x, x[i].x, fmaf(x[i].y, x[i].y, acc));
                    const float tv = sg * acc * sig * mult;  // this block's share of <Z_0 Z_1>
                    add_gp(-0.5f * float(C->weight) * tv, L.energy, gj);
                    if (L.terms) add_gp(tv, L.terms, C->rep * L.P + j);
                    break;
                }
                case kOpLamInit: {
                    if (GRAD) {
                        const float sg = ((lane ^ (lane >> 1)) & 1) ? 0.5f : -0.5f;
#pragma unroll
                        for (int i = 0; i < NR; ++i) r[i] = make_float2(sg * x[i].x, sg * x[i].y);
                    }
                    break;
                }
                case kOpUnmix: {
                    if (GRAD) {
                        const float4 c_s = __ldg(cs + l);
                        // At the last layer lambda = O psi (O = -1/2 Z_0 Z_1), and
                        // <psi|O X_q|psi> is real for every q other than 0 and 1 (X_q
                        // commutes with O and with the mixers of other qubits): only
                        // those two enter d/d beta_p, the others are rounding noise.
                        const int qd = l == p - 1 ? 2 : QAOA_MAX_CONE_QUBITS;
                        Dfl acc{0.f, 0.f};
                        for (int q = op.q0; q < op.q1; ++q) {
                            float d = 0.f;  // this qubit's terms, then added compensated
                            if (q < 5) {
                                const int m = 1 << q;
#pragma unroll
                                for (int i = 0; i < NR; ++i) {
                                    float2 xo, ro;
                                    xo.x = __shfl_xor_sync(kFull, x[i].x, m);
                                    xo.y = __shfl_xor_sync(kFull, x[i].y, m);
                                    ro.x = __shfl_xor_sync(kFull, r[i].x, m);
                                    ro.y = __shfl_xor_sync(kFull, r[i].y, m);
                                    d += imconj(r[i], xo);
                                    x[i] = unrot(x[i], xo, c_s);
                                    r[i] = unrot(r[i], ro, c_s);
                                }
                            } else {
                                const int rq = q - b;
#pragma unroll
                                for (int rb = 0; rb < kBigRegBits; ++rb) {
                                    if (rb != rq) continue;
#pragma unroll
                                    for (int i = 0; i < NR; ++i) {
                                        if (i & (1 << rb)) continue;
                                        const int i2 = i | (1 << rb);
                                        const float2 a = x[i], bb = x[i2], ra = r[i], rbv = r[i2];
                                        d += imconj(ra, bb) + imconj(rbv, a);
                                        x[i] = unrot(a, bb, c_s);
                                        x[i2] = unrot(bb, a, c_s);
                                        r[i] = unrot(ra, rbv, c_s);
                                        r[i2] = unrot(rbv, ra, c_s);
                                    }
                                }
                            }
                            if (q < qd) dfl_add(acc, d);
                        }
                        add_gp(acc, 2.f * wgt * sig, L.grad, gj * 2 * p + p + l);
                    }
                    break;
                }
                case kOpUnphase: {  // q0 = 1: also undo the phase
                    if (GRAD) {
                        const float2 *__restrict__ lt = lut + l * L.cmax1;
                        const float c0 = 0.5f * float(C->m);  // Im<r|x> = 0: C - c0 in place of C
                        Dfl acc{0.f, 0.f};
                        float d = 0.f;
#pragma unroll
                        for (int i = 0; i < NR; ++i) {
                            const int c = __popcll(lo[i & 3] ^ hi[i >> 2]);
                            d = fmaf(float(c) - c0, imconj(r[i], x[i]), d);
                            if ((i & 7) == 7) {  // eight terms at a time into the compensated sum
                                dfl_add(acc, d);
                                d = 0.f;
                            }
                            if (op.q0) {
                                const float2 ph = __ldg(lt + c);
                                x[i] = cmulc(x[i], ph);
                                r[i] = cmulc(r[i], ph);
                            }
                        }
                        add_gp(acc, 2.f * wgt * sig, L.grad, gj * 2 * p + l);
                    }
                    break;
                }
                default:
                    break;
            }
        }
        if (ps.store_psi) {
#pragma unroll
            for (int i = 0; i < NR; ++i) sp[int64_t(i) << b] = x[i];
        }
        if (GRAD && ps.store_lam) {
#pragma unroll
            for (int i = 0; i < NR; ++i) lp[int64_t(i) << b] = r[i];
        }
    }
}

// A pass made only of mixers: load, butterflies on the tile's qubits, store.
// No cut words or tables, so far fewer registers and more loads in flight.
__global__ void __launch_bounds__(128, 4) big_mix_kernel(const __grid_constant__ BigLaunch L) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const BigPass &ps = L.pass;
    const int b = ps.b;
    const int64_t tiles = int64_t(1) << (L.n_in - 10);
    const int64_t ntask = L.n_items * tiles;
    const int64_t block_amps = int64_t(1) << L.n_in;
    for (int64_t task = gw; task < ntask; task += nw) {
        const int64_t it = task / tiles;
        const int64_t tile = task - it * tiles;
        int ci;
        int64_t j, y;
        decode_item(L, L.item0 + it, ci, j, y);
        const DevCone *__restrict__ C = L.cones + L.cone_ids[ci];
        const float4 *__restrict__ cs = L.cs + (int64_t(C->graph) * L.P + j) * L.p;
        const int64_t lowmask = (int64_t(1) << (b - 5)) - 1;
        const int64_t xb = ((tile & lowmask) << 5) | ((tile >> (b - 5)) << (b + 5));
        float2 *__restrict__ sp = L.psi + it * block_amps + xb + lane;
        float2 x[NR];
#pragma unroll
        for (int i = 0; i < NR; ++i) x[i] = sp[int64_t(i) << b];
        for (int o = 0; o < ps.nops; ++o) {
            const BigOp op = ps.ops[o];
            const float4 c_s = __ldg(cs + op.layer);
            for (int q = op.q0; q < op.q1; ++q) {
                if (q < 5) {
                    const int m = 1 << q;
#pragma unroll
                    for (int i = 0; i < NR; ++i) {
                        float2 ot;
                        ot.x = __shfl_xor_sync(kFull, x[i].x, m);
                        ot.y = __shfl_xor_sync(kFull, x[i].y, m);
                        x[i] = rot(x[i], ot, c_s);
                    }
                } else {
                    const int rq = q - b;
#pragma unroll
                    for (int rb = 0; rb < kBigRegBits; ++rb) {
                        if (rb != rq) continue;
#pragma unroll
                        for (int i = 0; i < NR; ++i) {
                            if (i & (1 << rb)) continue;
                            const int i2 = i | (1 << rb);
                            const float2 a = x[i], bb = x[i2];
                            x[i] = rot(a, bb, c_s);
                            x[i2] = rot(bb, a, c_s);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NR; ++i) sp[int64_t(i) << b] = x[i];
    }
}

// (cos beta, sin beta) for the exact rotations, each as an FP32 pair hi + lo.
// Rounded to one FP32 number each, the gate becomes r exp(-i beta' X) with
// beta' - beta up to ~4e-8: the same shift for every amplitude, layer after
// layer, which a small gradient (near a stationary point, a second
// derivative times that shift) feels in full.  The lo parts (two more FMAs
// per output) take the shift away; what remains is per-operation rounding.
__global__ void big_prep_kernel(const double *params, int64_t GPp, int p, float4 *cs, float2 *fa) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < GPp; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t gj = i / p, l = i % p;
        double sn, c;
        sincos(params[gj * 2 * p + p + l], &sn, &c);
        const float ch = float(c), sh = float(sn);
        cs[i] = make_float4(ch, sh, float(c - double(ch)), float(sn - double(sh)));
        if (fa && l == 0) {
            // the first layer's factored coefficient: tan beta, or cot beta where
            // |tan beta| > 1 (the same choice, and the same rounded hi part, as
            // the register kernels' mixer table), with its FP32 rounding error
            const double a = fabs(sn) > fabs(c) ? c / sn : sn / c;
            const float ah = float(a);
            fa[gj] = make_float2(ah, float(a - double(ah)));
        }
    }
}

}  // namespace

cudaError_t launch_big_prep(const double *params, int64_t GP, int p, float4 *cs, float2 *fa, cudaStream_t s) {
    const int64_t n = GP * p;
    int blocks = int(std::min<int64_t>((n + 255) / 256, 1024));
    big_prep_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, s>>>(params, n, p, cs, fa);
    return cudaGetLastError();
}

int occupancy_grid(const void *fn, int block, size_t smem);

int big_grid(bool grad) {
    return grad ? occupancy_grid((const void *)big_pass_kernel<true>, 128, 0)
                : occupancy_grid((const void *)big_pass_kernel<false>, 128, 0);
}

static int mix_grid() { return occupancy_grid((const void *)big_mix_kernel, 128, 0); }

static bool mix_only(const BigPass &ps) {
    if (!ps.load_psi || !ps.store_psi || ps.load_lam || ps.store_lam) return false;
    for (int o = 0; o < ps.nops; ++o)
        if (ps.ops[o].type != kOpMix) return false;
    return true;
}

cudaError_t launch_big_pass(const BigLaunch &a, bool grad, int grid, cudaStream_t s) {
    const int64_t tasks = a.n_items * (int64_t(1) << (a.n_in - 10));
    const int64_t need = (tasks + 3) / 4;
    if (mix_only(a.pass)) {
        big_mix_kernel<<<int(std::min<int64_t>(mix_grid(), need < 1 ? 1 : need)), 128, 0, s>>>(a);
        return cudaGetLastError();
    }
    const int g = int(std::min<int64_t>(grid, need < 1 ? 1 : need));
    if (grad)
        big_pass_kernel<true><<<g, 128, 0, s>>>(a);
    else
        big_pass_kernel<false><<<g, 128, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------ pass lists

namespace {

// Register window [b, b+5) of the tile that holds qubits [lo, hi)
int window_for(int lo, int n_in) { return lo < 10 ? 5 : std::min(lo, n_in - 5); }

bool fits(const BigPass &ps, int q0, int q1) {
    for (int q = q0; q < q1; ++q)
        if (!(q < 5 || (q >= ps.b && q < ps.b + 5))) return false;
    return true;
}

}  // namespace

// Forward op list for one cone shape, split into passes.  Layer l applies
// its phase, then its mixer on the qubit groups [10,15), [15,20), ... (each
// in its own register window) and finally on [0, 10) in window 5, so that
// the low group fuses with the next layer's phase and, when that layer only
// mixes low qubits, with its mixer too.
std::vector<BigPass> big_forward_passes(int n_in, int p, const int32_t *k) {
    std::vector<BigPass> out;
    auto push_op = [&](uint8_t type, int layer, int q0, int q1, int want_b) {
        if (out.empty() || (type == kOpMix && !fits(out.back(), q0, q1)) || out.back().nops >= kBigMaxOps) {
            BigPass ps{};
            ps.b = want_b;
            out.push_back(ps);
        }
        BigPass &ps = out.back();
        ps.ops[ps.nops++] = BigOp{type, uint8_t(layer), uint8_t(q0), uint8_t(q1)};
    };
    for (int l = 0; l < p; ++l) {
        const int kl = k[l];
        std::vector<std::pair<int, int>> groups;
        for (int lo = 10; lo < kl; lo += 5) groups.emplace_back(lo, std::min(lo + 5, kl));
        groups.emplace_back(0, std::min(kl, 10));
        const int first_b = window_for(groups.front().first, n_in);
        push_op(l == 0 ? kOpGenPhase : kOpPhase, l, 0, 0, first_b);
        for (auto &gq : groups) push_op(kOpMix, l, gq.first, gq.second, window_for(gq.first, n_in));
    }
    push_op(kOpReduce, 0, 0, 0, 5);
    for (size_t i = 0; i < out.size(); ++i) {
        out[i].load_psi = i > 0;
        out[i].store_psi = i + 1 < out.size();
    }
    return out;
}

// Adjoint: the forward passes, except that the last one continues with the
// co-state initialisation and the inverse of its own ops; then the earlier
// passes in reverse order with inverted ops.  An inverted phase of layer 0
// only contributes its derivative.
std::vector<BigPass> big_grad_passes(int n_in, int p, const int32_t *k) {
    std::vector<BigPass> fwd = big_forward_passes(n_in, p, k);
    std::vector<BigPass> out;
    auto invert = [](const BigPass &src, BigPass &dst) {
        for (int o = src.nops - 1; o >= 0; --o) {
            const BigOp &op = src.ops[o];
            BigOp inv = op;
            if (op.type == kOpReduce) continue;
            if (op.type == kOpMix) inv.type = kOpUnmix;
            if (op.type == kOpPhase) inv = BigOp{kOpUnphase, op.layer, 1, 0};
            if (op.type == kOpGenPhase) inv = BigOp{kOpUnphase, op.layer, 0, 0};
            dst.ops[dst.nops++] = inv;
        }
    };
    for (size_t i = 0; i < fwd.size(); ++i) {
        BigPass ps = fwd[i];
        if (i + 1 < fwd.size()) {
            out.push_back(ps);  // forward part, stores psi
            continue;
        }
        // last forward pass: forward ops, reduce, co-state, inverse ops
        ps.ops[ps.nops++] = BigOp{kOpLamInit, 0, 0, 0};
        invert(fwd[i], ps);
        ps.store_psi = fwd.size() > 1;
        ps.store_lam = fwd.size() > 1;
        out.push_back(ps);
    }
    for (int i = int(fwd.size()) - 2; i >= 0; --i) {
        BigPass ps{};
        ps.b = fwd[i].b;
        invert(fwd[i], ps);
        ps.load_psi = true;
        ps.load_lam = true;
        ps.store_psi = i > 0;
        ps.store_lam = i > 0;
        out.push_back(ps);
    }
    return out;
}

}  // namespace qaoa
