// Depth-1 register kernel: energy, or energy and adjoint gradient, at p = 1.
//
// At p = 1 the mixer of the only layer acts, after gate pruning (Sec. 2.3),
// on the qubits within distance p - 1 = 0 of the edge: qubits 0 and 1 (u, v)
// alone.  Every other cone qubit stays classical, so a cone's state is a sum
// of independent 4-amplitude blocks, one per shell assignment (merged into
// shell blocks with multiplicities, see DevCone), and the amplitudes of one
// block never meet those of another.  The kernel therefore works on a flat
// list of blocks per graph (the blocks of all of the graph's representative
// cones, back to back): a thread takes kP1Blocks consecutive blocks and, for
// each parameter point, evolves them one after the other.  Only one block's
// amplitudes are live at a time, which leaves registers for more resident
// warps, and the per-point costs (table pointers, the output stash and the
// warp reductions) are shared by 16 blocks.
//
// Per block, with amplitude a = z_u + 2 z_v and c_a its cut value, and the
// record's weight W = (block multiplicity) x (orbit size) x 2^-n, all fixed
// at upload, in the stored form psi = kappa^2 2^-n/2 x of the general kernel:
//   s_a = exp(-i gamma c_a) from the phase table (|+> up to 2^-n/2),
//   x = (I - i tau X_v)(I - i tau X_u) s,
//   orbit-weighted <Z_u Z_v> = kappa^4 W (|x_0|^2 + |x_3|^2 - |x_1|^2 - |x_2|^2)  (Sec. 2.4),
// and E gets -1/2 of it.  Adjoint (co-state lambda = -1/2 Z_u Z_v psi, r =
// Z_u Z_v x):
//   dE/dbeta = 2 Im<lambda|X_u + X_v|psi>.  With r = Z_u Z_v x the two pair
//     terms of a qubit coincide, Im(conj r_i x_j) = Im(conj r_j x_i), so
//     Im<r|X_u + X_v|x> = 2 [Im(x_0* x_1) - Im(x_2* x_3) + Im(x_0* x_2) - Im(x_1* x_3)]
//     (half the products of the general form);
//   dE/dgamma = 2 Im<lambda|C|s> with the mixer undone on r.  Im<r|s> is
//     zero within every block (it equals <x|Z_u Z_v|x>, which is real), so C
//     may be shifted by any per-block constant: the block's first cut value
//     c_0, which drops one of the four terms.  The upload orders each block's
//     amplitudes so that c_0 is the one of its four cut values nearest their
//     middle (relabelling by X_u, X_v or both, which leave |+> and the mixers
//     unchanged and turn Z_u Z_v into -Z_u Z_v, +Z_u Z_v: the weight W takes
//     the sign).  That keeps the weights c_a - c_0 within about half the
//     block's spread, which limits how much of the FP32 state's rounding the
//     cancelling sum keeps.
// The block terms are accumulated per thread in four partial sums (blocks
// mod 4) and the lanes' shares of each point are summed with compensation
// (reg_flush).
#include "reg_common.cuh"

namespace qaoa {

int occupancy_grid(const void *fn, int block, size_t smem);

namespace {

// (I - i tau X) on qubit 0 (pairs (0,1), (2,3)), then on qubit 1 ((0,2), (1,3))
__device__ __forceinline__ void mix01(float2 (&x)[4], float tau) {
    float2 a = x[0], b = x[1];
    x[0] = bfly(a, b, tau);
    x[1] = bfly(b, a, tau);
    a = x[2];
    b = x[3];
    x[2] = bfly(a, b, tau);
    x[3] = bfly(b, a, tau);
    a = x[0];
    b = x[2];
    x[0] = bfly(a, b, tau);
    x[2] = bfly(b, a, tau);
    a = x[1];
    b = x[3];
    x[1] = bfly(a, b, tau);
    x[3] = bfly(b, a, tau);
}

// Count byte a of w as the FP32 value 2^23 + c (its bit pattern is
// 0x4B0000cc): one byte permute, and differences of two such values are
// exact FP32 subtractions
__device__ __forceinline__ uint32_t count_bits(uint32_t w, int a) { return __byte_perm(w, 0x4B000000u, 0x7540u | a); }

// float2 at a 32-bit shared-memory address
__device__ __forceinline__ float2 lds2(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

template <bool GRAD>
__global__ void __launch_bounds__(kRegBlock, GRAD ? kP1GradMinBlocks : kP1EnergyMinBlocks)
    reg_p1_kernel(const RegLaunch L) {
    extern __shared__ float2 s_tab[];
    constexpr int kWarps = kRegBlock / 32;
    constexpr int NOUT = reg_outputs(1, GRAD);
    constexpr int G = reg_p1_group(GRAD);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const RegWork &W = L.work;
    const int cm1 = L.cmax1;
    // per warp: the phase tables of the task's points (cmax1 float2 each),
    // (tau, kappa^4) per point, the slots' records, and the reduction buffer
    float2 *my_tab = s_tab + warp * (L.jpt * cm1);
    float2 *my_mix = s_tab + kWarps * (L.jpt * cm1) + warp * L.jpt;
    uint2 *my_rec = reinterpret_cast<uint2 *>(s_tab + kWarps * (L.jpt * (cm1 + 1))) + warp * (kP1Blocks * 32);
    float *red = reinterpret_cast<float *>(s_tab + kWarps * (L.jpt * (cm1 + 1) + kP1Blocks * 32)) +
                 warp * (NOUT * G * 32);
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int64_t nblk = (L.n_points + L.jpt - 1) / L.jpt;
    const int64_t ntask = W.warps * nblk;
    for (int64_t task = gw; task < ntask; task += nw) {
        const int64_t jb = task / W.warps;
        const int64_t w = task - jb * W.warps;
        const int64_t j0 = jb * L.jpt;
        const int jn = int(L.n_points - j0 < L.jpt ? L.n_points - j0 : L.jpt);
        const int64_t slot = w * 32 + lane;  // < W.slots: the slot count is a multiple of 32
        const int gwarp = __ldg(W.warp_graph + w);
        const int64_t row0 = int64_t(gwarp) * L.n_points + j0;
        __syncwarp();  // the previous task's reads of the staged data are done
        {
            const float2 *__restrict__ src = L.lut + row0 * cm1;
            for (int e = lane; e < jn * cm1; e += 32) cp_async8(my_tab + e, src + e);
            for (int e = lane; e < jn; e += 32) {
                cp_async4(&my_mix[e].x, &L.mix[row0 + e].x);
                cp_async4(&my_mix[e].y, L.kpow + (row0 + e) * kKpow + 2);  // kappa^(2 k), k = 2
            }
#pragma unroll
            for (int k = 0; k < kP1Blocks; ++k) cp_async8(my_rec + k * 32 + lane, W.rec_cw + k * W.slots + slot);
        }
        cp_async_wait_all();
        __syncwarp();  // the staged data are complete and visible to the warp
        for (int jj = 0; jj < jn; ++jj) {
            // address of entry c is lut0 + 8 (2^23 + c) (mod 2^32): the counts
            // are read as 2^23 + c, see count_bits
            const uint32_t lut0 = static_cast<uint32_t>(__cvta_generic_to_shared(my_tab + jj * cm1)) - (0x4B000000u << 3);
            const float2 tk = my_mix[jj];
            const float tau = tk.x;
            float e4[4] = {0.f, 0.f, 0.f, 0.f};
            float b4[4] = {0.f, 0.f, 0.f, 0.f};
            float g4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 16
            for (int b = 0; b < kP1Blocks; ++b) {
                const uint2 rc = my_rec[b * 32 + lane];
                const float wb = __uint_as_float(rc.y);
                uint32_t c[4];
                float2 s[4], x[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    c[a] = count_bits(rc.x, a);
                    s[a] = lds2(lut0 + (c[a] << 3));
                    x[a] = s[a];
                }
                mix01(x, tau);
                const float pos = fmaf(x[0].x, x[0].x, fmaf(x[0].y, x[0].y, fmaf(x[3].x, x[3].x, x[3].y * x[3].y)));
                const float neg = fmaf(x[1].x, x[1].x, fmaf(x[1].y, x[1].y, fmaf(x[2].x, x[2].x, x[2].y * x[2].y)));
                e4[b & 3] = fmaf(wb, pos - neg, e4[b & 3]);
                if constexpr (GRAD) {
                    // half of Im<r|X_u + X_v|x> (each pair term once)
                    float d = 0.f;
                    acc_imconj(d, x[0], x[1]);
                    acc_imconj(d, x[0], x[2]);
                    d = fmaf(-x[2].x, x[3].y, d);
                    d = fmaf(x[2].y, x[3].x, d);
                    d = fmaf(-x[1].x, x[3].y, d);
                    d = fmaf(x[1].y, x[3].x, d);
                    b4[b & 3] = fmaf(wb, d, b4[b & 3]);
                    // r = Z_u Z_v x, then the mixer undone on r
                    float2 r[4] = {x[0], make_float2(-x[1].x, -x[1].y), make_float2(-x[2].x, -x[2].y), x[3]};
                    mix01(r, -tau);
                    float dg = 0.f;
#pragma unroll
                    for (int a = 1; a < 4; ++a)
                        dg = fmaf(__uint_as_float(c[a]) - __uint_as_float(c[0]), imconj(r[a], s[a]), dg);
                    g4[b & 3] = fmaf(wb, dg, g4[b & 3]);
                }
            }
            const float k4 = tk.y;
            const int col = (lane + jj) & 31;
            red[(jj & (G - 1)) * 32 + col] = -0.5f * k4 * ((e4[0] + e4[1]) + (e4[2] + e4[3]));
            if constexpr (GRAD) {
                // gamma_1, then beta_1 (the pair terms were counted once above)
                red[(1 * G + (jj & (G - 1))) * 32 + col] = -k4 * ((g4[0] + g4[1]) + (g4[2] + g4[3]));
                red[(2 * G + (jj & (G - 1))) * 32 + col] = -2.f * k4 * ((b4[0] + b4[1]) + (b4[2] + b4[3]));
            }
            if ((jj & (G - 1)) == G - 1 || jj == jn - 1) {
                __syncwarp();
                reg_flush<NOUT>(red, NOUT, G, jj, lane, row0, 2, L.energy, L.grad);
                __syncwarp();
            }
        }
    }
}

}  // namespace

int reg_p1_grid(bool grad, size_t smem) {
    return grad ? occupancy_grid((const void *)reg_p1_kernel<true>, kRegBlock, smem)
                : occupancy_grid((const void *)reg_p1_kernel<false>, kRegBlock, smem);
}

cudaError_t reg_p1_prepare() {
    cudaError_t e = cudaFuncSetAttribute((const void *)reg_p1_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kRegMaxSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)reg_p1_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kRegMaxSmem);
    return e;
}

cudaError_t launch_reg_p1(const RegLaunch &a, bool grad, int grid, cudaStream_t s) {
    const size_t sm = reg_p1_smem_bytes(a.jpt, a.cmax1, grad);
    if (grad)
        reg_p1_kernel<true><<<grid, kRegBlock, sm, s>>>(a);
    else
        reg_p1_kernel<false><<<grid, kRegBlock, sm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace qaoa
