// Pieces shared by the register-resident cone kernels (the general kernel in
// cone_kernel.cuh and the depth-1 kernel in p1_kernel.cu): asynchronous
// staging of the point tables, the factored mixer butterfly, and the grouped
// warp reduction of the per-point outputs.
#pragma once

#include "dev_math.cuh"
#include "device.cuh"

namespace qaoa {

// cp.async copies of 8 and 4 bytes from global to shared memory (both
// addresses aligned to the size), and the wait for all of this thread's.
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// u - i tau v: one output of the butterfly (I - i tau X) on the pair (u, v)
__device__ __forceinline__ float2 bfly(float2 u, float2 v, float tau) {
    return make_float2(fmaf(tau, v.y, u.x), fmaf(-tau, v.x, u.y));
}

// d += Im(conj(a) b) as two FMAs (written out: the compiler may not contract
// a separate product and sum)
__device__ __forceinline__ void acc_imconj(float &d, float2 a, float2 b) {
    d = fmaf(a.x, b.y, d);
    d = fmaf(-a.y, b.x, d);
}

// Sum of v over the lanes of each run of equal keys (runs are contiguous);
// the result is valid in the run's first lane, which returns true.
__device__ __forceinline__ bool seg_sum(float &v, int key) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float ov = __shfl_down_sync(kFull, v, o);
        const int ok = __shfl_down_sync(kFull, key, o);
        if (lane + o < 32 && ok == key) v += ov;
    }
    const int prev = __shfl_up_sync(kFull, key, 1);
    return lane == 0 || prev != key;
}

// Warp sums of the per-point outputs of the group of points ending at jj.
// red holds this warp's FP32 shares: output c (0: energy, 1 + i: gradient
// component i) of point jj' of the group sits at [c][jj' mod G][(lane + jj')
// mod 32] (the skew keeps these reads free of bank conflicts).  Lane =
// (part, point): each lane adds G lanes' shares of its point with
// compensation, the parts meet by shuffles, and lanes of part 0 add hi and lo
// to the FP64 outputs of row row0 + point (row0 = g * n_points + first point
// of the task) with separate atomics (no FP64 arithmetic).  Called by the
// whole warp between __syncwarp()s.
template <int UNROLL>
__device__ __forceinline__ void reg_flush(const float *red, int nout, int G, int jj, int lane, int64_t row0,
                                          int n_grad, double *energy, double *grad) {
    const int gn = (jj & (G - 1)) + 1, jf = jj + 1 - gn;
    const int pt = lane & (G - 1), part = lane / G;
#pragma unroll(UNROLL)
    for (int c = 0; c < nout; ++c) {
        const float *src = red + (c * G + pt) * 32;
        Dfl acc{0.f, 0.f};
        for (int k = 0; k < G; ++k) dfl_add(acc, src[(part * G + k + jf + pt) & 31]);
        for (int o = G; o < 32; o <<= 1) {
            Dfl b;
            b.hi = __shfl_xor_sync(kFull, acc.hi, o);
            b.lo = __shfl_xor_sync(kFull, acc.lo, o);
            dfl_add(acc, b);
        }
        if (part == 0 && pt < gn) {
            const int64_t gjj = row0 + jf + pt;
            double *dst = c == 0 ? energy + gjj : grad + gjj * n_grad + (c - 1);
            atomicAdd(dst, f2d(acc.hi));
            if (acc.lo != 0.f) atomicAdd(dst, f2d(acc.lo));
        }
    }
}

}  // namespace qaoa
