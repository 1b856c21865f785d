// Device helpers shared by the large-state kernels.
#pragma once

#include "big.cuh"
#include "dev_math.cuh"

namespace qaoa {
namespace {

// c me - i s other: one output of exp(-i beta X) on the pair (me, other),
// with c = cs.x + cs.z and s = cs.y + cs.w (hi and lo FP32 parts)
__device__ __forceinline__ float2 rot(float2 me, float2 o, float4 cs) {
    return make_float2(fmaf(cs.x, me.x, fmaf(cs.y, o.y, fmaf(cs.z, me.x, cs.w * o.y))),
                       fmaf(cs.x, me.y, fmaf(-cs.y, o.x, fmaf(cs.z, me.y, -cs.w * o.x))));
}
// the same for exp(+i beta X)
__device__ __forceinline__ float2 unrot(float2 me, float2 o, float4 cs) {
    return make_float2(fmaf(cs.x, me.x, fmaf(-cs.y, o.y, fmaf(cs.z, me.x, -cs.w * o.y))),
                       fmaf(cs.x, me.y, fmaf(cs.y, o.x, fmaf(cs.z, me.y, cs.w * o.x))));
}

// Warp sum in FP32, then one FP64 atomic into base[idx] (energies and terms,
// whose sums do not cancel).
__device__ __forceinline__ void add_gp(float v, double *base, int64_t idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(base + idx, double(v));
}

// Compensated warp sum of a derivative partial times w, then one FP64
// atomic into base[idx].
__device__ __forceinline__ void add_gp(Dfl v, float w, double *base, int64_t idx) {
    v = dfl_warp_sum(dfl_scale(v, w));
    if ((threadIdx.x & 31) == 0) atomicAdd(base + idx, dfl_value(v));
}

// Item -> (cone of the shape, point j, shell block y).  Cone c owns the items
// P * [ystart[c], ystart[c+1]), ordered point-major.
__device__ __forceinline__ void decode_item(const BigLaunch &L, int64_t item, int &ci, int64_t &j, int64_t &y) {
    int lo = 0, hi = L.n_shape - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.P * L.ystart[mid] <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    const int64_t Y = L.ystart[lo + 1] - L.ystart[lo];
    const int64_t rem = item - L.P * L.ystart[lo];
    j = rem / Y;
    y = rem - j * Y;
    ci = lo;
}

}  // namespace
}  // namespace qaoa
