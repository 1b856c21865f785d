// Device helpers shared by the large-state kernels.
#pragma once

#include "big.cuh"

namespace qaoa {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// Im(conj(a) b)
__device__ __forceinline__ float imconj(float2 a, float2 b) { return a.x * b.y - a.y * b.x; }
// c me - i s other: one output of exp(-i beta X) on the pair (me, other)
__device__ __forceinline__ float2 rot(float2 me, float2 o, float c, float s) {
    return make_float2(fmaf(c, me.x, s * o.y), fmaf(c, me.y, -s * o.x));
}

// Warp sum in FP32, then one FP64 atomic into base[idx].
__device__ __forceinline__ void add_gp(float v, double *base, int64_t idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(base + idx, double(v));
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
