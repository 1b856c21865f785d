// Device arithmetic shared by every kernel: complex64 helpers and the
// compensated FP32 sums the derivative reductions use.
#pragma once

#include <cstdint>

namespace qaoa {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// Im(conj(a) b)
__device__ __forceinline__ float imconj(float2 a, float2 b) { return a.x * b.y - a.y * b.x; }

// An unevaluated FP32 sum hi + lo.  A derivative of E is a sum of terms of
// size O(1) (per amplitude, weighted by shell multiplicities and orbit sizes)
// that cancel to ~1e-4 of their size near a stationary point; a plain FP32
// running sum then loses about as many digits as the cancellation removes.
// Adding with an error-free transformation (Knuth's TwoSum: s = a + b exactly
// equals fl(a + b) + err) keeps the rounding error of every addition in lo,
// so the sum of hi + lo is exact up to the rounding of the lo additions,
// which are relative to lo.  The intrinsics keep the compiler from fusing or
// reassociating the steps.
struct Dfl {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc += v
__device__ __forceinline__ void dfl_add(Dfl &acc, float v) {
    float s, e;
    two_sum(acc.hi, v, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, e);
}

// acc += w * v with the product's rounding error kept as well
__device__ __forceinline__ void dfl_fma(Dfl &acc, float w, float v) {
    const float p = __fmul_rn(w, v);
    const float pe = __fmaf_rn(w, v, -p);  // w v - p, exact
    float s, e;
    two_sum(acc.hi, p, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pe));
}

// acc += other
__device__ __forceinline__ void dfl_add(Dfl &acc, Dfl o) {
    float s, e;
    two_sum(acc.hi, o.hi, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, o.lo));
}

// a * f with the rounding error of hi * f kept in lo
__device__ __forceinline__ Dfl dfl_scale(Dfl a, float f) {
    const float p = __fmul_rn(a.hi, f);
    const float pe = __fmaf_rn(a.hi, f, -p);  // a.hi f - p, exact
    return Dfl{p, __fmaf_rn(a.lo, f, pe)};
}

// Sum over the 32 lanes of the warp (every lane gets it).
__device__ __forceinline__ Dfl dfl_warp_sum(Dfl a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Dfl b;
        b.hi = __shfl_xor_sync(kFull, a.hi, o);
        b.lo = __shfl_xor_sync(kFull, a.lo, o);
        dfl_add(a, b);
    }
    return a;
}

__device__ __forceinline__ double dfl_value(Dfl a) { return double(a.hi) + double(a.lo); }

// float -> double by bit manipulation: the conversion instruction runs on the
// FP64 pipe, which on this part issues at 1/64 of the FP32 rate, so kernels
// that convert a partial sum for every FP64 atomic build the double's bits
// with integer operations instead.  Zero and subnormal floats (|x| < 2^-126)
// give 0; infinities and NaNs stay infinities and NaNs.
__device__ __forceinline__ double f2d(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    const uint32_t ed = e == 0xffu ? 0x7ffu : e + 896u;  // rebias 127 -> 1023
    const uint32_t hi = (b & 0x80000000u) | (ed << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double(int(hi), int(b << 29));
}

}  // namespace qaoa
