// Sums of many FP32 terms carried as an unevaluated pair hi + lo of FP32
// values (double-float arithmetic): every addition is Knuth's TwoSum, which
// returns the rounding error exactly, and every product x*y is split into its
// rounded value and the exact remainder fma(x, y, -x*y).  The pair carries
// about 48 significant bits, close to an FP64 accumulator, but every step runs
// on the FP32 pipes: on this GPU the FP64 rate is about 1/64 of the FP32 rate,
// so per-element FP64 accumulation would cost more than the loads it follows.
// The explicit _rn intrinsics keep the compiler from contracting or
// reassociating the error terms.
#pragma once

#include <cuda_runtime.h>

struct fpair {
    float hi, lo;
};

__device__ __forceinline__ fpair fpair_zero() { return fpair{0.0f, 0.0f}; }

// s + e == a + b exactly (TwoSum)
__device__ __forceinline__ void fpair_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a += x + t (t a small correction), renormalised so that |lo| stays within
// half an ulp of hi: without it lo grows with the number of terms and its own
// FP32 rounding takes over
__device__ __forceinline__ void fpair_accum(fpair& a, float x, float t) {
    float s, e;
    fpair_two_sum(a.hi, x, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, t));
    fpair_two_sum(s, e, a.hi, a.lo);
}

__device__ __forceinline__ void fpair_add(fpair& a, float x) { fpair_accum(a, x, 0.0f); }

// a += x * y, the product's rounding error kept
__device__ __forceinline__ void fpair_add_prod(fpair& a, float x, float y) {
    const float p = __fmul_rn(x, y);
    fpair_accum(a, p, __fmaf_rn(x, y, -p));
}

// a += (x - y)^2 with the difference and the square carried exactly to first order
__device__ __forceinline__ void fpair_add_sqdiff(fpair& a, float x, float y) {
    const float d = __fsub_rn(x, y);
    const float bb = __fsub_rn(d, x);
    const float de = __fsub_rn(__fsub_rn(x, __fsub_rn(d, bb)), __fadd_rn(y, bb));   // d + de == x - y
    const float p = __fmul_rn(d, d);
    fpair_accum(a, p, __fmaf_rn(__fmul_rn(2.0f, d), de, __fmaf_rn(d, d, -p)));
}

__device__ __forceinline__ void fpair_add(fpair& a, fpair b) { fpair_accum(a, b.hi, b.lo); }

// Sum over the warp, in lane order of a fixed tree (deterministic); the
// result is valid in lane 0.
__device__ __forceinline__ fpair fpair_warp_sum(fpair a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fpair b;
        b.hi = __shfl_down_sync(0xffffffffu, a.hi, o);
        b.lo = __shfl_down_sync(0xffffffffu, a.lo, o);
        fpair_add(a, b);
    }
    return a;
}

// Sum over the block (at most 32 warps, blockDim.x a multiple of 32; every
// thread calls it); the result is valid in thread 0.  Uses one shared array,
// so two calls in a row need a __syncthreads() between them.
__device__ __forceinline__ fpair fpair_block_sum(fpair a) {
    __shared__ fpair red[32];
    const int nw = (int)(blockDim.x >> 5);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = fpair_warp_sum(a);
    if (lane == 0) red[warp] = a;
    __syncthreads();
    fpair s = fpair_zero();
    if (warp == 0) {
        if (lane < nw) s = red[lane];
        s = fpair_warp_sum(s);
    }
    return s;
}

__device__ __forceinline__ double fpair_value(fpair a) { return (double)a.hi + (double)a.lo; }

