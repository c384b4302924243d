// Accumulators of the library's long sums: inner products, residual norms and
// the SSD (Eq. 10).  Every element's contribution enters an accumulator of
// type `lsum`; warps and blocks combine accumulators in a fixed shuffle tree
// (deterministic), and per-block results are stored and combined in FP64.
//
// Two accumulators, chosen when the library is built (LGNK_SUMS):
//
//  2 (default) FP64 per element.  Each FP32 operand is widened to FP64 by
//    rewriting its IEEE-754 fields (sign, exponent rebiased from 127 to 1023,
//    the 23 mantissa bits moved to the top of the 52), integer instructions
//    only; zero stays zero, and the rare subnormal, infinite or NaN operand
//    takes the hardware conversion.  The product of two widened operands is
//    exact in FP64 (24 + 24 bits), so x*y + acc is one FP64 fused multiply-add
//    per element: FP64's range and a 53-bit accumulator.  On this GPU the
//    FP64 rate is about 1/64 of the FP32 rate, which is why the widening does
//    not use the FP64 pipe as well.
//  1 FP64 per element with the hardware conversion (cvt.f64.f32).
//  0 Pairs of FP32 values (double-float arithmetic): every addition is
//    Knuth's TwoSum, which returns its rounding error exactly, and every
//    product x*y is split into its rounded value and the exact remainder
//    fma(x, y, -x*y).  About 48 significant bits on the FP32 pipes only, but
//    FP32's exponent range: a product below about 1e-38 loses its low word
//    and one below about 1e-45 vanishes.
//
// The explicit _rn intrinsics keep the compiler from contracting or
// reassociating the error terms of the pair arithmetic.
#pragma once

#include <cuda_runtime.h>

#ifndef LGNK_SUMS
#define LGNK_SUMS 2
#endif

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

__device__ __forceinline__ fpair fpair_shfl_down(fpair a, int o) {
    return fpair{__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}

__device__ __forceinline__ double fpair_value(fpair a) { return (double)a.hi + (double)a.lo; }

// ---- FP64 per element ----

// x widened to FP64 exactly.
__device__ __forceinline__ double widen(float x) {
#if LGNK_SUMS == 2
    const unsigned f = __float_as_uint(x);
    const unsigned e = (f >> 23) & 0xffu;
    if (e - 1u < 254u) {        // normal: rebias the exponent, move the mantissa
        const unsigned hi = (((f >> 3) & 0x0fffffffu) + 0x38000000u) | (f & 0x80000000u);
        return __hiloint2double((int)hi, (int)(f << 29));
    }
    if ((f & 0x7fffffffu) == 0u) return __hiloint2double((int)(f & 0x80000000u), 0);   // +-0
    return (double)x;           // subnormal, infinity, NaN
#else
    return (double)x;
#endif
}

struct dsum {
    double v;
};

__device__ __forceinline__ dsum dsum_zero() { return dsum{0.0}; }
__device__ __forceinline__ void dsum_add(dsum& a, dsum b) { a.v += b.v; }
__device__ __forceinline__ void dsum_add(dsum& a, float x) { a.v += widen(x); }
__device__ __forceinline__ void dsum_add_prod(dsum& a, float x, float y) { a.v = fma(widen(x), widen(y), a.v); }
// (x - y)^2: the FP64 difference of two FP32 values is exact unless their
// exponents differ by more than 29, and then the rounding is below 2^-53 of it
__device__ __forceinline__ void dsum_add_sqdiff(dsum& a, float x, float y) {
    const double d = widen(x) - widen(y);
    a.v = fma(d, d, a.v);
}
__device__ __forceinline__ dsum dsum_shfl_down(dsum a, int o) { return dsum{__shfl_down_sync(0xffffffffu, a.v, o)}; }
__device__ __forceinline__ double dsum_value(dsum a) { return a.v; }

// ---- the library's accumulator ----

#if LGNK_SUMS == 0
using lsum = fpair;
__device__ __forceinline__ lsum lsum_zero() { return fpair_zero(); }
__device__ __forceinline__ void lsum_add(lsum& a, lsum b) { fpair_add(a, b); }
__device__ __forceinline__ void lsum_add(lsum& a, float x) { fpair_add(a, x); }
__device__ __forceinline__ void lsum_add_prod(lsum& a, float x, float y) { fpair_add_prod(a, x, y); }
__device__ __forceinline__ void lsum_add_sqdiff(lsum& a, float x, float y) { fpair_add_sqdiff(a, x, y); }
__device__ __forceinline__ lsum lsum_shfl_down(lsum a, int o) { return fpair_shfl_down(a, o); }
__device__ __forceinline__ double lsum_value(lsum a) { return fpair_value(a); }
#else
using lsum = dsum;
__device__ __forceinline__ lsum lsum_zero() { return dsum_zero(); }
__device__ __forceinline__ void lsum_add(lsum& a, lsum b) { dsum_add(a, b); }
__device__ __forceinline__ void lsum_add(lsum& a, float x) { dsum_add(a, x); }
__device__ __forceinline__ void lsum_add_prod(lsum& a, float x, float y) { dsum_add_prod(a, x, y); }
__device__ __forceinline__ void lsum_add_sqdiff(lsum& a, float x, float y) { dsum_add_sqdiff(a, x, y); }
__device__ __forceinline__ lsum lsum_shfl_down(lsum a, int o) { return dsum_shfl_down(a, o); }
__device__ __forceinline__ double lsum_value(lsum a) { return dsum_value(a); }
#endif

// Sum over the warp, in lane order of a fixed tree (deterministic); the
// result is valid in lane 0.
__device__ __forceinline__ lsum lsum_warp_sum(lsum a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum_add(a, lsum_shfl_down(a, o));
    return a;
}

// Sum over the block (at most 32 warps, blockDim.x a multiple of 32; every
// thread calls it); the result is valid in thread 0.  Uses one shared array,
// so two calls in a row need a __syncthreads() between them.
__device__ __forceinline__ lsum lsum_block_sum(lsum a) {
    __shared__ lsum red[32];
    const int nw = (int)(blockDim.x >> 5);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = lsum_warp_sum(a);
    if (lane == 0) red[warp] = a;
    __syncthreads();
    lsum s = lsum_zero();
    if (warp == 0) {
        if (lane < nw) s = red[lane];
        s = lsum_warp_sum(s);
    }
    return s;
}
