// Float-float arithmetic for the refinement loop of the FP32 precisions.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers (about 48
// significant bits).  The building blocks are the classical error-free
// transformations: Knuth's TwoSum (s + e = a + b exactly, any order),
// Dekker's Fast2Sum (the same when |a| >= |b|) and the exact product through
// a fused multiply-add (a b = p + e with e = fma(a, b, -p)).  The operations
// on pairs are the short forms of Dekker's double-length arithmetic (the
// "double-single" arithmetic of Bailey's packages): the absolute error of a
// sum or product is a few units of 2^-48 times the operands' magnitude.
// That is what the residual b - L p needs: its terms cancel, so its error is
// set by the magnitude of the terms, not of the result.  GB300's FP32 rate is
// tens of times its FP64 rate: the FP64 versions of these kernels were bound
// by the FP64 units, the float-float ones come close to memory speed.
//
// The _rn intrinsics keep every step a separately rounded operation (no
// contraction into fused multiply-adds, no reassociation).
#pragma once

#include <cuda_runtime.h>

#include "fpconv.cuh"

namespace osm {

struct FF {
    float hi, lo;
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// the pair of a + b (two floats), exact
__device__ __forceinline__ FF ff_sum2(float a, float b) {
    FF r;
    two_sum(a, b, r.hi, r.lo);
    return r;
}

// a + b of two pairs, normalised
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    FF r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

// a - b of two pairs, not normalised: the high parts' difference exactly,
// plus the low parts' difference (for the face differences p_C - p_n, which
// are only summed afterwards)
__device__ __forceinline__ FF ff_diff(FF a, FF b) {
    FF r;
    two_sum(a.hi, -b.hi, r.hi, r.lo);
    r.lo = __fadd_rn(r.lo, __fsub_rn(a.lo, b.lo));
    return r;
}

// a * b of two pairs (the lo * lo term is below the pair's precision)
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    FF r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// the pair nearest a double (hi = x rounded to FP32, lo = the rest rounded)
__host__ __device__ inline FF ff_from_double(double x) {
    const float h = (float)x;
    return FF{h, (float)(x - (double)h)};
}

// the halves widen exactly on the integer units (fpconv.cuh): one FP64 add
__device__ __forceinline__ double ff_to_double(FF a) { return f32_to_f64(a.hi) + f32_to_f64(a.lo); }

// per-thread running sum for the reductions: a pair, with the rounding error
// of every addition carried in lo
struct FFAcc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x) {
        float s, e;
        two_sum(hi, x, s, e);
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

}  // namespace osm
