// Double-float arithmetic: a value is hi + lo with two float32 parts
// (|lo| <= ulp(hi)/2), about 48 significant bits. Used for the
// float64-accurate potential apply on GB300, whose float32 pipes are ~58x
// faster than its float64 ones (measured: 70.2 vs 1.20 TFLOP/s), so the
// float64-accurate FFT runs on the float32 units at a fraction of the cost.
//
// The algorithms are the classical error-free transformations: Knuth's
// TwoSum, Dekker's Fast2Sum (QuickTwoSum) and the fused-multiply-add
// TwoProd, combined as in the double-double arithmetic of Hida, Li and
// Bailey ("Algorithms for quad-double precision floating point
// arithmetic", 2001): the "sloppy" addition (one TwoSum of the high parts,
// the low parts added in plain arithmetic) and the FMA-based
// multiplication. The sloppy addition's error is a small multiple of
// 2^-47 (|a| + |b|) rather than of |a + b|; that is the form of bound an
// FFT's error analysis uses (errors relative to the norm of the data), and
// the potential apply built on it matches the oracle to 1e-12.
#pragma once

#include "common.cuh"

namespace bae {

struct __align__(8) dsf {
    float hi, lo;
    __host__ __device__ dsf() = default;
    __host__ __device__ constexpr dsf(float h, float l) : hi(h), lo(l) {}
    // nearest double-float to a double (exact for up to 48 significant bits)
    __host__ __device__ explicit dsf(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dsf fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return dsf(s, e);
}

__device__ __forceinline__ dsf two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dsf(s, e);
}

__device__ __forceinline__ dsf operator+(dsf a, dsf b) {
    dsf s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dsf operator-(dsf a) { return dsf(-a.hi, -a.lo); }
__device__ __forceinline__ dsf operator-(dsf a, dsf b) { return a + (-b); }

__device__ __forceinline__ dsf operator*(dsf a, dsf b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

// complex double-float
struct __align__(16) dsc {
    dsf x, y;
};

template <> struct Cplx<dsf> { using type = dsc; };

// a b + c d with one TwoSum: TwoProd (FMA) of both high products, the cross
// terms with the low parts added to their errors, a.lo b.lo and c.lo d.lo
// dropped as in the product above (19 float operations where two products
// and a sum take 25)
__device__ __forceinline__ dsf dot2(dsf a, dsf b, dsf c, dsf d) {
    const float p = __fmul_rn(a.hi, b.hi), q = __fmul_rn(c.hi, d.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float f = __fmaf_rn(c.hi, d.hi, -q);
    f = __fmaf_rn(c.hi, d.lo, f);
    f = __fmaf_rn(c.lo, d.hi, f);
    const dsf s = two_sum(p, q);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, f)));
}

// sum without the closing Fast2Sum: hi + lo is the same sloppy sum, lo is
// not brought below half an ulp of hi (it grows by about that much per sum
// until the next product renormalises). Only the complex sums of the
// transforms use it.
__device__ __forceinline__ dsf add_nr(dsf a, dsf b) {
    const dsf s = two_sum(a.hi, b.hi);
    return dsf(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

// complex operations of the transforms (found by argument-dependent lookup
// ahead of the generic templates)
__device__ __forceinline__ dsc cadd(dsc a, dsc b) { return dsc{add_nr(a.x, b.x), add_nr(a.y, b.y)}; }
__device__ __forceinline__ dsc csub(dsc a, dsc b) { return dsc{add_nr(a.x, -b.x), add_nr(a.y, -b.y)}; }
__device__ __forceinline__ dsc cmul(dsc a, dsc b) { return dsc{dot2(a.x, b.x, -a.y, b.y), dot2(a.x, b.y, a.y, b.x)}; }
__device__ __forceinline__ dsc cmulc(dsc a, dsc b) { return dsc{dot2(a.x, b.x, a.y, b.y), dot2(a.y, b.x, -a.x, b.y)}; }
__device__ __forceinline__ dsc crot(dsc x, dsf c, dsf s) { return dsc{dot2(x.x, c, -x.y, s), dot2(x.x, s, x.y, c)}; }

template <>
__device__ __forceinline__ dsc ldg_c<dsc>(const dsc* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    dsc r;
    r.x = dsf(v.x, v.y);
    r.y = dsf(v.z, v.w);
    return r;
}

// element type written by the last convolution pass
template <> struct OutOf<dsf> { using type = double; };
__device__ __forceinline__ double to_out(dsf v) { return (double)v.hi + (double)v.lo; }

}  // namespace bae
