// Sums of squares of FP64 values without the FP64 pipe.
//
// On this GPU the FP64 pipe completes two FMAs per clock per SM against 128
// FP32 FMAs, and the large-grid FP64 Leja iteration is bound by it: 13 FP64
// FMA-class instructions per cell, two of them the squares of the stopping
// rule's norms (Section 2).  SqSum forms those sums on the integer and FP32
// pipes instead, to about the accuracy of the FP64 sums they replace:
//
//  * x = 2^(e - 1023) (h + l), with h in [1, 2) the leading 24 bits of the
//    significand and l the next 23, both exact FP32 values cut from the bit
//    pattern by integer operations (the last 6 significand bits are dropped:
//    relative error below 2^-46);
//  * (h + l)^2 = s1 + t, s1 = h h rounded and t = (h h - s1) + 2 h l from two
//    FMAs (the product h h is exact in the pair; l^2 < 2^-46 is dropped);
//  * the terms are summed as an unevaluated FP32 pair (TwoSum, then a fast
//    renormalisation) scaled by 2^(E - 2046), E the largest 2e seen so far:
//    a larger exponent rescales the pair by an exact power of two, so the
//    pair neither over- nor underflows whatever the magnitude of x; the FP64
//    value of the sum overflows where an FP64 sum would;
//  * zeros and subnormals add nothing (their squares vanish in FP64 as well);
//    a NaN or an infinity makes the sum non-finite (NaN), as it does in FP64.
//
// Relative error of a sum: below about 2^-44, the order of a sequential FP64
// sum of a few hundred terms, far inside the 1e-9 the stopping rule needs.
#pragma once

namespace ad {
namespace {

// 2^k as an FP32 value for k <= 0 (0 below the normal range).
__device__ __forceinline__ float sq_pow2(int k) {
  return k < -126 ? 0.0f : __int_as_float((127 + k) << 23);
}

struct SqSum {
  float hi = 0.0f, lo = 0.0f;   // the sum / 2^(ea - 2046), as hi + lo
  int ea = -(1 << 20);          // the largest 2e of the terms so far
  bool bad = false;             // a NaN or an infinity was added

  __device__ __forceinline__ void add(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int w1 = (unsigned int)(b >> 32), w0 = (unsigned int)b;
    const int e = (int)((w1 >> 20) & 0x7ffu);
    bad |= e == 0x7ff;
    const bool use = e != 0 && e != 0x7ff;
    // h: significand bits 51..29 under an exponent of 0; l: bits 28..6 times
    // 2^-46, from the exact FP32 value 2^23 + r (the FMA result is exact)
    const float h = __int_as_float(0x3f800000u | ((w1 & 0xfffffu) << 3) | (w0 >> 29));
    const float l = fmaf(__int_as_float(0x4b000000u | ((w0 >> 6) & 0x7fffffu)), 0x1p-46f,
                         -0x1p-23f);
    const float s1 = h * h;
    const float t = fmaf(h + h, l, fmaf(h, h, -s1));
    const int E = use ? 2 * e : ea;
    const int en = ea > E ? ea : E;
    const float fa = sq_pow2(ea - en);
    const float ft = use ? sq_pow2(E - en) : 0.0f;
    ea = en;
    const float a1 = hi * fa, a2 = lo * fa, b1 = s1 * ft, b2 = t * ft;
    const float S = a1 + b1;                       // TwoSum(a1, b1)
    const float bv = S - a1;
    const float err = (a1 - (S - bv)) + (b1 - bv);
    const float L = (a2 + b2) + err;
    hi = S + L;                                    // renormalise (|S| >= |L|)
    lo = L - (hi - S);
  }

  // The sum in FP64 (a handful of FP64 operations, once per thread).
  __device__ __forceinline__ double value() const {
    if (bad) return __longlong_as_double(0x7ff8000000000000LL);
    if (hi == 0.0f && lo == 0.0f) return 0.0;
    return ldexp((double)hi + (double)lo, ea - 2046);
  }
};

}  // namespace
}  // namespace ad
