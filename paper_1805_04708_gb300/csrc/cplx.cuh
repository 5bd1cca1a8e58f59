// Complex helpers and the 2x2 update functors shared by the dense-encoding
// kernels (per-gate sweeps and shared-memory tile passes).
#pragma once
#ifndef QS_JIT
#include <cuda_runtime.h>
#endif

// ---------------------------------------------------------------------------
// Double-float ("float-float") numbers: a value hi + lo held as two FP32
// numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  The sum and the
// product follow the error-free transformations of Dekker (1971) and Knuth
// (TAOCP vol. 2): TwoSum gives a + b = s + e exactly, TwoProd (one FMA)
// a * b = p + e exactly, and a renormalisation keeps lo small.  Written with
// the _rn intrinsics so that no multiply-add contraction changes them.  The
// complex128 tile passes compute on these, on the FP32 pipes, instead of the
// FP64 units (1/64 of the FP32 rate on this GPU).
// ---------------------------------------------------------------------------
struct DF {
  float hi, lo;
  DF() = default;
  __host__ __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
  // also built on the host (gate coefficients of the per-gate kernels)
  __host__ __device__ __forceinline__ DF(double x) {
#ifdef __CUDA_ARCH__
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
#else
    hi = (float)x;
    lo = (float)(x - (double)hi);
#endif
  }
  __host__ __device__ __forceinline__ DF(int i) : hi((float)i), lo(0.f) {}
};
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ DF df_quick(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return DF(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return DF(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
// The sum: TwoSum of the high parts (exact), the low parts added in FP32, one
// renormalisation.  Its error is within a few units of 2^-44 of the larger
// operand (the low parts' rounding), far inside what the complex128 paths
// need (1e-12 absolute on amplitudes of magnitude <= 1), at about half the
// instructions of a second TwoSum on the low parts.
__device__ __forceinline__ DF operator+(DF a, DF b) {
  const DF s = df_two_sum(a.hi, b.hi);
  return df_quick(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
__device__ __forceinline__ DF operator*(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick(p, e);
}
// a * b + c with one renormalisation: the product's high part and its
// error-free remainder (TwoProd), the exact sum of the high parts (TwoSum),
// the low terms added in FP32
__device__ __forceinline__ DF fma(DF a, DF b, DF c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const DF s = df_two_sum(p, c.hi);
  return df_quick(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}
__device__ __forceinline__ bool operator!=(DF a, DF b) { return a.hi != b.hi || a.lo != b.lo; }

template <typename R> struct __align__(2 * sizeof(R)) Cx { R x, y; };

template <typename R>
__device__ __forceinline__ Cx<R> cx(R x, R y) { Cx<R> c; c.x = x; c.y = y; return c; }

// a * f, exact for the unit factors (code 0: 1, 1: i, 2: -1, 3: -i).
template <typename R>
__device__ __forceinline__ Cx<R> cmul_code(Cx<R> a, Cx<R> f, int code) {
  switch (code) {
    case 0: return a;
    case 1: return cx<R>(-a.y, a.x);
    case 2: return cx<R>(-a.x, -a.y);
    case 3: return cx<R>(a.y, -a.x);
    default: return cx<R>(fma(a.x, f.x, -(a.y * f.y)), fma(a.x, f.y, a.y * f.x));
  }
}

// u0 * a0 + u1 * a1
template <typename R>
__device__ __forceinline__ Cx<R> cmac2(Cx<R> u0, Cx<R> a0, Cx<R> u1, Cx<R> a1) {
  R re = u0.x * a0.x;
  re = fma(-u0.y, a0.y, re);
  re = fma(u1.x, a1.x, re);
  re = fma(-u1.y, a1.y, re);
  R im = u0.x * a0.y;
  im = fma(u0.y, a0.x, im);
  im = fma(u1.x, a1.y, im);
  im = fma(u1.y, a1.x, im);
  return cx<R>(re, im);
}

// complex128 amplitudes in memory are FP64 pairs; R = double computes on the
// FP64 units, R = DF on FP32 pairs
template <typename R> __device__ __forceinline__ Cx<R> from_mem(double2 x) { return cx<R>(R(x.x), R(x.y)); }
template <typename R> __device__ __forceinline__ double2 to_mem(Cx<R> a) {
  return make_double2(to_double(a.x), to_double(a.y));
}

#ifndef QS_JIT
// FP64 value -> (hi, lo) with integer operations, the same pair as
// hi = RN_float(x), lo = RN_float(x - hi) but without the FP64 units: hi is x's
// significand rounded to 24 bits (to nearest, ties to even); x - hi is the
// exact integer remainder d (|d| <= 2^28) times 2^(E - 1075), rounded to float
// by the integer conversion and scaled by two exact powers of two.  Values
// below 2^-126 in magnitude (no normal float hi) become 0, an absolute error
// under 1.2e-38; values of 2^76 and more take the FP64 conversion.
__device__ __forceinline__ DF df_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E < 897) return DF(0.f, 0.f);
  if (E > 1098) return DF(x);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  unsigned long long q = m >> 29;
  const unsigned long long r = m & 0x1FFFFFFFull;
  q += (r > 0x10000000ull || (r == 0x10000000ull && (q & 1ull))) ? 1ull : 0ull;
  const int d = (int)((long long)m - (long long)(q << 29));
  unsigned int eh = (unsigned int)(E - 896), qh = (unsigned int)q;
  if (qh == (1u << 24)) { qh >>= 1; ++eh; }
  const unsigned int sgn = (unsigned int)(b >> 32) & 0x80000000u;
  const float hi = __uint_as_float(sgn | (eh << 23) | (qh & 0x7FFFFFu));
  float lo = __fmul_rn(__int2float_rn(d), __uint_as_float((unsigned int)(E - 896) << 23));   // x 2^(E-1023)
  lo = __fmul_rn(lo, __uint_as_float(75u << 23));                                           // x 2^-52
  return DF(hi, sgn ? -lo : lo);
}
// float -> FP64 from the bits (exact for normal floats; subnormals, which the
// split above never produces for hi, give 0)
__device__ __forceinline__ double df_f2d(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xFFu;
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long body = ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)(e == 0 ? s : (s | body)));
}
template <> __device__ __forceinline__ Cx<DF> from_mem<DF>(double2 x) { return cx<DF>(df_split(x.x), df_split(x.y)); }
template <> __device__ __forceinline__ double2 to_mem<DF>(Cx<DF> a) {
  return make_double2(__dadd_rn(df_f2d(a.x.hi), df_f2d(a.x.lo)), __dadd_rn(df_f2d(a.y.hi), df_f2d(a.y.lo)));
}
#endif

// Storage <-> Cx conversions.
__device__ __forceinline__ Cx<double> ld(const double2& v) { return cx<double>(v.x, v.y); }
__device__ __forceinline__ Cx<float> ld(const float2& v) { return cx<float>(v.x, v.y); }
__device__ __forceinline__ void st(double2& v, Cx<double> a) { v.x = a.x; v.y = a.y; }
__device__ __forceinline__ void st(float2& v, Cx<float> a) { v.x = a.x; v.y = a.y; }

// ---------------------------------------------------------------------------
// 2x2 update functors.  pair(a0, a1) updates the two amplitudes of one pair
// (Eq. (NUM2) with the gate's matrix); one(a) multiplies one amplitude.
// ---------------------------------------------------------------------------
template <typename R> struct OpDense {
  Cx<R> u00, u01, u10, u11;
  __device__ __forceinline__ void pair(Cx<R>& a0, Cx<R>& a1) const {
    Cx<R> b0 = cmac2(u00, a0, u01, a1);
    Cx<R> b1 = cmac2(u10, a0, u11, a1);
    a0 = b0; a1 = b1;
  }
};
template <typename R> struct OpHad {
  R s;
  __device__ __forceinline__ void pair(Cx<R>& a0, Cx<R>& a1) const {
    Cx<R> b0 = cx<R>((a0.x + a1.x) * s, (a0.y + a1.y) * s);
    Cx<R> b1 = cx<R>((a0.x - a1.x) * s, (a0.y - a1.y) * s);
    a0 = b0; a1 = b1;
  }
};
template <typename R> struct OpDiag {
  Cx<R> d0, d1; int c0, c1;
  __device__ __forceinline__ void pair(Cx<R>& a0, Cx<R>& a1) const {
    a0 = cmul_code(a0, d0, c0);
    a1 = cmul_code(a1, d1, c1);
  }
};
template <typename R> struct OpAnti {
  Cx<R> f01, f10; int c0, c1;
  __device__ __forceinline__ void pair(Cx<R>& a0, Cx<R>& a1) const {
    Cx<R> b0 = cmul_code(a1, f01, c0);
    Cx<R> b1 = cmul_code(a0, f10, c1);
    a0 = b0; a1 = b1;
  }
};
// Real 2x2 (H, X, CNOT, TOFFOLI, +-Y, ...) on complex64 pairs with packed
// FP32x2 arithmetic on (re, im): two packed instructions per output.
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
#define QS_HAVE_F32X2 1
#endif
struct OpRealF {
  float2 u00, u01, u10, u11;   // (u, u) splats
  __device__ __forceinline__ void pair(Cx<float>& a0, Cx<float>& a1) const {
    const float2 A0 = make_float2(a0.x, a0.y), A1 = make_float2(a1.x, a1.y);
#ifdef QS_HAVE_F32X2
    const float2 B0 = __ffma2_rn(u00, A0, __fmul2_rn(u01, A1));
    const float2 B1 = __ffma2_rn(u10, A0, __fmul2_rn(u11, A1));
#else
    const float2 B0 = make_float2(fmaf(u00.x, A0.x, u01.x * A1.x), fmaf(u00.x, A0.y, u01.x * A1.y));
    const float2 B1 = make_float2(fmaf(u10.x, A0.x, u11.x * A1.x), fmaf(u10.x, A0.y, u11.x * A1.y));
#endif
    a0 = cx<float>(B0.x, B0.y);
    a1 = cx<float>(B1.x, B1.y);
  }
};
// Unscaled Hadamard butterfly (a0 + a1, a0 - a1).
template <typename R> struct OpBfly {
  __device__ __forceinline__ void pair(Cx<R>& a0, Cx<R>& a1) const {
    const Cx<R> b0 = cx<R>(a0.x + a1.x, a0.y + a1.y), b1 = cx<R>(a0.x - a1.x, a0.y - a1.y);
    a0 = b0;
    a1 = b1;
  }
};
// Unscaled Hadamard butterfly on complex64 pairs: one packed instruction per
// output (the pass applies the dropped scale factors elsewhere, once).
struct OpBflyF {
  __device__ __forceinline__ void pair(Cx<float>& a0, Cx<float>& a1) const {
    const float2 A0 = make_float2(a0.x, a0.y), A1 = make_float2(a1.x, a1.y);
#ifdef QS_HAVE_F32X2
    const float2 B0 = __fadd2_rn(A0, A1);
    const float2 B1 = __ffma2_rn(make_float2(-1.f, -1.f), A1, A0);
#else
    const float2 B0 = make_float2(A0.x + A1.x, A0.y + A1.y);
    const float2 B1 = make_float2(A0.x - A1.x, A0.y - A1.y);
#endif
    a0 = cx<float>(B0.x, B0.y);
    a1 = cx<float>(B1.x, B1.y);
  }
};
// The butterfly with the two amplitudes' roles possibly exchanged (a
// relabelled index bit: a0 then holds the pair's upper element): s0 = (1, 1),
// s1 = (-1, -1) give (a0 + a1, a0 - a1); s0 = (-1, -1), s1 = (1, 1) give
// (a1 - a0, a1 + a0).
struct OpBflyS {
  float2 s0, s1;
  __device__ __forceinline__ void pair(Cx<float>& a0, Cx<float>& a1) const {
    const float2 A0 = make_float2(a0.x, a0.y), A1 = make_float2(a1.x, a1.y);
#ifdef QS_HAVE_F32X2
    const float2 B0 = __ffma2_rn(s0, A0, A1);
    const float2 B1 = __ffma2_rn(s1, A1, A0);
#else
    const float2 B0 = make_float2(fmaf(s0.x, A0.x, A1.x), fmaf(s0.x, A0.y, A1.y));
    const float2 B1 = make_float2(fmaf(s1.x, A1.x, A0.x), fmaf(s1.x, A1.y, A0.y));
#endif
    a0 = cx<float>(B0.x, B0.y);
    a1 = cx<float>(B1.x, B1.y);
  }
};
// The unscaled butterfly computed in place, for a loop that keeps its values
// in fixed registers (no temporaries, hence no moves): a0 <- a0 + a1, then
// a1 <- a0_new - 2 a1 = a0 - a1 (one more rounding than the direct form).
// With SW the pair's roles are exchanged (a relabelled index bit).
template <bool SW> struct OpBflyIP {
  __device__ __forceinline__ void pair(Cx<float>& a0, Cx<float>& a1) const {
    Cx<float>& p = SW ? a1 : a0;
    Cx<float>& q = SW ? a0 : a1;
#ifdef QS_HAVE_F32X2
    const float2 P = __fadd2_rn(make_float2(p.x, p.y), make_float2(q.x, q.y));
    p = cx<float>(P.x, P.y);
    const float2 Q = __ffma2_rn(make_float2(-2.f, -2.f), make_float2(q.x, q.y), P);
    q = cx<float>(Q.x, Q.y);
#else
    p = cx<float>(p.x + q.x, p.y + q.y);
    q = cx<float>(fmaf(-2.f, q.x, p.x), fmaf(-2.f, q.y, p.y));
#endif
  }
};
template <typename R> struct OpMul {
  Cx<R> f; int c;
  __device__ __forceinline__ void one(Cx<R>& a) const { a = cmul_code(a, f, c); }
};
