// Complex arithmetic of the three storage precisions of the device path.
//
//   double : complex128, double2
//   float  : complex64,  float2
//   DF     : complex "double-float", float4 = (re.hi, re.lo, im.hi, im.lo):
//            every real is an unevaluated sum hi + lo of two FP32 numbers
//            (Dekker, "A floating-point technique for extending the available
//            precision", Numer. Math. 18 (1971); Knuth TAOCP vol. 2, 4.2.2),
//            about 48 significand bits computed on the FP32 pipe.
//
// The error-free transforms below rely on IEEE FP32 round-to-nearest and on
// the compiler not reassociating additions (nvcc does not without fast-math).
#pragma once

#include <cuda_runtime.h>

namespace ndgf {

struct DF {};

template <typename T> struct C2;
template <> struct C2<double> { using t = double2; };
template <> struct C2<float> { using t = float2; };
template <> struct C2<DF> { using t = float4; };
template <typename T> using cx = typename C2<T>::t;

template <typename T> struct Ops;

template <> struct Ops<double> {
  using C = double2;
  using R = double;  // magnitude type used for pivot comparisons
  struct Acc { double x, y; };
  static __device__ __forceinline__ C zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ C from_d2(double2 v) { return v; }
  static __device__ __forceinline__ double2 to_d2(C v) { return v; }
  static __device__ __forceinline__ C add(C a, C b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ C sub(C a, C b) { return make_double2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ C neg(C a) { return make_double2(-a.x, -a.y); }
  static __device__ __forceinline__ C conj(C a) { return make_double2(a.x, -a.y); }
  static __device__ __forceinline__ C mul(C a, C b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
  static __device__ __forceinline__ C scale(C a, double s) { return make_double2(s * a.x, s * a.y); }
  static __device__ __forceinline__ R mag2(C a) { return a.x * a.x + a.y * a.y; }
  static __device__ __forceinline__ C recip(C a) {
    const double s = fmax(fabs(a.x), fabs(a.y));
    const double ar = a.x / s, ai = a.y / s, d = (ar * ar + ai * ai) * s;
    return make_double2(ar / d, -ai / d);
  }
  static __device__ __forceinline__ Acc acc_zero() { return Acc{0.0, 0.0}; }
  static __device__ __forceinline__ void acc_fma(Acc& c, C a, C b) {
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(a.y, b.x, c.y);
  }
  static __device__ __forceinline__ C acc_get(const Acc& c) { return make_double2(c.x, c.y); }
  // a -= c r, the update of Gauss-Jordan elimination (gj_invert2)
  static __device__ __forceinline__ C norm(C a) { return a; }
  static __device__ __forceinline__ void sub_mul(C& a, C c, C r) {
    a.x = fma(-c.x, r.x, a.x);
    a.x = fma(c.y, r.y, a.x);
    a.y = fma(-c.x, r.y, a.y);
    a.y = fma(-c.y, r.x, a.y);
  }
  // 3-multiplication complex products (see Ops<DF>::Acc3)
  using S = double;
  struct Acc3 { double p1, p2, p3; };
  static __device__ __forceinline__ S sum(C a) { return a.x + a.y; }
  static __device__ __forceinline__ Acc3 acc3_zero() { return Acc3{0.0, 0.0, 0.0}; }
  static __device__ __forceinline__ void acc3_fma(Acc3& c, C a, S as, C b, S bs) {
    c.p1 = fma(a.x, b.x, c.p1);
    c.p2 = fma(a.y, b.y, c.p2);
    c.p3 = fma(as, bs, c.p3);
  }
  static __device__ __forceinline__ C acc3_get(const Acc3& c) { return make_double2(c.p1 - c.p2, (c.p3 - c.p1) - c.p2); }
};

template <> struct Ops<float> {
  using C = float2;
  using R = float;
  struct Acc { float x, y; };
  static __device__ __forceinline__ C zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ C from_d2(double2 v) { return make_float2(float(v.x), float(v.y)); }
  static __device__ __forceinline__ double2 to_d2(C v) { return make_double2(double(v.x), double(v.y)); }
  static __device__ __forceinline__ C add(C a, C b) { return make_float2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ C sub(C a, C b) { return make_float2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ C neg(C a) { return make_float2(-a.x, -a.y); }
  static __device__ __forceinline__ C conj(C a) { return make_float2(a.x, -a.y); }
  static __device__ __forceinline__ C mul(C a, C b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
  static __device__ __forceinline__ C scale(C a, double s) { return make_float2(float(s) * a.x, float(s) * a.y); }
  static __device__ __forceinline__ R mag2(C a) { return a.x * a.x + a.y * a.y; }
  static __device__ __forceinline__ C recip(C a) {
    const float s = fmaxf(fabsf(a.x), fabsf(a.y));
    const float ar = a.x / s, ai = a.y / s, d = (ar * ar + ai * ai) * s;
    return make_float2(ar / d, -ai / d);
  }
  static __device__ __forceinline__ Acc acc_zero() { return Acc{0.f, 0.f}; }
  static __device__ __forceinline__ void acc_fma(Acc& c, C a, C b) {
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(a.y, b.x, c.y);
  }
  static __device__ __forceinline__ C acc_get(const Acc& c) { return make_float2(c.x, c.y); }
  static __device__ __forceinline__ C norm(C a) { return a; }
  static __device__ __forceinline__ void sub_mul(C& a, C c, C r) {
    a.x = fmaf(-c.x, r.x, a.x);
    a.x = fmaf(c.y, r.y, a.x);
    a.y = fmaf(-c.x, r.y, a.y);
    a.y = fmaf(-c.y, r.x, a.y);
  }
  using S = float;
  struct Acc3 { float p1, p2, p3; };
  static __device__ __forceinline__ S sum(C a) { return a.x + a.y; }
  static __device__ __forceinline__ Acc3 acc3_zero() { return Acc3{0.f, 0.f, 0.f}; }
  static __device__ __forceinline__ void acc3_fma(Acc3& c, C a, S as, C b, S bs) {
    c.p1 = fmaf(a.x, b.x, c.p1);
    c.p2 = fmaf(a.y, b.y, c.p2);
    c.p3 = fmaf(as, bs, c.p3);
  }
  static __device__ __forceinline__ C acc3_get(const Acc3& c) { return make_float2(c.p1 - c.p2, (c.p3 - c.p1) - c.p2); }
};

// ---- double-float reals ----------------------------------------------------
struct f2 {
  float h, l;
};

// s + e = a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// s + e = a + b exactly when |a| >= |b| (Dekker's fast two-sum).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
// a + b with both the high and the low parts added by two-sum, so that the
// result stays accurate under cancellation of the high parts.
__device__ __forceinline__ f2 dd_add(f2 a, f2 b) {
  float s1, s2, t1, t2;
  two_sum(a.h, b.h, s1, s2);
  two_sum(a.l, b.l, t1, t2);
  s2 += t1;
  fast_two_sum(s1, s2, s1, s2);
  s2 += t2;
  f2 r;
  fast_two_sum(s1, s2, r.h, r.l);
  return r;
}
__device__ __forceinline__ f2 dd_neg(f2 a) { return f2{-a.h, -a.l}; }
__device__ __forceinline__ f2 dd_sub(f2 a, f2 b) { return dd_add(a, dd_neg(b)); }
// product: p + e = a.h * b.h exactly (FMA), plus the cross terms
__device__ __forceinline__ f2 dd_mul(f2 a, f2 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  f2 r;
  fast_two_sum(p, e, r.h, r.l);
  return r;
}
// 1/a by one Newton step from the FP32 reciprocal: y = y0 + y0 (1 - a y0)
__device__ __forceinline__ f2 dd_recip(f2 a) {
  const float y0 = 1.0f / a.h;
  const f2 r = dd_sub(f2{1.0f, 0.0f}, dd_mul(a, f2{y0, 0.0f}));
  return dd_add(f2{y0, 0.0f}, dd_mul(f2{y0, 0.0f}, r));
}
__device__ __forceinline__ f2 dd_from(double v) {
  const float h = __double2float_rn(v);
  return f2{h, __double2float_rn(v - double(h))};
}
__device__ __forceinline__ double dd_to(f2 a) { return double(a.h) + double(a.l); }

template <> struct Ops<DF> {
  using C = float4;  // (re.h, re.l, im.h, im.l)
  using R = float;
  // accumulator: hi parts summed with two-sum, low-order terms collected apart
  struct Acc { float rh, rl, ih, il; };
  static __device__ __forceinline__ f2 re(C a) { return f2{a.x, a.y}; }
  static __device__ __forceinline__ f2 im(C a) { return f2{a.z, a.w}; }
  static __device__ __forceinline__ C mk(f2 r, f2 i) { return make_float4(r.h, r.l, i.h, i.l); }
  static __device__ __forceinline__ C zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ C from_d2(double2 v) { return mk(dd_from(v.x), dd_from(v.y)); }
  static __device__ __forceinline__ double2 to_d2(C v) { return make_double2(dd_to(re(v)), dd_to(im(v))); }
  static __device__ __forceinline__ C add(C a, C b) { return mk(dd_add(re(a), re(b)), dd_add(im(a), im(b))); }
  static __device__ __forceinline__ C sub(C a, C b) { return mk(dd_sub(re(a), re(b)), dd_sub(im(a), im(b))); }
  static __device__ __forceinline__ C neg(C a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
  static __device__ __forceinline__ C conj(C a) { return make_float4(a.x, a.y, -a.z, -a.w); }
  static __device__ __forceinline__ C mul(C a, C b) {
    return mk(dd_sub(dd_mul(re(a), re(b)), dd_mul(im(a), im(b))), dd_add(dd_mul(re(a), im(b)), dd_mul(im(a), re(b))));
  }
  static __device__ __forceinline__ C scale(C a, double s) {
    const f2 f = dd_from(s);
    return mk(dd_mul(re(a), f), dd_mul(im(a), f));
  }
  static __device__ __forceinline__ R mag2(C a) { return a.x * a.x + a.z * a.z; }
  static __device__ __forceinline__ C recip(C a) {
    const f2 ar = re(a), ai = im(a);
    const f2 inv = dd_recip(dd_add(dd_mul(ar, ar), dd_mul(ai, ai)));
    return mk(dd_mul(ar, inv), dd_neg(dd_mul(ai, inv)));
  }
  static __device__ __forceinline__ Acc acc_zero() { return Acc{0.f, 0.f, 0.f, 0.f}; }
  // h + l += sign * (x * y), x, y double-float
  static __device__ __forceinline__ void acc_term(float& h, float& l, f2 x, f2 y, float sign) {
    const float p = x.h * y.h;
    float e = fmaf(x.h, y.h, -p);
    e = fmaf(x.h, y.l, e);
    e = fmaf(x.l, y.h, e);
    float s, t;
    two_sum(h, sign * p, s, t);
    h = s;
    l += t + sign * e;
  }
  static __device__ __forceinline__ void acc_fma(Acc& c, C a, C b) {
    acc_term(c.rh, c.rl, re(a), re(b), 1.f);
    acc_term(c.rh, c.rl, im(a), im(b), -1.f);
    acc_term(c.ih, c.il, re(a), im(b), 1.f);
    acc_term(c.ih, c.il, im(a), re(b), 1.f);
  }
  static __device__ __forceinline__ C acc_get(const Acc& c) {
    f2 r, i;
    two_sum(c.rh, c.rl, r.h, r.l);
    two_sum(c.ih, c.il, i.h, i.l);
    return mk(r, i);
  }
  // Elements updated by sub_mul are kept as unnormalised pairs (h, l), like
  // the accumulator above; norm() brings one back to a double-float before it
  // is used as a factor.
  static __device__ __forceinline__ C norm(C a) {
    f2 r, i;
    two_sum(a.x, a.y, r.h, r.l);
    two_sum(a.z, a.w, i.h, i.l);
    return mk(r, i);
  }
  static __device__ __forceinline__ void sub_mul(C& a, C c, C r) {  // a -= c r, c and r normalised
    acc_term(a.x, a.y, re(c), re(r), -1.f);
    acc_term(a.x, a.y, im(c), im(r), 1.f);
    acc_term(a.z, a.w, re(c), im(r), -1.f);
    acc_term(a.z, a.w, im(c), re(r), -1.f);
  }
  // 3-multiplication complex multiply-add (Gauss's trick; Higham, "Accuracy
  // and Stability of Numerical Algorithms", 2nd ed., Sec. 23.2.4):
  //   P1 += Re a Re b,  P2 += Im a Im b,  P3 += (Re a + Im a)(Re b + Im b),
  //   Re = P1 - P2,     Im = P3 - P1 - P2.
  // The sums Re + Im are formed once per staged element, so a multiply-add
  // costs three lazy double-float terms (36 FP32 operations) instead of four.
  // The error bound is normwise: |error| <~ eps (|Re a| + |Im a|)(|Re b| + |Im b|).
  using S = float2;  // double-float real (h, l)
  struct Acc3 { float h1, l1, h2, l2, h3, l3; };
  static __device__ __forceinline__ S sum(C a) {
    const f2 r = dd_add(re(a), im(a));
    return make_float2(r.h, r.l);
  }
  static __device__ __forceinline__ Acc3 acc3_zero() { return Acc3{0.f, 0.f, 0.f, 0.f, 0.f, 0.f}; }
  static __device__ __forceinline__ void acc3_fma(Acc3& c, C a, S as, C b, S bs) {
    acc_term(c.h1, c.l1, re(a), re(b), 1.f);
    acc_term(c.h2, c.l2, im(a), im(b), 1.f);
    acc_term(c.h3, c.l3, f2{as.x, as.y}, f2{bs.x, bs.y}, 1.f);
  }
  static __device__ __forceinline__ C acc3_get(const Acc3& c) {
    f2 p1, p2, p3;
    two_sum(c.h1, c.l1, p1.h, p1.l);
    two_sum(c.h2, c.l2, p2.h, p2.l);
    two_sum(c.h3, c.l3, p3.h, p3.l);
    return mk(dd_sub(p1, p2), dd_sub(dd_sub(p3, p1), p2));
  }
};

}  // namespace ndgf
