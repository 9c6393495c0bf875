// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi)/2, about 48 significant bits.  On GB300 the
// FP32 units issue ~58x the FP64 rate (34.8 TFMA/s vs 596 GFMA/s measured), so
// the FP64 plans run their FFTs and interpolation in this form.
//
// Error-free transforms (published methods, own code):
//   two_sum    Knuth, TAOCP vol. 2, Sec. 4.2.2: s + e = a + b exactly.
//   quick_two_sum  Dekker 1971 ("Fast2Sum"), valid for |a| >= |b|.
//   two_prod   a*b = p + e exactly, with e from one fused multiply-add.
// The add and multiply below are the usual "sloppy" double-float operations
// built from them (relative error a few units of 2^-48 barring cancellation
// of the high parts).  Intrinsics with explicit rounding keep the compiler
// from contracting the error terms into fused operations.
//
// Conversions between double and df64 use integer bit manipulation: on GB300
// the FP64<->FP32 conversion instructions run at ~280 G/s, against ~21 T/s
// for integer operations.  Magnitudes below ~1e-30 lose the low part (and
// below ~1e-38 flush to zero); values here are far from that range.
#pragma once

#include <cstdint>

namespace lpg {

struct dd {
  float hi, lo;
};

struct cdd {  // complex df64
  dd re, im;
};

__device__ __forceinline__ dd dd_make(float hi, float lo) { return dd{hi, lo}; }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  dd r;
  quick_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  dd r;
  quick_two_sum(p, e, r.hi, r.lo);
  return r;
}

// a * f for a float f
__device__ __forceinline__ dd dd_mul_f(dd a, float f) {
  const float p = __fmul_rn(a.hi, f);
  float e = __fmaf_rn(a.hi, f, -p);
  e = __fmaf_rn(a.lo, f, e);
  dd r;
  quick_two_sum(p, e, r.hi, r.lo);
  return r;
}

// exact scaling by a power of two
__device__ __forceinline__ dd dd_scale(dd a, float pow2) { return dd{a.hi * pow2, a.lo * pow2}; }

// a*b + c*d with one final renormalisation
__device__ __forceinline__ dd dd_dot2(dd a, dd b, dd c, dd d) {
  const float p1 = __fmul_rn(a.hi, b.hi);
  float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  e1 = __fmaf_rn(a.hi, b.lo, e1);
  e1 = __fmaf_rn(a.lo, b.hi, e1);
  const float p2 = __fmul_rn(c.hi, d.hi);
  float e2 = __fmaf_rn(c.hi, d.hi, -p2);
  e2 = __fmaf_rn(c.hi, d.lo, e2);
  e2 = __fmaf_rn(c.lo, d.hi, e2);
  float s, e;
  two_sum(p1, p2, s, e);
  e = __fadd_rn(e, __fadd_rn(e1, e2));
  dd r;
  quick_two_sum(s, e, r.hi, r.lo);
  return r;
}

// Running sum of products without renormalising every term: (s, c) with
// value s + c, c collecting the rounding errors.
struct dd_acc {
  float s, c;
};

__device__ __forceinline__ void acc_fma(dd_acc& a, dd w, dd g) {
  const float p = __fmul_rn(w.hi, g.hi);
  float e = __fmaf_rn(w.hi, g.hi, -p);
  e = __fmaf_rn(w.hi, g.lo, e);
  e = __fmaf_rn(w.lo, g.hi, e);
  float s, t;
  two_sum(a.s, p, s, t);
  a.s = s;
  a.c = __fadd_rn(a.c, __fadd_rn(t, e));
}

__device__ __forceinline__ dd acc_value(dd_acc a) {
  dd r;
  quick_two_sum(a.s, a.c, r.hi, r.lo);
  return r;
}

// acc * v + c with one renormalisation (Horner step)
__device__ __forceinline__ dd dd_horner(dd acc, dd v, float2 c) {
  const float p = __fmul_rn(acc.hi, v.hi);
  float e = __fmaf_rn(acc.hi, v.hi, -p);
  e = __fmaf_rn(acc.hi, v.lo, e);
  e = __fmaf_rn(acc.lo, v.hi, e);
  float s, t;
  two_sum(p, c.x, s, t);
  t = __fadd_rn(t, __fadd_rn(e, c.y));
  dd r;
  quick_two_sum(s, t, r.hi, r.lo);
  return r;
}

// The w stencil weights of one dimension from the kernel's per-offset
// polynomials (coefficient k of offset t at coef[k * stride + t], df64).
// The kernel is even, so offset w-1-t at v is offset t at -v: with
// P_t(v) = E_t(v^2) + v O_t(v^2), weights t and w-1-t are E_t +- v O_t, and
// only the first ceil(w/2) polynomials are evaluated, in v^2 (half the
// Horner steps of evaluating all w).  The first nf Horner steps of each
// chain, whose rounding the remaining steps damp by powers of v^2 <= 1/4,
// run in single precision on the coefficients' high parts (the plan chooses
// nf so that this adds at most 5% of the fit's error target).
template <int W>
__device__ __forceinline__ void dd_stencil_weights(const float2* coef, int stride, int nc, int nf, dd v, dd* w) {
  constexpr int WH = (W + 1) / 2;
  const dd v2 = dd_mul(v, v);
  const int ke = (nc - 1) & ~1, ko = (nc - 2) | 1;  // highest even / odd power present
  dd e[WH], o[WH];
  float ef[WH], of[WH];
#pragma unroll
  for (int t = 0; t < WH; ++t) {
    ef[t] = coef[ke * stride + t].x;
    of[t] = coef[ko * stride + t].x;
  }
  int k = ke - 2;
  for (int s = 0; s < nf && k >= 0; ++s, k -= 2) {
#pragma unroll
    for (int t = 0; t < WH; ++t) ef[t] = __fmaf_rn(ef[t], v2.hi, coef[k * stride + t].x);
  }
  int ko2 = ko - 2;
  for (int s = 0; s < nf && ko2 >= 1; ++s, ko2 -= 2) {
#pragma unroll
    for (int t = 0; t < WH; ++t) of[t] = __fmaf_rn(of[t], v2.hi, coef[ko2 * stride + t].x);
  }
#pragma unroll
  for (int t = 0; t < WH; ++t) {
    // no float steps: the leading coefficient keeps its low part
    e[t] = dd{ef[t], nf ? 0.f : coef[ke * stride + t].y};
    o[t] = dd{of[t], nf ? 0.f : coef[ko * stride + t].y};
  }
  for (; k >= 0; k -= 2) {
#pragma unroll
    for (int t = 0; t < WH; ++t) e[t] = dd_horner(e[t], v2, coef[k * stride + t]);
  }
  for (; ko2 >= 1; ko2 -= 2) {
#pragma unroll
    for (int t = 0; t < WH; ++t) o[t] = dd_horner(o[t], v2, coef[ko2 * stride + t]);
  }
#pragma unroll
  for (int t = 0; t < WH; ++t) {
    const dd vo = dd_mul(v, o[t]);
    w[t] = dd_add(e[t], vo);
    if (W - 1 - t != t) w[W - 1 - t] = dd_sub(e[t], vo);
  }
}

// ---- conversions (integer bit manipulation) ----

// float with sign bit s, unbiased exponent e and a significand m whose leading
// one is at bit 23 (0 if the exponent is below the normal range)
__device__ __forceinline__ float make_float(uint32_t s, int e, uint32_t m) {
  if (e < -126) return __uint_as_float(s);
  return __uint_as_float(s | ((uint32_t)(e + 127) << 23) | (m & 0x7fffffu));
}

// double -> df64: hi = the top 24 significand bits (truncated), lo = the next
// 24 bits of the remainder (truncated); hi + lo agrees with x to ~2^-48.
__device__ __forceinline__ dd dd_from_double(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t s = (uint32_t)(b >> 32) & 0x80000000u;
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) return dd{__uint_as_float(s), 0.f};     // zero (denormals flushed)
  if (ex == 0x7ff) return dd{(float)x, 0.f};           // inf / nan
  const int e = ex - 1023;
  if (e > 127) return dd{(float)x, 0.f};               // out of float range
  const uint64_t m = (b & 0xfffffffffffffull) | 0x10000000000000ull;  // 53-bit significand
  const uint32_t mh = (uint32_t)(m >> 29);              // 24 bits, leading one at bit 23
  const uint32_t r = (uint32_t)(m & 0x1fffffffu);       // remaining 29 bits, weight 2^(e-52)
  dd out;
  out.hi = make_float(s, e, mh);
  if (r == 0) {
    out.lo = __uint_as_float(s);
  } else {
    const int lz = __clz(r);                            // >= 3
    const int top = 31 - lz;                            // bit index of the leading one
    const uint32_t rn = top >= 23 ? (r >> (top - 23)) : (r << (23 - top));
    out.lo = make_float(s, e - 52 + top, rn);
  }
  return out;
}

// df64 -> double: hi widened exactly through its bits, plus lo (one FP64 add)
__device__ __forceinline__ double float_to_double_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t s = u & 0x80000000u;
  const uint32_t ef = (u >> 23) & 0xff;
  if (ef == 0) return __longlong_as_double((int64_t)((uint64_t)s << 32));  // zero (denormals flushed)
  if (ef == 0xff) return (double)f;
  const uint64_t bits = ((uint64_t)s << 32) | ((uint64_t)(ef - 127 + 1023) << 52) |
                        ((uint64_t)(u & 0x7fffffu) << 29);
  return __longlong_as_double((int64_t)bits);
}

__device__ __forceinline__ double dd_to_double(dd a) {
  return float_to_double_bits(a.hi) + float_to_double_bits(a.lo);
}

// ---- complex ----

__device__ __forceinline__ cdd cdd_add(cdd a, cdd b) { return cdd{dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
__device__ __forceinline__ cdd cdd_sub(cdd a, cdd b) { return cdd{dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; }
__device__ __forceinline__ cdd cdd_conj(cdd a) { return cdd{a.re, dd_neg(a.im)}; }
// a * (-i) and a * (+i)
__device__ __forceinline__ cdd cdd_mul_mi(cdd a) { return cdd{a.im, dd_neg(a.re)}; }
__device__ __forceinline__ cdd cdd_mul_pi(cdd a) { return cdd{dd_neg(a.im), a.re}; }

__device__ __forceinline__ cdd cdd_mul(cdd a, cdd b) {
  return cdd{dd_dot2(a.re, b.re, dd_neg(a.im), b.im), dd_dot2(a.re, b.im, a.im, b.re)};
}

// a * conj(b)
__device__ __forceinline__ cdd cdd_mul_conj(cdd a, cdd b) {
  return cdd{dd_dot2(a.re, b.re, a.im, b.im), dd_dot2(a.im, b.re, dd_neg(a.re), b.im)};
}

__device__ __forceinline__ cdd cdd_scale_dd(cdd a, dd m) { return cdd{dd_mul(a.re, m), dd_mul(a.im, m)}; }

__device__ __forceinline__ cdd cdd_load(const float4* p) {
  const float4 v = *p;
  return cdd{dd{v.x, v.y}, dd{v.z, v.w}};
}

__device__ __forceinline__ void cdd_store(float4* p, cdd a) { *p = make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }

}  // namespace lpg
