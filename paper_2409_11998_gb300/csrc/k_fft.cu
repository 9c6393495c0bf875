// FFT chain of the history part (Sec. 3, Steps 2-4: forward transform of the
// spread grids, diagonal multiplier, inverse transform): in double-float
// arithmetic for FP64 plans (FP64 cuFFT is bound by GB300's FP64 units) and
// in single precision for FP32 plans, with the same structure.
//
//   rows_fwd  real grid rows [row_lo, row_hi) (FP64, as spread) -> kept modes
//             0..K of each row's half spectrum, df64 complex, [g][Kp]
//   cols      per kept column m_x: forward transform along y, the
//             deconvolved multiplier (V, S: M F; D: M (-i)(k1 F1 + k2 F2)),
//             inverse transform along y -- the column never leaves shared
//             memory between the two transforms
//   rows_inv  rows [row_lo, row_hi) of the half spectrum -> real grid rows,
//             written in place over the grid (FP64 plans: as df64 (hi, lo)
//             pairs over the FP64 values)
//
// Transforms are unnormalised with the signs of the forward (e^{-i}) and
// inverse (e^{+i}) DFT, as the multiplier tables expect.  Each 1D transform
// runs in shared memory as a mixed-radix (4, 2, 3) Stockham autosort FFT
// (Govindaraju et al., "High performance discrete Fourier transforms on
// graphics processors", SC 2008): stage s with radix R combines R interleaved
// transforms of length Ns into transforms of length Ns R, reading with stride
// N/R and writing in natural order.  A real row of length g = 2N is
// transformed as the complex sequence x_2n + i x_2n+1 of length N followed by
// the usual even/odd split; the inverse runs the same steps backwards.
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <vector>

#include "df64.cuh"
#include "lp_internal.cuh"

namespace lpg {

namespace {

// sqrt(3)/2 = kS3h + kS3l (float(sqrt(3)/2) and the float of the remainder)
constexpr float kS3h = 0.8660253882408142f;
constexpr float kS3l = 1.5543625053737742e-08f;

// Arithmetic of one chain: DD = double-float complex values (float4 in
// memory: re.hi, re.lo, im.hi, im.lo), F32 = single-precision complex
// (float2).  Twiddles come from one df64 table; F32 uses its high parts.
struct DD {
  using V = cdd;
  using S = float4;
  __device__ static V load(const S* p) { return cdd_load(p); }
  __device__ static void store(S* p, V a) { cdd_store(p, a); }
  __device__ static V zero() { return cdd{dd{0.f, 0.f}, dd{0.f, 0.f}}; }
  __device__ static V add(V a, V b) { return cdd_add(a, b); }
  __device__ static V sub(V a, V b) { return cdd_sub(a, b); }
  __device__ static V conj(V a) { return cdd_conj(a); }
  __device__ static V mi(V a) { return cdd_mul_mi(a); }
  __device__ static V pi(V a) { return cdd_mul_pi(a); }
  __device__ static V half(V a) {
    return cdd{dd_scale(a.re, 0.5f), dd_scale(a.im, 0.5f)};
  }
  __device__ static V s3(V a) {
    const dd c = dd_make(kS3h, kS3l);
    return cdd{dd_mul(a.re, c), dd_mul(a.im, c)};
  }
  __device__ static V tw(const float4* t, int k) { return cdd_load(t + k); }
  __device__ static void store_tw(S* p, float4 v) { *p = v; }
  __device__ static V mul(V a, V t) { return cdd_mul(a, t); }
  __device__ static V mul_conj(V a, V t) { return cdd_mul_conj(a, t); }
};

struct F32 {
  using V = float2;
  using S = float2;
  __device__ static V load(const S* p) { return *p; }
  __device__ static void store(S* p, V a) { *p = a; }
  __device__ static V zero() { return make_float2(0.f, 0.f); }
  __device__ static V add(V a, V b) { return make_float2(a.x + b.x, a.y + b.y); }
  __device__ static V sub(V a, V b) { return make_float2(a.x - b.x, a.y - b.y); }
  __device__ static V conj(V a) { return make_float2(a.x, -a.y); }
  __device__ static V mi(V a) { return make_float2(a.y, -a.x); }
  __device__ static V pi(V a) { return make_float2(-a.y, a.x); }
  __device__ static V half(V a) { return make_float2(0.5f * a.x, 0.5f * a.y); }
  __device__ static V s3(V a) { return make_float2(kS3h * a.x, kS3h * a.y); }
  __device__ static V tw(const float4* t, int k) {
    const float4 v = t[k];
    return make_float2(v.x, v.z);
  }
  __device__ static void store_tw(S* p, float4 v) { *p = make_float2(v.x, v.z); }
  __device__ static V mul(V a, V t) { return make_float2(a.x * t.x - a.y * t.y, a.x * t.y + a.y * t.x); }
  __device__ static V mul_conj(V a, V t) { return make_float2(a.x * t.x + a.y * t.y, a.y * t.x - a.x * t.y); }
  template <int R>
  __device__ static V stw(int m);
};

// radices 8, 9 and 16 (two-level small DFTs) for the single-precision chain
// only; the double-float chain is bound by its arithmetic, not by the number
// of shared-memory passes, and keeps radices 2, 3 and 4 (its radix-8/9
// butterflies, with df64 internal twiddles, measured slower)
template <class A>
constexpr bool kHighRadix = false;
template <>
constexpr bool kHighRadix<F32> = true;
template <class A>
constexpr bool kRadix16 = kHighRadix<A>;

// e^{-2 pi i m / R} for the two-level small DFTs of the single-precision
// chain (R = 8, 9, 16; m < R)
template <int R>
__device__ __forceinline__ float2 small_tw(int m) {
  constexpr float t8[8][2] = {{1.f, 0.f}, {7.071067812e-01f, -7.071067812e-01f}, {0.f, -1.f},
                              {-7.071067812e-01f, -7.071067812e-01f}, {-1.f, 0.f},
                              {-7.071067812e-01f, 7.071067812e-01f}, {0.f, 1.f},
                              {7.071067812e-01f, 7.071067812e-01f}};
  constexpr float t9[9][2] = {{1.f, 0.f}, {7.660444431e-01f, -6.427876097e-01f},
                              {1.736481777e-01f, -9.848077530e-01f}, {-5.000000000e-01f, -8.660254038e-01f},
                              {-9.396926208e-01f, -3.420201433e-01f}, {-9.396926208e-01f, 3.420201433e-01f},
                              {-5.000000000e-01f, 8.660254038e-01f}, {1.736481777e-01f, 9.848077530e-01f},
                              {7.660444431e-01f, 6.427876097e-01f}};
  constexpr float t16[16][2] = {{1.f, 0.f}, {9.238795325e-01f, -3.826834324e-01f},
                                {7.071067812e-01f, -7.071067812e-01f}, {3.826834324e-01f, -9.238795325e-01f},
                                {0.f, -1.f}, {-3.826834324e-01f, -9.238795325e-01f},
                                {-7.071067812e-01f, -7.071067812e-01f}, {-9.238795325e-01f, -3.826834324e-01f},
                                {-1.f, 0.f}, {-9.238795325e-01f, 3.826834324e-01f},
                                {-7.071067812e-01f, 7.071067812e-01f}, {-3.826834324e-01f, 9.238795325e-01f},
                                {0.f, 1.f}, {3.826834324e-01f, 9.238795325e-01f},
                                {7.071067812e-01f, 7.071067812e-01f}, {9.238795325e-01f, 3.826834324e-01f}};
  if (R == 8) return make_float2(t8[m][0], t8[m][1]);
  if (R == 9) return make_float2(t9[m][0], t9[m][1]);
  return make_float2(t16[m][0], t16[m][1]);
}

template <int R>
__device__ float2 F32::stw(int m) {
  return small_tw<R>(m);
}

template <class A, int R>
__device__ __forceinline__ void dft_small(typename A::V* v, bool inv);

// DFT of length R = R1 R2 in registers from R2 DFTs of length R1 (over the
// inputs R2 n1 + n2), twiddles W_R^{n2 k1}, and R1 DFTs of length R2; the
// output k1 + R1 k2 (Cooley-Tukey with the index split n = R2 n1 + n2,
// k = k1 + R1 k2)
template <class A, int R1, int R2>
__device__ __forceinline__ void dft_two_level(typename A::V* v, bool inv) {
  using V = typename A::V;
  constexpr int R = R1 * R2;
  V y[R];
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    V t[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) t[n1] = v[R2 * n1 + n2];
    dft_small<A, R1>(t, inv);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      V z = t[k1];
      if (n2 * k1 != 0) {
        const V w = A::template stw<R>(n2 * k1);
        z = inv ? A::mul_conj(z, w) : A::mul(z, w);
      }
      y[n2 * R1 + k1] = z;
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    V t[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) t[n2] = y[n2 * R1 + k1];
    dft_small<A, R2>(t, inv);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = t[k2];
  }
}

template <class A, int R>
__device__ __forceinline__ void dft_small(typename A::V* v, bool inv) {
  using V = typename A::V;
  if constexpr (R == 8) {
    dft_two_level<A, 4, 2>(v, inv);
  } else if constexpr (R == 9) {
    dft_two_level<A, 3, 3>(v, inv);
  } else if constexpr (R == 16) {
    dft_two_level<A, 4, 4>(v, inv);
  } else if constexpr (R == 2) {
    const V a = v[0], b = v[1];
    v[0] = A::add(a, b);
    v[1] = A::sub(a, b);
  } else if constexpr (R == 4) {
    const V t0 = A::add(v[0], v[2]), t1 = A::sub(v[0], v[2]);
    const V t2 = A::add(v[1], v[3]);
    const V d = A::sub(v[1], v[3]);
    const V t3 = inv ? A::pi(d) : A::mi(d);
    v[0] = A::add(t0, t2);
    v[1] = A::add(t1, t3);
    v[2] = A::sub(t0, t2);
    v[3] = A::sub(t1, t3);
  } else {  // R == 3
    const V t1 = A::add(v[1], v[2]);
    const V t2 = A::sub(v[0], A::half(t1));
    const V ds = A::s3(A::sub(v[1], v[2]));
    const V t3 = inv ? A::pi(ds) : A::mi(ds);
    v[0] = A::add(v[0], t1);
    v[1] = A::add(t2, t3);
    v[2] = A::sub(t2, t3);
  }
}

// Twiddles e^{-2 pi i m / N} of a length-N transform: from a shared-memory
// table of the N values, or from the global df64 table of length g at
// stride tws = g / N.
template <class A>
struct SmemTw {
  const typename A::S* t;
  __device__ typename A::V operator()(int m) const { return A::load(t + m); }
};
template <class A>
struct GlobTw {
  const float4* __restrict__ t;
  int tws;
  __device__ typename A::V operator()(int m) const { return A::tw(t, m * tws); }
};

// the N twiddles of a length-N transform into shared memory (the caller
// synchronises before use)
template <class A>
__device__ __forceinline__ void load_twiddles(typename A::S* dst, const float4* __restrict__ tw, int N, int tws) {
  for (int m = threadIdx.x; m < N; m += blockDim.x) A::store_tw(dst + m, __ldg(tw + (size_t)m * tws));
}

template <class A, int R, class TW>
__device__ __forceinline__ void stockham_butterfly(const typename A::S* in, typename A::S* out, int j, int N,
                                                   int Ns, const TW& tw, bool inv) {
  using V = typename A::V;
  const int stride = N / R;
  V v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = A::load(in + j + r * stride);
  const int k = j % Ns;
  if (k != 0) {
    const int step = N / (Ns * R);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const V t = tw(k * r * step);
      v[r] = inv ? A::mul_conj(v[r], t) : A::mul(v[r], t);
    }
  }
  dft_small<A, R>(v, inv);
  const int base = (j - k) * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r) A::store(out + base + r * Ns, v[r]);
}

// Transform of length N held in a (scratch b); returns the buffer holding
// the result.  All threads of the CTA take part; the caller synchronises
// before (data in a) and the function synchronises after every stage.
// HIGH: the shape may hold radices 8, 9, 16 (compiled only where used, so
// that the row kernels keep their registers)
template <class A, bool HIGH, class TW>
__device__ typename A::S* fft_smem(typename A::S* a, typename A::S* b, const FftShape& sh, const TW& tw,
                                   bool inv) {
  const int N = sh.n;
  int Ns = 1;
  for (int s = 0; s < sh.nst; ++s) {
    const int R = sh.radix[s];
    const int nb = N / R;
    if (R == 4) {
      for (int j = threadIdx.x; j < nb; j += blockDim.x) stockham_butterfly<A, 4>(a, b, j, N, Ns, tw, inv);
    } else if (R == 2) {
      for (int j = threadIdx.x; j < nb; j += blockDim.x) stockham_butterfly<A, 2>(a, b, j, N, Ns, tw, inv);
    } else if (R == 3) {
      for (int j = threadIdx.x; j < nb; j += blockDim.x) stockham_butterfly<A, 3>(a, b, j, N, Ns, tw, inv);
    } else if constexpr (HIGH) {
      if (R == 8) {
        for (int j = threadIdx.x; j < nb; j += blockDim.x) stockham_butterfly<A, 8>(a, b, j, N, Ns, tw, inv);
      } else if (R == 9) {
        for (int j = threadIdx.x; j < nb; j += blockDim.x) stockham_butterfly<A, 9>(a, b, j, N, Ns, tw, inv);
      } else {
        for (int j = threadIdx.x; j < nb; j += blockDim.x) stockham_butterfly<A, 16>(a, b, j, N, Ns, tw, inv);
      }
    }
    __syncthreads();
    typename A::S* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// In-place mixed-radix transforms of one shared-memory buffer (used by the
// column pass, whose spectrum is only multiplied between the forward and the
// inverse transform).  Forward: decimation in frequency (Sande-Tukey) over the
// radices in order; stage s splits blocks of length L into R interleaved
// sub-blocks of length L/R (butterfly, then twiddles W_L^{t j}), leaving the
// transform in mixed-radix digit-reversed order (position p holds frequency
// fft_dif_order[p]).  Inverse: decimation in time over the radices in
// reverse order (conjugate twiddles, then the conjugate butterfly), taking
// that order back to natural order.  Unnormalised, like the Stockham form.
template <class A, int R, class TW>
__device__ __forceinline__ void dif_stage(typename A::S* x, int N, int L, const TW& tw, int t0, int nt) {
  using V = typename A::V;
  const int Lr = L / R, step = N / L;
  for (int q = t0; q < N / R; q += nt) {
    const int b = q / Lr, j = q - b * Lr;
    typename A::S* base = x + b * L + j;
    V v[R];
#pragma unroll
    for (int u = 0; u < R; ++u) v[u] = A::load(base + u * Lr);
    dft_small<A, R>(v, false);
    if (j != 0) {
#pragma unroll
      for (int t = 1; t < R; ++t) v[t] = A::mul(v[t], tw(t * j * step));
    }
#pragma unroll
    for (int t = 0; t < R; ++t) A::store(base + t * Lr, v[t]);
  }
}

template <class A, int R, class TW>
__device__ __forceinline__ void dit_stage_inv(typename A::S* x, int N, int L, const TW& tw, int t0, int nt) {
  using V = typename A::V;
  const int Lr = L / R, step = N / L;
  for (int q = t0; q < N / R; q += nt) {
    const int b = q / Lr, j = q - b * Lr;
    typename A::S* base = x + b * L + j;
    V v[R];
#pragma unroll
    for (int t = 0; t < R; ++t) v[t] = A::load(base + t * Lr);
    if (j != 0) {
#pragma unroll
      for (int t = 1; t < R; ++t) v[t] = A::mul_conj(v[t], tw(t * j * step));
    }
    dft_small<A, R>(v, true);
#pragma unroll
    for (int u = 0; u < R; ++u) A::store(base + u * Lr, v[u]);
  }
}

// Threads t0, t0 + nt, ... of the CTA transform x; the caller synchronises
// before (data in x); every stage ends with a CTA-wide barrier, so all
// thread groups of the CTA must run the same sequence of stages.
template <class A, class TW>
__device__ void fft_dif(typename A::S* x, const FftShape& sh, const TW& tw, int t0, int nt) {
  const int N = sh.n;
  int L = N;
  for (int s = 0; s < sh.nst; ++s) {
    const int R = sh.radix[s];
    if (R == 4) dif_stage<A, 4>(x, N, L, tw, t0, nt);
    else if (R == 2) dif_stage<A, 2>(x, N, L, tw, t0, nt);
    else if (R == 3) dif_stage<A, 3>(x, N, L, tw, t0, nt);
    else if constexpr (kHighRadix<A>) {
      if (R == 8) dif_stage<A, 8>(x, N, L, tw, t0, nt);
      else if (R == 9) dif_stage<A, 9>(x, N, L, tw, t0, nt);
      else if constexpr (kRadix16<A>) dif_stage<A, 16>(x, N, L, tw, t0, nt);
    }
    __syncthreads();
    L /= R;
  }
}

template <class A, class TW>
__device__ void fft_dit_inv(typename A::S* x, const FftShape& sh, const TW& tw, int t0, int nt) {
  const int N = sh.n;
  int L = sh.radix[sh.nst - 1];  // the block length of the last forward stage
  for (int s = sh.nst - 1; s >= 0; --s) {
    const int R = sh.radix[s];
    if (R == 4) dit_stage_inv<A, 4>(x, N, L, tw, t0, nt);
    else if (R == 2) dit_stage_inv<A, 2>(x, N, L, tw, t0, nt);
    else if (R == 3) dit_stage_inv<A, 3>(x, N, L, tw, t0, nt);
    else if constexpr (kHighRadix<A>) {
      if (R == 8) dit_stage_inv<A, 8>(x, N, L, tw, t0, nt);
      else if (R == 9) dit_stage_inv<A, 9>(x, N, L, tw, t0, nt);
      else if constexpr (kRadix16<A>) dit_stage_inv<A, 16>(x, N, L, tw, t0, nt);
    }
    __syncthreads();
    if (s > 0) L *= sh.radix[s - 1];
  }
}

// grid row -> complex sequence z_n = x_2n + i x_2n+1
__device__ __forceinline__ cdd load_pair(const void* row, int n, DD) {
  const double2 x = *((const double2*)row + n);
  return cdd{dd_from_double(x.x), dd_from_double(x.y)};
}
__device__ __forceinline__ float2 load_pair(const void* row, int n, F32) { return *((const float2*)row + n); }

// complex z_n -> grid row values x_2n, x_2n+1 (df64 pairs, or floats)
__device__ __forceinline__ void store_pair(void* row, int n, cdd z, DD) { cdd_store((float4*)row + n, z); }
__device__ __forceinline__ void store_pair(void* row, int n, float2 z, F32) { *((float2*)row + n) = z; }

// multiplier table entry: df64 pair, or float
__device__ __forceinline__ dd mult_value(const void* tab, size_t i, DD) {
  const float2 m = ((const float2*)tab)[i];
  return dd_make(m.x, m.y);
}
__device__ __forceinline__ float mult_value(const void* tab, size_t i, F32) { return ((const float*)tab)[i]; }

__device__ __forceinline__ cdd scale_real(cdd a, dd m) { return cdd_scale_dd(a, m); }
__device__ __forceinline__ float2 scale_real(float2 a, float m) { return make_float2(a.x * m, a.y * m); }

// m (-i)(kx f1 + ky f2), kx = dk mx, ky = dk my
__device__ __forceinline__ cdd dipole_mode(cdd f1, cdd f2, dd m, float2 dk2, int mx, int my) {
  const dd dk = dd_make(dk2.x, dk2.y);
  const dd kx = dd_mul_f(dk, (float)mx), ky = dd_mul_f(dk, (float)my);
  const dd re = dd_dot2(kx, f1.im, ky, f2.im);
  const dd im = dd_dot2(kx, f1.re, ky, f2.re);
  return cdd{dd_mul(m, re), dd_neg(dd_mul(m, im))};
}
__device__ __forceinline__ float2 dipole_mode(float2 f1, float2 f2, float m, float2 dk2, int mx, int my) {
  const float kx = dk2.x * (float)mx, ky = dk2.x * (float)my;
  return make_float2(m * (kx * f1.y + ky * f2.y), -m * (kx * f1.x + ky * f2.x));
}

// Single-precision chain, low modes: the FP64 table entry, the product in
// double, one rounding to float (k = 0 is excluded: its term is added in
// FP64 at the targets)
__device__ __forceinline__ float2 scale_low(float2 z, double m) {
  return make_float2((float)((double)z.x * m), (float)((double)z.y * m));
}
// (the double-float chain's forms, for the generic multiplier loop: it never
// takes this path, since its table is already in double-float)
__device__ __forceinline__ cdd scale_low(cdd z, double m) { return cdd_scale_dd(z, dd_from_double(m)); }
__device__ __forceinline__ cdd dipole_low(cdd f1, cdd f2, double m, float2 dk2, int mx, int my) {
  return dipole_mode(f1, f2, dd_from_double(m), dk2, mx, my);
}
__device__ __forceinline__ float2 dipole_low(float2 f1, float2 f2, double m, float2 dk2, int mx, int my) {
  const double dk = (double)dk2.x + (double)dk2.y;
  const double kx = dk * mx, ky = dk * my;
  return make_float2((float)(m * (kx * (double)f1.y + ky * (double)f2.y)),
                     (float)(-m * (kx * (double)f1.x + ky * (double)f2.x)));
}

// Twiddles in shared memory (a third buffer) for the single-precision chain:
// its butterflies are cheap and the per-stage global twiddle loads saturated
// the L1 pipe.  The double-float chain keeps the global table: a third
// 16-byte buffer cuts the CTAs per SM (measured slower) and, for columns of
// the largest grids, exceeds shared memory.
template <class A>
constexpr bool kTwSmem = false;
template <>
constexpr bool kTwSmem<F32> = true;

// Forward transform of real rows: one CTA per (row, channel).
template <class A>
__global__ void __launch_bounds__(kFftThreads) fft_rows_fwd_kernel(const __grid_constant__ FftRowArgs a) {
  using V = typename A::V;
  using S = typename A::S;
  extern __shared__ float4 sm_raw[];
  S* sm = (S*)sm_raw;
  const int N = a.half.n;
  const int row = a.row_lo + blockIdx.x, c = blockIdx.y;
  // a complex value of the chain takes twice the bytes of a real grid element
  const char* src = (const char*)a.grid[c] + (size_t)row * a.pitch * (sizeof(S) / 2);
  S* buf0 = sm;
  S* buf1 = sm + N;
  S* twt = sm + 2 * N;
  if (kTwSmem<A>) load_twiddles<A>(twt, a.tw, N, 2);
  for (int n = threadIdx.x; n < N; n += blockDim.x) A::store(buf0 + n, load_pair(src, n, A()));
  __syncthreads();
  const S* Z = kTwSmem<A> ? fft_smem<A, false>(buf0, buf1, a.half, SmemTw<A>{twt}, false)
                          : fft_smem<A, false>(buf0, buf1, a.half, GlobTw<A>{a.tw, 2}, false);
  S* dst = (S*)a.spec[c] + (size_t)row * a.kp;
  for (int k = threadIdx.x; k <= a.K; k += blockDim.x) {
    const V zk = A::load(Z + k), zn = A::conj(A::load(Z + (k == 0 ? 0 : N - k)));
    const V e = A::half(A::add(zk, zn));
    const V o = A::mi(A::half(A::sub(zk, zn)));
    A::store(dst + k, A::add(e, A::mul(o, A::tw(a.tw, k))));
  }
}

// strided column loads in flight per thread
template <class A>
constexpr int kColBatch = 4;
template <>
constexpr int kColBatch<F32> = 8;

// Column pass: one CTA per (C adjacent kept columns, job), one shared-memory
// buffer of g values per column (in-place transforms) and a group of
// kFftThreads threads per column.  Loads and stores interleave the C columns,
// so the C values of a spectrum row fill whole 32-byte sectors (the spectrum
// is stored row by row).  Jobs of kind 0 transform one spectrum and multiply
// by M; kind 1 (D) transforms two and combines them, parking the first
// transform (in digit-reversed order) in its own global columns meanwhile.
// The multiplier is applied in the forward transform's order.
template <class A, int C>
__device__ __forceinline__ void fft_cols_body(const FftColArgs& a) {
  using V = typename A::V;
  using S = typename A::S;
  extern __shared__ float4 sm_raw[];
  S* sm = (S*)sm_raw;
  const int g = a.full.n, K = a.K, mx0 = blockIdx.x * C;
  const int grp = threadIdx.x / kFftThreads, t0 = threadIdx.x % kFftThreads;
  const int mx = mx0 + grp;  // this group's column
  const FftColJob& job = a.job[blockIdx.y];
  S* x = sm + (size_t)grp * g;
  S* twt = sm + (size_t)C * g;
  if (kTwSmem<A>) load_twiddles<A>(twt, a.tw, g, 1);
  const SmemTw<A> tws{twt};
  const GlobTw<A> twg{a.tw, 1};
  // element e of the CTA's C x g block: row e / C, column mx0 + e % C; the
  // strided loads are issued kColBatch at a time before their stores, so
  // that several are in flight per thread
  auto load_cols = [&](const void* spec) {
    const S* sp = (const S*)spec;
    constexpr int U = kColBatch<A>;
    for (int e0 = threadIdx.x; e0 < C * g; e0 += U * blockDim.x) {
      S v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x, r = e / C, c = e - r * C;
        if (e < C * g && r >= a.row_lo && r < a.row_hi && mx0 + c < a.kp)
          v[u] = sp[(size_t)r * a.kp + mx0 + c];
        else
          A::store(v + u, A::zero());
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x, r = e / C, c = e - r * C;
        if (e < C * g) sm[(size_t)c * g + r] = v[u];
      }
    }
    __syncthreads();
  };
  auto forward = [&]() {
    if (kTwSmem<A>)
      fft_dif<A>(x, a.full, tws, t0, kFftThreads);
    else
      fft_dif<A>(x, a.full, twg, t0, kFftThreads);
  };
  // The multiplier on the forward-transformed column, in place (KIND 1:
  // the D combination with the parked D1 column).  FP32 plans: a column
  // with m_x < klo takes the FP64 entry for its modes |m_y| < klo (k = 0
  // excepted), decided once per column so that the other columns run the
  // plain loop.
  auto mult_loop = [&](const S* park, auto kind_tag, auto low_tag) {
    constexpr int KIND = decltype(kind_tag)::value;
    constexpr bool LOW = decltype(low_tag)::value && std::is_same<A, F32>::value;
    for (int p = t0; p < g; p += kFftThreads) {
      const int r = __ldg(a.freq + p);
      const int my = r <= g / 2 ? r : r - g;
      const int amy = my < 0 ? -my : my;
      V o = A::zero();
      if (amy <= K && mx <= K) {
        const size_t ti = (size_t)amy * (K + 1) + mx;
        bool done = false;
        if constexpr (LOW) {
          if (amy < a.klo && (mx | amy) != 0) {
            if constexpr (KIND == 1)
              o = dipole_low(A::load(park + (size_t)p * a.kp + mx), A::load(x + p), a.tab64[ti], a.dk, mx, my);
            else
              o = scale_low(A::load(x + p), a.tab64[ti]);
            done = true;
          }
        }
        if (!done) {
          if constexpr (KIND == 1)
            o = dipole_mode(A::load(park + (size_t)p * a.kp + mx), A::load(x + p), mult_value(a.tab, ti, A()),
                            a.dk, mx, my);
          else
            o = scale_real(A::load(x + p), mult_value(a.tab, ti, A()));
        }
      }
      A::store(x + p, o);
    }
  };
  auto mult_column = [&](const S* park, auto kind_tag) {
    if (a.tab64 != nullptr && mx < a.klo)
      mult_loop(park, kind_tag, std::true_type{});
    else
      mult_loop(park, kind_tag, std::false_type{});
  };
  if (job.kind == 1) {
    load_cols(job.in[0]);
    forward();
    S* park = (S*)job.out;  // the D1 spectrum columns, all g rows
    for (int e = threadIdx.x; e < C * g; e += blockDim.x) {
      const int p = e / C, c = e - p * C;
      if (mx0 + c < a.kp) park[(size_t)p * a.kp + mx0 + c] = sm[(size_t)c * g + p];
    }
    __syncthreads();
    load_cols(job.in[1]);
    forward();
    mult_column(park, std::integral_constant<int, 1>{});
  } else {
    load_cols(job.in[0]);
    forward();
    mult_column(nullptr, std::integral_constant<int, 0>{});
  }
  __syncthreads();
  if (kTwSmem<A>)
    fft_dit_inv<A>(x, a.full, tws, t0, kFftThreads);
  else
    fft_dit_inv<A>(x, a.full, twg, t0, kFftThreads);
  S* out = (S*)job.out;
  for (int e = threadIdx.x; e < C * (a.row_hi - a.row_lo); e += blockDim.x) {
    const int rr = e / C, c = e - rr * C, r = a.row_lo + rr;
    if (mx0 + c < a.kp) out[(size_t)r * a.kp + mx0 + c] = sm[(size_t)c * g + r];
  }
}

template <class A, int C>
__global__ void __launch_bounds__(kFftThreads * C) fft_cols_kernel(const __grid_constant__ FftColArgs a) {
  fft_cols_body<A, C>(a);
}

// FP32, two columns per CTA, compiled for two resident CTAs per SM (64
// registers): with the compiler's own choice (87) only one 512-thread CTA
// would fit
__global__ void __launch_bounds__(kFftThreads * 2, 2) fft_cols2_f32_kernel(const __grid_constant__ FftColArgs a) {
  fft_cols_body<F32, 2>(a);
}

// Inverse transform of rows: one CTA per (row, job); writes the g values of
// the row over the job's grid row (df64 pairs over the FP64 grid, or floats).
template <class A>
__global__ void __launch_bounds__(kFftThreads) fft_rows_inv_kernel(const __grid_constant__ FftRowArgs a) {
  using V = typename A::V;
  using S = typename A::S;
  extern __shared__ float4 sm_raw[];
  S* sm = (S*)sm_raw;
  const int N = a.half.n;
  const int row = a.row_lo + blockIdx.x, c = blockIdx.y;
  const S* spec = (const S*)a.spec[c] + (size_t)row * a.kp;
  S* buf0 = sm;
  S* buf1 = sm + N;
  S* twt = sm + 2 * N;
  if (kTwSmem<A>) load_twiddles<A>(twt, a.tw, N, 2);
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    V xk = k <= a.K ? A::load(spec + k) : A::zero();
    if (k == 0) xk = A::add(A::half(xk), A::half(A::conj(xk)));  // drop the imaginary part
    const int nk = N - k;
    const V xn = nk <= a.K ? A::conj(A::load(spec + nk)) : A::zero();
    const V B = A::mul_conj(A::sub(xk, xn), A::tw(a.tw, k));
    A::store(buf0 + k, A::add(A::add(xk, xn), A::pi(B)));
  }
  __syncthreads();
  const S* z = kTwSmem<A> ? fft_smem<A, false>(buf0, buf1, a.half, SmemTw<A>{twt}, true)
                          : fft_smem<A, false>(buf0, buf1, a.half, GlobTw<A>{a.tw, 2}, true);
  char* dst = (char*)a.grid[c] + (size_t)row * a.pitch * (sizeof(S) / 2);
  for (int n = threadIdx.x; n < N; n += blockDim.x) store_pair(dst, n, A::load(z + n), A());
}

__global__ void split_table_kernel(const double* __restrict__ src, float2* dst, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const dd v = dd_from_double(src[i]);
  dst[i] = make_float2(v.hi, v.lo);
}

}  // namespace

void launch_split_table(const double* src, float2* dst, int64_t n, cudaStream_t s) {
  if (n > 0) split_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
}

FftShape fft_shape(int n, bool high, bool r16) {
  FftShape s{};
  s.n = n;
  int m = n;
  auto take = [&](int r) {
    while (m % r == 0 && s.nst < kMaxFftStages) {
      s.radix[s.nst++] = r;
      m /= r;
    }
  };
  if (high) {  // powers of two as 16s (if r16) or 8s, then one 8, 4 or 2; powers of three as 9s, then one 3
    if (r16) take(16);
    if (m % 8 == 0) take(8);
  }
  take(4);
  if (m % 2 == 0 && s.nst < kMaxFftStages) {
    s.radix[s.nst++] = 2;
    m /= 2;
  }
  if (high) take(9);
  take(3);
  if (m != 1) s.nst = -1;  // not 3-smooth
  return s;
}

// e^{-2 pi i k / g}, k = 0..g-1, as df64 (hi, lo) pairs of the real and
// imaginary parts, from long double cos/sin
std::vector<float4> fft_twiddles(int g) {
  std::vector<float4> t(g);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < g; ++k) {
    const long double ang = -2.0L * pi * (long double)k / (long double)g;
    const long double c = cosl(ang), s = sinl(ang);
    const float ch = (float)c, sh = (float)s;
    t[k] = make_float4(ch, (float)(c - (long double)ch), sh, (float)(s - (long double)sh));
  }
  return t;
}

// rows: two buffers of the transform length, and for FP32 the twiddle table
size_t fft_rows_smem(int g, bool f64) { return f64 ? (size_t)2 * (g / 2) * sizeof(float4) : (size_t)3 * (g / 2) * sizeof(float2); }
// columns: one buffer per column of a CTA (in-place transforms), and for
// FP32 the twiddle table
size_t fft_cols_smem_c(int g, bool f64, int C) {
  return f64 ? (size_t)C * g * sizeof(float4) : (size_t)(C + 1) * g * sizeof(float2);
}
// Columns per CTA: FP64 two when they fit (their 16-byte values then fill
// whole sectors; measured 0.56 -> 0.54 ms on the starfish); FP32 two when
// at least two CTAs fit on an SM (adjacent lanes read the two columns' 8-byte
// values of a row as 16 contiguous bytes; four 1024-thread groups measured
// slower: 0.30 -> 0.32 ms).
int fft_cols_per_cta(int g, bool f64) {
  if (f64 && fft_cols_smem_c(g, f64, 2) <= 220 * 1024) return 2;
  if (!f64 && fft_cols_smem_c(g, f64, 2) <= 110 * 1024) return 2;
  return 1;
}
size_t fft_cols_smem(int g, bool f64) { return fft_cols_smem_c(g, f64, 1); }

// Position -> frequency of the in-place decimation-in-frequency transform:
// after stage s (radix R_s, block length L_s -> L_s / R_s) the digit of
// frequency weight R_0 ... R_{s-1} sits at position weight L_s / R_s.
std::vector<int> fft_dif_order(const FftShape& sh) {
  std::vector<int> fr(sh.n);
  for (int p = 0; p < sh.n; ++p) {
    int q = p, k = 0, prod = 1, L = sh.n;
    for (int s = 0; s < sh.nst; ++s) {
      L /= sh.radix[s];
      const int d = q / L;
      q -= d * L;
      k += d * prod;
      prod *= sh.radix[s];
    }
    fr[p] = k;
  }
  return fr;
}

bool fft_dd_configure() {
  const int bytes = 220 * 1024;
  const void* fns[8] = {(const void*)fft_rows_fwd_kernel<DD>,  (const void*)fft_rows_inv_kernel<DD>,
                        (const void*)fft_cols_kernel<DD, 1>,    (const void*)fft_cols_kernel<DD, 2>,
                        (const void*)fft_rows_fwd_kernel<F32>, (const void*)fft_rows_inv_kernel<F32>,
                        (const void*)fft_cols_kernel<F32, 1>,   (const void*)fft_cols2_f32_kernel};
  for (const void* f : fns)
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return false;
  return true;
}

// Threads per row transform: about one per radix-4 butterfly of a stage
// (N / 4, a whole number of warps, 32 .. kFftThreads), so that the short
// rows of small grids do not leave most of a 256-thread CTA idle; the row
// kernels stride by blockDim.
static int row_threads(int N) {
  const int t = ((N / 4 + 31) / 32) * 32;
  return std::min(kFftThreads, std::max(32, t));
}

void launch_fft_rows_fwd(const FftRowArgs& a, int nchan, bool f64, cudaStream_t s) {
  const int nrows = a.row_hi - a.row_lo;
  if (nrows <= 0 || nchan <= 0) return;
  const size_t smem = fft_rows_smem(2 * a.half.n, f64);
  if (f64)
    fft_rows_fwd_kernel<DD><<<dim3(nrows, nchan), row_threads(a.half.n), smem, s>>>(a);
  else
    fft_rows_fwd_kernel<F32><<<dim3(nrows, nchan), row_threads(a.half.n), smem, s>>>(a);
}

void launch_fft_rows_inv(const FftRowArgs& a, int nchan, bool f64, cudaStream_t s) {
  const int nrows = a.row_hi - a.row_lo;
  if (nrows <= 0 || nchan <= 0) return;
  const size_t smem = fft_rows_smem(2 * a.half.n, f64);
  if (f64)
    fft_rows_inv_kernel<DD><<<dim3(nrows, nchan), row_threads(a.half.n), smem, s>>>(a);
  else
    fft_rows_inv_kernel<F32><<<dim3(nrows, nchan), row_threads(a.half.n), smem, s>>>(a);
}

void launch_fft_cols(const FftColArgs& a, int njobs, bool f64, cudaStream_t s) {
  if (njobs <= 0) return;
  const int C = fft_cols_per_cta(a.full.n, f64);
  const size_t smem = fft_cols_smem_c(a.full.n, f64, C);
  const dim3 grid((a.K + C) / C, njobs);  // ceil((K + 1) / C) column groups
  if (f64) {
    if (C == 2)
      fft_cols_kernel<DD, 2><<<grid, kFftThreads * 2, smem, s>>>(a);
    else
      fft_cols_kernel<DD, 1><<<grid, kFftThreads, smem, s>>>(a);
  } else {
    if (C == 2)
      fft_cols2_f32_kernel<<<grid, kFftThreads * 2, smem, s>>>(a);
    else
      fft_cols_kernel<F32, 1><<<grid, kFftThreads, smem, s>>>(a);
  }
}

}  // namespace lpg
