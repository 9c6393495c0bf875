// Dyadic refinement of the local layer potentials (Sec. 4.4).  With
// delta_j = delta / 4^j the local parts satisfy
//   S_L[delta] = S_L[delta_J] + sum_{j=1..J} int_Gamma (G_H[delta_j] - G_H[delta_{j-1}]) sigma ds,
// and the same for D with the source-point normal derivative of the
// difference kernel.  The expansions are evaluated at delta_J (k_local.cu);
// the difference integrals are direct sums over the boundary panels split
// into m_j = 2^j equal parameter intervals of p Gauss-Legendre nodes each
// ("subnodes"), with position, weight and normal from the panel's Legendre
// interpolant.  In x = 4^{j-1} |x - x'|^2 / delta the kernels of level j are
//   S: F(x) = (E1(x/4) - E1(x)) / (4 pi)
//   D: (4^{j-1} / (2 pi delta)) H(x) nu.(x - x'),  H(x) = (e^{-x/4} - e^{-x}) / x,
// both negligible (below e^{-36}) for x >= 144 -- the level-j range is
// 12 sqrt(delta_{j-1}).  F and H are tabulated once per plan as piecewise
// polynomials on unit intervals of x.  FP64 plans sum in double-float
// arithmetic, FP32 plans in single precision.
#include <algorithm>
#include <cmath>
#include <vector>

#include "df64.cuh"
#include "lp_internal.cuh"

namespace lpg {

namespace {

// Legendre jets of order ND for NS series (coefficients / k!, scaled
// recurrence Q_k = k! P_k), as in the local pass.
template <int ND, int NS>
__device__ __forceinline__ void jets64(const double* const* c, const double* ref, int p, double t,
                                       double (*out)[ND + 1]) {
  double qm[ND + 1], qk[ND + 1];
#pragma unroll
  for (int j = 0; j <= ND; ++j) {
    qm[j] = 0;
    qk[j] = (j == 0) ? 1.0 : 0.0;
  }
#pragma unroll
  for (int q = 0; q < NS; ++q) {
#pragma unroll
    for (int j = 0; j <= ND; ++j) out[q][j] = 0;
    out[q][0] = ref[q] + c[q][0];
  }
  for (int k = 0; k + 1 < p; ++k) {
    const double a = 2 * k + 1, b = (double)k * k;
#pragma unroll
    for (int j = ND; j >= 0; --j) {
      const double prev = j ? qk[j - 1] : 0.0;
      const double qn = a * fma(t, qk[j], j * prev) - b * qm[j];
      qm[j] = qk[j];
      qk[j] = qn;
    }
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const double ck = c[q][k + 1];
#pragma unroll
      for (int j = 0; j <= ND; ++j) out[q][j] = fma(ck, qk[j], out[q][j]);
    }
  }
}

__device__ __forceinline__ float4 dd_pair(double a, double b) {
  const dd x = dd_from_double(a), y = dd_from_double(b);
  return make_float4(x.hi, x.lo, y.hi, y.lo);
}

// Subnode geometry of one level: offset from the panel's reference node,
// and the outward normal times the arc-length weight, both as df64 pairs.
__global__ void dyadic_geom_kernel(const double* __restrict__ geo_coef, const double* __restrict__ tau,
                                   const double* __restrict__ wgl, int n_panels, int p, int m, float4* rel,
                                   float4* nw) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nq = (int64_t)n_panels * m * p;
  if (q >= nq) return;
  const int i = (int)(q % p), k = (int)((q / p) % m), ip = (int)(q / ((int64_t)p * m));
  const double t = -1.0 + (2.0 * k + 1.0 + tau[i]) / m;
  const double* c[2] = {geo_coef + (size_t)(2 * ip) * p, geo_coef + (size_t)(2 * ip + 1) * p};
  const double zero[2] = {0.0, 0.0};
  double J[2][2];
  jets64<1, 2>(c, zero, p, t, J);
  const double sp = sqrt(J[0][1] * J[0][1] + J[1][1] * J[1][1]);
  const double w = sp * wgl[i] / m;
  rel[q] = dd_pair(J[0][0], J[1][0]);
  nw[q] = dd_pair(J[1][1] / sp * w, -J[0][1] / sp * w);  // outward normal of a counter-clockwise curve
}

// Densities at the subnodes of one level (at bind time): sigma times the
// weight, and mu, as df64 pairs.
__global__ void dyadic_dens_kernel(const double* __restrict__ coef, const double* __restrict__ ref,
                                   const double* __restrict__ tau, const double* __restrict__ wgl,
                                   const double* __restrict__ geo_coef, int n_panels, int p, int m, int times_w,
                                   float2* out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nq = (int64_t)n_panels * m * p;
  if (q >= nq) return;
  const int i = (int)(q % p), k = (int)((q / p) % m), ip = (int)(q / ((int64_t)p * m));
  const double t = -1.0 + (2.0 * k + 1.0 + tau[i]) / m;
  const double* c[1] = {coef + (size_t)ip * p};
  const double r[1] = {ref[ip]};
  double V[1][1];
  jets64<0, 1>(c, r, p, t, V);
  double v = V[0][0];
  if (times_w) {
    const double* g[2] = {geo_coef + (size_t)(2 * ip) * p, geo_coef + (size_t)(2 * ip + 1) * p};
    const double zero[2] = {0.0, 0.0};
    double J[2][2];
    jets64<1, 2>(g, zero, p, t, J);
    v *= sqrt(J[0][1] * J[0][1] + J[1][1] * J[1][1]) * wgl[i] / m;
  }
  const dd d = dd_from_double(v);
  out[q] = make_float2(d.hi, d.lo);
}

// Arithmetic of the sums: df64 (FP64 plans) or float (FP32 plans).  Acc is
// the running-sum form (for df64 a sum and a correction term).
struct SumDD {
  using V = dd;
  using Acc = dd_acc;
  __device__ static V make(float hi, float lo) { return dd{hi, lo}; }
  __device__ static V sub(V a, V b) { return dd_sub(a, b); }
  __device__ static V mul(V a, V b) { return dd_mul(a, b); }
  __device__ static V scale(V a, float pow2) { return dd_scale(a, pow2); }
  __device__ static V dot2(V a, V b, V c, V d) { return dd_dot2(a, b, c, d); }
  __device__ static float hi(V a) { return a.hi; }
  __device__ static V from_dd(dd a) { return a; }
  __device__ static double to_double(V a) { return dd_to_double(a); }
  __device__ static Acc zero() { return dd_acc{0.f, 0.f}; }
  __device__ static void fma(Acc& acc, V a, V b) { acc_fma(acc, a, b); }
  __device__ static V shfl(V a, int src) {
    return dd{__shfl_sync(0xffffffffu, a.hi, src), __shfl_sync(0xffffffffu, a.lo, src)};
  }
  __device__ static V warp_sum(Acc acc) {
    V v = acc_value(acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      v = dd_add(v, dd{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
    return v;
  }
  // piece polynomial: c4..c15 in single precision (their sum is below 1e-3
  // of the value on every piece), c3..c0 as df64 Horner steps
  __device__ static V poly(const float4* c, V s) {
    const float sh = s.hi;
    const float4 t2 = c[2], t3 = c[3], t4 = c[4];
    float t = t4.w;
    t = fmaf(t, sh, t4.z);
    t = fmaf(t, sh, t4.y);
    t = fmaf(t, sh, t4.x);
    t = fmaf(t, sh, t3.w);
    t = fmaf(t, sh, t3.z);
    t = fmaf(t, sh, t3.y);
    t = fmaf(t, sh, t3.x);
    t = fmaf(t, sh, t2.w);
    t = fmaf(t, sh, t2.z);
    t = fmaf(t, sh, t2.y);
    t = fmaf(t, sh, t2.x);
    const float4 h0 = c[0], h1 = c[1];
    dd acc = dd_horner(dd{t, 0.f}, s, make_float2(h1.z, h1.w));
    acc = dd_horner(acc, s, make_float2(h1.x, h1.y));
    acc = dd_horner(acc, s, make_float2(h0.z, h0.w));
    return dd_horner(acc, s, make_float2(h0.x, h0.y));
  }
};

struct SumF {
  using V = float;
  using Acc = float;
  __device__ static V make(float hi, float) { return hi; }
  __device__ static V sub(V a, V b) { return a - b; }
  __device__ static V mul(V a, V b) { return a * b; }
  __device__ static V scale(V a, float pow2) { return a * pow2; }
  __device__ static V dot2(V a, V b, V c, V d) { return fmaf(a, b, c * d); }
  __device__ static float hi(V a) { return a; }
  __device__ static V from_dd(dd a) { return a.hi; }
  __device__ static double to_double(V a) { return (double)a; }
  __device__ static Acc zero() { return 0.f; }
  __device__ static void fma(Acc& acc, V a, V b) { acc = fmaf(a, b, acc); }
  __device__ static V shfl(V a, int src) { return __shfl_sync(0xffffffffu, a, src); }
  __device__ static V warp_sum(Acc v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  }
  __device__ static V poly(const float4* c, V s) {
    const float4 h0 = c[0], h1 = c[1], t2 = c[2], t3 = c[3], t4 = c[4];
    float t = t4.w;
    t = fmaf(t, s, t4.z);
    t = fmaf(t, s, t4.y);
    t = fmaf(t, s, t4.x);
    t = fmaf(t, s, t3.w);
    t = fmaf(t, s, t3.z);
    t = fmaf(t, s, t3.y);
    t = fmaf(t, s, t3.x);
    t = fmaf(t, s, t2.w);
    t = fmaf(t, s, t2.z);
    t = fmaf(t, s, t2.y);
    t = fmaf(t, s, t2.x);
    t = fmaf(t, s, h1.z);
    t = fmaf(t, s, h1.x);
    t = fmaf(t, s, h0.z);
    return fmaf(t, s, h0.x);
  }
};

// 2^e for -126 <= e <= 127 (exact, no division)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// Level j of one panel: the warp's lanes take its m_j p subnodes in turn.
// (Tx, Ty) is the target relative to the panel's reference node.
template <class A>
__device__ __forceinline__ void level_sums(const DyadicArgs& a, const float4* __restrict__ tab, int ip, int j,
                                           typename A::V Tx, typename A::V Ty, int lane, typename A::Acc& s_acc,
                                           typename A::Acc& d_acc) {
  using V = typename A::V;
  const int m = 1 << j, n = m * a.p;
  const int64_t q0 = a.q_off[j - 1] + (int64_t)ip * n;
  const float scale = (float)(1 << (2 * (j - 1)));  // 4^{j-1}
  const V xs = A::scale(A::make(a.inv_delta.x, a.inv_delta.y), scale);
  const float range = a.range1f * pow2f(1 - j);
  const float r2max = range * range * 1.0001f;
  for (int u = lane; u < n; u += 32) {
    const int64_t q = q0 + u;
    const float4 rr = __ldg(a.rel + q);
    const V dx = A::sub(Tx, A::make(rr.x, rr.y)), dy = A::sub(Ty, A::make(rr.z, rr.w));
    const float dxh = A::hi(dx), dyh = A::hi(dy);
    if (dxh * dxh + dyh * dyh > r2max) continue;  // single-precision prefilter
    const V xv = A::mul(A::dot2(dx, dx, dy, dy), xs);
    const float xh = A::hi(xv);
    if (!(xh < (float)kDyPieces)) continue;
    // floor(xh) for 0 <= xh < 2^22 without conversion instructions: adding
    // 2^23 rounded down leaves floor(xh) in the low mantissa bits
    const float fl = __fadd_rd(fmaxf(xh, 0.f), 8388608.f);
    const int k = __float_as_int(fl) - 0x4B000000;
    const V s = A::sub(xv, A::make(__fsub_rn(fl, 8388608.f) + 0.5f, 0.f));
    if (a.sig_w) {
      const float2 sw = __ldg(a.sig_w + q);
      A::fma(s_acc, A::poly(tab + k * kDyTabVec, s), A::make(sw.x, sw.y));
    }
    if (a.mu) {
      const float4 nn = __ldg(a.nw + q);
      const float2 mu = __ldg(a.mu + q);
      const V h = A::poly(tab + (kDyPieces + k) * kDyTabVec, s);
      const V dot = A::dot2(dx, A::make(nn.x, nn.y), dy, A::make(nn.z, nn.w));
      A::fma(d_acc, A::mul(h, dot), A::scale(A::make(mu.x, mu.y), scale));
    }
  }
}

// One warp per target of the near list (every target within the band, which
// is the level-1 range, of the boundary).  The lanes first cull the panels of
// the 3x3 hash cells around the target (each lane one panel: how many levels
// reach the target), then the warp walks the surviving panels together.
template <class A>
__global__ void __launch_bounds__(kDyThreads, 4) dyadic_kernel(const __grid_constant__ DyadicArgs a,
                                                            const int2* __restrict__ list,
                                                            const int* __restrict__ count) {
  using V = typename A::V;
  __shared__ float4 tab[2 * kDyPieces * kDyTabVec];
  for (int k = threadIdx.x; k < 2 * kDyPieces * kDyTabVec; k += blockDim.x) tab[k] = __ldg(a.tab + k);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int n_near = *count;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int idx = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); idx < n_near; idx += warps) {
    const int64_t i = list[idx].x;
    // the target as df64 (integer conversion): FP64 runs at 1/58 of the FP32
    // rate on this part, so the per-target work avoids it
    const dd X = dd_from_double(a.txy[2 * i]), Y = dd_from_double(a.txy[2 * i + 1]);
    // cell index in single precision (the cells carry a relative slack of
    // 1e-4 for this), clamped before the integer conversion
    const float ux = (X.hi - a.hx0) * a.inv_hh, uy = (Y.hi - a.hy0) * a.inv_hh;
    const int cx = (int)fminf(fmaxf(floorf(ux), -2.f), (float)a.hnx + 1.f);
    const int cy = (int)fminf(fmaxf(floorf(uy), -2.f), (float)a.hny + 1.f);
    typename A::Acc s_acc = A::zero(), d_acc = A::zero();
    const int xa = max(cx - 1, 0), xb = min(cx + 1, a.hnx - 1);
    for (int yy = max(cy - 1, 0); yy <= min(cy + 1, a.hny - 1) && xa <= xb; ++yy) {
      // the cells xa..xb of row yy hold a contiguous run of panels
      const int k0 = a.cell_start[yy * a.hnx + xa], k1 = a.cell_start[yy * a.hnx + xb + 1];
      for (int base = k0; base < k1; base += 32) {
        const int k = base + lane;
        int ip = 0, reach = 0;
        dd tdx = dd{0.f, 0.f}, tdy = dd{0.f, 0.f};
        if (k < k1) {
          ip = a.cell_panel[k];
          const float4 r = __ldg(a.ref_dd + ip);
          tdx = dd_sub(X, dd{r.x, r.y});
          tdy = dd_sub(Y, dd{r.z, r.w});
          const float d = sqrtf(tdx.hi * tdx.hi + tdy.hi * tdy.hi) - a.panel_rad[ip];
          for (int j = 1; j <= a.levels; ++j) {
            if (d > a.range1f * pow2f(1 - j) * 1.0001f) break;  // ranges shrink with j
            reach = j;
          }
        }
        const V Tx = A::from_dd(tdx), Ty = A::from_dd(tdy);
        unsigned mask = __ballot_sync(0xffffffffu, reach > 0);
        while (mask) {
          const int src = __ffs(mask) - 1;
          mask &= mask - 1;
          const int pp = __shfl_sync(0xffffffffu, ip, src), pr = __shfl_sync(0xffffffffu, reach, src);
          const V px = A::shfl(Tx, src), py = A::shfl(Ty, src);
          for (int j = 1; j <= pr; ++j) level_sums<A>(a, tab, pp, j, px, py, lane, s_acc, d_acc);
        }
      }
    }
    const V s_sum = A::warp_sum(s_acc), d_sum = A::warp_sum(d_acc);
    if (lane == 0) {
      if (a.out_s && a.sig_w) a.out_s[i] += A::to_double(A::mul(s_sum, A::make(a.inv_4pi.x, a.inv_4pi.y)));
      if (a.out_d && a.mu) a.out_d[i] += A::to_double(A::mul(d_sum, A::make(a.dcoef.x, a.dcoef.y)));
    }
  }
}

// ---- host: tables of F and H ----

long double e1_host(long double x) {
  const long double gamma = 0.577215664901532860606512090082402431L;
  if (x <= 2.0L) {
    long double term = 1.0L, sum = 0.0L;
    for (int k = 1; k < 60; ++k) {
      term *= -x / k;
      sum += term / k;  // sum_{k>=1} (-1)^k x^k / (k k!)
    }
    return -gamma - logl(x) - sum;
  }
  // continued fraction (Abramowitz & Stegun 5.1.22), modified Lentz
  const long double tiny = 1e-300L;
  long double b = x + 1.0L, c = 1.0L / tiny, d = 1.0L / b, h = d;
  for (int i = 1; i < 500; ++i) {
    const long double an = -(long double)i * i;
    b += 2.0L;
    d = 1.0L / (an * d + b);
    c = b + an / c;
    const long double del = c * d;
    h *= del;
    if (fabsl(del - 1.0L) < 1e-19L) break;
  }
  return h * expl(-x);
}

// sum_{k>=1} (-1)^{k+1} x^k / (k k!)
long double ein_host(long double x) {
  long double term = 1.0L, sum = 0.0L;
  for (int k = 1; k < 80; ++k) {
    term *= -x / k;
    sum -= term / k;
  }
  return sum;
}

// 4 pi F(x) = E1(x/4) - E1(x); small x through Ein to avoid cancellation
long double f4pi_host(long double x) {
  if (x <= 8.0L) return logl(4.0L) + ein_host(0.25L * x) - ein_host(x);
  return e1_host(0.25L * x) - e1_host(x);
}

long double h_host(long double x) {
  if (x < 1e-12L) return 0.75L - 15.0L / 32.0L * x;
  return (expm1l(-0.25L * x) - expm1l(-x)) / x;
}

// Chebyshev interpolation of g on [k, k+1] at degree deg, as monomials in
// s = x - k - 1/2 (coef[k][0..deg], zero above deg); returns the largest error
// of the double coefficients on a fine grid over all pieces.
template <class G>
double fit_table(G g, int deg, std::vector<double>& coef) {
  const long double pi = 3.141592653589793238462643383279502884L;
  coef.assign((size_t)kDyPieces * (kDyMaxDeg + 1), 0.0);
  double err = 0.0;
  const int n = deg + 1;
  for (int k = 0; k < kDyPieces; ++k) {
    std::vector<long double> fx(n), cheb(n, 0.0L), mono(n, 0.0L);
    for (int j = 0; j < n; ++j) fx[j] = g(k + 0.5L + 0.5L * cosl(pi * (j + 0.5L) / n));
    for (int m = 0; m < n; ++m) {
      long double s = 0;
      for (int j = 0; j < n; ++j) s += fx[j] * cosl(pi * m * (j + 0.5L) / n);
      cheb[m] = s * (m == 0 ? 1.0L : 2.0L) / n;
    }
    // Chebyshev series in u = 2 s -> monomials in u -> monomials in s
    std::vector<long double> tm(n, 0.0L), tk(n, 0.0L), tn(n);
    tm[0] = 1.0L;
    if (n > 1) tk[1] = 1.0L;
    mono[0] += cheb[0];
    if (n > 1)
      for (int i = 0; i < n; ++i) mono[i] += cheb[1] * tk[i];
    for (int m = 1; m + 1 < n; ++m) {
      for (int i = 0; i < n; ++i) tn[i] = (i ? 2.0L * tk[i - 1] : 0.0L) - tm[i];
      for (int i = 0; i < n; ++i) mono[i] += cheb[m + 1] * tn[i];
      tm = tk;
      tk = tn;
    }
    double* cd = &coef[(size_t)k * (kDyMaxDeg + 1)];
    long double sc = 1.0L;
    for (int i = 0; i < n; ++i) {
      cd[i] = (double)(mono[i] * sc);
      sc *= 2.0L;
    }
    for (int j = 0; j <= 40; ++j) {
      const double s = -0.5 + j / 40.0;
      double acc = cd[n - 1];
      for (int i = n - 2; i >= 0; --i) acc = acc * s + cd[i];
      err = std::max(err, (double)fabsl((long double)acc - g(k + 0.5L + s)));
    }
  }
  return err;
}

// Device layout of one piece (kDyTabVec float4): c0, c1, c2, c3 as (hi, lo)
// pairs, then c4..c15 rounded to float.  Returns the largest error of the
// packed polynomial (the form the kernels evaluate, in long double) against g.
template <class G>
double pack_table(G g, const std::vector<double>& coef, float4* out) {
  double err = 0.0;
  for (int k = 0; k < kDyPieces; ++k) {
    const double* cd = &coef[(size_t)k * (kDyMaxDeg + 1)];
    float v[4 * kDyTabVec];
    long double c[kDyMaxDeg + 1];
    for (int i = 0; i < 4; ++i) {
      const float h = (float)cd[i];
      const float l = (float)(cd[i] - (double)h);
      v[2 * i] = h;
      v[2 * i + 1] = l;
      c[i] = (long double)h + (long double)l;
    }
    for (int i = 4; i <= kDyMaxDeg; ++i) {
      v[4 + i] = (float)cd[i];
      c[i] = (long double)v[4 + i];
    }
    for (int q = 0; q < kDyTabVec; ++q)
      out[k * kDyTabVec + q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    for (int j = 0; j <= 40; ++j) {
      const long double s = -0.5L + j / 40.0L;
      long double acc = c[kDyMaxDeg];
      for (int i = kDyMaxDeg - 1; i >= 0; --i) acc = acc * s + c[i];
      err = std::max(err, (double)fabsl(acc - g(k + 0.5L + s)));
    }
  }
  return err;
}

}  // namespace

lp_status setup_dyadic(Plan& P, int levels) {
  if (levels <= 0 || P.nb == 0) return LP_OK;
  if (levels > kMaxDyLevels) return LP_ERR_ARG;
  P.dy_levels = levels;
  // tables: the lowest degree (from 10) whose fit error is below 4e-16
  // (F <= 0.11, H <= 0.75; the double-coefficient floor is ~2e-16, reached
  // at degree 12); long double is slow on some hosts, so few fits
  std::vector<double> cf, ch;
  for (P.dy_deg_f = 10; P.dy_deg_f < kDyMaxDeg; ++P.dy_deg_f)
    if (fit_table(f4pi_host, P.dy_deg_f, cf) < 4e-16) break;
  if (P.dy_deg_f == kDyMaxDeg) fit_table(f4pi_host, kDyMaxDeg, cf);
  for (P.dy_deg_h = 10; P.dy_deg_h < kDyMaxDeg; ++P.dy_deg_h)
    if (fit_table(h_host, P.dy_deg_h, ch) < 4e-16) break;
  if (P.dy_deg_h == kDyMaxDeg) fit_table(h_host, kDyMaxDeg, ch);
  std::vector<float4> tab((size_t)2 * kDyPieces * kDyTabVec);
  const double ef = pack_table(f4pi_host, cf, tab.data());
  const double eh = pack_table(h_host, ch, tab.data() + (size_t)kDyPieces * kDyTabVec);
  P.dy_err = std::max(ef / (4.0 * 3.14159265358979323846), eh);
  auto dalloc_ = [&](void** ptr, size_t bytes) {
    if (cudaMalloc(ptr, bytes) != cudaSuccess) return false;
    P.device_bytes += bytes;
    return true;
  };
  if (!dalloc_((void**)&P.d_dy_tab, tab.size() * sizeof(float4))) return LP_ERR_NOMEM;
  cudaMemcpy(P.d_dy_tab, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice);
  // Gauss-Legendre weights of the panel order (nodes are the plan's tau)
  std::vector<double> tau(P.p), wgl(P.p);
  gauss_legendre(P.p, tau.data(), wgl.data());
  // per-panel radius about the reference node (for the range test)
  std::vector<double> hxy(P.nb * 2), href(P.n_panels * 2), rad(P.n_panels, 0.0);
  std::vector<float> radf(P.n_panels);
  std::vector<float4> refdd(P.n_panels);
  cudaMemcpy(hxy.data(), P.d_bxy, hxy.size() * sizeof(double), cudaMemcpyDeviceToHost);
  cudaMemcpy(href.data(), P.d_geo_ref, href.size() * sizeof(double), cudaMemcpyDeviceToHost);
  for (int64_t ip = 0; ip < P.n_panels; ++ip) {
    for (int i = 0; i < P.p; ++i) {
      const double* q = &hxy[2 * (ip * P.p + i)];
      rad[ip] = std::max(rad[ip], std::hypot(q[0] - href[2 * ip], q[1] - href[2 * ip + 1]));
    }
    rad[ip] *= 1.05;  // the interpolant between nodes bulges slightly
    radf[ip] = (float)rad[ip];
    const float rx = (float)href[2 * ip], ry = (float)href[2 * ip + 1];
    refdd[ip] = make_float4(rx, (float)(href[2 * ip] - rx), ry, (float)(href[2 * ip + 1] - ry));
  }
  // panel hash: reference nodes into cells of side >= range1 + max radius
  {
    const double range1 = 12.0 * std::sqrt(P.delta1);
    double rmax = 0.0, lo0 = href[0], hi0 = href[0], lo1 = href[1], hi1 = href[1];
    for (int64_t ip = 0; ip < P.n_panels; ++ip) {
      rmax = std::max(rmax, rad[ip]);
      lo0 = std::min(lo0, href[2 * ip]);
      hi0 = std::max(hi0, href[2 * ip]);
      lo1 = std::min(lo1, href[2 * ip + 1]);
      hi1 = std::max(hi1, href[2 * ip + 1]);
    }
    double hc = (range1 + rmax) * (1.0 + 1e-4);  // slack for the kernel's FP32 cell index
    int nx = (int)std::ceil((hi0 - lo0) / hc) + 3, ny = (int)std::ceil((hi1 - lo1) / hc) + 3;
    while ((int64_t)nx * ny > (int64_t)1 << 22) {  // bound the table for tiny deltas
      hc *= 2.0;
      nx = (int)std::ceil((hi0 - lo0) / hc) + 3;
      ny = (int)std::ceil((hi1 - lo1) / hc) + 3;
    }
    P.dy_hh = hc;
    P.dy_hx0 = lo0 - hc;
    P.dy_hy0 = lo1 - hc;
    P.dy_hnx = nx;
    P.dy_hny = ny;
    std::vector<int> start((size_t)nx * ny + 1, 0), cell(P.n_panels), panel(P.n_panels);
    for (int64_t ip = 0; ip < P.n_panels; ++ip) {
      int cx = (int)std::floor((href[2 * ip] - P.dy_hx0) / hc);
      int cy = (int)std::floor((href[2 * ip + 1] - P.dy_hy0) / hc);
      cx = std::min(std::max(cx, 0), nx - 1);
      cy = std::min(std::max(cy, 0), ny - 1);
      cell[ip] = cy * nx + cx;
      start[cell[ip] + 1]++;
    }
    for (size_t c = 0; c + 1 < start.size(); ++c) start[c + 1] += start[c];
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (int64_t ip = 0; ip < P.n_panels; ++ip) panel[fill[cell[ip]]++] = (int)ip;
    if (!dalloc_((void**)&P.d_dy_cell_start, start.size() * sizeof(int)) ||
        !dalloc_((void**)&P.d_dy_cell_panel, std::max<size_t>(panel.size(), 1) * sizeof(int)))
      return LP_ERR_NOMEM;
    cudaMemcpy(P.d_dy_cell_start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(P.d_dy_cell_panel, panel.data(), panel.size() * sizeof(int), cudaMemcpyHostToDevice);
  }
  int64_t total = 0;
  for (int j = 1; j <= levels; ++j) {
    P.dy_q_off[j - 1] = total;
    total += P.n_panels * ((int64_t)1 << j) * P.p;
  }
  P.dy_nq = total;
  if (!dalloc_((void**)&P.d_dy_rel, total * sizeof(float4)) ||
      !dalloc_((void**)&P.d_dy_nw, total * sizeof(float4)) ||
      !dalloc_((void**)&P.d_dy_sig, total * sizeof(float2)) ||
      !dalloc_((void**)&P.d_dy_mu, total * sizeof(float2)) ||
      !dalloc_((void**)&P.d_dy_rad, P.n_panels * sizeof(float)) ||
      !dalloc_((void**)&P.d_dy_ref, P.n_panels * sizeof(float4)) ||
      !dalloc_((void**)&P.d_dy_wgl, P.p * sizeof(double)))
    return LP_ERR_NOMEM;
  cudaMemcpy(P.d_dy_rad, radf.data(), radf.size() * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(P.d_dy_ref, refdd.data(), refdd.size() * sizeof(float4), cudaMemcpyHostToDevice);
  cudaMemcpy(P.d_dy_wgl, wgl.data(), wgl.size() * sizeof(double), cudaMemcpyHostToDevice);
  for (int j = 1; j <= levels; ++j) {
    const int m = 1 << j;
    const int64_t nq = P.n_panels * (int64_t)m * P.p;
    dyadic_geom_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, P.stream>>>(
        P.d_geo_coef, P.d_tau, P.d_dy_wgl, (int)P.n_panels, P.p, m, P.d_dy_rel + P.dy_q_off[j - 1],
        P.d_dy_nw + P.dy_q_off[j - 1]);
  }
  if (cudaStreamSynchronize(P.stream) != cudaSuccess) return LP_ERR_CUDA;
  return LP_OK;
}

// Densities at the subnodes after lp_single_layer (kind 0: sigma w) or
// lp_double_layer (kind 1: mu).
void launch_dyadic_dens(const Plan& P, int kind, cudaStream_t s) {
  for (int j = 1; j <= P.dy_levels; ++j) {
    const int m = 1 << j;
    const int64_t nq = P.n_panels * (int64_t)m * P.p;
    dyadic_dens_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(
        kind == 0 ? P.d_sigma_coef : P.d_mu_coef, kind == 0 ? P.d_sigma_ref : P.d_mu_ref, P.d_tau, P.d_dy_wgl,
        P.d_geo_coef, (int)P.n_panels, P.p, m, kind == 0, (kind == 0 ? P.d_dy_sig : P.d_dy_mu) + P.dy_q_off[j - 1]);
    ++P.launches;
  }
}

void launch_dyadic(const Plan& P, int64_t nt, const double* txy, double* S, double* D, const int2* list,
                   const int* count, cudaStream_t s) {
  if (P.dy_levels <= 0 || nt <= 0 || (!S && !D)) return;
  DyadicArgs a{};
  a.txy = txy;
  a.out_s = P.have_sigma ? S : nullptr;
  a.out_d = P.have_mu ? D : nullptr;
  a.sig_w = P.have_sigma && S ? P.d_dy_sig : nullptr;
  a.mu = P.have_mu && D ? P.d_dy_mu : nullptr;
  a.rel = P.d_dy_rel;
  a.nw = P.d_dy_nw;
  a.tab = P.d_dy_tab;
  a.levels = P.dy_levels;
  for (int j = 0; j < P.dy_levels; ++j) a.q_off[j] = P.dy_q_off[j];
  a.ref_dd = P.d_dy_ref;
  a.panel_rad = P.d_dy_rad;
  a.p = P.p;
  a.hx0 = (float)P.dy_hx0;
  a.hy0 = (float)P.dy_hy0;
  a.inv_hh = (float)(1.0 / P.dy_hh);
  a.hnx = P.dy_hnx;
  a.hny = P.dy_hny;
  a.cell_start = P.d_dy_cell_start;
  a.cell_panel = P.d_dy_cell_panel;
  a.range1f = (float)(12.0 * std::sqrt(P.delta1));
  auto split = [](double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  };
  a.inv_delta = split(1.0 / P.delta1);
  a.inv_4pi = split(1.0 / (4.0 * 3.14159265358979323846));
  a.dcoef = split(1.0 / (2.0 * 3.14159265358979323846 * P.delta1));
  a.status = P.d_status;
  // one warp per near target; the near count is on the device, so the grid
  // covers every target with a grid-stride loop (at most 152 x 8 blocks)
  const int64_t warps_per_block = kDyThreads / 32;
  const unsigned blocks =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>((nt + warps_per_block - 1) / warps_per_block, 152 * 8));
  ++P.launches;
  if (P.precision == LP_FP64)
    dyadic_kernel<SumDD><<<blocks, kDyThreads, 0, s>>>(a, list, count);
  else
    dyadic_kernel<SumF><<<blocks, kDyThreads, 0, s>>>(a, list, count);
}

}  // namespace lpg
