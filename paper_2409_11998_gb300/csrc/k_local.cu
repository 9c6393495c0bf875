// Local part (Sec. 4): per target, closest boundary point (Sec. 2.2:
// nearest node, then Newton on the panel polynomial), the tangent-line frame
// (eq. tanparams) and the asymptotic expansions of the local single-layer,
// double-layer and volume heat potentials, added onto the smooth part.
//
// Conventions (forced by the definitions of Sec. 1-2):
//   D[mu] differentiates in the source point, so D[1] = -1 inside; with it
//   the printed local D expansion changes sign.  The local S kernel is
//   positive, so the printed local S expansion changes sign.  In the volume
//   expansion, with eta the inward normal and kappa > 0 for convex
//   boundaries, the delta^{3/2} term reads (2 f_eta - kappa f).
//
// The passes are templated on the arithmetic type of the expansions: double
// for FP64 plans, float for FP32 plans (tolerance >= 1e-6; coordinates
// relative to the panel's reference node).  Both take the single-precision
// nearest node and foot search finished in double precision (panel_foot), so
// the distance and the side of the boundary are resolved to rounding.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "df64.cuh"
#include "lp_internal.cuh"

namespace cg = cooperative_groups;

namespace lpg {

namespace {


// d^j/dt^j of ref_s + sum_k c_s[k] P_k(t), j = 0..ND, for NS series sharing
// one recurrence.  The stored coefficients are c_k / k!, paired with
// Q_k = k! P_k, which obey the division-free recurrence
// Q_{k+1} = (2k+1) t Q_k - k^2 Q_{k-1}; differentiating j times gives
// Q_{k+1}^(j) = (2k+1) (t Q_k^(j) + j Q_k^(j-1)) - k^2 Q_{k-1}^(j).
template <int ND, int NS, typename T>
__device__ __forceinline__ void legendre_jets(const T* const* c, const T* ref, int p, T t,
                                              T (*out)[ND + 1]) {
  T qm[ND + 1], qk[ND + 1];
#pragma unroll
  for (int j = 0; j <= ND; ++j) {
    qm[j] = 0;
    qk[j] = (j == 0) ? T(1) : T(0);
  }
#pragma unroll
  for (int q = 0; q < NS; ++q) {
#pragma unroll
    for (int j = 0; j <= ND; ++j) out[q][j] = 0;
    out[q][0] = ref[q] + c[q][0];
  }
  for (int k = 0; k + 1 < p; ++k) {
    const T a = T(2 * k + 1), b = T(k) * T(k);
#pragma unroll
    for (int j = ND; j >= 0; --j) {
      T prev = j ? qk[j - 1] : T(0);
      T qn = a * fma(t, qk[j], T(j) * prev) - b * qm[j];
      qm[j] = qk[j];
      qk[j] = qn;
    }
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const T ck = c[q][k + 1];
#pragma unroll
      for (int j = 0; j <= ND; ++j) out[q][j] = fma(ck, qk[j], out[q][j]);
    }
  }
}

// legendre_jets in double-float arithmetic (the FP32 units; GB300's FP64 rate
// is 1/58 of theirs): the same recurrence, the stored coefficients as df64
// pairs, the sums accumulated with error-free transforms; out = ref + sum in
// double.  ~48 bits: the fourth derivatives, which enter at delta^2 and
// reach ~8e3 at the starfish's concave tips, keep ~1e-12 relative.
template <int ND, int NS>
__device__ __forceinline__ void legendre_jets_dd(const float2* const* c, const double* ref, int p, double t,
                                                 double (*out)[ND + 1]) {
  const dd td = dd_from_double(t);
  dd qm[ND + 1], qk[ND + 1];
  dd_acc acc[NS][ND + 1];
#pragma unroll
  for (int j = 0; j <= ND; ++j) {
    qm[j] = dd{0.f, 0.f};
    qk[j] = dd{j == 0 ? 1.f : 0.f, 0.f};
  }
#pragma unroll
  for (int q = 0; q < NS; ++q) {
#pragma unroll
    for (int j = 0; j <= ND; ++j) acc[q][j] = dd_acc{0.f, 0.f};
    acc[q][0] = dd_acc{c[q][0].x, c[q][0].y};
  }
  for (int k = 0; k + 1 < p; ++k) {
    const float a = (float)(2 * k + 1), b = (float)(k * k);
#pragma unroll
    for (int j = ND; j >= 0; --j) {
      dd tq = dd_mul(td, qk[j]);
      if (j) tq = dd_add(tq, dd_mul_f(qk[j - 1], (float)j));
      const dd qn = dd_sub(dd_mul_f(tq, a), dd_mul_f(qm[j], b));
      qm[j] = qk[j];
      qk[j] = qn;
    }
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const float2 ck = c[q][k + 1];
#pragma unroll
      for (int j = 0; j <= ND; ++j) acc_fma(acc[q][j], dd{ck.x, ck.y}, qk[j]);
    }
  }
#pragma unroll
  for (int q = 0; q < NS; ++q)
#pragma unroll
    for (int j = 0; j <= ND; ++j) out[q][j] = (j == 0 ? ref[q] : 0.0) + dd_to_double(acc_value(acc[q][j]));
}

// Foot of the perpendicular: panel, parameter, and the offset from the target
// to the foot (gx, gy) with its squared length, always evaluated in double
// precision so that the side of the boundary and the distance are exact to
// rounding whatever the arithmetic type of the expansions.
struct Foot {
  int panel;
  double t, d2, gx, gy;
  double s2;       // |gamma'|^2 at the last parameter
  bool converged;  // the double-precision phase met its stopping rule, or its
                   // last step was a gradient step (flat distance near a
                   // centre of curvature: slow, but downhill to the foot)
};

// Newton for the foot on panel ip from parameter t: a single-precision phase
// in coordinates relative to the panel's reference node (it ends within
// single-precision noise of the root, or after 16 steps), then double-
// precision steps until one moves t by less than 1e-6 -- Newton's quadratic
// convergence leaves ~1e-12 in t after it -- with the foot offset at the last
// parameter from the second-order Taylor expansion of that step (error ~|dt|^3
// times the third derivative), so that the distance of on-boundary targets
// and the side of the boundary are resolved to rounding.  Twenty double
// steps without a step below 1e-6, the last of them a Newton step proper,
// leave `converged` false.
__device__ Foot panel_foot(const LocalArgs& a, int ip, double t, double x, double y) {
  const size_t off = (size_t)(2 * ip) * a.p;
  const double rx = a.geo_ref[2 * ip], ry = a.geo_ref[2 * ip + 1];
  {
    const float* c32[2] = {a.geo_coef32 + off, a.geo_coef32 + off + a.p};
    const float zero2[2] = {0.f, 0.f};
    const float xr = (float)(x - rx), yr = (float)(y - ry);
    float tf = (float)t;
    for (int it = 0; it < 16; ++it) {
      float J[2][3];
      legendre_jets<2, 2, float>(c32, zero2, a.p, tf, J);
      float gx = J[0][0] - xr, gy = J[1][0] - yr;
      float f = gx * J[0][1] + gy * J[1][1];
      float s2 = J[0][1] * J[0][1] + J[1][1] * J[1][1];
      float fp = s2 + gx * J[0][2] + gy * J[1][2];
      if (fp < 0.1f * s2) fp = s2;
      float tn = fminf(1.f, fmaxf(-1.f, tf - f / fp));
      float dt = tn - tf;
      tf = tn;
      if (fabsf(dt) < 2e-7f) break;
    }
    if (tf == tf) t = (double)tf;  // keep the node start if the phase failed
  }
  const float2* cdd[2] = {a.geo_coef_dd + off, a.geo_coef_dd + off + a.p};
  const double ref[2] = {rx, ry};
  Foot r;
  r.panel = ip;
  r.converged = false;
  for (int it = 0; it < 20; ++it) {
    double J[2][3];
    legendre_jets_dd<2, 2>(cdd, ref, a.p, t, J);
    const double gx = J[0][0] - x, gy = J[1][0] - y;
    const double f = gx * J[0][1] + gy * J[1][1];
    const double s2 = J[0][1] * J[0][1] + J[1][1] * J[1][1];
    double fp = s2 + gx * J[0][2] + gy * J[1][2];
    const bool gradient = fp < 0.1 * s2;
    if (gradient) fp = s2;
    const double tn = fmin(1.0, fmax(-1.0, t - f / fp));
    const double dt = tn - t;
    t = tn;
    r.gx = gx + dt * (J[0][1] + 0.5 * dt * J[0][2]);
    r.gy = gy + dt * (J[1][1] + 0.5 * dt * J[1][2]);
    r.s2 = s2;
    r.converged = gradient;
    if (fabs(dt) < 1e-6) {
      r.converged = true;
      break;
    }
  }
  r.t = t;
  r.d2 = r.gx * r.gx + r.gy * r.gy;
  return r;
}

template <typename T>
__device__ __forceinline__ const T* coef_ptr(const double* c64, const float* c32);
template <>
__device__ __forceinline__ const double* coef_ptr<double>(const double* c64, const float*) { return c64; }
template <>
__device__ __forceinline__ const float* coef_ptr<float>(const double*, const float* c32) { return c32; }

// Coefficients of xi^1..xi^4 of F(s(xi)) with F(s) = sum_{k>=1} F[k] s^k and
// s(xi) = sum_{k>=1} c[k] xi^k.
template <typename T>
__device__ void compose4(const T* F, const T* c, T* o) {
  o[1] = F[1] * c[1];
  o[2] = F[1] * c[2] + F[2] * c[1] * c[1];
  o[3] = F[1] * c[3] + T(2) * F[2] * c[1] * c[2] + F[3] * c[1] * c[1] * c[1];
  o[4] = F[1] * c[4] + F[2] * (c[2] * c[2] + T(2) * c[1] * c[3]) + T(3) * F[3] * c[1] * c[1] * c[2] +
         F[4] * c[1] * c[1] * c[1] * c[1];
}

// Local volume integral over the quadrant of a convex right-angle corner
// (the expansions of Sec. 4 assume a smooth boundary) for the quadratic f of the jet J, at distances ea, eb from the edges
// with inward normals n1, n2: the heat kernel separates along n1 and n2, so
// the integrand at time t is the product of the one-dimensional moments
// M_k(e) = int_{-e}^inf s^k g_t(s) ds of the Gaussian g_t of variance 2t,
//   M0 = erfc(-e / 2 sqrt t) / 2, M1 = sqrt(t / pi) exp(-e^2 / 4t),
//   M2 = 2t (M0 - e g_t(e)),
// contracted with f and its derivatives along n1, n2; the time integral on
// the plan's graded nodes.  Evaluated by a whole warp (every lane calls it,
// with the same target): lane l takes the nodes l, l + 32, ..., and the
// partial sums are combined by shuffles; every lane returns the total.
// The integrand is evaluated in single precision for both plan precisions
// and summed in double: the quadrant term is of size delta f (the heat
// kernel's mass over the quadrant), so single-precision rounding perturbs V
// by ~1e-7 delta |f|, far below the FP64 plans' tolerance, while the FP64
// erfc and exp cost ten times the rest of the local pass.
__device__ double corner_volume_warp(const LocalArgs& a, const double* J, const double* c, double ea, double eb,
                                     int lane) {
  const float f = (float)J[0];
  const float d1 = (float)(J[1] * c[2] + J[2] * c[3]), d2 = (float)(J[1] * c[4] + J[2] * c[5]);
  const float h11 = (float)(J[3] * c[2] * c[2] + 2.0 * J[4] * c[2] * c[3] + J[5] * c[3] * c[3]);
  const float h22 = (float)(J[3] * c[4] * c[4] + 2.0 * J[4] * c[4] * c[5] + J[5] * c[5] * c[5]);
  const float h12 = (float)(J[3] * c[2] * c[4] + J[4] * (c[2] * c[5] + c[3] * c[4]) + J[5] * c[3] * c[5]);
  const float inv_sqrt_pi = 0.5641895835f;
  const float eaf = (float)ea, ebf = (float)eb;
  double v = 0.0;
  for (int k = lane; k < kCornerQuad; k += 32) {
    const float t = (float)a.corner_q[k], st = sqrtf(t), is = 1.0f / st;
    const float xa = eaf * is, xb = ebf * is;  // e / sqrt t
    const float ga = expf(-0.25f * xa * xa), gb = expf(-0.25f * xb * xb);
    const float A0 = 0.5f * erfcf(-0.5f * xa), B0 = 0.5f * erfcf(-0.5f * xb);
    const float A1 = st * inv_sqrt_pi * ga, B1 = st * inv_sqrt_pi * gb;
    const float A2 = 2.0f * t * A0 - eaf * A1, B2 = 2.0f * t * B0 - ebf * B1;
    const float I = f * A0 * B0 + d1 * A1 * B0 + d2 * A0 * B1 + 0.5f * h11 * A2 * B0 + h12 * A1 * B1 +
                    0.5f * h22 * A0 * B2;
    v += a.corner_q[kCornerQuad + k] * (double)I;
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double far_volume(const LocalArgs& a, const double* J) {
  // delta f + delta^2/2 lap f (Sec. 4, after eq. vplocO5)
  double v = a.delta * J[0];
  if (a.order >= 5) v += 0.5 * a.delta * a.delta * (J[3] + J[5]);
  return v;
}

// Returns the index of the corner whose quadrant holds the target (its V
// term is then left to the corner pass), or -1.
template <typename T>
__device__ int local_near_one(const LocalArgs& a, int64_t i, int best) {
  const double x = a.txy[2 * i], y = a.txy[2 * i + 1];
  const T dl = (T)a.delta_sd;  // S and D expansions (V uses a.delta)
  const double* J = a.jet ? a.jet + 6 * i : nullptr;
  T vl = 0, sl = 0, dlv = 0;
  bool far = false;
  int corner = -1;
  Foot ft{-1, 0.0, 1e300, 0.0, 0.0, 1.0, true};
  {
    const int p = a.p;
    const int ip0 = best / p;
    ft = panel_foot(a, ip0, a.tau[best - ip0 * p], x, y);
    if (fabs(ft.t) == 1.0) {
      // the foot lies beyond this panel's end: continue on the adjacent panel
      int ip = ((ip0 + (ft.t > 0.0 ? 1 : -1)) % a.n_panels + a.n_panels) % a.n_panels;
      int kb = 0;
      double kd = 1e300;
      for (int k = 0; k < p; ++k) {
        const double* q = a.bxy + 2 * ((size_t)ip * p + k);
        double d2 = (x - q[0]) * (x - q[0]) + (y - q[1]) * (y - q[1]);
        if (d2 < kd) {
          kd = d2;
          kb = k;
        }
      }
      Foot f = panel_foot(a, ip, a.tau[kb], x, y);
      // past the adjacent panel's far end as well: no foot on either panel
      const bool beyond = ft.t > 0.0 ? f.t == 1.0 : f.t == -1.0;
      if (!f.converged || beyond) atomicOr(a.status, kStatusNewton);
      if (f.d2 < ft.d2) ft = f;
    } else if (!ft.converged) {
      atomicOr(a.status, kStatusNewton);
    }
    if (sqrt(ft.d2) >= a.band) far = true;
    // a foot where the parametrisation's speed vanishes (a cusp, a panel of
    // nearly coincident nodes) has no tangent frame: the expansions below
    // divide by that speed
    if (!far && ft.s2 < 1e6 * a.on_tol * a.on_tol) atomicOr(a.status, kStatusNewton);
  }

  if (far) {
    if (J) vl = (T)far_volume(a, J);
  } else {
    const int p = a.p, ip = ft.panel;
    const bool want_s = a.out[1] && a.sig_coef, want_d = a.out[2] && a.mu_coef;
    const T* cgx = coef_ptr<T>(a.geo_coef, a.geo_coef32) + (size_t)(2 * ip) * p;
    // value and four derivatives of x, y (relative to the panel's reference
    // node), sigma, mu at the foot (one recurrence)
    const T* cs[4] = {cgx, cgx + p, want_s ? coef_ptr<T>(a.sig_coef, a.sig_coef32) + (size_t)ip * p : cgx,
                      want_d ? coef_ptr<T>(a.mu_coef, a.mu_coef32) + (size_t)ip * p : cgx};
    const T rs[4] = {T(0), T(0), want_s ? (T)a.sig_ref[ip] : T(0), want_d ? (T)a.mu_ref[ip] : T(0)};
    T JJ[4][5];
    if constexpr (sizeof(T) == 8) {
      // FP64 plans: the jets in double-float (the expansions themselves in double)
      const float2* gdd = a.geo_coef_dd + (size_t)(2 * ip) * p;
      const float2* cd[4] = {gdd, gdd + p, want_s ? a.sig_coef_dd + (size_t)ip * p : gdd,
                             want_d ? a.mu_coef_dd + (size_t)ip * p : gdd};
      const double rd[4] = {0.0, 0.0, want_s ? a.sig_ref[ip] : 0.0, want_d ? a.mu_ref[ip] : 0.0};
      legendre_jets_dd<4, 4>(cd, rd, p, ft.t, JJ);
    } else {
      legendre_jets<4, 4, T>(cs, rs, p, (T)ft.t, JJ);
    }
    const T* X = JJ[0];
    const T* Y = JJ[1];
    const T sp = hypot(X[1], Y[1]);
    const T Tx = X[1] / sp, Ty = Y[1] / sp;
    const T Nx = -Ty, Ny = Tx;  // inward normal of a counter-clockwise curve
    const double rd = sqrt(ft.d2);
    const T r = (T)rd;
    T sgn = 0;
    if (rd > a.on_tol) sgn = (-(ft.gx * (double)Nx + ft.gy * (double)Ny) > 0.0) ? T(1) : T(-1);
    // Taylor coefficients in s = t - t*: xi(s) = sum a_k s^k, eta(s) = sum e_k s^k
    const T fact[5] = {T(1), T(1), T(0.5), T(1.0 / 6.0), T(1.0 / 24.0)};
    T A[5], E[5];
    for (int k = 1; k <= 4; ++k) {
      A[k] = (X[k] * Tx + Y[k] * Ty) * fact[k];
      E[k] = (X[k] * Nx + Y[k] * Ny) * fact[k];
    }
    E[1] = 0;
    // series reversion s(xi)
    T C[5];
    const T i1 = T(1.0) / A[1];
    const T i2 = i1 * i1, i3 = i2 * i1, i5 = i3 * i2, i7 = i5 * i2;
    C[1] = i1;
    C[2] = -A[2] * i3;
    C[3] = (T(2.0) * A[2] * A[2] - A[1] * A[3]) * i5;
    C[4] = (T(5.0) * A[1] * A[2] * A[3] - A[1] * A[1] * A[4] - T(5.0) * A[2] * A[2] * A[2]) * i7;
    T H[5];
    compose4<T>(E, C, H);
    const T kap = T(2.0) * H[2], g3 = T(6.0) * H[3], g4 = T(24.0) * H[4];
    const T c = r / sqrt(dl);
    const T sq = sqrt(dl), d15 = dl * sq, d2 = dl * dl;
    const T Ex = exp(-T(0.25) * c * c) * T(0.56418958354775628695);  // e^{-c^2/4}/sqrt(pi)
    const T Cc = erfc(T(0.5) * c);
    const T c2 = c * c, c3 = c2 * c;
    if (want_s) {
      const T* Sv = JJ[2];
      T F[5], o[5];
      for (int k = 1; k <= 4; ++k) F[k] = Sv[k] * fact[k];
      compose4<T>(F, C, o);
      const T s0 = Sv[0], s1 = o[1], s2 = T(2.0) * o[2];
      const T Aq = c * Cc - T(2.0) * Ex;
      const T Q = T(2.0) * (c2 - T(2.0)) * Ex - c3 * Cc;
      T s = sq * T(0.5) * s0 * Aq + sgn * dl * T(0.25) * c * kap * s0 * Aq;
      if (a.order >= 4)
        s += d15 * (s0 * kap * kap / T(12.0) * (T(2.0) * c3 * Cc - (T(4.0) * c2 + T(1.0)) * Ex) + s2 / T(12.0) * Q);
      if (a.order >= 5)
        s += d2 * sgn * c *
             (kap * kap * kap * s0 / T(16.0) * (T(3.0) * c3 * Cc - (T(6.0) * c2 - T(2.0)) * Ex) +
              (kap * s2 / T(8.0) + s0 * g4 / T(48.0) + s1 * g3 / T(12.0)) * Q);
      sl = -s;
    }
    if (want_d) {
      const T* Mv = JJ[3];
      T F[5], o[5];
      for (int k = 1; k <= 4; ++k) F[k] = Mv[k] * fact[k];
      compose4<T>(F, C, o);
      const T m0 = Mv[0], m1 = o[1], m2 = T(2.0) * o[2], m4 = T(24.0) * o[4];
      const T R1 = T(2.0) * (c2 + T(1.0)) * Ex - c3 * Cc;
      const T R4 = T(2.0) * (c2 + T(4.0)) * Ex - c3 * Cc;
      T s = sgn * T(0.5) * m0 * Cc + sq * T(0.5) * kap * m0 * Ex +
            dl * sgn * (T(0.375) * c * kap * kap * m0 * Ex + T(0.25) * c * m2 * (T(2.0) * Ex - c * Cc));
      if (a.order >= 4)
        s += d15 * (T(5.0 / 16.0) * (c2 - T(2.0)) * kap * kap * kap * m0 * Ex + T(0.25) * g4 * m0 * Ex +
                    T(0.25) * kap * m2 * R1 + g3 * m1 / T(12.0) * R4);
      if (a.order >= 5)
        s += d2 * sgn * c *
             (T(35.0 / 128.0) * kap * kap * kap * kap * m0 * (c2 - T(6.0)) * Ex +
              T(5.0 / 12.0) * g3 * g3 * m0 * Ex + T(0.625) * kap * g4 * m0 * Ex +
              T(5.0) * (kap * kap * m2 / T(16.0) * R1 + kap * g3 * m1 / T(24.0) * R4) +
              m4 / T(48.0) * (c3 * Cc - T(2.0) * (c2 - T(2.0)) * Ex));
      dlv = -s;
    }
    if (J) {
      if (sgn < T(0.0)) {
        atomicOr(a.status, kStatusExteriorBandV);
      } else {
        T Jt[6];
        for (int k = 0; k < 6; ++k) Jt[k] = (T)J[k];
        const T f = Jt[0];
        const T fe = Jt[1] * Nx + Jt[2] * Ny;
        const T fxx = Jt[3] * Tx * Tx + T(2.0) * Jt[4] * Tx * Ty + Jt[5] * Ty * Ty;
        const T fee = Jt[3] * Nx * Nx + T(2.0) * Jt[4] * Nx * Ny + Jt[5] * Ny * Ny;
        // V keeps delta: the c-dependent factors again when refinement
        // evaluates S and D at a smaller delta
        const bool same = a.delta_sd == a.delta;
        const T dv = (T)a.delta;
        const T cv = same ? c : r / sqrt(dv);
        const T d15v = same ? d15 : dv * sqrt(dv), d2v = dv * dv;
        const T Exv = same ? Ex : exp(-T(0.25) * cv * cv) * T(0.56418958354775628695);
        const T Ccv = same ? Cc : erfc(T(0.5) * cv);
        const T c2v = cv * cv, c3v = c2v * cv;
        const T Ef = erf(T(0.5) * cv);
        T v = T(0.25) * dv * (T(2.0) * Ef + T(2.0) * cv * Exv - c2v * Ccv + T(2.0)) * f;
        if (a.order >= 4) v += d15v * ((T(4.0) - T(2.0) * c2v) * Exv + c3v * Ccv) * (T(2.0) * fe - kap * f) / T(12.0);
        if (a.order >= 5) {
          const T c4 = c2v * c2v;
          v += d2v / T(48.0) *
               (Ccv * (T(4.0) * c4 * kap * fe - T(3.0) * (c4 + T(4.0)) * fee + (c4 - T(12.0)) * fxx -
                      T(3.0) * c4 * kap * kap * f) +
                T(2.0) * cv * (c2v - T(2.0)) * Exv * (-T(4.0) * kap * fe + T(3.0) * fee - fxx + T(3.0) * kap * kap * f) +
                T(24.0) * (fxx + fee));
        }
        vl = v;
        // within the band of both edges of a right-angle corner: the
        // quadrant integral replaces the expansion (corner pass)
        if (a.order >= 5)
          for (int q = 0; q < a.n_corners; ++q) {
            const double* c = a.corners + 6 * q;
            const double ea = (x - c[0]) * c[2] + (y - c[1]) * c[3];
            const double eb = (x - c[0]) * c[4] + (y - c[1]) * c[5];
            if (ea > -a.on_tol && eb > -a.on_tol && ea < a.band && eb < a.band) {
              vl = 0;
              corner = q;
              break;
            }
          }
      }
    }
  }
  if (a.out[0]) a.out[0][i] += (double)vl;
  if (a.out[1]) a.out[1][i] += (double)sl;
  if (a.out[2]) a.out[2][i] += (double)dlv;
  return corner;
}

// Pass 1: nearest boundary node among the 3x3 hash cells, by a single-
// precision scan over node coordinates stored relative to their cell origin
// (every squared distance within 2e-5 h^2, h the cell side).  The node only
// seeds the foot search; at the band edge, where a rounding-level error can
// move a target between the near and far branches, the near and far
// expansions agree.  Targets whose nearest node is farther than band + margin
// get the far-field volume term here; the others are appended to a compact
// list for pass 2.  Returns the nearest node for a band candidate, -1 when
// the far-field term was applied.
__device__ int local_classify_one(const LocalArgs& a, int64_t i) {
  // The classification runs for every target, so it avoids FP64 arithmetic
  // (1/58 of the FP32 rate): the cell index from a float product, the offset
  // from the target's own cell corner from one FMA split into floats by
  // integer operations, the neighbouring cells' offsets and the band test
  // in float.  A target within ~1e-7 of the band edge may fall on either
  // side; the local terms there are below e^{-36}.
  const double x = a.txy[2 * i], y = a.txy[2 * i + 1];
  int best = -1;
  float m32 = 3.0e38f;
  if (a.nb > 0) {
    const double dx0 = x - a.hx0, dy0 = y - a.hy0;
    const float ux = dd_from_double(dx0).hi * a.inv_hh32, uy = dd_from_double(dy0).hi * a.inv_hh32;
    if (ux >= 0.f && ux < (float)a.hnx && uy >= 0.f && uy < (float)a.hny) {
      const int cx = min((int)ux, a.hnx - 1), cy = min((int)uy, a.hny - 1);
      const float rx = dd_from_double(fma(-(double)cx, a.hh, dx0)).hi;
      const float ry = dd_from_double(fma(-(double)cy, a.hh, dy0)).hi;
      const int x0c = max(cx - 1, 0), x1c = min(cx + 1, a.hnx - 1);
      const int y0c = max(cy - 1, 0), y1c = min(cy + 1, a.hny - 1);
      int k32 = -1;
      const bool scan = a.cell_near[cy * a.hnx + cx] != 0;  // else every neighbouring cell is empty
      for (int yy = y0c; scan && yy <= y1c; ++yy) {
        const float ty = fmaf(-(float)(yy - cy), a.hh32, ry);
        for (int xx = x0c; xx <= x1c; ++xx) {
          const float tx = fmaf(-(float)(xx - cx), a.hh32, rx);
          const int c = yy * a.hnx + xx;
          const int k1 = a.cell_start[c + 1];
          for (int k = a.cell_start[c]; k < k1; ++k) {
            float2 q = a.cell_xy32[k];
            float dx = tx - q.x, dy = ty - q.y;
            const float d2 = fmaf(dx, dx, dy * dy);
            if (d2 < m32) {
              m32 = d2;
              k32 = k;
            }
          }
        }
      }
      if (k32 >= 0) best = a.cell_node[k32];
    }
  }
  if (best < 0 || sqrtf(m32) - a.margin32 >= a.band32) {
    if (a.out[0] && a.jet) a.out[0][i] += far_volume(a, a.jet + 6 * i);
    return -1;
  }
  return best;
}

__global__ void local_classify_kernel(const __grid_constant__ LocalArgs a, int2* list, int* count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int best = local_classify_one(a, i);
  if (best < 0) return;
  auto g = cg::coalesced_threads();
  int base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(count, (int)g.size());
  base = g.shfl(base, 0);
  list[base + g.thread_rank()] = make_int2((int)i, best);
}

// Batched: one launch over the targets of many plans; list entries are
// (plan, target, nearest node).
__global__ void local_classify_batch_kernel(const LocalArgs* __restrict__ args, const int2* __restrict__ work,
                                            int4* list, int* count) {
  const int2 wk = work[blockIdx.x];
  const LocalArgs& a = args[wk.x];
  int64_t i = (int64_t)wk.y + threadIdx.x;
  if (i >= a.n) return;
  const int best = local_classify_one(a, i);
  if (best < 0) return;
  auto g = cg::coalesced_threads();
  int base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(count, (int)g.size());
  base = g.shfl(base, 0);
  list[base + g.thread_rank()] = make_int4(wk.x, (int)i, best, 0);
}

// Pass 2: closest point, frame and expansions for the listed targets.  A
// target in a corner's quadrant gets its entry marked for pass 3: the
// nearest-node field (no longer needed) becomes -1 - corner.
template <typename T>
__global__ void local_near_kernel(const __grid_constant__ LocalArgs a, int2* __restrict__ list,
                                  const int* __restrict__ count) {
  const int n_near = *count;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n_near; idx += gridDim.x * blockDim.x) {
    const int q = local_near_one<T>(a, list[idx].x, list[idx].y);
    if (q >= 0) list[idx].y = -1 - q;
  }
}

template <typename T>
__global__ void local_near_batch_kernel(const LocalArgs* __restrict__ args, int4* __restrict__ list,
                                        const int* __restrict__ count) {
  const int n_near = *count;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n_near; idx += gridDim.x * blockDim.x) {
    const int4 e = list[idx];
    const int q = local_near_one<T>(args[e.x], e.y, e.z);
    if (q >= 0) list[idx].w = 1 + q;
  }
}

// Pass 3: the quadrant integrals of the marked entries, one warp per target.
// Each warp scans 32 list entries per round (the round count depends only on
// the warp, so every lane takes part in the ballot and the shuffles) and
// evaluates the marked ones one after the other with all its lanes.
__device__ __forceinline__ void corner_entry(int2 e, int& plan, int& t, int& q) {
  plan = 0;
  t = e.x;
  q = e.y < 0 ? -1 - e.y : -1;
}
__device__ __forceinline__ void corner_entry(int4 e, int& plan, int& t, int& q) {
  plan = e.x;
  t = e.y;
  q = e.w > 0 ? e.w - 1 : -1;
}

template <typename E>
__device__ void corner_pass(const LocalArgs* one, const LocalArgs* args, const E* __restrict__ list,
                            const int* __restrict__ count) {
  const int n = *count;
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int base = warp * 32; base < n; base += nwarps * 32) {
    int plan = 0, t = 0, q = -1;
    if (base + lane < n) corner_entry(list[base + lane], plan, t, q);
    unsigned m = __ballot_sync(0xffffffffu, q >= 0);
    while (m != 0u) {
      const int src = __ffs(m) - 1;
      m &= m - 1u;
      const int pp = __shfl_sync(0xffffffffu, plan, src);
      const int tt = __shfl_sync(0xffffffffu, t, src);
      const int qq = __shfl_sync(0xffffffffu, q, src);
      const LocalArgs& a = one ? *one : args[pp];
      const double x = a.txy[2 * (int64_t)tt], y = a.txy[2 * (int64_t)tt + 1];
      const double* c = a.corners + 6 * qq;
      const double ea = (x - c[0]) * c[2] + (y - c[1]) * c[3];
      const double eb = (x - c[0]) * c[4] + (y - c[1]) * c[5];
      const double v = corner_volume_warp(a, a.jet + 6 * (int64_t)tt, c, fmax(ea, 0.0), fmax(eb, 0.0), lane);
      if (lane == 0) a.out[0][tt] += v;
    }
  }
}

__global__ void local_corner_kernel(const __grid_constant__ LocalArgs a, const int2* __restrict__ list,
                                    const int* __restrict__ count) {
  corner_pass(&a, nullptr, list, count);
}

__global__ void local_corner_batch_kernel(const LocalArgs* __restrict__ args, const int4* __restrict__ list,
                                          const int* __restrict__ count) {
  corner_pass<int4>(nullptr, args, list, count);
}

template <typename T>
void local_two_pass(const LocalArgs& a, int64_t nt, int2* list, int* count, cudaStream_t s) {
  const int threads = 128;
  const unsigned blocks = (unsigned)((nt + threads - 1) / threads);
  cudaMemsetAsync(count, 0, sizeof(int), s);
  local_classify_kernel<<<blocks, threads, 0, s>>>(a, list, count);
  const unsigned nblk = std::min<unsigned>(blocks, 152u * 16u);
  local_near_kernel<T><<<nblk, threads, 0, s>>>(a, list, count);
  if (a.n_corners > 0 && a.out[0] && a.jet && a.order >= 5)
    local_corner_kernel<<<std::min<unsigned>(blocks, 152u * 4u), threads, 0, s>>>(a, list, count);
}

}  // namespace

LocalArgs make_local_args(const Plan& P, int64_t nt, const double* txy, const double* jet, double* V,
                          double* S, double* D) {
  LocalArgs a;
  a.txy = txy;
  a.jet = V ? jet : nullptr;
  a.n = nt;
  a.out[0] = V;
  a.out[1] = S;
  a.out[2] = D;
  a.bxy = P.d_bxy;
  a.nb = P.nb;
  a.n_panels = (int)P.n_panels;
  a.p = P.p;
  a.tau = P.d_tau;
  a.geo_coef = P.d_geo_coef;
  a.geo_ref = P.d_geo_ref;
  a.sig_coef = P.have_sigma ? P.d_sigma_coef : nullptr;
  a.sig_ref = P.d_sigma_ref;
  a.mu_coef = P.have_mu ? P.d_mu_coef : nullptr;
  a.mu_ref = P.d_mu_ref;
  a.hx0 = P.hash_x0;
  a.hy0 = P.hash_y0;
  a.hh = P.hash_h;
  a.hh32 = (float)P.hash_h;
  a.inv_hh32 = (float)(1.0 / P.hash_h);
  a.hnx = P.hash_nx;
  a.hny = P.hash_ny;
  a.cell_start = P.d_cell_start;
  a.cell_near = P.d_cell_near;
  a.cell_node = P.d_cell_node;
  a.cell_xy32 = P.d_cell_xy32;
  a.geo_coef32 = P.d_geo_coef32;
  a.sig_coef32 = P.d_sigma_coef32;
  a.mu_coef32 = P.d_mu_coef32;
  a.geo_coef_dd = P.d_geo_coef_dd;
  a.sig_coef_dd = P.d_sigma_coef_dd;
  a.mu_coef_dd = P.d_mu_coef_dd;
  a.margin = P.margin;
  a.band = P.band;
  a.margin32 = (float)P.margin;
  a.band32 = (float)P.band;
  a.delta = P.delta1;
  a.delta_sd = P.dy_levels > 0 ? P.delta1 / std::pow(4.0, P.dy_levels) : P.delta1;
  a.on_tol = P.on_tol;
  a.order = P.order;
  a.status = P.d_status;
  a.corners = P.d_corners;
  a.n_corners = P.d_corner_q ? P.n_corners : 0;
  a.corner_q = P.d_corner_q;
  return a;
}

void launch_local(const Plan& P, int64_t nt, const double* txy, const double* jet, double* V,
                  double* S, double* D, cudaStream_t s) {
  launch_local_list(P, nt, txy, jet, V, S, D, P.d_near, P.d_near_count, s);
}

// Same two passes with a caller-provided list and counter (the counter is
// cleared here).
void launch_local_list(const Plan& P, int64_t nt, const double* txy, const double* jet, double* V,
                       double* S, double* D, int2* list, int* count, cudaStream_t s) {
  if (nt <= 0) return;
  LocalArgs a = make_local_args(P, nt, txy, jet, V, S, D);
  P.launches += 2 + (a.n_corners > 0 && a.out[0] && a.jet && a.order >= 5 ? 1 : 0);
  if (P.precision == LP_FP64)
    local_two_pass<double>(a, nt, list, count, s);
  else
    local_two_pass<float>(a, nt, list, count, s);
}

// Batched local pass over a wave of plans: one classify launch over every
// plan's targets (work entries of kBatchThreads targets), one near launch over
// the combined candidate list.
void launch_local_batch(int precision, const LocalArgs* d_args, const int2* d_work, int nwork, int4* d_list,
                        int* d_count, int64_t n_total, bool corners, cudaStream_t s) {
  if (nwork <= 0) return;
  cudaMemsetAsync(d_count, 0, sizeof(int), s);
  const unsigned nblk = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_total + 127) / 128, 152 * 16));
  local_classify_batch_kernel<<<nwork, kBatchThreads, 0, s>>>(d_args, d_work, d_list, d_count);
  if (precision == LP_FP64)
    local_near_batch_kernel<double><<<nblk, 128, 0, s>>>(d_args, d_list, d_count);
  else
    local_near_batch_kernel<float><<<nblk, 128, 0, s>>>(d_args, d_list, d_count);
  if (corners) local_corner_batch_kernel<<<std::min<unsigned>(nblk, 152u * 4u), 128, 0, s>>>(d_args, d_list, d_count);
}

}  // namespace lpg
