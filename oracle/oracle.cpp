// FP64 CPU oracle for the heat-kernel-split evaluation of 2D log-kernel
// volume and layer potentials (Fryklund, Greengard, Jiang, Potter,
// arXiv 2409.11998).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file: only tests/, the smoke check of the entry module and the
// CPU-baseline leg of the benchmark use it.  It shares no code with the CUDA
// implementation.
//
// What it computes (plainly, slowly, in double precision):
//   smooth part   u_H(x) = sum_j q_j G_H[delta](x - x_j)          (Sec. 2, eq. splitting2)
//                 D_H(x) = sum_b m_b d/dnu_b G_H[delta](x - y_b)
//   local part    the asymptotic expansions of Sec. 4 (lemmas for S_L, D_L,
//                 V_L), with the sign readings listed below, evaluated per
//                 target after a closest-point search on the boundary panels.
//
// Readings of the paper used here (each is forced by the definitions the
// paper gives, see the tests that pin them):
//   * D uses the derivative in the source point x' (eq. dlpot), so
//     D[1] = -1 inside, -1/2 on, 0 outside; the printed local D expansion
//     (eq. dlplocO5 and its on-surface corollary) is negated.
//   * The local S kernel is positive (eq. sheatloc); the printed S expansion
//     (eq. slplocO5, corollary) is negated.
//   * In the volume expansion (eq. vplocO5) with eta the inward normal and
//     kappa > 0 on convex boundaries, the delta^{3/2} term reads
//     (2 f_eta - kappa f); the printed on-boundary formula already does.
//   * Density and curve derivatives are with respect to the tangent-line
//     coordinate xi (Sec. 4, eq. tanparams), obtained by series reversion.
//   * Closest point: nearest boundary node, then Newton to |dt| < 1e-14
//     (at most 20 steps) on that node's panel; when the iterate stops at a
//     panel end, Newton again on the adjacent panel past that end.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

namespace {

const double kPi = 3.14159265358979323846;
const double kEulerGamma = 0.57721566490153286061;

// ---------------------------------------------------------------------------
// Exponential integral.  E1(z) = int_1^inf e^{-zt}/t dt  (Sec. 2, below
// eq. splitting2).  Ein(z) = sum_{k>=1} (-1)^{k+1} z^k / (k k!) is the entire
// part: E1(z) = -gamma - ln z + Ein(z).
// ---------------------------------------------------------------------------
double ein_series(double z) {
  double term = z, sum = z;
  for (int k = 2; k < 200; ++k) {
    term *= -z / k;                 // (-1)^{k+1} z^k / k!
    double add = term / k;
    sum += add;
    if (std::fabs(add) < 1e-18 * std::fabs(sum)) break;
  }
  return sum;
}

// Continued fraction for E1 (Abramowitz & Stegun 5.1.22), evaluated with the
// modified Lentz method, valid for z >= 1.
double e1_cfrac(double z) {
  const double tiny = 1e-300;
  double b = z + 1.0;
  double c = 1.0 / tiny;
  double d = 1.0 / b;
  double h = d;
  for (int i = 1; i < 500; ++i) {
    double an = -(double)i * i;
    b += 2.0;
    d = 1.0 / (an * d + b);
    c = b + an / c;
    double del = c * d;
    h *= del;
    if (std::fabs(del - 1.0) < 1e-16) break;
  }
  return h * std::exp(-z);
}

double e1(double z) {
  if (z <= 1.0) return -kEulerGamma - std::log(z) + ein_series(z);
  return e1_cfrac(z);
}

// G_H[delta](r) = -ln r /(2 pi) - E1(r^2/(4 delta)) /(4 pi)   (eq. splitting2).
// For r^2/(4 delta) <= 1 the two logarithms are cancelled analytically:
// G_H = (gamma - ln(4 delta) - Ein(z)) / (4 pi), which also gives the
// limit at r = 0.
double green_smooth(double r2, double delta) {
  double z = r2 / (4.0 * delta);
  if (z <= 1.0) return (kEulerGamma - std::log(4.0 * delta) - ein_series(z)) / (4.0 * kPi);
  double e = (z > 700.0) ? 0.0 : e1_cfrac(z);
  return (-std::log(r2) - e) / (4.0 * kPi);
}

// d/dnu_y G_H[delta](x - y) = (1 - exp(-r^2/4delta)) nu.(x - y) / (2 pi r^2):
// the normal derivative in the source point of G - G_L, with
// grad_y G_L(x-y) = exp(-r^2/4delta) (x-y)/(2 pi r^2).  Zero at r = 0.
double green_smooth_dipole(double dx, double dy, double nx, double ny, double delta) {
  double r2 = dx * dx + dy * dy;
  if (r2 == 0.0) return 0.0;
  double one_minus = -std::expm1(-r2 / (4.0 * delta));
  return one_minus * (nx * dx + ny * dy) / (2.0 * kPi * r2);
}

// ---------------------------------------------------------------------------
// Panel polynomials: Lagrange interpolation through the Gauss-Legendre
// abscissae tau[0..p-1] of one panel, expanded as a truncated Taylor series
// in s around t: P(t+s) = sum_k coef[k] s^k, k = 0..nd.
// ---------------------------------------------------------------------------
void lagrange_taylor(const double* tau, int p, const double* vals, int stride, double t,
                     int nd, double* coef) {
  for (int k = 0; k <= nd; ++k) coef[k] = 0.0;
  double c[8];
  // Interpolate v_i - v_mid (exact for neighbouring values) and add v_mid
  // back: the derivatives then carry rounding relative to the panel's
  // variation rather than to the coordinates' magnitude.
  const double vref = vals[(size_t)(p / 2) * stride];
  for (int i = 0; i < p; ++i) {
    for (int k = 0; k <= nd; ++k) c[k] = 0.0;
    c[0] = 1.0;
    for (int j = 0; j < p; ++j) {
      if (j == i) continue;
      double inv = 1.0 / (tau[i] - tau[j]);
      double a = (t - tau[j]) * inv;
      // multiply by (a + s*inv)
      for (int k = nd; k >= 1; --k) c[k] = a * c[k] + inv * c[k - 1];
      c[0] *= a;
    }
    double v = vals[(size_t)i * stride] - vref;
    for (int k = 0; k <= nd; ++k) coef[k] += v * c[k];
  }
  coef[0] += vref;
}

// Gauss-Legendre abscissae on [-1,1] by Newton iteration on P_p.
void gl_nodes(int p, double* x) {
  for (int i = 0; i < p; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (p + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= p; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = p * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[p - 1 - i] = z;  // ascending order
  }
}

// Gauss-Legendre weights for the abscissae x[0..p-1]: 2 / ((1 - x^2) P_p'(x)^2).
void gl_weights(int p, const double* x, double* w) {
  for (int i = 0; i < p; ++i) {
    const double z = x[i];
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= p; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    const double dp = p * (z * p1 - p0) / (z * z - 1.0);
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

struct Panels {
  int n_panels = 0, p = 0;
  const double* xy = nullptr;   // [n_panels*p][2]
  const double* sigma = nullptr;
  const double* mu = nullptr;
  std::vector<double> tau;
};

struct Foot {
  int panel;
  double t;
  double dist2;
};

// Newton on f(t) = (Gamma(t) - x) . Gamma'(t) for one panel, from t0.
Foot newton_on_panel(const Panels& P, int ip, double t0, double x, double y) {
  const double* base = P.xy + (size_t)ip * P.p * 2;
  double t = t0;
  double cx[5], cy[5];
  for (int it = 0; it < 20; ++it) {
    lagrange_taylor(P.tau.data(), P.p, base, 2, t, 2, cx);
    lagrange_taylor(P.tau.data(), P.p, base + 1, 2, t, 2, cy);
    double gx = cx[0] - x, gy = cy[0] - y;
    double d1x = cx[1], d1y = cy[1], d2x = 2 * cx[2], d2y = 2 * cy[2];
    double f = gx * d1x + gy * d1y;
    double sp2 = d1x * d1x + d1y * d1y;
    double fp = sp2 + gx * d2x + gy * d2y;
    if (fp < 0.1 * sp2) fp = sp2;  // Gauss-Newton safeguard
    double tn = t - f / fp;
    if (tn > 1.0) tn = 1.0;
    if (tn < -1.0) tn = -1.0;
    double dt = tn - t;
    t = tn;
    if (std::fabs(dt) < 1e-14) break;
  }
  lagrange_taylor(P.tau.data(), P.p, base, 2, t, 0, cx);
  lagrange_taylor(P.tau.data(), P.p, base + 1, 2, t, 0, cy);
  Foot f;
  f.panel = ip;
  f.t = t;
  f.dist2 = (cx[0] - x) * (cx[0] - x) + (cy[0] - y) * (cy[0] - y);
  return f;
}

// Truncated power-series product (degree <= 4).
void ps_mul(const double* a, const double* b, double* c) {
  for (int k = 0; k <= 4; ++k) {
    double s = 0.0;
    for (int i = 0; i <= k; ++i) s += a[i] * b[k - i];
    c[k] = s;
  }
}

// Compose F(s) = sum F_k s^k with s(xi) = sum_{k>=1} c_k xi^k, degree <= 4.
void ps_compose(const double* F, const double* s, double* out) {
  double powk[5] = {1, 0, 0, 0, 0}, tmp[5];
  for (int k = 0; k <= 4; ++k) out[k] = 0.0;
  for (int k = 0; k <= 4; ++k) {
    for (int j = 0; j <= 4; ++j) out[j] += F[k] * powk[j];
    ps_mul(powk, s, tmp);
    std::memcpy(powk, tmp, sizeof(tmp));
  }
}

struct LocalGeom {
  double r, sgn, c;
  double kappa, g3, g4;          // curve derivatives in xi (gamma'', ''', '''')
  double s0, s1, s2;             // sigma and its xi-derivatives
  double m0, m1, m2, m4;         // mu and its xi-derivatives
  double Tx, Ty, Nx, Ny;         // tangent, inward normal at b
};

// Geometry at the foot point: tangent-line frame and xi-derivatives
// (Sec. 4, eq. tanparams), by reversion of xi(s) = (Gamma(t*+s) - b).T.
void frame_at_foot(const Panels& P, const Foot& ft, double x, double y, double on_tol,
                   LocalGeom& g) {
  const double* base = P.xy + (size_t)ft.panel * P.p * 2;
  double cx[5], cy[5];
  lagrange_taylor(P.tau.data(), P.p, base, 2, ft.t, 4, cx);
  lagrange_taylor(P.tau.data(), P.p, base + 1, 2, ft.t, 4, cy);
  double sp = std::hypot(cx[1], cy[1]);
  g.Tx = cx[1] / sp;
  g.Ty = cy[1] / sp;
  g.Nx = -g.Ty;  // counter-clockwise curve: left normal points inward
  g.Ny = g.Tx;
  double bx = cx[0], by = cy[0];
  g.r = std::hypot(x - bx, y - by);
  if (g.r <= on_tol) {
    g.sgn = 0.0;
  } else {
    // sgn = sign((b - x) . nu), nu = -N the outward normal
    double s = -((bx - x) * g.Nx + (by - y) * g.Ny);
    g.sgn = (s > 0) ? 1.0 : -1.0;
  }
  double a[5], e[5];
  a[0] = 0.0;
  e[0] = 0.0;
  for (int k = 1; k <= 4; ++k) {
    a[k] = cx[k] * g.Tx + cy[k] * g.Ty;
    e[k] = cx[k] * g.Nx + cy[k] * g.Ny;
  }
  e[1] = 0.0;  // tangent direction by construction
  // reversion of xi(s) = a1 s + a2 s^2 + a3 s^3 + a4 s^4
  double a1 = a[1], a2 = a[2], a3 = a[3], a4 = a[4];
  double srev[5];
  srev[0] = 0.0;
  srev[1] = 1.0 / a1;
  srev[2] = -a2 / (a1 * a1 * a1);
  srev[3] = (2.0 * a2 * a2 - a1 * a3) / std::pow(a1, 5);
  srev[4] = (5.0 * a1 * a2 * a3 - a1 * a1 * a4 - 5.0 * a2 * a2 * a2) / std::pow(a1, 7);
  double eta_xi[5];
  ps_compose(e, srev, eta_xi);
  g.kappa = 2.0 * eta_xi[2];
  g.g3 = 6.0 * eta_xi[3];
  g.g4 = 24.0 * eta_xi[4];
  double sc[5], sx[5];
  if (P.sigma) {
    lagrange_taylor(P.tau.data(), P.p, P.sigma + (size_t)ft.panel * P.p, 1, ft.t, 4, sc);
    ps_compose(sc, srev, sx);
    g.s0 = sx[0];
    g.s1 = sx[1];
    g.s2 = 2.0 * sx[2];
  } else {
    g.s0 = g.s1 = g.s2 = 0.0;
  }
  if (P.mu) {
    lagrange_taylor(P.tau.data(), P.p, P.mu + (size_t)ft.panel * P.p, 1, ft.t, 4, sc);
    ps_compose(sc, srev, sx);
    g.m0 = sx[0];
    g.m1 = sx[1];
    g.m2 = 2.0 * sx[2];
    g.m4 = 24.0 * sx[4];
  } else {
    g.m0 = g.m1 = g.m2 = g.m4 = 0.0;
  }
}

// S_L, Sec. 4 single-layer lemma (eq. slplocO5) with the overall sign fixed
// so that S_L equals the positive heat integral of eq. sheatloc.
double local_single(const LocalGeom& g, double delta, int order) {
  double c = g.c, sg = g.sgn, k = g.kappa;
  double sd = std::sqrt(delta), sp = std::sqrt(kPi);
  double E = std::exp(-c * c / 4.0), Ec = std::erfc(c / 2.0);
  double A = c * Ec - 2.0 * E / sp;                         // c erfc - 2e/sqrt(pi)
  double B = 2.0 * c * c * c * Ec - (4.0 * c * c + 1.0) * E / sp;
  double Cq = 2.0 * (c * c - 2.0) * E / sp - c * c * c * Ec;
  double s = 0.0;
  s += sd * g.s0 / 2.0 * A;
  s += sg * delta * c * k * g.s0 / 4.0 * A;
  if (order >= 4) {
    s += std::pow(delta, 1.5) * g.s0 * k * k / 12.0 * B;
    s += std::pow(delta, 1.5) * g.s2 / 12.0 * Cq;
  }
  if (order >= 5) {
    double d2 = delta * delta;
    double Dq = 3.0 * c * c * c * Ec - (6.0 * c * c - 2.0) * E / sp;
    s += d2 * sg * (c * k * k * k * g.s0 / 16.0 * Dq + c * k * g.s2 / 8.0 * Cq);
    s += d2 * sg * (c * g.s0 * g.g4 / 48.0 * Cq + c * g.s1 * g.g3 / 12.0 * Cq);
  }
  return -s;
}

// D_L, Sec. 4 double-layer lemma (eq. dlplocO5), negated to the convention
// of eq. dlpot (derivative in the source point).
double local_double(const LocalGeom& g, double delta, int order) {
  double c = g.c, sg = g.sgn, k = g.kappa;
  double sd = std::sqrt(delta), sp = std::sqrt(kPi);
  double E = std::exp(-c * c / 4.0), Ec = std::erfc(c / 2.0);
  double c2 = c * c, c3 = c2 * c;
  double d15 = std::pow(delta, 1.5);
  double s = 0.0;
  s += sg * g.m0 / 2.0 * Ec;
  s += sd * k * g.m0 / (2.0 * sp) * E;
  s += delta * sg * (3.0 * c * k * k * g.m0 / (8.0 * sp) * E +
                     c * g.m2 / 4.0 * (2.0 * E / sp - c * Ec));
  if (order >= 4) {
    s += d15 * 5.0 * (c2 - 2.0) * k * k * k * g.m0 / (16.0 * sp) * E;
    s += d15 * g.g4 * g.m0 / (4.0 * sp) * E;
    s += d15 * k * g.m2 / 4.0 * (2.0 * (c2 + 1.0) * E / sp - c3 * Ec);
    s += d15 * g.g3 * g.m1 / 12.0 * (2.0 * E * (c2 + 4.0) / sp - c3 * Ec);
  }
  if (order >= 5) {
    double d2 = delta * delta;
    s += d2 * sg * (35.0 * c * k * k * k * k * g.m0 * (c2 - 6.0) / (128.0 * sp) * E +
                    5.0 * c * g.g3 * g.g3 * g.m0 / (12.0 * sp) * E +
                    5.0 * c * k * g.g4 * g.m0 / (8.0 * sp) * E);
    s += d2 * sg * 5.0 * c *
         (k * k * g.m2 / 16.0 * (2.0 * (c2 + 1.0) * E / sp - c3 * Ec) +
          k * g.g3 * g.m1 / 24.0 * (2.0 * (c2 + 4.0) * E / sp - c3 * Ec));
    s += d2 * sg * c * g.m4 / 48.0 * (c3 * Ec - 2.0 * (c2 - 2.0) * E / sp);
  }
  return -s;
}

// V_L, Sec. 4 volume lemma (eq. vplocO5), eta = inward normal, kappa > 0 on
// convex boundaries; the delta^{3/2} term carries (2 f_eta - kappa f).
double local_volume(const LocalGeom& g, const double* jet, double delta, int order) {
  double c = g.c, k = g.kappa;
  double fx = jet[1], fy = jet[2], fxx = jet[3], fxy = jet[4], fyy = jet[5], f = jet[0];
  double feta = fx * g.Nx + fy * g.Ny;
  double fxixi = fxx * g.Tx * g.Tx + 2.0 * fxy * g.Tx * g.Ty + fyy * g.Ty * g.Ty;
  double fetaeta = fxx * g.Nx * g.Nx + 2.0 * fxy * g.Nx * g.Ny + fyy * g.Ny * g.Ny;
  double sp = std::sqrt(kPi);
  double E = std::exp(-c * c / 4.0), Ec = std::erfc(c / 2.0), Ef = std::erf(c / 2.0);
  double c2 = c * c, c3 = c2 * c, c4 = c2 * c2;
  double v = 0.0;
  v += delta / 4.0 * (2.0 * Ef + 2.0 * E * c / sp - c2 * Ec + 2.0) * f;
  if (order >= 4)
    v += std::pow(delta, 1.5) * ((4.0 - 2.0 * c2) * E + sp * c3 * Ec) * (2.0 * feta - k * f) /
         (12.0 * sp);
  if (order >= 5) {
    v += delta * delta / 48.0 *
         (Ec * (4.0 * c4 * k * feta - 3.0 * (c4 + 4.0) * fetaeta + (c4 - 12.0) * fxixi -
                3.0 * c4 * k * k * f) +
          2.0 * c * (c2 - 2.0) * E * (-4.0 * k * feta + 3.0 * fetaeta - fxixi + 3.0 * k * k * f) /
              sp +
          24.0 * (fxixi + fetaeta));
  }
  return v;
}

}  // namespace

extern "C" {

double oracle_e1(double z) { return e1(z); }
double oracle_ein(double z) { return ein_series(z); }
double oracle_green_smooth(double r2, double delta) { return green_smooth(r2, delta); }

// out[i] = sum_j q[j] G_H[delta](t_i - s_j)   (charges; V_H and S_H)
void oracle_smooth_charge(int64_t ns, const double* sxy, const double* q, int64_t nt,
                          const double* txy, double delta, double* out) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nt; ++i) {
    double x = txy[2 * i], y = txy[2 * i + 1];
    double acc = 0.0;
    for (int64_t j = 0; j < ns; ++j) {
      double dx = x - sxy[2 * j], dy = y - sxy[2 * j + 1];
      acc += q[j] * green_smooth(dx * dx + dy * dy, delta);
    }
    out[i] = acc;
  }
}

// out[i] = sum_b m[b] d/dnu_b G_H[delta](t_i - y_b)   (dipoles; D_H)
void oracle_smooth_dipole(int64_t ns, const double* sxy, const double* nrm, const double* m,
                          int64_t nt, const double* txy, double delta, double* out) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nt; ++i) {
    double x = txy[2 * i], y = txy[2 * i + 1];
    double acc = 0.0;
    for (int64_t j = 0; j < ns; ++j) {
      double dx = x - sxy[2 * j], dy = y - sxy[2 * j + 1];
      acc += m[j] * green_smooth_dipole(dx, dy, nrm[2 * j], nrm[2 * j + 1], delta);
    }
    out[i] = acc;
  }
}

void oracle_gl_nodes(int p, double* x) { gl_nodes(p, x); }
void oracle_gl_weights(int p, const double* x, double* w) { gl_weights(p, x, w); }

// Expansion order p (3, 4 or 5): terms through delta^{(p-1)/2} are kept, so
// the truncation error is O(delta^{p/2}) (Sec. 4; Sec. 6.1 uses p = 4, 5 and
// Sec. 6.2 keeps terms up to O(delta), i.e. p = 3).
//
// Local part per target.  Boundary: n_panels x p nodes in order along a
// closed counter-clockwise curve; sigma/mu may be NULL.  jet: nt x 6 (may be
// NULL -> volume part skipped).  Outputs (any may be NULL): VL, SL, DL.
// info[i*4 + {0,1,2,3}] = {panel or -1 if far, t*, r, sgn}.  status bit 1:
// Right-angle corners of a polygonal boundary (a reading beyond Sec. 4, which assumes a smooth curve): a junction
// of two straight panels (every node on the chord to 1e-12 of its length)
// whose directions are perpendicular to 1e-9 and turn left (a convex corner
// of a counter-clockwise curve).  For each: the corner point (the two lines'
// intersection) and the inward unit normals of the edge before (n1) and after
// (n2) it.
struct Corner {
  double cx, cy, n1x, n1y, n2x, n2y;
};

static bool straight_panel(const Panels& P, int ip, double* tx, double* ty) {
  const double* a = P.xy + (size_t)ip * P.p * 2;
  const double* b = a + (size_t)(P.p - 1) * 2;
  const double L = std::hypot(b[0] - a[0], b[1] - a[1]);
  if (!(L > 0.0)) return false;
  *tx = (b[0] - a[0]) / L;
  *ty = (b[1] - a[1]) / L;
  for (int k = 1; k + 1 < P.p; ++k) {
    const double* q = a + 2 * k;
    const double off = (q[0] - a[0]) * (-*ty) + (q[1] - a[1]) * (*tx);
    if (std::fabs(off) > 1e-12 * L) return false;
  }
  return true;
}

static std::vector<Corner> right_angle_corners(const Panels& P) {
  std::vector<Corner> out;
  for (int i = 0; i < P.n_panels; ++i) {
    const int j = (i + 1) % P.n_panels;
    double t1x, t1y, t2x, t2y;
    if (!straight_panel(P, i, &t1x, &t1y) || !straight_panel(P, j, &t2x, &t2y)) continue;
    if (std::fabs(t1x * t2x + t1y * t2y) > 1e-9 || t1x * t2y - t1y * t2x <= 0.0) continue;
    // intersection of the line through panel i's last node along t1 and the
    // line through panel j's first node along t2
    const double* a = P.xy + ((size_t)i * P.p + P.p - 1) * 2;
    const double* b = P.xy + (size_t)j * P.p * 2;
    const double det = t1x * (-t2y) - t1y * (-t2x);
    const double s = ((b[0] - a[0]) * (-t2y) - (b[1] - a[1]) * (-t2x)) / det;
    Corner c;
    c.cx = a[0] + s * t1x;
    c.cy = a[1] + s * t1y;
    c.n1x = -t1y;  // inward normal: the tangent turned left
    c.n1y = t1x;
    c.n2x = -t2y;
    c.n2y = t2x;
    out.push_back(c);
  }
  return out;
}

// Local volume integral over the quadrant {(y - c).n1 >= 0, (y - c).n2 >= 0}
// for the quadratic f of the jet at x, at distances a = (x - c).n1 and
// b = (x - c).n2 from the two edges: the heat kernel separates along n1 and
// n2, so
//   V = int_0^delta [f A0 B0 + f_1 A1 B0 + f_2 A0 B1 + f_11 A2 B0 / 2
//                    + f_12 A1 B1 + f_22 A0 B2 / 2] dt,
// with the one-dimensional moments M_k(e, t) = int_{-e}^inf s^k g_t(s) ds of
// g_t(s) = exp(-s^2 / 4t) / sqrt(4 pi t):
//   M0 = 1 - erfc(e / 2 sqrt t) / 2, M1 = sqrt(t / pi) exp(-e^2 / 4t),
//   M2 = 2 t M0 - 2 t e g_t(e),
// and derivatives of f along n1, n2.  The time integral: t = delta s^2,
// composite Gauss-Legendre (16 points per piece) on s in [0, 1] with pieces
// graded towards s = 0, where the moments behave like exp(-e^2 / 4 delta s^2).
static double quadrant_volume(const double* J, double a, double b, const Corner& c, double delta) {
  const double f = J[0];
  const double f1 = J[1] * c.n1x + J[2] * c.n1y, f2 = J[1] * c.n2x + J[2] * c.n2y;
  auto hess = [&](double ux, double uy, double vx, double vy) {
    return J[3] * ux * vx + J[4] * (ux * vy + uy * vx) + J[5] * uy * vy;
  };
  const double f11 = hess(c.n1x, c.n1y, c.n1x, c.n1y), f22 = hess(c.n2x, c.n2y, c.n2x, c.n2y);
  const double f12 = hess(c.n1x, c.n1y, c.n2x, c.n2y);
  const double pi = 3.14159265358979323846;
  auto moments = [&](double e, double t, double* m) {
    const double g = std::exp(-e * e / (4.0 * t)) / std::sqrt(4.0 * pi * t);
    m[0] = 1.0 - 0.5 * std::erfc(e / (2.0 * std::sqrt(t)));
    m[1] = std::sqrt(t / pi) * std::exp(-e * e / (4.0 * t));
    m[2] = 2.0 * t * m[0] - 2.0 * t * e * g;
  };
  double x16[16], w16[16];
  gl_nodes(16, x16);
  gl_weights(16, x16, w16);
  const double edges[8] = {0.0, 1.0 / 1024, 1.0 / 256, 1.0 / 64, 1.0 / 16, 0.25, 0.5, 1.0};
  double v = 0.0;
  for (int piece = 0; piece < 7; ++piece)
    for (int k = 0; k < 16; ++k) {
      const double h = edges[piece + 1] - edges[piece];
      const double sv = edges[piece] + 0.5 * h * (x16[k] + 1.0);
      const double t = delta * sv * sv;
      double A[3], B[3];
      moments(a, t, A);
      moments(b, t, B);
      const double F = f * A[0] * B[0] + f1 * A[1] * B[0] + f2 * A[0] * B[1] + 0.5 * f11 * A[2] * B[0] +
                       f12 * A[1] * B[1] + 0.5 * f22 * A[0] * B[2];
      v += 0.5 * h * w16[k] * F * 2.0 * delta * sv;  // dt = 2 delta s ds; ds = (h/2) dx
    }
  return v;
}

// an exterior target lies inside the band where V_L is not available.
// At order 5, a target within 12 sqrt(delta) of both edges of a convex
// right-angle corner takes the quadrant integral (the same reading) instead of
// the nearest edge's half-plane.
int oracle_local(int n_panels, int p, const double* bxy, const double* sigma, const double* mu,
                 int64_t nt, const double* txy, const double* jet, double delta, int order,
                 double on_tol, double* VL, double* SL, double* DL, double* info) {
  Panels P;
  P.n_panels = n_panels;
  P.p = p;
  P.xy = bxy;
  P.sigma = sigma;
  P.mu = mu;
  P.tau.resize(p > 0 ? p : 1);
  if (p > 0) gl_nodes(p, P.tau.data());
  const int64_t nb = (int64_t)n_panels * p;
  // margin: longest chord between consecutive boundary nodes (cyclic)
  double margin = 0.0;
  for (int64_t j = 0; j < nb; ++j) {
    int64_t k = (j + 1) % nb;
    margin = std::max(margin, std::hypot(bxy[2 * k] - bxy[2 * j], bxy[2 * k + 1] - bxy[2 * j + 1]));
  }
  const double band = 12.0 * std::sqrt(delta);
  const std::vector<Corner> corners = (jet && order >= 5 && p > 1) ? right_angle_corners(P) : std::vector<Corner>();
  int status = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : status)
  for (int64_t i = 0; i < nt; ++i) {
    double x = txy[2 * i], y = txy[2 * i + 1];
    int64_t jbest = -1;
    double dbest = 1e300;
    for (int64_t j = 0; j < nb; ++j) {
      double dx = x - bxy[2 * j], dy = y - bxy[2 * j + 1];
      double d2 = dx * dx + dy * dy;
      if (d2 < dbest) {
        dbest = d2;
        jbest = j;
      }
    }
    bool far = (nb == 0) || (std::sqrt(dbest) - margin >= band);
    LocalGeom g;
    Foot best{-1, 0.0, 1e300};
    if (!far) {
      // Newton on the panel of the nearest node, started at that node; if
      // the iterate stops at a panel end, the foot lies beyond it: Newton
      // again on the adjacent panel, started at its node nearest the target,
      // and keep the closer foot (the first on ties).
      int ip0 = (int)(jbest / p);
      best = newton_on_panel(P, ip0, P.tau[jbest % p], x, y);
      if (std::fabs(best.t) == 1.0) {
        int ip = ((ip0 + (best.t > 0 ? 1 : -1)) % n_panels + n_panels) % n_panels;
        int kbest = 0;
        double kd = 1e300;
        for (int k = 0; k < p; ++k) {
          const double* q = bxy + ((size_t)ip * p + k) * 2;
          double d2 = (x - q[0]) * (x - q[0]) + (y - q[1]) * (y - q[1]);
          if (d2 < kd) {
            kd = d2;
            kbest = k;
          }
        }
        Foot f = newton_on_panel(P, ip, P.tau[kbest], x, y);
        if (f.dist2 < best.dist2) best = f;
      }
      if (std::sqrt(best.dist2) >= band) far = true;
    }
    double vl = 0.0, sl = 0.0, dl = 0.0;
    if (far) {
      if (jet) {
        const double* J = jet + 6 * i;
        vl = delta * J[0];
        if (order >= 5) vl += 0.5 * delta * delta * (J[3] + J[5]);
      }
      if (info) {
        info[4 * i] = -1;
        info[4 * i + 1] = 0;
        info[4 * i + 2] = std::sqrt(dbest);
        info[4 * i + 3] = 0;
      }
    } else {
      frame_at_foot(P, best, x, y, on_tol, g);
      g.c = g.r / std::sqrt(delta);
      if (sigma) sl = local_single(g, delta, order);
      if (mu) dl = local_double(g, delta, order);
      if (jet) {
        if (g.sgn < 0) {
          status |= 1;
          vl = 0.0;
        } else {
          vl = local_volume(g, jet + 6 * i, delta, order);
          for (const Corner& c : corners) {
            const double a = (x - c.cx) * c.n1x + (y - c.cy) * c.n1y;
            const double b = (x - c.cx) * c.n2x + (y - c.cy) * c.n2y;
            if (a > -on_tol && b > -on_tol && a < band && b < band) {
              vl = quadrant_volume(jet + 6 * i, std::max(a, 0.0), std::max(b, 0.0), c, delta);
              break;
            }
          }
        }
      }
      if (info) {
        info[4 * i] = best.panel;
        info[4 * i + 1] = best.t;
        info[4 * i + 2] = g.r;
        info[4 * i + 3] = g.sgn;
      }
    }
    if (VL) VL[i] = vl;
    if (SL) SL[i] = sl;
    if (DL) DL[i] = dl;
  }
  return status;
}

// Dyadic refinement of the local layer potentials (Sec. 4.4).  With
// delta_j = delta / 4^j (j = 0..J):
//   S_L[delta] = S_L[delta_J] + sum_{j=1..J} int_Gamma (G_H[delta_j] - G_H[delta_{j-1}]) sigma ds
//   D_L[delta] = D_L[delta_J] + sum_{j=1..J} int_Gamma d/dnu (G_H[delta_j] - G_H[delta_{j-1}]) mu ds
// (S_L[delta] = S - S_H[delta] for every delta; G_H[delta_j] - G_H[delta_{j-1}]
// is the smooth difference kernel (E1(4^{j-2} r) - E1(4^{j-1} r)) / (4 pi),
// r = |x - x'|^2 / delta).  S_L[delta_J], D_L[delta_J] are the asymptotic
// expansions of order `order`; each difference integral is a direct sum over
// every panel split into m0 2^{j-1} equal parameter intervals of p
// Gauss-Legendre nodes, with the panel's Lagrange interpolant giving the
// position, |Gamma'|, the outward normal and sigma, mu at each node.
// Outputs SL, DL (either may be NULL).
int oracle_local_dyadic(int n_panels, int p, const double* bxy, const double* sigma, const double* mu,
                        int64_t nt, const double* txy, double delta, int order, double on_tol, int J,
                        int m0, double* SL, double* DL) {
  const double delta_J = delta / std::pow(4.0, J);
  int st = oracle_local(n_panels, p, bxy, sigma, mu, nt, txy, nullptr, delta_J, order, on_tol, nullptr, SL,
                        DL, nullptr);
  if (J <= 0) return st;
  std::vector<double> tau(p), wgl(p);
  gl_nodes(p, tau.data());
  gl_weights(p, tau.data(), wgl.data());
  for (int j = 1; j <= J; ++j) {
    const double d_new = delta / std::pow(4.0, j), d_old = delta / std::pow(4.0, j - 1);
    const int m = m0 << (j - 1);
    // quadrature nodes of this level: position, outward normal, weight, densities
    const int64_t nq = (int64_t)n_panels * m * p;
    std::vector<double> qx(nq), qy(nq), qnx(nq), qny(nq), qw(nq), qs(nq), qm(nq);
    for (int ip = 0; ip < n_panels; ++ip) {
      const double* base = bxy + (size_t)ip * p * 2;
      for (int k = 0; k < m; ++k)
        for (int i = 0; i < p; ++i) {
          const double t = -1.0 + (2.0 * k + 1.0 + tau[i]) / m;
          double cx[2], cy[2];
          lagrange_taylor(tau.data(), p, base, 2, t, 1, cx);
          lagrange_taylor(tau.data(), p, base + 1, 2, t, 1, cy);
          const double sp = std::hypot(cx[1], cy[1]);
          const int64_t q = ((int64_t)ip * m + k) * p + i;
          qx[q] = cx[0];
          qy[q] = cy[0];
          qnx[q] = cy[1] / sp;  // outward normal of a counter-clockwise curve
          qny[q] = -cx[1] / sp;
          qw[q] = sp * wgl[i] / m;
          double v[1];
          if (sigma) {
            lagrange_taylor(tau.data(), p, sigma + (size_t)ip * p, 1, t, 0, v);
            qs[q] = v[0];
          }
          if (mu) {
            lagrange_taylor(tau.data(), p, mu + (size_t)ip * p, 1, t, 0, v);
            qm[q] = v[0];
          }
        }
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; ++i) {
      const double x = txy[2 * i], y = txy[2 * i + 1];
      double s_acc = 0.0, d_acc = 0.0;
      for (int64_t q = 0; q < nq; ++q) {
        const double dx = x - qx[q], dy = y - qy[q];
        const double r2 = dx * dx + dy * dy;
        if (sigma) s_acc += (green_smooth(r2, d_new) - green_smooth(r2, d_old)) * qs[q] * qw[q];
        if (mu)
          d_acc += (green_smooth_dipole(dx, dy, qnx[q], qny[q], d_new) -
                    green_smooth_dipole(dx, dy, qnx[q], qny[q], d_old)) *
                   qm[q] * qw[q];
      }
      if (SL && sigma) SL[i] += s_acc;
      if (DL && mu) DL[i] += d_acc;
    }
  }
  return st;
}

// Frame quantities at a given foot (for tests): out = {kappa, g3, g4, s0, s1,
// s2, m0, m1, m2, m4, Tx, Ty, bx, by}.
void oracle_frame(int n_panels, int p, const double* bxy, const double* sigma, const double* mu,
                  int panel, double t, double* out) {
  Panels P;
  P.n_panels = n_panels;
  P.p = p;
  P.xy = bxy;
  P.sigma = sigma;
  P.mu = mu;
  P.tau.resize(p);
  gl_nodes(p, P.tau.data());
  Foot f{panel, t, 0.0};
  LocalGeom g;
  double cx[1], cy[1];
  lagrange_taylor(P.tau.data(), p, bxy + (size_t)panel * p * 2, 2, t, 0, cx);
  lagrange_taylor(P.tau.data(), p, bxy + (size_t)panel * p * 2 + 1, 2, t, 0, cy);
  frame_at_foot(P, f, cx[0], cy[0], 1.0, g);
  double v[14] = {g.kappa, g.g3, g.g4, g.s0, g.s1, g.s2, g.m0, g.m1, g.m2, g.m4,
                  g.Tx, g.Ty, cx[0], cy[0]};
  std::memcpy(out, v, sizeof(v));
}

// Local expansions for given frame data (for tests): geom = {r, sgn, kappa,
// g3, g4, s0, s1, s2, m0, m1, m2, m4, Tx, Ty}; jet6 in the global frame.
void oracle_local_formulas(const double* geom, const double* jet6, double delta, int order,
                           double* out3) {
  LocalGeom g;
  g.r = geom[0];
  g.sgn = geom[1];
  g.kappa = geom[2];
  g.g3 = geom[3];
  g.g4 = geom[4];
  g.s0 = geom[5];
  g.s1 = geom[6];
  g.s2 = geom[7];
  g.m0 = geom[8];
  g.m1 = geom[9];
  g.m2 = geom[10];
  g.m4 = geom[11];
  g.Tx = geom[12];
  g.Ty = geom[13];
  g.Nx = -g.Ty;
  g.Ny = g.Tx;
  g.c = g.r / std::sqrt(delta);
  out3[0] = local_volume(g, jet6, delta, order);
  out3[1] = local_single(g, delta, order);
  out3[2] = local_double(g, delta, order);
}

}  // extern "C"
