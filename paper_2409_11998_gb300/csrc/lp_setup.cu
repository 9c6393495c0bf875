// Plan-time host computations: history-grid sizing (Sec. 2.3 and Sec. 3,
// Step 1, generalised to an arbitrary box), the deconvolved Fourier
// multiplier tables (eq. vnearkspace, eq. vfarkspace, eq. Wdef), and the
// boundary search structures used by the local part (Sec. 2.2, Sec. 4).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lp_internal.cuh"

namespace lpg {

namespace {
const double kPi = 3.14159265358979323846;

// Smallest k > 1/sqrt(2 delta) (beyond the maximum of k e^{-k^2 delta}) with
// k e^{-k^2 delta} < eps: the truncation rule of Sec. 3 (input of the
// history algorithm), used for every channel.
double fourier_cutoff(double delta, double eps) {
  double lo = 1.0 / std::sqrt(2.0 * delta), hi = lo;
  while (hi * std::exp(-hi * hi * delta) >= eps) hi *= 1.5;
  for (int i = 0; i < 200; ++i) {
    double mid = 0.5 * (lo + hi);
    if (mid * std::exp(-mid * mid * delta) >= eps) lo = mid; else hi = mid;
  }
  return hi;
}

}  // namespace

void gauss_legendre(int p, double* x, double* w) {
  // Newton on P_p from Chebyshev-like initial guesses; ascending order.
  for (int i = 0; i < p; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (p + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= p; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = p * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[p - 1 - i] = z;
    w[p - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Smallest even 3-smooth integer (2^a 3^b) >= n: on GB300 cuFFT's FP64
// transforms of such sizes are ~25% faster per point than 5- or 7-smooth ones.
int fft_size(int n) {
  int m = std::max(n, 8);
  if (m & 1) ++m;
  for (;; m += 2) {
    int k = m;
    for (int f : {2, 3})
      while (k % f == 0) k /= f;
    if (k == 1) return m;
  }
}

lp_status choose_levels(Plan& P) {
  const double eps = P.tol;
  const double D = P.side;
  const double cx = 0.5 * (P.box_lo[0] + P.box_hi[0]);
  const double cy = 0.5 * (P.box_lo[1] + P.box_hi[1]);
  // Reach of the Gaussian tails beyond which the history kernels are below
  // eps: e^{-R^2 / (4 delta_2)} = eps.
  const double R = std::sqrt(4.0 * P.delta2 * std::log(1.0 / eps));
  for (int l = P.l0; l < 2; ++l) {
    GridLevel& G = P.lv[l];
    G.kind = l;
    G.R = R;
    double kmax;
    if (l == 0) {
      kmax = fourier_cutoff(P.delta1, 0.1 * eps);
      G.P = D + R;                 // period excludes aliasing of F_NH over the box
      G.L = 0.0;
    } else {
      kmax = fourier_cutoff(P.delta2, 0.1 * eps);
      G.L = std::sqrt(2.0) * D + R;  // truncation radius of eq. Wdef, generalised
      G.P = D + G.L + R;
    }
    G.dk = 2.0 * kPi / G.P;
    G.K = (int)std::ceil(kmax / G.dk);
    int g = fft_size(std::max((int)std::ceil(P.sigma * (2 * G.K + 1)), 2 * P.ker.w + 8));
    // the spreading stencil of every point in the box must stay inside the
    // grid (no periodic wrap): margin (P - D)/2 >= (w/2 + 2) h
    while ((G.P - D) / 2.0 < (P.ker.half_w + 2.0) * (G.P / g)) g = fft_size(g + 2);
    G.g = g;
    G.h = G.P / g;
    G.pitch = 2 * (g / 2 + 1);
    G.x0 = cx - 0.5 * G.P;
    G.y0 = cy - 0.5 * G.P;
    // rows touched by the stencils of points in the box: the only rows the
    // row transforms need (other rows of the spread grid are zero, other rows
    // of the output grid are never read)
    G.row_lo = std::max(0, (int)std::floor((P.box_lo[1] - G.y0) / G.h - P.ker.half_w) - 2);
    G.row_hi = std::min(g, (int)std::ceil((P.box_hi[1] - G.y0) / G.h + P.ker.half_w) + 3);
    if (G.K > g / 2 - 1) return LP_ERR_ARG;
  }
  // ES shape parameter for the realised upsampling (the smaller of the two
  // levels): beta = 0.97 pi (1 - 1/(2 sigma)) w, the exponential-of-semicircle
  // choice of Barnett, Magland and af Klinteberg (SISC 2019).
  P.sigma_eff = P.lv[1].g / (2.0 * P.lv[1].K + 1.0);
  if (P.l0 == 0) P.sigma_eff = std::min(P.sigma_eff, P.lv[0].g / (2.0 * P.lv[0].K + 1.0));
  P.ker.beta = 0.97 * kPi * (1.0 - 0.5 / P.sigma_eff) * P.ker.w;
  return LP_OK;
}

// Deconvolution factors: the Fourier transform, at the kept modes, of the
// kernel the spread and the interpolation evaluate -- the fitted piecewise
// polynomial (double coefficients for FP64 plans, their float roundings for
// FP32 plans), not the exponential of semicircle it approximates.  Weight t
// of a point at offset v in [-1/2, 1/2) is the kernel at grid distance
// x = v + (w-1)/2 - t, so piece t covers x in [w/2 - t - 1, w/2 - t); the
// kernel is even, and its cosine transform is summed piece by piece with 16
// Gauss-Legendre nodes each.  Deconvolving by the kernel actually used
// removes the fit error from the normalisation of every mode (measured on the
// FP32 starfish: a systematic relative error of ~2.7e-6, proportional to the
// potential itself, from a fit to 1e-7).
lp_status build_tables(Plan& P) {
  const int w = P.es.w, nc = P.es.nc;
  const bool f32 = P.precision == LP_FP32;
  double gx[16], gw[16];
  gauss_legendre(16, gx, gw);
  std::vector<double> px((size_t)w * 16), pv((size_t)w * 16), pw((size_t)w * 16);
  for (int t = 0; t < w; ++t)
    for (int q = 0; q < 16; ++q) {
      const double v = 0.5 * gx[q];
      double acc = f32 ? (double)P.es32.c[nc - 1][t] : P.es.c[nc - 1][t];
      for (int k = nc - 2; k >= 0; --k) acc = acc * v + (f32 ? (double)P.es32.c[k][t] : P.es.c[k][t]);
      px[t * 16 + q] = v + 0.5 * (w - 1) - t;
      pv[t * 16 + q] = acc;
      pw[t * 16 + q] = 0.5 * gw[q];
    }
  for (int l = P.l0; l < 2; ++l) {
    GridLevel& G = P.lv[l];
    const int K = G.K;
    std::vector<double> ph(K + 1);
    for (int m = 0; m <= K; ++m) {
      const double xi = 2.0 * kPi * m / G.g;
      double s = 0.0;
      for (size_t i = 0; i < px.size(); ++i) s += pw[i] * pv[i] * std::cos(xi * px[i]);
      ph[m] = s;
    }
    const double scale = (G.dk / (2.0 * kPi)) * (G.dk / (2.0 * kPi));
    // the k = 0 multiplier without deconvolution (FP32 path adds it in FP64)
    G.zero_mode = scale * (l == 0 ? (P.delta2 - P.delta1) : G.L * G.L * (1.0 - 2.0 * std::log(G.L)) / 4.0);
    const size_t n = (size_t)(K + 1) * (K + 1);
    double* d_ph = nullptr;
    if (cudaMalloc(&G.mtab, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G.mtab32, n * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&d_ph, (K + 1) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      if (d_ph) cudaFree(d_ph);
      return LP_ERR_NOMEM;
    }
    P.device_bytes += n * (sizeof(double) + sizeof(float));
    cudaMemcpy(d_ph, ph.data(), (K + 1) * sizeof(double), cudaMemcpyHostToDevice);
    launch_mult_table(l, K, G.dk, P.delta1, P.delta2, G.L, scale, d_ph, G.mtab, G.mtab32, P.stream);
    cudaStreamSynchronize(P.stream);
    cudaFree(d_ph);
  }
  return LP_OK;
}

// Leading Horner steps of the df64 weight chains (even and odd parts in
// v^2, see dd_stencil_weights) that may run in single precision: the largest
// m <= 4 for which the float steps -- coefficients rounded to float, v^2
// rounded to float, fused multiply-adds rounded to float, the rest exact --
// move no weight by more than 5% of the fit's error target, over a fine grid
// of v in [-1/2, 1/2].
static int float_horner_steps(const Plan& P, double target) {
  const int w = P.es.w, nc = P.es.nc;
  const int ke = (nc - 1) & ~1, ko = (nc - 2) | 1;
  int best = 0;
  for (int m = 1; m <= 4; ++m) {
    double worst = 0.0;
    for (int t = 0; t < (w + 1) / 2; ++t)
      for (int j = 0; j <= 400; ++j) {
        const double v = -0.5 + j / 400.0 * (1.0 - 1e-12), u = v * v;
        double err = 0.0;
        for (int par = 0; par < 2; ++par) {
          const int top = par ? ko : ke;
          double exact = P.es.c[top][t];
          float f = (float)P.es.c[top][t];
          int s = 0;
          for (int k = top - 2; k >= par; k -= 2, ++s) {
            exact = exact * u + P.es.c[k][t];
            if (s < m)
              f = std::fmaf(f, (float)u, (float)P.es.c[k][t]);
          }
          // the exact continuation from the float partial sum after m steps
          double mixed = (double)f;
          s = 0;
          for (int k = top - 2; k >= par; k -= 2, ++s)
            if (s >= m) mixed = mixed * u + P.es.c[k][t];
          err += std::fabs(mixed - exact) * (par ? std::fabs(v) : 1.0);
        }
        worst = std::max(worst, err);
      }
    if (worst > 0.05 * target) break;
    best = m;
  }
  return best;
}

// Chebyshev interpolation of each stencil weight phi_t(v), v in [-1/2, 1/2),
// converted to monomials in v (long double on the host).  The degree grows
// until the interior weights are within tol/100 of the kernel; the two edge
// weights reach the support edge z = +-1, where sqrt(1 - z^2) is not smooth,
// and are accepted once within 4 e^{-beta} (the kernel's own value there,
// below the kernel's truncation error).
lp_status fit_kernel_poly(Plan& P) {
  const int w = P.ker.w;
  const double beta = P.ker.beta, hw = P.ker.half_w;
  auto phi = [&](int t, long double v) -> long double {
    long double z = (v + (long double)(hw - 0.5) - t) / hw;
    long double a = 1.0L - z * z;
    return a > 0 ? std::exp((long double)beta * (std::sqrt(a) - 1.0L)) : 0.0L;
  };
  const double target = std::max(0.01 * P.tol, 1e-15);
  const double target_edge = std::max(target, 4.0 * std::exp(-beta));
  for (int nc = w + 1; nc <= kMaxNC; ++nc) {
    double err = 0.0, err_edge = 0.0;
    for (int t = 0; t < w; ++t) {
      // Chebyshev coefficients from values at Chebyshev points on [-1,1] (x = 2 v)
      std::vector<long double> fx(nc), cheb(nc, 0.0L);
      for (int j = 0; j < nc; ++j) {
        long double x = std::cos((long double)M_PI * (j + 0.5L) / nc);
        fx[j] = phi(t, 0.5L * x);
      }
      for (int k = 0; k < nc; ++k) {
        long double s = 0;
        for (int j = 0; j < nc; ++j) s += fx[j] * std::cos((long double)M_PI * k * (j + 0.5L) / nc);
        cheb[k] = s * (k == 0 ? 1.0L : 2.0L) / nc;
      }
      // monomials in x: T_0 = 1, T_1 = x, T_{k+1} = 2x T_k - T_{k-1}
      std::vector<long double> mono(nc, 0.0L), tm(nc, 0.0L), tk(nc, 0.0L), tn(nc);
      tm[0] = 1.0L;
      if (nc > 1) tk[1] = 1.0L;
      mono[0] += cheb[0];
      for (int i = 0; i < nc; ++i) mono[i] += (nc > 1 ? cheb[1] : 0.0L) * tk[i];
      for (int k = 1; k + 1 < nc; ++k) {
        for (int i = 0; i < nc; ++i) tn[i] = (i ? 2.0L * tk[i - 1] : 0.0L) - tm[i];
        for (int i = 0; i < nc; ++i) mono[i] += cheb[k + 1] * tn[i];
        tm = tk;
        tk = tn;
      }
      // x = 2 v: coefficient of v^i is mono[i] 2^i
      long double sc = 1.0L;
      for (int i = 0; i < nc; ++i) {
        P.es.c[i][t] = (double)(mono[i] * sc);
        P.es32.c[i][t] = (float)(mono[i] * sc);
        sc *= 2.0L;
      }
      double e = 0.0;
      for (int j = 0; j <= 400; ++j) {
        double v = -0.5 + j / 400.0 * (1.0 - 1e-12);
        double acc = P.es.c[nc - 1][t];
        for (int i = nc - 2; i >= 0; --i) acc = acc * v + P.es.c[i][t];
        e = std::max(e, (double)std::fabs((long double)acc - phi(t, v)));
      }
      if (t == 0 || t == w - 1) err_edge = std::max(err_edge, e);
      else err = std::max(err, e);
    }
    P.es.w = P.es32.w = w;
    P.es.nc = P.es32.nc = nc;
    P.es_fit_err = std::max(err, err_edge);
    if (err <= target && err_edge <= target_edge) {
      P.es_float_steps = float_horner_steps(P, target);
      return LP_OK;
    }
  }
  P.es_float_steps = float_horner_steps(P, target);
  return LP_OK;  // best effort at the maximum degree (error recorded)
}

// Convex right-angle corners of a polygonal boundary (outside the smooth-curve setting of Sec. 4): consecutive
// panels whose nodes lie on their chords (to 1e-12 of the chord) with
// perpendicular directions (to 1e-9) turning left (counter-clockwise
// curve).  Each: the intersection of the two edge lines and the inward
// normals of the edge before and after the corner.  Targets within 12
// sqrt(delta) of both edges take the quadrant form of the local volume
// integral (order 5).
static std::vector<double> find_corners(int64_t n_panels, int p, const double* xy) {
  std::vector<double> out;
  auto dir = [&](int64_t ip, double& tx, double& ty) {
    const double* a = xy + (size_t)ip * p * 2;
    const double* b = a + (size_t)(p - 1) * 2;
    const double len = std::hypot(b[0] - a[0], b[1] - a[1]);
    if (!(len > 0.0)) return false;
    tx = (b[0] - a[0]) / len;
    ty = (b[1] - a[1]) / len;
    for (int k = 1; k < p - 1; ++k) {
      const double* q = a + 2 * k;
      if (std::fabs((q[1] - a[1]) * tx - (q[0] - a[0]) * ty) > 1e-12 * len) return false;
    }
    return true;
  };
  for (int64_t i = 0; i < n_panels && p > 1; ++i) {
    const int64_t j = (i + 1) % n_panels;
    double ux, uy, vx, vy;
    if (!dir(i, ux, uy) || !dir(j, vx, vy)) continue;
    if (std::fabs(ux * vx + uy * vy) > 1e-9 || ux * vy - uy * vx <= 0.0) continue;
    const double* e = xy + ((size_t)i * p + p - 1) * 2;  // last node of the edge before
    const double* f = xy + (size_t)j * p * 2;            // first node of the edge after
    // e + s u = f + r v  =>  s = ((f - e) x v) / (u x v)
    const double s = ((f[0] - e[0]) * vy - (f[1] - e[1]) * vx) / (ux * vy - uy * vx);
    const double c[6] = {e[0] + s * ux, e[1] + s * uy, -uy, ux, -vy, vx};
    out.insert(out.end(), c, c + 6);
  }
  return out;
}

lp_status build_boundary(Plan& P, const double* h_xy, const double* h_w, const double* h_nrm) {
  const int p = P.p;
  const int64_t nb = P.nb;
  {
    const std::vector<double> cor = find_corners(P.n_panels, p, h_xy);
    if (!cor.empty()) {
      P.n_corners = (int)(cor.size() / 6);
      // time integral: t = delta s^2 on six pieces of s in [0, 1] graded
      // towards 0, 16 Gauss-Legendre nodes each; weight = piece / 2 * w * 2 delta s
      double x[16], w[16];
      gauss_legendre(16, x, w);
      const double edges[7] = {0.0, 1.0 / 2048, 1.0 / 128, 1.0 / 32, 1.0 / 8, 0.375, 1.0};
      std::vector<double> q(2 * kCornerQuad);
      for (int piece = 0; piece < 6; ++piece)
        for (int k = 0; k < 16; ++k) {
          const double h = edges[piece + 1] - edges[piece];
          const double sv = edges[piece] + 0.5 * h * (x[k] + 1.0);
          q[piece * 16 + k] = P.delta1 * sv * sv;
          q[kCornerQuad + piece * 16 + k] = 0.5 * h * w[k] * 2.0 * P.delta1 * sv;
        }
      if (cudaMalloc((void**)&P.d_corners, cor.size() * sizeof(double)) != cudaSuccess ||
          cudaMalloc((void**)&P.d_corner_q, q.size() * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return LP_ERR_NOMEM;
      }
      P.device_bytes += cor.size() * sizeof(double) + q.size() * sizeof(double);
      cudaMemcpy(P.d_corners, cor.data(), cor.size() * sizeof(double), cudaMemcpyHostToDevice);
      cudaMemcpy(P.d_corner_q, q.data(), q.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
  }
  // margin: longest chord between consecutive nodes along the curve; any
  // point of the curve is within it of a node, so a target whose nearest
  // node is farther than band + margin is outside the band.
  double margin = 0.0;
  for (int64_t j = 0; j < nb; ++j) {
    int64_t k = (j + 1) % nb;
    margin = std::max(margin, std::hypot(h_xy[2 * k] - h_xy[2 * j], h_xy[2 * k + 1] - h_xy[2 * j + 1]));
  }
  P.margin = margin;
  P.band = 12.0 * std::sqrt(P.delta1);
  // hash of nodes: cells of side >= band + margin over the box (+ one cell)
  double hc = P.band + P.margin;
  double lo0 = P.box_lo[0], lo1 = P.box_lo[1], hi0 = P.box_hi[0], hi1 = P.box_hi[1];
  for (int64_t j = 0; j < nb; ++j) {
    lo0 = std::min(lo0, h_xy[2 * j]);
    hi0 = std::max(hi0, h_xy[2 * j]);
    lo1 = std::min(lo1, h_xy[2 * j + 1]);
    hi1 = std::max(hi1, h_xy[2 * j + 1]);
  }
  int nx = std::max(1, (int)std::ceil((hi0 - lo0) / hc) + 2);
  int ny = std::max(1, (int)std::ceil((hi1 - lo1) / hc) + 2);
  while ((int64_t)nx * ny > (int64_t)1 << 24) {  // bound the table for tiny deltas
    hc *= 2.0;
    nx = std::max(1, (int)std::ceil((hi0 - lo0) / hc) + 2);
    ny = std::max(1, (int)std::ceil((hi1 - lo1) / hc) + 2);
  }
  P.hash_h = hc;
  P.hash_x0 = lo0 - hc;
  P.hash_y0 = lo1 - hc;
  P.hash_nx = nx;
  P.hash_ny = ny;
  std::vector<int> cnt((size_t)nx * ny + 1, 0), cell(nb), order(nb);
  for (int64_t j = 0; j < nb; ++j) {
    int cx = (int)std::floor((h_xy[2 * j] - P.hash_x0) / hc);
    int cy = (int)std::floor((h_xy[2 * j + 1] - P.hash_y0) / hc);
    cx = std::min(std::max(cx, 0), nx - 1);
    cy = std::min(std::max(cy, 0), ny - 1);
    cell[j] = cy * nx + cx;
    cnt[cell[j] + 1]++;
  }
  for (size_t c = 0; c + 1 < cnt.size(); ++c) cnt[c + 1] += cnt[c];
  // cells whose 3x3 neighbourhood holds no node: every target there is far
  // from the boundary, and the classification skips the scan
  std::vector<unsigned char> near((size_t)nx * ny, 0);
  for (int cy = 0; cy < ny; ++cy)
    for (int cx = 0; cx < nx; ++cx) {
      const int c = cy * nx + cx;
      if (cnt[c + 1] == cnt[c]) continue;
      for (int yy = std::max(cy - 1, 0); yy <= std::min(cy + 1, ny - 1); ++yy)
        for (int xx = std::max(cx - 1, 0); xx <= std::min(cx + 1, nx - 1); ++xx) near[(size_t)yy * nx + xx] = 1;
    }
  std::vector<int> fill(cnt.begin(), cnt.end() - 1);
  for (int64_t j = 0; j < nb; ++j) order[fill[cell[j]]++] = (int)j;  // stable: ascending ids
  // FP32 coordinates of each sorted node relative to its cell's origin, for
  // the single-precision prefilter of the nearest-node search
  std::vector<float2> rel(std::max<int64_t>(nb, 1));
  for (int64_t k = 0; k < nb; ++k) {
    int j = order[k];
    int c = cell[j];
    double ox = P.hash_x0 + (c % nx) * hc, oy = P.hash_y0 + (c / nx) * hc;
    rel[k] = make_float2((float)(h_xy[2 * j] - ox), (float)(h_xy[2 * j + 1] - oy));
  }

  // Legendre transform of the panel interpolant: coef_k = (2k+1)/2 sum_i w_i v_i P_k(tau_i)
  // (exact: the interpolant has degree p-1 and the Gauss rule degree 2p-1)
  std::vector<double> tau(p), wq(p), T((size_t)p * p);
  gauss_legendre(p, tau.data(), wq.data());
  for (int i = 0; i < p; ++i) {
    double p0 = 1.0, p1 = tau[i];
    for (int k = 0; k < p; ++k) {
      double pk;
      if (k == 0) pk = 1.0;
      else if (k == 1) pk = tau[i];
      else {
        double p2 = ((2.0 * k - 1.0) * tau[i] * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
        pk = p2;
      }
      // coefficients are stored divided by k!, for the recurrence of Q_k = k! P_k
      T[(size_t)k * p + i] = 0.5 * (2.0 * k + 1.0) * wq[i] * pk / std::tgamma(k + 1.0);
    }
  }
  auto dmalloc = [&](void** ptr, size_t bytes) -> bool {
    if (cudaMalloc(ptr, bytes) != cudaSuccess) return false;
    P.device_bytes += bytes;
    return true;
  };
  if (!dmalloc((void**)&P.d_bxy, nb * 2 * sizeof(double)) ||
      !dmalloc((void**)&P.d_bw, nb * sizeof(double)) ||
      !dmalloc((void**)&P.d_bnrm, nb * 2 * sizeof(double)) ||
      !dmalloc((void**)&P.d_geo_coef, (size_t)P.n_panels * 2 * p * sizeof(double)) ||
      !dmalloc((void**)&P.d_geo_ref, (size_t)P.n_panels * 2 * sizeof(double)) ||
      !dmalloc((void**)&P.d_leg_T, (size_t)p * p * sizeof(double)) ||
      !dmalloc((void**)&P.d_tau, p * sizeof(double)) ||
      !dmalloc((void**)&P.d_cell_start, cnt.size() * sizeof(int)) ||
      !dmalloc((void**)&P.d_cell_near, near.size()) ||
      !dmalloc((void**)&P.d_cell_node, std::max<int64_t>(nb, 1) * sizeof(int)) ||
      !dmalloc((void**)&P.d_cell_xy32, std::max<int64_t>(nb, 1) * sizeof(float2)) ||
      !dmalloc((void**)&P.d_geo_coef32, (size_t)P.n_panels * 2 * p * sizeof(float)) ||
      !dmalloc((void**)&P.d_bq, 3 * nb * sizeof(double)) ||
      !dmalloc((void**)&P.d_sigma, nb * sizeof(double)) ||
      !dmalloc((void**)&P.d_mu, nb * sizeof(double)) ||
      !dmalloc((void**)&P.d_sigma_coef, (size_t)P.n_panels * p * sizeof(double)) ||
      !dmalloc((void**)&P.d_sigma_ref, (size_t)P.n_panels * sizeof(double)) ||
      !dmalloc((void**)&P.d_mu_coef, (size_t)P.n_panels * p * sizeof(double)) ||
      !dmalloc((void**)&P.d_mu_ref, (size_t)P.n_panels * sizeof(double)) ||
      !dmalloc((void**)&P.d_sigma_coef32, (size_t)P.n_panels * p * sizeof(float)) ||
      !dmalloc((void**)&P.d_mu_coef32, (size_t)P.n_panels * p * sizeof(float)) ||
      !dmalloc((void**)&P.d_geo_coef_dd, (size_t)P.n_panels * 2 * p * sizeof(float2)) ||
      !dmalloc((void**)&P.d_sigma_coef_dd, (size_t)P.n_panels * p * sizeof(float2)) ||
      !dmalloc((void**)&P.d_mu_coef_dd, (size_t)P.n_panels * p * sizeof(float2)))
    return LP_ERR_NOMEM;
  cudaMemcpy(P.d_bxy, h_xy, nb * 2 * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(P.d_bw, h_w, nb * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(P.d_bnrm, h_nrm, nb * 2 * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(P.d_leg_T, T.data(), T.size() * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(P.d_tau, tau.data(), p * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(P.d_cell_start, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(P.d_cell_near, near.data(), near.size(), cudaMemcpyHostToDevice);
  if (nb) cudaMemcpy(P.d_cell_node, order.data(), nb * sizeof(int), cudaMemcpyHostToDevice);
  if (nb) cudaMemcpy(P.d_cell_xy32, rel.data(), nb * sizeof(float2), cudaMemcpyHostToDevice);
  launch_panel_coef(P, P.d_bxy, 2, 2, P.d_geo_coef, P.d_geo_ref, P.stream);
  launch_to_float(P.d_geo_coef, P.d_geo_coef32, P.n_panels * 2 * p, P.stream);
  launch_split_table(P.d_geo_coef, P.d_geo_coef_dd, P.n_panels * 2 * p, P.stream);
  if (cudaStreamSynchronize(P.stream) != cudaSuccess) return LP_ERR_CUDA;
  return LP_OK;
}

}  // namespace lpg
