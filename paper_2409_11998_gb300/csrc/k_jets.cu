// f-jets at targets from the bound node values (lp_volume_jets).  The
// volume expansion of Sec. 4 (eq. vplocO5, and delta f + delta^2/2 lap f
// away from the boundary) needs f and its first and second derivatives at
// each target; the paper computes them analytically (Sec. 6.1).  For a
// caller that has f only at the quadrature nodes, each target gets a
// weighted least-squares quadratic through the nodes within
// rho = sqrt(3 delta_1), weights (1 - r^2/rho^2)^2, basis 1, u, v, u^2,
// u v, v^2 in (u, v) = (y - x)/rho: with at least 10 such nodes; a linear
// fit with 4 to 9; the weighted mean with 1 to 3; a zero jet with none.  At
// a node (within 1e-12 of the box side) the value is that node's f.
//
// Nodes are counting-sorted into square cells of side rho (the cells around
// a target hold every node within rho of it) with single-precision offsets
// from their cell's corner, which prefilter the candidates; the neighbour
// test, the normal equations and their Cholesky solution use the nodes'
// double coordinates: on coarse meshes the fitted value enters delta f at
// full weight.
#include <cmath>

#include "lp_internal.cuh"

namespace lpg {

namespace {

// Cholesky solve of the n x n system (packed upper triangle, row-major:
// A[i][j] for j >= i at idx(i, j)); false if a pivot is not positive.
template <int N>
__device__ bool chol_solve(const double* Ap, const double* bp, double* c) {
  double L[N][N], y[N];
  int k = 0;
  double A[N][N];
  for (int i = 0; i < 6; ++i)
    for (int j = i; j < 6; ++j, ++k)
      if (i < N && j < N) A[i][j] = A[j][i] = Ap[k];
  for (int j = 0; j < N; ++j) {
    double d = A[j][j];
    for (int p = 0; p < j; ++p) d -= L[j][p] * L[j][p];
    if (!(d > 1e-12 * A[0][0])) return false;
    L[j][j] = sqrt(d);
    for (int i = j + 1; i < N; ++i) {
      double s = A[i][j];
      for (int p = 0; p < j; ++p) s -= L[i][p] * L[j][p];
      L[i][j] = s / L[j][j];
    }
  }
  for (int i = 0; i < N; ++i) {
    double s = bp[i];
    for (int p = 0; p < i; ++p) s -= L[i][p] * y[p];
    y[i] = s / L[i][i];
  }
  for (int i = N - 1; i >= 0; --i) {
    double s = y[i];
    for (int p = i + 1; p < N; ++p) s -= L[p][i] * c[p];
    c[i] = s / L[i][i];
  }
  return true;
}

__global__ void jet_fit_kernel(const __grid_constant__ JetArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const double x = a.txy[2 * i], y = a.txy[2 * i + 1];
  double jet[6] = {0, 0, 0, 0, 0, 0};
  const double fxc = (x - a.x0) / a.bt, fyc = (y - a.y0) / a.bt;
  if (fxc >= 0.0 && fxc < a.nbx && fyc >= 0.0 && fyc < a.nby) {
    const int cx = (int)fxc, cy = (int)fyc;
    const double inv_rho = 1.0 / a.rho;
    const float ir = (float)inv_rho;
    double A[21], b[6];
    for (int k = 0; k < 21; ++k) A[k] = 0.0;
    for (int k = 0; k < 6; ++k) b[k] = 0.0;
    int cnt = 0, bestk = -1;
    float best = 2.f;
    for (int yy = max(cy - 1, 0); yy <= min(cy + 1, a.nby - 1); ++yy)
      for (int xx = max(cx - 1, 0); xx <= min(cx + 1, a.nbx - 1); ++xx) {
        const int key = yy * a.nbx + xx;
        // the target relative to this cell's corner, in units of rho
        const double tx = (x - (a.x0 + xx * a.bt)) * inv_rho;
        const double ty = (y - (a.y0 + yy * a.bt)) * inv_rho;
        for (int k = a.start[key]; k < a.start[key + 1]; ++k) {
          const float2 r = a.rel[k];
          const float u = fmaf(r.x, ir, -(float)tx), v = fmaf(r.y, ir, -(float)ty);
          const float r2 = fmaf(u, u, v * v);
          if (!(r2 < 1.0001f)) continue;
          const int j = a.perm[k];
          const double ud = (a.vxy[2 * j] - x) * inv_rho, vd = (a.vxy[2 * j + 1] - y) * inv_rho;
          const double r2d = ud * ud + vd * vd;
          if (!(r2d < 1.0)) continue;
          ++cnt;
          if (r2 < best) {
            best = r2;
            bestk = k;
          }
          const double wgt = (1.0 - r2d) * (1.0 - r2d);
          const double ph[6] = {1.0, ud, vd, ud * ud, ud * vd, vd * vd};
          const double wf = wgt * a.vf[j];
          int q = 0;
#pragma unroll
          for (int s = 0; s < 6; ++s) {
            const double ws = wgt * ph[s];
#pragma unroll
            for (int t = s; t < 6; ++t, ++q) A[q] = fma(ws, ph[t], A[q]);
            b[s] = fma(wf, ph[s], b[s]);
          }
        }
      }
    double c[6] = {0, 0, 0, 0, 0, 0};
    bool ok = false;
    int nb = 0;
    if (cnt >= 10 && chol_solve<6>(A, b, c)) {
      ok = true;
      nb = 6;
    }
    if (!ok && cnt >= 4 && chol_solve<3>(A, b, c)) {
      ok = true;
      nb = 3;
    }
    if (!ok && cnt >= 1) {
      c[0] = b[0] / A[0];
      ok = true;
      nb = 1;
    }
    if (ok) {
      jet[0] = c[0];
      if (nb >= 3) {
        jet[1] = c[1] * inv_rho;
        jet[2] = c[2] * inv_rho;
      }
      if (nb == 6) {
        jet[3] = 2.0 * c[3] * inv_rho * inv_rho;
        jet[4] = c[4] * inv_rho * inv_rho;
        jet[5] = 2.0 * c[5] * inv_rho * inv_rho;
      }
      const int j = a.perm[bestk];
      const double dx = a.vxy[2 * j] - x, dy = a.vxy[2 * j + 1] - y;
      if (sqrt(dx * dx + dy * dy) <= a.on_tol) jet[0] = a.vf[j];
    }
  }
  for (int k = 0; k < 6; ++k) a.jet[6 * i + k] = jet[k];
}

}  // namespace

void launch_jet_fit(const JetArgs& a, cudaStream_t s) {
  if (a.n <= 0) return;
  jet_fit_kernel<<<(unsigned)((a.n + 127) / 128), 128, 0, s>>>(a);
}

}  // namespace lpg
