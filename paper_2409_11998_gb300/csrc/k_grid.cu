// History part on the periodic grids (Sec. 3, Steps 2-4): type-1 spreading of
// weighted sources with the exponential-of-semicircle kernel, the diagonal
// Fourier multiplier with kernel deconvolution, and type-2 interpolation.
#include <cmath>

#include "lp_internal.cuh"

namespace lpg {

namespace {

template <typename T>
struct SpreadArgs {
  const double* xy;
  const double* q[3];
  void* grid[3];
  int nq;
  int64_t n;
  GridDev gd;
  unsigned* status;
  EsPoly<T> es;
};

// Grid coordinate split: first stencil index i0 = floor(u - w/2) + 1 and the
// offset d0 = u - i0 of the point from it (in [w/2 - 1, w/2)).
__device__ __forceinline__ bool stencil_origin(double u, int w, int g, int& i0, double& d0) {
  if (!(u > -1e9 && u < 1e9)) return false;  // rejects NaN / inf
  double f = floor(u - 0.5 * w);
  i0 = (int)f + 1;
  d0 = u - (double)i0;
  return i0 >= 0 && i0 + w <= g;
}

// The W stencil weights of one dimension (Horner on the plan's polynomials).
template <typename T, int W>
__device__ __forceinline__ void es_weights(const EsPoly<T>& P, T v, T* out) {
#pragma unroll
  for (int t = 0; t < W; ++t) out[t] = P.c[P.nc - 1][t];
  for (int k = P.nc - 2; k >= 0; --k) {
#pragma unroll
    for (int t = 0; t < W; ++t) out[t] = fma(out[t], v, P.c[k][t]);
  }
}

template <typename T, int W>
__global__ void spread_atomic_kernel(const __grid_constant__ SpreadArgs<T> a) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.n) return;
  double ux = (a.xy[2 * j] - a.gd.x0) * a.gd.inv_h;
  double uy = (a.xy[2 * j + 1] - a.gd.y0) * a.gd.inv_h;
  int ix, iy;
  double dx, dy;
  if (!stencil_origin(ux, W, a.gd.g, ix, dx) || !stencil_origin(uy, W, a.gd.g, iy, dy)) {
    atomicOr(a.status, kStatusOutOfBox);
    return;
  }
  T kx[W], ky[W];
  es_weights<T, W>(a.es, (T)(dx - 0.5 * (W - 1)), kx);
  es_weights<T, W>(a.es, (T)(dy - 0.5 * (W - 1)), ky);
  for (int c = 0; c < a.nq; ++c) {
    T qv = (T)a.q[c][j];
    T* grid = (T*)a.grid[c];
#pragma unroll
    for (int b = 0; b < W; ++b) {
      T qb = qv * ky[b];
      T* row = grid + (size_t)(iy + b) * a.gd.pitch + ix;
#pragma unroll
      for (int t = 0; t < W; ++t) atomicAdd(row + t, qb * kx[t]);
    }
  }
}

template <typename C, typename R>
__global__ void multiplier_kernel(int g, int K, double dk, const R* __restrict__ tab, C* V, C* S,
                                  C* D1, const C* __restrict__ D2) {
  const int ncol = g / 2 + 1;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)g * ncol) return;
  int row = (int)(idx / ncol), mx = (int)(idx - (int64_t)row * ncol);
  int my = row <= g / 2 ? row : row - g;
  int amy = my < 0 ? -my : my;
  R m = 0;
  if (mx <= K && amy <= K) m = tab[(size_t)amy * (K + 1) + mx];
  if (V) {
    C z = V[idx];
    z.x *= m;
    z.y *= m;
    V[idx] = z;
  }
  if (S) {
    C z = S[idx];
    z.x *= m;
    z.y *= m;
    S[idx] = z;
  }
  if (D1) {
    // D channel: multiplier times -i (k1 F1 + k2 F2), derivative in the
    // source point (eq. dlpot convention).
    C z1 = D1[idx], z2 = D2[idx];
    R kx = (R)(dk * mx), ky = (R)(dk * my);
    C o;
    o.x = m * (kx * z1.y + ky * z2.y);
    o.y = -m * (kx * z1.x + ky * z2.x);
    D1[idx] = o;
  }
}

template <typename T>
struct InterpArgs {
  const double* txy;
  int64_t n;
  const void* grid[2][3];  // [level][V,S,D]
  GridDev gd[2];
  const double* qsum;      // FP64 strength sums of V and S (FP32 path), or null
  double zero_factor;      // sum over levels of (dk/2pi)^2 M(0)
  double* out[3];
  unsigned* status;
  EsPoly<T> es;
};

template <typename T, int W>
__global__ void interp_kernel(const __grid_constant__ InterpArgs<T> a) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  // FP32 path: the k = 0 term (the log constant) is summed and added in FP64.
  double acc[3] = {0.0, 0.0, 0.0};
  if (a.qsum) {
    acc[0] = a.zero_factor * a.qsum[0];
    acc[1] = a.zero_factor * a.qsum[1];
  }
  bool bad = false;
  for (int l = 0; l < 2; ++l) {
    const GridDev gd = a.gd[l];
    double ux = (a.txy[2 * i] - gd.x0) * gd.inv_h;
    double uy = (a.txy[2 * i + 1] - gd.y0) * gd.inv_h;
    int ix, iy;
    double dx, dy;
    if (!stencil_origin(ux, W, gd.g, ix, dx) || !stencil_origin(uy, W, gd.g, iy, dy)) {
      bad = true;
      break;
    }
    T kx[W], ky[W];
    es_weights<T, W>(a.es, (T)(dx - 0.5 * (W - 1)), kx);
    es_weights<T, W>(a.es, (T)(dy - 0.5 * (W - 1)), ky);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T* grid = (const T*)a.grid[l][c];
      if (!grid) continue;
      T s = 0;
#pragma unroll
      for (int b = 0; b < W; ++b) {
        const T* row = grid + (size_t)(iy + b) * gd.pitch + ix;
        T r = 0;
#pragma unroll
        for (int t = 0; t < W; ++t) r = fma(row[t], kx[t], r);
        s = fma(r, ky[b], s);
      }
      acc[c] += (double)s;
    }
  }
  if (bad) {
    atomicOr(a.status, kStatusOutOfBox);
    for (int c = 0; c < 3; ++c)
      if (a.out[c]) a.out[c][i] = 0.0;
    return;
  }
  for (int c = 0; c < 3; ++c)
    if (a.out[c]) a.out[c][i] = acc[c];
}

GridDev grid_dev(const GridLevel& G) {
  GridDev d;
  d.g = G.g;
  d.pitch = G.pitch;
  d.x0 = G.x0;
  d.y0 = G.y0;
  d.inv_h = 1.0 / G.h;
  return d;
}

}  // namespace

#define LP_WIDTH_CASES(X) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

template <typename T>
static void spread_dispatch(const SpreadArgs<T>& a, int w, unsigned blocks, int threads, cudaStream_t s) {
  switch (w) {
#define LP_CASE(W) \
  case W:          \
    spread_atomic_kernel<T, W><<<blocks, threads, 0, s>>>(a); \
    break;
    LP_WIDTH_CASES(LP_CASE)
#undef LP_CASE
    default: break;
  }
}

void launch_spread(const Plan& P, int level, const double* xy, const double* const* q, int nq,
                   void* const* grids, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  int threads = 128;
  unsigned blocks = (unsigned)((n + threads - 1) / threads);
  ++P.launches;
  auto fill = [&](auto& a) {
    a.xy = xy;
    for (int c = 0; c < 3; ++c) {
      a.q[c] = c < nq ? q[c] : nullptr;
      a.grid[c] = c < nq ? grids[c] : nullptr;
    }
    a.nq = nq;
    a.n = n;
    a.gd = grid_dev(P.lv[level]);
    a.status = P.d_status;
  };
  if (P.precision == LP_FP64) {
    SpreadArgs<double> a;
    fill(a);
    a.es = P.es;
    spread_dispatch(a, P.ker.w, blocks, threads, s);
  } else {
    SpreadArgs<float> a;
    fill(a);
    a.es = P.es32;
    spread_dispatch(a, P.ker.w, blocks, threads, s);
  }
}

void launch_multiplier(const Plan& P, int level, bool want_v, bool want_s, bool want_d,
                       cudaStream_t s) {
  const GridLevel& G = P.lv[level];
  int64_t total = (int64_t)G.g * (G.g / 2 + 1);
  int threads = 256;
  unsigned blocks = (unsigned)((total + threads - 1) / threads);
  ++P.launches;
  if (P.precision == LP_FP64) {
    using C = cufftDoubleComplex;
    multiplier_kernel<C, double><<<blocks, threads, 0, s>>>(
        G.g, G.K, G.dk, G.mtab, want_v ? (C*)G.chan[0] : nullptr, want_s ? (C*)G.chan[1] : nullptr,
        want_d ? (C*)G.chan[2] : nullptr, want_d ? (const C*)G.chan[3] : nullptr);
  } else {
    using C = cufftComplex;
    multiplier_kernel<C, float><<<blocks, threads, 0, s>>>(
        G.g, G.K, G.dk, G.mtab32, want_v ? (C*)G.chan[0] : nullptr, want_s ? (C*)G.chan[1] : nullptr,
        want_d ? (C*)G.chan[2] : nullptr, want_d ? (const C*)G.chan[3] : nullptr);
  }
}

template <typename T>
static void interp_dispatch(const InterpArgs<T>& a, int w, unsigned blocks, int threads, cudaStream_t s) {
  switch (w) {
#define LP_CASE(W) \
  case W:          \
    interp_kernel<T, W><<<blocks, threads, 0, s>>>(a); \
    break;
    LP_WIDTH_CASES(LP_CASE)
#undef LP_CASE
    default: break;
  }
}

void launch_interp(const Plan& P, int64_t nt, const double* txy, double* V, double* S, double* D,
                   cudaStream_t s) {
  if (nt <= 0) return;
  auto fill = [&](auto& a) {
    a.txy = txy;
    a.n = nt;
    a.status = P.d_status;
    a.out[0] = V;
    a.out[1] = S;
    a.out[2] = D;
    for (int l = 0; l < 2; ++l) {
      a.gd[l] = grid_dev(P.lv[l]);
      for (int c = 0; c < 3; ++c) a.grid[l][c] = a.out[c] ? P.lv[l].chan[c] : nullptr;
    }
    a.qsum = nullptr;
    a.zero_factor = P.lv[0].zero_mode + P.lv[1].zero_mode;
  };
  int threads = 128;
  unsigned blocks = (unsigned)((nt + threads - 1) / threads);
  ++P.launches;
  if (P.precision == LP_FP64) {
    InterpArgs<double> a;
    fill(a);
    a.es = P.es;
    interp_dispatch(a, P.ker.w, blocks, threads, s);
  } else {
    // FP32 path: the zero mode was removed from the FP32 tables
    InterpArgs<float> a;
    fill(a);
    a.es = P.es32;
    a.qsum = P.d_qsum;
    interp_dispatch(a, P.ker.w, blocks, threads, s);
  }
}

}  // namespace lpg
