// History part on the periodic grids (Sec. 3, Steps 2-4): type-1 spreading of
// weighted sources with the exponential-of-semicircle kernel, the diagonal
// Fourier multiplier with kernel deconvolution, and type-2 interpolation.
#include <cmath>

#include "lp_internal.cuh"

namespace lpg {

namespace {

struct SpreadArgs {
  const double* xy;
  const double* q[3];
  void* grid[3];
  int nq;
  int64_t n;
  GridDev gd;
  Kernel ker;
  unsigned* status;
};

__device__ __forceinline__ double es_phi(double z, double beta) {
  double a = 1.0 - z * z;
  return a > 0.0 ? exp(beta * (sqrt(a) - 1.0)) : 0.0;
}
__device__ __forceinline__ float es_phi_f(float z, float beta) {
  float a = 1.0f - z * z;
  return a > 0.0f ? __expf(beta * (sqrtf(a) - 1.0f)) : 0.0f;
}

// Grid coordinate split: first stencil index i0 = floor(u - w/2) + 1 and the
// offset d0 = u - i0 of the point from it (in [w/2 - 1, w/2)).
__device__ __forceinline__ bool stencil_origin(double u, int w, double hw, int g, int& i0, double& d0) {
  if (!(u > -1e9 && u < 1e9)) return false;  // rejects NaN / inf
  double f = floor(u - hw);
  i0 = (int)f + 1;
  d0 = u - (double)i0;
  return i0 >= 0 && i0 + w <= g;
}

template <typename T>
__global__ void spread_atomic_kernel(SpreadArgs a) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.n) return;
  const int w = a.ker.w;
  const double hw = a.ker.half_w;
  double ux = (a.xy[2 * j] - a.gd.x0) * a.gd.inv_h;
  double uy = (a.xy[2 * j + 1] - a.gd.y0) * a.gd.inv_h;
  int ix, iy;
  double dx, dy;
  if (!stencil_origin(ux, w, hw, a.gd.g, ix, dx) || !stencil_origin(uy, w, hw, a.gd.g, iy, dy)) {
    atomicOr(a.status, kStatusOutOfBox);
    return;
  }
  T kx[kMaxW], ky[kMaxW];
  const double inv_hw = 1.0 / hw;
  for (int t = 0; t < w; ++t) {
    if (sizeof(T) == 8) {
      kx[t] = (T)es_phi((dx - t) * inv_hw, a.ker.beta);
      ky[t] = (T)es_phi((dy - t) * inv_hw, a.ker.beta);
    } else {
      kx[t] = (T)es_phi_f((float)((dx - t) * inv_hw), (float)a.ker.beta);
      ky[t] = (T)es_phi_f((float)((dy - t) * inv_hw), (float)a.ker.beta);
    }
  }
  for (int c = 0; c < a.nq; ++c) {
    T qv = (T)a.q[c][j];
    T* grid = (T*)a.grid[c];
    for (int b = 0; b < w; ++b) {
      T qb = qv * ky[b];
      T* row = grid + (size_t)(iy + b) * a.gd.pitch + ix;
      for (int t = 0; t < w; ++t) atomicAdd(row + t, qb * kx[t]);
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

struct InterpArgs {
  const double* txy;
  int64_t n;
  const void* grid[2][3];  // [level][V,S,D]
  GridDev gd[2];
  const double* qsum;      // FP64 strength sums of V and S (FP32 path), or null
  double zero_factor;      // sum over levels of (dk/2pi)^2 M(0)
  Kernel ker;
  double* out[3];
  unsigned* status;
};

template <typename T>
__global__ void interp_kernel(InterpArgs a) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int w = a.ker.w;
  const double hw = a.ker.half_w, inv_hw = 1.0 / hw;
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
    if (!stencil_origin(ux, w, hw, gd.g, ix, dx) || !stencil_origin(uy, w, hw, gd.g, iy, dy)) {
      bad = true;
      break;
    }
    T kx[kMaxW], ky[kMaxW];
    for (int t = 0; t < w; ++t) {
      if (sizeof(T) == 8) {
        kx[t] = (T)es_phi((dx - t) * inv_hw, a.ker.beta);
        ky[t] = (T)es_phi((dy - t) * inv_hw, a.ker.beta);
      } else {
        kx[t] = (T)es_phi_f((float)((dx - t) * inv_hw), (float)a.ker.beta);
        ky[t] = (T)es_phi_f((float)((dy - t) * inv_hw), (float)a.ker.beta);
      }
    }
    for (int c = 0; c < 3; ++c) {
      const T* grid = (const T*)a.grid[l][c];
      if (!grid) continue;
      T s = 0;
      for (int b = 0; b < w; ++b) {
        const T* row = grid + (size_t)(iy + b) * gd.pitch + ix;
        T r = 0;
        for (int t = 0; t < w; ++t) r += row[t] * kx[t];
        s += r * ky[b];
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

void launch_spread(const Plan& P, int level, const double* xy, const double* const* q, int nq,
                   void* const* grids, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  SpreadArgs a;
  a.xy = xy;
  for (int c = 0; c < 3; ++c) {
    a.q[c] = c < nq ? q[c] : nullptr;
    a.grid[c] = c < nq ? grids[c] : nullptr;
  }
  a.nq = nq;
  a.n = n;
  a.gd = grid_dev(P.lv[level]);
  a.ker = P.ker;
  a.status = P.d_status;
  int threads = 128;
  unsigned blocks = (unsigned)((n + threads - 1) / threads);
  ++P.launches;
  if (P.precision == LP_FP64)
    spread_atomic_kernel<double><<<blocks, threads, 0, s>>>(a);
  else
    spread_atomic_kernel<float><<<blocks, threads, 0, s>>>(a);
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

void launch_interp(const Plan& P, int64_t nt, const double* txy, double* V, double* S, double* D,
                   cudaStream_t s) {
  if (nt <= 0) return;
  InterpArgs a;
  a.txy = txy;
  a.n = nt;
  a.ker = P.ker;
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
  int threads = 128;
  unsigned blocks = (unsigned)((nt + threads - 1) / threads);
  ++P.launches;
  if (P.precision == LP_FP64) {
    interp_kernel<double><<<blocks, threads, 0, s>>>(a);
  } else {
    // FP32 path: the zero mode was removed from the FP32 tables
    a.qsum = P.d_qsum;
    interp_kernel<float><<<blocks, threads, 0, s>>>(a);
  }
}

}  // namespace lpg
