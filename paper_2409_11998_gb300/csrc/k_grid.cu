// History part on the periodic grids (Sec. 3, Steps 2-4): type-1 spreading of
// weighted sources with the exponential-of-semicircle kernel, the diagonal
// Fourier multiplier with kernel deconvolution, and type-2 interpolation.
// Each kernel body is a per-item device function shared by the single-plan
// launch (arguments by value) and the batched launch (an array of argument
// records plus a per-block work list, one launch for a whole wave of plans).
#include <cmath>
#include <vector>

#include "lp_internal.cuh"

namespace lpg {

namespace {

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
__device__ __forceinline__ void spread_point(const SpreadArgs<T>& a, int64_t j) {
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

template <typename T, int W>
__global__ void spread_atomic_kernel(const __grid_constant__ SpreadArgs<T> a) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < a.n) spread_point<T, W>(a, j);
}

template <typename T, int W>
__global__ void spread_batch_kernel(const SpreadArgs<T>* __restrict__ args, const int2* __restrict__ work) {
  const int2 wk = work[blockIdx.x];
  const SpreadArgs<T>& a = args[wk.x];
  int64_t j = (int64_t)wk.y + threadIdx.x;
  if (j < a.n) spread_point<T, W>(a, j);
}

// Multiplier on the half spectrum (row index = m_y mod g, column = m_x):
// kept modes |m| <= K get the deconvolved history multiplier, every other
// mode is zeroed.  D channel: multiplier times -i (k1 F1 + k2 F2), the
// source-point derivative of eq. dlpot.
template <typename C, typename R>
__device__ __forceinline__ void multiplier_mode(const MultArgs& a, int64_t idx) {
  const int g = a.g, K = a.K, ncol = g / 2 + 1;
  int row = (int)(idx / ncol), mx = (int)(idx - (int64_t)row * ncol);
  int my = row <= g / 2 ? row : row - g;
  int amy = my < 0 ? -my : my;
  if (sizeof(R) == 4 && a.tab64 && mx < a.klo && amy < a.klo && (mx | amy) != 0) {
    // FP32 plans, low modes: the FP64 entry, products in double, one rounding
    const double md = a.tab64[(size_t)amy * (K + 1) + mx];
    C* chan[2] = {(C*)a.V, (C*)a.S};
    for (C* c : chan)
      if (c) {
        C z = c[idx];
        z.x = (R)((double)z.x * md);
        z.y = (R)((double)z.y * md);
        c[idx] = z;
      }
    if (a.D1) {
      const C z1 = ((C*)a.D1)[idx], z2 = ((const C*)a.D2)[idx];
      const double kx = a.dk * mx, ky = a.dk * my;
      C o;
      o.x = (R)(md * (kx * (double)z1.y + ky * (double)z2.y));
      o.y = (R)(-md * (kx * (double)z1.x + ky * (double)z2.x));
      ((C*)a.D1)[idx] = o;
    }
    return;
  }
  R m = 0;
  if (mx <= K && amy <= K) m = ((const R*)a.tab)[(size_t)amy * (K + 1) + mx];
  if (a.V) {
    C z = ((C*)a.V)[idx];
    z.x *= m;
    z.y *= m;
    ((C*)a.V)[idx] = z;
  }
  if (a.S) {
    C z = ((C*)a.S)[idx];
    z.x *= m;
    z.y *= m;
    ((C*)a.S)[idx] = z;
  }
  if (a.D1) {
    C z1 = ((C*)a.D1)[idx], z2 = ((const C*)a.D2)[idx];
    R kx = (R)(a.dk * mx), ky = (R)(a.dk * my);
    C o;
    o.x = m * (kx * z1.y + ky * z2.y);
    o.y = -m * (kx * z1.x + ky * z2.x);
    ((C*)a.D1)[idx] = o;
  }
}

template <typename C, typename R>
__global__ void multiplier_kernel(const __grid_constant__ MultArgs a) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < (int64_t)a.g * (a.g / 2 + 1)) multiplier_mode<C, R>(a, idx);
}

template <typename C, typename R>
__global__ void multiplier_batch_kernel(const MultArgs* __restrict__ args, const int2* __restrict__ work) {
  const int2 wk = work[blockIdx.x];
  const MultArgs& a = args[wk.x];
  int64_t idx = (int64_t)wk.y * blockDim.x + threadIdx.x;
  if (idx < (int64_t)a.g * (a.g / 2 + 1)) multiplier_mode<C, R>(a, idx);
}

template <typename T, int W>
__device__ __forceinline__ void interp_target(const InterpArgs<T>& a, int64_t i) {
  // FP32 path: the k = 0 term (the log constant) is summed and added in FP64.
  double acc[3] = {0.0, 0.0, 0.0};
  if (a.qsum) {
    acc[0] = a.zero_factor * a.qsum[0];
    acc[1] = a.zero_factor * a.qsum[1];
  }
  bool bad = false;
  for (int l = a.l0; l < 2; ++l) {
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
    if constexpr (sizeof(T) == 4) {
      // single precision: a row is read as W/2 + 1 eight-byte cell pairs from
      // the even cell ix0 at or below ix (rows start 8-byte aligned: the
      // pitch is even), with the x weights shifted once onto the W + 1 cells
      // ix0 .. ix0 + W; the unused end cell (possibly the row's padding, whose
      // bits need not be a finite float) is dropped
      const int ix0 = ix & ~1;
      const bool odd = (ix & 1) != 0;
      T ks[W + 1];
#pragma unroll
      for (int t = 0; t <= W; ++t) {
        const T here = t < W ? kx[t] : T(0), prev = t > 0 ? kx[t - 1] : T(0);
        ks[t] = odd ? prev : here;
      }
      constexpr int NQ = (W + 2) / 2;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T* grid = (const T*)a.grid[l][c];
        if (!grid) continue;
        T s = 0;
#pragma unroll
        for (int b = 0; b < W; ++b) {
          const float2* row = (const float2*)(grid + (size_t)(iy + b) * gd.pitch + ix0);
          float2 q[NQ];
#pragma unroll
          for (int u = 0; u < NQ; ++u) q[u] = __ldg(row + u);
          T r = 0;
#pragma unroll
          for (int t = 0; t <= W; ++t) {
            T v = (t & 1) ? q[t / 2].y : q[t / 2].x;
            if (t == W) v = odd ? v : T(0);
            r = fma(v, ks[t], r);
          }
          s = fma(r, ky[b], s);
        }
        acc[c] += (double)s;
      }
    } else {
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

template <typename T, int W>
__global__ void interp_kernel(const __grid_constant__ InterpArgs<T> a) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) interp_target<T, W>(a, i);
}

template <typename T, int W>
__global__ void interp_batch_kernel(const InterpArgs<T>* __restrict__ args, const int2* __restrict__ work) {
  const int2 wk = work[blockIdx.x];
  const InterpArgs<T>& a = args[wk.x];
  int64_t i = (int64_t)wk.y + threadIdx.x;
  if (i < a.n) interp_target<T, W>(a, i);
}

// Zero a list of buffers (the grids of a wave) in one launch; each work item
// clears kZeroChunk 16-byte words of one segment.
__global__ void zero_batch_kernel(const ZeroSeg* __restrict__ segs, const int2* __restrict__ work) {
  const int2 wk = work[blockIdx.x];
  const ZeroSeg sg = segs[wk.x];
  const int64_t base = (int64_t)wk.y * kZeroChunk;
  float4* p = (float4*)sg.ptr;
  for (int k = threadIdx.x; k < kZeroChunk; k += blockDim.x) {
    int64_t e = base + k;
    if (e < sg.n16) p[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

}  // namespace

GridDev grid_dev(const GridLevel& G) {
  GridDev d;
  d.g = G.g;
  d.pitch = G.pitch;
  d.x0 = G.x0;
  d.y0 = G.y0;
  d.inv_h = 1.0 / G.h;
  return d;
}

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

template <typename T>
SpreadArgs<T> make_spread_args(const Plan& P, int level, const double* xy, const double* const* q, int nq,
                               void* const* grids, int64_t n) {
  SpreadArgs<T> a;
  a.xy = xy;
  for (int c = 0; c < 3; ++c) {
    a.q[c] = c < nq ? q[c] : nullptr;
    a.grid[c] = c < nq ? grids[c] : nullptr;
  }
  a.nq = nq;
  a.n = n;
  a.gd = grid_dev(P.lv[level]);
  a.status = P.d_status;
  if constexpr (sizeof(T) == 8) a.es = P.es; else a.es = P.es32;
  return a;
}
template SpreadArgs<double> make_spread_args<double>(const Plan&, int, const double*, const double* const*,
                                                     int, void* const*, int64_t);
template SpreadArgs<float> make_spread_args<float>(const Plan&, int, const double*, const double* const*,
                                                   int, void* const*, int64_t);

void launch_spread(const Plan& P, int level, const double* xy, const double* const* q, int nq,
                   void* const* grids, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  int threads = 128;
  unsigned blocks = (unsigned)((n + threads - 1) / threads);
  ++P.launches;
  if (P.precision == LP_FP64)
    spread_dispatch(make_spread_args<double>(P, level, xy, q, nq, grids, n), P.ker.w, blocks, threads, s);
  else
    spread_dispatch(make_spread_args<float>(P, level, xy, q, nq, grids, n), P.ker.w, blocks, threads, s);
}

MultArgs make_mult_args(const Plan& P, int level, bool want_v, bool want_s, bool want_d) {
  const GridLevel& G = P.lv[level];
  MultArgs a;
  a.g = G.g;
  a.K = G.K;
  a.dk = G.dk;
  a.tab = P.precision == LP_FP64 ? (const void*)G.mtab : (const void*)G.mtab32;
  a.tab64 = P.precision == LP_FP64 ? nullptr : G.mtab;
  a.klo = P.precision == LP_FP64 ? 0 : kLowKFP64;
  a.V = want_v ? G.chan[0] : nullptr;
  a.S = want_s ? G.chan[1] : nullptr;
  a.D1 = want_d ? G.chan[2] : nullptr;
  a.D2 = want_d ? G.chan[3] : nullptr;
  return a;
}

void launch_multiplier(const Plan& P, int level, bool want_v, bool want_s, bool want_d,
                       cudaStream_t s) {
  const GridLevel& G = P.lv[level];
  int64_t total = (int64_t)G.g * (G.g / 2 + 1);
  int threads = 256;
  unsigned blocks = (unsigned)((total + threads - 1) / threads);
  ++P.launches;
  MultArgs a = make_mult_args(P, level, want_v, want_s, want_d);
  if (P.precision == LP_FP64)
    multiplier_kernel<cufftDoubleComplex, double><<<blocks, threads, 0, s>>>(a);
  else
    multiplier_kernel<cufftComplex, float><<<blocks, threads, 0, s>>>(a);
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

template <typename T>
InterpArgs<T> make_interp_args(const Plan& P, int64_t nt, const double* txy, double* V, double* S, double* D) {
  InterpArgs<T> a;
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
  a.zero_factor = P.lv[0].zero_mode + P.lv[1].zero_mode;  // 0 for an unused level
  a.l0 = P.l0;
  // FP32 path: the zero mode was removed from the FP32 tables
  a.qsum = sizeof(T) == 8 ? nullptr : (P.use_qred ? P.d_qred : P.d_qsum);
  if constexpr (sizeof(T) == 8) a.es = P.es; else a.es = P.es32;
  return a;
}
template InterpArgs<double> make_interp_args<double>(const Plan&, int64_t, const double*, double*, double*, double*);
template InterpArgs<float> make_interp_args<float>(const Plan&, int64_t, const double*, double*, double*, double*);

void launch_interp(const Plan& P, int64_t nt, const double* txy, double* V, double* S, double* D,
                   cudaStream_t s) {
  if (nt <= 0) return;
  int threads = 128;
  unsigned blocks = (unsigned)((nt + threads - 1) / threads);
  ++P.launches;
  if (P.precision == LP_FP64)
    interp_dispatch(make_interp_args<double>(P, nt, txy, V, S, D), P.ker.w, blocks, threads, s);
  else
    interp_dispatch(make_interp_args<float>(P, nt, txy, V, S, D), P.ker.w, blocks, threads, s);
}

// ---- batched launches ---------------------------------------------------------

void launch_zero_batch(const ZeroSeg* d_segs, const int2* d_work, int nwork, cudaStream_t s) {
  if (nwork > 0) zero_batch_kernel<<<nwork, 256, 0, s>>>(d_segs, d_work);
}

void launch_spread_batch(int precision, int w, const void* d_args, const int2* d_work, int nwork,
                         cudaStream_t s) {
  if (nwork <= 0) return;
  switch (w) {
#define LP_CASE(W)                                                                              \
  case W:                                                                                       \
    if (precision == LP_FP64)                                                                   \
      spread_batch_kernel<double, W>                                                            \
          <<<nwork, kBatchThreads, 0, s>>>((const SpreadArgs<double>*)d_args, d_work);          \
    else                                                                                        \
      spread_batch_kernel<float, W><<<nwork, kBatchThreads, 0, s>>>((const SpreadArgs<float>*)d_args, d_work); \
    break;
    LP_WIDTH_CASES(LP_CASE)
#undef LP_CASE
    default: break;
  }
}

void launch_multiplier_batch(int precision, const MultArgs* d_args, const int2* d_work, int nwork,
                             cudaStream_t s) {
  if (nwork <= 0) return;
  if (precision == LP_FP64)
    multiplier_batch_kernel<cufftDoubleComplex, double><<<nwork, kBatchThreads, 0, s>>>(d_args, d_work);
  else
    multiplier_batch_kernel<cufftComplex, float><<<nwork, kBatchThreads, 0, s>>>(d_args, d_work);
}

void launch_interp_batch(int precision, int w, const void* d_args, const int2* d_work, int nwork,
                         cudaStream_t s) {
  if (nwork <= 0) return;
  switch (w) {
#define LP_CASE(W)                                                                              \
  case W:                                                                                       \
    if (precision == LP_FP64)                                                                   \
      interp_batch_kernel<double, W>                                                            \
          <<<nwork, kBatchThreads, 0, s>>>((const InterpArgs<double>*)d_args, d_work);          \
    else                                                                                        \
      interp_batch_kernel<float, W><<<nwork, kBatchThreads, 0, s>>>((const InterpArgs<float>*)d_args, d_work); \
    break;
    LP_WIDTH_CASES(LP_CASE)
#undef LP_CASE
    default: break;
  }
}

}  // namespace lpg
