// Small device kernels: panel Legendre coefficients, source strengths
// (Sec. 3, input: f w for volume nodes, sigma w and mu nu w for boundary
// nodes) and FP64 strength sums.
#include "lp_internal.cuh"

namespace lpg {

namespace {

// coef[(ip*ncomp + comp)*p + k] = sum_i T[k][i] (v_i - v_ref), v_ref = middle
// node; ref[ip*ncomp + comp] = v_ref.  Interpolating the centred values keeps
// the rounding of high derivatives at the size of the panel's variation.
__global__ void panel_coef_kernel(const double* __restrict__ vals, int stride, int ncomp, int p,
                                  int64_t n_panels, const double* __restrict__ T, double* coef,
                                  double* ref) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = n_panels * ncomp * p;
  if (idx >= total) return;
  int k = (int)(idx % p);
  int64_t pc = idx / p;
  int comp = (int)(pc % ncomp);
  int64_t ip = pc / ncomp;
  const double* v = vals + (size_t)ip * p * stride + comp;
  double vr = v[(size_t)(p / 2) * stride];
  double s = 0.0;
  for (int i = 0; i < p; ++i) s += T[(size_t)k * p + i] * (v[(size_t)i * stride] - vr);
  coef[idx] = s;
  if (k == 0) ref[pc] = vr;
}

__global__ void strengths_kernel(int kind, const double* __restrict__ dens, const double* __restrict__ w,
                                 const double* __restrict__ nrm, double* bq, int64_t nb) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  double dw = dens[j] * w[j];
  if (kind == 0) {
    bq[j] = dw;
  } else {
    bq[nb + j] = dw * nrm[2 * j];
    bq[2 * nb + j] = dw * nrm[2 * j + 1];
  }
}

__global__ void volume_q_kernel(const double* __restrict__ f, const double* __restrict__ w, double* q,
                                int64_t n) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) q[j] = f[j] * w[j];
}

__global__ void sum_kernel(const double* __restrict__ x, int64_t n, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    s += x[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(out, s);
  }
}

// Deconvolved history multiplier (eq. vnearkspace; eq. vfarkspace with W of
// eq. Wdef) on the kept modes, tab[my][mx] = scale M(dk |m|) / (ph[mx] ph[my])^2;
// the FP32 copy omits the k = 0 entry (its term is added in FP64).
__device__ double one_minus_j0_dev(double z) {
  if (z < 2.0) {  // power series: no cancellation at small z
    double q = 0.25 * z * z, term = 1.0, s = 0.0;
    for (int k = 1; k < 40; ++k) {
      term *= -q / ((double)k * k);
      s -= term;
      if (fabs(term) < 1e-18 * fabs(s)) break;
    }
    return s;
  }
  return 1.0 - j0(z);
}
__device__ double j1_over_z_dev(double z) {
  if (z < 2.0) {
    double q = 0.25 * z * z, term = 0.5, s = 0.5;
    for (int k = 1; k < 40; ++k) {
      term *= -q / ((double)k * (k + 1));
      s += term;
      if (fabs(term) < 1e-18 * fabs(s)) break;
    }
    return s;
  }
  return j1(z) / z;
}

__global__ void mult_table_kernel(int kind, int K, double dk, double d1, double d2, double L, double scale,
                                  const double* __restrict__ ph, double* tab, float* tab32) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n = (int64_t)(K + 1) * (K + 1);
  if (idx >= n) return;
  int my = (int)(idx / (K + 1)), mx = (int)(idx - (int64_t)my * (K + 1));
  double k = dk * sqrt((double)mx * mx + (double)my * my);
  double M;
  if (kind == 0) {
    M = (k == 0.0) ? (d2 - d1) : (expm1(-k * k * d1) - expm1(-k * k * d2)) / (k * k);
  } else {
    double z = L * k;
    double W = (z == 0.0) ? 0.25 * L * L : L * L * (one_minus_j0_dev(z) / (z * z));
    W -= L * L * log(L) * j1_over_z_dev(z);
    M = exp(-k * k * d2) * W;
  }
  double d = ph[mx] * ph[my];
  double v = scale * M / (d * d);
  tab[idx] = v;
  tab32[idx] = (idx == 0) ? 0.0f : (float)v;
}

__global__ void to_float_kernel(const double* __restrict__ src, float* dst, int64_t n) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) dst[j] = (float)src[j];
}

}  // namespace

void launch_mult_table(int kind, int K, double dk, double d1, double d2, double L, double scale,
                       const double* d_ph, double* tab, float* tab32, cudaStream_t s) {
  int64_t n = (int64_t)(K + 1) * (K + 1);
  mult_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(kind, K, dk, d1, d2, L, scale, d_ph, tab,
                                                                 tab32);
}

void launch_to_float(const double* src, float* dst, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  to_float_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
}

void launch_panel_coef(const Plan& P, const double* vals, int stride, int ncomp, double* coef,
                       double* ref, cudaStream_t s) {
  int64_t total = P.n_panels * ncomp * P.p;
  if (total <= 0) return;
  int threads = 128;
  ++P.launches;
  panel_coef_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, s>>>(
      vals, stride, ncomp, P.p, P.n_panels, P.d_leg_T, coef, ref);
}

void launch_strengths(const Plan& P, int kind, cudaStream_t s) {
  if (P.nb <= 0) return;
  int threads = 256;
  const double* dens = kind == 0 ? P.d_sigma : P.d_mu;
  ++P.launches;
  strengths_kernel<<<(unsigned)((P.nb + threads - 1) / threads), threads, 0, s>>>(
      kind, dens, P.d_bw, P.d_bnrm, P.d_bq, P.nb);
}

void launch_volume_q(const Plan& P, const double* f, const double* w, double* q, int64_t n,
                     cudaStream_t s) {
  if (n <= 0) return;
  int threads = 256;
  ++P.launches;
  volume_q_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(f, w, q, n);
}

void launch_sum(const Plan& P, const double* x, int64_t n, double* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(double), s);
  if (n <= 0) return;
  int threads = 256;
  int64_t blocks = (n + threads - 1) / threads;
  if (blocks > 1024) blocks = 1024;
  ++P.launches;
  sum_kernel<<<(unsigned)blocks, threads, 0, s>>>(x, n, out);
}

}  // namespace lpg
