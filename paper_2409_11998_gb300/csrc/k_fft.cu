// FFT chain of the FP64 plans in double-float arithmetic (Sec. 3, Steps 2-4:
// forward transform of the spread grids, diagonal multiplier, inverse
// transform), replacing FP64 cuFFT, which on GB300 is bound by the FP64 units.
//
//   rows_fwd  real grid rows [row_lo, row_hi) (FP64, as spread) -> kept modes
//             0..K of each row's half spectrum, df64 complex, [g][Kp]
//   cols      per kept column m_x: forward transform along y, the
//             deconvolved multiplier (V, S: M F; D: M (-i)(k1 F1 + k2 F2)),
//             inverse transform along y -- the column never leaves shared
//             memory between the two transforms
//   rows_inv  rows [row_lo, row_hi) of the half spectrum -> real grid rows,
//             written in place over the FP64 grid as df64 (hi, lo) pairs
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
#include <cmath>
#include <vector>

#include "df64.cuh"
#include "lp_internal.cuh"

namespace lpg {

namespace {

// sqrt(3)/2 = kS3h + kS3l (float(sqrt(3)/2) and the float of the remainder)
constexpr float kS3h = 0.8660253882408142f;
constexpr float kS3l = 1.5543625053737742e-08f;

template <int R>
__device__ __forceinline__ void dft_small(cdd* v, bool inv) {
  if (R == 2) {
    const cdd a = v[0], b = v[1];
    v[0] = cdd_add(a, b);
    v[1] = cdd_sub(a, b);
  } else if (R == 4) {
    const cdd t0 = cdd_add(v[0], v[2]), t1 = cdd_sub(v[0], v[2]);
    const cdd t2 = cdd_add(v[1], v[3]);
    const cdd d = cdd_sub(v[1], v[3]);
    const cdd t3 = inv ? cdd_mul_pi(d) : cdd_mul_mi(d);
    v[0] = cdd_add(t0, t2);
    v[1] = cdd_add(t1, t3);
    v[2] = cdd_sub(t0, t2);
    v[3] = cdd_sub(t1, t3);
  } else {  // R == 3
    const cdd t1 = cdd_add(v[1], v[2]);
    const cdd t2 = cdd_sub(v[0], cdd{dd_scale(t1.re, 0.5f), dd_scale(t1.im, 0.5f)});
    const cdd d = cdd_sub(v[1], v[2]);
    const dd s3 = dd_make(kS3h, kS3l);
    const cdd ds = cdd{dd_mul(d.re, s3), dd_mul(d.im, s3)};
    const cdd t3 = inv ? cdd_mul_pi(ds) : cdd_mul_mi(ds);
    v[0] = cdd_add(v[0], t1);
    v[1] = cdd_add(t2, t3);
    v[2] = cdd_sub(t2, t3);
  }
}

template <int R>
__device__ __forceinline__ void stockham_butterfly(const float4* in, float4* out, int j, int N, int Ns,
                                                   const float4* __restrict__ tw, int tws, bool inv) {
  const int stride = N / R;
  cdd v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = cdd_load(in + j + r * stride);
  const int k = j % Ns;
  if (k != 0) {
    const int step = (N / (Ns * R)) * tws;
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const cdd t = cdd_load(tw + k * r * step);
      v[r] = inv ? cdd_mul_conj(v[r], t) : cdd_mul(v[r], t);
    }
  }
  dft_small<R>(v, inv);
  const int base = (j - k) * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r) cdd_store(out + base + r * Ns, v[r]);
}

// Transform of length N held in a (scratch b); returns the buffer holding
// the result.  All threads of the CTA take part; the caller synchronises
// before (data in a) and the function synchronises after every stage.
__device__ float4* fft_smem(float4* a, float4* b, const FftShape& sh, const float4* __restrict__ tw, int tws,
                            bool inv) {
  const int N = sh.n;
  int Ns = 1;
  for (int s = 0; s < sh.nst; ++s) {
    const int R = sh.radix[s];
    const int nb = N / R;
    if (R == 4) {
      for (int j = threadIdx.x; j < nb; j += blockDim.x) stockham_butterfly<4>(a, b, j, N, Ns, tw, tws, inv);
    } else if (R == 2) {
      for (int j = threadIdx.x; j < nb; j += blockDim.x) stockham_butterfly<2>(a, b, j, N, Ns, tw, tws, inv);
    } else {
      for (int j = threadIdx.x; j < nb; j += blockDim.x) stockham_butterfly<3>(a, b, j, N, Ns, tw, tws, inv);
    }
    __syncthreads();
    float4* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

__device__ __forceinline__ cdd cdd_zero() { return cdd{dd{0.f, 0.f}, dd{0.f, 0.f}}; }

// Forward transform of real rows: one CTA per (row, channel).
__global__ void __launch_bounds__(kFftThreads) fft_rows_fwd_kernel(const __grid_constant__ FftRowArgs a) {
  extern __shared__ float4 sm[];
  const int N = a.half.n;
  const int row = a.row_lo + blockIdx.x, c = blockIdx.y;
  const double* src = (const double*)a.grid[c] + (size_t)row * a.pitch;
  float4* buf0 = sm;
  float4* buf1 = sm + N;
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    const double2 x = *(const double2*)(src + 2 * n);
    cdd_store(buf0 + n, cdd{dd_from_double(x.x), dd_from_double(x.y)});
  }
  __syncthreads();
  const float4* Z = fft_smem(buf0, buf1, a.half, a.tw, 2, false);
  float4* dst = a.spec[c] + (size_t)row * a.kp;
  for (int k = threadIdx.x; k <= a.K; k += blockDim.x) {
    const cdd zk = cdd_load(Z + k), zn = cdd_conj(cdd_load(Z + (k == 0 ? 0 : N - k)));
    const cdd s = cdd_add(zk, zn), d = cdd_sub(zk, zn);
    const cdd e = cdd{dd_scale(s.re, 0.5f), dd_scale(s.im, 0.5f)};
    const cdd o = cdd_mul_mi(cdd{dd_scale(d.re, 0.5f), dd_scale(d.im, 0.5f)});
    cdd_store(dst + k, cdd_add(e, cdd_mul(cdd_load(a.tw + k), o)));
  }
}

// Column pass: one CTA per (kept column m_x, job).  Jobs of kind 0 transform
// one spectrum and multiply by M; kind 1 (D) transforms two and combines
// them, parking the first transform in its own (global) column meanwhile so
// that every job needs only two shared-memory buffers of g values.
__global__ void __launch_bounds__(kFftThreads) fft_cols_kernel(const __grid_constant__ FftColArgs a) {
  extern __shared__ float4 sm[];
  const int g = a.full.n, K = a.K, mx = blockIdx.x;
  const FftColJob& job = a.job[blockIdx.y];
  float4* buf0 = sm;
  float4* buf1 = sm + g;
  auto load_col = [&](const float4* spec) {
    for (int r = threadIdx.x; r < g; r += blockDim.x) {
      if (r >= a.row_lo && r < a.row_hi)
        buf0[r] = spec[(size_t)r * a.kp + mx];
      else
        cdd_store(buf0 + r, cdd_zero());
    }
    __syncthreads();
  };
  const dd dk = dd_make(a.dk.x, a.dk.y);
  float4* X;
  if (job.kind == 1) {
    load_col(job.in[0]);
    const float4* F1 = fft_smem(buf0, buf1, a.full, a.tw, 1, false);
    float4* park = job.out;  // the D1 spectrum column, all g rows
    for (int r = threadIdx.x; r < g; r += blockDim.x) park[(size_t)r * a.kp + mx] = F1[r];
    __syncthreads();
    load_col(job.in[1]);
    X = fft_smem(buf0, buf1, a.full, a.tw, 1, false);
    const dd kx = dd_mul_f(dk, (float)mx);
    for (int r = threadIdx.x; r < g; r += blockDim.x) {
      const int my = r <= g / 2 ? r : r - g;
      const int amy = my < 0 ? -my : my;
      cdd o = cdd_zero();
      if (amy <= K) {
        const float2 mt = a.tab[(size_t)amy * (K + 1) + mx];
        const dd m = dd_make(mt.x, mt.y);
        const dd ky = dd_mul_f(dk, (float)my);
        const cdd f1 = cdd_load(park + (size_t)r * a.kp + mx), f2 = cdd_load(X + r);
        // m (-i)(kx f1 + ky f2)
        const dd re = dd_dot2(kx, f1.im, ky, f2.im);
        const dd im = dd_dot2(kx, f1.re, ky, f2.re);
        o = cdd{dd_mul(m, re), dd_neg(dd_mul(m, im))};
      }
      cdd_store(X + r, o);
    }
  } else {
    load_col(job.in[0]);
    X = fft_smem(buf0, buf1, a.full, a.tw, 1, false);
    for (int r = threadIdx.x; r < g; r += blockDim.x) {
      const int my = r <= g / 2 ? r : r - g;
      const int amy = my < 0 ? -my : my;
      cdd o = cdd_zero();
      if (amy <= K) {
        const float2 mt = a.tab[(size_t)amy * (K + 1) + mx];
        o = cdd_scale_dd(cdd_load(X + r), dd_make(mt.x, mt.y));
      }
      cdd_store(X + r, o);
    }
  }
  __syncthreads();
  const float4* Y = fft_smem(X, X == buf0 ? buf1 : buf0, a.full, a.tw, 1, true);
  for (int r = a.row_lo + threadIdx.x; r < a.row_hi; r += blockDim.x) job.out[(size_t)r * a.kp + mx] = Y[r];
}

// Inverse transform of rows: one CTA per (row, job); writes g df64 values
// over the row of the job's FP64 grid.
__global__ void __launch_bounds__(kFftThreads) fft_rows_inv_kernel(const __grid_constant__ FftRowArgs a) {
  extern __shared__ float4 sm[];
  const int N = a.half.n;
  const int row = a.row_lo + blockIdx.x, c = blockIdx.y;
  const float4* spec = a.spec[c] + (size_t)row * a.kp;
  float4* buf0 = sm;
  float4* buf1 = sm + N;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    cdd xk = k <= a.K ? cdd_load(spec + k) : cdd_zero();
    if (k == 0) xk.im = dd{0.f, 0.f};
    const int nk = N - k;
    const cdd xn = nk <= a.K ? cdd_conj(cdd_load(spec + nk)) : cdd_zero();
    const cdd A = cdd_add(xk, xn);
    const cdd B = cdd_mul_conj(cdd_sub(xk, xn), cdd_load(a.tw + k));
    cdd_store(buf0 + k, cdd_add(A, cdd_mul_pi(B)));
  }
  __syncthreads();
  const float4* z = fft_smem(buf0, buf1, a.half, a.tw, 2, true);
  float4* dst = (float4*)((float2*)a.grid[c] + (size_t)row * a.pitch);  // 2 df64 values per float4
  for (int n = threadIdx.x; n < N; n += blockDim.x) dst[n] = z[n];
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

FftShape fft_shape(int n) {
  FftShape s{};
  s.n = n;
  int m = n;
  while (m % 4 == 0 && s.nst < kMaxFftStages) {
    s.radix[s.nst++] = 4;
    m /= 4;
  }
  if (m % 2 == 0 && s.nst < kMaxFftStages) {
    s.radix[s.nst++] = 2;
    m /= 2;
  }
  while (m % 3 == 0 && s.nst < kMaxFftStages) {
    s.radix[s.nst++] = 3;
    m /= 3;
  }
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

size_t fft_rows_smem(int g) { return (size_t)2 * (g / 2) * sizeof(float4); }
size_t fft_cols_smem(int g) { return (size_t)2 * g * sizeof(float4); }

bool fft_dd_configure() {
  const int bytes = 220 * 1024;
  return cudaFuncSetAttribute(fft_rows_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
             cudaSuccess &&
         cudaFuncSetAttribute(fft_rows_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
             cudaSuccess &&
         cudaFuncSetAttribute(fft_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
             cudaSuccess;
}

void launch_fft_rows_fwd(const FftRowArgs& a, int nchan, cudaStream_t s) {
  const int nrows = a.row_hi - a.row_lo;
  if (nrows <= 0 || nchan <= 0) return;
  fft_rows_fwd_kernel<<<dim3(nrows, nchan), kFftThreads, fft_rows_smem(2 * a.half.n), s>>>(a);
}

void launch_fft_rows_inv(const FftRowArgs& a, int nchan, cudaStream_t s) {
  const int nrows = a.row_hi - a.row_lo;
  if (nrows <= 0 || nchan <= 0) return;
  fft_rows_inv_kernel<<<dim3(nrows, nchan), kFftThreads, fft_rows_smem(2 * a.half.n), s>>>(a);
}

void launch_fft_cols(const FftColArgs& a, int njobs, cudaStream_t s) {
  if (njobs <= 0) return;
  fft_cols_kernel<<<dim3(a.K + 1, njobs), kFftThreads, fft_cols_smem(a.full.n), s>>>(a);
}

}  // namespace lpg
