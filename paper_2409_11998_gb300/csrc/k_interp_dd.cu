// Type-2 interpolation of the FP64 plans in double-float arithmetic (Sec. 3,
// Step 4): u(x) = sum over both history grids of the w x w stencil weights
// times the grid values, which the df64 FFT chain left as (hi, lo) pairs.
// The stencil weights are the plan's per-offset polynomials (coefficients
// split from the FP64 fit) evaluated in df64 through the kernel's symmetry
// (dd_stencil_weights); products are accumulated with error-free transforms
// and the three outputs are converted to double once per target.
#include <cmath>

#include "df64.cuh"
#include "lp_internal.cuh"

namespace lpg {

namespace {

// Stencil origin i0 = floor(u - W/2) + 1 of a df64 grid coordinate, and the
// offset v = u - i0 - (W-1)/2 in [-1/2, 1/2).
template <int W>
__device__ __forceinline__ bool dd_stencil(dd u, int g, int& i0, dd& v) {
  const dd t = dd_add(u, dd{-0.5f * W, 0.f});
  float f = floorf(t.hi);
  if (t.hi == f && t.lo < 0.f) f -= 1.f;
  if (!(f > -1e7f && f < 1e7f)) return false;
  i0 = (int)f + 1;
  v = dd_add(u, dd{-((float)i0 + 0.5f * (W - 1)), 0.f});
  return i0 >= 0 && i0 + W <= g;
}

template <int W>
__device__ __forceinline__ void interp_dd_target(const InterpDDArgs& a, int64_t i) {
  const dd X = dd_from_double(a.txy[2 * i]), Y = dd_from_double(a.txy[2 * i + 1]);
  dd_acc acc[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  bool bad = false;
  for (int l = a.l0; l < 2; ++l) {
    const InterpDDLevel& L = a.lv[l];
    const dd ux = dd_mul(dd_sub(X, dd{L.x0.x, L.x0.y}), dd{L.inv_h.x, L.inv_h.y});
    const dd uy = dd_mul(dd_sub(Y, dd{L.y0.x, L.y0.y}), dd{L.inv_h.x, L.inv_h.y});
    int ix, iy;
    dd vx, vy;
    if (!dd_stencil<W>(ux, L.g, ix, vx) || !dd_stencil<W>(uy, L.g, iy, vy)) {
      bad = true;
      continue;
    }
    dd wx[W], wy[W];
    dd_stencil_weights<W>(&a.coef[0][0], kMaxW, a.nc, a.nf, vx, wx);
    dd_stencil_weights<W>(&a.coef[0][0], kMaxW, a.nc, a.nf, vy, wy);
    // rows and channels stay rolled (wy spills to L1-resident local memory):
    // unrolling all w^2 C products overflows the instruction cache.
    // Rows are read as 16-byte pairs of cells from the even cell ix0 at or
    // below ix (grid rows start 16-byte aligned: the pitch is even), W/2 + 1
    // loads instead of W.  The x weights are shifted once per target onto
    // the W + 1 cells ix0 .. ix0 + W (a zero weight at the unused end), so
    // that every row takes the loaded values in a fixed order.
    const int ix0 = ix & ~1;
    const bool odd = (ix & 1) != 0;
    dd ws[W + 1];
#pragma unroll
    for (int t = 0; t <= W; ++t) {
      const dd here = t < W ? wx[t] : dd{0.f, 0.f};
      const dd prev = t > 0 ? wx[t - 1] : dd{0.f, 0.f};
      ws[t] = odd ? prev : here;
    }
    constexpr int NQ = (W + 2) / 2;  // 16-byte loads covering cells 0 .. W
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
      if (!a.out[c]) continue;
      const float4* base = (const float4*)((const float2*)L.grid[c] + (size_t)iy * L.pitch + ix0);
#pragma unroll 1
      for (int b = 0; b < W; ++b) {
        const float4* row = base + (size_t)b * (L.pitch / 2);
        float4 q[NQ];
#pragma unroll
        for (int u = 0; u < NQ; ++u) q[u] = __ldg(row + u);
        dd_acc r = {0.f, 0.f};
#pragma unroll
        for (int t = 0; t <= W; ++t) {
          const float4 qq = q[t / 2];
          dd gv = (t & 1) ? dd{qq.z, qq.w} : dd{qq.x, qq.y};
          // cell ix0 + W of an even origin may be the row's padding, whose
          // bits need not be finite floats: its (zero-weight) value is dropped
          if (t == W) gv = odd ? gv : dd{0.f, 0.f};
          acc_fma(r, ws[t], gv);
        }
        acc_fma(acc[c], wy[b], acc_value(r));
      }
    }
  }
  if (bad) {
    atomicOr(a.status, kStatusOutOfBox);
    return;
  }
  for (int c = 0; c < 3; ++c)
    if (a.out[c]) a.out[c][i] = dd_to_double(acc_value(acc[c]));
}

template <int W>
__global__ void __launch_bounds__(128) interp_dd_kernel(const __grid_constant__ InterpDDArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) interp_dd_target<W>(a, i);
}

// A wave of plans in one launch: block b serves record r = the last with
// first[r] <= b (first[] ascending, each record's first block), targets
// 128 (b - first[r]) + threadIdx.x of it.
template <int W>
__global__ void __launch_bounds__(128) interp_dd_wave_kernel(const InterpDDArgs* __restrict__ recs,
                                                             const int* __restrict__ first, int nrec) {
  // the block's record in shared memory: the per-target code reads its
  // weight coefficients and level data many times (from global memory each
  // read would be a load; the single-plan kernel has them in parameter space)
  __shared__ InterpDDArgs sa;
  int lo = 0, hi = nrec - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  static_assert(sizeof(InterpDDArgs) % sizeof(int) == 0, "record copied as words");
  const int* src = (const int*)(recs + lo);
  int* dst = (int*)&sa;
  for (int k = threadIdx.x; k < (int)(sizeof(InterpDDArgs) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
  __syncthreads();
  const int64_t i = (int64_t)(blockIdx.x - first[lo]) * 128 + threadIdx.x;
  if (i < sa.n) interp_dd_target<W>(sa, i);
}

}  // namespace

void launch_interp_dd(const InterpDDArgs& a, int w, cudaStream_t s) {
  if (a.n <= 0) return;
  const unsigned blocks = (unsigned)((a.n + 127) / 128);
  switch (w) {
#define LP_CASE(W)                                         \
  case W:                                                  \
    interp_dd_kernel<W><<<blocks, 128, 0, s>>>(a);         \
    break;
    LP_CASE(4) LP_CASE(5) LP_CASE(6) LP_CASE(7) LP_CASE(8) LP_CASE(9) LP_CASE(10) LP_CASE(11) LP_CASE(12)
    LP_CASE(13) LP_CASE(14) LP_CASE(15) LP_CASE(16)
#undef LP_CASE
    default: break;
  }
}

void launch_interp_dd_wave(const InterpDDArgs* recs, const int* first, int nrec, int nblocks, int w,
                           cudaStream_t s) {
  if (nrec <= 0 || nblocks <= 0) return;
  switch (w) {
#define LP_CASE(W)                                                       \
  case W:                                                                \
    interp_dd_wave_kernel<W><<<nblocks, 128, 0, s>>>(recs, first, nrec); \
    break;
    LP_CASE(4) LP_CASE(5) LP_CASE(6) LP_CASE(7) LP_CASE(8) LP_CASE(9) LP_CASE(10) LP_CASE(11) LP_CASE(12)
    LP_CASE(13) LP_CASE(14) LP_CASE(15) LP_CASE(16)
#undef LP_CASE
    default: break;
  }
}

}  // namespace lpg
