// Volume nodes sorted into square bins of kTile near-history cells
// (counting sort), and the single-precision spread that uses them.  One CTA
// owns one bin on each level's grid: it accumulates every point of the bin
// into shared-memory copies of the grid patch their stencils cover (the bin
// plus a w-cell halo), then adds the patch to the grid with global atomics.
// Each point is read once per level, its stencil weights are evaluated once,
// and the w^2 updates hit shared memory only.  Positions are stored relative
// to their bin's corner in single precision (bins are ~0.03 wide, so ~2e-9
// absolute).
#include <algorithm>
#include <cmath>

#include "lp_internal.cuh"

namespace lpg {

namespace {

// Key = bin of the point; points outside the bin grid (or NaN) go to the
// overflow bin nbx*nby, which no CTA reads, and are reported.
__global__ void bin_keys_kernel(const double* __restrict__ xy, int64_t n, double x0, double y0, double inv_bt,
                                int nbx, int nby, int* keys, int* counts, unsigned* status) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double fx = (xy[2 * j] - x0) * inv_bt, fy = (xy[2 * j + 1] - y0) * inv_bt;
  int key;
  if (fx >= 0.0 && fx < nbx && fy >= 0.0 && fy < nby) {
    key = (int)fy * nbx + (int)fx;
  } else {
    key = nbx * nby;
    atomicOr(status, kStatusOutOfBox);
  }
  keys[j] = key;
  atomicAdd(&counts[key], 1);
}

// Exclusive scan of counts[0..n) into starts[0..n], one block.
__global__ void scan_kernel(const int* __restrict__ counts, int n, int* starts) {
  __shared__ int part[1024];
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per, hi = min(n, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += counts[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < blockDim.x; off <<= 1) {
    int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - s;
  for (int i = lo; i < hi; ++i) {
    starts[i] = run;
    run += counts[i];
  }
  if (threadIdx.x == blockDim.x - 1) starts[n] = part[threadIdx.x];
}

// Scatter into bin order; positions become offsets from the bin's corner.
__global__ void scatter_kernel(const double* __restrict__ xy, int64_t n, const int* __restrict__ keys,
                               const int* __restrict__ starts, int* cursor, BinGeom bg, float2* rel_s,
                               int* perm) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int key = keys[j];
  const int pos = starts[key] + atomicAdd(&cursor[key], 1);
  const int bx = key % bg.nbx, by = key / bg.nbx;  // overflow bin: never read
  const double bt = 1.0 / bg.inv_bt;
  rel_s[pos] = make_float2((float)(xy[2 * j] - (bg.x0 + bx * bt)), (float)(xy[2 * j + 1] - (bg.y0 + by * bt)));
  perm[pos] = (int)j;
}

// q_s[c][k] = q[c][perm[k]] in single precision
__global__ void gather_q_kernel(const double* __restrict__ q, int64_t stride, int nq, const int* __restrict__ perm,
                                int64_t n, float* q_s) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int j = perm[k];
  for (int c = 0; c < nq; ++c) q_s[c * n + k] = (float)q[c * stride + j];
}

// Binned spread of the volume nodes on one level.  One warp handles one point
// at a time: lane i < 2w evaluates one stencil weight polynomial (x weights
// in lanes 0..w-1, y weights in lanes w..2w-1, coefficients held in
// registers); the lanes then take the w^2 stencil cells in row-major order, 32
// per pass.  The cells of one point are distinct and each warp accumulates
// into its own patch, so the updates are plain loads and stores; the CTA sums
// its warps' patches at the end and adds the sum to the grid with global
// atomics (neighbouring bins' patches overlap in the halo).
template <int W, int NCW>
__global__ void __launch_bounds__(kSubThreads) spread_sub_kernel(const __grid_constant__ SubArgs a) {
  extern __shared__ float smem[];  // [NCW][W] weight coefficients, then [nwarp][M*M] patches
  constexpr int NC = W * W, NP = (NC + 31) / 32;
  constexpr int NWARP = kSubThreads / 32;
  const int M = a.M, MM = M * M;
  const int bx = blockIdx.x, by = blockIdx.y;
  const int key = by * a.nbx + bx;
  const int k0 = a.start[key], n_here = a.start[key + 1] - k0;
  if (n_here == 0) return;
  float* coef = smem;
  float* patch = smem + ((NCW * W + 3) & ~3);
  for (int e = threadIdx.x; e < NCW * W; e += blockDim.x)
    coef[e] = (e / W < a.es.nc) ? a.es.c[e / W][e % W] : 0.f;
  for (int e = threadIdx.x; e < NWARP * MM; e += blockDim.x) patch[e] = 0.f;
  // grid index of patch cell (0, 0): the lowest stencil origin a point of
  // this bin can have, minus one for rounding
  const double ux = (a.org_x + bx * a.bt - a.gd.x0) * a.gd.inv_h;
  const double uy = (a.org_y + by * a.bt - a.gd.y0) * a.gd.inv_h;
  const int ox = (int)floor(ux - 0.5 * W), oy = (int)floor(uy - 0.5 * W);
  const float u0 = (float)(ux - ox), v0 = (float)(uy - oy);
  const float inv_h = (float)a.gd.inv_h;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int cell[NP], src_x[NP], src_y[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int i = lane + 32 * p;
    const int r = i / W, c = i % W;
    cell[p] = i < NC ? r * M + c : -1;
    src_x[p] = c;
    src_y[p] = W + (r < W ? r : 0);
  }
  __syncthreads();
  float cf[NCW];  // this lane's weight polynomial (lanes < 2W)
  {
    const int t = lane < W ? lane : (lane < 2 * W ? lane - W : 0);
#pragma unroll
    for (int j = 0; j < NCW; ++j) cf[j] = coef[j * W + t];
  }
  float* my = patch + warp * MM;
  const float half = 0.5f * (W - 1);
  // warp `warp` takes points k0 + warp + NWARP j; each round loads 32 of them
  // (one per lane) and walks them through the shuffles
  const int n_warp = n_here > warp ? (n_here - warp + NWARP - 1) / NWARP : 0;
  for (int j0 = 0; j0 < n_warp; j0 += 32) {
    const int jl = j0 + lane;
    float2 rl = make_float2(0.f, 0.f);
    float ql = 0.f;
    if (jl < n_warp) {
      rl = a.rel[k0 + warp + NWARP * jl];
      ql = a.q[k0 + warp + NWARP * jl];
    }
    const int cnt = min(32, n_warp - j0);
    for (int jj = 0; jj < cnt; ++jj) {
      const float rx = __shfl_sync(0xffffffffu, rl.x, jj);
      const float ry = __shfl_sync(0xffffffffu, rl.y, jj);
      const float qv = __shfl_sync(0xffffffffu, ql, jj);
      const float u = u0 + rx * inv_h, v = v0 + ry * inv_h;
      const int ix = (int)floorf(u - 0.5f * W) + 1, iy = (int)floorf(v - 0.5f * W) + 1;
      if (ix < 0 || iy < 0 || ix + W > M || iy + W > M) {
        if (lane == 0) atomicOr(a.status, kStatusOutOfBox);
        continue;
      }
      const float z = lane < W ? u - ix - half : v - iy - half;
      float wgt = cf[NCW - 1];
#pragma unroll
      for (int j = NCW - 2; j >= 0; --j) wgt = fmaf(wgt, z, cf[j]);
      float* dst = my + iy * M + ix;
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const float wx = __shfl_sync(0xffffffffu, wgt, src_x[p]);
        const float wy = __shfl_sync(0xffffffffu, wgt, src_y[p]);
        if (cell[p] >= 0) dst[cell[p]] = fmaf(qv * wy, wx, dst[cell[p]]);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  float* grid = (float*)a.grid;
  for (int e = threadIdx.x; e < MM; e += blockDim.x) {
    float val = 0.f;
#pragma unroll
    for (int w = 0; w < NWARP; ++w) val += patch[w * MM + e];
    if (val == 0.f) continue;
    const int gy = oy + e / M, gx = ox + e % M;
    if (gx < 0 || gy < 0 || gx >= a.gd.g || gy >= a.gd.g) {
      atomicOr(a.status, kStatusOutOfBox);
      continue;
    }
    atomicAdd(grid + (size_t)gy * a.gd.pitch + gx, val);
  }
}

}  // namespace

void launch_bin_sort(const double* xy, int64_t n, const BinGeom& bg, int* keys, int* counts, int* cursor,
                     int* starts, float2* rel_s, int* perm, unsigned* status, cudaStream_t s) {
  const int nbins = bg.nbx * bg.nby + 1;  // + overflow bin
  cudaMemsetAsync(counts, 0, nbins * sizeof(int), s);
  cudaMemsetAsync(cursor, 0, nbins * sizeof(int), s);
  if (n > 0)
    bin_keys_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xy, n, bg.x0, bg.y0, bg.inv_bt, bg.nbx, bg.nby,
                                                                keys, counts, status);
  scan_kernel<<<1, 1024, 0, s>>>(counts, nbins, starts);
  if (n > 0)
    scatter_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xy, n, keys, starts, cursor, bg, rel_s, perm);
}

void launch_gather_q(const double* q, int64_t stride, int nq, const int* perm, int64_t n, float* q_s,
                     cudaStream_t s) {
  if (n > 0) gather_q_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(q, stride, nq, perm, n, q_s);
}

size_t spread_sub_smem(const SubArgs& a, int w) {
  return (size_t)(((sub_ncw(w) * w + 3) & ~3) + (kSubThreads / 32) * a.M * a.M) * sizeof(float);
}

#define LP_SUB_CASES LP_CASE(4) LP_CASE(5) LP_CASE(6) LP_CASE(7) LP_CASE(8) LP_CASE(9) LP_CASE(10)

bool spread_sub_configure(int w) {
  const int bytes = 200 * 1024;
  switch (w) {
#define LP_CASE(W)                                                                         \
  case W:                                                                                  \
    return cudaFuncSetAttribute(spread_sub_kernel<W, W + 3>,                               \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
    LP_SUB_CASES
#undef LP_CASE
    default: return false;
  }
}

void launch_spread_sub(const SubArgs& a, int w, cudaStream_t s) {
  dim3 grid(a.nbx, a.nby);
  const size_t smem = spread_sub_smem(a, w);
  switch (w) {
#define LP_CASE(W)                                                  \
  case W:                                                           \
    spread_sub_kernel<W, W + 3><<<grid, kSubThreads, smem, s>>>(a); \
    break;
    LP_SUB_CASES
#undef LP_CASE
    default: break;
  }
}

}  // namespace lpg
