// Volume nodes sorted into square bins of near-history cells (counting
// sort; 32 cells for FP32 plans, 24 for FP64 plans), and the binned spreads
// that use them.  One CTA owns one bin on each level's grid: it accumulates
// every point of the bin into shared-memory copies of the grid patch their
// stencils cover (the bin plus a w-cell halo), then adds the patch to the
// grid with global atomics.  Each point is read once per level, its stencil
// weights are evaluated once, and the w^2 updates hit shared memory only.
// Positions are stored relative to their bin's corner: in single precision
// for FP32 plans (bins are ~0.03 wide, so ~2e-9 absolute), as df64 pairs for
// FP64 plans.
#include <algorithm>
#include <cmath>

#include "df64.cuh"
#include "lp_internal.cuh"

namespace lpg {

namespace {

// Key = bin of the point; points outside the bin grid (or NaN) go to the
// overflow bin nbx*nby, which no CTA reads, and are reported.
// Warp-aggregated reservation: the lanes holding the same key (-1: none)
// share one atomic add of their number on ctr[key]; returns the lane's slot
// (the counter's old value plus its rank among those lanes).  Every lane of
// the warp calls it.  Consecutive nodes (the six of a triangle) mostly share
// a bin, so this divides the atomics on the bin counters several-fold.
__device__ __forceinline__ int warp_reserve(int* ctr, int key) {
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (key >= 0 && lane == leader) base = atomicAdd(ctr + key, __popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

__global__ void bin_keys_kernel(const double* __restrict__ xy, int64_t n, double x0, double y0, double inv_bt,
                                int nbx, int nby, int* keys, int* counts, unsigned* status) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int key = -1;
  if (j < n) {
    const double fx = (xy[2 * j] - x0) * inv_bt, fy = (xy[2 * j + 1] - y0) * inv_bt;
    if (fx >= 0.0 && fx < nbx && fy >= 0.0 && fy < nby) {
      key = (int)fy * nbx + (int)fx;
    } else {
      key = nbx * nby;
      atomicOr(status, kStatusOutOfBox);
    }
    keys[j] = key;
  }
  warp_reserve(counts, key);
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
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int key = j < n ? keys[j] : -1;
  const int slot = warp_reserve(cursor, key);
  if (key < 0) return;
  const int pos = starts[key] + slot;
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
__device__ __forceinline__ void spread_sub_bin(const SubArgs& a, int bx, int by) {
  extern __shared__ float smem[];  // [NCW][W] weight coefficients, then [nwarp][M*M] patches
  constexpr int NC = W * W, NP = (NC + 31) / 32;
  constexpr int NWARP = kSubThreads / 32;
  const int M = a.M, MM = M * M;
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
      float cur[NP];
#pragma unroll
      for (int p = 0; p < NP; ++p)
        if (cell[p] >= 0) cur[p] = dst[cell[p]];
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const float wx = __shfl_sync(0xffffffffu, wgt, src_x[p]);
        const float wy = __shfl_sync(0xffffffffu, wgt, src_y[p]);
        if (cell[p] >= 0) dst[cell[p]] = fmaf(qv * wy, wx, cur[p]);
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

// Scatter of the FP64 plans: offsets from the bin corner as df64 pairs
// (x.hi, x.lo, y.hi, y.lo), exact to ~2^-48 of the bin side.
__global__ void scatter_dd_kernel(const double* __restrict__ xy, int64_t n, const int* __restrict__ keys,
                                  const int* __restrict__ starts, int* cursor, BinGeom bg, float4* rel_s,
                                  int* perm) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int key = j < n ? keys[j] : -1;
  const int slot = warp_reserve(cursor, key);
  if (key < 0) return;
  const int pos = starts[key] + slot;
  const int bx = key % bg.nbx, by = key / bg.nbx;  // overflow bin: never read
  const double bt = 1.0 / bg.inv_bt;
  const dd rx = dd_from_double(xy[2 * j] - (bg.x0 + bx * bt));
  const dd ry = dd_from_double(xy[2 * j + 1] - (bg.y0 + by * bt));
  rel_s[pos] = make_float4(rx.hi, rx.lo, ry.hi, ry.lo);
  perm[pos] = (int)j;
}

// q_s[k] = q[perm[k]] as a df64 pair
__global__ void gather_q_dd_kernel(const double* __restrict__ q, const int* __restrict__ perm, int64_t n,
                                   float2* q_s) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const dd v = dd_from_double(q[perm[k]]);
  q_s[k] = make_float2(v.hi, v.lo);
}

// Stencil origin of a df64 patch coordinate u (see dd_stencil of the
// interpolation): i0 = floor(u - W/2) + 1 and v = u - i0 - (W-1)/2.
template <int W>
__device__ __forceinline__ bool stencil_dd(dd u, int M, int& i0, dd& v) {
  const dd t = dd_add(u, dd{-0.5f * W, 0.f});
  float f = floorf(t.hi);
  if (t.hi == f && t.lo < 0.f) f -= 1.f;
  if (!(f > -1e6f && f < 1e6f)) return false;
  i0 = (int)f + 1;
  v = dd_add(u, dd{-((float)i0 + 0.5f * (W - 1)), 0.f});
  return i0 >= 0 && i0 + W <= M;
}

// Binned spread of the volume nodes of FP64 plans, in fixed point.  One
// CTA per bin and one shared patch per CTA: every patch cell holds two
// 32-bit integer accumulators, a coarse count of quanta e1 and a fine count
// of quanta e2 = e1 / 2^s2, both chosen from the bin's largest strength and
// node count so that neither can overflow.  A contribution p = q wy wx
// (df64 product: high part ph plus error pe) is rounded to the coarse grid
// by one addition of a magic constant -- exact, since ph < 2^22 e1 -- the
// exact remainder plus pe to the fine grid the same way, and both counts
// are added with shared-memory integer atomics.  Integer sums are exact and
// independent of order, so the warps of the CTA share one patch; the
// result carries about 2^-44 of the bin's largest strength per
// contribution, below the df64 rounding of the transforms.
//   Phase 1 (per chunk of up to kSubDDChunk nodes): the CTA evaluates the 2w
//   df64 weight polynomials as (node, axis) tasks, one per thread, and stores
//   x weights and q times y weights with the stencil origins.
//   Phase 2: each warp takes one node at a time, its lanes the w^2 cells.
//   Flush: each cell's counts become one double (integer normalisation, no
//   FP64 arithmetic) added to the grid with an FP64 atomic.
template <int W, int NT>
__device__ __forceinline__ void spread_fx_bin(const SubDDArgs& a, const float2* __restrict__ q_s, void* grid_out,
                                              int bx, int by) {
  extern __shared__ float2 smd[];
  constexpr int NC = W * W, NP = (NC + 31) / 32, NWARP = NT / 32, CH = kSubDDChunk;
  constexpr int WS = 2 * W + 1;  // weight row stride (odd: conflict-free task stores)
  const int M = a.M, MM = M * M, nc = a.nc;
  const int key = by * a.nbx + bx;
  const int k0 = a.start[key], n_here = a.start[key + 1] - k0;
  if (n_here == 0) return;
  float2* coef = smd;                        // [nc][W]
  float2* wbuf = coef + kMaxNC * W;          // [CH][WS]: x weights, then q * y weights
  int* wpos = (int*)(wbuf + CH * WS);        // [CH][2] stencil origins (-1: outside the patch)
  int* pc = wpos + 2 * CH;                   // [MM] coarse counts
  int* pf = pc + MM;                         // [MM] fine counts
  __shared__ float red_q[NWARP];
  for (int e = threadIdx.x; e < nc * W; e += NT) coef[e] = a.coef[e / W][e % W];
  for (int e = threadIdx.x; e < 2 * MM; e += NT) pc[e] = 0;
  // largest |q| of the bin (high parts; the quanta only need its binade);
  // a non-finite strength is reported and the bin skipped
  float qmax = 0.f;
  bool bad_q = false;
  for (int k = threadIdx.x; k < n_here; k += NT) {
    const float qx = fabsf(q_s[k0 + k].x);
    bad_q |= !(qx <= 3.4e38f);
    qmax = fmaxf(qmax, qx);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) qmax = fmaxf(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red_q[warp] = qmax;
  if (__syncthreads_or(bad_q)) {
    if (threadIdx.x == 0) atomicOr(a.status, kStatusOutOfBox);
    return;
  }
  qmax = red_q[0];
#pragma unroll
  for (int w = 1; w < NWARP; ++w) qmax = fmaxf(qmax, red_q[w]);
  if (qmax == 0.f) return;
  // strengths scaled by 2^-eq (exact) so that the largest lies in [1/2, 1);
  // quanta: e1 = 2^E1 with every |ph| < 1 <= 2^(E1 + 21) and, for bins of
  // more than 512 nodes, 2^xs coarser so that the coarse counts stay below
  // 2^31; e2 = e1 / 2^(22 - xs) with the same bound for the fine counts
  int xs = 0;
  while ((512 << xs) < n_here && xs < 20) ++xs;
  int eq;
  frexpf(qmax * 1.000001f, &eq);             // qmax * (1 + 1e-6) < 2^eq
  eq = max(eq, -126);                        // a finite scale for subnormal strengths
  const float qscale = ldexpf(1.f, -eq);
  const int E1 = -21 + xs, E2 = E1 - 22 + xs;
  const float M1 = ldexpf(1.5f, E1 + 23), M2 = ldexpf(1.5f, E2 + 23);
  const int M1b = __float_as_int(M1), M2b = __float_as_int(M2);
  const double ux = (a.org_x + bx * a.bt - a.gd.x0) * a.gd.inv_h;
  const double uy = (a.org_y + by * a.bt - a.gd.y0) * a.gd.inv_h;
  const int ox = (int)floor(ux - 0.5 * W), oy = (int)floor(uy - 0.5 * W);
  const dd u0[2] = {dd_from_double(ux - ox), dd_from_double(uy - oy)};
  const dd inv_h = dd{a.inv_h.x, a.inv_h.y};
  int cell[NP], wxo[NP], wyo[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int i = lane + 32 * p;
    const int r = i / W, c = i % W;
    cell[p] = i < NC ? r * M + c : -1;
    wxo[p] = c;
    wyo[p] = W + (r < W ? r : 0);
  }
  __syncthreads();
  for (int c0 = 0; c0 < n_here; c0 += CH) {
    const int nch = min(CH, n_here - c0);
    // phase 1: task t = (node t / 2, axis t % 2)
    for (int t = threadIdx.x; t < 2 * nch; t += NT) {
      const int j = t >> 1, ax = t & 1;
      const int kk = k0 + c0 + j;
      const float4 r = a.rel[kk];
      const dd off = ax ? dd{r.z, r.w} : dd{r.x, r.y};
      const dd u = dd_add(u0[ax], dd_mul(off, inv_h));
      int i0;
      dd v;
      if (stencil_dd<W>(u, M, i0, v)) {
        dd w[W];
        dd_stencil_weights<W>(coef, W, nc, a.nf, v, w);
        float2* out = wbuf + j * WS + ax * W;
        if (ax) {
          const float2 q = q_s[kk];
          const dd qd = dd{q.x * qscale, q.y * qscale};
#pragma unroll
          for (int s = 0; s < W; ++s) {
            const dd qw = dd_mul(w[s], qd);
            out[s] = make_float2(qw.hi, qw.lo);
          }
        } else {
#pragma unroll
          for (int s = 0; s < W; ++s) out[s] = make_float2(w[s].hi, w[s].lo);
        }
        wpos[2 * j + ax] = i0;
      } else {
        wpos[2 * j + ax] = -1;
        atomicOr(a.status, kStatusOutOfBox);
      }
    }
    __syncthreads();
    // phase 2: warp per node, lanes over cells
    for (int j = warp; j < nch; j += NWARP) {
      const int ix = wpos[2 * j], iy = wpos[2 * j + 1];
      if (ix < 0 || iy < 0) continue;
      const int base = iy * M + ix;
      const float2* wrow = wbuf + j * WS;
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        if (cell[p] < 0) continue;
        const float2 wx = wrow[wxo[p]], qwy = wrow[wyo[p]];
        const float ph = __fmul_rn(qwy.x, wx.x);
        float pe = __fmaf_rn(qwy.x, wx.x, -ph);
        pe = __fmaf_rn(qwy.x, wx.y, pe);
        pe = __fmaf_rn(qwy.y, wx.x, pe);
        const float t1 = __fadd_rn(ph, M1);                        // ph rounded to a multiple of e1
        const float rem = __fsub_rn(ph, __fsub_rn(t1, M1));        // exact remainder
        const float t2 = __fadd_rn(__fadd_rn(rem, pe), M2);        // remainder + error, multiple of e2
        atomicAdd(pc + base + cell[p], __float_as_int(t1) - M1b);
        atomicAdd(pf + base + cell[p], __float_as_int(t2) - M2b);
      }
    }
    __syncthreads();
  }
  // flush: value = (coarse * 2^(E1 - E2) + fine) * 2^E2, an integer below
  // 2^53 times a power of two, assembled as a double by integer operations
  double* grid = (double*)grid_out;
  const int sh = E1 - E2;
  for (int e = threadIdx.x; e < MM; e += NT) {
    const long long n = ((long long)pc[e] << sh) + (long long)pf[e];
    if (n == 0) continue;
    const int gy = oy + e / M, gx = ox + e % M;
    if (gx < 0 || gy < 0 || gx >= a.gd.g || gy >= a.gd.g) {
      atomicOr(a.status, kStatusOutOfBox);
      continue;
    }
    const unsigned long long sign = n < 0 ? (1ull << 63) : 0ull;
    const unsigned long long m = (unsigned long long)(n < 0 ? -n : n);
    const int lz = __clzll(m);                                     // >= 11
    const unsigned long long frac = ((m << lz) >> 11) & 0xfffffffffffffull;
    const long long ex = (long long)(63 - lz + E2 + eq + 1023);
    const double v = __longlong_as_double((long long)(sign | ((unsigned long long)ex << 52) | frac));
    atomicAdd(grid + (size_t)gy * a.gd.pitch + gx, v);
  }
}


// The binned spreads as kernels: one CTA per bin of one plan (grid = bins),
// or, for a wave of plans, one CTA per bin of every record of the wave: the
// record of block b is the last r with first[r] <= b (first[] holds each
// record's first block, ascending; first[nrec] the total).
__device__ __forceinline__ int wave_record(const int* __restrict__ first, int nrec, int b) {
  int lo = 0, hi = nrec - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int W, int NCW>
__global__ void __launch_bounds__(kSubThreads) spread_sub_kernel(const __grid_constant__ SubArgs a) {
  spread_sub_bin<W, NCW>(a, blockIdx.x, blockIdx.y);
}

template <int W, int NCW>
__global__ void __launch_bounds__(kSubThreads) spread_sub_wave_kernel(const SubArgs* __restrict__ recs,
                                                                      const int* __restrict__ first, int nrec) {
  const int r = wave_record(first, nrec, blockIdx.x);
  const SubArgs& a = recs[r];
  const int key = blockIdx.x - first[r];
  spread_sub_bin<W, NCW>(a, key % a.nbx, key / a.nbx);
}

template <int W, int NT>
__global__ void __launch_bounds__(NT, kSubDDMinBlocks) spread_fx_kernel(const __grid_constant__ SubDDArgs a) {
  spread_fx_bin<W, NT>(a, a.q, a.grid, blockIdx.x, blockIdx.y);
}

// Listed bins x channels: block (b, c) spreads channel c of bin bins[b].
template <int W, int NT>
__global__ void __launch_bounds__(NT, kSubDDMinBlocks) spread_fx_list_kernel(const __grid_constant__ SubDDArgs a,
                                                               const int2* __restrict__ bins, FxChan ch) {
  const int2 b = bins[blockIdx.x];
  spread_fx_bin<W, NT>(a, ch.q[blockIdx.y], ch.grid[blockIdx.y], b.x, b.y);
}

template <int W, int NT>
__global__ void __launch_bounds__(NT, kSubDDMinBlocks) spread_fx_list_wave_kernel(
    const SubDDArgs* __restrict__ recs, const FxListRec* __restrict__ lrecs, const int* __restrict__ first,
    int nrec) {
  const int r = wave_record(first, nrec, blockIdx.x);
  const FxListRec& L = lrecs[r];
  const int key = blockIdx.x - first[r];
  const int c = key % L.nch;
  const int2 b = L.bins[key / L.nch];
  spread_fx_bin<W, NT>(recs[r], L.ch.q[c], L.ch.grid[c], b.x, b.y);
}

template <int W, int NT>
__global__ void __launch_bounds__(NT, kSubDDMinBlocks) spread_fx_wave_kernel(const SubDDArgs* __restrict__ recs,
                                                               const int* __restrict__ first, int nrec) {
  const int r = wave_record(first, nrec, blockIdx.x);
  const SubDDArgs& a = recs[r];
  const int key = blockIdx.x - first[r];
  spread_fx_bin<W, NT>(a, a.q, a.grid, key % a.nbx, key / a.nbx);
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

void launch_bin_sort_dd(const double* xy, int64_t n, const BinGeom& bg, int* keys, int* counts, int* cursor,
                        int* starts, float4* rel_s, int* perm, unsigned* status, cudaStream_t s) {
  const int nbins = bg.nbx * bg.nby + 1;  // + overflow bin
  cudaMemsetAsync(counts, 0, nbins * sizeof(int), s);
  cudaMemsetAsync(cursor, 0, nbins * sizeof(int), s);
  if (n > 0)
    bin_keys_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xy, n, bg.x0, bg.y0, bg.inv_bt, bg.nbx, bg.nby,
                                                                keys, counts, status);
  scan_kernel<<<1, 1024, 0, s>>>(counts, nbins, starts);
  if (n > 0)
    scatter_dd_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xy, n, keys, starts, cursor, bg, rel_s, perm);
}

void launch_gather_q_dd(const double* q, const int* perm, int64_t n, float2* q_s, cudaStream_t s) {
  if (n > 0) gather_q_dd_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(q, perm, n, q_s);
}

// Shared memory of the fixed-point spread: coefficient table, one chunk of
// weight rows and stencil origins, and the two count arrays of the patch.
static size_t spread_fx_smem_nt(int M, int w, int nt) {
  return (size_t)(kMaxNC * w + nt * (2 * w + 1)) * sizeof(float2) + (size_t)2 * nt * sizeof(int) +
         (size_t)2 * M * M * sizeof(int);
}

size_t spread_sub_dd_smem(int M, int w) { return spread_fx_smem_nt(M, w, kSubDDChunk); }

// dynamic shared memory of either binned spread for patch side M
size_t spread_sub_smem(int M, int w, bool f64) {
  if (f64) return spread_fx_smem_nt(M, w, kSubDDChunk);
  return (size_t)(((sub_ncw(w) * w + 3) & ~3) + (kSubThreads / 32) * M * M) * sizeof(float);
}

#define LP_SUB_DD_CASES LP_CASE(4) LP_CASE(5) LP_CASE(6) LP_CASE(7) LP_CASE(8) LP_CASE(9) LP_CASE(10) \
  LP_CASE(11) LP_CASE(12) LP_CASE(13) LP_CASE(14) LP_CASE(15) LP_CASE(16)

bool spread_sub_dd_configure(int w) {
  const int bytes = 200 * 1024;
  switch (w) {
#define LP_CASE(W)                                                                                     \
  case W:                                                                                              \
    return cudaFuncSetAttribute(spread_fx_kernel<W, kSubDDThreads>,                                     \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess &&   \
           cudaFuncSetAttribute(spread_fx_wave_kernel<W, kSubDDThreads>,                                \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess &&   \
           cudaFuncSetAttribute(spread_fx_list_kernel<W, kSubDDThreads>,                                \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess &&   \
           cudaFuncSetAttribute(spread_fx_list_wave_kernel<W, kSubDDThreads>,                           \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
    LP_SUB_DD_CASES
#undef LP_CASE
    default: return false;
  }
}

void launch_spread_fx_list(const SubDDArgs& a, const int2* bins, int nbins, const FxChan& ch, int nch, int w,
                           cudaStream_t s) {
  if (nbins <= 0 || nch <= 0) return;
  dim3 grid(nbins, nch);
  const size_t smem = spread_fx_smem_nt(a.M, w, kSubDDChunk);
  switch (w) {
#define LP_CASE(W)                                                                      \
  case W:                                                                               \
    spread_fx_list_kernel<W, kSubDDThreads><<<grid, kSubDDThreads, smem, s>>>(a, bins, ch); \
    break;
    LP_SUB_DD_CASES
#undef LP_CASE
    default: break;
  }
}

void launch_spread_sub_dd(const SubDDArgs& a, int w, cudaStream_t s) {
  dim3 grid(a.nbx, a.nby);
  const size_t smem = spread_fx_smem_nt(a.M, w, kSubDDChunk);
  switch (w) {
#define LP_CASE(W)                                                               \
  case W:                                                                        \
    spread_fx_kernel<W, kSubDDThreads><<<grid, kSubDDThreads, smem, s>>>(a);     \
    break;
    LP_SUB_DD_CASES
#undef LP_CASE
    default: break;
  }
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
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess && \
           cudaFuncSetAttribute(spread_sub_wave_kernel<W, W + 3>,                          \
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

// One launch for the binned spreads of a wave: recs[nrec] in device memory,
// first[nrec + 1] their first blocks; smem: the largest record's need.
void launch_spread_fx_list_wave(int w, const SubDDArgs* recs, const FxListRec* lrecs, const int* first, int nrec,
                                int nblocks, size_t smem, cudaStream_t s) {
  if (nrec <= 0 || nblocks <= 0) return;
  switch (w) {
#define LP_CASE(W)                                                                                            \
  case W:                                                                                                     \
    spread_fx_list_wave_kernel<W, kSubDDThreads><<<nblocks, kSubDDThreads, smem, s>>>(recs, lrecs, first, nrec); \
    break;
    LP_SUB_DD_CASES
#undef LP_CASE
    default: break;
  }
}

void launch_spread_wave(int precision, int w, const void* recs, const int* first, int nrec, int nblocks,
                        size_t smem, cudaStream_t s) {
  if (nrec <= 0 || nblocks <= 0) return;
  if (precision == LP_FP64) {
    switch (w) {
#define LP_CASE(W)                                                                                       \
  case W:                                                                                                \
    spread_fx_wave_kernel<W, kSubDDThreads><<<nblocks, kSubDDThreads, smem, s>>>((const SubDDArgs*)recs, \
                                                                                 first, nrec);          \
    break;
      LP_SUB_DD_CASES
#undef LP_CASE
      default: break;
    }
  } else {
    switch (w) {
#define LP_CASE(W)                                                                                           \
  case W:                                                                                                    \
    spread_sub_wave_kernel<W, W + 3><<<nblocks, kSubThreads, smem, s>>>((const SubArgs*)recs, first, nrec); \
    break;
      LP_SUB_CASES
#undef LP_CASE
      default: break;
    }
  }
}

}  // namespace lpg
