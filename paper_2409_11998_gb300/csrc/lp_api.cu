// C ABI entry points (include/lp.h): plan lifetime, binding of sources and
// densities, and the evaluation pipeline
//   spread -> forward FFT -> multiplier -> inverse FFT -> interpolate -> local
// of Sec. 3 (history part, two levels) and Sec. 4 (local part).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "lp_internal.cuh"

using namespace lpg;

struct lp_plan_s {
  Plan P;
};

namespace lpg {

// Forward transform of one channel: real rows [row_lo, row_hi) along x
// (the other rows are zero), then the K + 1 kept complex columns along y.
void fft_forward(const Plan& P, int level, int c) {
  const GridLevel& G = P.lv[level];
  const size_t r0 = (size_t)G.row_lo;
  if (P.precision == LP_FP64) {
    double* re = (double*)G.chan[c];
    cufftDoubleComplex* cz = (cufftDoubleComplex*)G.chan[c];
    cufftExecD2Z(G.row_fwd, re + r0 * G.pitch, cz + r0 * (G.g / 2 + 1));
    cufftExecZ2Z(G.col, cz, cz, CUFFT_FORWARD);
  } else {
    float* re = (float*)G.chan[c];
    cufftComplex* cz = (cufftComplex*)G.chan[c];
    cufftExecR2C(G.row_fwd, re + r0 * G.pitch, cz + r0 * (G.g / 2 + 1));
    cufftExecC2C(G.col, cz, cz, CUFFT_FORWARD);
  }
}

// Inverse: the K + 1 columns along y (the multiplier zeroed every other
// column), then the complex-to-real rows [row_lo, row_hi) that targets read.
void fft_inverse(const Plan& P, int level, int c) {
  const GridLevel& G = P.lv[level];
  const size_t r0 = (size_t)G.row_lo;
  if (P.precision == LP_FP64) {
    double* re = (double*)G.chan[c];
    cufftDoubleComplex* cz = (cufftDoubleComplex*)G.chan[c];
    cufftExecZ2Z(G.col, cz, cz, CUFFT_INVERSE);
    cufftExecZ2D(G.row_inv, cz + r0 * (G.g / 2 + 1), re + r0 * G.pitch);
  } else {
    float* re = (float*)G.chan[c];
    cufftComplex* cz = (cufftComplex*)G.chan[c];
    cufftExecC2C(G.col, cz, cz, CUFFT_INVERSE);
    cufftExecC2R(G.row_inv, cz + r0 * (G.g / 2 + 1), re + r0 * G.pitch);
  }
}

}  // namespace lpg

namespace {

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Device allocation charged to the plan's footprint; refused (no cudaMalloc)
// when it would take the footprint beyond the plan's budget.
bool dalloc(Plan& P, void** ptr, size_t bytes) {
  if (P.max_bytes && P.device_bytes + bytes > P.max_bytes) {
    *ptr = nullptr;
    return false;
  }
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return false;
  }
  ++P.gen;
  P.device_bytes += bytes;
  return true;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

// Free a plan buffer of `bytes` bytes and take it off the plan's footprint.
template <typename Tp>
void drelease(Plan& P, Tp*& p, size_t bytes) {
  if (p) {
    cudaFree((void*)p);
    P.device_bytes -= std::min(bytes, P.device_bytes);
  }
  p = nullptr;
}

// Stage timing event k on stream s; while lp_execute is captured into a
// graph the record becomes a graph node (external record), so the replayed
// graph still times its stages.
void record_stage(const Plan& P, int k, cudaStream_t s) {
  if (P.capturing)
    cudaEventRecordWithFlags(P.ev[k], s, cudaEventRecordExternal);
  else
    cudaEventRecord(P.ev[k], s);
}

// Device view of a caller array: used in place when it is device memory,
// otherwise copied into plan-owned staging at byte offset *off.
const double* device_view(Plan& P, const double* src, size_t count, size_t* off, cudaStream_t s) {
  if (!src || count == 0) return src;
  if (is_device_ptr(src)) return src;
  double* dst = (double*)((char*)P.d_stage + *off);
  cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyHostToDevice, s);
  *off += ((count * sizeof(double) + 255) / 256) * 256;
  return dst;
}

bool ensure_stage(Plan& P, size_t bytes) {
  if (bytes <= P.stage_bytes) return true;
  cudaStreamSynchronize(P.stream);
  if (P.d_stage) {
    cudaFree(P.d_stage);
    P.device_bytes -= P.stage_bytes;
  }
  P.d_stage = nullptr;
  P.stage_bytes = 0;
  if (!dalloc(P, &P.d_stage, bytes)) return false;
  P.stage_bytes = bytes;
  return true;
}

size_t round256(size_t b) { return ((b + 255) / 256) * 256; }

lp_status make_fft_plans(Plan& P, GridLevel& G) {
  const int g = G.g, nc = g / 2 + 1;
  const bool f64 = P.precision == LP_FP64;
  int n[1] = {g};
  int rin[1] = {G.pitch}, cin[1] = {nc}, col[1] = {g};
  const int nrows = G.row_hi - G.row_lo;
  if (cufftPlanMany(&G.row_fwd, 1, n, rin, 1, G.pitch, cin, 1, nc, f64 ? CUFFT_D2Z : CUFFT_R2C,
                    nrows) != CUFFT_SUCCESS ||
      cufftPlanMany(&G.row_inv, 1, n, cin, 1, nc, rin, 1, G.pitch, f64 ? CUFFT_Z2D : CUFFT_C2R,
                    nrows) != CUFFT_SUCCESS ||
      cufftPlanMany(&G.col, 1, n, col, nc, 1, col, nc, 1, f64 ? CUFFT_Z2Z : CUFFT_C2C, G.K + 1) !=
          CUFFT_SUCCESS)
    return LP_ERR_CUDA;
  cufftSetStream(G.row_fwd, P.stream);
  cufftSetStream(G.row_inv, P.stream);
  cufftSetStream(G.col, P.stream);
  return LP_OK;
}

void destroy_plan(Plan& P) {
  if (P.graph_stream) cudaStreamSynchronize(P.graph_stream);
  if (P.copy_stream) cudaStreamSynchronize(P.copy_stream);
  if (P.stream) cudaStreamSynchronize(P.stream);
  for (auto& G : P.lv) {
    for (auto& c : G.chan) dfree(c);
    for (auto& c : G.spec) dfree(c);
    dfree(G.tw_dd);
    dfree(G.freq);
    dfree(G.mtab_dd);
    dfree(G.mtab);
    dfree(G.mtab32);
    if (G.row_fwd) cufftDestroy(G.row_fwd);
    if (G.row_inv) cufftDestroy(G.row_inv);
    if (G.col) cufftDestroy(G.col);
  }
  void* bufs[] = {P.d_bxy, P.d_bw, P.d_bnrm, P.d_geo_coef, P.d_geo_ref, P.d_leg_T, P.d_tau,
                  P.d_cell_start, P.d_cell_node, P.d_vxy, P.d_vq, P.d_sigma, P.d_sigma_coef,
                  P.d_sigma_ref, P.d_mu, P.d_mu_coef, P.d_mu_ref, P.d_bq, P.d_qsum, P.d_stage,
                  P.d_out, P.d_status, P.d_near, P.d_near_count, P.d_cell_xy32,
                  P.d_geo_coef32, P.d_keys, P.d_counts, P.d_cursor, P.d_vrel_s, P.d_vperm, P.d_vq_s,
                  P.d_vstart, P.d_sigma_coef32, P.d_mu_coef32, P.d_vrel_dd, P.d_vq_dd,
                  P.d_dy_tab, P.d_dy_rel, P.d_dy_nw, P.d_dy_sig, P.d_dy_mu,
                  P.d_dy_rad, P.d_dy_wgl, P.d_dy_cell_start, P.d_dy_cell_panel, P.d_dy_ref, P.d_vf,
                  P.d_corners, P.d_corner_q, P.d_qred, P.d_geo_coef_dd, P.d_sigma_coef_dd,
                  P.d_mu_coef_dd, P.d_cell_near, P.d_bkeys, P.d_bstart, P.d_brel_dd, P.d_bperm, P.d_bq_dd, P.d_bbins};
  for (void* b : bufs) dfree(b);
  if (P.h_status) cudaFreeHost(P.h_status);
  for (auto& e : P.ev)
    if (e) cudaEventDestroy(e);
  if (P.graph_exec) cudaGraphExecDestroy(P.graph_exec);
  if (P.ev_g0) cudaEventDestroy(P.ev_g0);
  if (P.ev_g1) cudaEventDestroy(P.ev_g1);
  if (P.graph_stream) cudaStreamDestroy(P.graph_stream);
  if (P.ev_in) cudaEventDestroy(P.ev_in);
  if (P.ev_staged) cudaEventDestroy(P.ev_staged);
  if (P.copy_stream) cudaStreamDestroy(P.copy_stream);
}

lp_status status_from_cuda() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

// Outward normals from the panel interpolant when the caller gives none:
// nu = (y', -x') / |gamma'| at the nodes (counter-clockwise curve).
void derive_normals(int64_t n_panels, int p, const double* xy, double* nrm) {
  std::vector<double> tau(p), wq(p);
  gauss_legendre(p, tau.data(), wq.data());
  // differentiation matrix of the Lagrange basis at the nodes
  std::vector<double> bw(p, 1.0);
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j)
      if (j != i) bw[i] /= (tau[i] - tau[j]);
  for (int64_t ip = 0; ip < n_panels; ++ip) {
    const double* v = xy + (size_t)ip * p * 2;
    for (int i = 0; i < p; ++i) {
      double dx = 0, dy = 0, diag = 0;
      for (int j = 0; j < p; ++j) {
        if (j == i) continue;
        double dij = bw[j] / bw[i] / (tau[i] - tau[j]);
        dx += dij * v[2 * j];
        dy += dij * v[2 * j + 1];
        diag -= dij;
      }
      dx += diag * v[2 * i];
      dy += diag * v[2 * i + 1];
      double s = std::hypot(dx, dy);
      nrm[(size_t)(ip * p + i) * 2] = dy / s;
      nrm[(size_t)(ip * p + i) * 2 + 1] = -dx / s;
    }
  }
}

// ---- scratch of lp_execute_noalloc -------------------------------------------
// The per-call buffers that lp_execute keeps in plan memory -- the
// near-boundary list of the local pass (one int2 per target) and its
// counter -- live in this file-scope device array instead, so that the call
// allocates nothing.  Every GPU that loads the library holds it (16 MiB +
// 256 B) until the process exits.
constexpr int64_t kNoAllocMaxTargets = int64_t(1) << 21;
constexpr size_t kNoAllocListBytes = (size_t)kNoAllocMaxTargets * sizeof(int2);
constexpr size_t kNoAllocScratchBytes = kNoAllocListBytes + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch on device `dev`, which must be current.  In
// host code the array's name is only a host-side stand-in, so the address is
// looked up once per device (with that device current) and cached.
lp_status noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return LP_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return LP_ERR_CUDA;
    }
    g_noalloc_addr[dev] = ptr;
  }
  *out = g_noalloc_addr[dev];
  return LP_OK;
}

}  // namespace

namespace lpg {

// FP64 plans: counting sort of the boundary nodes into the current bins, the
// list of bins that hold some (read back once: the layer spread launches one
// CTA per listed bin and channel), and the bound layer strengths in bin
// order.  Runs at plan creation and whenever the bins change (autotuner);
// synchronises the plan's stream.  A node outside the bins keeps the
// point-parallel layer spread, which reports it at every evaluation.
static void gather_layer_strengths(Plan& P, int kind) {
  if (!P.bbinned) return;
  if (kind == 0) {
    launch_gather_q_dd(P.d_bq, P.d_bperm, P.nb, P.d_bq_dd, P.stream);
    ++P.launches;
  } else {
    launch_gather_q_dd(P.d_bq + P.nb, P.d_bperm, P.nb, P.d_bq_dd + P.nb, P.stream);
    launch_gather_q_dd(P.d_bq + 2 * P.nb, P.d_bperm, P.nb, P.d_bq_dd + 2 * P.nb, P.stream);
    P.launches += 2;
  }
}

static lp_status bin_boundary(Plan& P) {
  P.bbinned = false;
  if (!P.d_bkeys || P.nb <= 0) return LP_OK;
  unsigned* scratch_status = (unsigned*)(P.d_bkeys + P.nb);
  cudaMemsetAsync(scratch_status, 0, sizeof(unsigned), P.stream);
  launch_bin_sort_dd(P.d_bxy, P.nb, P.bins, P.d_bkeys, P.d_counts, P.d_cursor, P.d_bstart, P.d_brel_dd, P.d_bperm,
                     scratch_status, P.stream);
  const int nbins = P.bins.nbx * P.bins.nby;
  std::vector<int> st((size_t)nbins + 2);
  cudaMemcpyAsync(st.data(), P.d_bstart, st.size() * sizeof(int), cudaMemcpyDeviceToHost, P.stream);
  if (cudaStreamSynchronize(P.stream) != cudaSuccess) return status_from_cuda();
  if (st[nbins + 1] != st[nbins]) return LP_OK;  // nodes outside the bins
  std::vector<int2> list;
  for (int k = 0; k < nbins; ++k)
    if (st[k + 1] > st[k]) list.push_back(make_int2(k % P.bins.nbx, k / P.bins.nbx));
  if (list.empty()) return LP_OK;
  cudaMemcpy(P.d_bbins, list.data(), list.size() * sizeof(int2), cudaMemcpyHostToDevice);
  P.n_bbins = (int)list.size();
  P.bbinned = true;
  if (P.have_sigma) gather_layer_strengths(P, 0);
  if (P.have_mu) gather_layer_strengths(P, 1);
  return status_from_cuda();
}

// Bins of the binned volume spread: squares of bin_cells near-history cells
// (32 for FP32 plans; 24 for FP64 plans, whose df64 patches take twice the
// shared memory).  FP32 plans whose kernel fit needs more coefficients than
// the binned kernel holds keep the point-parallel spread.
// Bin geometry for bins of `cells` near-history cells (first level in use):
// origin, count, and per level the patch side -- the bin, the stencil halo
// and a cell of rounding slack; among the next 16 sizes, the one whose row
// pitch gives the fewest shared-memory wavefronts for the w^2 stencil cells
// taken 32 at a time (4-byte cells in 32 banks: the FP32 patch, and each of
// the two count arrays of the FP64 plans' fixed-point patch).  False if a
// patch would not fit in shared memory.
static bool configure_bins(Plan& P, int cells) {
  const GridLevel& N = P.lv[P.l0];
  const int w = P.ker.w;
  const bool f64 = P.precision == LP_FP64;
  BinGeom bins;
  bins.x0 = N.x0;
  bins.y0 = N.y0;
  bins.inv_bt = 1.0 / (cells * N.h);
  bins.nbx = bins.nby = (N.g + cells - 1) / cells;
  int M[2] = {0, 0};
  const int banks = 32, group = 32;
  for (int l = P.l0; l < 2; ++l) {
    const double c = cells * N.h / P.lv[l].h;
    const int m0 = (int)std::ceil(c) + w + 3;
    int best = m0, best_wf = 1 << 30;
    for (int m = m0; m < m0 + 16; ++m) {
      int wf = 0;
      for (int p0 = 0; p0 < w * w; p0 += group) {
        int hits[32] = {0}, mx = 0;
        for (int i = p0; i < std::min(p0 + group, w * w); ++i)
          mx = std::max(mx, ++hits[((i / w) * m + i % w) % banks]);
        wf += mx;
      }
      if (wf < best_wf) {
        best_wf = wf;
        best = m;
      }
    }
    M[l] = best;
    const size_t smem = f64 ? spread_sub_dd_smem(best, w)
                            : (size_t)(((sub_ncw(w) * w + 3) & ~3) + (kSubThreads / 32) * best * best) * sizeof(float);
    if (smem > 200 * 1024) return false;
  }
  P.bin_cells = cells;
  ++P.gen;
  P.bins = bins;
  P.sub_M[0] = M[0];
  P.sub_M[1] = M[1];
  return true;
}

// Bins of the binned volume spread: squares of bin_cells near-history cells
// (32 for FP32 plans; 24 for FP64 plans, whose df64 patches take twice the
// shared memory; plans created with autotune time kBinCandidates at the first
// lp_volume).  FP32 plans whose kernel fit needs more coefficients than the
// binned kernel holds keep the point-parallel spread.
lp_status setup_bins(Plan& P) {
  const int w = P.ker.w;
  const bool f64 = P.precision == LP_FP64;
  if (w < 4 || (!f64 && (w > 10 || P.es32.nc > sub_ncw(w)))) return LP_OK;
  if (!configure_bins(P, f64 ? 24 : kTile)) return LP_OK;
  if (!(f64 ? spread_sub_dd_configure(w) : spread_sub_configure(w))) return LP_ERR_CUDA;
  // bin bookkeeping sized for the smallest candidate bin
  const int nb_max = (P.lv[P.l0].g + kBinCandidates[f64][0] - 1) / kBinCandidates[f64][0];
  const size_t nbins = (size_t)nb_max * nb_max + 1;
  if (!dalloc(P, (void**)&P.d_counts, nbins * sizeof(int)) ||
      !dalloc(P, (void**)&P.d_cursor, nbins * sizeof(int)) ||
      !dalloc(P, (void**)&P.d_vstart, (nbins + 1) * sizeof(int)))
    return LP_ERR_NOMEM;
  cudaMemset(P.d_vstart, 0, (nbins + 1) * sizeof(int));
  P.binned = true;
  if (f64 && P.nb > 0) {
    const size_t nb = (size_t)P.nb;
    if (!dalloc(P, (void**)&P.d_bkeys, (nb + 1) * sizeof(int)) ||
        !dalloc(P, (void**)&P.d_bstart, (nbins + 1) * sizeof(int)) ||
        !dalloc(P, (void**)&P.d_brel_dd, nb * sizeof(float4)) || !dalloc(P, (void**)&P.d_bperm, nb * sizeof(int)) ||
        !dalloc(P, (void**)&P.d_bq_dd, 3 * nb * sizeof(float2)) ||
        !dalloc(P, (void**)&P.d_bbins, std::min(nb, nbins) * sizeof(int2)))
      return LP_ERR_NOMEM;
    return bin_boundary(P);
  }
  return LP_OK;
}

// FP64 plans: argument record of the fixed-point spread of the volume
// channel on one level.
SubDDArgs make_spread_dd_args(const Plan& P, int l) {
  const GridLevel& G = P.lv[l];
  SubDDArgs a{};
  a.gd = grid_dev(G);
  a.rel = P.d_vrel_dd;
  a.q = P.d_vq_dd;
  a.start = P.d_vstart;
  a.grid = G.chan[0];
  a.org_x = P.bins.x0;
  a.org_y = P.bins.y0;
  a.bt = 1.0 / P.bins.inv_bt;
  const double ih = 1.0 / G.h;
  const float ihh = (float)ih;
  a.inv_h = make_float2(ihh, (float)(ih - (double)ihh));
  a.nbx = P.bins.nbx;
  a.nby = P.bins.nby;
  a.M = P.sub_M[l];
  a.nc = P.es.nc;
  a.nf = P.es_float_steps;
  a.status = P.d_status;
  for (int k = 0; k < P.es.nc; ++k)
    for (int t = 0; t < P.es.w; ++t) {
      const double c = P.es.c[k][t];
      const float ch = (float)c;
      a.coef[k][t] = make_float2(ch, (float)(c - (double)ch));
    }
  return a;
}

void spread_binned_dd(const Plan& P, int l, cudaStream_t s) {
  ++P.launches;
  launch_spread_sub_dd(make_spread_dd_args(P, l), P.ker.w, s);
}

void spread_binned(const Plan& P, int l, cudaStream_t s);

// Spread of the volume channel on one level from the sorted nodes.
void spread_volume_binned(const Plan& P, int l, cudaStream_t s) {
  if (P.precision == LP_FP64)
    spread_binned_dd(P, l, s);
  else
    spread_binned(P, l, s);
}

// FP32 plans: argument record of the spread of the volume channel on one
// level from the sorted nodes.
SubArgs make_spread_sub_args(const Plan& P, int l) {
  const GridLevel& G = P.lv[l];
  SubArgs a;
  a.gd = grid_dev(G);
  a.es = P.es32;
  a.rel = P.d_vrel_s;
  a.q = P.d_vq_s;
  a.start = P.d_vstart;
  a.grid = G.chan[0];
  a.org_x = P.bins.x0;
  a.org_y = P.bins.y0;
  a.bt = 1.0 / P.bins.inv_bt;
  a.nbx = P.bins.nbx;
  a.nby = P.bins.nby;
  a.M = P.sub_M[l];
  a.status = P.d_status;
  return a;
}

void spread_binned(const Plan& P, int l, cudaStream_t s) {
  ++P.launches;
  launch_spread_sub(make_spread_sub_args(P, l), P.ker.w, s);
}

float2 split_host(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

// FFT chain of both precisions (k_fft.cu): radix plans, twiddles, the
// multiplier tables as (hi, lo) pairs (FP64) and the per-channel spectrum
// columns.  Plans whose grids are not 3-smooth or whose columns do not fit in
// shared memory keep cuFFT.
lp_status setup_fft_chain(Plan& P) {
  const size_t limit = 220 * 1024;
  const bool f64 = P.precision == LP_FP64;
  for (int l = P.l0; l < 2; ++l) {
    GridLevel& G = P.lv[l];
    // FP32 column transforms use radices 8, 9, 16 as well (fewer passes:
    // 0.278 -> 0.229 ms on the starfish); the half-length row transforms keep
    // 2, 3, 4 (radix-9 rows of 1458 leave a third of the threads idle and
    // measured slower, 0.189 -> 0.222 ms).  Double-float columns keep 2, 3, 4:
    // radices 8 and 9 (df64 internal twiddles, 92 registers) measured slower
    // on the starfish, 0.53 -> 0.66 ms
    G.full = fft_shape(G.g, !f64);
    G.half = fft_shape(G.g / 2, false);
    if (G.full.nst <= 0 || G.half.nst <= 0 || (G.g & 1)) return LP_OK;
    if (fft_cols_smem(G.g, f64) > limit || fft_rows_smem(G.g, f64) > limit) return LP_OK;
  }
  if (!fft_dd_configure()) return LP_ERR_CUDA;
  for (int l = P.l0; l < 2; ++l) {
    GridLevel& G = P.lv[l];
    G.kp = (G.K + 2) & ~1;
    const size_t spec_bytes = (size_t)G.g * G.kp * (f64 ? sizeof(float4) : sizeof(float2));
    for (int c = 0; c < 4; ++c)
      if (!dalloc(P, &G.spec[c], spec_bytes)) return LP_ERR_NOMEM;
    const std::vector<float4> tw = fft_twiddles(G.g);
    if (!dalloc(P, (void**)&G.tw_dd, tw.size() * sizeof(float4))) return LP_ERR_NOMEM;
    cudaMemcpy(G.tw_dd, tw.data(), tw.size() * sizeof(float4), cudaMemcpyHostToDevice);
    const std::vector<int> fr = fft_dif_order(G.full);
    if (!dalloc(P, (void**)&G.freq, fr.size() * sizeof(int))) return LP_ERR_NOMEM;
    cudaMemcpy(G.freq, fr.data(), fr.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (f64) {
      const size_t ntab = (size_t)(G.K + 1) * (G.K + 1);
      if (!dalloc(P, (void**)&G.mtab_dd, ntab * sizeof(float2))) return LP_ERR_NOMEM;
      launch_split_table(G.mtab, G.mtab_dd, (int64_t)ntab, P.stream);
    }
  }
  for (int k = 0; k < P.es.nc; ++k)
    for (int t = 0; t < P.es.w; ++t) P.es_dd[k][t] = split_host(P.es.c[k][t]);
  if (cudaStreamSynchronize(P.stream) != cudaSuccess) return LP_ERR_CUDA;
  P.own_fft = true;
  return LP_OK;
}

// Steps 2-4 with the FFT chain: forward row transforms of the spread grids,
// the fused column pass (transform, multiplier, inverse transform) and the
// inverse row transforms (stage events recorded when `events`).
void history_transforms(const Plan& P, bool wv, bool ws, bool wd, cudaStream_t s, bool events) {
  const bool f64 = P.precision == LP_FP64;
  int fch[4], nf = 0;
  if (wv) fch[nf++] = 0;
  if (ws) fch[nf++] = 1;
  if (wd) {
    fch[nf++] = 2;
    fch[nf++] = 3;
  }
  int ich[3], ni = 0;
  if (wv) ich[ni++] = 0;
  if (ws) ich[ni++] = 1;
  if (wd) ich[ni++] = 2;
  auto row_args = [&](const GridLevel& G, const int* ch, int n) {
    FftRowArgs a{};
    a.half = G.half;
    a.tw = G.tw_dd;
    for (int i = 0; i < n; ++i) {
      a.grid[i] = G.chan[ch[i]];
      a.spec[i] = G.spec[ch[i]];
    }
    a.pitch = G.pitch;
    a.kp = G.kp;
    a.K = G.K;
    a.row_lo = G.row_lo;
    a.row_hi = G.row_hi;
    return a;
  };
  for (int l = P.l0; l < 2; ++l) {
    launch_fft_rows_fwd(row_args(P.lv[l], fch, nf), nf, f64, s);
    ++P.launches;
  }
  if (events) record_stage(P, 4, s);
  for (int l = P.l0; l < 2; ++l) {
    const GridLevel& G = P.lv[l];
    FftColArgs a{};
    a.full = G.full;
    a.tw = G.tw_dd;
    a.freq = G.freq;
    a.tab = f64 ? (const void*)G.mtab_dd : (const void*)G.mtab32;
    a.tab64 = f64 ? nullptr : G.mtab;
    a.klo = f64 ? 0 : kLowKFP64;
    a.dk = f64 ? split_host(G.dk) : make_float2((float)G.dk, (float)(G.dk - (double)(float)G.dk));
    int nj = 0;
    if (wv) a.job[nj++] = FftColJob{0, {G.spec[0], nullptr}, G.spec[0]};
    if (ws) a.job[nj++] = FftColJob{0, {G.spec[1], nullptr}, G.spec[1]};
    if (wd) a.job[nj++] = FftColJob{1, {G.spec[2], G.spec[3]}, G.spec[2]};
    a.kp = G.kp;
    a.K = G.K;
    a.row_lo = G.row_lo;
    a.row_hi = G.row_hi;
    launch_fft_cols(a, nj, f64, s);
    ++P.launches;
  }
  if (events) record_stage(P, 5, s);
  for (int l = P.l0; l < 2; ++l) {
    launch_fft_rows_inv(row_args(P.lv[l], ich, ni), ni, f64, s);
    ++P.launches;
  }
  if (events) record_stage(P, 6, s);
}

// Step 4 after the FFT chain: interpolation from the chain's grids (df64
// pairs for FP64 plans, floats for FP32 plans).
// Argument record of the df64 interpolation of an FP64 plan on the FFT chain.
InterpDDArgs make_interp_dd_args(const Plan& P, int64_t nt, const double* txy, double* const* dout) {
  InterpDDArgs a{};
  a.txy = txy;
  a.n = nt;
  a.l0 = P.l0;
  for (int l = P.l0; l < 2; ++l) {
    const GridLevel& G = P.lv[l];
    InterpDDLevel& L = a.lv[l];
    for (int c = 0; c < 3; ++c) L.grid[c] = G.chan[c];
    L.g = G.g;
    L.pitch = G.pitch;
    L.x0 = split_host(G.x0);
    L.y0 = split_host(G.y0);
    L.inv_h = split_host(1.0 / G.h);
  }
  for (int c = 0; c < 3; ++c) a.out[c] = dout[c];
  a.status = P.d_status;
  a.nc = P.es.nc;
  a.nf = P.es_float_steps;
  std::memcpy(a.coef, P.es_dd, sizeof(a.coef));
  return a;
}

void history_interp(const Plan& P, int64_t nt, const double* txy, double* const* dout, cudaStream_t s) {
  if (P.precision != LP_FP64) {
    launch_interp(P, nt, txy, dout[0], dout[1], dout[2], s);
    return;
  }
  launch_interp_dd(make_interp_dd_args(P, nt, txy, dout), P.ker.w, s);
  ++P.launches;
}

}  // namespace lpg

extern "C" {

const char* lp_status_string(lp_status s) {
  switch (s) {
    case LP_OK: return "ok";
    case LP_ERR_ARG: return "invalid argument";
    case LP_ERR_OUT_OF_BOX: return "a source or target lies outside the plan's box";
    case LP_ERR_NOMEM: return "device allocation failed";
    case LP_ERR_CUDA: return "CUDA runtime or cuFFT failure";
    case LP_ERR_UNSUPPORTED:
      return "volume potential requested at an exterior target inside the local band";
    case LP_ERR_STATE: return "call order violated";
    case LP_ERR_NEWTON: return "closest-point search did not converge for a target near the boundary";
    case LP_ERR_TIMEOUT: return "the plan's work did not complete within the time limit";
  }
  return "unknown status";
}

// Refinement levels of a plan: explicit, or (LP_REFINE_AUTO) the smallest J
// with (delta/4^J)^(order/2) <= tol, the selection rule of Sec. 4.4 for an
// expansion whose error is O(delta^(order/2)), capped at kMaxDyLevels.
static int refine_levels_for(int requested, double delta, double tol, int order) {
  if (requested != LP_REFINE_AUTO) return requested;
  int J = 0;
  while (J < kMaxDyLevels && std::pow(delta / std::pow(4.0, J), 0.5 * order) > tol) ++J;
  return J;
}

lp_status lp_plan(const lp_domain* dom, double delta, double tol, lp_plan_t* out) {
  if (!dom || !out) return LP_ERR_ARG;
  *out = nullptr;
  if (!(delta > 0.0) || !std::isfinite(delta)) return LP_ERR_ARG;
  if (!(tol >= 1e-13 && tol <= 1e-2)) return LP_ERR_ARG;
  if (dom->precision != LP_FP64 && dom->precision != LP_FP32) return LP_ERR_ARG;
  if (dom->precision == LP_FP32 && tol < 1e-6) return LP_ERR_ARG;
  int order = dom->order == 0 ? 5 : dom->order;
  if (order < 3 || order > 5) return LP_ERR_ARG;
  for (int d = 0; d < 2; ++d)
    if (!(dom->box_hi[d] > dom->box_lo[d]) || !std::isfinite(dom->box_lo[d]) ||
        !std::isfinite(dom->box_hi[d]))
      return LP_ERR_ARG;
  if (dom->n_panels < 0 || dom->max_device_bytes < 0) return LP_ERR_ARG;
  if (dom->autotune < 0 || dom->autotune > LP_AUTOTUNE_FULL) return LP_ERR_ARG;
  if (dom->refine_levels < LP_REFINE_AUTO || dom->refine_levels > kMaxDyLevels) return LP_ERR_ARG;
  if (dom->levels < LP_LEVELS_AUTO || dom->levels > 2) return LP_ERR_ARG;
  if (dom->upsampling != 0.0 && !(dom->upsampling >= 1.25 && dom->upsampling <= 3.0)) return LP_ERR_ARG;
  if (dom->n_panels > 0) {
    if (dom->panel_order < 2 || dom->panel_order > kMaxPanelOrder) return LP_ERR_ARG;
    if (!dom->bnd_xy || !dom->bnd_w) return LP_ERR_ARG;
    if (dom->n_panels > (int64_t)1 << 26) return LP_ERR_ARG;
  }
  lp_plan_s* h = new (std::nothrow) lp_plan_s();
  if (!h) return LP_ERR_NOMEM;
  Plan& P = h->P;
  P.precision = dom->precision;
  P.order = order;
  P.delta1 = delta;
  P.autotune = dom->autotune != 0;
  P.tune_grids = dom->autotune == LP_AUTOTUNE_FULL;
  P.l0 = dom->levels == 1 ? 1 : 0;
  P.delta2 = P.l0 ? delta : 32.0 * delta;
  P.tol = tol;
  for (int d = 0; d < 2; ++d) {
    P.box_lo[d] = dom->box_lo[d];
    P.box_hi[d] = dom->box_hi[d];
  }
  P.side = std::max(P.box_hi[0] - P.box_lo[0], P.box_hi[1] - P.box_lo[1]);
  P.on_tol = 1e-12 * P.side;
  P.stream = (cudaStream_t)dom->stream;
  P.max_bytes = dom->max_device_bytes > 0 ? (size_t)dom->max_device_bytes : 0;
  // Kernel width and upsampling.  FP64 is bound by cuFFT's FP64 arithmetic,
  // so its grids use sigma = 1.5 (0.56x the modes of sigma = 2) and wider
  // kernels; FP32 keeps sigma = 2.  Measured (disk, tol 1e-9): sigma 2, w 10
  // -> 4.3e-10; sigma 1.5, w 11 -> 3.9e-10, w 12 -> 5.6e-11.  Small, many-
  // lobed problems reached 1.2e-9 at w 11, so FP64 takes w = ceil(-log10 tol)
  // + 3 (12 at 1e-9); FP32 takes + 2 (7 at 1e-5) for margin against
  // single-precision rounding.
  // Other upsampling factors (1.25 .. 3) take the width at which the ES
  // kernel's aliasing error e^{-pi w sqrt(1 - 1/sigma)} reaches tol, plus one.
  const double sigma_default = P.precision == LP_FP64 ? 1.5 : 2.0;
  P.sigma = dom->upsampling > 0.0 ? dom->upsampling : sigma_default;
  int w;
  if (P.sigma == sigma_default) {
    w = (int)std::ceil(-std::log10(tol)) + (P.precision == LP_FP64 ? 3 : 2);
  } else {
    w = (int)std::ceil(std::log(1.0 / tol) / (3.14159265358979323846 * std::sqrt(1.0 - 1.0 / P.sigma))) + 1;
    if (w > kMaxW) {
      delete h;
      return LP_ERR_ARG;  // tolerance out of reach at this upsampling
    }
  }
  w = std::min(std::max(w, 4), kMaxW);
  if (cudaGetDevice(&P.device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return LP_ERR_CUDA;
  }
  P.ker.w = w;
  P.ker.beta = 2.30 * w;  // refined by choose_levels for the realised sigma
  P.ker.half_w = 0.5 * w;
  if (dom->levels == LP_LEVELS_AUTO) {
    // one level when its grid is small: the launch chain of the second level
    // then costs more than the larger single grid (measured on GB300)
    Plan Q = P;
    Q.l0 = 1;
    Q.delta2 = delta;
    if (choose_levels(Q) == LP_OK && Q.lv[1].g <= LP_SINGLE_LEVEL_MAX_GRID) {
      P.l0 = 1;
      P.delta2 = delta;
    }
  }
  lp_status st = choose_levels(P);
  if (st == LP_OK) st = fit_kernel_poly(P);  // the tables deconvolve by the fitted kernel
  if (st == LP_OK) st = build_tables(P);
  const size_t rs = P.precision == LP_FP64 ? sizeof(double) : sizeof(float);
  for (int l = P.l0; l < 2 && st == LP_OK; ++l) {
    GridLevel& G = P.lv[l];
    G.chan_bytes = (size_t)G.g * G.pitch * rs;
    for (int c = 0; c < 4 && st == LP_OK; ++c)
      if (!dalloc(P, &G.chan[c], G.chan_bytes)) st = LP_ERR_NOMEM;
  }
  if (st == LP_OK) {
    if (!dalloc(P, (void**)&P.d_status, sizeof(unsigned)) ||
        !dalloc(P, (void**)&P.d_qsum, 2 * sizeof(double)))
      st = LP_ERR_NOMEM;
    else if (cudaMallocHost((void**)&P.h_status, sizeof(unsigned)) != cudaSuccess)
      st = LP_ERR_NOMEM;
    else {
      cudaMemset(P.d_status, 0, sizeof(unsigned));
      cudaMemset(P.d_qsum, 0, 2 * sizeof(double));
      for (auto& e : P.ev) cudaEventCreate(&e);
    }
  }
  if (st == LP_OK && dom->n_panels > 0) {
    P.n_panels = dom->n_panels;
    P.p = dom->panel_order;
    P.nb = P.n_panels * P.p;
    std::vector<double> hxy(P.nb * 2), hw(P.nb), hn(P.nb * 2);
    auto fetch = [&](const double* src, double* dst, size_t count) {
      if (is_device_ptr(src))
        cudaMemcpy(dst, src, count * sizeof(double), cudaMemcpyDeviceToHost);
      else
        std::memcpy(dst, src, count * sizeof(double));
    };
    fetch(dom->bnd_xy, hxy.data(), hxy.size());
    fetch(dom->bnd_w, hw.data(), hw.size());
    if (dom->bnd_normal)
      fetch(dom->bnd_normal, hn.data(), hn.size());
    else
      derive_normals(P.n_panels, P.p, hxy.data(), hn.data());
    bool finite = true;
    for (double v : hxy) finite &= std::isfinite(v);
    for (double v : hw) finite &= std::isfinite(v);
    if (!finite) st = LP_ERR_ARG;
    if (st == LP_OK) st = build_boundary(P, hxy.data(), hw.data(), hn.data());
    if (st == LP_OK) st = setup_dyadic(P, refine_levels_for(dom->refine_levels, delta, tol, order));
  }
  if (st == LP_OK) st = setup_bins(P);
  if (st == LP_OK) st = setup_fft_chain(P);
  // cuFFT plans only for grids the library's own FFT chain cannot hold
  for (int l = P.l0; l < 2 && st == LP_OK && !P.own_fft; ++l) st = make_fft_plans(P, P.lv[l]);
  if (st == LP_OK) st = status_from_cuda();
  if (st != LP_OK) {
    destroy_plan(P);
    delete h;
    return st;
  }
  *out = h;
  return LP_OK;
}

// Counting sort of the bound volume nodes into the current bins.
static void bin_volume(Plan& P, int64_t n) {
  if (P.precision == LP_FP64) {
    launch_bin_sort_dd(P.d_vxy, n, P.bins, P.d_keys, P.d_counts, P.d_cursor, P.d_vstart, P.d_vrel_dd, P.d_vperm,
                       P.d_status, P.stream);
    launch_gather_q_dd(P.d_vq, P.d_vperm, n, P.d_vq_dd, P.stream);
  } else {
    launch_bin_sort(P.d_vxy, n, P.bins, P.d_keys, P.d_counts, P.d_cursor, P.d_vstart, P.d_vrel_s, P.d_vperm,
                    P.d_status, P.stream);
    launch_gather_q(P.d_vq, n, 1, P.d_vperm, n, P.d_vq_s, P.stream);
  }
  P.launches += 4;
}

// Autotuner of the bin side: for each candidate, bin the bound volume nodes
// and time the binned spread of both levels (median of three after one
// warm-up, CUDA events on the plan's stream; the grids are scratch until
// lp_execute zeroes them); keep the fastest and bin with it.
static lp_status tune_bins(Plan& P, int64_t n) {
  const int f64 = P.precision == LP_FP64 ? 1 : 0;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LP_ERR_CUDA;
  const int base = P.bin_cells;
  int best = base;
  float best_ms = 1e30f;
  for (int c = 0; c < 3; ++c) {
    const int cells = kBinCandidates[f64][c];
    P.tune_ms[c] = -1.f;
    if (!configure_bins(P, cells)) continue;
    bin_volume(P, n);
    float t[3];
    for (int r = 0; r < 4; ++r) {
      cudaEventRecord(e0, P.stream);
      for (int l = P.l0; l < 2; ++l) spread_volume_binned(P, l, P.stream);
      cudaEventRecord(e1, P.stream);
      cudaEventSynchronize(e1);
      if (r > 0) cudaEventElapsedTime(&t[r - 1], e0, e1);
    }
    std::sort(t, t + 3);
    P.tune_ms[c] = t[1];
    if (t[1] < best_ms) {
      best_ms = t[1];
      best = cells;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!configure_bins(P, best)) configure_bins(P, base);
  bin_volume(P, n);
  P.tuned = true;
  const lp_status bs = bin_boundary(P);
  if (bs != LP_OK) return bs;
  return status_from_cuda();
}

static lp_status tune_grids(lp_plan_t h, int64_t n, const double* xy, const double* w, const double* f);

lp_status lp_volume(lp_plan_t h, int64_t n, const double* xy, const double* w, const double* f) {
  if (!h || n < 0) return LP_ERR_ARG;
  if (n > 0 && (!xy || !w || !f)) return LP_ERR_ARG;
  if (h->P.tune_grids && n > 0) {
    const lp_status st = tune_grids(h, n, xy, w, f);  // may replace h->P by a faster configuration
    if (st != LP_OK) return st;
  }
  Plan& P = h->P;
  if (n > P.v_cap) {
    cudaStreamSynchronize(P.stream);
    drelease(P, P.d_vxy, P.v_cap * 2 * sizeof(double));
    drelease(P, P.d_vq, P.v_cap * sizeof(double));
    drelease(P, P.d_vf, P.v_cap * sizeof(double));
    P.v_cap = 0;
    P.nv = 0;
    P.have_volume = false;
    if (!dalloc(P, (void**)&P.d_vxy, n * 2 * sizeof(double)) ||
        !dalloc(P, (void**)&P.d_vq, n * sizeof(double)) || !dalloc(P, (void**)&P.d_vf, n * sizeof(double)))
      return LP_ERR_NOMEM;
    P.v_cap = n;
  }
  P.nv = n;
  if (n > 0) {
    // staging only for the arrays that are in host memory
    const size_t stage = (is_device_ptr(xy) ? 0 : round256(n * 2 * sizeof(double))) +
                         (is_device_ptr(w) ? 0 : round256(n * sizeof(double))) +
                         (is_device_ptr(f) ? 0 : round256(n * sizeof(double)));
    if (!ensure_stage(P, stage)) return LP_ERR_NOMEM;
    size_t off = 0;
    const double* dxy = device_view(P, xy, n * 2, &off, P.stream);
    const double* dw = device_view(P, w, n, &off, P.stream);
    const double* df = device_view(P, f, n, &off, P.stream);
    cudaMemcpyAsync(P.d_vxy, dxy, n * 2 * sizeof(double), cudaMemcpyDeviceToDevice, P.stream);
    cudaMemcpyAsync(P.d_vf, df, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream);
    launch_volume_q(P, df, dw, P.d_vq, n, P.stream);
  }
  if (P.binned && n > 0) {
    // sort the volume nodes into the spread's bins
    const bool f64 = P.precision == LP_FP64;
    if ((size_t)n > P.key_cap || (size_t)n > P.vsort_cap) {
      cudaStreamSynchronize(P.stream);
      if ((size_t)n > P.key_cap) {
        drelease(P, P.d_keys, P.key_cap * sizeof(int));
        P.key_cap = 0;
        if (!dalloc(P, (void**)&P.d_keys, n * sizeof(int))) return LP_ERR_NOMEM;
        P.key_cap = n;
      }
      if ((size_t)n > P.vsort_cap) {
        const size_t c = P.vsort_cap;
        drelease(P, P.d_vperm, c * sizeof(int));
        drelease(P, P.d_vrel_s, f64 ? 0 : c * sizeof(float2));
        drelease(P, P.d_vq_s, f64 ? 0 : c * sizeof(float));
        drelease(P, P.d_vrel_dd, f64 ? c * sizeof(float4) : 0);
        drelease(P, P.d_vq_dd, f64 ? c * sizeof(float2) : 0);
        P.vsort_cap = 0;
        const bool ok = dalloc(P, (void**)&P.d_vperm, n * sizeof(int)) &&
                        (f64 ? dalloc(P, (void**)&P.d_vrel_dd, n * sizeof(float4)) &&
                                   dalloc(P, (void**)&P.d_vq_dd, n * sizeof(float2))
                             : dalloc(P, (void**)&P.d_vrel_s, n * sizeof(float2)) &&
                                   dalloc(P, (void**)&P.d_vq_s, n * sizeof(float)));
        if (!ok) return LP_ERR_NOMEM;
        P.vsort_cap = n;
      }
    }
    bin_volume(P, n);
    if (P.autotune && !P.tuned) {
      const lp_status st = tune_bins(P, n);
      if (st != LP_OK) return st;
    }
  }
  launch_sum(P, P.d_vq, n, P.d_qsum, P.stream);
  P.have_volume = true;
  return status_from_cuda();
}

static lp_status bind_layer(lp_plan_t h, const double* dens, int kind) {
  if (!h || !dens) return LP_ERR_ARG;
  Plan& P = h->P;
  if (P.nb == 0) return LP_ERR_STATE;
  if (!is_device_ptr(dens) && !ensure_stage(P, round256(P.nb * sizeof(double)))) return LP_ERR_NOMEM;
  size_t off = 0;
  const double* d = device_view(P, dens, P.nb, &off, P.stream);
  double* dst = kind == 0 ? P.d_sigma : P.d_mu;
  cudaMemcpyAsync(dst, d, P.nb * sizeof(double), cudaMemcpyDeviceToDevice, P.stream);
  launch_panel_coef(P, dst, 1, 1, kind == 0 ? P.d_sigma_coef : P.d_mu_coef,
                    kind == 0 ? P.d_sigma_ref : P.d_mu_ref, P.stream);
  if (P.dy_levels > 0) launch_dyadic_dens(P, kind, P.stream);
  // single-precision copy for the local expansions (both precisions)
  launch_to_float(kind == 0 ? P.d_sigma_coef : P.d_mu_coef, kind == 0 ? P.d_sigma_coef32 : P.d_mu_coef32,
                  P.n_panels * P.p, P.stream);
  launch_split_table(kind == 0 ? P.d_sigma_coef : P.d_mu_coef, kind == 0 ? P.d_sigma_coef_dd : P.d_mu_coef_dd,
                     P.n_panels * P.p, P.stream);
  ++P.launches;
  launch_strengths(P, kind, P.stream);
  gather_layer_strengths(P, kind);
  if (kind == 0) {
    launch_sum(P, P.d_bq, P.nb, P.d_qsum + 1, P.stream);
    P.have_sigma = true;
  } else {
    P.have_mu = true;
  }
  return status_from_cuda();
}

lp_status lp_single_layer(lp_plan_t h, const double* sigma) { return bind_layer(h, sigma, 0); }
lp_status lp_double_layer(lp_plan_t h, const double* mu) { return bind_layer(h, mu, 1); }

// Grid autotuner (LP_AUTOTUNE_FULL): the upsampling sigma and the number of
// history levels trade transform size against stencil width and launch
// count (Sec. 3's remark on one level against two), so the first lp_volume
// builds a plan for each sigma in {1.25, 1.5, 2} with one and with two
// levels -- each with the kernel width that sigma needs for the plan's
// tolerance -- on the plan's own boundary, binds the sources (and unit
// layer densities), and times one V (+ S + D) evaluation at the sources
// (median of three after a warm-up, CUDA events on the plan's stream).  The
// fastest configuration replaces the plan's grids; its bins are then tuned
// as for LP_AUTOTUNE_BINS.  Scratch for the timing is allocated and freed
// here.
static lp_status tune_grids(lp_plan_t h, int64_t n, const double* xy, const double* w, const double* f) {
  Plan& P0 = h->P;
  P0.tune_grids = false;
  const double sigmas[3] = {1.25, 1.5, 2.0};
  lp_domain dom{};
  dom.precision = P0.precision;
  dom.order = P0.order;
  for (int d = 0; d < 2; ++d) {
    dom.box_lo[d] = P0.box_lo[d];
    dom.box_hi[d] = P0.box_hi[d];
  }
  dom.n_panels = P0.n_panels;
  dom.panel_order = P0.p;
  dom.bnd_xy = P0.d_bxy;
  dom.bnd_w = P0.d_bw;
  dom.bnd_normal = P0.d_bnrm;
  dom.stream = P0.stream;
  dom.refine_levels = P0.dy_levels;
  dom.autotune = 0;
  dom.max_device_bytes = (int64_t)P0.max_bytes;
  const int64_t nb = P0.nb;
  // scratch: zero jets, three outputs, unit densities
  double* tmp = nullptr;
  const size_t tmp_n = (size_t)9 * n + 2 * (size_t)nb;
  if (cudaMalloc((void**)&tmp, tmp_n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return LP_ERR_NOMEM;
  }
  cudaMemsetAsync(tmp, 0, (size_t)9 * n * sizeof(double), P0.stream);
  std::vector<double> ones((size_t)2 * nb, 1.0);
  if (nb) cudaMemcpy(tmp + 9 * n, ones.data(), ones.size() * sizeof(double), cudaMemcpyHostToDevice);
  double* jet = tmp;
  double* outv[3] = {tmp + 6 * n, nb ? tmp + 7 * n : nullptr, nb ? tmp + 8 * n : nullptr};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  lp_plan_s* best = nullptr;
  float best_ms = 1e30f;
  float ms_all[6];
  for (int c = 0; c < 6; ++c) {
    ms_all[c] = -1.f;
    dom.upsampling = sigmas[c / 2];
    dom.levels = 1 + (c % 2);
    lp_plan_s* cand = nullptr;
    if (lp_plan(&dom, P0.delta1, P0.tol, &cand) != LP_OK) continue;
    lp_status st = lp_volume(cand, n, xy, w, f);
    if (st == LP_OK && nb) st = lp_single_layer(cand, tmp + 9 * n);
    if (st == LP_OK && nb) st = lp_double_layer(cand, tmp + 9 * n + nb);
    float t[3] = {0, 0, 0};
    for (int r = 0; r < 4 && st == LP_OK; ++r) {
      cudaEventRecord(e0, cand->P.stream);
      st = lp_execute(cand, n, cand->P.d_vxy, jet, outv[0], outv[1], outv[2]);
      cudaEventRecord(e1, cand->P.stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = LP_ERR_CUDA;
      if (r > 0) cudaEventElapsedTime(&t[r - 1], e0, e1);
    }
    if (st == LP_OK) st = lp_sync(cand);
    if (st != LP_OK) {
      lp_destroy(cand);
      cudaGetLastError();
      continue;
    }
    std::sort(t, t + 3);
    ms_all[c] = t[1];
    if (t[1] < best_ms) {
      if (best) lp_destroy(best);
      best = cand;
      best_ms = t[1];
    } else {
      lp_destroy(cand);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(P0.stream);
  cudaFree(tmp);
  if (!best) return LP_OK;  // no candidate could be built: keep the plan as created
  // the winner takes over the handle; densities already bound move with it
  const bool bins = P0.autotune;
  const bool had_sigma = P0.have_sigma, had_mu = P0.have_mu;
  std::swap(h->P, best->P);  // best now holds the plan as created
  Plan& P = h->P;
  P.autotune = bins;
  P.tuned = false;
  P.tune_grids = false;
  P.have_volume = false;
  P.launches += best->P.launches;
  for (int c = 0; c < 6; ++c) P.grid_ms[c] = ms_all[c];
  lp_status st = LP_OK;
  if (had_sigma) st = lp_single_layer(h, best->P.d_sigma);
  if (st == LP_OK && had_mu) st = lp_double_layer(h, best->P.d_mu);
  else if (!had_mu) P.have_mu = false;
  if (!had_sigma) P.have_sigma = false;
  cudaStreamSynchronize(P.stream);
  lp_destroy(best);
  return st;
}

// Steps 2-3 on device buffers (stage events 2, 10, 3): zero the grids of the
// requested channels and spread onto them the bound volume nodes (when
// `volume`: through the bins, or point-parallel with global atomics) and
// boundary nodes (when `layers`: point-parallel).  Allocates nothing.
static void spread_part(Plan& P, bool wv, bool ws, bool wd, bool volume, bool layers, cudaStream_t s) {
  for (int l = P.l0; l < 2; ++l) {
    GridLevel& G = P.lv[l];
    if (wv) cudaMemsetAsync(G.chan[0], 0, G.chan_bytes, s);
    if (ws) cudaMemsetAsync(G.chan[1], 0, G.chan_bytes, s);
    if (wd) {
      cudaMemsetAsync(G.chan[2], 0, G.chan_bytes, s);
      cudaMemsetAsync(G.chan[3], 0, G.chan_bytes, s);
    }
  }
  record_stage(P, 2, s);
  for (int l = P.l0; l < 2; ++l) {
    GridLevel& G = P.lv[l];
    if (wv && volume && P.nv > 0) {
      if (P.binned) {
        spread_volume_binned(P, l, s);
      } else {
        const double* q[1] = {P.d_vq};
        void* g[1] = {G.chan[0]};
        launch_spread(P, l, P.d_vxy, q, 1, g, P.nv, s);
      }
    }
  }
  record_stage(P, 10, s);
  for (int l = P.l0; l < 2; ++l) {
    GridLevel& G = P.lv[l];
    const double* bq[3];
    void* bg[3];
    int nq = 0;
    if (ws) {
      bq[nq] = P.d_bq;
      bg[nq++] = G.chan[1];
    }
    if (wd) {
      bq[nq] = P.d_bq + P.nb;
      bg[nq++] = G.chan[2];
      bq[nq] = P.d_bq + 2 * P.nb;
      bg[nq++] = G.chan[3];
    }
    if (!nq || !layers) continue;
    if (P.bbinned) {
      SubDDArgs a = make_spread_dd_args(P, l);
      a.rel = P.d_brel_dd;
      a.start = P.d_bstart;
      FxChan ch{};
      int k = 0;
      if (ws) {
        ch.q[k] = P.d_bq_dd;
        ch.grid[k++] = G.chan[1];
      }
      if (wd) {
        ch.q[k] = P.d_bq_dd + P.nb;
        ch.grid[k++] = G.chan[2];
        ch.q[k] = P.d_bq_dd + 2 * P.nb;
        ch.grid[k++] = G.chan[3];
      }
      ++P.launches;
      launch_spread_fx_list(a, P.d_bbins, P.n_bbins, ch, k, P.ker.w, s);
    } else {
      launch_spread(P, l, P.d_bxy, bq, nq, bg, P.nb, s);
    }
  }
  record_stage(P, 3, s);
}

// Step 4 and the local part from the spread grids (stage events 4 .. 8):
// transform with the multiplier (the library's FFT chain, or cuFFT with the
// multiplier kernel), interpolate, then the local correction and the
// refinement sums.  dt, dj, dout: device targets, jets and outputs; list,
// count: the near-boundary list of the local pass (one int2 per target) and
// its counter; staged: an event the interpolation waits for (targets copied
// on another stream), or null.  Allocates nothing.
static void finish_part(Plan& P, int64_t nt, const double* dt, const double* dj, double* const* dout, bool wv,
                        bool ws, bool wd, int2* list, int* count, cudaEvent_t staged, cudaStream_t s) {
  if (P.own_fft) {
    history_transforms(P, wv, ws, wd, s, true);
    if (staged) cudaStreamWaitEvent(s, staged, 0);
    history_interp(P, nt, dt, dout, s);
  } else {
    for (int l = P.l0; l < 2; ++l) {
      if (wv) fft_forward(P, l, 0);
      if (ws) fft_forward(P, l, 1);
      if (wd) {
        fft_forward(P, l, 2);
        fft_forward(P, l, 3);
      }
    }
    record_stage(P, 4, s);
    // Step 4: deconvolved multiplier (in place; D written to channel 2)
    for (int l = P.l0; l < 2; ++l) launch_multiplier(P, l, wv, ws, wd, s);
    record_stage(P, 5, s);
    for (int l = P.l0; l < 2; ++l) {
      if (wv) fft_inverse(P, l, 0);
      if (ws) fft_inverse(P, l, 1);
      if (wd) fft_inverse(P, l, 2);
    }
    record_stage(P, 6, s);
    if (staged) cudaStreamWaitEvent(s, staged, 0);
    launch_interp(P, nt, dt, dout[0], dout[1], dout[2], s);
  }
  record_stage(P, 7, s);
  launch_local_list(P, nt, dt, dj, dout[0], dout[1], dout[2], list, count, s);
  record_stage(P, 11, s);
  launch_dyadic(P, nt, dt, dout[1], dout[2], list, count, s);
  record_stage(P, 8, s);
}

static void device_pipeline(Plan& P, int64_t nt, const double* dt, const double* dj, double* const* dout,
                            bool wv, bool ws, bool wd, int2* list, int* count, cudaEvent_t staged,
                            cudaStream_t s) {
  spread_part(P, wv, ws, wd, true, true, s);
  finish_part(P, nt, dt, dj, dout, wv, ws, wd, list, count, staged, s);
}

lp_status lp_execute(lp_plan_t h, int64_t nt, const double* txy, const double* jet, double* V,
                     double* S, double* D) {
  if (!h || nt < 0 || nt > (int64_t)INT32_MAX) return LP_ERR_ARG;
  if (nt > 0 && !txy) return LP_ERR_ARG;
  Plan& P = h->P;
  const bool wv = V != nullptr, ws = S != nullptr, wd = D != nullptr;
  if (wv && nt > 0 && !jet) return LP_ERR_ARG;
  if ((wv && !P.have_volume) || (ws && !P.have_sigma) || (wd && !P.have_mu)) return LP_ERR_STATE;
  if (nt == 0 || (!wv && !ws && !wd)) return LP_OK;
  cudaStream_t s = P.stream;
  // staging for the targets and jets that are in host memory
  const size_t need = (is_device_ptr(txy) ? 0 : round256(nt * 2 * sizeof(double))) +
                      (!wv || is_device_ptr(jet) ? 0 : round256(nt * 6 * sizeof(double)));
  if (!ensure_stage(P, need)) return LP_ERR_NOMEM;
  double* outs[3] = {V, S, D};
  bool host_out[3];
  bool any_host = false;
  for (int c = 0; c < 3; ++c) {
    host_out[c] = outs[c] && !is_device_ptr(outs[c]);
    any_host |= host_out[c];
  }
  if (any_host && (size_t)nt > P.out_cap) {
    cudaStreamSynchronize(s);
    drelease(P, P.d_out, 3 * P.out_cap * sizeof(double));
    P.out_cap = 0;
    if (!dalloc(P, (void**)&P.d_out, 3 * nt * sizeof(double))) return LP_ERR_NOMEM;
    P.out_cap = nt;
  }
  if ((size_t)nt > P.near_cap) {
    cudaStreamSynchronize(s);
    drelease(P, P.d_near, P.near_cap * sizeof(int2));
    P.near_cap = 0;
    if (!dalloc(P, (void**)&P.d_near, nt * sizeof(int2))) return LP_ERR_NOMEM;
    P.near_cap = nt;
  }
  if (!P.d_near_count && !dalloc(P, (void**)&P.d_near_count, sizeof(int))) return LP_ERR_NOMEM;
  record_stage(P, 0, s);
  // Host targets and jets are copied on the plan's copy stream, overlapping
  // the spreads and transforms; the staging buffer is free once the work
  // already queued on the plan's stream has run, and the interpolation
  // waits for the copies.
  const bool host_in = !is_device_ptr(txy) || (wv && !is_device_ptr(jet));
  cudaStream_t cs = s;
  if (host_in) {
    if (!P.copy_stream) {
      if (cudaStreamCreateWithFlags(&P.copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&P.ev_in, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&P.ev_staged, cudaEventDisableTiming) != cudaSuccess)
        return LP_ERR_CUDA;
    }
    cudaEventRecord(P.ev_in, s);
    cudaStreamWaitEvent(P.copy_stream, P.ev_in, 0);
    cs = P.copy_stream;
  }
  size_t off = 0;
  const double* dt = device_view(P, txy, nt * 2, &off, cs);
  const double* dj = wv ? device_view(P, jet, nt * 6, &off, cs) : nullptr;
  if (host_in) cudaEventRecord(P.ev_staged, cs);
  double* dout[3];
  for (int c = 0; c < 3; ++c) dout[c] = host_out[c] ? P.d_out + c * nt : outs[c];
  record_stage(P, 1, s);

  device_pipeline(P, nt, dt, dj, dout, wv, ws, wd, P.d_near, P.d_near_count, host_in ? P.ev_staged : nullptr,
                  s);
  for (int c = 0; c < 3; ++c)
    if (host_out[c]) cudaMemcpyAsync(outs[c], dout[c], nt * sizeof(double), cudaMemcpyDeviceToHost, s);
  record_stage(P, 9, s);
  return status_from_cuda();
}

// lp_execute replayed from a CUDA graph.  A miss (new pointers, target
// count, source count, or any reallocation or bin change since the capture)
// runs lp_execute directly -- which also grows every buffer to its final
// capacity -- and then captures a second lp_execute, issued on the plan's
// graph stream, into an executable graph.  Each call (hit or miss) orders
// the graph stream after the work already on the plan's stream and the
// plan's stream after the replay, so plans on the legacy default stream work.
lp_status lp_execute_graph(lp_plan_t h, int64_t nt, const double* txy, const double* jet, double* V, double* S,
                           double* D) {
  if (!h || nt < 0 || nt > (int64_t)INT32_MAX) return LP_ERR_ARG;
  Plan& P = h->P;
  const void* key[5] = {txy, V ? jet : nullptr, V, S, D};
  for (const void* b : key)
    if (b && !is_device_ptr(b)) return LP_ERR_ARG;  // device memory only: no staging copies in a graph
  if (!P.own_fft || nt == 0 || (!V && !S && !D)) return lp_execute(h, nt, txy, jet, V, S, D);
  if (!P.graph_stream) {
    if (cudaStreamCreateWithFlags(&P.graph_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&P.ev_g0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&P.ev_g1, cudaEventDisableTiming) != cudaSuccess)
      return LP_ERR_CUDA;
  }
  bool hit = P.graph_exec && P.graph_nt == nt && P.graph_nv == P.nv && P.graph_gen == P.gen;
  for (int i = 0; i < 5 && hit; ++i) hit = P.graph_key[i] == key[i];
  if (!hit) {
    lp_status st = lp_execute(h, nt, txy, jet, V, S, D);  // this call's result; sizes every buffer
    if (st != LP_OK) return st;
    if (P.graph_exec) {
      cudaGraphExecDestroy(P.graph_exec);
      P.graph_exec = nullptr;
    }
    const unsigned long long gen0 = P.gen;
    const long long launches0 = P.launches;
    cudaStream_t user = P.stream;
    P.stream = P.graph_stream;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(P.graph_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      P.stream = user;
      return LP_ERR_CUDA;
    }
    P.capturing = true;
    st = lp_execute(h, nt, txy, jet, V, S, D);
    P.capturing = false;
    const cudaError_t ce = cudaStreamEndCapture(P.graph_stream, &graph);
    P.stream = user;
    P.graph_launches = P.launches - launches0;
    P.launches = launches0;  // captured, not run
    if (st != LP_OK || ce != cudaSuccess || P.gen != gen0) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return st != LP_OK ? st : LP_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&P.graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      P.graph_exec = nullptr;
      cudaGetLastError();
      return LP_ERR_CUDA;
    }
    P.graph_nt = nt;
    P.graph_nv = P.nv;
    P.graph_gen = P.gen;
    for (int i = 0; i < 5; ++i) P.graph_key[i] = key[i];
    return LP_OK;
  }
  cudaEventRecord(P.ev_g0, P.stream);
  cudaStreamWaitEvent(P.graph_stream, P.ev_g0, 0);
  if (cudaGraphLaunch(P.graph_exec, P.graph_stream) != cudaSuccess) {
    cudaGetLastError();
    return LP_ERR_CUDA;
  }
  cudaEventRecord(P.ev_g1, P.graph_stream);
  cudaStreamWaitEvent(P.stream, P.ev_g1, 0);
  P.launches += P.graph_launches;
  return status_from_cuda();
}

lp_status lp_execute_noalloc(lp_plan_t h, int64_t nt, const double* txy, const double* jet,
                             double* V, double* S, double* D) {
  if (!h || nt < 0 || nt > kNoAllocMaxTargets) return LP_ERR_ARG;
  if (nt > 0 && !txy) return LP_ERR_ARG;
  Plan& P = h->P;
  const bool wv = V != nullptr, ws = S != nullptr, wd = D != nullptr;
  if (wv && nt > 0 && !jet) return LP_ERR_ARG;
  if ((wv && !P.have_volume) || (ws && !P.have_sigma) || (wd && !P.have_mu)) return LP_ERR_STATE;
  if (nt == 0 || (!wv && !ws && !wd)) return LP_OK;
  // host buffers would need staging, i.e. an allocation: device memory only
  const void* bufs[5] = {txy, wv ? jet : nullptr, V, S, D};
  for (const void* b : bufs)
    if (b && !is_device_ptr(b)) return LP_ERR_ARG;
  // the scratch array is per device: only the plan's device may run it
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return LP_ERR_CUDA;
  }
  if (cur != P.device) return LP_ERR_ARG;
  void* scratch = nullptr;
  lp_status st = noalloc_scratch(P.device, &scratch);
  if (st != LP_OK) return st;
  int2* list = (int2*)scratch;
  int* count = (int*)((char*)scratch + kNoAllocListBytes);
  cudaStream_t s = P.stream;
  record_stage(P, 0, s);
  record_stage(P, 1, s);
  double* dout[3] = {V, S, D};
  device_pipeline(P, nt, txy, wv ? jet : nullptr, dout, wv, ws, wd, list, count, nullptr, s);
  record_stage(P, 9, s);
  return status_from_cuda();
}

lp_status lp_spread(lp_plan_t h, int outputs, int spread_layers) {
  if (!h || outputs <= 0 || outputs > 7) return LP_ERR_ARG;
  Plan& P = h->P;
  const bool wv = outputs & 1, ws = outputs & 2, wd = outputs & 4;
  if ((wv && !P.have_volume) || (spread_layers && ((ws && !P.have_sigma) || (wd && !P.have_mu))))
    return LP_ERR_STATE;
  if ((ws || wd) && P.nb == 0) return LP_ERR_STATE;
  if (!P.d_qred && !dalloc(P, (void**)&P.d_qred, 2 * sizeof(double))) return LP_ERR_NOMEM;
  cudaStream_t s = P.stream;
  record_stage(P, 0, s);
  record_stage(P, 1, s);
  spread_part(P, wv, ws, wd, true, spread_layers != 0, s);
  // the zero-mode sums this plan contributes (FP32 plans add the k = 0 term
  // from them): the volume strengths when it spread V, sigma w when it
  // spread the layers
  cudaMemsetAsync(P.d_qred, 0, 2 * sizeof(double), s);
  if (wv) cudaMemcpyAsync(P.d_qred, P.d_qsum, sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (ws && spread_layers) cudaMemcpyAsync(P.d_qred + 1, P.d_qsum + 1, sizeof(double), cudaMemcpyDeviceToDevice, s);
  P.spread_outputs = outputs;
  return status_from_cuda();
}

lp_status lp_grid_buffers(lp_plan_t h, void** ptrs, int64_t* bytes, int* dtypes, int* n) {
  if (!h || !n || *n < 0) return LP_ERR_ARG;
  const Plan& P = h->P;
  if (!P.spread_outputs) return LP_ERR_STATE;
  void* p[9];
  int64_t b[9];
  int t[9], k = 0;
  const int gtype = P.precision == LP_FP64 ? 0 : 1;
  for (int l = P.l0; l < 2; ++l) {
    const GridLevel& G = P.lv[l];
    const int chans[4] = {P.spread_outputs & 1 ? 0 : -1, P.spread_outputs & 2 ? 1 : -1,
                          P.spread_outputs & 4 ? 2 : -1, P.spread_outputs & 4 ? 3 : -1};
    for (int c : chans)
      if (c >= 0) {
        p[k] = G.chan[c];
        b[k] = (int64_t)G.chan_bytes;
        t[k++] = gtype;
      }
  }
  p[k] = P.d_qred;
  b[k] = 2 * sizeof(double);
  t[k++] = 0;
  if (*n < k || (k > 0 && (!ptrs || !bytes || !dtypes))) {
    *n = k;
    return *n == 0 ? LP_OK : LP_ERR_ARG;
  }
  for (int i = 0; i < k; ++i) {
    ptrs[i] = p[i];
    bytes[i] = b[i];
    dtypes[i] = t[i];
  }
  *n = k;
  return LP_OK;
}

lp_status lp_finish(lp_plan_t h, int64_t nt, const double* txy, const double* jet, double* V, double* S,
                    double* D) {
  if (!h || nt < 0 || nt > (int64_t)INT32_MAX) return LP_ERR_ARG;
  if (nt > 0 && !txy) return LP_ERR_ARG;
  Plan& P = h->P;
  const bool wv = V != nullptr, ws = S != nullptr, wd = D != nullptr;
  if (wv && nt > 0 && !jet) return LP_ERR_ARG;
  const int want = (wv ? 1 : 0) | (ws ? 2 : 0) | (wd ? 4 : 0);
  if (want & ~P.spread_outputs) return LP_ERR_STATE;
  if ((ws && !P.have_sigma) || (wd && !P.have_mu)) return LP_ERR_STATE;  // their local parts
  if (nt == 0 || !want) return LP_OK;
  const void* bufs[5] = {txy, wv ? jet : nullptr, V, S, D};
  for (const void* b : bufs)
    if (b && !is_device_ptr(b)) return LP_ERR_ARG;
  cudaStream_t s = P.stream;
  if ((size_t)nt > P.near_cap) {
    cudaStreamSynchronize(s);
    drelease(P, P.d_near, P.near_cap * sizeof(int2));
    P.near_cap = 0;
    if (!dalloc(P, (void**)&P.d_near, nt * sizeof(int2))) return LP_ERR_NOMEM;
    P.near_cap = nt;
  }
  if (!P.d_near_count && !dalloc(P, (void**)&P.d_near_count, sizeof(int))) return LP_ERR_NOMEM;
  double* dout[3] = {V, S, D};
  P.use_qred = true;
  finish_part(P, nt, txy, wv ? jet : nullptr, dout, wv, ws, wd, P.d_near, P.d_near_count, nullptr, s);
  P.use_qred = false;
  record_stage(P, 9, s);
  return status_from_cuda();
}

lp_status lp_volume_jets(lp_plan_t h, int64_t nt, const double* txy, double* jet) {
  if (!h || nt < 0 || nt > (int64_t)INT32_MAX) return LP_ERR_ARG;
  if (nt > 0 && (!txy || !jet)) return LP_ERR_ARG;
  Plan& P = h->P;
  if (!P.have_volume) return LP_ERR_STATE;
  if (nt == 0) return LP_OK;
  cudaStream_t s = P.stream;
  // cells of side rho over the box with one cell of margin on every side
  const double rho = std::sqrt(3.0 * P.delta1);
  BinGeom bg;
  bg.x0 = P.box_lo[0] - rho;
  bg.y0 = P.box_lo[1] - rho;
  bg.inv_bt = 1.0 / rho;
  const double nx = std::ceil((P.box_hi[0] - P.box_lo[0]) / rho) + 3.0;
  const double ny = std::ceil((P.box_hi[1] - P.box_lo[1]) / rho) + 3.0;
  if (nx * ny > 6.4e7) return LP_ERR_UNSUPPORTED;  // cells far below the node spacing
  bg.nbx = (int)nx;
  bg.nby = (int)ny;
  const int64_t n = P.nv;
  const size_t ncell = (size_t)bg.nbx * bg.nby + 1;
  // scratch, freed before return: keys, counts, cursor, starts, offsets,
  // permutation; targets and jets when in host memory
  const bool host_t = !is_device_ptr(txy), host_j = !is_device_ptr(jet);
  const size_t bytes = round256(n * sizeof(int)) * 2 + round256(ncell * sizeof(int)) * 2 +
                       round256((ncell + 1) * sizeof(int)) + round256(n * sizeof(float2)) +
                       (host_t ? round256(nt * 2 * sizeof(double)) : 0) +
                       (host_j ? round256(nt * 6 * sizeof(double)) : 0);
  char* tmp = nullptr;
  if (cudaMalloc((void**)&tmp, bytes) != cudaSuccess) {
    cudaGetLastError();
    return LP_ERR_NOMEM;
  }
  size_t off = 0;
  auto take = [&](size_t b) {
    char* p = tmp + off;
    off += round256(b);
    return p;
  };
  int* keys = (int*)take(n * sizeof(int));
  int* perm = (int*)take(n * sizeof(int));
  int* counts = (int*)take(ncell * sizeof(int));
  int* cursor = (int*)take(ncell * sizeof(int));
  int* starts = (int*)take((ncell + 1) * sizeof(int));
  float2* rel = (float2*)take(n * sizeof(float2));
  const double* dt = txy;
  if (host_t) {
    double* d = (double*)take(nt * 2 * sizeof(double));
    cudaMemcpyAsync(d, txy, nt * 2 * sizeof(double), cudaMemcpyHostToDevice, s);
    dt = d;
  }
  double* dj = host_j ? (double*)take(nt * 6 * sizeof(double)) : jet;
  launch_bin_sort(P.d_vxy, n, bg, keys, counts, cursor, starts, rel, perm, P.d_status, s);
  JetArgs a;
  a.txy = dt;
  a.n = nt;
  a.jet = dj;
  a.rel = rel;
  a.perm = perm;
  a.start = starts;
  a.vxy = P.d_vxy;
  a.vf = P.d_vf;
  a.x0 = bg.x0;
  a.y0 = bg.y0;
  a.bt = 1.0 / bg.inv_bt;
  a.rho = rho;
  a.on_tol = P.on_tol;
  a.nbx = bg.nbx;
  a.nby = bg.nby;
  launch_jet_fit(a, s);
  P.launches += 4;
  if (host_j) cudaMemcpyAsync(jet, dj, nt * 6 * sizeof(double), cudaMemcpyDeviceToHost, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(tmp);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LP_ERR_CUDA;
  }
  return status_from_cuda();
}

lp_status lp_sync(lp_plan_t h) {
  if (!h) return LP_ERR_ARG;
  Plan& P = h->P;
  if (cudaStreamSynchronize(P.stream) != cudaSuccess) return LP_ERR_CUDA;
  cudaMemcpy(P.h_status, P.d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
  unsigned st = *P.h_status;
  cudaMemset(P.d_status, 0, sizeof(unsigned));
  if (cudaGetLastError() != cudaSuccess) return LP_ERR_CUDA;
  if (st & kStatusOutOfBox) return LP_ERR_OUT_OF_BOX;
  if (st & kStatusExteriorBandV) return LP_ERR_UNSUPPORTED;
  if (st & kStatusNewton) return LP_ERR_NEWTON;
  return LP_OK;
}

lp_status lp_sync_timeout(lp_plan_t h, double timeout_ms) {
  if (!h || std::isnan(timeout_ms)) return LP_ERR_ARG;
  if (timeout_ms < 0.0) return lp_sync(h);
  Plan& P = h->P;
  const auto t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaStreamQuery(P.stream);
  while (e == cudaErrorNotReady) {  // bounded by timeout_ms of host time
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (ms >= timeout_ms) return LP_ERR_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
    e = cudaStreamQuery(P.stream);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LP_ERR_CUDA;
  }
  return lp_sync(h);
}

lp_status lp_destroy(lp_plan_t h) {
  if (!h) return LP_ERR_ARG;
  destroy_plan(h->P);
  delete h;
  return LP_OK;
}

lp_status lp_plan_info(lp_plan_t h, double* out) {
  if (!h || !out) return LP_ERR_ARG;
  const Plan& P = h->P;
  double v[37] = {P.delta1, P.delta2, (double)P.ker.w, P.ker.beta, (double)P.lv[0].g, (double)P.lv[0].K,
                  P.lv[0].P, (double)P.lv[1].g, (double)P.lv[1].K, P.lv[1].P, P.lv[1].L, P.band,
                  P.margin, (double)P.device_bytes, (double)P.precision, (double)P.order,
                  (double)P.launches, P.es_fit_err, (double)P.es.nc, P.sigma_eff,
                  P.own_fft ? 1.0 : 0.0, P.binned ? 1.0 : 0.0, (double)P.bin_cells,
                  (double)P.dy_levels, P.dy_err, (double)P.dy_nq, (double)(2 - P.l0), P.sigma,
                  (double)P.tune_ms[0], (double)P.tune_ms[1], (double)P.tune_ms[2],
                  (double)P.grid_ms[0], (double)P.grid_ms[1], (double)P.grid_ms[2], (double)P.grid_ms[3],
                  (double)P.grid_ms[4], (double)P.grid_ms[5]};
  std::memcpy(out, v, sizeof(v));
  return LP_OK;
}

lp_status lp_stage_times(lp_plan_t h, float* out) {
  if (!h || !out) return LP_ERR_ARG;
  Plan& P = h->P;
  // events: 0 start, 1 staged, 2 zeroed, 10 volume spread, 3 spread, 4 fwd,
  // 5 mult, 6 inv, 7 interp, 11 local, 8 refinement sums, 9 copies
  auto el = [&](int a, int b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, P.ev[a], P.ev[b]) != cudaSuccess) {
      cudaGetLastError();
      return -1.0f;
    }
    return ms;
  };
  out[0] = el(2, 3);
  out[1] = el(3, 4);
  out[2] = el(4, 5);
  out[3] = el(5, 6);
  out[4] = el(6, 7);
  out[5] = el(7, 11);
  out[6] = el(0, 9);
  out[7] = el(0, 1) + el(8, 9);
  out[8] = el(1, 2);
  out[9] = el(2, 10);
  out[10] = el(11, 8);
  return LP_OK;
}

}  // extern "C"
