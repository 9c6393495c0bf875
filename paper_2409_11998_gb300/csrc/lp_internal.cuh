// Internal declarations of the GB300 evaluator (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/lp.h"

namespace lpg {

constexpr int kMaxW = 16;           // widest spreading kernel (grid points)
constexpr int kMaxNC = 20;          // coefficients per piece of the kernel polynomial
constexpr int kBatchThreads = 128;  // threads per block (and items per work entry) of batched launches
constexpr int kZeroChunk = 4096;    // 16-byte words cleared per work entry of the batched zeroing
constexpr int kTile = 32;           // bin side (near-history cells) of the binned spread
// bin sides the autotuner times, [FP64 plan][candidate], smallest first
constexpr int kBinCandidates[2][3] = {{16, 32, 48}, {16, 24, 32}};
constexpr int kSubThreads = 256;    // threads per CTA of the binned spread
constexpr int kSubDDThreads = 128;  // threads per CTA of the binned df64 spread (FP64 plans)
constexpr int kSubDDChunk = 64;     // nodes per weight chunk of that spread (one task per thread)
constexpr int kSubDDMinBlocks = 6;  // resident CTAs per SM it is compiled for (80 registers)
// Coefficient count of the binned spread's weight polynomials for width w
// (the plan's fit is zero-padded; plans whose fit needs more use the
// point-parallel spread).
constexpr int sub_ncw(int w) { return w + 3; }
constexpr int kMaxPanelOrder = 32;  // Gauss-Legendre nodes per boundary panel
constexpr int kNumEvents = 12;
constexpr int kFftThreads = 256;    // threads per CTA of the df64 FFT kernels
constexpr int kMaxDyLevels = 6;     // dyadic refinement levels of the local layer potentials
constexpr int kDyPieces = 144;      // unit pieces of the difference-kernel tables, x in [0, 144)
constexpr int kDyMaxDeg = 15;       // highest polynomial degree of a table piece
constexpr int kDyTabVec = 5;        // float4 per table piece: c0..c3 as df64 pairs, c4..c15 as floats
constexpr int kDyThreads = 256;     // threads per block of the refinement sums
constexpr int kMaxFftStages = 24;   // radix stages of one df64 transform
constexpr int kCornerQuad = 96;     // nodes of the corner time integral (6 graded pieces x 16)

// Device status bits (OR-ed by kernels, read by lp_sync).
enum : unsigned {
  kStatusOutOfBox = 1u,
  kStatusExteriorBandV = 2u,
  kStatusNewton = 4u,  // closest-point Newton did not converge (Sec. 2.2)
};

// Exponential-of-semicircle spreading kernel phi(z) = exp(beta (sqrt(1-z^2) - 1))
// on |z| < 1, z = (u - l) / (w/2) for grid coordinate u and grid index l.
struct Kernel {
  int w;
  double beta;
  double half_w;  // w/2
};

// Piecewise-polynomial form of the same kernel: for a point at grid
// coordinate u with stencil origin i0 = floor(u - w/2) + 1 and
// v = u - i0 - (w - 1)/2 in [-1/2, 1/2), the w stencil weights are
// phi_t = sum_k c[k][t] v^k (t = 0..w-1), fitted at plan time to within a
// hundredth of the plan tolerance.
template <typename T>
struct EsPoly {
  int w, nc;
  T c[kMaxNC][kMaxW];
};

// Radix plan of one df64 transform of length n (n = 2^a 3^b).
struct FftShape {
  int n, nst;
  int radix[kMaxFftStages];
};

// One periodic grid of the history part (Sec. 3): near history (kind 0,
// multiplier (e^{-k^2 d1} - e^{-k^2 d2})/k^2) or far history (kind 1,
// multiplier e^{-k^2 d2} W(k) with truncation radius L).
struct GridLevel {
  int kind = 0;
  int g = 0;          // grid points per dimension (7-smooth, even)
  int K = 0;          // kept modes |m| <= K per dimension
  int pitch = 0;      // row pitch of the in-place real layout, 2 (g/2 + 1)
  double P = 0, dk = 0, h = 0, L = 0, R = 0;
  double x0 = 0, y0 = 0;  // coordinates of grid index 0
  double zero_mode = 0;   // (dk/2pi)^2 M(0): the k = 0 multiplier without deconvolution
  void* chan[4] = {nullptr, nullptr, nullptr, nullptr};  // V, S, D1, D2 in-place buffers
  double* mtab = nullptr;  // (K+1)^2 deconvolved multiplier table, FP64
  float* mtab32 = nullptr; // same in FP32 with the zero mode removed (FP32 path)
  // pruned transforms: real rows [row_lo, row_hi) along x, then complex
  // columns 0..K along y (forward), and the reverse for the inverse
  int row_lo = 0, row_hi = 0;
  cufftHandle row_fwd = 0, row_inv = 0, col = 0;
  size_t chan_bytes = 0;
  // FFT chain: twiddles e^{-2 pi i k/g} as df64, the multiplier table as
  // (hi, lo) pairs (FP64 plans), and per channel the kept half-spectrum
  // columns [g][kp] (kp = K + 1 rounded up to even), df64 or FP32 complex
  FftShape full{}, half{};
  float4* tw_dd = nullptr;
  int* freq = nullptr;  // digit-reversed order of the in-place column transform, [g]
  float2* mtab_dd = nullptr;
  void* spec[4] = {nullptr, nullptr, nullptr, nullptr};
  int kp = 0;
};

// Grid geometry passed to kernels by value.
struct GridDev {
  int g, pitch;
  double x0, y0, inv_h;
};

// Argument records of the grid kernels.  A single-plan launch passes one by
// value; a batched launch passes an array of them in device memory plus a
// per-block work list.
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

template <typename T>
struct InterpArgs {
  const double* txy;
  int64_t n;
  const void* grid[2][3];  // [level][V,S,D]
  GridDev gd[2];
  const double* qsum;      // FP64 strength sums of V and S (FP32 path), or null
  double zero_factor;      // sum over levels of (dk/2pi)^2 M(0)
  int l0;                  // first level in use (1 for single-level plans)
  double* out[3];
  unsigned* status;
  EsPoly<T> es;
};

struct MultArgs {
  int g, K;
  double dk;
  const void* tab;        // double (FP64) or float (FP32) table
  const double* tab64;    // FP32 plans: the FP64 table, taken for 0 < max(|m_x|, |m_y|) < klo
  int klo;
  void* V;
  void* S;
  void* D1;
  const void* D2;
};

// A buffer to clear in a batched launch: ptr (16-byte aligned), n16 16-byte words.
struct ZeroSeg {
  void* ptr;
  int64_t n16;
};

// Bins of the sorted-source spread: squares of side kTile near-history cells
// from the near-history grid origin (physical, so both levels use them).
struct BinGeom {
  double x0, y0, inv_bt;  // origin and 1 / (kTile h_NH)
  int nbx, nby;
};

// One level of the binned spread of the volume nodes: one CTA per bin.
struct SubArgs {
  GridDev gd;
  const float2* rel;  // positions relative to their bin's corner, in bin order
  const float* q;     // strengths in the same order
  const int* start;   // [nbins + 2] bin starts (last bin: overflow)
  void* grid;
  double org_x, org_y, bt;  // bin grid origin and bin side
  int nbx, nby, M;          // bins per dimension; patch side (row pitch)
  unsigned* status;
  EsPoly<float> es;
};

// One level of the binned df64 spread of the volume nodes (FP64 plans).
struct SubDDArgs {
  GridDev gd;
  const float4* rel;  // offsets from the bin corner, df64 (x.hi, x.lo, y.hi, y.lo), in bin order
  const float2* q;    // strengths, df64, same order
  const int* start;   // [nbins + 2] bin starts
  void* grid;         // FP64 grid
  double org_x, org_y, bt;
  float2 inv_h;       // 1 / h, df64
  int nbx, nby, M, nc, nf;  // nf: leading Horner steps in float
  unsigned* status;
  float2 coef[kMaxNC][kMaxW];  // weight polynomials, df64
};

// FP32 plans: modes with |m_x|, |m_y| below this take the FP64 multiplier
// entry, the product formed in double (the low modes carry most of the
// log kernel's weight, and its multiplier is where the terms cancel)
constexpr int kLowKFP64 = 16;

// df64 FFT chain (k_fft.cu)
struct FftRowArgs {
  FftShape half;
  const float4* tw;
  void* grid[4];      // grids: forward input (FP64 or FP32), inverse output (df64 pairs or FP32)
  void* spec[4];      // kept half spectra (df64 or FP32 complex)
  int pitch, kp, K, row_lo, row_hi;
};

struct FftColJob {
  int kind;           // 0: M F (V, S); 1: M (-i)(k1 F1 + k2 F2) (D)
  const void* in[2];
  void* out;
};

struct FftColArgs {
  FftShape full;
  const float4* tw;
  const int* freq;    // frequency index of each position of the in-place forward transform's output
  const void* tab;    // deconvolved multiplier, (K+1)^2: df64 pairs (FP64) or floats without k = 0 (FP32)
  const double* tab64;  // FP32 plans: the FP64 table, taken for 0 < max(|m_x|, |m_y|) < klo
  int klo;
  float2 dk;          // mode spacing (df64 pair; FP32 uses .x)
  FftColJob job[3];
  int kp, K, row_lo, row_hi;
};

// df64 interpolation (k_interp_dd.cu)
struct InterpDDLevel {
  const void* grid[3];  // V, S, D grids as df64 (hi, lo) pairs
  int g, pitch;
  float2 x0, y0, inv_h;
};

struct InterpDDArgs {
  const double* txy;
  int64_t n;
  InterpDDLevel lv[2];
  int l0;                  // first level in use (1 for single-level plans)
  double* out[3];
  unsigned* status;
  int nc, nf;               // coefficients; leading Horner steps in float
  float2 coef[kMaxNC][kMaxW];  // weight polynomials, df64
};

// f-jet estimation from node values (k_jets.cu): nodes sorted into square
// cells of side bt >= rho from (x0, y0), offsets from their cell corner.
struct JetArgs {
  const double* txy;
  int64_t n;
  double* jet;         // [n][6] out
  const float2* rel;   // node offsets from their cell's corner, in cell order
  const int* perm;     // node index of each sorted entry
  const int* start;    // [ncells + 2] cell starts
  const double* vxy;   // node coordinates (input order)
  const double* vf;    // f at the nodes (input order)
  double x0, y0, bt, rho, on_tol;
  int nbx, nby;
};
void launch_jet_fit(const JetArgs& a, cudaStream_t s);

// Argument record of the local pass (one per plan).
struct LocalArgs {
  const double* txy;
  const double* jet;
  int64_t n;
  double* out[3];  // V, S, D: local part added in place
  const double* bxy;
  int64_t nb;
  int n_panels, p;
  const double* tau;
  const double* geo_coef;
  const double* geo_ref;
  const double* sig_coef;
  const double* sig_ref;
  const double* mu_coef;
  const double* mu_ref;
  double hx0, hy0, hh;
  float hh32, inv_hh32, band32, margin32;  // single-precision copies for the classification
  int hnx, hny;
  const unsigned char* cell_near;  // per hash cell: a boundary node within its 3x3 cells
  const int* cell_start;
  const int* cell_node;
  const float2* cell_xy32;   // node coordinates relative to their cell origin
  const float* geo_coef32;   // FP32 copy of geo_coef
  const float* sig_coef32;   // FP32 copies of sig_coef / mu_coef (FP32 plans)
  const float* mu_coef32;
  const float2* geo_coef_dd;  // df64 copies of geo_coef, sig_coef, mu_coef
  const float2* sig_coef_dd;
  const float2* mu_coef_dd;
  double margin, band, delta, on_tol;
  double delta_sd;  // delta of the S and D expansions (delta / 4^J with dyadic refinement)
  int order;
  unsigned* status;
  // convex right-angle corners [n_corners][6]: corner point, inward normals
  // of the edge before and after it; time integral nodes t_k and weights
  const double* corners;
  int n_corners;
  const double* corner_q;  // [2][kCornerQuad]: t, weight (dt included)
};

// Dyadic refinement sums over the band targets (k_dyadic.cu).
struct DyadicArgs {
  const double* txy;
  double* out_s;
  double* out_d;
  const float2* sig_w;   // sigma * weight at the subnodes (df64), or null
  const float2* mu;      // mu at the subnodes (df64), or null
  const float4* rel;     // subnode offset from its panel's reference node (df64 x, y)
  const float4* nw;      // outward normal times weight (df64 x, y)
  const float4* tab;     // piecewise polynomials of F, then H (kDyTabVec float4 per piece)
  int levels, p;
  int64_t q_off[kMaxDyLevels];  // first subnode of each level
  const float4* ref_dd;    // panel reference node (df64 x, y)
  const float* panel_rad;  // panel radius about its reference node
  // panels hashed by their reference node into cells of side >= range1 +
  // the largest panel radius: every panel within range1 of a target lies in
  // the 3x3 cells around it, each panel in exactly one cell
  float hx0, hy0;         // grid origin (single precision suffices for cells)
  float inv_hh;           // 1 / cell side
  int hnx, hny;
  const int* cell_start;
  const int* cell_panel;
  float range1f;          // 12 sqrt(delta): the level-1 range
  float2 inv_delta, inv_4pi, dcoef;  // 1/delta, 1/(4 pi), 1/(2 pi delta), df64
  unsigned* status;
};

struct Plan {
  int precision = LP_FP64;
  int order = 5;
  double delta1 = 0, delta2 = 0, tol = 0;
  // history levels: two (near history at delta_1..delta_2, far history from
  // delta_2), or one (l0 = 1: the far-history level alone with delta_2 =
  // delta_1, so the near-history multiplier would vanish identically)
  int l0 = 0;
  double box_lo[2] = {0, 0}, box_hi[2] = {0, 0};
  double side = 0;        // max box extent
  double sigma = 2.0;     // target upsampling of the history grids (g >= sigma (2K+1))
  double sigma_eff = 2.0; // smallest realised g / (2K+1) over the two levels
  double on_tol = 0;      // on-surface classification radius
  Kernel ker{};
  EsPoly<double> es{};
  EsPoly<float> es32{};
  int es_float_steps = 0;  // leading Horner steps of the df64 weight chains taken in float
  float2 es_dd[kMaxNC][kMaxW] = {};  // es as df64 (hi, lo) pairs
  // dyadic refinement (k_dyadic.cu): levels J, difference-kernel tables,
  // subnodes of every level (offsets, normal x weight, densities)
  int dy_levels = 0, dy_deg_f = 0, dy_deg_h = 0;  // levels; fitted table degrees
  double dy_err = 0;
  int64_t dy_q_off[kMaxDyLevels] = {};
  int64_t dy_nq = 0;
  float4* d_dy_tab = nullptr;
  float4* d_dy_rel = nullptr;
  float4* d_dy_nw = nullptr;
  float2* d_dy_sig = nullptr;
  float2* d_dy_mu = nullptr;
  float* d_dy_rad = nullptr;
  float4* d_dy_ref = nullptr;
  double* d_dy_wgl = nullptr;
  double dy_hx0 = 0, dy_hy0 = 0, dy_hh = 0;
  int dy_hnx = 0, dy_hny = 0;
  int* d_dy_cell_start = nullptr;
  int* d_dy_cell_panel = nullptr;
  bool own_fft = false;              // transforms run in this library's FFT chain (df64 for FP64 plans,
                                     // with the df64 interpolation), not cuFFT
  double es_fit_err = 0;
  GridLevel lv[2];
  cudaStream_t stream = nullptr;

  // boundary
  int64_t n_panels = 0;
  int p = 0;              // nodes per panel
  int64_t nb = 0;         // n_panels * p
  double* d_bxy = nullptr;     // [nb][2]
  double* d_bw = nullptr;      // [nb]
  double* d_bnrm = nullptr;    // [nb][2]
  double* d_geo_coef = nullptr;  // [n_panels][2][p] Legendre coefficients of x - xref, y - yref
  double* d_geo_ref = nullptr;   // [n_panels][2] reference (middle node) coordinates
  double* d_leg_T = nullptr;     // [p][p] values -> Legendre coefficients
  double* d_tau = nullptr;       // [p] Gauss-Legendre abscissae
  double margin = 0, band = 0;
  // uniform hash of boundary nodes for the nearest-node search
  double hash_x0 = 0, hash_y0 = 0, hash_h = 0;
  int hash_nx = 0, hash_ny = 0;
  int* d_cell_start = nullptr;  // [nx*ny + 1]
  unsigned char* d_cell_near = nullptr;  // [nx*ny] 1 where the cell's 3x3 neighbourhood holds a node
  int* d_cell_node = nullptr;   // [nb] node ids sorted by cell
  float2* d_cell_xy32 = nullptr;  // [nb] node coordinates relative to their cell's origin (FP32)
  float* d_geo_coef32 = nullptr;  // FP32 copy of d_geo_coef (Newton start)
  float2* d_geo_coef_dd = nullptr;    // df64 copies of the panel coefficients (foot search,
  float2* d_sigma_coef_dd = nullptr;  // jets of the FP64 expansions)
  float2* d_mu_coef_dd = nullptr;
  float* d_sigma_coef32 = nullptr;  // FP32 copies of the density coefficients (FP32 local pass)
  float* d_mu_coef32 = nullptr;
  double* d_corners = nullptr;   // [n_corners][6] convex right-angle corners (V_L by the quadrant)
  int n_corners = 0;
  double* d_corner_q = nullptr;  // [2][kCornerQuad] quadrature of the corner time integral

  // sorted-bin spread (FP32 path)
  BinGeom bins{};
  int sub_M[2] = {0, 0};           // shared-memory patch side (row pitch), per level
  int* d_keys = nullptr;           // scratch [max(nv, nb)]
  int* d_counts = nullptr;         // scratch [nbins + 1]
  int* d_cursor = nullptr;         // scratch [nbins + 1]
  float2* d_vrel_s = nullptr;      // volume nodes sorted by bin (offsets from the bin corner)
  int* d_vperm = nullptr;
  float* d_vq_s = nullptr;
  int* d_vstart = nullptr;         // [nbins + 2]
  bool binned = false;             // volume spread through the bins
  int bin_cells = kTile;           // bin side in near-history cells (FP32 32, FP64 24)
  bool autotune = false;           // time the bin candidates at the first lp_volume
  bool tuned = false;
  float tune_ms[3] = {0, 0, 0};    // spread time of each candidate (both levels)
  bool tune_grids = false;         // time upsampling x level candidates at the first lp_volume
  float grid_ms[6] = {0, 0, 0, 0, 0, 0};  // their evaluation times (ms; -1: not built)
  float4* d_vrel_dd = nullptr;     // FP64 plans: offsets from the bin corner, df64
  float2* d_vq_dd = nullptr;       // FP64 plans: strengths in bin order, df64
  // FP64 plans: the boundary nodes sorted into the same bins (fixed-point
  // spread of the layers over the non-empty bins); re-sorted when the bins change
  bool bbinned = false;
  int* d_bkeys = nullptr;          // [nb + 1] sort scratch (the last entry: its status word)
  int* d_bstart = nullptr;         // [nbins + 2]
  float4* d_brel_dd = nullptr;     // [nb] offsets from the bin corner, df64
  int* d_bperm = nullptr;          // [nb]
  float2* d_bq_dd = nullptr;       // [3][nb] sigma w, mu nu_x w, mu nu_y w in bin order, df64
  int2* d_bbins = nullptr;         // [n_bbins] the bins holding boundary nodes
  int n_bbins = 0;
  size_t key_cap = 0;
  size_t vsort_cap = 0;

  // bound sources
  int64_t nv = 0;
  int64_t v_cap = 0;         // capacity of d_vxy / d_vq
  double* d_vxy = nullptr;   // [nv][2]
  double* d_vq = nullptr;    // [nv] f w
  double* d_vf = nullptr;    // [nv] f (node values, for lp_volume_jets)
  bool have_volume = false;
  double* d_sigma = nullptr;   // [nb]
  double* d_sigma_coef = nullptr;  // [n_panels][p] Legendre coefficients (centred)
  double* d_sigma_ref = nullptr;   // [n_panels]
  double* d_mu = nullptr;
  double* d_mu_coef = nullptr;
  double* d_mu_ref = nullptr;
  double* d_bq = nullptr;    // [3][nb]: sigma w, mu nu1 w, mu nu2 w
  bool have_sigma = false, have_mu = false;
  double* d_qsum = nullptr;  // [2] FP64 sums of the V and S strengths (zero mode)
  double* d_qred = nullptr;  // [2] the sums this plan's lp_spread contributed (summed across ranks)
  int spread_outputs = 0;    // outputs (1 V, 2 S, 4 D) of the last lp_spread; 0: none
  bool use_qred = false;     // lp_finish: the zero mode from d_qred

  // staging for host pointers
  void* d_stage = nullptr;
  size_t stage_bytes = 0;
  double* d_out = nullptr;   // [3][cap] outputs for host destinations
  size_t out_cap = 0;
  int2* d_near = nullptr;    // [near_cap] (target, nearest node) of band candidates
  int* d_near_count = nullptr;
  size_t near_cap = 0;

  unsigned* d_status = nullptr;
  unsigned* h_status = nullptr;  // pinned
  cudaEvent_t ev[kNumEvents] = {};
  // host targets are staged on a second stream while the spreads and
  // transforms run (created at the first execute with host inputs)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_staged = nullptr;
  // graph replay of lp_execute (lp_execute_graph): one cached executable
  // graph per argument signature, captured on graph_stream
  unsigned long long gen = 0;      // bumped by every allocation or bin change
  cudaStream_t graph_stream = nullptr;
  cudaEvent_t ev_g0 = nullptr, ev_g1 = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  const void* graph_key[5] = {};
  int64_t graph_nt = -1, graph_nv = -1;
  unsigned long long graph_gen = 0;
  long long graph_launches = 0;
  bool capturing = false;          // lp_execute is being captured into a graph
  size_t device_bytes = 0;
  size_t max_bytes = 0;            // device-memory budget (0: none)
  int device = 0;                  // CUDA device current at lp_plan
  mutable long long launches = 0;  // kernels launched by this plan (all calls)
};

// ---- host helpers (lp_setup.cu) ----
lp_status choose_levels(Plan& P);
lp_status build_tables(Plan& P);
lp_status fit_kernel_poly(Plan& P);
lp_status build_boundary(Plan& P, const double* h_xy, const double* h_w, const double* h_nrm);
void gauss_legendre(int p, double* x, double* w);
int fft_size(int n);

// ---- argument builders and batched launches ----
GridDev grid_dev(const GridLevel& G);
template <typename T>
SpreadArgs<T> make_spread_args(const Plan& P, int level, const double* xy, const double* const* q, int nq,
                               void* const* grids, int64_t n);
template <typename T>
InterpArgs<T> make_interp_args(const Plan& P, int64_t nt, const double* txy, double* V, double* S, double* D);
MultArgs make_mult_args(const Plan& P, int level, bool want_v, bool want_s, bool want_d);
LocalArgs make_local_args(const Plan& P, int64_t nt, const double* txy, const double* jet, double* V,
                          double* S, double* D);
void launch_zero_batch(const ZeroSeg* d_segs, const int2* d_work, int nwork, cudaStream_t s);
void launch_spread_batch(int precision, int w, const void* d_args, const int2* d_work, int nwork,
                         cudaStream_t s);
void launch_multiplier_batch(int precision, const MultArgs* d_args, const int2* d_work, int nwork,
                             cudaStream_t s);
void launch_interp_batch(int precision, int w, const void* d_args, const int2* d_work, int nwork,
                         cudaStream_t s);
void launch_local_batch(int precision, const LocalArgs* d_args, const int2* d_work, int nwork, int4* d_list,
                        int* d_count, int64_t n_total, bool corners, cudaStream_t s);

// ---- launches (kernels in k_*.cu) ----
void launch_spread(const Plan& P, int level, const double* xy, const double* const* q, int nq,
                   void* const* grids, int64_t n, cudaStream_t s);
void launch_multiplier(const Plan& P, int level, bool want_v, bool want_s, bool want_d,
                       cudaStream_t s);
void launch_interp(const Plan& P, int64_t nt, const double* txy, double* V, double* S, double* D,
                   cudaStream_t s);
void launch_local(const Plan& P, int64_t nt, const double* txy, const double* jet, double* V,
                  double* S, double* D, cudaStream_t s);
void launch_local_list(const Plan& P, int64_t nt, const double* txy, const double* jet, double* V,
                       double* S, double* D, int2* list, int* count, cudaStream_t s);
void launch_bin_sort(const double* xy, int64_t n, const BinGeom& bg, int* keys, int* counts, int* cursor,
                     int* starts, float2* rel_s, int* perm, unsigned* status, cudaStream_t s);
void launch_gather_q(const double* q, int64_t stride, int nq, const int* perm, int64_t n, float* q_s,
                     cudaStream_t s);
bool spread_sub_configure(int w);
bool spread_sub_dd_configure(int w);
size_t spread_sub_dd_smem(int M, int w);
void launch_spread_sub_dd(const SubDDArgs& a, int w, cudaStream_t s);
// up to three channels (strengths in bin order, FP64 grid) spread over a
// list of bins with the fixed-point kernel: one CTA per (bin, channel)
struct FxChan {
  const float2* q[3];
  void* grid[3];
};
void launch_spread_fx_list(const SubDDArgs& a, const int2* bins, int nbins, const FxChan& ch, int nch, int w,
                           cudaStream_t s);
// the same over a wave of plans: record r (SubDDArgs recs[r], its bin list
// and channels lrecs[r]) covers blocks first[r] .. first[r + 1] - 1, one per
// (listed bin, channel)
struct FxListRec {
  const int2* bins;
  FxChan ch;
  int nch;
};
void launch_spread_fx_list_wave(int w, const SubDDArgs* recs, const FxListRec* lrecs, const int* first, int nrec,
                                int nblocks, size_t smem, cudaStream_t s);
void launch_bin_sort_dd(const double* xy, int64_t n, const BinGeom& bg, int* keys, int* counts, int* cursor,
                        int* starts, float4* rel_s, int* perm, unsigned* status, cudaStream_t s);
void launch_gather_q_dd(const double* q, const int* perm, int64_t n, float2* q_s, cudaStream_t s);
size_t spread_sub_smem(const SubArgs& a, int w);
void launch_spread_sub(const SubArgs& a, int w, cudaStream_t s);
FftShape fft_shape(int n, bool high = false, bool r16 = true);  // high: radices 8, 9 (and 16 if r16) too
std::vector<float4> fft_twiddles(int g);
std::vector<int> fft_dif_order(const FftShape& sh);
bool fft_dd_configure();
size_t fft_rows_smem(int g, bool f64);
size_t fft_cols_smem(int g, bool f64);
void launch_fft_rows_fwd(const FftRowArgs& a, int nchan, bool f64, cudaStream_t s);
void launch_fft_rows_inv(const FftRowArgs& a, int nchan, bool f64, cudaStream_t s);
void launch_fft_cols(const FftColArgs& a, int njobs, bool f64, cudaStream_t s);
void launch_split_table(const double* src, float2* dst, int64_t n, cudaStream_t s);
void launch_interp_dd(const InterpDDArgs& a, int w, cudaStream_t s);
void launch_interp_dd_wave(const InterpDDArgs* recs, const int* first, int nrec, int nblocks, int w,
                           cudaStream_t s);
void launch_spread_wave(int precision, int w, const void* recs, const int* first, int nrec, int nblocks,
                        size_t smem, cudaStream_t s);
size_t spread_sub_smem(int M, int w, bool f64);
SubDDArgs make_spread_dd_args(const Plan& P, int l);
SubArgs make_spread_sub_args(const Plan& P, int l);
InterpDDArgs make_interp_dd_args(const Plan& P, int64_t nt, const double* txy, double* const* dout);
lp_status setup_dyadic(Plan& P, int levels);
void launch_dyadic_dens(const Plan& P, int kind, cudaStream_t s);
void launch_dyadic(const Plan& P, int64_t nt, const double* txy, double* S, double* D, const int2* list,
                   const int* count, cudaStream_t s);
// pipeline pieces shared by lp_execute and lp_batch_execute (lp_api.cu)
void spread_volume_binned(const Plan& P, int l, cudaStream_t s);
void history_transforms(const Plan& P, bool wv, bool ws, bool wd, cudaStream_t s, bool events);
void history_interp(const Plan& P, int64_t nt, const double* txy, double* const* dout, cudaStream_t s);
void fft_forward(const Plan& P, int level, int chan);
void fft_inverse(const Plan& P, int level, int chan);
void launch_panel_coef(const Plan& P, const double* vals, int stride, int ncomp, double* coef,
                       double* ref, cudaStream_t s);
void launch_strengths(const Plan& P, int kind, cudaStream_t s);
void launch_to_float(const double* src, float* dst, int64_t n, cudaStream_t s);
void launch_mult_table(int kind, int K, double dk, double d1, double d2, double L, double scale,
                       const double* d_ph, double* tab, float* tab32, cudaStream_t s);
void launch_volume_q(const Plan& P, const double* f, const double* w, double* q, int64_t n,
                     cudaStream_t s);
void launch_sum(const Plan& P, const double* x, int64_t n, double* out, cudaStream_t s);

}  // namespace lpg
