// Interior boundary value problems by boundary integral equations (Sec. 5),
// for -lap u = f in Omega:
//   Dirichlet (u = g):       u = V[f] + D[mu],  -mu/2 + D[mu] = g - V[f]
//                            at the boundary nodes (eq. dir_inteq);
//   Neumann (du/dnu = g):    u = V[f] + S[g] - D[u],  u/2 + D[u] = V[f] + S[g]
//                            at the boundary nodes; constants are in the null
//                            space (D[1] = -1/2 on the boundary), so the
//                            operator carries the rank-one term
//                            (sum_i w_i u_i / |Gamma|) 1, which selects the
//                            solution of zero boundary mean.
// Restarted GMRES (Saad and Schultz, SISSC 1986) with classical Gram-Schmidt
// applied twice.  Each operator application binds the iterate as the
// double-layer density and evaluates D at the plan's own boundary nodes
// (on-surface targets: the smooth part plus the on-surface local expansions,
// refined when the plan refines) -- the paper's FMM is replaced by this
// evaluator.  The Krylov basis, its inner products and updates live on the
// device; only the (m+1) x m Hessenberg recurrences run on the host.
#include <cmath>
#include <vector>

#include "lp_internal.cuh"

using namespace lpg;

struct lp_plan_s {
  Plan P;
};

namespace {

constexpr int kDotThreads = 256;
constexpr int kMaxRestart = 64;

// out[i] = <V_i, w> for i < nv; one block per vector, fixed reduction order
__global__ void __launch_bounds__(kDotThreads) dots_kernel(const double* __restrict__ V, int64_t ld, int nv,
                                                           const double* __restrict__ w, int64_t n,
                                                           double* __restrict__ out) {
  __shared__ double red[kDotThreads];
  const int i = blockIdx.x;
  if (i >= nv) return;
  const double* v = V + (int64_t)i * ld;
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += kDotThreads) s = fma(v[k], w[k], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kDotThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[i] = red[0];
}

// w -= sum_{i < nv} h_i V_i
__global__ void subtract_kernel(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ h,
                                double* __restrict__ w, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s = w[k];
  for (int i = 0; i < nv; ++i) s = fma(-h[i], V[(int64_t)i * ld + k], s);
  w[k] = s;
}

// y = a x + b y (x may be y: no restrict qualifiers)
__global__ void axpby_kernel(double a, const double* x, double b, double* y, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) y[k] = fma(a, x[k], b * y[k]);
}

// y += scale * (*a) (a device scalar)
__global__ void add_scaled_kernel(const double* __restrict__ a, double scale, double* __restrict__ y, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) y[k] = fma(scale, *a, y[k]);
}

__global__ void fill_kernel(double* __restrict__ y, double v, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) y[k] = v;
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

struct Solver {
  lp_plan_t h;
  Plan& P;
  int64_t n;
  int m;
  double* V = nullptr;    // (m + 1) Krylov vectors of length n
  double* x = nullptr;    // iterate
  double* b = nullptr;    // right-hand side
  double* t = nullptr;    // scratch
  double* dh = nullptr;   // [2 (m + 1) + 1]: two Gram-Schmidt passes and a norm
  long long launches = 0;

  Solver(lp_plan_t h_, int64_t n_, int m_) : h(h_), P(h_->P), n(n_), m(m_) {}
  ~Solver() {
    for (void* p : {(void*)V, (void*)x, (void*)b, (void*)t, (void*)dh})
      if (p) cudaFree(p);
  }
  bool alloc() {
    return cudaMalloc(&V, (size_t)(m + 1) * n * sizeof(double)) == cudaSuccess &&
           cudaMalloc(&x, n * sizeof(double)) == cudaSuccess && cudaMalloc(&b, n * sizeof(double)) == cudaSuccess &&
           cudaMalloc(&t, n * sizeof(double)) == cudaSuccess &&
           cudaMalloc(&dh, (2 * (m + 1) + 1) * sizeof(double)) == cudaSuccess;
  }
  double* vec(int i) { return V + (int64_t)i * n; }

  // <a, a> through the device reduction, returned to the host
  double norm(const double* a) {
    dots_kernel<<<1, kDotThreads, 0, P.stream>>>(a, n, 1, a, n, dh);
    ++launches;
    double v = 0.0;
    cudaMemcpyAsync(&v, dh, sizeof(double), cudaMemcpyDeviceToHost, P.stream);
    cudaStreamSynchronize(P.stream);
    return std::sqrt(v);
  }
};

// Restarted GMRES for A x = b with A applied by `apply(in, out)` (device
// vectors); x starts at 0.  Returns the status; *iterations and *rel receive
// the iterations taken and the true relative residual of x (one more
// application).
template <class Op>
lp_status gmres(Solver& S, const Op& apply, double tol, int max_iter, int* iterations, double* residual) {
  Plan& P = S.P;
  const int m = S.m;
  const int64_t n = S.n;
  cudaStream_t s = P.stream;
  cudaMemsetAsync(S.x, 0, n * sizeof(double), s);
  const double bnorm = S.norm(S.b);
  if (!(bnorm > 0.0)) {  // b = 0: x = 0
    if (iterations) *iterations = 0;
    if (residual) *residual = 0.0;
    return LP_OK;
  }
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gam(m + 1), y(m), hv(2 * (m + 1) + 1);
  int it = 0;
  double rel = 1.0;
  lp_status st = LP_OK;
  bool first = true;
  while (it < max_iter && st == LP_OK) {
    // r = b - A x into V_0
    double beta;
    if (first) {
      cudaMemcpyAsync(S.vec(0), S.b, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
      beta = bnorm;
      first = false;
    } else {
      if ((st = apply(S.x, S.t)) != LP_OK) break;
      cudaMemcpyAsync(S.vec(0), S.b, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
      axpby_kernel<<<blocks_for(n), 256, 0, s>>>(-1.0, S.t, 1.0, S.vec(0), n);
      ++S.launches;
      beta = S.norm(S.vec(0));
    }
    rel = beta / bnorm;
    if (rel <= tol) break;
    axpby_kernel<<<blocks_for(n), 256, 0, s>>>(1.0 / beta, S.vec(0), 0.0, S.vec(0), n);
    ++S.launches;
    std::fill(gam.begin(), gam.end(), 0.0);
    gam[0] = beta;
    int k = 0;
    for (; k < m && it < max_iter; ++k, ++it) {
      double* w = S.vec(k + 1);
      if ((st = apply(S.vec(k), w)) != LP_OK) break;
      // two classical Gram-Schmidt passes against V_0..V_k, then |w|
      double* h1 = S.dh;
      double* h2 = S.dh + (m + 1);
      double* nr = S.dh + 2 * (m + 1);
      dots_kernel<<<k + 1, kDotThreads, 0, s>>>(S.V, n, k + 1, w, n, h1);
      subtract_kernel<<<blocks_for(n), 256, 0, s>>>(S.V, n, k + 1, h1, w, n);
      dots_kernel<<<k + 1, kDotThreads, 0, s>>>(S.V, n, k + 1, w, n, h2);
      subtract_kernel<<<blocks_for(n), 256, 0, s>>>(S.V, n, k + 1, h2, w, n);
      dots_kernel<<<1, kDotThreads, 0, s>>>(w, n, 1, w, n, nr);
      S.launches += 5;
      cudaMemcpyAsync(hv.data(), S.dh, hv.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) {
        st = LP_ERR_CUDA;
        break;
      }
      for (int i = 0; i <= k; ++i) H[(size_t)i * m + k] = hv[i] + hv[m + 1 + i];
      const double hk1 = std::sqrt(std::max(hv[2 * (m + 1)], 0.0));
      H[(size_t)(k + 1) * m + k] = hk1;
      if (hk1 > 0.0) {
        axpby_kernel<<<blocks_for(n), 256, 0, s>>>(1.0 / hk1, w, 0.0, w, n);
        ++S.launches;
      }
      // Givens rotations: earlier ones on the new column, then a new one
      for (int i = 0; i < k; ++i) {
        const double a = H[(size_t)i * m + k], c = H[(size_t)(i + 1) * m + k];
        H[(size_t)i * m + k] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + k] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[(size_t)k * m + k], c = H[(size_t)(k + 1) * m + k];
      const double r = std::hypot(a, c);
      cs[k] = r > 0.0 ? a / r : 1.0;
      sn[k] = r > 0.0 ? c / r : 0.0;
      H[(size_t)k * m + k] = r;
      H[(size_t)(k + 1) * m + k] = 0.0;
      gam[k + 1] = -sn[k] * gam[k];
      gam[k] = cs[k] * gam[k];
      rel = std::fabs(gam[k + 1]) / bnorm;
      if (rel <= tol || hk1 == 0.0) {
        ++k;
        ++it;
        break;
      }
    }
    if (st != LP_OK) break;
    // x += V_0..V_{k-1} y with H y = gamma (upper triangular)
    for (int i = k - 1; i >= 0; --i) {
      double acc = gam[i];
      for (int j = i + 1; j < k; ++j) acc -= H[(size_t)i * m + j] * y[j];
      y[i] = acc / H[(size_t)i * m + i];
    }
    for (int i = 0; i < k; ++i) hv[i] = -y[i];
    cudaMemcpyAsync(S.dh, hv.data(), k * sizeof(double), cudaMemcpyHostToDevice, s);
    subtract_kernel<<<blocks_for(n), 256, 0, s>>>(S.V, n, k, S.dh, S.x, n);
    ++S.launches;
    cudaStreamSynchronize(s);
    if (rel <= tol) break;
  }
  // the true residual of the returned iterate
  if (st == LP_OK) st = apply(S.x, S.t);
  if (st == LP_OK) {
    axpby_kernel<<<blocks_for(n), 256, 0, s>>>(1.0, S.b, -1.0, S.t, n);
    ++S.launches;
    rel = S.norm(S.t) / bnorm;
  }
  if (iterations) *iterations = it;
  if (residual) *residual = rel;
  return st;
}

// out = c * in + D[in] at the boundary nodes (c = -1/2: Dirichlet; +1/2:
// Neumann), plus, for Neumann, (sum_i w_i in_i / |Gamma|) 1
struct LayerOp {
  Solver* S;
  double c;
  bool mean_term;
  double inv_len;
  lp_status operator()(const double* in, double* out) const {
    Plan& P = S->P;
    lp_status st = lp_double_layer(S->h, in);
    if (st != LP_OK) return st;
    st = lp_execute(S->h, S->n, P.d_bxy, nullptr, nullptr, nullptr, out);
    if (st != LP_OK) return st;
    axpby_kernel<<<blocks_for(S->n), 256, 0, P.stream>>>(c, in, 1.0, out, S->n);
    ++S->launches;
    if (mean_term) {
      dots_kernel<<<1, kDotThreads, 0, P.stream>>>(P.d_bw, S->n, 1, in, S->n, S->dh);
      add_scaled_kernel<<<blocks_for(S->n), 256, 0, P.stream>>>(S->dh, inv_len, out, S->n);
      S->launches += 2;
    }
    return LP_OK;
  }
};

}  // namespace

extern "C" lp_status lp_solve_dirichlet(lp_plan_t h, const double* g, const double* f_jet_b, double* mu, double tol,
                                        int max_iter, int restart, int* iterations, double* residual) {
  if (!h || !g || !mu || !(tol > 0.0) || max_iter < 1 || restart < 0 || restart > kMaxRestart) return LP_ERR_ARG;
  Plan& P = h->P;
  if (P.n_panels == 0 || P.nb == 0) return LP_ERR_STATE;
  if (f_jet_b && !P.have_volume) return LP_ERR_STATE;
  const int64_t n = P.nb;
  Solver S(h, n, restart == 0 ? 30 : restart);
  if (!S.alloc()) {
    cudaGetLastError();
    return LP_ERR_NOMEM;
  }
  cudaStream_t s = P.stream;
  // right-hand side b = g - V[f] at the boundary nodes
  cudaMemcpyAsync(S.b, g, n * sizeof(double), cudaMemcpyDefault, s);
  if (f_jet_b) {
    lp_status st = lp_execute(h, n, P.d_bxy, f_jet_b, S.t, nullptr, nullptr);
    if (st != LP_OK) return st;
    axpby_kernel<<<blocks_for(n), 256, 0, s>>>(-1.0, S.t, 1.0, S.b, n);
    ++S.launches;
  }
  lp_status st = gmres(S, LayerOp{&S, -0.5, false, 0.0}, tol, max_iter, iterations, residual);
  if (st == LP_OK) {
    cudaMemcpyAsync(mu, S.x, n * sizeof(double), cudaMemcpyDefault, s);
    st = lp_double_layer(h, S.x);  // leave the solution bound as the double-layer density
  }
  P.launches += S.launches;
  const lp_status st_sync = lp_sync(h);
  return st == LP_OK ? st_sync : st;
}

extern "C" lp_status lp_solve_neumann(lp_plan_t h, const double* g, const double* f_jet_b, double* u, double tol,
                                      int max_iter, int restart, int* iterations, double* residual) {
  if (!h || !g || !u || !(tol > 0.0) || max_iter < 1 || restart < 0 || restart > kMaxRestart) return LP_ERR_ARG;
  Plan& P = h->P;
  if (P.n_panels == 0 || P.nb == 0) return LP_ERR_STATE;
  if (f_jet_b && !P.have_volume) return LP_ERR_STATE;
  const int64_t n = P.nb;
  Solver S(h, n, restart == 0 ? 30 : restart);
  if (!S.alloc()) {
    cudaGetLastError();
    return LP_ERR_NOMEM;
  }
  cudaStream_t s = P.stream;
  // |Gamma| = sum of the boundary weights
  fill_kernel<<<blocks_for(n), 256, 0, s>>>(S.t, 1.0, n);
  dots_kernel<<<1, kDotThreads, 0, s>>>(P.d_bw, n, 1, S.t, n, S.dh);
  double len = 0.0;
  cudaMemcpyAsync(&len, S.dh, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  S.launches += 2;
  if (!(len > 0.0)) return LP_ERR_STATE;
  // right-hand side b = V[f] + S[g] at the boundary nodes
  lp_status st = lp_single_layer(h, g);
  if (st != LP_OK) return st;
  st = lp_execute(h, n, P.d_bxy, f_jet_b, f_jet_b ? S.t : nullptr, S.b, nullptr);
  if (st != LP_OK) return st;
  if (f_jet_b) {
    axpby_kernel<<<blocks_for(n), 256, 0, s>>>(1.0, S.t, 1.0, S.b, n);
    ++S.launches;
  }
  st = gmres(S, LayerOp{&S, 0.5, true, 1.0 / len}, tol, max_iter, iterations, residual);
  if (st == LP_OK) {
    cudaMemcpyAsync(u, S.x, n * sizeof(double), cudaMemcpyDefault, s);
    st = lp_double_layer(h, S.x);  // u bound as the double-layer density (and g as the single layer)
  }
  P.launches += S.launches;
  const lp_status st_sync = lp_sync(h);
  return st == LP_OK ? st_sync : st;
}
