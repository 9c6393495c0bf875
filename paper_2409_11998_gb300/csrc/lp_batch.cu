// Batched evaluation of a wave of independent plans (problems of different
// sizes): one zeroing launch, one point-parallel spread launch (boundary
// nodes), one binned-spread launch over every bin of every plan, one
// interpolation launch and one local classify + one near launch for the whole
// wave, each over an array of per-plan argument records (with a per-block
// work list, or each record's first block); each plan's transform chain runs
// in between on one of several worker streams, so that small plans' chains
// overlap.  The arithmetic per item is the single-plan kernels' (same device
// functions).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "lp_internal.cuh"

using namespace lpg;

struct lp_plan_s {
  Plan P;
};

constexpr int kBatchWorkers = 8;  // streams the plans' transform chains are spread over

struct lp_batch_s {
  cudaStream_t stream = nullptr;
  cudaStream_t work[kBatchWorkers] = {};
  cudaEvent_t fork = nullptr, join[kBatchWorkers] = {};
  void* d_buf = nullptr;  // per-wave records and work lists
  void* h_buf = nullptr;  // pinned mirror
  size_t buf_cap = 0;
  int4* d_list = nullptr;  // near-boundary candidates of the wave
  size_t list_cap = 0;
  int* d_count = nullptr;
  cudaEvent_t ev[8] = {};
  bool pending = false;   // h_buf is in use by an enqueued copy until ev[7]
  long long launches = 0;
};

namespace {

bool dev_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Append records of type R to the packed host image; returns their offset.
struct Packer {
  std::vector<unsigned char> img;
  template <typename R>
  size_t put(const std::vector<R>& v) {
    size_t off = align_up(img.size(), 256);
    img.resize(off + v.size() * sizeof(R));
    if (!v.empty()) std::memcpy(img.data() + off, v.data(), v.size() * sizeof(R));
    return off;
  }
};

}  // namespace

extern "C" {

lp_status lp_batch_create(void* stream, lp_batch_t* out) {
  if (!out) return LP_ERR_ARG;
  *out = nullptr;
  lp_batch_s* b = new (std::nothrow) lp_batch_s();
  if (!b) return LP_ERR_NOMEM;
  b->stream = (cudaStream_t)stream;
  if (cudaMalloc(&b->d_count, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return LP_ERR_NOMEM;
  }
  for (auto& e : b->ev) cudaEventCreate(&e);
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < kBatchWorkers && ok; ++k)
    ok = cudaStreamCreateWithFlags(&b->work[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lp_batch_destroy(b);
    return LP_ERR_CUDA;
  }
  *out = b;
  return LP_OK;
}

lp_status lp_batch_destroy(lp_batch_t b) {
  if (!b) return LP_ERR_ARG;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  if (b->d_buf) cudaFree(b->d_buf);
  if (b->h_buf) cudaFreeHost(b->h_buf);
  if (b->d_list) cudaFree(b->d_list);
  if (b->d_count) cudaFree(b->d_count);
  for (auto& e : b->ev)
    if (e) cudaEventDestroy(e);
  for (int k = 0; k < kBatchWorkers; ++k) {
    if (b->work[k]) cudaStreamDestroy(b->work[k]);
    if (b->join[k]) cudaEventDestroy(b->join[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
  return LP_OK;
}

static long long sum_launches(const lp_plan_t* plans, int n) {
  long long t = 0;
  for (int i = 0; i < n; ++i) t += plans[i]->P.launches;
  return t;
}

lp_status lp_batch_execute(lp_batch_t b, int n, const lp_plan_t* plans, const int64_t* n_t,
                           const double* const* t_xy, const double* const* f_jet, double* const* V,
                           double* const* S, double* const* D) {
  if (!b || n <= 0 || !plans || !n_t || !t_xy || !plans[0]) return LP_ERR_ARG;
  const int prec = plans[0]->P.precision, w = plans[0]->P.ker.w;
  int64_t total_t = 0;
  for (int i = 0; i < n; ++i) {
    if (!plans[i]) return LP_ERR_ARG;
    const Plan& P = plans[i]->P;
    if (P.precision != prec || P.ker.w != w) return LP_ERR_ARG;  // one kernel shape per wave
    if (P.dy_levels > 0) return LP_ERR_UNSUPPORTED;              // refinement: lp_execute only
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return LP_ERR_ARG;  // a plan's grids serve one problem
    if (n_t[i] < 0 || n_t[i] > (int64_t)INT32_MAX) return LP_ERR_ARG;
    const bool wv = V && V[i], ws = S && S[i], wd = D && D[i];
    if ((wv && !P.have_volume) || (ws && !P.have_sigma) || (wd && !P.have_mu)) return LP_ERR_STATE;
    if (n_t[i] == 0) continue;
    if (!dev_ptr(t_xy[i])) return LP_ERR_ARG;
    if (wv && (!f_jet || !dev_ptr(f_jet[i]))) return LP_ERR_ARG;
    if ((wv && !dev_ptr(V[i])) || (ws && !dev_ptr(S[i])) || (wd && !dev_ptr(D[i]))) return LP_ERR_ARG;
    total_t += n_t[i];
  }
  cudaStream_t s = b->stream;
  if (b->pending) {
    cudaEventSynchronize(b->ev[7]);  // the previous wave's records were copied
    b->pending = false;
  }

  // ---- per-wave records ----
  std::vector<ZeroSeg> zsegs;
  std::vector<int2> zwork;
  std::vector<SpreadArgs<double>> sp64;
  std::vector<SpreadArgs<float>> sp32;
  std::vector<int2> swork;
  std::vector<MultArgs> mult;
  std::vector<int2> mwork;
  std::vector<InterpArgs<double>> in64;
  std::vector<InterpArgs<float>> in32;
  std::vector<int2> iwork;
  std::vector<LocalArgs> loc;
  std::vector<int2> lwork;
  // binned volume spreads and df64 interpolations: one record per plan and
  // level (per plan), each with its first block in the wave's launch
  std::vector<SubDDArgs> bdd;
  std::vector<SubArgs> b32;
  std::vector<int> bfirst(1, 0);
  size_t bsmem = 0;
  std::vector<InterpDDArgs> idd;
  std::vector<int> ifirst(1, 0);
  // FP64 plans whose boundary nodes sit in the bins: the layer spreads over
  // their listed bins, one record per plan and level
  std::vector<SubDDArgs> ldd;
  std::vector<FxListRec> lrec;
  std::vector<int> lfirst(1, 0);
  size_t lsmem = 0;
  const bool f64 = prec == LP_FP64;
  for (int i = 0; i < n; ++i) {
    const Plan& P = plans[i]->P;
    const bool wv = V && V[i], ws = S && S[i], wd = D && D[i];
    const int64_t nt = n_t[i];
    if (nt == 0 || (!wv && !ws && !wd)) continue;
    for (int l = P.l0; l < 2; ++l) {
      const GridLevel& G = P.lv[l];
      const bool need[4] = {wv, ws, wd, wd};
      for (int c = 0; c < 4; ++c) {
        if (!need[c]) continue;
        int rec = (int)zsegs.size();
        ZeroSeg zs{G.chan[c], (int64_t)(G.chan_bytes / 16)};
        zsegs.push_back(zs);
        for (int64_t e = 0; e < zs.n16; e += kZeroChunk) zwork.push_back(make_int2(rec, (int)(e / kZeroChunk)));
      }
      // spread records: volume sources, then boundary channels
      auto add_spread = [&](const double* xy, const double* const* q, int nq, void* const* grids, int64_t cnt) {
        if (cnt <= 0 || nq == 0) return;
        int rec = f64 ? (int)sp64.size() : (int)sp32.size();
        if (f64) sp64.push_back(make_spread_args<double>(P, l, xy, q, nq, grids, cnt));
        else sp32.push_back(make_spread_args<float>(P, l, xy, q, nq, grids, cnt));
        for (int64_t j = 0; j < cnt; j += kBatchThreads) swork.push_back(make_int2(rec, (int)j));
      };
      if (wv && !P.binned) {  // binned plans: one launch over every bin of the wave below
        const double* q[1] = {P.d_vq};
        void* g[1] = {G.chan[0]};
        add_spread(P.d_vxy, q, 1, g, P.nv);
      }
      if (wv && P.binned && P.nv > 0) {
        if (f64) bdd.push_back(make_spread_dd_args(P, l));
        else b32.push_back(make_spread_sub_args(P, l));
        bfirst.push_back(bfirst.back() + P.bins.nbx * P.bins.nby);
        bsmem = std::max(bsmem, spread_sub_smem(P.sub_M[l], P.ker.w, f64));
      }
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
      if (nq && f64 && P.bbinned) {
        SubDDArgs a = make_spread_dd_args(P, l);
        a.rel = P.d_brel_dd;
        a.start = P.d_bstart;
        FxListRec r{};
        r.bins = P.d_bbins;
        int k = 0;
        if (ws) {
          r.ch.q[k] = P.d_bq_dd;
          r.ch.grid[k++] = G.chan[1];
        }
        if (wd) {
          r.ch.q[k] = P.d_bq_dd + P.nb;
          r.ch.grid[k++] = G.chan[2];
          r.ch.q[k] = P.d_bq_dd + 2 * P.nb;
          r.ch.grid[k++] = G.chan[3];
        }
        r.nch = k;
        ldd.push_back(a);
        lrec.push_back(r);
        lfirst.push_back(lfirst.back() + P.n_bbins * k);
        lsmem = std::max(lsmem, spread_sub_smem(P.sub_M[l], P.ker.w, true));
      } else {
        add_spread(P.d_bxy, bq, nq, bg, P.nb);
      }
      if (!P.own_fft) {  // plans on the FFT chain apply the multiplier inside it
        int rec = (int)mult.size();
        mult.push_back(make_mult_args(P, l, wv, ws, wd));
        int64_t modes = (int64_t)G.g * (G.g / 2 + 1);
        for (int64_t j = 0; j * kBatchThreads < modes; ++j) mwork.push_back(make_int2(rec, (int)j));
      }
    }
    double* vo = wv ? V[i] : nullptr;
    double* so = ws ? S[i] : nullptr;
    double* dout = wd ? D[i] : nullptr;
    // FP64 plans on the FFT chain interpolate from df64 grids: one launch
    // over all of them below
    if (f64 && P.own_fft) {
      double* outs[3] = {vo, so, dout};
      idd.push_back(make_interp_dd_args(P, nt, t_xy[i], outs));
      ifirst.push_back(ifirst.back() + (int)((nt + 127) / 128));
    } else {
      int rec = f64 ? (int)in64.size() : (int)in32.size();
      if (f64) in64.push_back(make_interp_args<double>(P, nt, t_xy[i], vo, so, dout));
      else in32.push_back(make_interp_args<float>(P, nt, t_xy[i], vo, so, dout));
      for (int64_t j = 0; j < nt; j += kBatchThreads) iwork.push_back(make_int2(rec, (int)j));
    }
    int lrec = (int)loc.size();
    loc.push_back(make_local_args(P, nt, t_xy[i], wv ? f_jet[i] : nullptr, vo, so, dout));
    for (int64_t j = 0; j < nt; j += kBatchThreads) lwork.push_back(make_int2(lrec, (int)j));
  }
  if (lwork.empty()) return LP_OK;
  Packer pk;
  const size_t o_zs = pk.put(zsegs), o_zw = pk.put(zwork);
  const size_t o_sa = f64 ? pk.put(sp64) : pk.put(sp32), o_sw = pk.put(swork);
  const size_t o_ma = pk.put(mult), o_mw = pk.put(mwork);
  const size_t o_ia = f64 ? pk.put(in64) : pk.put(in32), o_iw = pk.put(iwork);
  const size_t o_la = pk.put(loc), o_lw = pk.put(lwork);
  const size_t o_ba = f64 ? pk.put(bdd) : pk.put(b32), o_bf = pk.put(bfirst);
  const size_t o_da = pk.put(idd), o_df = pk.put(ifirst);
  const size_t o_lda = pk.put(ldd), o_lre = pk.put(lrec), o_lfi = pk.put(lfirst);
  const int nbrec = (int)(f64 ? bdd.size() : b32.size()), ndrec = (int)idd.size();
  const size_t bytes = align_up(pk.img.size(), 256);
  if (bytes > b->buf_cap) {
    cudaStreamSynchronize(s);
    if (b->d_buf) cudaFree(b->d_buf);
    if (b->h_buf) cudaFreeHost(b->h_buf);
    b->d_buf = b->h_buf = nullptr;
    b->buf_cap = 0;
    size_t cap = std::max(bytes, (size_t)1 << 20);
    if (cudaMalloc(&b->d_buf, cap) != cudaSuccess || cudaMallocHost(&b->h_buf, cap) != cudaSuccess) {
      cudaGetLastError();
      return LP_ERR_NOMEM;
    }
    b->buf_cap = cap;
  }
  if ((size_t)total_t > b->list_cap) {
    cudaStreamSynchronize(s);
    if (b->d_list) cudaFree(b->d_list);
    b->d_list = nullptr;
    b->list_cap = 0;
    if (cudaMalloc(&b->d_list, total_t * sizeof(int4)) != cudaSuccess) {
      cudaGetLastError();
      return LP_ERR_NOMEM;
    }
    b->list_cap = total_t;
  }
  std::memcpy(b->h_buf, pk.img.data(), pk.img.size());
  char* d = (char*)b->d_buf;
  cudaEventRecord(b->ev[0], s);
  cudaMemcpyAsync(d, b->h_buf, pk.img.size(), cudaMemcpyHostToDevice, s);
  launch_zero_batch((const ZeroSeg*)(d + o_zs), (const int2*)(d + o_zw), (int)zwork.size(), s);
  cudaEventRecord(b->ev[1], s);
  launch_spread_batch(prec, w, d + o_sa, (const int2*)(d + o_sw), (int)swork.size(), s);
  b->launches += 2;
  launch_spread_wave(prec, w, d + o_ba, (const int*)(d + o_bf), nbrec, bfirst.back(), bsmem, s);
  if (nbrec) ++b->launches;
  launch_spread_fx_list_wave(w, (const SubDDArgs*)(d + o_lda), (const FxListRec*)(d + o_lre),
                             (const int*)(d + o_lfi), (int)ldd.size(), lfirst.back(), lsmem, s);
  if (!ldd.empty()) ++b->launches;
  const long long before = sum_launches(plans, n);
  cudaEventRecord(b->ev[2], s);
  // each plan's transforms: the whole FFT chain for plans on it (counted as
  // forward transforms), spread round-robin over the worker streams, which
  // fork from the batch stream here and join it after; else pruned cuFFT
  // transforms on the batch stream
  cudaEventRecord(b->fork, s);
  for (int k = 0; k < kBatchWorkers; ++k) cudaStreamWaitEvent(b->work[k], b->fork, 0);
  int next = 0;
  for (int i = 0; i < n; ++i) {
    const Plan& P = plans[i]->P;
    const bool wv = V && V[i], ws = S && S[i], wd = D && D[i];
    if (n_t[i] == 0 || (!wv && !ws && !wd)) continue;
    if (P.own_fft) {
      history_transforms(P, wv, ws, wd, b->work[next], false);
      next = (next + 1) % kBatchWorkers;
      continue;
    }
    for (int l = P.l0; l < 2; ++l) {
      const GridLevel& G = P.lv[l];
      cufftSetStream(G.row_fwd, s);
      cufftSetStream(G.col, s);
      if (wv) fft_forward(P, l, 0);
      if (ws) fft_forward(P, l, 1);
      if (wd) {
        fft_forward(P, l, 2);
        fft_forward(P, l, 3);
      }
    }
  }
  for (int k = 0; k < kBatchWorkers; ++k) {
    cudaEventRecord(b->join[k], b->work[k]);
    cudaStreamWaitEvent(s, b->join[k], 0);
  }
  cudaEventRecord(b->ev[3], s);
  launch_multiplier_batch(prec, (const MultArgs*)(d + o_ma), (const int2*)(d + o_mw), (int)mwork.size(), s);
  cudaEventRecord(b->ev[4], s);
  for (int i = 0; i < n; ++i) {
    const Plan& P = plans[i]->P;
    const bool wv = V && V[i], ws = S && S[i], wd = D && D[i];
    if (n_t[i] == 0 || (!wv && !ws && !wd) || P.own_fft) continue;
    for (int l = P.l0; l < 2; ++l) {
      const GridLevel& G = P.lv[l];
      cufftSetStream(G.row_inv, s);
      if (wv) fft_inverse(P, l, 0);
      if (ws) fft_inverse(P, l, 1);
      if (wd) fft_inverse(P, l, 2);
      cufftSetStream(G.row_fwd, P.stream);
      cufftSetStream(G.row_inv, P.stream);
      cufftSetStream(G.col, P.stream);
    }
  }
  cudaEventRecord(b->ev[5], s);
  launch_interp_batch(prec, w, d + o_ia, (const int2*)(d + o_iw), (int)iwork.size(), s);
  launch_interp_dd_wave((const InterpDDArgs*)(d + o_da), (const int*)(d + o_df), ndrec, ifirst.back(), w, s);
  if (ndrec) ++b->launches;
  cudaEventRecord(b->ev[6], s);
  bool corners = false;
  for (const LocalArgs& la : loc) corners = corners || (la.n_corners > 0 && la.out[0] && la.jet && la.order >= 5);
  launch_local_batch(prec, (const LocalArgs*)(d + o_la), (const int2*)(d + o_lw), (int)lwork.size(), b->d_list,
                     b->d_count, total_t, corners, s);
  cudaEventRecord(b->ev[7], s);
  b->launches += 5 + (corners ? 1 : 0) + (sum_launches(plans, n) - before);
  b->pending = true;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

lp_status lp_batch_sync(lp_batch_t b) {
  if (!b) return LP_ERR_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LP_ERR_CUDA;
  b->pending = false;
  return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

lp_status lp_batch_stage_times(lp_batch_t b, float* out) {
  if (!b || !out) return LP_ERR_ARG;
  auto el = [&](int x, int y) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->ev[x], b->ev[y]) != cudaSuccess) {
      cudaGetLastError();
      return -1.0f;
    }
    return ms;
  };
  // {zero+copy, spread, forward FFTs, multiplier, inverse FFTs, interp, local, total, launches}
  out[0] = el(0, 1);
  out[1] = el(1, 2);
  out[2] = el(2, 3);
  out[3] = el(3, 4);
  out[4] = el(4, 5);
  out[5] = el(5, 6);
  out[6] = el(6, 7);
  out[7] = el(0, 7);
  out[8] = (float)b->launches;
  return LP_OK;
}

}  // extern "C"
