// The batched path of include/feast_gb300.h: many independent standard
// pencils (B = I), each with its own order, subspace size and contour,
// iterated together with Algorithm R-FEAST in mixed precision.
//
// Per iteration, for every active pencil at once:
//   1. right-hand sides: Y (first iteration) or the residual form
//      select(E, X) with its coefficients (one grouped kernel);
//   2. ONE persistent launch factors every shifted matrix (first call only)
//      and solves every (matrix, 32-column chunk) -- batch_lu.cu;
//   3. Q = c0 .* X + sum_k coef_k .* S_k^{-1} R (grouped accumulation);
//   4. Rayleigh-Ritz as grouped kernels: CGS2 (one cooperative launch for all
//      blocks), the FP64 projections on DMMA, the reduced problem (FP32 Schur
//      + two FP64 refinement sweeps), Ritz vectors and residuals.
// Steps 1-4 of the steady iterations are captured once into a CUDA graph and
// replayed; the host reads ~m0 eigenvalues and residuals per pencil per
// iteration and takes the Sec. 5 decisions per pencil.  Converged pencils are
// switched off through a device flag array, so the graph never changes.
//
// The task order of the persistent launch comes from a list-scheduling
// simulation on the host (plan_order): each task's priority is its bottom
// level (longest cost path to the end of its matrix's DAG), so the largest
// pencils start first and their panels run ahead of their updates.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <queue>
#include <cstdio>
#include <vector>

#include "../../include/feast_gb300.h"
#include "batch.cuh"
#include "blas1.cuh"
#include "gemm.cuh"
#include "lu.cuh"
#include "norm2.cuh"
#include "ozaki.cuh"
#include "small.cuh"
#include "tc_deep.cuh"
#include "tc_update.cuh"
#include "tune.cuh"

using zc = std::complex<double>;

bool feast_quadrature_host(const feast_contour& c, std::vector<zc>& z, std::vector<zc>& w);

namespace {

inline double2 d2(zc v) { return make_double2(v.real(), v.imag()); }
inline zc zz(double2 v) { return zc(v.x, v.y); }

// ---------------------------------------------------------------- scheduling
// Model costs in microseconds of one SM (only their ratios matter).  The
// per-row panel and per-tile update rates are the autotuner's parameters
// (defaults below; tuned values come from options.tune_cache).
struct CostModel {
  double panel_row = 0.06, update_tile = 4.5;
};
double cost_panel(const CostModel& c, int rows) { return 8.0 + c.panel_row * rows; }
double cost_update(const CostModel& c, int tiles) { return 3.0 + c.update_tile * tiles; }
double cost_lswap(int panels) { return 1.0 + 1.0 * panels; }
double cost_solve(int nb, int w) { return 6.0 * nb + 2.2 * nb * (nb - 1) * (w / 32.0); }

struct Plan {
  std::vector<int> nb, m;
  bool lu = true, solve = true;
  const std::vector<char>* lu_mask = nullptr;  // per matrix: factored here (1) or elsewhere (0)
  std::vector<long long> base;
  bool lu_of(int i) const { return lu && (!lu_mask || (*lu_mask)[i]); }
  long long count_of(int i) const {
    const long long n = nb[i];
    return (lu_of(i) ? n + n * (n - 1) / 2 + (n - 1) : 0) + (solve ? (m[i] + BATCH_SOLVE_W - 1) / BATCH_SOLVE_W : 0);
  }
  long long P(int i, int k) const { return base[i] + k; }
  long long U(int i, int k, int j) const {
    const long long n = nb[i];
    return base[i] + n + (long long)k * (2 * n - k - 1) / 2 + (j - k - 1);
  }
  long long L(int i, int j) const {
    const long long n = nb[i];
    return base[i] + n + n * (n - 1) / 2 + j;
  }
  long long S(int i, int c) const {
    const long long n = nb[i];
    return base[i] + (lu_of(i) ? n + n * (n - 1) / 2 + (n - 1) : 0) + c;
  }
  int nch(int i) const { return solve ? (m[i] + BATCH_SOLVE_W - 1) / BATCH_SOLVE_W : 0; }
};

// Topological task order by list scheduling on `workers` identical workers.
std::vector<int4> plan_order(const std::vector<int>& nbv, const std::vector<int>& mv, bool lu, bool solve,
                             int workers, double* makespan, const CostModel& cm = CostModel(),
                             const std::vector<char>* lu_mask = nullptr) {
  Plan pl;
  pl.nb = nbv;
  pl.m = mv;
  pl.lu = lu;
  pl.solve = solve;
  pl.lu_mask = lu_mask;
  const int nm = (int)nbv.size();
  pl.base.assign(nm + 1, 0);
  for (int i = 0; i < nm; ++i) pl.base[i + 1] = pl.base[i] + pl.count_of(i);
  const long long T = pl.base[nm];
  std::vector<int4> task(T);
  std::vector<double> cost(T), bl(T);
  std::vector<int> pend(T, 0);
  for (int i = 0; i < nm; ++i) {
    const int nb = nbv[i], ch = pl.nch(i);
    if (pl.lu_of(i)) {
      for (int k = 0; k < nb; ++k) {
        task[pl.P(i, k)] = make_int4(BT_PANEL, i, k, k);
        cost[pl.P(i, k)] = cost_panel(cm, BATCH_TILE * (nb - k));
        pend[pl.P(i, k)] = k > 0 ? 1 : 0;
        for (int j = k + 1; j < nb; ++j) {
          task[pl.U(i, k, j)] = make_int4(BT_UPDATE, i, k, j);
          cost[pl.U(i, k, j)] = cost_update(cm, nb - k - 1);
          pend[pl.U(i, k, j)] = 1 + (k > 0 ? 1 : 0);
        }
      }
      for (int j = 0; j + 1 < nb; ++j) {
        task[pl.L(i, j)] = make_int4(BT_LSWAP, i, 0, j);
        cost[pl.L(i, j)] = cost_lswap(nb - 1 - j);
        pend[pl.L(i, j)] = 1;
      }
    }
    double maxS = 0.0;
    for (int c = 0; c < ch; ++c) {
      const int w = std::min(BATCH_SOLVE_W, mv[i] - BATCH_SOLVE_W * c);
      task[pl.S(i, c)] = make_int4(BT_SOLVE, i, 0, c);
      cost[pl.S(i, c)] = cost_solve(nb, w);
      pend[pl.S(i, c)] = pl.lu_of(i) ? nb : 0;  // the last panel and the nb - 1 fix-ups
      bl[pl.S(i, c)] = cost[pl.S(i, c)];
      maxS = std::max(maxS, bl[pl.S(i, c)]);
    }
    if (!pl.lu_of(i)) continue;
    double maxL = 0.0;
    for (int j = 0; j + 1 < nb; ++j) {
      bl[pl.L(i, j)] = cost[pl.L(i, j)] + maxS;
      maxL = std::max(maxL, bl[pl.L(i, j)]);
    }
    bl[pl.P(i, nb - 1)] = cost[pl.P(i, nb - 1)] + std::max(maxL, maxS);
    for (int k = nb - 2; k >= 0; --k) {
      double mx = 0.0;
      for (int j = k + 1; j < nb; ++j) {
        const double nxt = j == k + 1 ? bl[pl.P(i, k + 1)] : bl[pl.U(i, k + 1, j)];
        bl[pl.U(i, k, j)] = cost[pl.U(i, k, j)] + nxt;
        mx = std::max(mx, bl[pl.U(i, k, j)]);
      }
      bl[pl.P(i, k)] = cost[pl.P(i, k)] + mx;
    }
  }
  auto for_succ = [&](long long id, const std::function<void(long long)>& fn) {
    const int4 t = task[id];
    const int i = t.y, nb = nbv[i];
    switch (t.x) {
      case BT_PANEL:
        for (int j = t.z + 1; j < nb; ++j) fn(pl.U(i, t.z, j));
        if (t.z == nb - 1) {
          for (int j = 0; j + 1 < nb; ++j) fn(pl.L(i, j));
          for (int c = 0; c < pl.nch(i); ++c) fn(pl.S(i, c));
        }
        break;
      case BT_UPDATE: fn(t.w == t.z + 1 ? pl.P(i, t.z + 1) : pl.U(i, t.z + 1, t.w)); break;
      case BT_LSWAP:
        for (int c = 0; c < pl.nch(i); ++c) fn(pl.S(i, c));
        break;
      default: break;
    }
  };
  std::priority_queue<std::pair<double, long long>> ready;  // (bottom level, -id)
  for (long long id = 0; id < T; ++id)
    if (pend[id] == 0) ready.push({bl[id], -id});
  using Ev = std::pair<double, long long>;
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> run;
  std::vector<int4> order;
  order.reserve(T);
  double now = 0.0;
  int free = std::max(1, workers);
  while ((long long)order.size() < T) {
    while (free > 0 && !ready.empty()) {
      const long long id = -ready.top().second;
      ready.pop();
      order.push_back(task[id]);
      run.push({now + cost[id], id});
      --free;
    }
    if (run.empty()) break;
    const Ev e = run.top();
    run.pop();
    now = e.first;
    ++free;
    for_succ(e.second, [&](long long s) {
      if (--pend[s] == 0) ready.push({bl[s], -s});
    });
  }
  while (!run.empty()) {
    now = std::max(now, run.top().first);
    run.pop();
  }
  if (makespan) *makespan = now;
  return order;
}

feast_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return FEAST_OK;
  if (e == cudaErrorMemoryAllocation) return FEAST_ERR_ALLOC;
  return FEAST_ERR_CUDA;
}
#define CK(expr)                                   \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)
#define FS(expr)                       \
  do {                                 \
    feast_status s_ = (expr);          \
    if (s_ != FEAST_OK) return s_;     \
  } while (0)

struct GG {  // one grouped GEMM call site
  void* tab = nullptr;
  int* tstart = nullptr;
  int total = 0;
  size_t split_mn = 0;
  bool f32 = false;
};

}  // namespace

struct feast_batch {
  int np = 0, nmat = 0, Nmax = 0, nmax = 0, mmax = 0;
  feast_options opt;
  cudaStream_t st = nullptr;
  cudaStream_t own_stream = nullptr;  // created when the caller passes no stream (the legacy stream cannot be captured)
  std::vector<GrpDesc> pd;
  std::vector<BMat> mats;
  std::vector<std::vector<zc>> z, w;
  std::vector<zc> center;
  std::vector<double> R, aspect, normA;
  std::vector<int> fdom;  // per pencil: CUSTOM nodes without an ellipse (domain test by the filter value)
  int tuned = 0;          // launch parameters read from options.tune_cache
  // tensor-core size classes: pencils of order >= tc_min are padded to a multiple
  // of 256 and their shifted matrices of one padded order are factored together
  // by the two-level tcgen05 LU, each class on its own stream
  struct TcClass {
    int N = 0, mat0 = 0, count = 0;
    TcStaging st;
    DeepStaging dst;
    float2* T = nullptr;
    int32_t *mv = nullptr, *pinv = nullptr, *rowmaps = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    // the class's factorisation captured once into a graph, so that all
    // classes are submitted at once and run side by side (one host call each
    // instead of about a thousand launches one class after another)
    cudaGraphExec_t gexec = nullptr;
    bool graph_failed = false;
  };
  std::vector<TcClass> tcc;
  int tc_min = 768;
  std::vector<char> lu_mask;  // per matrix: 1 = factored by the persistent launch
  int* d_fcnt0 = nullptr;     // per matrix: the completion count a class-factored matrix starts with
  cudaEvent_t fork_ev = nullptr;
  size_t snn = 0, snm = 0, smm = 0, sm = 0, sqm = 0, slog = 0, sS = 0, sX = 0, sN = 0, snb = 0;
  // device
  GrpDesc* d_pd = nullptr;
  BMat* d_mats = nullptr;
  double2 *A = nullptr, *Y = nullptr, *Q = nullptr, *AQ = nullptr, *X = nullptr, *AX = nullptr, *E = nullptr,
          *Rhs = nullptr;
  double2 *Ahat = nullptr, *Bhat = nullptr, *LUB = nullptr, *Cm = nullptr, *Zs = nullptr, *V = nullptr,
          *W = nullptr, *LUW = nullptr, *Minv = nullptr, *Binv = nullptr;
  float2 *C32 = nullptr, *Z32 = nullptr, *V32 = nullptr, *W32 = nullptr, *lam32 = nullptr;
  double2 *lam = nullptr, *coef = nullptr, *c0 = nullptr, *dz = nullptr;
  int *pivB = nullptr, *pivW = nullptr, *useres = nullptr, *active = nullptr, *gate = nullptr;
  double *res = nullptr, *xn = nullptr, *scal = nullptr;
  char* logs = nullptr;
  void* pw_scratch = nullptr;
  float2 *S = nullptr, *Xs = nullptr;
  int *head = nullptr, *cver = nullptr, *pdone = nullptr, *fcnt = nullptr, *mv = nullptr, *perm = nullptr,
      *piv = nullptr, *info = nullptr;
  unsigned* flags = nullptr;
  int4 *t_factor = nullptr, *t_first = nullptr, *t_solve = nullptr;
  int n_factor = 0, n_first = 0, n_solve = 0;
  double makespan = 0.0;
  int grid = 0;
  GG g_AQ, g_Ahat, g_Bhat, g_W32, g_Cm, g_V, g_Zs, g_LUW, g_X, g_AX;
  // A_p Q_p, FP64-accurate on the BF16 tensor cores: digits of every A_p (made at
  // creation) and one work area that the pencils' products use in turn
  std::vector<OzOperator> ozop;
  void* oz_work = nullptr;
  int* orth_cta0 = nullptr;
  int orth_total = 0;
  double2* orth_part = nullptr;
  unsigned* orth_bars = nullptr;
  bool factored = false;
  std::vector<void*> allocs;
  // pinned host staging (graph-capturable copies)
  double2 *h_coef = nullptr, *h_c0 = nullptr, *h_lam = nullptr;
  int *h_use = nullptr, *h_active = nullptr;
  double* h_res = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool graph_failed = false;
  int graph_err = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
};

namespace {

template <typename P>
cudaError_t dalloc(feast_batch* b, P** p, size_t bytes) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, bytes ? bytes : 16);
  if (e != cudaSuccess) return e;
  b->allocs.push_back(v);
  *p = reinterpret_cast<P*>(v);
  return cudaSuccess;
}

BatchLuArgs lu_args(feast_batch* b, const int4* tasks, int ntasks) {
  BatchLuArgs a;
  a.S = b->S;
  a.mats = b->d_mats;
  a.tasks = tasks;
  a.ntasks = ntasks;
  a.head = b->head;
  a.cver = b->cver;
  a.pdone = b->pdone;
  a.fcnt = b->fcnt;
  a.mv = b->mv;
  a.perm = b->perm;
  a.piv = b->piv;
  a.info = b->info;
  a.R = b->Rhs;
  a.X = b->Xs;
  a.active = b->active;
  a.flags = b->flags;
  a.wait_ns = feast_wait_limit_ns(2000000000ull);
  return a;
}

// One grouped GEMM call site: entries ordered by per-tile work (longest first,
// so the long-K tiles do not form the tail), complex128 products with few
// output tiles and a long K cut into K-chunks of at least 256.
template <typename T>
feast_status make_gg(feast_batch* b, GG& g, const std::function<GemmArgs<T>(const GrpDesc&)>& f) {
  std::vector<GemmArgs<T>> tab(b->np);
  size_t ws_total = 0;
  for (int p = 0; p < b->np; ++p) {
    tab[p] = f(b->pd[p]);
    tab[p].batch = 1;
    tab[p].tag = p;
    int sk = 1;
    if (!std::is_same<T, float>::value && gemm_tiles(tab[p].M, tab[p].N) <= 4 && tab[p].K >= 512)
      sk = std::min(8, tab[p].K / 256);
    tab[p].splitk = sk;
    if (sk > 1) {
      ws_total += (size_t)sk * tab[p].M * tab[p].N;
      g.split_mn = std::max(g.split_mn, (size_t)tab[p].M * tab[p].N);
    }
  }
  std::stable_sort(tab.begin(), tab.end(), [](const GemmArgs<T>& x, const GemmArgs<T>& y) {
    return (long long)x.K / x.splitk > (long long)y.K / y.splitk;
  });
  if (ws_total) {
    cplx<T>* ws = nullptr;
    CK(dalloc(b, &ws, ws_total * sizeof(cplx<T>)));
    size_t off = 0;
    for (auto& e : tab)
      if (e.splitk > 1) {
        e.ws = ws + off;
        e.ws_elems = (size_t)e.splitk * e.M * e.N;
        off += e.ws_elems;
      }
  }
  std::vector<int> ts(b->np + 1, 0);
  for (int p = 0; p < b->np; ++p) ts[p + 1] = ts[p] + gemm_tiles(tab[p].M, tab[p].N) * tab[p].splitk;
  CK(dalloc(b, &g.tab, tab.size() * sizeof(GemmArgs<T>)));
  CK(dalloc(b, &g.tstart, ts.size() * sizeof(int)));
  CK(cudaMemcpyAsync(g.tab, tab.data(), tab.size() * sizeof(GemmArgs<T>), cudaMemcpyHostToDevice, b->st));
  CK(cudaMemcpyAsync(g.tstart, ts.data(), ts.size() * sizeof(int), cudaMemcpyHostToDevice, b->st));
  CK(cudaStreamSynchronize(b->st));
  g.total = ts[b->np];
  g.f32 = std::is_same<T, float>::value;
  return FEAST_OK;
}

cudaError_t run_gg(feast_batch* b, const GG& g) {
  if (g.f32)
    return gemm_grouped<float>(reinterpret_cast<const GemmArgs<float>*>(g.tab), g.tstart, b->np, g.total, b->active,
                               0, b->st);
  return gemm_grouped<double>(reinterpret_cast<const GemmArgs<double>*>(g.tab), g.tstart, b->np, g.total, b->active,
                              g.split_mn, b->st);
}

GemmArgs<double> zargs(int M, int N, int K, const double2* A, long long lda, int opA, const double2* B, long long ldb,
                       int opB, double2* C, long long ldc) {
  GemmArgs<double> g;
  g.M = M; g.N = N; g.K = K;
  g.alpha = make_double2(1.0, 0.0);
  g.beta = make_double2(0.0, 0.0);
  g.A = A; g.lda = lda; g.opA = opA;
  g.B = B; g.ldb = ldb; g.opB = opB;
  g.C = C; g.ldc = ldc;
  return g;
}

feast_status read_flags(feast_batch* b) {
  unsigned f = 0;
  CK(cudaMemcpyAsync(&f, b->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, b->st));
  CK(cudaStreamSynchronize(b->st));
  if (f & DEVFLAG_TIMEOUT) return FEAST_ERR_DEVICE_TIMEOUT;
  if (f & DEVFLAG_NONFINITE) return FEAST_ERR_NONFINITE;
  if (f & DEVFLAG_BADARG) return FEAST_ERR_CUDA;
  return FEAST_OK;
}

// The far and deep steps of a class's two-level LU (Sec. 5.5's factorisations
// with 256-column outer blocks): every panel's interchanges on the columns
// beyond the block, U12 = L11^{-1} A12 as one deep product with T = -L11^{-1},
// then the K = 256 product of the block's L and U off everything below-right.
cudaError_t class_far(const LuBatch<float>& lu, int K0, int KB, void* c, cudaStream_t s) {
  const feast_batch::TcClass* cls = reinterpret_cast<const feast_batch::TcClass*>(c);
  const int far0 = K0 + KB, nfar = lu.n - far0;
  if (nfar <= 0) return cudaSuccess;
  cudaError_t e;
  if ((e = block_swaps_far(lu, K0, KB, s)) != cudaSuccess) return e;
  if ((e = block_inverse_negated(lu, false, KB, K0 / KB, 1, cls->T, s)) != cudaSuccess) return e;
  return tc_far_gemm(lu, K0, KB, cls->T, cls->dst, s);
}

cudaError_t class_deep(const LuBatch<float>& lu, int K0, int KB, void* c, cudaStream_t s) {
  const feast_batch::TcClass* cls = reinterpret_cast<const feast_batch::TcClass*>(c);
  cudaError_t e = tc_deep_stage(lu, K0, KB, cls->dst, s);
  if (e != cudaSuccess) return e;
  return tc_deep_run(lu, K0, KB, cls->dst, s);
}

// Every tensor-core class factored on its own stream (forked from and joined
// back into the batch's stream): the class's shifted matrices are consecutive
// in every arena with stride N, so one LuBatch view of q = count matrices
// covers them; the factor lands in the layout the persistent solve tasks read
// (P S = L U in place, perm with (P S)[r] = S[perm[r]]).
cudaError_t factor_classes(feast_batch* b) {
  if (b->tcc.empty()) return cudaSuccess;
  cudaError_t e;
  int dev = 0, nsm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(b->fork_ev, b->st)) != cudaSuccess) return e;
  for (feast_batch::TcClass& c : b->tcc) {
    if ((e = cudaStreamWaitEvent(c.s, b->fork_ev, 0)) != cudaSuccess) return e;
    const BMat& M0 = b->mats[c.mat0];
    LuBatch<float> lu;
    lu.S = b->S + M0.soff;
    lu.ld = c.N;
    lu.stride = (long long)c.N * c.N;
    lu.n = c.N;  // the padding is an identity block: it is never a pivot and stays untouched
    lu.q = c.count;
    lu.piv = b->piv + M0.poff;
    lu.perm = b->perm + M0.poff;
    lu.pinv = c.pinv;
    lu.info = b->info + c.mat0;
    lu.flags = b->flags;
    lu.tc = &c.st;
    lu.mv = c.mv;
    lu.mv_panels = c.N / 64;
    lu.rowmaps = c.rowmaps;
    lu.u12_in_stage = true;
    // the four-CTA cluster panel while the class's panels alone leave SMs idle
    lu.panel_cluster = 4 * c.count <= nsm;
    TrailingUpdateFn<float> upd = nullptr;
    void* ctx = nullptr;
    select_trailing_update<float>(&upd, &ctx, &c.st);
    auto run = [&]() -> cudaError_t {
      return c.dst.Ast ? lu_factor_two_level(lu, 64, 256, upd, ctx, class_far, class_deep, &c, c.s)
                       : lu_factor_batched<float>(lu, 64, upd, ctx, c.s);
    };
    if (!c.gexec && !c.graph_failed && !b->opt.batch_direct) {
      cudaGraph_t g = nullptr;
      cudaError_t ce = cudaStreamBeginCapture(c.s, cudaStreamCaptureModeRelaxed);
      cudaError_t re = ce == cudaSuccess ? run() : ce;
      if (ce == cudaSuccess) ce = cudaStreamEndCapture(c.s, &g);
      if (ce == cudaSuccess && re == cudaSuccess && g) ce = cudaGraphInstantiate(&c.gexec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (ce != cudaSuccess || re != cudaSuccess || !c.gexec) {
        c.graph_failed = true;  // direct launches from here on
        if (c.gexec) cudaGraphExecDestroy(c.gexec);
        c.gexec = nullptr;
        cudaGetLastError();
      }
    }
    e = c.gexec ? cudaGraphLaunch(c.gexec, c.s) : run();
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(c.done, c.s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The batch's stream waits for every class.
cudaError_t join_classes(feast_batch* b) {
  cudaError_t e;
  for (feast_batch::TcClass& c : b->tcc)
    if ((e = cudaStreamWaitEvent(b->st, c.done, 0)) != cudaSuccess) return e;
  return cudaSuccess;
}

// Persistent launch over one of the task lists.  A factorisation launch also
// factors the tensor-core classes on their streams: beside the persistent
// kernel when it only factors (its tasks never touch a class matrix), before it
// when it also solves (the class matrices' solve tasks need their factors).
cudaError_t launch_lu(feast_batch* b, const int4* tasks, int n) {
  if (tasks == b->t_factor || tasks == b->t_first) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(b->cver, 0, b->snb * sizeof(int), b->st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b->pdone, 0, b->snb * sizeof(int), b->st)) != cudaSuccess) return e;
    if (b->d_fcnt0)
      e = cudaMemcpyAsync(b->fcnt, b->d_fcnt0, b->nmat * sizeof(int), cudaMemcpyDeviceToDevice, b->st);
    else
      e = cudaMemsetAsync(b->fcnt, 0, b->nmat * sizeof(int), b->st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b->info, 0, b->nmat * sizeof(int), b->st)) != cudaSuccess) return e;
    if ((e = factor_classes(b)) != cudaSuccess) return e;
    if (tasks == b->t_first && (e = join_classes(b)) != cudaSuccess) return e;
    if ((e = batch_lu_launch(lu_args(b, tasks, n), b->Nmax, b->grid, b->st)) != cudaSuccess) return e;
    return tasks == b->t_factor ? join_classes(b) : cudaSuccess;
  }
  return batch_lu_launch(lu_args(b, tasks, n), b->Nmax, b->grid, b->st);
}

// Rayleigh-Ritz for every active pencil (Algorithm R-FEAST steps 4-5 with Q^ = Q).
cudaError_t enqueue_rr(feast_batch* b) {
  cudaError_t e;
  const size_t mmb = b->smm * sizeof(double2);
#define CE(x) if ((e = (x)) != cudaSuccess) return e
  CE(orth_cgs2_grp(b->Q, b->d_pd, b->orth_cta0, b->np, b->orth_total, b->orth_part, b->orth_bars, b->active,
                   b->flags, b->st));
  for (int p = 0; p < b->np; ++p) {
    const GrpDesc& d = b->pd[p];
    OzWork w;
    oz_work_layout(b->oz_work, d.n, d.m, &w);
    CE(oz_apply(b->ozop[p], b->Q + d.onm, d.n, d.m, b->AQ + d.onm, d.n, w, b->flags, b->st, b->active + p));
  }
  CE(run_gg(b, b->g_Ahat));
  CE(run_gg(b, b->g_Bhat));
  // C = B^^{-1} A^.  Q is orthonormal, so B^ = I + E with E at rounding level:
  // B^^{-1} = 2I - B^ to O(|E|^2) while max |E_ij| <= 1e-10 (for m <= 128 the
  // dropped terms stay below 2e-16); a pencil past that gets B^^{-1} by LU.
  CE(inverse_check_grp(b->Bhat, b->d_pd, b->np, b->active, 1e-10, b->gate, b->Binv, b->st));
  CE(small_inverse_gated_grp(b->Bhat, b->LUB, b->pivB, b->Binv, b->d_pd, b->np, b->flags, b->gate, b->st));
  CE(run_gg(b, b->g_Cm));
  CE(to_c64(b->Cm, b->C32, b->smm, b->st));
  CE(small_schur_grp(b->C32, b->Z32, b->lam32, b->d_pd, b->np, b->mmax, b->active, b->flags, b->logs, b->st));
  CE(small_trevc_grp(b->C32, b->V32, b->d_pd, b->np, b->mmax, b->active, b->st));
  CE(run_gg(b, b->g_W32));
  CE(to_c128(b->W32, b->W, b->smm, b->st));
  // Two refinement sweeps E = W^{-1} C W, lam = diag(E), W <- W (I + Delta); W^{-1}
  // by one LU per pencil (a CTA each: at m <= 128 this beats Newton-Schulz on the
  // FP64 tensor cores, whose m x m products leave most SMs idle)
  for (int sweep = 0; sweep < 2; ++sweep) {
    CE(cudaMemcpyAsync(b->LUW, b->W, mmb, cudaMemcpyDeviceToDevice, b->st));
    CE(small_lu_grp(b->LUW, b->d_pd, b->np, b->active, b->pivW, b->flags, b->st));
    CE(batch_identity(b->Minv, b->d_pd, b->np, b->mmax, b->active, b->st));
    CE(small_lu_solve_grp(b->LUW, b->pivW, b->d_pd, b->np, b->mmax, b->active, b->Minv, 0, b->st));
    CE(run_gg(b, b->g_V));
    CE(run_gg(b, b->g_Zs));
    CE(eig_refine_step_grp(b->Zs, b->Ahat, b->lam, b->d_pd, b->np, b->active, b->st));
    CE(run_gg(b, b->g_LUW));
    CE(cudaMemcpyAsync(b->W, b->LUW, mmb, cudaMemcpyDeviceToDevice, b->st));
  }
  CE(run_gg(b, b->g_X));
  CE(run_gg(b, b->g_AX));
  CE(batch_normalize(b->X, b->AX, b->d_pd, b->np, b->mmax, b->active, b->xn, b->st));
  CE(batch_residual(b->AX, b->X, b->lam, b->d_pd, b->np, b->mmax, b->active, b->E, b->res, b->st));
  CE(cudaMemcpyAsync(b->h_lam, b->lam, b->sm * sizeof(double2), cudaMemcpyDeviceToHost, b->st));
  CE(cudaMemcpyAsync(b->h_res, b->res, b->sm * sizeof(double), cudaMemcpyDeviceToHost, b->st));
#undef CE
  return cudaSuccess;
}

cudaError_t enqueue_inputs(feast_batch* b) {
  cudaError_t e;
  if ((e = cudaMemcpyAsync(b->coef, b->h_coef, b->sqm * sizeof(double2), cudaMemcpyHostToDevice, b->st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(b->c0, b->h_c0, b->sm * sizeof(double2), cudaMemcpyHostToDevice, b->st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(b->useres, b->h_use, b->sm * sizeof(int), cudaMemcpyHostToDevice, b->st)) != cudaSuccess)
    return e;
  return cudaMemcpyAsync(b->active, b->h_active, b->np * sizeof(int), cudaMemcpyHostToDevice, b->st);
}

// A steady iteration: residual-form right-hand sides, solves, accumulation, Rayleigh-Ritz.
cudaError_t enqueue_steady(feast_batch* b) {
  cudaError_t e;
  if ((e = enqueue_inputs(b)) != cudaSuccess) return e;
  if ((e = batch_select(b->E, b->X, b->useres, b->d_pd, b->np, b->nmax, b->mmax, b->active, b->Rhs, b->st)) !=
      cudaSuccess)
    return e;
  if ((e = launch_lu(b, b->t_solve, b->n_solve)) != cudaSuccess) return e;
  if ((e = batch_accumulate(b->Xs, b->d_mats, b->d_pd, b->np, b->nmax, b->mmax, b->coef, b->c0, b->X, b->active,
                            b->Q, b->st)) != cudaSuccess)
    return e;
  return enqueue_rr(b);
}

// Host: coefficients of pencil p for Ritz values theta (or the plain filter when null).
void host_coefs(feast_batch* b, int p, const double2* theta) {
  const GrpDesc& d = b->pd[p];
  for (int i = 0; i < d.m; ++i) {
    bool u = false;
    zc th(0.0);
    if (theta) {
      th = zz(theta[d.om + i]);
      if (std::isfinite(th.real()) && std::isfinite(th.imag())) {
        double dmin = 1e300;
        for (int k = 0; k < d.q; ++k) dmin = std::min(dmin, std::abs(b->z[p][k] - th));
        u = dmin >= 1e-10 * b->R[p];
      }
    }
    zc acc = 0.0;
    for (int k = 0; k < d.q; ++k) {
      const zc g = u ? b->w[p][k] / (b->z[p][k] - th) : b->w[p][k];
      acc += g;
      b->h_coef[d.oqm + (size_t)k * d.m + i] = d2(g);
    }
    b->h_c0[d.om + i] = d2(u ? acc : zc(0.0));
    b->h_use[d.om + i] = u ? 1 : 0;
  }
}

bool inside(const feast_batch* b, int p, zc l) {
  if (b->fdom[p]) {
    zc r = 0.0;
    for (size_t k = 0; k < b->z[p].size(); ++k) r += b->w[p][k] / (b->z[p][k] - l);
    return std::abs(r) >= 0.5;
  }
  const double x = (l.real() - b->center[p].real()) / b->R[p];
  const double y = (l.imag() - b->center[p].imag()) / (b->R[p] * b->aspect[p]);
  return x * x + y * y < 1.0;
}

std::vector<int> candidates(const feast_batch* b, int p) {
  const GrpDesc& d = b->pd[p];
  std::vector<int> idx;
  for (int i = 0; i < d.m; ++i) {
    const zc l = zz(b->h_lam[d.om + i]);
    const double r = b->h_res[d.om + i];
    if (!std::isfinite(l.real()) || !std::isfinite(l.imag()) || !std::isfinite(r)) continue;
    if (inside(b, p, l) && r <= b->opt.cand_tol) idx.push_back(i);
  }
  std::sort(idx.begin(), idx.end(), [&](int x, int y) {
    const zc a = zz(b->h_lam[d.om + x]), c = zz(b->h_lam[d.om + y]);
    if (a.real() != c.real()) return a.real() < c.real();
    return a.imag() < c.imag();
  });
  return idx;
}

feast_status ensure_factored_first(feast_batch* b, bool with_solve) {
  // with_solve: the first launch also solves the current right-hand sides
  const int4* t = with_solve ? (b->factored ? b->t_solve : b->t_first) : (b->factored ? nullptr : b->t_factor);
  const int n = with_solve ? (b->factored ? b->n_solve : b->n_first) : (b->factored ? 0 : b->n_factor);
  if (!t) return FEAST_OK;
  const bool timing = b->opt.timing && !b->factored;
  if (timing) CK(cudaEventRecord(b->ev[0], b->st));
  CK(launch_lu(b, t, n));
  if (timing) CK(cudaEventRecord(b->ev[1], b->st));
  if (!b->factored) {
    FS(read_flags(b));
    std::vector<int> info(b->nmat);
    CK(cudaMemcpyAsync(info.data(), b->info, b->nmat * sizeof(int), cudaMemcpyDeviceToHost, b->st));
    CK(cudaStreamSynchronize(b->st));
    b->factored = true;
    for (int v : info)
      if (v != 0) return FEAST_ERR_SINGULAR_SHIFT;
  }
  return FEAST_OK;
}

}  // namespace

extern "C" {

void feast_batch_destroy(feast_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  for (auto& c : b->tcc)
    if (c.s) cudaStreamSynchronize(c.s);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (void* p : b->allocs) cudaFree(p);
  for (void* p : {(void*)b->h_coef, (void*)b->h_c0, (void*)b->h_lam, (void*)b->h_use, (void*)b->h_active,
                  (void*)b->h_res})
    if (p) cudaFreeHost(p);
  for (auto& e : b->ev)
    if (e) cudaEventDestroy(e);
  for (auto& c : b->tcc) {
    if (c.gexec) cudaGraphExecDestroy(c.gexec);
    if (c.s) cudaStreamDestroy(c.s);
    if (c.done) cudaEventDestroy(c.done);
  }
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  delete b;
}

feast_status feast_batch_plan(int nmat, const int* nb, const int* m, int with_lu, int with_solve, int workers,
                              int* tasks, int capacity, int* ntasks, double* makespan_us) {
  if (nmat < 1 || !nb || !m || !ntasks || workers < 1) return FEAST_ERR_ARG;
  std::vector<int> nbv(nb, nb + nmat), mv(m, m + nmat);
  for (int i = 0; i < nmat; ++i)
    if (nbv[i] < 1 || mv[i] < 0) return FEAST_ERR_ARG;
  double ms = 0.0;
  const std::vector<int4> order = plan_order(nbv, mv, with_lu != 0, with_solve != 0, workers, &ms);
  *ntasks = (int)order.size();
  if (makespan_us) *makespan_us = ms;
  if (tasks) {
    if (capacity < (int)order.size()) return FEAST_ERR_ARG;
    for (size_t t = 0; t < order.size(); ++t) {
      tasks[4 * t] = order[t].x;
      tasks[4 * t + 1] = order[t].y;
      tasks[4 * t + 2] = order[t].z;
      tasks[4 * t + 3] = order[t].w;
    }
  }
  return FEAST_OK;
}

feast_status feast_batch_create(feast_batch** out, int count, const int64_t* n, const feast_z* const* A,
                                const int64_t* lda, const feast_contour* contours, const int* m0,
                                const feast_options* o, void* stream) {
  if (!out) return FEAST_ERR_ARG;
  *out = nullptr;
  if (count < 1 || count > 4096 || !n || !A || !contours || !m0) return FEAST_ERR_ARG;
  feast_batch* b = new (std::nothrow) feast_batch();
  if (!b) return FEAST_ERR_ALLOC;
  if (o) b->opt = *o; else feast_default_options(&b->opt);
  if (b->opt.tol <= 0) b->opt.tol = 1e-10;
  if (b->opt.max_iter < 1) b->opt.max_iter = 20;
  if (b->opt.max_iter > 64) b->opt.max_iter = 64;
  if (b->opt.cand_tol <= 0) b->opt.cand_tol = 1e-4;
  auto bad = [&](feast_status s) { feast_batch_destroy(b); return s; };
  if (b->opt.algo != FEAST_ALGO_R || b->opt.precision != FEAST_PREC_MIXED) return bad(FEAST_ERR_ARG);
  b->st = reinterpret_cast<cudaStream_t>(stream);
  if (!b->st) {
    // a blocking stream: it stays ordered with the legacy default stream
    if (cudaStreamCreate(&b->own_stream) != cudaSuccess) return bad(FEAST_ERR_CUDA);
    b->st = b->own_stream;
  }
  b->np = count;
  b->pd.resize(count);
  b->z.resize(count);
  b->w.resize(count);
  for (int p = 0; p < count; ++p) {
    const int64_t np_ = n[p];
    const int64_t ld = lda ? lda[p] : np_;
    if (np_ < 1 || np_ > BATCH_MAX_N || m0[p] < 1 || m0[p] > np_ || m0[p] > 160 || !A[p] || ld < np_)
      return bad(FEAST_ERR_ARG);
    const feast_contour& c = contours[p];
    // CUSTOM nodes with R = 0: no ellipse, the domain test is |rho(lambda)| >= 1/2
    const bool fdom = c.rule == FEAST_RULE_CUSTOM && c.R == 0.0;
    if (!fdom && (c.R <= 0.0 || c.aspect <= 0.0)) return bad(FEAST_ERR_ARG);
    if (!feast_quadrature_host(c, b->z[p], b->w[p]) || b->z[p].size() > 256) return bad(FEAST_ERR_ARG);
    b->center.push_back(zc(c.center.re, c.center.im));
    b->R.push_back(fdom ? 1.0 : c.R);
    b->aspect.push_back(fdom ? 1.0 : c.aspect);
    b->fdom.push_back(fdom ? 1 : 0);
    GrpDesc& d = b->pd[p];
    d.n = (int)np_;
    d.m = m0[p];
    d.q = (int)b->z[p].size();
    d.mat0 = b->nmat;
    d.onn = (long long)b->snn;
    d.onm = (long long)b->snm;
    d.omm = (long long)b->smm;
    d.om = (long long)b->sm;
    d.oqm = (long long)b->sqm;
    d.olog = (long long)b->slog;
    b->snn += (size_t)d.n * d.n;
    b->snm += (size_t)d.n * d.m;
    b->smm += (size_t)d.m * d.m;
    b->sm += (size_t)d.m;
    b->sqm += (size_t)d.q * d.m;
    b->slog += (schur_log_bytes(d.m) + 255) / 256 * 256;
    b->nmax = std::max(b->nmax, d.n);
    b->mmax = std::max(b->mmax, d.m);
  }
  // padded orders: multiples of 64, or of 256 for the tensor-core classes
  // (orders from tc_min on; tc_min = 0: none)
  if (b->opt.batch_tc_min < 0) {
    b->tc_min = 0;
  } else if (b->opt.batch_tc_min > 0) {
    b->tc_min = std::max(512, b->opt.batch_tc_min);
  } else if (b->opt.tune_cache) {
    char key[256];
    std::snprintf(key, sizeof(key), "%s|batch|count%d|nmax%lld|mixed", tune_gpu_name().c_str(), b->np,
                  tune_bucket(((b->nmax + BATCH_TILE - 1) / BATCH_TILE) * BATCH_TILE));
    std::map<std::string, double> t;
    if (tune_lookup(b->opt.tune_cache, key, t) && t.count("tc_min"))
      b->tc_min = t["tc_min"] > 0 ? std::max(512, (int)t["tc_min"]) : 0;
  }
  std::vector<int> Np(count), order(count);
  for (int p = 0; p < count; ++p) {
    const int nn = b->pd[p].n;
    Np[p] = (b->tc_min > 0 && nn >= b->tc_min) ? (nn + 255) / 256 * 256 : (nn + BATCH_TILE - 1) / BATCH_TILE * BATCH_TILE;
    order[p] = p;
  }
  // class pencils first (largest order first), then the others in the given order
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const bool tx = b->tc_min > 0 && b->pd[x].n >= b->tc_min, ty = b->tc_min > 0 && b->pd[y].n >= b->tc_min;
    if (tx != ty) return tx;
    if (tx) return Np[x] > Np[y];
    return false;
  });
  for (int p : order) {
    GrpDesc& d = b->pd[p];
    const int N = Np[p];
    const bool tc = b->tc_min > 0 && d.n >= b->tc_min;
    b->Nmax = std::max(b->Nmax, N);
    d.mat0 = b->nmat;
    if (tc) {
      if (b->tcc.empty() || b->tcc.back().N != N) {
        feast_batch::TcClass c;
        c.N = N;
        c.mat0 = b->nmat;
        b->tcc.push_back(c);
      }
      b->tcc.back().count += d.q;
    }
    for (int k = 0; k < d.q; ++k) {
      BMat M;
      M.soff = (long long)b->sS;
      M.xoff = (long long)b->sX;
      M.roff = d.onm;
      M.N = N;
      M.n = d.n;
      M.m = d.m;
      M.nb = N / BATCH_TILE;
      M.coff = (int)b->snb;
      M.poff = (int)b->sN;
      M.pencil = p;
      M.shift = k;
      b->sS += (size_t)N * N;
      b->sX += (size_t)N * d.m;
      b->snb += (size_t)M.nb;
      b->sN += (size_t)N;
      b->mats.push_back(M);
      b->lu_mask.push_back(tc ? 0 : 1);
      ++b->nmat;
    }
  }
  cudaError_t e;
#define AL(p, bytes) if ((e = dalloc(b, &(p), (bytes))) != cudaSuccess) return bad(cuda_status(e))
  AL(b->d_pd, b->np * sizeof(GrpDesc));
  AL(b->d_mats, b->nmat * sizeof(BMat));
  AL(b->A, b->snn * sizeof(double2));
  double2** nms[] = {&b->Y, &b->Q, &b->AQ, &b->X, &b->AX, &b->E, &b->Rhs};
  for (double2** p : nms) AL(*p, b->snm * sizeof(double2));
  double2** mms[] = {&b->Ahat, &b->Bhat, &b->LUB, &b->Cm, &b->Zs, &b->V, &b->W, &b->LUW, &b->Minv, &b->Binv};
  for (double2** p : mms) AL(*p, b->smm * sizeof(double2));
  float2** m32[] = {&b->C32, &b->Z32, &b->V32, &b->W32};
  for (float2** p : m32) AL(*p, b->smm * sizeof(float2));
  AL(b->lam32, b->sm * sizeof(float2));
  AL(b->lam, b->sm * sizeof(double2));
  AL(b->c0, b->sm * sizeof(double2));
  AL(b->coef, b->sqm * sizeof(double2));
  AL(b->dz, b->nmat * sizeof(double2));
  AL(b->pivB, b->sm * sizeof(int));
  AL(b->pivW, b->sm * sizeof(int));
  AL(b->useres, b->sm * sizeof(int));
  AL(b->active, b->np * sizeof(int));
  AL(b->gate, b->np * sizeof(int));
  AL(b->res, b->sm * sizeof(double));
  AL(b->xn, b->sm * sizeof(double));
  AL(b->scal, 64);
  AL(b->logs, b->slog);
  AL(b->pw_scratch, norm2_scratch_bytes(b->nmax));
  AL(b->S, b->sS * sizeof(float2));
  AL(b->Xs, b->sX * sizeof(float2));
  AL(b->head, 64);
  AL(b->cver, b->snb * sizeof(int));
  AL(b->pdone, b->snb * sizeof(int));
  AL(b->fcnt, b->nmat * sizeof(int));
  AL(b->info, b->nmat * sizeof(int));
  AL(b->mv, b->snb * BATCH_MVSTRIDE * sizeof(int));
  AL(b->perm, b->sN * sizeof(int));
  AL(b->piv, b->sN * sizeof(int));
  AL(b->flags, 64);
  // tensor-core classes: the update's and the deep product's staging, the far
  // step's -L11^{-1}, the panels' moved-row lists, inverse permutations, a stream
  for (auto& c : b->tcc) {
    AL(c.st.Ast, tc_staging_bytes_A(c.N, c.count));
    AL(c.st.Bst, tc_staging_bytes_B(c.N, c.count));
    c.st.rows_max = 2LL * c.N;
    c.st.cols_max = c.N;
    c.st.q = c.count;
    if (c.N >= 1024) {  // two-level LU with 256-column outer blocks
      AL(c.dst.Ast, deep_staging_bytes_A(c.N, c.count));
      AL(c.dst.Bst, deep_staging_bytes_B(c.N, c.count));
      c.dst.rows_max = 2LL * c.N;
      c.dst.cols_max = c.N;
      c.dst.q = c.count;
      AL(c.T, (size_t)c.count * 256 * 256 * sizeof(float2));
    }
    AL(c.mv, (size_t)(c.N / 64) * c.count * LU_MV_STRIDE * sizeof(int32_t));
    AL(c.pinv, (size_t)c.count * c.N * sizeof(int32_t));
    AL(c.rowmaps, lu_rowmap_ints(c.N, c.count, c.N >= 1024 ? 256 : 64) * sizeof(int32_t));
    if ((e = cudaStreamCreateWithFlags(&c.s, cudaStreamNonBlocking)) != cudaSuccess) return bad(cuda_status(e));
    if ((e = cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming)) != cudaSuccess) return bad(cuda_status(e));
  }
  if (!b->tcc.empty()) {
    // a class-factored matrix enters the persistent launch as finished
    // (completion count = its block columns), so only its solves run there
    if ((e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming)) != cudaSuccess) return bad(cuda_status(e));
    std::vector<int> f0(b->nmat, 0);
    for (int i = 0; i < b->nmat; ++i)
      if (!b->lu_mask[i]) f0[i] = b->mats[i].nb;
    AL(b->d_fcnt0, b->nmat * sizeof(int));
    if ((e = cudaMemcpyAsync(b->d_fcnt0, f0.data(), f0.size() * sizeof(int), cudaMemcpyHostToDevice, b->st)) !=
        cudaSuccess)
      return bad(cuda_status(e));
    if ((e = cudaStreamSynchronize(b->st)) != cudaSuccess) return bad(cuda_status(e));
  }
  for (void** hp : {(void**)&b->h_coef, (void**)&b->h_c0, (void**)&b->h_lam}) {
    if ((e = cudaMallocHost(hp, (hp == (void**)&b->h_coef ? b->sqm : b->sm) * sizeof(double2))) != cudaSuccess)
      return bad(cuda_status(e));
  }
  if ((e = cudaMallocHost((void**)&b->h_use, b->sm * sizeof(int))) != cudaSuccess) return bad(cuda_status(e));
  if ((e = cudaMallocHost((void**)&b->h_active, b->np * sizeof(int))) != cudaSuccess) return bad(cuda_status(e));
  if ((e = cudaMallocHost((void**)&b->h_res, b->sm * sizeof(double))) != cudaSuccess) return bad(cuda_status(e));
  for (auto& ev : b->ev)
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bad(cuda_status(e));
  // tables
  std::vector<double2> zd;  // the node of every shifted matrix, in matrix order
  for (const BMat& M : b->mats) zd.push_back(d2(b->z[M.pencil][M.shift]));
  if ((e = cudaMemcpyAsync(b->d_pd, b->pd.data(), b->np * sizeof(GrpDesc), cudaMemcpyHostToDevice, b->st)) != cudaSuccess)
    return bad(cuda_status(e));
  if ((e = cudaMemcpyAsync(b->d_mats, b->mats.data(), b->nmat * sizeof(BMat), cudaMemcpyHostToDevice, b->st)) !=
      cudaSuccess)
    return bad(cuda_status(e));
  if ((e = cudaMemcpyAsync(b->dz, zd.data(), zd.size() * sizeof(double2), cudaMemcpyHostToDevice, b->st)) != cudaSuccess)
    return bad(cuda_status(e));
  if ((e = cudaMemsetAsync(b->flags, 0, 64, b->st)) != cudaSuccess) return bad(cuda_status(e));
  for (int p = 0; p < b->np; ++p) {
    const GrpDesc& d = b->pd[p];
    const int64_t ld = lda ? lda[p] : d.n;
    if ((e = cudaMemcpy2DAsync(b->A + d.onn, d.n * sizeof(double2), A[p], ld * sizeof(double2), d.n * sizeof(double2),
                               d.n, cudaMemcpyDefault, b->st)) != cudaSuccess)
      return bad(cuda_status(e));
  }
  if ((e = check_finite(b->A, b->snn, b->flags, b->st)) != cudaSuccess) return bad(cuda_status(e));
  {
    feast_status s = read_flags(b);
    if (s != FEAST_OK) return bad(s);
  }
  for (int p = 0; p < b->np; ++p) {
    const GrpDesc& d = b->pd[p];
    if ((e = norm2_power(b->A + d.onn, d.n, d.n, 50, b->pw_scratch, b->scal, b->flags, b->st)) != cudaSuccess)
      return bad(cuda_status(e));
    double s = 0.0;
    if ((e = cudaMemcpyAsync(&s, b->scal, sizeof(double), cudaMemcpyDeviceToHost, b->st)) != cudaSuccess)
      return bad(cuda_status(e));
    if ((e = cudaStreamSynchronize(b->st)) != cudaSuccess) return bad(cuda_status(e));
    b->normA.push_back(s);
  }
  // digits of every A_p for the emulated-FP64 products A_p Q_p
  {
    size_t wmax = 0;
    b->ozop.resize(b->np);
    for (int p = 0; p < b->np; ++p) {
      const GrpDesc& d = b->pd[p];
      void* base = nullptr;
      if ((e = dalloc(b, &base, oz_operator_bytes(d.n))) != cudaSuccess) return bad(cuda_status(e));
      oz_operator_layout(base, d.n, &b->ozop[p]);
      if ((e = oz_make_operator(b->A + d.onn, d.n, OP_N, b->ozop[p], b->st)) != cudaSuccess) return bad(cuda_status(e));
      wmax = std::max(wmax, oz_work_bytes(d.n, d.m));
    }
    if ((e = dalloc(b, &b->oz_work, wmax)) != cudaSuccess) return bad(cuda_status(e));
  }
  // persistent launch: resident CTAs and the three task lists
  b->grid = batch_lu_grid(b->Nmax);
  if (b->grid < 1) return bad(FEAST_ERR_CUDA);
  CostModel cm;
  if (b->opt.tune_cache) {
    // the autotuner's choice for this GPU, batch size and largest order
    char key[256];
    std::snprintf(key, sizeof(key), "%s|batch|count%d|nmax%lld|mixed", tune_gpu_name().c_str(), b->np,
                  tune_bucket(b->Nmax));
    std::map<std::string, double> t;
    if (tune_lookup(b->opt.tune_cache, key, t)) {
      if (t.count("grid")) b->grid = std::max(1, std::min(b->grid, (int)t["grid"]));
      if (t.count("cost_panel_row") && t["cost_panel_row"] > 0) cm.panel_row = t["cost_panel_row"];
      if (t.count("cost_update_tile") && t["cost_update_tile"] > 0) cm.update_tile = t["cost_update_tile"];
      b->tuned = 1;
    }
  }
  {
    std::vector<int> nbv, mv;
    for (const BMat& M : b->mats) {
      nbv.push_back(M.nb);
      mv.push_back(M.m);
    }
    auto upload = [&](bool lu, bool solve, int4** dst, int* cnt, double* mk) -> cudaError_t {
      const std::vector<int4> ord = plan_order(nbv, mv, lu, solve, b->grid, mk, cm, &b->lu_mask);
      *cnt = (int)ord.size();
      cudaError_t ee = dalloc(b, dst, ord.size() * sizeof(int4));
      if (ee != cudaSuccess) return ee;
      ee = cudaMemcpyAsync(*dst, ord.data(), ord.size() * sizeof(int4), cudaMemcpyHostToDevice, b->st);
      if (ee != cudaSuccess) return ee;
      return cudaStreamSynchronize(b->st);
    };
    double mk = 0.0;
    if ((e = upload(true, false, &b->t_factor, &b->n_factor, &b->makespan)) != cudaSuccess) return bad(cuda_status(e));
    if ((e = upload(true, true, &b->t_first, &b->n_first, &mk)) != cudaSuccess) return bad(cuda_status(e));
    if ((e = upload(false, true, &b->t_solve, &b->n_solve, &mk)) != cudaSuccess) return bad(cuda_status(e));
  }
  // S_i = z_i I - A_p
  if ((e = batch_form_shifted(b->A, b->d_pd, b->d_mats, b->dz, b->nmat, b->Nmax, b->S, b->st, b->np)) != cudaSuccess)
    return bad(cuda_status(e));
  // grouped CGS2: CTAs per block in proportion to n, within the resident limit
  {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int cap = nsm * std::max(1, orth_grp_ctas_per_sm());
    std::vector<int> G(b->np);
    long long tot = 0;
    for (int p = 0; p < b->np; ++p) {
      G[p] = std::max(1, std::min(16, (b->pd[p].n + 127) / 128));
      tot += G[p];
    }
    while (tot > cap) {
      tot = 0;
      for (int p = 0; p < b->np; ++p) {
        G[p] = std::max(1, G[p] / 2);
        tot += G[p];
      }
      if (tot > cap && *std::max_element(G.begin(), G.end()) == 1) return bad(FEAST_ERR_ARG);
    }
    std::vector<int> c0(b->np + 1, 0);
    for (int p = 0; p < b->np; ++p) c0[p + 1] = c0[p] + G[p];
    b->orth_total = c0[b->np];
    AL(b->orth_cta0, c0.size() * sizeof(int));
    AL(b->orth_part, (size_t)2 * b->orth_total * 256 * sizeof(double2));
    AL(b->orth_bars, (size_t)2 * b->np * sizeof(unsigned));
    if ((e = cudaMemcpyAsync(b->orth_cta0, c0.data(), c0.size() * sizeof(int), cudaMemcpyHostToDevice, b->st)) !=
        cudaSuccess)
      return bad(cuda_status(e));
  }
#undef AL
  // grouped GEMM call sites
  {
    feast_batch* B = b;
    feast_status s;
    if ((s = make_gg<double>(b, b->g_AQ, [B](const GrpDesc& d) {
           return zargs(d.n, d.m, d.n, B->A + d.onn, d.n, OP_N, B->Q + d.onm, d.n, OP_N, B->AQ + d.onm, d.n);
         })) != FEAST_OK) return bad(s);
    if ((s = make_gg<double>(b, b->g_Ahat, [B](const GrpDesc& d) {
           return zargs(d.m, d.m, d.n, B->Q + d.onm, d.n, OP_C, B->AQ + d.onm, d.n, OP_N, B->Ahat + d.omm, d.m);
         })) != FEAST_OK) return bad(s);
    if ((s = make_gg<double>(b, b->g_Bhat, [B](const GrpDesc& d) {
           return zargs(d.m, d.m, d.n, B->Q + d.onm, d.n, OP_C, B->Q + d.onm, d.n, OP_N, B->Bhat + d.omm, d.m);
         })) != FEAST_OK) return bad(s);
    if ((s = make_gg<float>(b, b->g_W32, [B](const GrpDesc& d) {
           GemmArgs<float> g;
           g.M = d.m; g.N = d.m; g.K = d.m;
           g.alpha = make_float2(1.f, 0.f);
           g.beta = make_float2(0.f, 0.f);
           g.A = B->Z32 + d.omm; g.lda = d.m;
           g.B = B->V32 + d.omm; g.ldb = d.m;
           g.C = B->W32 + d.omm; g.ldc = d.m;
           return g;
         })) != FEAST_OK) return bad(s);
    if ((s = make_gg<double>(b, b->g_Cm, [B](const GrpDesc& d) {
           return zargs(d.m, d.m, d.m, B->Binv + d.omm, d.m, OP_N, B->Ahat + d.omm, d.m, OP_N, B->Cm + d.omm, d.m);
         })) != FEAST_OK) return bad(s);
    if ((s = make_gg<double>(b, b->g_V, [B](const GrpDesc& d) {
           return zargs(d.m, d.m, d.m, B->Cm + d.omm, d.m, OP_N, B->W + d.omm, d.m, OP_N, B->V + d.omm, d.m);
         })) != FEAST_OK) return bad(s);
    if ((s = make_gg<double>(b, b->g_Zs, [B](const GrpDesc& d) {
           return zargs(d.m, d.m, d.m, B->Minv + d.omm, d.m, OP_N, B->V + d.omm, d.m, OP_N, B->Zs + d.omm, d.m);
         })) != FEAST_OK) return bad(s);
    if ((s = make_gg<double>(b, b->g_LUW, [B](const GrpDesc& d) {
           return zargs(d.m, d.m, d.m, B->W + d.omm, d.m, OP_N, B->Ahat + d.omm, d.m, OP_N, B->LUW + d.omm, d.m);
         })) != FEAST_OK) return bad(s);
    if ((s = make_gg<double>(b, b->g_X, [B](const GrpDesc& d) {
           return zargs(d.n, d.m, d.m, B->Q + d.onm, d.n, OP_N, B->W + d.omm, d.m, OP_N, B->X + d.onm, d.n);
         })) != FEAST_OK) return bad(s);
    if ((s = make_gg<double>(b, b->g_AX, [B](const GrpDesc& d) {
           return zargs(d.n, d.m, d.m, B->AQ + d.onm, d.n, OP_N, B->W + d.omm, d.m, OP_N, B->AX + d.onm, d.n);
         })) != FEAST_OK) return bad(s);
  }
  for (int p = 0; p < b->np; ++p) b->h_active[p] = 1;
  if ((e = cudaMemcpyAsync(b->active, b->h_active, b->np * sizeof(int), cudaMemcpyHostToDevice, b->st)) != cudaSuccess)
    return bad(cuda_status(e));
  if ((e = cudaStreamSynchronize(b->st)) != cudaSuccess) return bad(cuda_status(e));
  *out = b;
  return FEAST_OK;
}

feast_status feast_batch_factor(feast_batch* b) {
  if (!b) return FEAST_ERR_ARG;
  if (b->factored) {  // an explicit call factors again
    CK(batch_form_shifted(b->A, b->d_pd, b->d_mats, b->dz, b->nmat, b->Nmax, b->S, b->st, b->np));
    b->factored = false;
  }
  return ensure_factored_first(b, false);
}

feast_status feast_batch_filter(feast_batch* b, const feast_z* const* Y, feast_z* const* Q) {
  if (!b || !Y || !Q) return FEAST_ERR_ARG;
  for (int p = 0; p < b->np; ++p) {
    const GrpDesc& d = b->pd[p];
    if (!Y[p]) return FEAST_ERR_ARG;
    CK(cudaMemcpyAsync(b->Y + d.onm, Y[p], (size_t)d.n * d.m * sizeof(double2), cudaMemcpyDefault, b->st));
    host_coefs(b, p, nullptr);
    b->h_active[p] = 1;
  }
  CK(enqueue_inputs(b));
  CK(cudaMemcpyAsync(b->Rhs, b->Y, b->snm * sizeof(double2), cudaMemcpyDeviceToDevice, b->st));
  FS(ensure_factored_first(b, true));
  CK(batch_accumulate(b->Xs, b->d_mats, b->d_pd, b->np, b->nmax, b->mmax, b->coef, nullptr, nullptr, b->active, b->Q,
                      b->st));
  for (int p = 0; p < b->np; ++p) {
    const GrpDesc& d = b->pd[p];
    if (Q[p]) CK(cudaMemcpyAsync(Q[p], b->Q + d.onm, (size_t)d.n * d.m * sizeof(double2), cudaMemcpyDefault, b->st));
  }
  CK(cudaStreamSynchronize(b->st));
  return read_flags(b);
}

feast_status feast_batch_solve(feast_batch* b, const feast_z* const* Y0, feast_z* const* lambda, feast_z* const* X,
                               double* const* res, int* m_found, feast_batch_stats* stats) {
  if (!b || !Y0 || !lambda) return FEAST_ERR_ARG;
  feast_batch_stats st;
  std::memset(&st, 0, sizeof(st));
  st.grid = b->grid;
  st.tuned = b->tuned;
  st.tasks_factor = b->n_factor;
  st.plan_makespan_us = b->makespan;
  const bool was_factored = b->factored;
  // iteration 1: plain filter of Y0
  for (int p = 0; p < b->np; ++p) {
    const GrpDesc& d = b->pd[p];
    if (!Y0[p] || !lambda[p]) return FEAST_ERR_ARG;
    CK(cudaMemcpyAsync(b->Y + d.onm, Y0[p], (size_t)d.n * d.m * sizeof(double2), cudaMemcpyDefault, b->st));
    host_coefs(b, p, nullptr);
    b->h_active[p] = 1;
  }
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (b->opt.timing) {
    CK(cudaEventCreate(&t0));
    CK(cudaEventCreate(&t1));
    CK(cudaEventRecord(t0, b->st));
  }
  CK(cudaMemsetAsync(b->flags, 0, sizeof(unsigned), b->st));
  CK(enqueue_inputs(b));
  CK(cudaMemcpyAsync(b->Rhs, b->Y, b->snm * sizeof(double2), cudaMemcpyDeviceToDevice, b->st));
  feast_status fs = ensure_factored_first(b, true);
  if (fs != FEAST_OK) return fs;
  if (b->opt.timing && !was_factored) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
    st.t_factor_ms = ms;
  }
  CK(batch_accumulate(b->Xs, b->d_mats, b->d_pd, b->np, b->nmax, b->mmax, b->coef, nullptr, nullptr, b->active, b->Q,
                      b->st));
  CK(enqueue_rr(b));
  CK(cudaStreamSynchronize(b->st));
  FS(read_flags(b));
  if (b->opt.timing) {
    CK(cudaEventRecord(t1, b->st));
    CK(cudaEventSynchronize(t1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    st.t_iter_ms[0] = ms;
  }
  std::vector<int> prev(b->np, -1), conv(b->np, 0);
  std::vector<std::vector<int>> cand(b->np);
  int it = 1;
  for (;; ++it) {
    int nconv = 0;
    for (int p = 0; p < b->np; ++p) {
      if (conv[p]) { ++nconv; continue; }
      cand[p] = candidates(b, p);
      const int count = (int)cand[p].size();
      double mx = count ? 0.0 : INFINITY;
      for (int i : cand[p]) mx = std::max(mx, b->h_res[b->pd[p].om + i] / b->normA[p]);
      if (count > 0 && count == prev[p] && mx <= b->opt.tol) {
        conv[p] = 1;
        ++nconv;
      }
      prev[p] = count;
    }
    st.iters = it;
    st.converged = nconv;
    if (nconv == b->np || it >= b->opt.max_iter) break;
    // next iteration: residual form for the pencils still active
    for (int p = 0; p < b->np; ++p) {
      b->h_active[p] = conv[p] ? 0 : 1;
      if (!conv[p]) host_coefs(b, p, b->h_lam);
    }
    if (b->opt.timing) CK(cudaEventRecord(t0, b->st));
    bool done = false;
    if (!b->graph_failed) {
      if (!b->gexec) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
          cudaError_t e2 = enqueue_steady(b);
          e = cudaStreamEndCapture(b->st, &g);
          if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          cudaGetLastError();
          b->graph_err = (int)e;
          if (b->gexec) cudaGraphExecDestroy(b->gexec);
          b->gexec = nullptr;
          b->graph_failed = true;
        }
      }
      if (b->gexec) {
        CK(cudaGraphLaunch(b->gexec, b->st));
        done = true;
        st.graph = 1;
      }
    }
    if (!done) {
      st.graph = -b->graph_err;  // the capture's CUDA error, negated
      CK(enqueue_steady(b));
    }
    CK(cudaStreamSynchronize(b->st));
    FS(read_flags(b));
    if (b->opt.timing) {
      CK(cudaEventRecord(t1, b->st));
      CK(cudaEventSynchronize(t1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      if (it < 64) st.t_iter_ms[it] = ms;
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  // outputs: candidates first, sorted by (Re, Im)
  int nconv = 0;
  for (int p = 0; p < b->np; ++p) {
    const GrpDesc& d = b->pd[p];
    const int k = (int)cand[p].size();
    std::vector<double2> lam(d.m, make_double2(0.0, 0.0));
    std::vector<double> r(d.m, 0.0);
    for (int j = 0; j < k; ++j) {
      lam[j] = b->h_lam[d.om + cand[p][j]];
      r[j] = b->h_res[d.om + cand[p][j]] / b->normA[p];
    }
    CK(cudaMemcpyAsync(lambda[p], lam.data(), d.m * sizeof(double2), cudaMemcpyDefault, b->st));
    if (res && res[p]) CK(cudaMemcpyAsync(res[p], r.data(), d.m * sizeof(double), cudaMemcpyDefault, b->st));
    if (X && X[p]) {  // gather through the (now free) AQ arena, then one copy out
      double2* tmp = b->AQ + d.onm;
      for (int j = 0; j < d.m; ++j) {
        if (j < k)
          CK(cudaMemcpyAsync(tmp + (size_t)j * d.n, b->X + d.onm + (size_t)cand[p][j] * d.n, d.n * sizeof(double2),
                             cudaMemcpyDeviceToDevice, b->st));
        else
          CK(cudaMemsetAsync(tmp + (size_t)j * d.n, 0, d.n * sizeof(double2), b->st));
      }
      CK(cudaMemcpyAsync(X[p], tmp, (size_t)d.n * d.m * sizeof(double2), cudaMemcpyDefault, b->st));
    }
    if (m_found) m_found[p] = k;
    nconv += conv[p];
    CK(cudaStreamSynchronize(b->st));  // the host vectors go out of scope
  }
  if (stats) *stats = st;
  return nconv == b->np ? FEAST_OK : FEAST_ERR_NOCONV;
}

feast_status feast_batch_get_factor(feast_batch* b, int pencil, int shift, feast_z* LU, int32_t* perm) {
  if (!b || pencil < 0 || pencil >= b->np || shift < 0 || shift >= b->pd[pencil].q) return FEAST_ERR_ARG;
  if (!b->factored) return FEAST_ERR_STATE;
  const BMat& M = b->mats[b->pd[pencil].mat0 + shift];
  if (LU) {
    std::vector<float2> f((size_t)M.N * M.N);
    CK(cudaMemcpyAsync(f.data(), b->S + M.soff, f.size() * sizeof(float2), cudaMemcpyDeviceToHost, b->st));
    CK(cudaStreamSynchronize(b->st));
    std::vector<double2> d((size_t)M.n * M.n);
    for (int c = 0; c < M.n; ++c)
      for (int r = 0; r < M.n; ++r) {
        const float2 v = f[(size_t)r + (size_t)c * M.N];
        d[(size_t)r + (size_t)c * M.n] = make_double2(v.x, v.y);
      }
    CK(cudaMemcpyAsync(LU, d.data(), d.size() * sizeof(double2), cudaMemcpyDefault, b->st));
    CK(cudaStreamSynchronize(b->st));
  }
  if (perm) {
    CK(cudaMemcpyAsync(perm, b->perm + M.poff, M.n * sizeof(int32_t), cudaMemcpyDefault, b->st));
    CK(cudaStreamSynchronize(b->st));
  }
  return FEAST_OK;
}

feast_status feast_batch_tc_info(const feast_batch* b, int* tc_min, int* classes, int* matrices) {
  if (!b) return FEAST_ERR_ARG;
  if (tc_min) *tc_min = b->tc_min;
  if (classes) *classes = (int)b->tcc.size();
  if (matrices) {
    int m = 0;
    for (const auto& c : b->tcc) m += c.count;
    *matrices = m;
  }
  return FEAST_OK;
}

feast_status feast_batch_info(const feast_batch* b, int* count, int* nmat, int* grid, int* tasks_factor,
                              double* plan_makespan_us, double* lu_flops) {
  if (!b) return FEAST_ERR_ARG;
  if (count) *count = b->np;
  if (nmat) *nmat = b->nmat;
  if (grid) *grid = b->grid;
  if (tasks_factor) *tasks_factor = b->n_factor;
  if (plan_makespan_us) *plan_makespan_us = b->makespan;
  if (lu_flops) {
    double f = 0.0;
    for (const BMat& M : b->mats) f += 8.0 / 3.0 * (double)M.n * M.n * M.n;
    *lu_flops = f;
  }
  return FEAST_OK;
}

}  // extern "C"
