// The C ABI of include/feast_gb300.h: handle, quadrature (Sec. 3), the
// factor-once shifted LUs, the filter (Eq. Rasp / Eq. Lasp), Rayleigh-Ritz
// (Algorithms R-FEAST and Bi-FEAST) and the iteration with the Sec. 5
// candidate monitoring.  All arithmetic runs in the kernels of this library;
// the host only orders launches, computes the q quadrature nodes and weights
// and takes the per-iteration decisions from a few hundred bytes of results.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <new>
#include <type_traits>
#include <mutex>
#include <vector>

#include "../../include/feast_gb300.h"
#include "blas1.cuh"
#include "gemm.cuh"
#include "lu.cuh"
#include "norm2.cuh"
#include "small.cuh"
#include "ozaki.cuh"
#include "refine.cuh"
#include "tc_deep.cuh"
#include "tune.cuh"
#include "tc_update.cuh"

using zc = std::complex<double>;

static std::atomic<unsigned long long> g_launches{0};
void feast_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

inline double2 d2(zc v) { return make_double2(v.real(), v.imag()); }
inline zc zz(double2 v) { return zc(v.x, v.y); }

// ---------------------------------------------------------------- quadrature (host)
// Gauss-Legendre nodes on [-1, 1] by Newton's method on P_K (three-term
// recurrence), weights 2 / ((1 - t^2) P_K'(t)^2).
void gauss_legendre(int K, std::vector<double>& t, std::vector<double>& w) {
  t.assign(K, 0.0);
  w.assign(K, 0.0);
  for (int k = 1; k <= K; ++k) {
    double x = std::cos(M_PI * (k - 0.25) / (K + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int j = 2; j <= K; ++j) {
        const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      if (K == 1) { p0 = 1.0; p1 = x; }
      dp = K * (p0 - x * p1) / (1.0 - x * x);
      const double step = p1 / dp;
      x -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    double p0 = 1.0, p1 = x;
    for (int j = 2; j <= K; ++j) {
      const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    dp = K * (p0 - x * p1) / (1.0 - x * x);
    t[K - k] = x;  // increasing order
    w[K - k] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

// Eq. ellipses: phi(t) = c + R (cos th + i a sin th), th = pi/2 (1 + t), and dphi/dt.
zc ellipse(double t, zc c, double R, double a) {
  const double th = 0.5 * M_PI * (1.0 + t);
  return c + R * zc(std::cos(th), a * std::sin(th));
}
zc ellipse_d(double t, double R, double a) {
  const double th = 0.5 * M_PI * (1.0 + t);
  return R * 0.5 * M_PI * zc(-std::sin(th), a * std::cos(th));
}

// Eq. quadrature_for_pi: sigma_k = w_k phi'(t_k) / (2 pi i) over both folded halves (Eq. pi).
bool build_quadrature(const feast_contour& c, std::vector<zc>& z, std::vector<zc>& s) {
  const zc cc(c.center.re, c.center.im);
  const double R = c.R, a = c.aspect;
  const zc twopii(0.0, 2.0 * M_PI);
  z.clear();
  s.clear();
  if (c.rule == FEAST_RULE_CUSTOM) {
    if (!c.nodes || !c.weights || c.q_custom < 1) return false;
    for (int k = 0; k < c.q_custom; ++k) {
      z.push_back(zc(c.nodes[k].re, c.nodes[k].im));
      s.push_back(zc(c.weights[k].re, c.weights[k].im));
    }
    return true;
  }
  if (c.N_e < 1) return false;
  if (c.rule == FEAST_RULE_TRAP_MID) {
    const int q = c.N_e;
    for (int j = 0; j < q; ++j) {
      const double th = 2.0 * M_PI * (j + 0.5) / q;
      const double t = 2.0 * th / M_PI - 1.0;
      z.push_back(ellipse(t, cc, R, a));
      s.push_back((4.0 / q) * ellipse_d(t, R, a) / twopii);
    }
    return true;
  }
  std::vector<double> t, w;
  const int K = c.N_e;
  if (c.rule == FEAST_RULE_GAUSS) {
    gauss_legendre(K, t, w);
    for (int k = 0; k < K; ++k) { z.push_back(ellipse(t[k], cc, R, a)); s.push_back(w[k] * ellipse_d(t[k], R, a) / twopii); }
    for (int k = 0; k < K; ++k) {
      const double t2 = 2.0 - t[k];
      z.push_back(ellipse(t2, cc, R, a));
      s.push_back(w[k] * ellipse_d(t2, R, a) / twopii);
    }
    return true;
  }
  if (c.rule == FEAST_RULE_TRAP_END) {
    if (K < 2) return false;
    // endpoints of the two folded halves coincide pairwise: q = 2(K - 1) points,
    // angle-uniform on the closed contour, each with the full step h = 2/(K-1).
    const double h = 2.0 / (K - 1);
    for (int k = 0; k < K; ++k) {
      const double tk = -1.0 + h * k;
      z.push_back(ellipse(tk, cc, R, a));
      const double wk = (k == 0 || k == K - 1) ? h : h;  // h/2 + h/2 at the merged endpoints
      s.push_back(wk * ellipse_d(tk, R, a) / twopii);
    }
    for (int k = K - 2; k >= 1; --k) {
      const double t2 = 2.0 - (-1.0 + h * k);
      z.push_back(ellipse(t2, cc, R, a));
      s.push_back(h * ellipse_d(t2, R, a) / twopii);
    }
    return true;
  }
  return false;
}

}  // namespace

// Nodes and weights for the batched path (same rules as the handle).
bool feast_quadrature_host(const feast_contour& c, std::vector<zc>& z, std::vector<zc>& w) {
  return build_quadrature(c, z, w);
}

// ---------------------------------------------------------------- the handle
struct feast_handle {
  int64_t n = 0;
  int m0 = 0, q = 0;
  feast_options opt;
  cudaStream_t st = nullptr;
  bool hasB = false;
  zc center;
  double R = 1.0, aspect = 1.0;
  bool filter_domain = false;  // CUSTOM nodes without an ellipse: inside = |rho| >= 1/2
  std::vector<zc> z, w;        // the nodes this handle factors (a range of the contour's)
  std::vector<zc> z_all, w_all;  // every node of the contour
  int shift0 = 0;              // index of z[0] among z_all
  bool partial = false;        // a proper sub-range: the filter returns its subtree, without c0 Y
  AccTree tree;                // the summation tree of this handle's leaves
  double2* combine_buf = nullptr;  // feast_filter_combine's staging of the partial blocks
  std::vector<int> h_info;     // per shift: 0 or 1 + first zero-pivot column (last factorisation)
  // real pencils: each factored system k stands for node gidx[k] and, when
  // pidx[k] >= 0, for its conjugate node pidx[k] as well
  bool realp = false;
  std::vector<int> gidx, pidx;
  double2 *coefc = nullptr, *coefch = nullptr;
  double normA = 0.0;
  double2* At = nullptr;
  // ||A||_2 is estimated on its own stream at creation, beside the first
  // factorisation; norm_ev marks its end and the value is read on first use
  cudaStream_t norm_st = nullptr;
  // U's diagonal-block inverses for the blocked solves, made during the
  // factorisation on a low-priority stream as each outer block finishes
  cudaStream_t tinv_st = nullptr;
  cudaEvent_t tinv_fork = nullptr, tinv_join = nullptr;
  cudaEvent_t norm_ev = nullptr;
  bool norm_ready = false;
  bool factored = false;
  feast_status factor_status = FEAST_OK;
  int nb = 64, nbs = 64;
  // device data
  double2 *A = nullptr, *B = nullptr, *dz = nullptr, *dw = nullptr, *dmu = nullptr;
  void* S = nullptr;
  int32_t *piv = nullptr, *perm = nullptr, *pinv = nullptr, *mv = nullptr;
  int32_t* rowmaps = nullptr;  // complex64 LU: row maps of the deferred interchanges (blocks x q x n)
  int* info = nullptr;
  unsigned* flags = nullptr;
  void *Xs = nullptr, *Xsh = nullptr;
  double2 *Y = nullptr, *Yh = nullptr, *Rr = nullptr, *Rl = nullptr, *Q = nullptr, *Qh = nullptr;
  double2 *Qo = nullptr, *Qho = nullptr, *AQ = nullptr, *BQ = nullptr, *AhQ = nullptr, *BhQ = nullptr;
  double2 *X = nullptr, *Xl = nullptr, *AX = nullptr, *BX = nullptr, *AhX = nullptr, *BhX = nullptr;
  double2 *E = nullptr, *Eh = nullptr, *tmp = nullptr;
  double2 *Ahat = nullptr, *Bhat = nullptr, *LUB = nullptr, *Cm = nullptr, *Zs = nullptr, *V = nullptr;
  double2 *W = nullptr, *LUW = nullptr, *Minv = nullptr, *Binv = nullptr, *Zl = nullptr, *lam = nullptr, *dd = nullptr;
  double2 *coef = nullptr, *coefh = nullptr, *c0 = nullptr, *c0h = nullptr;
  int *pivB = nullptr, *pivW = nullptr, *useres = nullptr, *useresh = nullptr, *colidx = nullptr;
  int* gate = nullptr;  // device flag: the Newton-Schulz inverse of W missed its tolerance
  double *res = nullptr, *resl = nullptr, *xn = nullptr, *xln = nullptr, *scal = nullptr;
  void* orth_scratch = nullptr;
  void* orth_scratch2 = nullptr;       // the left block's orthonormalisation (side stream)
  void* pw_scratch = nullptr;
  TcStaging staging;
  DeepStaging deep;                    // the two-level LU's deep-update operands (and the right solves')
  DeepStaging deep_left;               // the left solves' own (they run beside the right ones)
  // -D^{-1} of every diagonal block (lu_outer columns) of the unit lower L and
  // of the upper U, for the far steps of the LU and the blocked solves
  float2 *TL = nullptr, *TU = nullptr;
  int nblk = 0;
  // the blocked solves' factor operands, staged once per factorisation (per side)
  void* pre[2] = {nullptr, nullptr};
  bool pre_valid[2] = {false, false};
  int lu_outer = 0;                    // its outer block (0: one-level LU)
  bool tuned = false;                  // launch parameters read from the tune cache
  std::vector<cudaEvent_t> deep_ev;
  int n_deep = 0;
  double t_deep = 0, deep_flops = 0, deep_bytes = 0;
  double upd_flops = 0, upd_bytes = 0;
  TcStaging staging_left;              // the left solves' own staging (they run beside the right ones)
  cudaStream_t side = nullptr;         // stream of the left solves
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr, join_ev2 = nullptr;
  void* schur_log = nullptr;
  double2* gemm_ws = nullptr;  // split-K partial products
  // mixed path: FP64-accurate n x n x m0 products on the BF16 tensor cores
  // (digits of A, A^H, B, B^H made on first use)
  bool use_oz = false;
  OzOperator oz[4];
  bool oz_ready[4] = {false, false, false, false};
  OzWork ozw;
  OzWork ozw2;           // the left side's products on the side stream (Bi-FEAST)
  bool has_ozw2 = false;
  float2* s32 = nullptr;       // FP32 Schur work: C, Z, V, W, lambda (m0 x m0 each)
  size_t gemm_ws_elems = 0;
  std::vector<void*> allocs;
  // classical refinement (options.max_refine > 0): per-shift stall records
  std::vector<int> h_refine_fail;
  double2 *X64r = nullptr, *X64l = nullptr, *r64 = nullptr, *T1 = nullptr, *T2 = nullptr, *ones = nullptr;
  double2* S64 = nullptr;  // one shifted matrix in FP64 (refactorisation of a stalled shift)
  int32_t *piv64 = nullptr, *perm64 = nullptr, *pinv64 = nullptr;
  int* info64 = nullptr;
  double *rnorm = nullptr, *Rn = nullptr;
  int refine_sweeps = 0, n_refactored = 0;
  // host mirrors of the last Rayleigh-Ritz step
  std::vector<zc> h_lam;
  std::vector<double> h_res, h_resl;
  bool have_rr = false;
  // timing
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> rr_ev;  // phase marks of the Rayleigh-Ritz step (timing)
  double t_factor = 0, t_filter = 0, t_rr = 0, t_update = 0;
  int n_update = 0;
  std::vector<cudaEvent_t> upd_ev;
};

namespace {

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

// Device memory of the handles comes from one stream-ordered pool per device
// that keeps the blocks it gets back (release threshold: unlimited), so a
// handle created after another was destroyed reuses that memory instead of
// paying for cudaMalloc and cudaFree again.  The pool holds the largest set of
// handles alive at once until the process exits.
cudaMemPool_t handle_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pl = nullptr;
    if (cudaMemPoolCreate(&pl, &props) != cudaSuccess) return nullptr;
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pl, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = pl;
  }
  return pools[dev];
}

template <typename P>
cudaError_t dalloc(feast_handle* h, P** p, size_t bytes) {
  void* v = nullptr;
  cudaMemPool_t pool = handle_pool();
  cudaError_t e = pool ? cudaMallocFromPoolAsync(&v, bytes ? bytes : 16, pool, h->st) : cudaErrorMemoryAllocation;
  if (e != cudaSuccess) return e;
  h->allocs.push_back(v);
  *p = reinterpret_cast<P*>(v);
  return cudaSuccess;
}

bool mixed(const feast_handle* h) { return h->opt.precision == FEAST_PREC_MIXED; }

template <typename T>
LuBatch<T> lu_view(feast_handle* h) {
  LuBatch<T> lu;
  lu.S = reinterpret_cast<cplx<T>*>(h->S);
  lu.ld = h->n;
  lu.stride = h->n * h->n;
  lu.n = (int)h->n;
  lu.q = h->q;
  lu.piv = h->piv;
  lu.perm = h->perm;
  lu.pinv = h->pinv;
  lu.info = h->info;
  lu.flags = h->flags;
  lu.mv = h->mv;
  lu.mv_panels = (int)((h->n + 63) / 64);
  if (std::is_same<T, float>::value) lu.rowmaps = h->rowmaps;
  if (std::is_same<T, float>::value && h->staging.Ast) lu.tc = &h->staging;
  lu.panel_cluster = std::is_same<T, float>::value && h->opt.panel_cluster >= 0;
  lu.cluster_min_rows = h->opt.panel_cluster > 0 ? h->opt.panel_cluster : 0;
  return lu;
}

cudaError_t zg(feast_handle* h, int opA, int opB, int M, int N, int K, zc alpha, const double2* A, long long lda,
               const double2* B, long long ldb, zc beta, double2* C, long long ldc) {
  GemmArgs<double> g;
  g.M = M; g.N = N; g.K = K; g.batch = 1;
  g.alpha = d2(alpha); g.beta = d2(beta);
  g.A = A; g.lda = lda; g.opA = opA;
  g.B = B; g.ldb = ldb; g.opB = opB;
  g.C = C; g.ldc = ldc;
  g.ws = h->gemm_ws;
  g.ws_elems = h->gemm_ws_elems;
  return gemm_batched<double>(g, h->st);
}

// C (n x cols, cols <= m0; default m0) = op(M) X for M = A (which = 0) or B (which = 1), op = OP_N or OP_C:
// on the emulated-FP64 tensor-core path when the handle uses it (the digits of
// op(M) are made on first use), else the DMMA GEMM.
// side = true: on the side stream with its own work area (the operator's
// digits are made on that stream at first use, and only that side uses them)
cudaError_t big_product(feast_handle* h, int which, int op, const double2* X, double2* C, int cols = -1,
                        bool side = false) {
  const int n = (int)h->n, m = cols < 0 ? h->m0 : cols;
  const double2* Mx = which == 0 ? h->A : h->B;
  if (!h->use_oz) return zg(h, op, OP_N, n, m, n, zc(1.0), Mx, n, X, n, zc(0.0), C, n);
  cudaStream_t s = side ? h->side : h->st;
  const int slot = which * 2 + (op == OP_C ? 1 : 0);
  if (!h->oz_ready[slot]) {
    void* base = nullptr;
    cudaError_t e = dalloc(h, &base, oz_operator_bytes(n));
    if (e != cudaSuccess) return e;
    oz_operator_layout(base, n, &h->oz[slot]);
    e = oz_make_operator(Mx, n, op, h->oz[slot], s);
    if (e != cudaSuccess) return e;
    h->oz_ready[slot] = true;
  }
  return oz_apply(h->oz[slot], X, n, m, C, n, side ? h->ozw2 : h->ozw, h->flags, s);
}

feast_status read_flags(feast_handle* h) {
  unsigned f = 0;
  CK(cudaMemcpyAsync(&f, h->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (f & DEVFLAG_TIMEOUT) return FEAST_ERR_DEVICE_TIMEOUT;
  if (f & DEVFLAG_NONFINITE) return FEAST_ERR_NONFINITE;
  return FEAST_OK;
}

void ev_mark(feast_handle* h, int i) {
  if (h->opt.timing) cudaEventRecord(h->ev[i], h->st);
}
double ev_ms(feast_handle* h, int a, int b) {
  if (!h->opt.timing) return 0.0;
  float ms = 0.f;
  cudaEventSynchronize(h->ev[b]);
  cudaEventElapsedTime(&ms, h->ev[a], h->ev[b]);
  return ms;
}

// ---------------------------------------------------------------- factorisation
// Trailing-update wrapper that brackets every launch with CUDA events (timing mode).
template <typename T>
struct UpdateTimer {
  TrailingUpdateFn<T> inner;
  void* ctx;
  feast_handle* h;
  int used;
  double ms;
  double flops = 0.0, bytes = 0.0;  // algorithmic work of the timed launches
};

template <typename T>
cudaError_t timed_update(const LuBatch<T>& lu, int k0, int w, int c0, int nc, bool stage, void* c, cudaStream_t s) {
  auto* t = reinterpret_cast<UpdateTimer<T>*>(c);
  if (lu.n - k0 - w <= 0 || nc <= 0) return cudaSuccess;
  if (stage) {  // the operands' staging (nc = 0: stage only) stays outside the timed kernel
    cudaError_t e = t->inner(lu, k0, w, c0, 0, true, t->ctx, s);
    if (e != cudaSuccess) return e;
  }
  if (2 * t->used + 1 >= (int)t->h->upd_ev.size()) return t->inner(lu, k0, w, c0, nc, false, t->ctx, s);
  cudaEventRecord(t->h->upd_ev[2 * t->used], s);
  cudaError_t e = t->inner(lu, k0, w, c0, nc, false, t->ctx, s);
  cudaEventRecord(t->h->upd_ev[2 * t->used + 1], s);
  ++t->used;
  const double M = (double)(lu.n - k0 - w);
  t->flops += 8.0 * lu.q * M * nc * w;
  t->bytes += 8.0 * lu.q * (2.0 * M * nc + M * w + (double)w * nc);
  return e;
}

// The far step of the two-level LU: every panel's interchanges on the columns
// beyond the block, then U12 = L11^{-1} A12 as one deep product with
// T = -L11^{-1} that overwrites A12 (timed with the deep updates).
cudaError_t far_hook(const LuBatch<float>& lu, int K0, int KB, void* c, cudaStream_t s) {
  feast_handle* h = reinterpret_cast<feast_handle*>(c);
  const int far0 = K0 + KB, nfar = lu.n - far0;
  if (nfar <= 0) return cudaSuccess;
  // the block's U part is final: -U_II^{-1} on the low-priority stream
  if (h->tinv_st) {
    cudaError_t e2 = cudaEventRecord(h->tinv_fork, s);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(h->tinv_st, h->tinv_fork, 0);
    if (e2 == cudaSuccess)
      e2 = block_inverse_negated(lu, true, KB, K0 / KB, 1, h->TU + (size_t)(K0 / KB) * lu.q * KB * KB, h->tinv_st);
    if (e2 != cudaSuccess) return e2;
  }
  cudaError_t e = block_swaps_far(lu, K0, KB, s);
  if (e != cudaSuccess) return e;
  // T = -L11^{-1} of this block, kept for the solves (block-major, all blocks)
  float2* T = h->TL + (size_t)(K0 / KB) * lu.q * KB * KB;
  e = block_inverse_negated(lu, false, KB, K0 / KB, 1, T, s);
  if (e != cudaSuccess) return e;
  const bool timing = h->opt.timing && 2 * h->n_deep + 1 < (int)h->deep_ev.size();
  if (timing) cudaEventRecord(h->deep_ev[2 * h->n_deep], s);
  e = tc_far_gemm(lu, K0, KB, T, h->deep, s);
  if (timing) {
    cudaEventRecord(h->deep_ev[2 * h->n_deep + 1], s);
    ++h->n_deep;
  }
  h->deep_flops += 8.0 * lu.q * (double)KB * KB * nfar;
  h->deep_bytes += 8.0 * lu.q * (2.0 * KB * nfar + (double)KB * KB + (double)KB * nfar);
  return e;
}

// The deep update of the two-level LU: operands staged, then the timed kernel.
cudaError_t deep_hook(const LuBatch<float>& lu, int K0, int KB, void* c, cudaStream_t s) {
  feast_handle* h = reinterpret_cast<feast_handle*>(c);
  cudaError_t e = tc_deep_stage(lu, K0, KB, h->deep, s);
  if (e != cudaSuccess) return e;
  const bool timing = h->opt.timing && 2 * h->n_deep + 1 < (int)h->deep_ev.size();
  if (timing) cudaEventRecord(h->deep_ev[2 * h->n_deep], s);
  e = tc_deep_run(lu, K0, KB, h->deep, s);
  if (timing) {
    cudaEventRecord(h->deep_ev[2 * h->n_deep + 1], s);
    ++h->n_deep;
  }
  h->deep_flops += tc_deep_flops(lu.n, lu.q, K0, KB);
  h->deep_bytes += tc_deep_bytes(lu.n, lu.q, K0, KB);
  return e;
}

template <typename T>
feast_status factor_impl(feast_handle* h) {
  LuBatch<T> lu = lu_view<T>(h);
  h->pre_valid[0] = h->pre_valid[1] = false;  // the solves' staged operands belong to the old factors
  CK(form_shifted<T>(h->A, h->n, h->hasB ? h->B : nullptr, h->n, h->dz, h->q, (int)h->n, lu.S, lu.stride, h->st));
  TrailingUpdateFn<T> upd = nullptr;
  void* ctx = nullptr;
  select_trailing_update<T>(&upd, &ctx, &h->staging);
  if (!upd) upd = default_trailing_update<T>;
  // complex64 with staging: the tensor-core update (its operands always fit the
  // staging sized for n and q) solves U12 while staging it
  lu.u12_in_stage = std::is_same<T, float>::value && h->staging.Ast != nullptr;
  UpdateTimer<T> timer{upd, ctx, h, 0, 0.0, 0.0, 0.0};
  if (h->opt.timing) {
    const int panels = (int)((h->n + h->nb - 1) / h->nb);
    while ((int)h->upd_ev.size() < 4 * panels) {  // two update launches per step
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      h->upd_ev.push_back(e);
    }
  }
  h->n_deep = 0;
  h->t_deep = h->deep_flops = h->deep_bytes = 0.0;
  TrailingUpdateFn<T> use_upd = h->opt.timing ? timed_update<T> : upd;
  void* use_ctx = h->opt.timing ? (void*)&timer : ctx;
  if constexpr (std::is_same<T, float>::value) {
    if (h->lu_outer > 0) {
      if (h->opt.timing) {
        const int blocks = (int)((h->n + h->lu_outer - 1) / h->lu_outer);
        while ((int)h->deep_ev.size() < 4 * blocks + 2) {  // far and deep products per block
          cudaEvent_t e;
          CK(cudaEventCreate(&e));
          h->deep_ev.push_back(e);
        }
      }
      CK(lu_factor_two_level(lu, 64, h->lu_outer, use_upd, use_ctx, far_hook, deep_hook, h, h->st));
      // -D^{-1} of the last L block (the far steps made the others) and of every
      // U block, for the blocked solves
      const int KB = h->lu_outer;
      CK(block_inverse_negated(lu, false, KB, h->nblk - 1, 1, h->TL + (size_t)(h->nblk - 1) * h->q * KB * KB,
                                  h->st));
      if (h->tinv_st) {  // the far steps started the other blocks' U inverses on their stream
        CK(block_inverse_negated(lu, true, KB, h->nblk - 1, 1, h->TU + (size_t)(h->nblk - 1) * h->q * KB * KB,
                                    h->st));
        CK(cudaEventRecord(h->tinv_join, h->tinv_st));
        CK(cudaStreamWaitEvent(h->st, h->tinv_join, 0));
      } else {
        CK(block_inverse_negated(lu, true, KB, 0, h->nblk, h->TU, h->st));
      }
    } else {
      CK(lu_factor_batched<T>(lu, h->nb, use_upd, use_ctx, h->st));
    }
  } else {
    CK(lu_factor_batched<T>(lu, h->nb, use_upd, use_ctx, h->st));
  }
  std::vector<int> info(h->q);
  CK(cudaMemcpyAsync(info.data(), h->info, sizeof(int) * h->q, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  h->t_update = 0.0;
  h->n_update = timer.used;
  h->upd_flops = timer.flops;
  h->upd_bytes = timer.bytes;
  for (int i = 0; i < h->n_deep; ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->deep_ev[2 * i], h->deep_ev[2 * i + 1]);
    h->t_deep += ms;
  }
  for (int i = 0; i < timer.used; ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->upd_ev[2 * i], h->upd_ev[2 * i + 1]);
    h->t_update += ms;
  }
  h->h_info = info;
  feast_status fs = read_flags(h);
  if (fs == FEAST_ERR_NONFINITE) return fs;
  for (int k = 0; k < h->q; ++k)
    if (info[k] != 0) return FEAST_ERR_SINGULAR_SHIFT;
  return fs;
}

feast_status ensure_factored(feast_handle* h) {
  if (h->factored) return h->factor_status;
  ev_mark(h, 0);
  feast_status s = mixed(h) ? factor_impl<float>(h) : factor_impl<double>(h);
  ev_mark(h, 1);
  h->t_factor = ev_ms(h, 0, 1);
  h->factored = true;
  h->factor_status = s;
  return s;
}

// ---------------------------------------------------------------- filter
// Classical refinement of all q solves of one side (MIXED, max_refine > 0).
// X64 starts from the complex64 solutions in Xs; each sweep forms every
// shift's FP64 residual r_k = R - S_k X_k (right: S_k = phi_k B - A; left:
// S_k^H = conj(phi_k) B^H - A^H; the n x n x m products on the emulated-FP64
// tensor-core path) and, unless every shift already has max_j ||r_kj|| /
// ||R_j|| <= refine_tol, solves S_k d_k = r_k with the complex64 factor and
// adds d_k in FP64.  A shift still above the tolerance after max_refine sweeps
// (its refinement stalled) is refactored in FP64 on the GPU and solved again;
// if even that misses the tolerance the call returns FEAST_ERR_REFINE_NOCONV.
feast_status refine_side(feast_handle* h, int side, const double2* R, float2* Xs, const int32_t* rowmap,
                         double2* X64) {
  const int n = (int)h->n, m = h->m0, q = h->q;
  const size_t nm = (size_t)n * m;
  LuBatch<float> lu = lu_view<float>(h);
  if (side == 1) lu.tc = h->staging_left.Ast ? &h->staging_left : nullptr;
  CK(refine_widen(Xs, q, n, m, rowmap, X64, false, h->st));
  CK(column_norms(R, n, m, h->Rn, h->st));
  std::vector<double> rn(m), nr((size_t)q * m), prev(q, INFINITY), rel(q, INFINITY);
  CK(cudaMemcpyAsync(rn.data(), h->Rn, m * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  const double tau = h->opt.refine_tol;
  auto residuals = [&](int k) -> cudaError_t {
    double2* xk = X64 + (size_t)k * nm;
    cudaError_t e = big_product(h, 0, side ? OP_C : OP_N, xk, h->T1);
    const double2* T2 = xk;
    if (e == cudaSuccess && h->hasB) {
      e = big_product(h, 1, side ? OP_C : OP_N, xk, h->T2);
      T2 = h->T2;
    }
    const zc zk = side ? std::conj(h->z[k]) : h->z[k];
    if (e == cudaSuccess) e = refine_residual(R, h->T1, T2, d2(zk), n, m, h->r64 + (size_t)k * nm, h->rnorm + (size_t)k * m, h->st);
    return e;
  };
  auto measure = [&]() -> feast_status {
    for (int k = 0; k < q; ++k) CK(residuals(k));
    CK(cudaMemcpyAsync(nr.data(), h->rnorm, nr.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    for (int k = 0; k < q; ++k) {
      double r = 0.0;
      for (int j = 0; j < m; ++j) r = std::max(r, rn[j] > 0 ? nr[(size_t)k * m + j] / rn[j] : nr[(size_t)k * m + j]);
      rel[k] = std::isfinite(r) ? r : INFINITY;
    }
    return FEAST_OK;
  };
  feast_status st;
  int sweeps = 0;
  for (;;) {
    if ((st = measure()) != FEAST_OK) return st;
    bool all = true;
    for (int k = 0; k < q; ++k) all = all && rel[k] <= tau;
    if (all || sweeps == h->opt.max_refine) break;
    // corrections for every shift from its FP64 residual, one batched solve
    CK(refine_gather(h->r64, h->perm, Xs, q, n, m, side == 0, h->st));
    CK(lu_solve_batched<float>(lu, side, Xs, m, h->nbs, h->st));
    CK(refine_widen(Xs, q, n, m, rowmap, X64, true, h->st));
    prev = rel;
    ++sweeps;
  }
  h->refine_sweeps = std::max(h->refine_sweeps, sweeps);
  // shifts whose refinement did not reach the tolerance: FP64 factor and solve
  for (int k = 0; k < q; ++k) {
    if (rel[k] <= tau) continue;
    if (!h->S64) {
      CK(dalloc(h, &h->S64, (size_t)n * n * sizeof(double2)));
      CK(dalloc(h, &h->piv64, (size_t)n * sizeof(int32_t)));
      CK(dalloc(h, &h->perm64, (size_t)n * sizeof(int32_t)));
      CK(dalloc(h, &h->pinv64, (size_t)n * sizeof(int32_t)));
      CK(dalloc(h, &h->info64, 64));
    }
    LuBatch<double> l1;
    l1.S = h->S64; l1.ld = n; l1.stride = (long long)n * n; l1.n = n; l1.q = 1;
    l1.piv = h->piv64; l1.perm = h->perm64; l1.pinv = h->pinv64; l1.info = h->info64; l1.flags = h->flags;
    CK(form_shifted<double>(h->A, h->n, h->hasB ? h->B : nullptr, h->n, h->dz + k, 1, n, h->S64, l1.stride, h->st));
    CK(lu_factor_batched<double>(l1, 64, nullptr, nullptr, h->st));
    double2* X1 = h->r64 + (size_t)k * nm;  // this shift's residual slot as the solve's work block
    CK(rows_gather<double>(l1, R, X1, m, side == 0, h->st));
    CK(lu_solve_batched<double>(l1, side, X1, m, h->nbs, h->st));
    CK(accumulate<double>(X1, acc_tree_single(1), n, m, h->ones, nullptr, nullptr, side ? h->pinv64 : nullptr,
                          X64 + (size_t)k * nm, h->st));
    ++h->n_refactored;
    CK(residuals(k));
    std::vector<double> nk(m);
    CK(cudaMemcpyAsync(nk.data(), h->rnorm + (size_t)k * m, m * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    double r = 0.0;
    for (int j = 0; j < m; ++j) r = std::max(r, rn[j] > 0 ? nk[j] / rn[j] : nk[j]);
    if ((int)h->h_refine_fail.size() < q) h->h_refine_fail.assign(q, 0);
    if (!(r <= tau)) h->h_refine_fail[k] = sweeps + 1;
  }
  for (int v : h->h_refine_fail)
    if (v) return FEAST_ERR_REFINE_NOCONV;
  return FEAST_OK;
}

feast_status refine_alloc(feast_handle* h) {
  if (h->X64r) return FEAST_OK;
  const size_t nm = (size_t)h->n * h->m0;
  CK(dalloc(h, &h->X64r, (size_t)h->q * nm * sizeof(double2)));
  if (h->opt.algo == FEAST_ALGO_BI && !h->opt.symmetric) CK(dalloc(h, &h->X64l, (size_t)h->q * nm * sizeof(double2)));
  CK(dalloc(h, &h->r64, (size_t)h->q * nm * sizeof(double2)));
  CK(dalloc(h, &h->T1, nm * sizeof(double2)));
  CK(dalloc(h, &h->T2, nm * sizeof(double2)));
  CK(dalloc(h, &h->rnorm, (size_t)h->q * h->m0 * sizeof(double)));
  CK(dalloc(h, &h->Rn, (size_t)h->m0 * sizeof(double)));
  CK(dalloc(h, &h->ones, (size_t)h->m0 * sizeof(double2)));
  std::vector<double2> one(h->m0, make_double2(1.0, 0.0));
  CK(cudaMemcpyAsync(h->ones, one.data(), h->m0 * sizeof(double2), cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  return FEAST_OK;
}

// Right: Q = c0 .* Y + sum_k coef_k .* S_k^{-1} R;  left: Qh = c0h .* Yh + sum_k coefh_k .* S_k^{-H} Rh
// The filter's triangular solves of all shifts: with the two-level factors the
// blocked deep-K form (diagonal blocks through -D^{-1}, K = lu_outer updates),
// else the 64-row block form.
template <typename T>
cudaError_t solve_all(feast_handle* h, const LuBatch<T>& lu, int side, cplx<T>* X, int m, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    const DeepStaging& st = side == 0 ? h->deep : h->deep_left;
    if (h->opt.deep_solves >= 0 && h->lu_outer > 0 && h->TU && st.Ast && m <= st.cols_max)
      return tc_solve_deep(lu, side, X, m, h->lu_outer, h->TL, h->TU, st, s, h->pre_valid[side] ? h->pre[side] : nullptr);
  }
  return lu_solve_batched<T>(lu, side, X, m, h->nbs, s);
}

template <typename T>
feast_status filter_impl(feast_handle* h, const double2* R, const double2* Yc0, bool use_c0, const double2* Rh,
                         const double2* Yhc0, double2* Qout, double2* Qhout) {
  LuBatch<T> lu = lu_view<T>(h);
  const int n = (int)h->n, m = h->m0;
  cplx<T>* Xs = reinterpret_cast<cplx<T>*>(h->Xs);
  const bool split = Rh && !h->opt.symmetric && h->side;
  // the first filter after a factorisation stages the solves' factor operands,
  // each side on the stream of its own solves (the two stagings side by side)
  bool stage_right = false, stage_left = false;
  if constexpr (std::is_same<T, float>::value) {
    const bool deep = h->opt.deep_solves >= 0 && h->lu_outer > 0 && h->TU;
    stage_left = deep && Rh && !h->opt.symmetric && h->pre[1] && !h->pre_valid[1];
    stage_right = deep && h->pre[0] && !h->pre_valid[0];
  }
  if (split) CK(cudaEventRecord(h->fork_ev, h->st));  // the left solves start from here
  if constexpr (std::is_same<T, float>::value) {
    if (stage_right) {
      CK(tc_solve_prestage(lu, 0, h->lu_outer, h->TL, h->TU, h->pre[0], h->st));
      h->pre_valid[0] = true;
    }
  }
  const bool add_c0 = use_c0 && !h->partial;  // a partial handle returns its subtree alone
  const int ms = h->realp ? 2 * m : m;          // real pencils: [R, conj(R)] per factor
  CK(rows_gather<T>(lu, R, Xs, m, true, h->st, h->realp));
  CK(solve_all<T>(h, lu, 0, Xs, ms, h->st));
  const bool refine = std::is_same<T, float>::value && h->opt.max_refine > 0;
  feast_status rstat = FEAST_OK;
  if (refine) {
    // classical refinement: FP64 solutions per shift, then the accumulation of those
    h->h_refine_fail.assign(h->q, 0);
    h->refine_sweeps = h->n_refactored = 0;
    feast_status st2;
    if ((st2 = refine_alloc(h)) != FEAST_OK) return st2;
    rstat = refine_side(h, 0, R, reinterpret_cast<float2*>(Xs), nullptr, h->X64r);
    if (rstat != FEAST_OK && rstat != FEAST_ERR_REFINE_NOCONV) return rstat;
    CK(accumulate<double>(h->X64r, h->tree, n, m, h->coef, add_c0 ? h->c0 : nullptr, add_c0 ? Yc0 : nullptr, nullptr,
                          Qout, h->st));
    if (Rh && !h->opt.symmetric) {
      cplx<T>* Xsh = reinterpret_cast<cplx<T>*>(h->Xsh);
      LuBatch<T> lul = lu;
      if (std::is_same<T, float>::value) lul.tc = h->staging_left.Ast ? &h->staging_left : nullptr;
      CK(rows_gather<T>(lul, Rh, Xsh, m, false, h->st));
      CK(lu_solve_batched<T>(lul, 1, Xsh, m, h->nbs, h->st));
      feast_status r2 = refine_side(h, 1, Rh, reinterpret_cast<float2*>(Xsh), lu.pinv, h->X64l);
      if (r2 != FEAST_OK && r2 != FEAST_ERR_REFINE_NOCONV) return r2;
      if (r2 != FEAST_OK) rstat = r2;
      CK(accumulate<double>(h->X64l, h->tree, n, m, h->coefh, add_c0 ? h->c0h : nullptr, add_c0 ? Yhc0 : nullptr,
                            nullptr, Qhout, h->st));
    } else if (Rh) {
      CK(conj_copy(Qout, Qhout, (size_t)n * m, h->st));
    }
    return rstat;
  }
  if (h->realp) {
    CK(accumulate_conj_pairs<T>(Xs, h->q, n, m, h->coef, h->coefc, add_c0 ? h->c0 : nullptr,
                                add_c0 ? Yc0 : nullptr, nullptr, Qout, h->st));
  } else {
    CK(accumulate<T>(Xs, h->tree, n, m, h->coef, add_c0 ? h->c0 : nullptr, add_c0 ? Yc0 : nullptr, nullptr, Qout,
                     h->st));
  }
  if (Rh && h->opt.symmetric) {
    // complex symmetric pencil: (phi B - A)^{-H} conj(V) = conj((phi B - A)^{-1} V),
    // and the left inputs are the conjugates of the right ones
    CK(conj_copy(Qout, Qhout, (size_t)n * m, h->st));
  } else if (Rh) {
    // the left solves (U^H, then L^H) run on the side stream, beside the right
    // ones: both are chains of small block steps that leave most SMs idle
    cplx<T>* Xsh = reinterpret_cast<cplx<T>*>(h->Xsh);
    LuBatch<T> lul = lu;
    if (std::is_same<T, float>::value) lul.tc = h->staging_left.Ast ? &h->staging_left : nullptr;
    cudaStream_t ls = split ? h->side : h->st;
    if (split) CK(cudaStreamWaitEvent(h->side, h->fork_ev, 0));
    if constexpr (std::is_same<T, float>::value) {
      if (stage_left) {
        CK(tc_solve_prestage(lu, 1, h->lu_outer, h->TL, h->TU, h->pre[1], ls));
        h->pre_valid[1] = true;
      }
    }
    CK(rows_gather<T>(lul, Rh, Xsh, m, false, ls, h->realp));
    CK(solve_all<T>(h, lul, 1, Xsh, ms, ls));
    if (h->realp) {
      CK(accumulate_conj_pairs<T>(Xsh, h->q, n, m, h->coefh, h->coefch, add_c0 ? h->c0h : nullptr,
                                  add_c0 ? Yhc0 : nullptr, lu.pinv, Qhout, ls));
    } else {
      CK(accumulate<T>(Xsh, h->tree, n, m, h->coefh, add_c0 ? h->c0h : nullptr, add_c0 ? Yhc0 : nullptr, lu.pinv,
                       Qhout, ls));
    }
    if (split) {
      CK(cudaEventRecord(h->join_ev, h->side));
      CK(cudaStreamWaitEvent(h->st, h->join_ev, 0));
    }
  }
  return FEAST_OK;
}

// Host-side coefficients.  Plain form: coef_k = sigma_k.  Residual form for
// column i (Ritz value theta_i not on a node):
//   S_k^{-1} B x = x / (phi_k - theta) + S_k^{-1} (A x - theta B x) / (phi_k - theta)
// so coef_k,i = sigma_k / (phi_k - theta_i) and c0_i = sum_k coef_k,i = rho(theta_i).
feast_status upload_coefs(feast_handle* h, const zc* theta, std::vector<int>* use_out) {
  const int q = h->q, m = h->m0, qa = (int)h->z_all.size();
  std::vector<double2> coef((size_t)q * m), coefh((size_t)q * m), c0(m), c0h(m);
  std::vector<double2> coefc_v(h->realp ? (size_t)q * m : 0), coefch_v(h->realp ? (size_t)q * m : 0);
  std::vector<int> use(m, 0);
  for (int i = 0; i < m; ++i) {
    bool u = false;
    if (theta && std::isfinite(theta[i].real()) && std::isfinite(theta[i].imag())) {
      double dmin = 1e300;
      for (int k = 0; k < qa; ++k) dmin = std::min(dmin, std::abs(h->z_all[k] - theta[i]));
      // The identity holds for every theta != phi_k; for a converged pair the
      // initial iterate x / (phi_k - theta) is already close to the solution, so
      // a Ritz value next to a node brings no cancellation.  Only a value on top
      // of a node (division by ~0) takes the plain right-hand side.  Every node
      // of the contour decides, so that the handles of a shift partition agree.
      u = dmin >= 1e-10 * h->R;
    }
    use[i] = u;
    for (int k = 0; k < q; ++k) {
      const int kg = h->gidx[k];
      const zc g = u ? h->w_all[kg] / (h->z_all[kg] - theta[i]) : h->w_all[kg];
      coef[(size_t)k * m + i] = d2(g);
      coefh[(size_t)k * m + i] = d2(std::conj(g));
      if (h->realp) {
        const int kp = h->pidx[k];
        const zc gp = kp < 0 ? zc(0.0) : (u ? h->w_all[kp] / (h->z_all[kp] - theta[i]) : h->w_all[kp]);
        coefc_v[(size_t)k * m + i] = d2(gp);
        coefch_v[(size_t)k * m + i] = d2(std::conj(gp));
      }
    }
    zc acc = 0.0;  // c0 = rho(theta) over all the contour's nodes
    if (u)
      for (int k = 0; k < qa; ++k) acc += h->w_all[k] / (h->z_all[k] - theta[i]);
    c0[i] = d2(u ? acc : zc(0.0));
    c0h[i] = d2(u ? std::conj(acc) : zc(0.0));
  }
  CK(cudaMemcpyAsync(h->coef, coef.data(), coef.size() * sizeof(double2), cudaMemcpyHostToDevice, h->st));
  if (h->realp) {
    CK(cudaMemcpyAsync(h->coefc, coefc_v.data(), coefc_v.size() * sizeof(double2), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->coefch, coefch_v.data(), coefch_v.size() * sizeof(double2), cudaMemcpyHostToDevice,
                       h->st));
  }
  CK(cudaMemcpyAsync(h->coefh, coefh.data(), coefh.size() * sizeof(double2), cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(h->c0, c0.data(), c0.size() * sizeof(double2), cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(h->c0h, c0h.data(), c0h.size() * sizeof(double2), cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(h->useres, use.data(), m * sizeof(int), cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));  // the host vectors go out of scope
  if (use_out) *use_out = use;
  return FEAST_OK;
}

feast_status run_filter(feast_handle* h, const double2* R, const double2* Yc0, bool use_c0, const double2* Rh,
                        const double2* Yhc0) {
  return mixed(h) ? filter_impl<float>(h, R, Yc0, use_c0, Rh, Yhc0, h->Q, h->Qh)
                  : filter_impl<double>(h, R, Yc0, use_c0, Rh, Yhc0, h->Q, h->Qh);
}

// ---------------------------------------------------------------- Rayleigh-Ritz
feast_status rr_impl(feast_handle* h, const double2* Qin, const double2* Qhin) {
  const int n = (int)h->n, m = h->m0;
  const bool bi = Qhin != nullptr;
  if (h->opt.timing) {
    while (h->rr_ev.size() < 9) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      h->rr_ev.push_back(e);
    }
  }
  auto mark = [&](int i) {
    if (h->opt.timing) cudaEventRecord(h->rr_ev[i], h->st);
  };
  mark(0);
  const size_t blk = (size_t)n * m * sizeof(double2);
  const zc one(1.0), zero(0.0);
  CK(cudaMemsetAsync(h->flags, 0, sizeof(unsigned), h->st));
  CK(cudaMemcpyAsync(h->Qo, Qin, blk, cudaMemcpyDeviceToDevice, h->st));
  if (bi) CK(cudaMemcpyAsync(h->Qho, Qhin, blk, cudaMemcpyDeviceToDevice, h->st));
  // the left block is orthonormalised on the side stream, beside the right one
  // and the products A Q, B Q (the two latency-bound kernels share the SMs)
  const bool par = bi && h->side && h->orth_scratch2;
  // with its own work area the side stream also forms A^H Qhat and B^H Qhat,
  // hidden behind the reduced problem (one-CTA kernels) on the main stream
  const bool side_products = par && !h->opt.symmetric && h->use_oz && h->has_ozw2;
  if (par) {
    CK(cudaEventRecord(h->fork_ev, h->st));
    CK(cudaStreamWaitEvent(h->side, h->fork_ev, 0));
    CK(orth_cgs2(h->Qho, n, m, h->orth_scratch2, h->flags, h->side, 0, true));
    CK(cudaEventRecord(h->join_ev, h->side));
    if (side_products) {
      CK(big_product(h, 0, OP_C, h->Qho, h->AhQ, -1, true));
      if (h->hasB) CK(big_product(h, 1, OP_C, h->Qho, h->BhQ, -1, true));
      CK(cudaEventRecord(h->join_ev2, h->side));
    }
  }
  // the bases need the span exactly and orthonormality only to FP32 level: the
  // reduced problem forms and inverts their Gram matrix Bhat in FP64 below
  CK(orth_cgs2(h->Qo, n, m, h->orth_scratch, h->flags, h->st, 0, true));
  if (bi && !par) CK(orth_cgs2(h->Qho, n, m, h->orth_scratch, h->flags, h->st, 0, true));
  mark(1);
  const double2* Vb = bi ? h->Qho : h->Qo;
  CK(big_product(h, 0, OP_N, h->Qo, h->AQ));
  const double2* BQp = h->Qo;
  if (h->hasB) {
    CK(big_product(h, 1, OP_N, h->Qo, h->BQ));
    BQp = h->BQ;
  }
  if (par) CK(cudaStreamWaitEvent(h->st, h->join_ev, 0));
  mark(2);
  CK(zg(h, OP_C, OP_N, m, m, n, one, Vb, n, h->AQ, n, zero, h->Ahat, m));
  CK(zg(h, OP_C, OP_N, m, m, n, one, Vb, n, BQp, n, zero, h->Bhat, m));
  mark(3);
  // reduced problem: C = B^{-1} A^, Schur form, eigenvectors
  const size_t sm = (size_t)m * m * sizeof(double2);
  // X <- X (2I - M X): quadratic convergence to M^{-1} (DMMA products; LUW, Zs scratch)
  auto newton_schulz = [&](const double2* Mx, double2* X, int steps) -> cudaError_t {
    for (int it = 0; it < steps; ++it) {
      cudaError_t e = set_identity(h->LUW, m, h->st);
      if (e == cudaSuccess) e = zg(h, OP_N, OP_N, m, m, m, zc(-1.0), Mx, m, X, m, zc(2.0), h->LUW, m);
      if (e == cudaSuccess) e = zg(h, OP_N, OP_N, m, m, m, one, X, m, h->LUW, m, zero, h->Zs, m);
      if (e == cudaSuccess) e = cudaMemcpyAsync(X, h->Zs, sm, cudaMemcpyDeviceToDevice, h->st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  // guard: when ||M X - I|| > 1e-12 (an ill-conditioned M, or a start too far
  // off for the iteration) the inverse is recomputed by LU on the device
  auto inverse_guard = [&](const double2* Mx, double2* X, double2* LU, int* piv) -> cudaError_t {
    cudaError_t e = zg(h, OP_N, OP_N, m, m, m, one, Mx, m, X, m, zero, h->Zs, m);
    if (e == cudaSuccess) e = inverse_check(h->Zs, m, 1e-12, h->gate, h->st);
    if (e == cudaSuccess) e = small_inverse_gated(Mx, LU, piv, X, m, h->flags, h->gate, h->st);
    return e;
  };
  // B^^{-1}: FP32 Gauss-Jordan start, three Newton-Schulz steps, checked
  CK(gj_inverse32(h->Bhat, m, h->Binv, h->st));
  CK(newton_schulz(h->Bhat, h->Binv, 3));
  CK(inverse_guard(h->Bhat, h->Binv, h->LUB, h->pivB));
  CK(zg(h, OP_N, OP_N, m, m, m, one, h->Binv, m, h->Ahat, m, zero, h->Cm, m));
  mark(4);
  // Schur form and eigenvectors in FP32, then two FP64 refinement sweeps:
  // E = W^{-1} C W (DMMA products), lam = diag(E), W <- W (I + Delta).
  {
    const size_t mm = (size_t)m * m;
    float2* C32 = h->s32;
    float2* Z32 = C32 + mm;
    float2* V32 = Z32 + mm;
    float2* W32 = V32 + mm;
    float2* lam32 = W32 + mm;
    CK(to_c64(h->Cm, C32, mm, h->st));
    CK(small_schur<float>(C32, Z32, lam32, m, h->flags, h->schur_log, h->st));
    CK(small_trevc<float>(C32, V32, m, h->st));
    GemmArgs<float> g32;
    g32.M = m; g32.N = m; g32.K = m;
    g32.alpha = make_float2(1.f, 0.f);
    g32.beta = make_float2(0.f, 0.f);
    g32.A = Z32; g32.lda = m; g32.B = V32; g32.ldb = m; g32.C = W32; g32.ldc = m;
    CK(gemm_batched<float>(g32, h->st));
    CK(to_c128(W32, h->W, mm, h->st));
    // W^{-1} = V^{-1} Z^H from the Schur factors (FP32), made FP64-accurate by
    // Newton-Schulz steps X <- X (2I - W X) (quadratic convergence, DMMA products)
    CK(small_triu_inv<float>(V32, C32, m, h->st));
    GemmArgs<float> gi = g32;
    gi.A = C32; gi.B = Z32; gi.opB = OP_C; gi.C = W32;
    CK(gemm_batched<float>(gi, h->st));
    CK(to_c128(W32, h->Minv, mm, h->st));
    CK(newton_schulz(h->W, h->Minv, 3));
    CK(inverse_guard(h->W, h->Minv, h->LUW, h->pivW));
    mark(5);
    for (int sweep = 0; sweep < 2; ++sweep) {
      CK(zg(h, OP_N, OP_N, m, m, m, one, h->Cm, m, h->W, m, zero, h->V, m));
      CK(zg(h, OP_N, OP_N, m, m, m, one, h->Minv, m, h->V, m, zero, h->Zs, m));
      CK(eig_refine_step(h->Zs, h->Ahat, h->lam, m, h->st));
      CK(zg(h, OP_N, OP_N, m, m, m, one, h->W, m, h->Ahat, m, zero, h->LUW, m));
      CK(cudaMemcpyAsync(h->W, h->LUW, sm, cudaMemcpyDeviceToDevice, h->st));
      CK(newton_schulz(h->W, h->Minv, 2 - sweep));  // W changed by O(Delta): quadratic steps from the old inverse
      CK(inverse_guard(h->W, h->Minv, h->LUW, h->pivW));
    }
  }
  mark(6);
  // Ritz vectors and residuals
  CK(zg(h, OP_N, OP_N, n, m, m, one, h->Qo, n, h->W, m, zero, h->X, n));
  CK(zg(h, OP_N, OP_N, n, m, m, one, h->AQ, n, h->W, m, zero, h->AX, n));
  double2* BXp = h->X;
  if (h->hasB) {
    CK(zg(h, OP_N, OP_N, n, m, m, one, h->BQ, n, h->W, m, zero, h->BX, n));
    BXp = h->BX;
  }
  CK(column_norms(h->X, n, m, h->xn, h->st));
  CK(scale_columns_inv(h->X, h->AX, h->hasB ? h->BX : nullptr, n, m, h->xn, nullptr, h->st));
  CK(residual_columns(h->AX, BXp, h->lam, 0, n, m, h->E, h->res, nullptr, h->st));
  mark(7);
  if (bi) {
    const double2* BhQp = h->Qho;
    if (h->opt.symmetric) {
      // Qho = conj(Qo) and A = A^T: A^H conj(Qo) = conj(A Qo), likewise for B
      CK(conj_copy(h->AQ, h->AhQ, (size_t)n * m, h->st));
      if (h->hasB) {
        CK(conj_copy(h->BQ, h->BhQ, (size_t)n * m, h->st));
        BhQp = h->BhQ;
      }
    } else if (side_products) {
      CK(cudaStreamWaitEvent(h->st, h->join_ev2, 0));
      if (h->hasB) BhQp = h->BhQ;
    } else {
      CK(big_product(h, 0, OP_C, h->Qho, h->AhQ));
      if (h->hasB) {
        CK(big_product(h, 1, OP_C, h->Qho, h->BhQ));
        BhQp = h->BhQ;
      }
    }
    // Zl = (W^{-1} B^^{-1})^H from the two inverses above
    CK(zg(h, OP_C, OP_C, m, m, m, one, h->Binv, m, h->Minv, m, zero, h->Zl, m));
    CK(zg(h, OP_N, OP_N, n, m, m, one, h->Qho, n, h->Zl, m, zero, h->Xl, n));
    CK(zg(h, OP_N, OP_N, n, m, m, one, h->AhQ, n, h->Zl, m, zero, h->AhX, n));
    double2* BhXp = h->Xl;
    if (h->hasB) {
      CK(zg(h, OP_N, OP_N, n, m, m, one, BhQp, n, h->Zl, m, zero, h->BhX, n));
      BhXp = h->BhX;
    }
    CK(column_dots(h->Xl, BXp, n, m, h->dd, h->st));
    CK(scale_columns_inv(h->Xl, h->AhX, h->hasB ? h->BhX : nullptr, n, m, nullptr, h->dd, h->st));
    CK(column_norms(h->Xl, n, m, h->xln, h->st));
    CK(residual_columns(h->AhX, BhXp, h->lam, 1, n, m, h->Eh, h->resl, h->xln, h->st));
  }
  mark(8);
  h->h_lam.resize(m);
  h->h_res.resize(m);
  h->h_resl.assign(m, 0.0);
  std::vector<double2> lam(m);
  CK(cudaMemcpyAsync(lam.data(), h->lam, m * sizeof(double2), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(h->h_res.data(), h->res, m * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  if (bi) CK(cudaMemcpyAsync(h->h_resl.data(), h->resl, m * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  for (int i = 0; i < m; ++i) h->h_lam[i] = zz(lam[i]);
  h->have_rr = true;
  return read_flags(h);
}

bool inside_ellipse(const feast_handle* h, zc l) {
  if (h->filter_domain) {  // rho of all the contour's nodes approximates the indicator
    zc r = 0.0;
    for (size_t k = 0; k < h->z_all.size(); ++k) r += h->w_all[k] / (h->z_all[k] - l);
    return std::abs(r) >= 0.5;
  }
  const double x = (l.real() - h->center.real()) / h->R;
  const double y = (l.imag() - h->center.imag()) / (h->R * h->aspect);
  return x * x + y * y < 1.0;
}

// candidates of the last Rayleigh-Ritz step, sorted by (Re, Im)
std::vector<int> candidates(const feast_handle* h) {
  std::vector<int> idx;
  for (int i = 0; i < h->m0; ++i) {
    const zc l = h->h_lam[i];
    if (!std::isfinite(l.real()) || !std::isfinite(l.imag())) continue;
    if (!std::isfinite(h->h_res[i])) continue;
    if (inside_ellipse(h, l) && h->h_res[i] <= h->opt.cand_tol) idx.push_back(i);
  }
  std::sort(idx.begin(), idx.end(), [&](int a, int b) {
    const zc la = h->h_lam[a], lb = h->h_lam[b];
    if (la.real() != lb.real()) return la.real() < lb.real();
    return la.imag() < lb.imag();
  });
  return idx;
}

feast_status copy_in(feast_handle* h, double2* dst, const feast_z* src, size_t count) {
  CK(cudaMemcpyAsync(dst, src, count * sizeof(double2), cudaMemcpyDefault, h->st));
  return FEAST_OK;
}
feast_status copy_out(feast_handle* h, feast_z* dst, const double2* src, size_t count) {
  if (!dst) return FEAST_OK;
  CK(cudaMemcpyAsync(dst, src, count * sizeof(double2), cudaMemcpyDefault, h->st));
  return FEAST_OK;
}

// Start the ||A||_2 estimate on the handle's norm stream (after the upload of A
// on the main stream); norm_of() waits for it where the value is first needed.
feast_status estimate_norm2(feast_handle* h) {
  CK(cudaEventRecord(h->norm_ev, h->st));
  CK(cudaStreamWaitEvent(h->norm_st, h->norm_ev, 0));
  CK(norm2_power(h->A, h->n, (int)h->n, 50, h->pw_scratch, h->scal, h->flags + 8, h->norm_st, h->At));  // own flag word
  CK(cudaEventRecord(h->norm_ev, h->norm_st));
  return FEAST_OK;
}

double norm_of(feast_handle* h) {
  if (!h->norm_ready) {
    double s = 0.0;
    unsigned f = 0;
    if (cudaEventSynchronize(h->norm_ev) == cudaSuccess &&
        cudaMemcpy(&s, h->scal, sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess &&
        cudaMemcpy(&f, h->flags + 8, sizeof(unsigned), cudaMemcpyDeviceToHost) == cudaSuccess)
      h->normA = (f & DEVFLAG_TIMEOUT) ? NAN : s;  // a timed-out estimate poisons the residuals
    h->norm_ready = true;
  }
  return h->normA;
}

// per-shift status of the last factorisation and refinement
void fill_shift_stats(const feast_handle* h, feast_stats* st) {
  st->q = h->q;
  for (int k = 0; k < h->q && k < 256; ++k) {
    st->shift_info[k] = k < (int)h->h_info.size() ? h->h_info[k] : 0;
    if (k < (int)h->h_refine_fail.size() && h->h_refine_fail[k]) st->shift_info[k] = (1 << 30) + h->h_refine_fail[k];
  }
  st->refine_sweeps = h->refine_sweeps;
  st->refactored = h->n_refactored;
}

std::atomic<unsigned long long> g_wait_ns{0};

}  // namespace

// the time limit of the cross-CTA waits (0 = each kernel's built-in limit)
unsigned long long feast_wait_limit_ns(unsigned long long dflt) {
  const unsigned long long v = g_wait_ns.load(std::memory_order_relaxed);
  return v ? v : dflt;
}

// ================================================================= C ABI
extern "C" {

uint64_t feast_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void feast_set_wait_limit(double seconds) {
  g_wait_ns.store(seconds > 0 ? (unsigned long long)(seconds * 1e9) + 1ull : 0ull, std::memory_order_relaxed);
}

feast_status feast_piecewise_nodes(const feast_segment* seg, int nseg, int K, int rule, int* q, feast_z* nodes,
                                   feast_z* weights) {
  if (!seg || nseg < 1 || !q) return FEAST_ERR_ARG;
  if (rule != FEAST_RULE_TRAP_END && rule != FEAST_RULE_GAUSS) return FEAST_ERR_ARG;
  if (K < (rule == FEAST_RULE_TRAP_END ? 2 : 1)) return FEAST_ERR_ARG;
  for (int s2 = 0; s2 < nseg; ++s2)
    if (seg[s2].kind != 0 && seg[s2].kind != 1) return FEAST_ERR_ARG;
  const int count = rule == FEAST_RULE_TRAP_END ? nseg * (K - 1) : nseg * K;
  if (count > 256) return FEAST_ERR_ARG;
  *q = count;
  if (!nodes && !weights) return FEAST_OK;
  const zc twopii(0.0, 2.0 * M_PI);
  auto point = [&](const feast_segment& g, double t) -> zc {
    const zc a(g.a.re, g.a.im), b(g.b.re, g.b.im);
    if (g.kind == 0) return a + (b - a) * t;
    return a + g.r * std::exp(zc(0.0, g.t0 + (g.t1 - g.t0) * t));
  };
  auto deriv = [&](const feast_segment& g, double t) -> zc {
    const zc a(g.a.re, g.a.im), b(g.b.re, g.b.im);
    if (g.kind == 0) return b - a;
    return zc(0.0, (g.t1 - g.t0) * g.r) * std::exp(zc(0.0, g.t0 + (g.t1 - g.t0) * t));
  };
  std::vector<zc> z, w;
  if (rule == FEAST_RULE_TRAP_END) {
    const double h = 1.0 / (K - 1);
    for (int s2 = 0; s2 < nseg; ++s2) {
      const feast_segment& g = seg[s2];
      const feast_segment& prev = seg[(s2 + nseg - 1) % nseg];
      for (int j = 0; j < K - 1; ++j) {
        const double t = j * h;
        zc d = (j == 0 ? 0.5 * h : h) * deriv(g, t);
        if (j == 0) d += 0.5 * h * deriv(prev, 1.0);  // the merged end node of the previous segment
        z.push_back(point(g, t));
        w.push_back(d / twopii);
      }
    }
  } else {
    std::vector<double> tg, wg;
    gauss_legendre(K, tg, wg);
    for (int s2 = 0; s2 < nseg; ++s2)
      for (int j = 0; j < K; ++j) {
        const double t = 0.5 * (tg[j] + 1.0);
        z.push_back(point(seg[s2], t));
        w.push_back(0.5 * wg[j] * deriv(seg[s2], t) / twopii);
      }
  }
  for (int k = 0; k < count; ++k) {
    if (nodes) { nodes[k].re = z[k].real(); nodes[k].im = z[k].imag(); }
    if (weights) { weights[k].re = w[k].real(); weights[k].im = w[k].imag(); }
  }
  return FEAST_OK;
}

feast_status feast_eta_indicator(const feast_contour* c, const double* r, int nr, int ntheta, double* eta) {
  if (!c || !r || !eta || nr < 1 || ntheta < 1 || c->R <= 0.0 || c->aspect <= 0.0) return FEAST_ERR_ARG;
  std::vector<zc> z, w;
  if (!build_quadrature(*c, z, w)) return FEAST_ERR_ARG;
  const zc cc(c->center.re, c->center.im);
  for (int i = 0; i < nr; ++i) {
    double lo = INFINITY, hi = 0.0;
    for (int j = 0; j < ntheta; ++j) {
      const double th = 2.0 * M_PI * j / ntheta;
      const zc mu = cc + r[i] * c->R * zc(std::cos(th), c->aspect * std::sin(th));
      zc rho = 0.0;
      for (size_t k = 0; k < z.size(); ++k) rho += w[k] / (z[k] - mu);
      const double a = std::abs(rho);
      lo = std::min(lo, a);
      hi = std::max(hi, a);
    }
    eta[i] = r[i] < 1.0 ? lo : hi;
  }
  return FEAST_OK;
}

feast_status feast_contour_nodes(const feast_contour* c, int* q, feast_z* nodes, feast_z* weights) {
  if (!c || !q) return FEAST_ERR_ARG;
  std::vector<zc> z, w;
  if (!build_quadrature(*c, z, w) || z.size() > 256) return FEAST_ERR_ARG;
  *q = (int)z.size();
  for (size_t k = 0; k < z.size(); ++k) {
    if (nodes) { nodes[k].re = z[k].real(); nodes[k].im = z[k].imag(); }
    if (weights) { weights[k].re = w[k].real(); weights[k].im = w[k].imag(); }
  }
  return FEAST_OK;
}

void feast_default_options(feast_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->algo = FEAST_ALGO_BI;
  o->precision = FEAST_PREC_MIXED;
  o->tol = 1e-10;
  o->max_iter = 20;
  o->cand_tol = 1e-4;
  o->panel = 0;
  o->timing = 0;
}

const char* feast_status_str(feast_status s) {
  switch (s) {
    case FEAST_OK: return "ok";
    case FEAST_ERR_ARG: return "invalid argument";
    case FEAST_ERR_ALLOC: return "device allocation failed";
    case FEAST_ERR_SINGULAR_SHIFT: return "a shifted matrix is exactly singular";
    case FEAST_ERR_REFINE_NOCONV: return "refinement did not converge";
    case FEAST_ERR_M0_TOO_SMALL: return "subspace too small";
    case FEAST_ERR_NOCONV: return "no convergence within max_iter";
    case FEAST_ERR_NONFINITE: return "non-finite value";
    case FEAST_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case FEAST_ERR_CUDA: return "CUDA error";
    case FEAST_ERR_STATE: return "call out of order";
    case FEAST_ERR_TOO_LARGE: return "size exceeds the fixed scratch of the allocation-free entry point";
  }
  return "unknown status";
}

void feast_destroy(feast_handle* h) {
  if (!h) return;
  if (h->side) cudaStreamSynchronize(h->side);
  if (h->norm_st) cudaStreamSynchronize(h->norm_st);
  cudaStreamSynchronize(h->st);
  for (void* p : h->allocs) cudaFreeAsync(p, h->st);  // back to the pool
  cudaStreamSynchronize(h->st);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : h->upd_ev) cudaEventDestroy(e);
  for (auto& e : h->deep_ev) cudaEventDestroy(e);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->fork_ev) cudaEventDestroy(h->fork_ev);
  if (h->join_ev) cudaEventDestroy(h->join_ev);
  if (h->join_ev2) cudaEventDestroy(h->join_ev2);
  for (cudaEvent_t e : h->rr_ev) cudaEventDestroy(e);
  if (h->norm_st) cudaStreamDestroy(h->norm_st);
  if (h->tinv_st) {
    cudaStreamSynchronize(h->tinv_st);
    cudaStreamDestroy(h->tinv_st);
  }
  if (h->tinv_fork) cudaEventDestroy(h->tinv_fork);
  if (h->tinv_join) cudaEventDestroy(h->tinv_join);
  if (h->norm_ev) cudaEventDestroy(h->norm_ev);
  delete h;
}

feast_status feast_create(feast_handle** out, int64_t n, const feast_z* A, int64_t lda, const feast_z* B,
                          int64_t ldb, const feast_contour* c, int m0, const feast_options* o, void* stream) {
  if (!out) return FEAST_ERR_ARG;
  *out = nullptr;
  if (n < 1 || !A || !c || lda < n || (B && ldb < n) || m0 < 1 || m0 > n || m0 > 160) return FEAST_ERR_ARG;
  const bool no_ellipse = c->rule == FEAST_RULE_CUSTOM && c->R == 0.0;
  if (!no_ellipse && (c->R <= 0.0 || c->aspect <= 0.0)) return FEAST_ERR_ARG;
  feast_handle* h = new (std::nothrow) feast_handle();
  if (!h) return FEAST_ERR_ALLOC;
  if (o) h->opt = *o; else feast_default_options(&h->opt);
  if (h->opt.tol <= 0) h->opt.tol = 1e-10;
  if (h->opt.max_iter < 1) h->opt.max_iter = 20;
  if (h->opt.max_iter > 64) h->opt.max_iter = 64;
  if (h->opt.cand_tol <= 0) h->opt.cand_tol = 1e-4;
  if (h->opt.algo != FEAST_ALGO_R && h->opt.algo != FEAST_ALGO_BI) { delete h; return FEAST_ERR_ARG; }
  if (h->opt.precision != FEAST_PREC_FP64 && h->opt.precision != FEAST_PREC_MIXED) { delete h; return FEAST_ERR_ARG; }
  h->n = n;
  h->m0 = m0;
  h->st = reinterpret_cast<cudaStream_t>(stream);
  h->hasB = B != nullptr;
  h->center = zc(c->center.re, c->center.im);
  h->R = no_ellipse ? 1.0 : c->R;
  h->aspect = no_ellipse ? 1.0 : c->aspect;
  h->filter_domain = no_ellipse;
  if (!build_quadrature(*c, h->z_all, h->w_all) || h->z_all.size() > 256) { delete h; return FEAST_ERR_ARG; }
  {
    // this handle's range of the linear systems (the shift-partitioned filter)
    const int qa = (int)h->z_all.size();
    int b0 = h->opt.shift_begin, b1 = h->opt.shift_end;
    if (b0 == 0 && b1 == 0) b1 = qa;
    if (b0 < 0 || b1 > qa || b0 >= b1) { delete h; return FEAST_ERR_ARG; }
    // the range must be an aligned run of L = 1, 2, 4 or 8 of the eight leaves
    // gb[g] = floor(g qa / 8) of the fixed summation tree
    int gb[9];
    for (int g = 0; g <= 8; ++g) gb[g] = (int)(((long long)g * qa) / 8);
    bool found = false;
    for (int L = 8; L >= 1 && !found; L /= 2)
      for (int j = 0; j < 8 / L && !found; ++j)
        if (gb[j * L] == b0 && gb[(j + 1) * L] == b1) {
          h->tree.nleaf = L;
          for (int i = 0; i <= L; ++i) h->tree.b[i] = gb[j * L + i] - b0;
          found = true;
        }
    if (!found) { delete h; return FEAST_ERR_ARG; }
    h->shift0 = b0;
    // a handle created with a range is a member of a shift partition (even when
    // the range is every node: the partition of one process)
    h->partial = h->opt.shift_begin != 0 || h->opt.shift_end != 0;
    h->z.assign(h->z_all.begin() + b0, h->z_all.begin() + b1);
    h->w.assign(h->w_all.begin() + b0, h->w_all.begin() + b1);
    for (int k = b0; k < b1; ++k) {
      h->gidx.push_back(k);
      h->pidx.push_back(-1);
    }
  }
  if (h->opt.real_pencil) {
    // (conj(phi) B - A) = conj(phi B - A) for real A and B: factor one node of
    // each conjugate pair (the one with Im phi > 0) and every real node
    if (h->partial) { delete h; return FEAST_ERR_ARG; }
    const int qa = (int)h->z_all.size();
    std::vector<int> g, pp;
    std::vector<char> used(qa, 0);
    for (int k = 0; k < qa; ++k) {
      const zc zk = h->z_all[k];
      const double tol = 1e-12 * std::max(1.0, std::abs(zk));
      if (std::abs(zk.imag()) <= tol) { g.push_back(k); pp.push_back(-1); used[k] = 1; continue; }
      if (zk.imag() < 0) continue;
      int p = -1;
      for (int j = 0; j < qa; ++j)
        if (!used[j] && j != k && std::abs(h->z_all[j] - std::conj(zk)) <= tol &&
            std::abs(h->w_all[j] - std::conj(h->w_all[k])) <= 1e-12 * std::max(std::abs(h->w_all[k]), 1e-300)) {
          p = j;
          break;
        }
      if (p < 0) { delete h; return FEAST_ERR_ARG; }  // the contour is not symmetric about the real axis
      used[k] = used[p] = 1;
      g.push_back(k);
      pp.push_back(p);
    }
    for (int k = 0; k < qa; ++k)
      if (!used[k]) { delete h; return FEAST_ERR_ARG; }
    h->gidx = g;
    h->pidx = pp;
    h->z.clear();
    h->w.clear();
    for (int k : g) {
      h->z.push_back(h->z_all[k]);
      h->w.push_back(h->w_all[k]);
    }
    h->realp = true;
    h->tree = acc_tree_single((int)g.size());
    if (h->opt.max_refine > 0) { delete h; return FEAST_ERR_ARG; }
    if (2 * m0 > n) { delete h; return FEAST_ERR_ARG; }
  }
  if (h->opt.refine_tol <= 0) h->opt.refine_tol = 1e-12;
  if (h->opt.max_refine < 0 || h->opt.max_refine > 16) { delete h; return FEAST_ERR_ARG; }
  h->q = (int)h->z.size();
  const bool mx = h->opt.precision == FEAST_PREC_MIXED;
  h->nb = h->opt.panel > 0 ? std::min(h->opt.panel, mx ? 128 : 64) : 64;
  h->nbs = 64;
  const size_t esz = mx ? sizeof(float2) : sizeof(double2);
  const size_t nn = (size_t)n * n, nm = (size_t)n * m0, mm = (size_t)m0 * m0;
  auto fail = [&](cudaError_t e) { feast_destroy(h); return cuda_status(e); };
  cudaError_t e;
#define AL(p, bytes) if ((e = dalloc(h, &(p), (bytes))) != cudaSuccess) return fail(e)
  AL(h->A, nn * sizeof(double2));
  AL(h->At, nn * sizeof(double2));  // A^T for the norm estimate
  if (h->hasB) AL(h->B, nn * sizeof(double2));
  AL(h->dz, h->q * sizeof(double2));
  AL(h->dw, h->q * sizeof(double2));
  AL(h->dmu, (size_t)(h->q + 64) * sizeof(double2));
  AL(h->S, nn * h->q * esz);
  AL(h->piv, (size_t)h->q * n * sizeof(int32_t));
  AL(h->perm, (size_t)h->q * n * sizeof(int32_t));
  AL(h->pinv, (size_t)h->q * n * sizeof(int32_t));
  AL(h->mv, (size_t)((n + 63) / 64) * h->q * LU_MV_STRIDE * sizeof(int32_t));
  AL(h->info, h->q * sizeof(int));
  AL(h->flags, 64);
  const size_t xq = h->realp ? 2 * (size_t)h->q : (size_t)h->q;  // real pencils solve [R, conj(R)]
  AL(h->Xs, nm * std::max(xq, (size_t)2) * esz);
  if (h->opt.algo == FEAST_ALGO_BI) AL(h->Xsh, nm * xq * esz);
  if (h->realp) {
    AL(h->coefc, (size_t)h->q * m0 * sizeof(double2));
    AL(h->coefch, (size_t)h->q * m0 * sizeof(double2));
  }
  double2** blocks[] = {&h->Y, &h->Yh, &h->Rr, &h->Rl, &h->Q, &h->Qh, &h->Qo, &h->Qho, &h->AQ, &h->BQ,
                        &h->AhQ, &h->BhQ, &h->X, &h->Xl, &h->AX, &h->BX, &h->AhX, &h->BhX, &h->E, &h->Eh, &h->tmp};
  for (double2** p : blocks) AL(*p, nm * sizeof(double2) + 2 * n * sizeof(double2));
  double2** smalls[] = {&h->Ahat, &h->Bhat, &h->LUB, &h->Cm, &h->Zs, &h->V, &h->W, &h->LUW, &h->Minv, &h->Binv, &h->Zl};
  for (double2** p : smalls) AL(*p, mm * sizeof(double2));
  AL(h->lam, m0 * sizeof(double2));
  AL(h->dd, m0 * sizeof(double2));
  AL(h->coef, (size_t)h->q * m0 * sizeof(double2));
  AL(h->coefh, (size_t)h->q * m0 * sizeof(double2));
  AL(h->c0, m0 * sizeof(double2));
  AL(h->c0h, m0 * sizeof(double2));
  AL(h->pivB, m0 * sizeof(int));
  AL(h->pivW, m0 * sizeof(int));
  AL(h->useres, m0 * sizeof(int));
  AL(h->useresh, m0 * sizeof(int));
  AL(h->colidx, m0 * sizeof(int));
  AL(h->gate, 64);
  AL(h->res, m0 * sizeof(double));
  AL(h->resl, m0 * sizeof(double));
  AL(h->xn, m0 * sizeof(double));
  AL(h->xln, m0 * sizeof(double));
  AL(h->scal, 64);
  AL(h->orth_scratch, orth_scratch_bytes((int)n, m0));
  AL(h->pw_scratch, norm2_scratch_bytes((int)n));
  AL(h->schur_log, schur_log_bytes(m0));
  h->gemm_ws_elems = (size_t)64 * 160 * 160;
  AL(h->gemm_ws, h->gemm_ws_elems * sizeof(double2));
  AL(h->s32, (size_t)5 * m0 * m0 * sizeof(float2));
  if (mx && n >= 256) {  // FP64-accurate Rayleigh-Ritz products on the BF16 tensor cores
    void* ozbase = nullptr;
    AL(ozbase, oz_work_bytes((int)n, m0));
    oz_work_layout(ozbase, (int)n, m0, &h->ozw);
    h->use_oz = true;
    if (h->opt.algo == FEAST_ALGO_BI && !h->opt.symmetric) {
      void* ozbase2 = nullptr;
      AL(ozbase2, oz_work_bytes((int)n, m0));
      oz_work_layout(ozbase2, (int)n, m0, &h->ozw2);
      h->has_ozw2 = true;
    }
  }
  if (mx) {
    AL(h->staging.Ast, tc_staging_bytes_A(n, h->q));
    AL(h->staging.Bst, tc_staging_bytes_B(n, h->q));
    h->staging.rows_max = 2 * n;
    h->staging.cols_max = n;
    h->staging.q = h->q;
    // the autotuner's choice for this GPU, order bucket, m0, shift count and precision
    if (h->opt.tune_cache) {
      char key[256];
      std::snprintf(key, sizeof(key), "%s|single|n%lld|m0%d|q%d|mixed", tune_gpu_name().c_str(),
                    tune_bucket(n), m0, (int)h->z_all.size());
      std::map<std::string, double> t;
      if (tune_lookup(h->opt.tune_cache, key, t)) {
        if (h->opt.lu_outer == 0 && t.count("lu_outer")) {
          const int v = (int)t["lu_outer"];
          if (v < 0 || (v % 64 == 0 && v <= 256 && n > v)) h->opt.lu_outer = v;
        }
        if (h->opt.panel_cluster == 0 && t.count("panel_cluster")) h->opt.panel_cluster = (int)t["panel_cluster"];
        h->tuned = true;
      }
    }
    // two-level LU: outer blocks of lu_outer columns with deep (K = lu_outer) updates
    int outer = h->opt.lu_outer;
    if (outer == 0) outer = n >= 1024 ? 256 : -1;
    if (outer > 0 && (outer % 64 || outer > 256 || n <= outer || n > 16384)) { feast_destroy(h); return FEAST_ERR_ARG; }
    if (outer > 0 && h->nb == 64) {
      AL(h->deep.Ast, deep_staging_bytes_A(n, h->q));
      AL(h->deep.Bst, deep_staging_bytes_B(n, h->q));
      h->deep.rows_max = 2 * n;
      h->deep.cols_max = n;
      h->deep.q = h->q;
      if (h->opt.algo == FEAST_ALGO_BI && !h->opt.symmetric) {
        AL(h->deep_left.Ast, deep_staging_bytes_A(n, h->q));
        AL(h->deep_left.Bst, deep_staging_bytes_B(n, h->q));
        h->deep_left.rows_max = 2 * n;
        h->deep_left.cols_max = n;
        h->deep_left.q = h->q;
      }
      h->nblk = (int)((n + outer - 1) / outer);
      AL(h->TL, (size_t)h->nblk * h->q * outer * outer * sizeof(float2));
      AL(h->TU, (size_t)h->nblk * h->q * outer * outer * sizeof(float2));
      h->lu_outer = outer;
      if (h->opt.deep_solves >= 0) {
        // the blocked solves' factor operands, staged once per factorisation, when
        // they fit in half of the free memory (otherwise each solve stages its own)
        const int sides = (h->opt.algo == FEAST_ALGO_BI && !h->opt.symmetric) ? 2 : 1;
        const size_t bytes = tc_solve_prestage_bytes(n, h->q, outer);
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && (double)bytes * sides < 0.5 * (double)fr)
          for (int sd = 0; sd < sides; ++sd) AL(h->pre[sd], bytes);
      }
    }
    {  // row maps of the interchanges: blocks of lu_outer columns, or of 64 for the one-level LU
      const long long kb = h->lu_outer > 0 ? h->lu_outer : 64;
      const size_t bytes = lu_rowmap_ints(n, h->q, (int)kb) * sizeof(int32_t);
      if (bytes <= ((size_t)1 << 30)) AL(h->rowmaps, bytes);
    }
    if (h->opt.algo == FEAST_ALGO_BI && !h->opt.symmetric) {
      AL(h->staging_left.Ast, tc_staging_bytes_A(n, h->q));
      AL(h->staging_left.Bst, tc_staging_bytes_B(n, h->q));
      h->staging_left.rows_max = 2 * n;
      h->staging_left.cols_max = n;
      h->staging_left.q = h->q;
    }
  }
  if (h->opt.algo == FEAST_ALGO_BI && !h->opt.symmetric) {
    AL(h->orth_scratch2, orth_scratch_bytes((int)n, m0));
    if ((e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreateWithFlags(&h->join_ev2, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  }
#undef AL
  if ((e = cudaStreamCreateWithFlags(&h->norm_st, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
  if (h->lu_outer > 0) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if ((e = cudaStreamCreateWithPriority(&h->tinv_st, cudaStreamNonBlocking, lo)) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreateWithFlags(&h->tinv_fork, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreateWithFlags(&h->tinv_join, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  }
  if ((e = cudaEventCreateWithFlags(&h->norm_ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  if (h->opt.timing)
    for (auto& ev : h->ev) cudaEventCreate(&ev);
  std::vector<double2> zd(h->q);
  for (int k = 0; k < h->q; ++k) zd[k] = d2(h->z[k]);
  if ((e = cudaMemcpyAsync(h->dz, zd.data(), h->q * sizeof(double2), cudaMemcpyHostToDevice, h->st)) != cudaSuccess) return fail(e);
  std::vector<double2> wd(h->q);
  for (int k = 0; k < h->q; ++k) wd[k] = d2(h->w[k]);
  if ((e = cudaMemcpyAsync(h->dw, wd.data(), h->q * sizeof(double2), cudaMemcpyHostToDevice, h->st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemsetAsync(h->flags, 0, 64, h->st)) != cudaSuccess) return fail(e);
  // contiguous operands go as one linear copy (the faster path for large
  // host-to-device transfers), strided ones column by column
  auto upload = [&](double2* dst, const feast_z* src, int64_t ld) -> cudaError_t {
    if (ld == n) return cudaMemcpyAsync(dst, src, nn * sizeof(double2), cudaMemcpyDefault, h->st);
    return cudaMemcpy2DAsync(dst, n * sizeof(double2), src, ld * sizeof(double2), n * sizeof(double2), n,
                             cudaMemcpyDefault, h->st);
  };
  if ((e = upload(h->A, A, lda)) != cudaSuccess) return fail(e);
  if (h->hasB && (e = upload(h->B, B, ldb)) != cudaSuccess) return fail(e);
  if ((e = check_finite(h->A, nn, h->flags, h->st)) != cudaSuccess) return fail(e);
  if (h->hasB && (e = check_finite(h->B, nn, h->flags, h->st)) != cudaSuccess) return fail(e);
  feast_status s = read_flags(h);
  if (s != FEAST_OK) { feast_destroy(h); return s; }
  s = estimate_norm2(h);
  if (s != FEAST_OK) { feast_destroy(h); return s; }
  *out = h;
  return FEAST_OK;
}

feast_status feast_get_quadrature(const feast_handle* h, int* q, feast_z* nodes, feast_z* weights) {
  if (!h) return FEAST_ERR_ARG;
  if (q) *q = h->q;
  for (int k = 0; k < h->q; ++k) {
    if (nodes) { nodes[k].re = h->z[k].real(); nodes[k].im = h->z[k].imag(); }
    if (weights) { weights[k].re = h->w[k].real(); weights[k].im = h->w[k].imag(); }
  }
  return FEAST_OK;
}

feast_status feast_get_stats(const feast_handle* h, feast_stats* st) {
  if (!h || !st) return FEAST_ERR_ARG;
  std::memset(st, 0, sizeof(*st));
  fill_shift_stats(h, st);
  st->normA = norm_of(const_cast<feast_handle*>(h));
  st->t_factor_ms = h->t_factor;
  st->t_update_ms = h->t_update;
  st->update_launches = h->n_update;
  st->lu_outer = h->lu_outer;
  st->t_deep_ms = h->t_deep;
  st->deep_launches = h->n_deep;
  st->deep_flops = h->deep_flops;
  st->deep_bytes = h->deep_bytes;
  st->update_flops = h->upd_flops;
  st->update_bytes = h->upd_bytes;
  st->tuned = h->tuned ? 1 : 0;
  st->t_filter_ms = h->t_filter;
  st->t_rr_ms = h->t_rr;
  if (h->opt.timing && h->rr_ev.size() >= 9) {
    for (int i = 0; i < 8; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, h->rr_ev[i], h->rr_ev[i + 1]) == cudaSuccess) st->t_rr_phase_ms[i] = ms;
    }
  }
  return FEAST_OK;
}

feast_status feast_factor(feast_handle* h) {
  if (!h) return FEAST_ERR_ARG;
  h->factored = false;  // an explicit call always forms and factors again
  return ensure_factored(h);
}

feast_status feast_get_factor(feast_handle* h, int k, feast_z* LU, int32_t* piv) {
  if (!h || k < 0 || k >= h->q) return FEAST_ERR_ARG;
  if (!h->factored) return FEAST_ERR_STATE;
  const size_t nn = (size_t)h->n * h->n;
  if (LU) {
    if (mixed(h)) {
      std::vector<float2> tmp(nn);
      CK(cudaMemcpyAsync(tmp.data(), reinterpret_cast<float2*>(h->S) + k * nn, nn * sizeof(float2),
                         cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
      std::vector<double2> d(nn);
      for (size_t i = 0; i < nn; ++i) d[i] = make_double2(tmp[i].x, tmp[i].y);
      CK(cudaMemcpyAsync(LU, d.data(), nn * sizeof(double2), cudaMemcpyDefault, h->st));
      CK(cudaStreamSynchronize(h->st));
    } else {
      CK(cudaMemcpyAsync(LU, reinterpret_cast<double2*>(h->S) + k * nn, nn * sizeof(double2), cudaMemcpyDefault, h->st));
    }
  }
  if (piv) CK(cudaMemcpyAsync(piv, h->piv + (size_t)k * h->n, h->n * sizeof(int32_t), cudaMemcpyDefault, h->st));
  CK(cudaStreamSynchronize(h->st));
  return FEAST_OK;
}

}  // extern "C"

namespace {
template <typename T>
feast_status solve_shift_impl(feast_handle* h, int k, int side, int nrhs, double2* out) {
  LuBatch<T> lu = lu_view<T>(h);
  const size_t nn = (size_t)h->n * h->n;
  lu.S += nn * k;
  lu.piv += (size_t)k * h->n;
  lu.perm += (size_t)k * h->n;
  lu.pinv += (size_t)k * h->n;
  lu.info += k;
  lu.q = 1;
  cplx<T>* X = reinterpret_cast<cplx<T>*>(h->Xs);
  cplx<T>* X2 = X + (size_t)h->n * nrhs;
  CK(rows_gather<T>(lu, h->Rr, X, nrhs, side == 0, h->st));
  CK(lu_solve_batched<T>(lu, side, X, nrhs, h->nbs, h->st));
  const cplx<T>* res = X;
  if (side == 1) {
    CK(rows_scatter<T>(lu, X, X2, nrhs, h->st));
    res = X2;
  }
  // widen into `out` through the accumulation kernel with unit coefficients
  std::vector<double2> ones((size_t)nrhs, make_double2(1.0, 0.0));
  CK(cudaMemcpyAsync(h->coef, ones.data(), nrhs * sizeof(double2), cudaMemcpyHostToDevice, h->st));
  CK(accumulate<T>(res, acc_tree_single(1), (int)h->n, nrhs, h->coef, nullptr, nullptr, nullptr, out, h->st));
  CK(cudaStreamSynchronize(h->st));
  return FEAST_OK;
}
}  // namespace

extern "C" {

feast_status feast_solve_shift(feast_handle* h, int k, int side, const feast_z* R, feast_z* X, int nrhs) {
  if (!h || k < 0 || k >= h->q || (side != 0 && side != 1) || !R || !X || nrhs < 1 || nrhs > h->m0)
    return FEAST_ERR_ARG;
  feast_status s = ensure_factored(h);
  if (s != FEAST_OK && s != FEAST_ERR_SINGULAR_SHIFT) return s;
  const size_t cnt = (size_t)h->n * nrhs;
  if ((s = copy_in(h, h->Rr, R, cnt)) != FEAST_OK) return s;
  s = mixed(h) ? solve_shift_impl<float>(h, k, side, nrhs, h->tmp) : solve_shift_impl<double>(h, k, side, nrhs, h->tmp);
  if (s != FEAST_OK) return s;
  if ((s = copy_out(h, X, h->tmp, cnt)) != FEAST_OK) return s;
  CK(cudaStreamSynchronize(h->st));
  return FEAST_OK;
}

}  // extern "C"

namespace {
template <typename T>
feast_status moments_impl(feast_handle* h, const double2* BV, int S, int kmax) {
  LuBatch<T> lu = lu_view<T>(h);
  cplx<T>* Xs = reinterpret_cast<cplx<T>*>(h->Xs);
  CK(rows_gather<T>(lu, BV, Xs, S, true, h->st));
  CK(lu_solve_batched<T>(lu, 0, Xs, S, h->nbs, h->st));
  CK(probe_dots<T>(h->Y, Xs, (int)h->n, S, h->q, h->dmu + 64, h->st));
  CK(moments_combine(h->dmu + 64, h->dz, h->dw, d2(h->center), h->R, h->q, kmax, S, h->dmu, h->st));
  return FEAST_OK;
}
}  // namespace

extern "C" {

feast_status feast_moments(feast_handle* h, const feast_z* V, int S, int kmax, feast_z* mu) {
  if (!h || !V || !mu || S < 1 || S > h->m0 || kmax < 0 || kmax > 31) return FEAST_ERR_ARG;
  if (h->realp) return FEAST_ERR_STATE;  // the moments need every node's own solve
  feast_status s = ensure_factored(h);
  if (s != FEAST_OK) return s;
  const int n = (int)h->n;
  const size_t cnt = (size_t)n * S;
  if ((s = copy_in(h, h->Y, V, cnt)) != FEAST_OK) return s;
  const double2* BV = h->Y;
  if (h->hasB) {
    CK(big_product(h, 1, OP_N, h->Y, h->BX, S));
    BV = h->BX;
  }
  s = mixed(h) ? moments_impl<float>(h, BV, S, kmax) : moments_impl<double>(h, BV, S, kmax);
  if (s != FEAST_OK) return s;
  CK(cudaMemcpyAsync(mu, h->dmu, (kmax + 1) * sizeof(double2), cudaMemcpyDefault, h->st));
  CK(cudaStreamSynchronize(h->st));
  return read_flags(h);
}

feast_status feast_filter(feast_handle* h, const feast_z* Y, const feast_z* Yhat, const feast_z* theta, feast_z* Q,
                          feast_z* Qhat) {
  if (!h || !Y || !Q || (Yhat && !Qhat)) return FEAST_ERR_ARG;
  if (Yhat && h->opt.algo != FEAST_ALGO_BI) return FEAST_ERR_ARG;
  feast_status s = ensure_factored(h);
  if (s != FEAST_OK) return s;
  const int n = (int)h->n, m = h->m0;
  const size_t cnt = (size_t)n * m;
  if ((s = copy_in(h, h->Y, Y, cnt)) != FEAST_OK) return s;
  if (Yhat && (s = copy_in(h, h->Yh, Yhat, cnt)) != FEAST_OK) return s;
  std::vector<zc> th;
  const bool resform = theta && mixed(h);
  if (resform) {
    std::vector<double2> t(m);
    CK(cudaMemcpyAsync(t.data(), theta, m * sizeof(double2), cudaMemcpyDefault, h->st));
    CK(cudaStreamSynchronize(h->st));
    for (int i = 0; i < m; ++i) th.push_back(zz(t[i]));
  }
  if ((s = upload_coefs(h, resform ? th.data() : nullptr, nullptr)) != FEAST_OK) return s;
  // right-hand sides: B Y (plain) or (A Y - B Y Theta) per column (residual form)
  double2* BY = h->Y;
  if (h->hasB) { CK(big_product(h, 1, OP_N, h->Y, h->BX)); BY = h->BX; }
  const double2* R = BY;
  if (resform) {
    CK(cudaMemcpyAsync(h->lam, theta, m * sizeof(double2), cudaMemcpyDefault, h->st));
    CK(big_product(h, 0, OP_N, h->Y, h->AX));
    CK(residual_columns(h->AX, BY, h->lam, 0, n, m, h->E, h->res, nullptr, h->st));
    CK(select_columns(h->E, BY, h->useres, n, m, h->Rr, h->st));
    R = h->Rr;
  }
  const double2* Rh = nullptr;
  if (Yhat) {
    double2* BhY = h->Yh;
    if (h->hasB) { CK(big_product(h, 1, OP_C, h->Yh, h->BhX)); BhY = h->BhX; }
    Rh = BhY;
    if (resform) {
      CK(big_product(h, 0, OP_C, h->Yh, h->AhX));
      CK(residual_columns(h->AhX, BhY, h->lam, 1, n, m, h->Eh, h->resl, nullptr, h->st));
      CK(select_columns(h->Eh, BhY, h->useres, n, m, h->Rl, h->st));
      Rh = h->Rl;
    }
  }
  if ((s = run_filter(h, R, h->Y, resform, Rh, h->Yh)) != FEAST_OK) return s;
  if ((s = copy_out(h, Q, h->Q, cnt)) != FEAST_OK) return s;
  if (Yhat && (s = copy_out(h, Qhat, h->Qh, cnt)) != FEAST_OK) return s;
  CK(cudaStreamSynchronize(h->st));
  return read_flags(h);
}

feast_status feast_candidates(const feast_handle* h, int* count, int* idx, double* max_res) {
  if (!h || !count) return FEAST_ERR_ARG;
  if (!h->have_rr) return FEAST_ERR_STATE;
  const std::vector<int> c = candidates(h);
  *count = (int)c.size();
  double mr = c.empty() ? INFINITY : 0.0;
  const double nA = norm_of(const_cast<feast_handle*>(h));
  for (size_t j = 0; j < c.size(); ++j) {
    if (idx) idx[j] = c[j];
    mr = std::max(mr, h->h_res[c[j]] / nA);
  }
  if (max_res) *max_res = mr;
  return FEAST_OK;
}

feast_status feast_filter_combine(feast_handle* h, int nparts, const feast_z* const* parts,
                                  const feast_z* const* parts_hat, const feast_z* Y, const feast_z* Yhat,
                                  const feast_z* theta, feast_z* Q, feast_z* Qhat) {
  if (!h || !parts || !Q || nparts < 1 || nparts > 8 || (nparts & (nparts - 1))) return FEAST_ERR_ARG;
  if ((parts_hat && !Qhat) || (Qhat && !parts_hat)) return FEAST_ERR_ARG;
  const bool resform = theta && mixed(h);
  if (resform && (!Y || (parts_hat && !Yhat))) return FEAST_ERR_ARG;
  const int n = (int)h->n, m = h->m0;
  const size_t cnt = (size_t)n * m;
  if (!h->combine_buf) CK(dalloc(h, &h->combine_buf, 8 * cnt * sizeof(double2)));
  feast_status s;
  if (resform) {
    std::vector<double2> t(m);
    CK(cudaMemcpyAsync(t.data(), theta, m * sizeof(double2), cudaMemcpyDefault, h->st));
    CK(cudaStreamSynchronize(h->st));
    std::vector<zc> th(m);
    for (int i = 0; i < m; ++i) th[i] = zz(t[i]);
    if ((s = upload_coefs(h, th.data(), nullptr)) != FEAST_OK) return s;
  }
  for (int side = 0; side < (parts_hat ? 2 : 1); ++side) {
    const feast_z* const* P = side ? parts_hat : parts;
    for (int j = 0; j < nparts; ++j) {
      if (!P[j]) return FEAST_ERR_ARG;
      if ((s = copy_in(h, h->combine_buf + j * cnt, P[j], cnt)) != FEAST_OK) return s;
    }
    double2* Yd = side ? h->Yh : h->Y;
    if (resform && (s = copy_in(h, Yd, side ? Yhat : Y, cnt)) != FEAST_OK) return s;
    double2* out = side ? h->Qh : h->Q;
    CK(accumulate_tree_combine(h->combine_buf, nparts, n, m, resform ? (side ? h->c0h : h->c0) : nullptr,
                               resform ? Yd : nullptr, out, h->st));
    if ((s = copy_out(h, side ? Qhat : Q, out, cnt)) != FEAST_OK) return s;
  }
  CK(cudaStreamSynchronize(h->st));
  return FEAST_OK;
}

feast_status feast_rayleigh_ritz(feast_handle* h, const feast_z* Q, const feast_z* Qhat, feast_z* lambda, feast_z* X,
                                 feast_z* Xl, double* res, int* m_inside) {
  if (!h || !Q || !lambda) return FEAST_ERR_ARG;
  if (Qhat && h->opt.algo != FEAST_ALGO_BI) return FEAST_ERR_ARG;
  const int n = (int)h->n, m = h->m0;
  const size_t cnt = (size_t)n * m;
  feast_status s;
  if ((s = copy_in(h, h->Q, Q, cnt)) != FEAST_OK) return s;
  if (Qhat && (s = copy_in(h, h->Qh, Qhat, cnt)) != FEAST_OK) return s;
  if ((s = rr_impl(h, h->Q, Qhat ? h->Qh : nullptr)) != FEAST_OK) return s;
  std::vector<double2> lam(m);
  for (int i = 0; i < m; ++i) lam[i] = d2(h->h_lam[i]);
  CK(cudaMemcpyAsync(lambda, lam.data(), m * sizeof(double2), cudaMemcpyDefault, h->st));
  if ((s = copy_out(h, X, h->X, cnt)) != FEAST_OK) return s;
  if (Qhat && (s = copy_out(h, Xl, h->Xl, cnt)) != FEAST_OK) return s;
  std::vector<double> r(m);
  const double nA = norm_of(h);
  for (int i = 0; i < m; ++i) r[i] = h->h_res[i] / nA;
  if (res) CK(cudaMemcpyAsync(res, r.data(), m * sizeof(double), cudaMemcpyDefault, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (m_inside) *m_inside = (int)candidates(h).size();
  return FEAST_OK;
}

feast_status feast_solve(feast_handle* h, const feast_z* Y0, const feast_z* Vrand, feast_z* lambda, feast_z* Xout,
                         feast_z* Xlout, double* res, int* m_found, feast_stats* stats) {
  if (!h || !Y0 || !lambda) return FEAST_ERR_ARG;
  if (h->partial) return FEAST_ERR_STATE;  // a shift range filters only part of the sum
  const bool bi = h->opt.algo == FEAST_ALGO_BI;
  const int n = (int)h->n, m = h->m0;
  const size_t cnt = (size_t)n * m;
  const zc one(1.0), zero(0.0);
  feast_stats st;
  std::memset(&st, 0, sizeof(st));
  if (h->opt.timing) cudaEventRecord(h->ev[2], h->st);
  h->t_filter = h->t_rr = 0.0;
  feast_status s = ensure_factored(h);
  st.t_factor_ms = h->t_factor;
  if (s != FEAST_OK) return s;
  if ((s = copy_in(h, h->Y, Y0, cnt)) != FEAST_OK) return s;
  if (bi && h->opt.symmetric) {
    // complex symmetric pencil: the left block is the conjugate of the right one
    CK(conj_copy(h->Y, h->Yh, cnt, h->st));
  } else if (bi) {
    // Bi-FEAST step 2: V0 = Vr (Vr^H B Y0)^{-H}
    if ((s = copy_in(h, h->Yh, Vrand ? Vrand : Y0, cnt)) != FEAST_OK) return s;
    const double2* BY0 = h->Y;
    if (h->hasB) { CK(big_product(h, 1, OP_N, h->Y, h->BX)); BY0 = h->BX; }
    CK(zg(h, OP_C, OP_N, m, m, n, one, h->Yh, n, BY0, n, zero, h->LUW, m));
    CK(small_lu(h->LUW, m, h->pivW, h->flags, h->st));
    CK(set_identity(h->Minv, m, h->st));
    CK(small_lu_solve(h->LUW, h->pivW, m, h->Minv, m, 0, h->st));
    CK(cudaMemcpyAsync(h->tmp, h->Yh, cnt * sizeof(double2), cudaMemcpyDeviceToDevice, h->st));
    CK(zg(h, OP_N, OP_C, n, m, m, one, h->tmp, n, h->Minv, m, zero, h->Yh, n));
  }
  int prev = -1;
  bool converged = false;
  std::vector<int> cand;
  double max_res = INFINITY;
  int it = 0;
  for (it = 1; it <= h->opt.max_iter; ++it) {
    ev_mark(h, 0);
    const bool resform = mixed(h) && it > 1;
    const double2 *R, *Rh = nullptr, *Yc0 = nullptr, *Yhc0 = nullptr;
    if (it == 1) {
      if ((s = upload_coefs(h, nullptr, nullptr)) != FEAST_OK) return s;
      double2* BY = h->Y;
      if (h->hasB) { CK(big_product(h, 1, OP_N, h->Y, h->BX)); BY = h->BX; }
      R = BY;
      if (bi) {
        double2* BhY = h->Yh;
        if (h->hasB) { CK(big_product(h, 1, OP_C, h->Yh, h->BhX)); BhY = h->BhX; }
        Rh = BhY;
      }
    } else if (!resform) {
      if ((s = upload_coefs(h, nullptr, nullptr)) != FEAST_OK) return s;
      R = h->hasB ? h->BX : h->X;  // B U with U the unit Ritz vectors of the last step
      if (bi) Rh = h->hasB ? h->BhX : h->Xl;
    } else {
      if ((s = upload_coefs(h, h->h_lam.data(), nullptr)) != FEAST_OK) return s;
      const double2* BXp = h->hasB ? h->BX : h->X;
      CK(select_columns(h->E, BXp, h->useres, n, m, h->Rr, h->st));
      R = h->Rr;
      Yc0 = h->X;
      if (bi) {
        const double2* BhXp = h->hasB ? h->BhX : h->Xl;
        CK(select_columns(h->Eh, BhXp, h->useres, n, m, h->Rl, h->st));
        Rh = h->Rl;
        Yhc0 = h->Xl;
      }
    }
    if ((s = run_filter(h, R, Yc0, resform, Rh, Yhc0)) != FEAST_OK) return s;
    ev_mark(h, 1);
    if ((s = rr_impl(h, h->Q, bi ? h->Qh : nullptr)) != FEAST_OK) return s;
    ev_mark(h, 3);
    h->t_filter += ev_ms(h, 0, 1);
    h->t_rr += ev_ms(h, 1, 3);
    cand = candidates(h);
    const int count = (int)cand.size();
    max_res = count ? 0.0 : INFINITY;
    for (int i : cand) max_res = std::max(max_res, h->h_res[i] / norm_of(h));
    if (it - 1 < 64) {
      st.res_hist[it - 1] = max_res;
      st.count_hist[it - 1] = count;
      st.res_hist_len = it;
    }
    if (count > 0 && count == prev && max_res <= h->opt.tol) {
      converged = true;
      break;
    }
    prev = count;
  }
  if (it > h->opt.max_iter) it = h->opt.max_iter;
  // outputs: candidates first, sorted by (Re, Im)
  const int k = (int)cand.size();
  std::vector<double2> lam(m, make_double2(0.0, 0.0));
  std::vector<double> r(m, 0.0);
  for (int j = 0; j < k; ++j) {
    lam[j] = d2(h->h_lam[cand[j]]);
    r[j] = h->h_res[cand[j]] / norm_of(h);
  }
  CK(cudaMemcpyAsync(lambda, lam.data(), m * sizeof(double2), cudaMemcpyDefault, h->st));
  if (res) CK(cudaMemcpyAsync(res, r.data(), m * sizeof(double), cudaMemcpyDefault, h->st));
  std::vector<int> idx(m, 0);
  for (int j = 0; j < k; ++j) idx[j] = cand[j];
  CK(cudaMemcpyAsync(h->colidx, idx.data(), m * sizeof(int), cudaMemcpyHostToDevice, h->st));
  if (Xout) {
    CK(gather_columns(h->X, h->colidx, k, n, m, h->tmp, h->st));
    if ((s = copy_out(h, Xout, h->tmp, cnt)) != FEAST_OK) return s;
  }
  if (Xlout && bi) {
    CK(gather_columns(h->Xl, h->colidx, k, n, m, h->tmp, h->st));
    if ((s = copy_out(h, Xlout, h->tmp, cnt)) != FEAST_OK) return s;
  }
  CK(cudaStreamSynchronize(h->st));
  if (m_found) *m_found = k;
  st.iters = it;
  st.m_found = k;
  st.max_res = max_res;
  st.normA = norm_of(h);
  st.t_filter_ms = h->t_filter;
  st.t_rr_ms = h->t_rr;
  if (h->opt.timing) {
    cudaEventRecord(h->ev[3], h->st);
    st.t_total_ms = ev_ms(h, 2, 3);
  }
  fill_shift_stats(h, &st);
  if (stats) *stats = st;
  // every Ritz value of the subspace inside C: m0 does not exceed the count
  int inside_all = 0;
  for (int i = 0; i < m; ++i) {
    const zc l = h->h_lam[i];
    if (std::isfinite(l.real()) && std::isfinite(l.imag()) && inside_ellipse(h, l)) ++inside_all;
  }
  if (inside_all == m) return FEAST_ERR_M0_TOO_SMALL;
  return converged ? FEAST_OK : FEAST_ERR_NOCONV;
}

}  // extern "C"

extern "C" {

feast_status feast_emulated_zgemm(int64_t n, int64_t m, const feast_z* A, int64_t lda, int op, const feast_z* X,
                                  int64_t ldx, feast_z* C, int64_t ldc, void* stream) {
  if (n < 1 || m < 1 || m > 4096 || !A || !X || !C || lda < n || ldx < n || ldc < n || (op != OP_N && op != OP_C))
    return FEAST_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::vector<void*> mem;
  auto release = [&](feast_status s) {
    cudaStreamSynchronize(st);
    for (void* p : mem) cudaFree(p);
    return s;
  };
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
    mem.push_back(p);
    return p;
  };
  double2* dA = static_cast<double2*>(alloc((size_t)n * n * sizeof(double2)));
  double2* dX = static_cast<double2*>(alloc((size_t)n * m * sizeof(double2)));
  double2* dC = static_cast<double2*>(alloc((size_t)n * m * sizeof(double2)));
  void* opb = alloc(oz_operator_bytes((int)n));
  void* wb = alloc(oz_work_bytes((int)n, (int)m));
  unsigned* flags = static_cast<unsigned*>(alloc(64));
  if (!dA || !dX || !dC || !opb || !wb || !flags) return release(FEAST_ERR_ALLOC);
  if (cudaMemcpy2DAsync(dA, n * sizeof(double2), A, lda * sizeof(double2), n * sizeof(double2), n, cudaMemcpyDefault,
                        st) != cudaSuccess ||
      cudaMemcpy2DAsync(dX, n * sizeof(double2), X, ldx * sizeof(double2), n * sizeof(double2), m, cudaMemcpyDefault,
                        st) != cudaSuccess ||
      cudaMemsetAsync(flags, 0, 64, st) != cudaSuccess)
    return release(FEAST_ERR_CUDA);
  OzOperator L;
  OzWork w;
  oz_operator_layout(opb, (int)n, &L);
  oz_work_layout(wb, (int)n, (int)m, &w);
  if (oz_make_operator(dA, n, op, L, st) != cudaSuccess) return release(FEAST_ERR_CUDA);
  if (oz_apply(L, dX, n, (int)m, dC, n, w, flags, st) != cudaSuccess) return release(FEAST_ERR_CUDA);
  if (cudaMemcpy2DAsync(C, ldc * sizeof(double2), dC, n * sizeof(double2), n * sizeof(double2), m, cudaMemcpyDefault,
                        st) != cudaSuccess)
    return release(FEAST_ERR_CUDA);
  unsigned f = 0;
  if (cudaMemcpyAsync(&f, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return release(FEAST_ERR_CUDA);
  return release(f & DEVFLAG_TIMEOUT ? FEAST_ERR_DEVICE_TIMEOUT : FEAST_OK);
}

feast_status feast_orthonormalize(int64_t n, int64_t m, feast_z* Q, int64_t ldq, void* stream) {
  if (n < 1 || m < 1 || m > 256 || m > n || !Q || ldq < n) return FEAST_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double2* dQ = nullptr;
  void* scratch = nullptr;
  unsigned* flags = nullptr;
  auto release = [&](feast_status s) {
    cudaStreamSynchronize(st);
    cudaFree(dQ);
    cudaFree(scratch);
    cudaFree(flags);
    return s;
  };
  if (cudaMalloc(&dQ, (size_t)n * m * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&scratch, orth_scratch_bytes((int)n, (int)m)) != cudaSuccess ||
      cudaMalloc(&flags, 64) != cudaSuccess)
    return release(FEAST_ERR_ALLOC);
  if (cudaMemcpy2DAsync(dQ, n * sizeof(double2), Q, ldq * sizeof(double2), n * sizeof(double2), m, cudaMemcpyDefault,
                        st) != cudaSuccess ||
      cudaMemsetAsync(flags, 0, 64, st) != cudaSuccess)
    return release(FEAST_ERR_CUDA);
  if (orth_cgs2(dQ, (int)n, (int)m, scratch, flags, st) != cudaSuccess) return release(FEAST_ERR_CUDA);
  if (cudaMemcpy2DAsync(Q, ldq * sizeof(double2), dQ, n * sizeof(double2), n * sizeof(double2), m, cudaMemcpyDefault,
                        st) != cudaSuccess)
    return release(FEAST_ERR_CUDA);
  unsigned f = 0;
  if (cudaMemcpyAsync(&f, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return release(FEAST_ERR_CUDA);
  return release(f & DEVFLAG_TIMEOUT ? FEAST_ERR_DEVICE_TIMEOUT : FEAST_OK);
}

}  // extern "C"
