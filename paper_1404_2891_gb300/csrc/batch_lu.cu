// Persistent factor-and-solve kernel of the batched path: every shifted
// matrix S = z_j I - A_p of every pencil of the batch (Eq. Rasp's systems for
// many pencils at once) is factored with partial pivoting and solved for its
// pencil's right-hand sides, all in ONE launch.
//
// Each CTA pulls tasks from a device queue (one atomic counter over a task
// list that the host orders topologically by critical path, longest pencils
// first).  The tasks of one matrix are the nodes of the right-looking tiled
// LU with 64 x 64 tiles:
//   PANEL(k)     factor block column k (rows 64k..N) with partial pivoting
//   UPDATE(k,j)  apply panel k's row interchanges to block column j, solve
//                U_kj = L_kk^{-1} A_kj, then A_rj -= L_rk U_kj for r > k
//   LSWAP(j)     apply the later panels' interchanges to the L part of
//                block column j (so that P S = L U in the usual layout)
//   SOLVE(c)     X = U^{-1} L^{-1} P R for 32 right-hand sides
// A task waits for its predecessors through acquire loads of per-block-column
// counters that the producers publish with release stores.  Every wait is
// bounded (%globaltimer, 2 s): on expiry the CTA sets DEVFLAG_TIMEOUT and all
// CTAs leave the queue.  Because tasks are fetched in list order and every
// dependency points to an earlier task, the earliest unfinished task always
// belongs to a running CTA, so the queue makes progress without co-residency.
//
// Arithmetic is complex64 (FFMA): tiles are staged in shared memory with
// cp.async (L2 only, so data written by other CTAs is never read through a
// stale L1 line), each thread owns a 4 x 4 (update) or 4 x 2 (solve) block of
// the output tile, and the 64 x 64 triangular solves run one warp per 8 (or 4)
// columns with shuffles and no block barriers.
#include "batch.cuh"
#include "panel_ll.cuh"

namespace {

constexpr int NT = 256;  // threads per CTA
constexpr int TT = BATCH_TILE * BATCH_TILE;

struct Shared {
  int task, ok;
  int tmp[BATCH_MAXMV];
  PanelShared ps;
};

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Thread 0 only: wait until *p >= v.  False after the time limit or when
// another CTA has already given up.
__device__ bool wait_ge(const int* p, int v, unsigned* flags, unsigned long long limit) {
  if (ld_acquire(p) >= v) return true;
  const unsigned long long t0 = gtime();
  for (;;) {
    __nanosleep(64);
    if (ld_acquire(p) >= v) return true;
    if (*(volatile unsigned*)flags & DEVFLAG_TIMEOUT) return false;
    if (gtime() - t0 > limit) {
      atomicOr(flags, (unsigned)DEVFLAG_TIMEOUT);
      return false;
    }
  }
}

// 64 rows x ncols columns of a column-major matrix (ld in elements) into a
// shared tile with column stride 64.  Rows start at an even index and ld is a
// multiple of 64, so every 16-byte chunk is aligned.
__device__ __forceinline__ void tile_load_async(float2* dst, const float2* src, long long ld, int ncols) {
  for (int c = threadIdx.x; c < ncols * 32; c += NT) {
    const int col = c >> 5, part = c & 31;
    cp_async16(dst + col * 64 + part * 2, src + (size_t)col * ld + part * 2);
  }
}

// C (64 x 16 NJ, global, ld) -= A (64 x 64, shared) * B (64 x 16 NJ, shared);
// columns >= nvalid of C are left alone.
template <int NJ>
__device__ __forceinline__ void tile_gemm_sub(float2* C, long long ldc, const float2* As, const float2* Bs,
                                              int nvalid) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float2 cv[4][NJ], acc[4][NJ];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int col = ty + 16 * j;
      cv[i][j] = col < nvalid ? __ldcg(C + (tx + 16 * i) + (size_t)col * ldc) : make_float2(0.f, 0.f);
      acc[i][j] = make_float2(0.f, 0.f);
    }
#pragma unroll 8
  for (int k = 0; k < 64; ++k) {
    float2 av[4], bv[NJ];
#pragma unroll
    for (int i = 0; i < 4; ++i) av[i] = As[k * 64 + tx + 16 * i];
#pragma unroll
    for (int j = 0; j < NJ; ++j) bv[j] = Bs[(ty + 16 * j) * 64 + k];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < NJ; ++j) cfma<float>(acc[i][j], av[i], bv[j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int col = ty + 16 * j;
      if (col < nvalid) C[(tx + 16 * i) + (size_t)col * ldc] = csub<float>(cv[i][j], acc[i][j]);
    }
}

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// X (64 x 8 CPW columns in shared memory, column stride 64) <- L^{-1} X with L
// unit lower triangular (shared, column-major).  Warp w owns columns
// w, w + 8, ...; lane l holds rows l and l + 32.
template <int CPW>
__device__ __forceinline__ void trsm_lower_unit(const float2* Ls, float2* Xs) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float2 x0[CPW], x1[CPW];
#pragma unroll
  for (int c = 0; c < CPW; ++c) {
    x0[c] = Xs[(w + 8 * c) * 64 + lane];
    x1[c] = Xs[(w + 8 * c) * 64 + lane + 32];
  }
  for (int t = 0; t < 63; ++t) {
    const float2 l0 = Ls[t * 64 + lane], l1 = Ls[t * 64 + lane + 32];
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      const float2 xt = shfl2(t < 32 ? x0[c] : x1[c], t & 31);
      if (lane > t) x0[c] = csub<float>(x0[c], cmul<float>(l0, xt));
      if (lane + 32 > t) x1[c] = csub<float>(x1[c], cmul<float>(l1, xt));
    }
  }
#pragma unroll
  for (int c = 0; c < CPW; ++c) {
    Xs[(w + 8 * c) * 64 + lane] = x0[c];
    Xs[(w + 8 * c) * 64 + lane + 32] = x1[c];
  }
}

// X <- U^{-1} X with U upper triangular (non-unit diagonal), same layout.
template <int CPW>
__device__ __forceinline__ void trsm_upper(const float2* Us, float2* Xs) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float2 x0[CPW], x1[CPW];
#pragma unroll
  for (int c = 0; c < CPW; ++c) {
    x0[c] = Xs[(w + 8 * c) * 64 + lane];
    x1[c] = Xs[(w + 8 * c) * 64 + lane + 32];
  }
  for (int t = 63; t >= 0; --t) {
    const float2 dinv = crecip<float>(Us[t * 64 + t]);
    const float2 u0 = Us[t * 64 + lane], u1 = Us[t * 64 + lane + 32];
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      if (t < 32) {
        if (lane == t) x0[c] = cmul<float>(x0[c], dinv);
      } else {
        if (lane == t - 32) x1[c] = cmul<float>(x1[c], dinv);
      }
      const float2 xt = shfl2(t < 32 ? x0[c] : x1[c], t & 31);
      if (lane < t) x0[c] = csub<float>(x0[c], cmul<float>(u0, xt));
      if (lane + 32 < t) x1[c] = csub<float>(x1[c], cmul<float>(u1, xt));
    }
  }
#pragma unroll
  for (int c = 0; c < CPW; ++c) {
    Xs[(w + 8 * c) * 64 + lane] = x0[c];
    Xs[(w + 8 * c) * 64 + lane + 32] = x1[c];
  }
}

// Rows r0 + dst[e] <- rows r0 + src[e] of the 64 columns starting at c0 (one
// panel's moved-row list), staged through shared memory.
__device__ void apply_moves(float2* A, int N, int r0, int c0, const int* mvp, float2* stage) {
  const int cnt = __ldcg(mvp);
  if (cnt <= 0) return;
  for (int idx = threadIdx.x; idx < cnt * 64; idx += NT) {
    const int e = idx % cnt, c = idx / cnt;
    const int src = __ldcg(mvp + 2 + 2 * e);
    stage[idx] = __ldcg(A + (size_t)(r0 + src) + (size_t)(c0 + c) * N);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < cnt * 64; idx += NT) {
    const int e = idx % cnt, c = idx / cnt;
    const int dst = __ldcg(mvp + 1 + 2 * e);
    A[(size_t)(r0 + dst) + (size_t)(c0 + c) * N] = stage[idx];
  }
  __syncthreads();
}

// ---------------------------------------------------------------- PANEL
// The shared left-looking panel (panel_ll.cuh), then the batch bookkeeping:
// the moved-row list for the update and fix-up tasks, the release of the
// panel, and after the last panel the composed row permutation.
template <int GW>
__device__ void panel_task(const BatchLuArgs& a, const BMat& M, int mat, int k, char* smem, int gcap, Shared& sh) {
  const int tid = threadIdx.x;
  const int N = M.N, r0 = k * 64;
  float2* A = a.S + M.soff;
  float2* Lt = reinterpret_cast<float2*>(smem);
  float2* G = Lt + TT;
  int* pl = reinterpret_cast<int*>(G + gcap);
  panel_ll<GW, NT>(A, N, N, r0, 64, a.piv + M.poff + r0, a.info + mat, a.flags, Lt, G, pl, sh.ps);
  const int cnt = sh.ps.cnt;
  int* mvp = a.mv + (size_t)(M.coff + k) * BATCH_MVSTRIDE;
  for (int e = tid; e < cnt; e += NT) {
    mvp[1 + 2 * e] = sh.ps.mvd[e];
    mvp[2 + 2 * e] = sh.ps.mvs[e];
  }
  if (tid == 0) mvp[0] = cnt;
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    st_release(a.pdone + M.coff + k, 1);
  }
  if (k != M.nb - 1) return;
  // last panel: compose the whole row permutation from the panels' lists
  int* P = pl;
  for (int r = tid; r < N; r += NT) P[r] = r;
  __syncthreads();
  for (int kk = 0; kk < M.nb; ++kk) {
    const int* lst = a.mv + (size_t)(M.coff + kk) * BATCH_MVSTRIDE;
    const int c2 = __ldcg(lst);
    const int rb = 64 * kk;
    for (int e = tid; e < c2; e += NT) sh.tmp[e] = P[rb + __ldcg(lst + 2 + 2 * e)];
    __syncthreads();
    for (int e = tid; e < c2; e += NT) P[rb + __ldcg(lst + 1 + 2 * e)] = sh.tmp[e];
    __syncthreads();
  }
  for (int r = tid; r < N; r += NT) a.perm[M.poff + r] = P[r];
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    red_release_add(a.fcnt + mat, 1);
  }
}

// ---------------------------------------------------------------- UPDATE
__device__ void update_task(const BatchLuArgs& a, const BMat& M, int k, int j, char* smem) {
  const int N = M.N, nb = M.nb, r0 = 64 * k, cj = 64 * j;
  float2* A = a.S + M.soff;
  float2* Ls = reinterpret_cast<float2*>(smem);
  float2* Us = Ls + TT;
  float2* As = Us + TT;  // two tiles; also the staging area of the interchanges
  apply_moves(A, N, r0, cj, a.mv + (size_t)(M.coff + k) * BATCH_MVSTRIDE, As);
  tile_load_async(Ls, A + r0 + (size_t)r0 * N, N, 64);
  tile_load_async(Us, A + r0 + (size_t)cj * N, N, 64);
  cp_commit();
  tile_load_async(As, A + (r0 + 64) + (size_t)r0 * N, N, 64);  // j > k, so row tile k+1 exists
  cp_commit();
  cp_wait<1>();
  __syncthreads();
  trsm_lower_unit<8>(Ls, Us);
  __syncthreads();
  for (int idx = threadIdx.x; idx < TT; idx += NT) {
    const int c = idx >> 6, r = idx & 63;
    A[(size_t)(r0 + r) + (size_t)(cj + c) * N] = Us[idx];
  }
  for (int rt = k + 1; rt < nb; ++rt) {
    const int buf = (rt - k - 1) & 1;
    if (rt + 1 < nb) {
      tile_load_async(As + (buf ^ 1) * TT, A + 64 * (rt + 1) + (size_t)r0 * N, N, 64);
      cp_commit();
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    tile_gemm_sub<4>(A + 64 * rt + (size_t)cj * N, N, As + buf * TT, Us, 64);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(a.cver + M.coff + j, k + 1);
  }
}

// ---------------------------------------------------------------- LSWAP
__device__ void lswap_task(const BatchLuArgs& a, const BMat& M, int mat, int j, char* smem) {
  float2* A = a.S + M.soff;
  float2* stage = reinterpret_cast<float2*>(smem) + 2 * TT;
  for (int kk = j + 1; kk < M.nb; ++kk)
    apply_moves(A, M.N, 64 * kk, 64 * j, a.mv + (size_t)(M.coff + kk) * BATCH_MVSTRIDE, stage);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    red_release_add(a.fcnt + mat, 1);
  }
}

// ---------------------------------------------------------------- SOLVE
__device__ void solve_task(const BatchLuArgs& a, const BMat& M, int ch, char* smem) {
  const int N = M.N, n = M.n, nb = M.nb;
  const int c0 = ch * BATCH_SOLVE_W, w = min(BATCH_SOLVE_W, M.m - c0);
  if (w <= 0) return;
  const float2* A = a.S + M.soff;
  float2* X = a.X + M.xoff + (size_t)c0 * N;
  const double2* Rp = a.R + M.roff + (size_t)c0 * n;
  const int* P = a.perm + M.poff;
  float2* Lt = reinterpret_cast<float2*>(smem);
  float2* Ys = Lt + TT;  // 64 x 32
  float2* As = Lt + 2 * TT;
  for (int idx = threadIdx.x; idx < N * w; idx += NT) {
    const int c = idx / N, r = idx - c * N;
    float2 v = make_float2(0.f, 0.f);
    if (r < n) {
      const int pr = min(max(__ldcg(P + r), 0), n - 1);  // always < n: padding rows are never pivots
      const double2 d = Rp[(size_t)pr + (size_t)c * n];
      v = make_float2((float)d.x, (float)d.y);
    }
    X[(size_t)r + (size_t)c * N] = v;
  }
  for (int idx = threadIdx.x; idx < (BATCH_SOLVE_W - w) * 64; idx += NT) Ys[w * 64 + idx] = make_float2(0.f, 0.f);
  __syncthreads();
  // forward: L y = P r
  for (int t = 0; t < nb; ++t) {
    const int rt = 64 * t;
    tile_load_async(Lt, A + rt + (size_t)rt * N, N, 64);
    tile_load_async(Ys, X + rt, N, w);
    cp_commit();
    if (t + 1 < nb) {
      tile_load_async(As, A + (rt + 64) + (size_t)rt * N, N, 64);
      cp_commit();
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    trsm_lower_unit<4>(Lt, Ys);
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * 64; idx += NT) X[(size_t)(rt + (idx & 63)) + (size_t)(idx >> 6) * N] = Ys[idx];
    __syncthreads();  // Ys is refilled by the next block row's copy
    for (int t2 = t + 1; t2 < nb; ++t2) {
      const int buf = (t2 - t - 1) & 1;
      if (t2 + 1 < nb) {
        tile_load_async(As + (buf ^ 1) * TT, A + 64 * (t2 + 1) + (size_t)rt * N, N, 64);
        cp_commit();
        cp_wait<1>();
      } else {
        cp_wait<0>();
      }
      __syncthreads();
      tile_gemm_sub<2>(X + 64 * t2, N, As + buf * TT, Ys, w);
      __syncthreads();
    }
  }
  // backward: U x = y
  for (int t = nb - 1; t >= 0; --t) {
    const int rt = 64 * t;
    tile_load_async(Lt, A + rt + (size_t)rt * N, N, 64);
    tile_load_async(Ys, X + rt, N, w);
    cp_commit();
    if (t > 0) {
      tile_load_async(As, A + (size_t)rt * N, N, 64);
      cp_commit();
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    trsm_upper<4>(Lt, Ys);
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * 64; idx += NT) X[(size_t)(rt + (idx & 63)) + (size_t)(idx >> 6) * N] = Ys[idx];
    __syncthreads();  // Ys is refilled by the next block row's copy
    for (int t2 = 0; t2 < t; ++t2) {
      const int buf = t2 & 1;
      if (t2 + 1 < t) {
        tile_load_async(As + (buf ^ 1) * TT, A + 64 * (t2 + 1) + (size_t)rt * N, N, 64);
        cp_commit();
        cp_wait<1>();
      } else {
        cp_wait<0>();
      }
      __syncthreads();
      tile_gemm_sub<2>(X + 64 * t2, N, As + buf * TT, Ys, w);
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(NT, 1) k_batch_lu(BatchLuArgs a, int gcap) {
  extern __shared__ __align__(16) char smem[];
  __shared__ Shared sh;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      int t = atomicAdd(a.head, 1);
      if (*(volatile unsigned*)a.flags & DEVFLAG_TIMEOUT) t = a.ntasks;
      sh.task = t;
    }
    __syncthreads();
    const int t = sh.task;
    if (t >= a.ntasks) return;
    const int4 tk = a.tasks[t];
    const BMat M = a.mats[tk.y];
    if (tid == 0) {
      bool ok = true;
      switch (tk.x) {
        case BT_PANEL: ok = tk.z == 0 || wait_ge(a.cver + M.coff + tk.z, tk.z, a.flags, a.wait_ns); break;
        case BT_UPDATE:
          ok = wait_ge(a.pdone + M.coff + tk.z, 1, a.flags, a.wait_ns) &&
               (tk.z == 0 || wait_ge(a.cver + M.coff + tk.w, tk.z, a.flags, a.wait_ns));
          break;
        case BT_LSWAP: ok = wait_ge(a.pdone + M.coff + M.nb - 1, 1, a.flags, a.wait_ns); break;
        default: ok = !a.active[M.pencil] || wait_ge(a.fcnt + tk.y, M.nb, a.flags, a.wait_ns); break;
      }
      sh.ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!sh.ok) return;
    switch (tk.x) {
      case BT_PANEL:
        switch (panel_group_width(M.N - 64 * tk.z, gcap)) {
          case 8: panel_task<8>(a, M, tk.y, tk.z, smem, gcap, sh); break;
          case 4: panel_task<4>(a, M, tk.y, tk.z, smem, gcap, sh); break;
          case 2: panel_task<2>(a, M, tk.y, tk.z, smem, gcap, sh); break;
          default: panel_task<1>(a, M, tk.y, tk.z, smem, gcap, sh); break;
        }
        break;
      case BT_UPDATE: update_task(a, M, tk.z, tk.w, smem); break;
      case BT_LSWAP: lswap_task(a, M, tk.y, tk.w, smem); break;
      default:
        if (a.active[M.pencil]) solve_task(a, M, tk.w, smem);
        break;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- batch helpers
// One CTA row per pencil: each entry of A_p is read once and written into all
// of the pencil's shifted matrices (z_k - a, the padding as identity).
__global__ void k_batch_form_p(const double2* A, const GrpDesc* pd, const BMat* mats, const double2* z, float2* S) {
  __shared__ long long s_off[256];
  const GrpDesc d = pd[blockIdx.y];
  const int q = min(d.q, 256);
  for (int k = threadIdx.x; k < q; k += blockDim.x) s_off[k] = mats[d.mat0 + k].soff;
  __syncthreads();
  const int N = mats[d.mat0].N, n = d.n;
  const double2* Ap = A + d.onn;
  for (int c = blockIdx.x; c < N; c += gridDim.x)
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      const bool in = r < n && c < n;
      double2 av = make_double2(0.0, 0.0);
      if (in) av = Ap[(size_t)r + (size_t)c * n];
      const size_t idx = (size_t)r + (size_t)c * N;
      for (int k = 0; k < q; ++k) {
        float2 v;
        if (in) {
          // the same arithmetic as the per-matrix form: FP64 difference, then rounding
          const double2 zz = z[d.mat0 + k];
          v = make_float2((float)((r == c ? zz.x : 0.0) - av.x), (float)((r == c ? zz.y : 0.0) - av.y));
        } else {
          v = make_float2(r == c ? 1.f : 0.f, 0.f);
        }
        S[s_off[k] + idx] = v;
      }
    }
}

__global__ void k_batch_form(const double2* A, const GrpDesc* pd, const BMat* mats, const double2* z, float2* S) {
  const BMat M = mats[blockIdx.y];
  const GrpDesc d = pd[M.pencil];
  const double2 zz = z[blockIdx.y];
  const double2* Ap = A + d.onn;
  float2* Sm = S + M.soff;
  // columns strided over the CTAs, rows over the threads (coalesced on both sides)
  for (int c = blockIdx.x; c < M.N; c += gridDim.x) {
    for (int r = threadIdx.x; r < M.N; r += blockDim.x) {
      double2 v = make_double2(r == c ? 1.0 : 0.0, 0.0);
      if (r < M.n && c < M.n) {
        const double2 av = Ap[(size_t)r + (size_t)c * M.n];
        v = make_double2((r == c ? zz.x : 0.0) - av.x, (r == c ? zz.y : 0.0) - av.y);
      }
      Sm[(size_t)r + (size_t)c * M.N] = make_float2((float)v.x, (float)v.y);
    }
  }
}

__global__ void k_batch_acc(const float2* X, const BMat* mats, const GrpDesc* pd, const double2* coef,
                            const double2* c0, const double2* Y, const int* active, double2* Q) {
  const int p = blockIdx.y;
  if (!active[p]) return;
  const GrpDesc d = pd[p];
  const size_t total = (size_t)d.n * d.m;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % d.n), i = (int)(idx / d.n);
    double2 acc = make_double2(0.0, 0.0);
    if (c0) acc = cmul<double>(c0[d.om + i], Y[d.onm + idx]);
    for (int s = 0; s < d.q; ++s) {
      const BMat& M = mats[d.mat0 + s];
      const float2 x = X[M.xoff + (size_t)i * M.N + r];
      cfma<double>(acc, coef[d.oqm + (size_t)s * d.m + i], make_double2(x.x, x.y));
    }
    Q[d.onm + idx] = acc;
  }
}

__global__ void k_batch_select(const double2* E, const double2* F, const int* use, const GrpDesc* pd,
                               const int* active, double2* R) {
  const int p = blockIdx.y;
  if (!active[p]) return;
  const GrpDesc d = pd[p];
  const size_t total = (size_t)d.n * d.m;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / d.n);
    R[d.onm + idx] = use[d.om + i] ? E[d.onm + idx] : F[d.onm + idx];
  }
}

__device__ double bsum256(double v) {
  __shared__ double red[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += red[k];
  return t;
}

// nrm[i] = ||X[:, i]||, then X[:, i] and Y[:, i] scaled by 1 / nrm[i]; grid (m, pencils)
__global__ void __launch_bounds__(256) k_bnormalize(double2* X, double2* Y, const GrpDesc* pd, const int* active,
                                                    double* nrm) {
  const int p = blockIdx.y, i = blockIdx.x;
  if (!active[p] || i >= pd[p].m) return;
  const GrpDesc d = pd[p];
  double2* x = X + d.onm + (size_t)i * d.n;
  double2* y = Y ? Y + d.onm + (size_t)i * d.n : nullptr;
  double s = 0.0;
  for (int r = threadIdx.x; r < d.n; r += 256) s += cnorm2<double>(x[r]);
  s = sqrt(bsum256(s));
  const double f = s > 0.0 ? 1.0 / s : 0.0;
  for (int r = threadIdx.x; r < d.n; r += 256) {
    x[r] = cscale<double>(x[r], f);
    if (y) y[r] = cscale<double>(y[r], f);
  }
  if (threadIdx.x == 0) nrm[d.om + i] = s;
}

// E[:, i] = AX[:, i] - lam_i X[:, i], res[i] = ||E[:, i]||; grid (m, pencils)
__global__ void __launch_bounds__(256) k_bresidual(const double2* AX, const double2* X, const double2* lam,
                                                   const GrpDesc* pd, const int* active, double2* E, double* res) {
  const int p = blockIdx.y, i = blockIdx.x;
  if (!active[p] || i >= pd[p].m) return;
  const GrpDesc d = pd[p];
  const size_t off = d.onm + (size_t)i * d.n;
  const double2 l = lam[d.om + i];
  double s = 0.0;
  for (int r = threadIdx.x; r < d.n; r += 256) {
    const double2 e = csub<double>(AX[off + r], cmul<double>(X[off + r], l));
    E[off + r] = e;
    s += cnorm2<double>(e);
  }
  s = bsum256(s);
  if (threadIdx.x == 0) res[d.om + i] = sqrt(s);
}

__global__ void k_bidentity(double2* M, const GrpDesc* pd, const int* active) {
  const int p = blockIdx.y;
  if (!active[p]) return;
  const GrpDesc d = pd[p];
  const int total = d.m * d.m;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x)
    M[d.omm + idx] = make_double2((idx % d.m) == (idx / d.m) ? 1.0 : 0.0, 0.0);
}

unsigned blocks_for(size_t count) {
  const size_t b = (count + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 512 ? 512 : b));
}

}  // namespace

size_t batch_lu_gcap(int Nmax) { return (size_t)Nmax * (Nmax <= 2048 ? 8 : 4); }

size_t batch_lu_smem_bytes(int Nmax) {
  const size_t panel = batch_lu_gcap(Nmax) * sizeof(float2) + (size_t)Nmax * sizeof(int);
  const size_t other = (size_t)3 * TT * sizeof(float2);  // Us + two A tiles (update), Ys + two tiles (solve)
  return (size_t)TT * sizeof(float2) + (panel > other ? panel : other);
}

int batch_lu_grid(int Nmax) {
  const size_t smem = batch_lu_smem_bytes(Nmax);
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaFuncSetAttribute(k_batch_lu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_lu, NT, smem);
  return nsm * (per > 0 ? per : 0);
}

cudaError_t batch_lu_launch(const BatchLuArgs& a, int Nmax, int grid, cudaStream_t s) {
  if (grid < 1 || a.ntasks < 1) return cudaSuccess;
  if (Nmax < 64 || Nmax > BATCH_MAX_N || Nmax % 64) return cudaErrorInvalidValue;
  const size_t smem = batch_lu_smem_bytes(Nmax);
  cudaError_t e = cudaFuncSetAttribute(k_batch_lu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.head, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  feast_count_launch();
  k_batch_lu<<<grid, NT, smem, s>>>(a, (int)batch_lu_gcap(Nmax));
  return cudaGetLastError();
}

cudaError_t batch_form_shifted(const double2* A, const GrpDesc* pd, const BMat* mats, const double2* z, int nmat,
                               int Nmax, float2* S, cudaStream_t s, int np) {
  if (nmat < 1) return cudaSuccess;
  feast_count_launch();
  if (np > 0) {  // per pencil: A_p read once
    k_batch_form_p<<<dim3(std::min(Nmax, 512), np), 256, 0, s>>>(A, pd, mats, z, S);
    return cudaGetLastError();
  }
  dim3 grid(std::min(Nmax, 256), nmat);
  k_batch_form<<<grid, 256, 0, s>>>(A, pd, mats, z, S);
  return cudaGetLastError();
}

cudaError_t batch_accumulate(const float2* X, const BMat* mats, const GrpDesc* pd, int np, int nmax, int mmax,
                             const double2* coef, const double2* c0, const double2* Y, const int* active,
                             double2* Q, cudaStream_t s) {
  if (np < 1) return cudaSuccess;
  dim3 grid(blocks_for((size_t)nmax * mmax), np);
  feast_count_launch();
  k_batch_acc<<<grid, 256, 0, s>>>(X, mats, pd, coef, c0, Y, active, Q);
  return cudaGetLastError();
}

cudaError_t batch_select(const double2* E, const double2* F, const int* use, const GrpDesc* pd, int np, int nmax,
                         int mmax, const int* active, double2* R, cudaStream_t s) {
  if (np < 1) return cudaSuccess;
  dim3 grid(blocks_for((size_t)nmax * mmax), np);
  feast_count_launch();
  k_batch_select<<<grid, 256, 0, s>>>(E, F, use, pd, active, R);
  return cudaGetLastError();
}

cudaError_t batch_normalize(double2* X, double2* Y, const GrpDesc* pd, int np, int mmax, const int* active,
                            double* nrm, cudaStream_t s) {
  if (np < 1) return cudaSuccess;
  feast_count_launch();
  k_bnormalize<<<dim3(mmax, np), 256, 0, s>>>(X, Y, pd, active, nrm);
  return cudaGetLastError();
}

cudaError_t batch_residual(const double2* AX, const double2* X, const double2* lam, const GrpDesc* pd, int np,
                           int mmax, const int* active, double2* E, double* res, cudaStream_t s) {
  if (np < 1) return cudaSuccess;
  feast_count_launch();
  k_bresidual<<<dim3(mmax, np), 256, 0, s>>>(AX, X, lam, pd, active, E, res);
  return cudaGetLastError();
}

cudaError_t batch_identity(double2* M, const GrpDesc* pd, int np, int mmax, const int* active, cudaStream_t s) {
  if (np < 1) return cudaSuccess;
  feast_count_launch();
  k_bidentity<<<dim3(blocks_for((size_t)mmax * mmax), np), 256, 0, s>>>(M, pd, active);
  return cudaGetLastError();
}
