// Batched dense complex LU with partial pivoting and the triangular solves
// that reuse it, for the q shifted systems (phi_k B - A) of Eq. Rasp.
#pragma once
#include "common.cuh"
#include "gemm.cuh"

// q matrices of order n, column-major, leading dimension ld, batch stride `stride`.
template <typename T>
struct LuBatch {
  cplx<T>* S = nullptr;
  long long ld = 0, stride = 0;
  int n = 0, q = 0;
  int32_t* piv = nullptr;   // q x n, LAPACK style (0-based): row i exchanged with piv[i]
  int32_t* perm = nullptr;  // q x n, row i of P S is row perm[i] of S
  int32_t* pinv = nullptr;  // q x n, inverse permutation: pinv[perm[i]] = i
  int* info = nullptr;      // q ints: 0 or 1 + first column with an exact zero pivot
  unsigned* flags = nullptr;
  void* tc = nullptr;       // tensor-core staging (complex64 path), or nullptr
  // mv_panels x q x LU_MV_STRIDE ints, or nullptr: each panel's moved rows
  // {count, dst[128], src[128]} (relative to the panel's first row), written by
  // the complex64 panel for the interchanges on the other columns
  int32_t* mv = nullptr;
  int mv_panels = 0;
  // the trailing update's staging kernel solves U12 = L11^{-1} A12 (in place)
  // when it stages U12, so the interchange kernel leaves that solve out
  bool u12_in_stage = false;
  // two-level LU: the inner steps see only the columns before col_end (the
  // current outer block); 0 = all n columns
  int col_end = 0;
  // complex64 panels of >= cluster_min_rows rows (0: 1024) on a cluster of four CTAs per shift
  bool panel_cluster = false;
  int cluster_min_rows = 0;
  // complex64 with moved-row lists: lu_rowmap_ints(n, q, KB) ints of row maps
  // and moved-row lists (KB the outer block, or 64 for the one-level LU), or
  // nullptr.  With them the interchanges of the later outer blocks reach the
  // finished L columns in one deferred pass at the end (each column's moved
  // rows read and written once) instead of one pass per panel
  int32_t* rowmaps = nullptr;
};
constexpr int LU_MV_STRIDE = 257;

// Trailing-update hook of panel step (k0, w): the columns c0 .. c0+nc-1 of
// the trailing block, C = S[k0+w:, c0:c0+nc] -= L21 U12[:, c0 - (k0+w) ...],
// for all shifts.  `stage` is true on the first call of a step (an
// implementation that prepares the step's operands once does it then).
// Defaults to gemm_batched<T>; the mixed path installs its tensor-core kernel.
template <typename T>
using TrailingUpdateFn = cudaError_t (*)(const LuBatch<T>& lu, int k0, int w, int c0, int nc, bool stage, void* ctx,
                                         cudaStream_t s);

// The batched-GEMM trailing update (used when no other kernel is installed).
template <typename T>
cudaError_t default_trailing_update(const LuBatch<T>& lu, int k0, int w, int c0, int nc, bool stage, void* ctx,
                                    cudaStream_t s);

// Look-ahead: after panel k, the trailing update of block column k+1 runs
// first; panel k+1 then factors on a high-priority side stream while the rest
// of step k's trailing update runs on `s` (joined through events).
template <typename T>
cudaError_t lu_factor_batched(const LuBatch<T>& lu, int nb, TrailingUpdateFn<T> upd, void* ctx,
                              cudaStream_t s);

// Two-level form (complex64 with the tensor-core updates): outer blocks of KB
// columns (a multiple of nb).  Inside an outer block the panels and their
// trailing updates touch only the block's own columns (lu.col_end); at the end
// of the block, far(lu, K0, KB) applies the block's panels to the rows K0 ..
// K0+KB of the columns beyond it (interchanges, U12 solve, updates inside the
// block's rows), and deep(lu, K0, KB) subtracts the K = KB product of the
// block's L and U from everything below and to the right of it.
using FarFn = cudaError_t (*)(const LuBatch<float>& lu, int K0, int KB, void* ctx, cudaStream_t s);
// T = -D^{-1} for the diagonal blocks block0 .. block0+nblocks-1 of size KB
// (a multiple of 64, at most 256) of every shift: D the unit lower part of the
// factor (upper = false) or its upper part with the diagonal (upper = true);
// rows and columns beyond n act as the identity.  T holds nblocks x q matrices
// KB x KB, column-major with leading dimension KB, block-major.
cudaError_t block_inverse_negated(const LuBatch<float>& lu, bool upper, int KB, int block0, int nblocks, float2* T,
                                  cudaStream_t s);
// The moved rows of the panel at k0 (its list in lu.mv) applied to the columns
// col0 .. col0+ncols-1 of every shifted matrix.
cudaError_t laswp_moved_rows(const LuBatch<float>& lu, int k0, int col0, int ncols, cudaStream_t s);
// The interchanges of all panels of the outer block [K0, K0+KB) applied to the
// columns beyond it (K0+KB .. n-1) in one launch: the panels' moved-row lists
// in order, one warp per column.
cudaError_t block_swaps_far(const LuBatch<float>& lu, int K0, int KB, cudaStream_t s);
// Size of LuBatch::rowmaps for blocks of KB columns.
size_t lu_rowmap_ints(long long n, int q, int KB);
using DeepFn = cudaError_t (*)(const LuBatch<float>& lu, int K0, int KB, void* ctx, cudaStream_t s);
cudaError_t lu_factor_two_level(const LuBatch<float>& lu, int nb, int KB, TrailingUpdateFn<float> upd, void* ctx,
                                FarFn far, DeepFn deep, void* dctx, cudaStream_t s);

// Complex64 panel of rows k0 .. n-1, columns k0 .. k0+w-1 of every shift on a
// thread-block cluster of four CTAs per shift (panel_cluster.cu); for panels of
// min_rows (0: 1024) to 8192 rows.
bool panel_cluster_applies(int rows, int w, int min_rows);
cudaError_t panel_cluster(const LuBatch<float>& lu, int k0, int w, cudaStream_t s);

// X (q x n x m, leading dimension n, batch stride n*m) overwritten with
//   side 0:  S_b^{-1} X_b          side 1:  S_b^{-H} X_b
// using the stored factors; `X` must already hold P R (side 0) or R (side 1),
// see rows_gather; the final P^T of side 1 is applied by rows_scatter.
template <typename T>
cudaError_t lu_solve_batched(const LuBatch<T>& lu, int side, cplx<T>* X, int m, int nbs,
                             cudaStream_t s);

// X_b[i, c] = R[perm_b[i], c]   (R: n x m double2, shared by all b; X in T);
// conj_dup: X_b is n x 2m and X_b[i, m + c] = conj(R[perm_b[i], c])
template <typename T>
cudaError_t rows_gather(const LuBatch<T>& lu, const double2* R, cplx<T>* X, int m, bool permute,
                        cudaStream_t s, bool conj_dup = false);
// Out_b[perm_b[i], c] = V_b[i, c]  in place through a scratch copy
template <typename T>
cudaError_t rows_scatter(const LuBatch<T>& lu, const cplx<T>* V, cplx<T>* Out, int m,
                         cudaStream_t s);
