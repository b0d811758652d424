// Tables of the batched path: many independent pencils (each with its own
// order n, subspace size m0 and contour) solved together.  Every per-pencil
// array lives in one device arena per kind, and the kernels find their
// problem's slice through these descriptors.
#pragma once
#include "common.cuh"

// One pencil of a batch.  Offsets are in elements of the arena they index.
struct GrpDesc {
  int n = 0, m = 0, q = 0, mat0 = 0;  // order, subspace size, shifts, index of its first shifted matrix
  long long onn = 0;                  // n x n FP64 arena (A)
  long long onm = 0;                  // n x m FP64 arenas (Y, Q, AQ, X, AX, E, R)
  long long omm = 0;                  // m x m arenas (FP64 and FP32)
  long long om = 0;                   // length-m arenas
  long long oqm = 0;                  // q x m coefficient arena
  long long olog = 0;                 // byte offset into the Schur rotation-log arena
};

// One shifted matrix S = z I - A of the batch, stored in complex64 with its
// order padded to N (a multiple of 64; the padding is an identity block, which
// the factorisation leaves untouched).
struct BMat {
  long long soff = 0;  // factor arena offset (N x N, column-major, ld N)
  long long xoff = 0;  // solution arena offset (N x m, ld N)
  long long roff = 0;  // right-hand-side offset in the FP64 n x m arena (ld n)
  int N = 0, n = 0, m = 0, nb = 0;
  int coff = 0;  // offset into the per-block-column state arrays (sum of nb)
  int poff = 0;  // offset into the permutation / pivot arrays (sum of N)
  int pencil = 0, shift = 0;
};

// Task kinds of the persistent factor/solve kernel.
enum BTaskKind { BT_PANEL = 0, BT_UPDATE = 1, BT_LSWAP = 2, BT_SOLVE = 3 };

constexpr int BATCH_TILE = 64;      // tile order of the batched factorisation
constexpr int BATCH_MAXMV = 128;    // rows moved by one panel's pivoting (at most 2 x 64)
constexpr int BATCH_MVSTRIDE = 1 + 2 * BATCH_MAXMV;
constexpr int BATCH_SOLVE_W = 32;   // right-hand sides per solve task
constexpr int BATCH_MAX_N = 4096;   // largest padded order handled by the panel task

struct BatchLuArgs {
  float2* S = nullptr;          // factors
  const BMat* mats = nullptr;
  const int4* tasks = nullptr;  // {kind, matrix, k, j}
  int ntasks = 0;
  int* head = nullptr;          // task counter (zeroed before every launch)
  int* cver = nullptr;          // per block column: elimination steps applied
  int* pdone = nullptr;         // per block column: panel factored
  int* fcnt = nullptr;          // per matrix: finished row-interchange fix-ups + last panel
  int* mv = nullptr;            // per block column: moved-row list of its panel
  int* perm = nullptr;          // per matrix: row permutation, (P S)[r] = S[perm[r]]
  int* piv = nullptr;           // per matrix: LAPACK-style interchanges (0-based global rows)
  int* info = nullptr;          // per matrix: first zero pivot (1-based), 0 if none
  const double2* R = nullptr;   // right-hand sides (FP64, per pencil)
  float2* X = nullptr;          // solutions (complex64, per matrix)
  const int* active = nullptr;  // per pencil: solve tasks of inactive pencils are skipped
  unsigned* flags = nullptr;
  unsigned long long wait_ns = 2000000000ull;  // limit of each dependency wait
};

// ---- persistent factor/solve (batch_lu.cu)
// Nmax: largest padded order of the batch (multiple of 64, at most BATCH_MAX_N).
size_t batch_lu_smem_bytes(int Nmax);
int batch_lu_grid(int Nmax);  // resident CTAs on this device (0 if the kernel cannot run)
cudaError_t batch_lu_launch(const BatchLuArgs& a, int Nmax, int grid, cudaStream_t s);
// S_i = z_i I - A_p for every matrix of the batch (A_p FP64 n x n, ld n).
// np > 0: one pass per pencil (A_p read once for all its shifts); else per matrix.
cudaError_t batch_form_shifted(const double2* A, const GrpDesc* pd, const BMat* mats, const double2* z, int nmat,
                               int Nmax, float2* S, cudaStream_t s, int np = 0);
// Q_p = c0_p .* Y_p + sum_s coef_{p,s} .* X_{p,s}   (fixed order in s)
cudaError_t batch_accumulate(const float2* X, const BMat* mats, const GrpDesc* pd, int np, int nmax, int mmax,
                             const double2* coef, const double2* c0, const double2* Y, const int* active,
                             double2* Q, cudaStream_t s);
// R_p[:, i] = use_p[i] ? E_p[:, i] : F_p[:, i]
cudaError_t batch_select(const double2* E, const double2* F, const int* use, const GrpDesc* pd, int np, int nmax,
                         int mmax, const int* active, double2* R, cudaStream_t s);
// nrm_p[i] = ||X_p[:, i]||; X_p[:, i] and (if Y) Y_p[:, i] scaled by 1 / nrm_p[i]
cudaError_t batch_normalize(double2* X, double2* Y, const GrpDesc* pd, int np, int mmax, const int* active,
                            double* nrm, cudaStream_t s);
// E_p = AX_p - X_p diag(lam_p), res_p[i] = ||E_p[:, i]||
cudaError_t batch_residual(const double2* AX, const double2* X, const double2* lam, const GrpDesc* pd, int np,
                           int mmax, const int* active, double2* E, double* res, cudaStream_t s);
cudaError_t batch_identity(double2* M, const GrpDesc* pd, int np, int mmax, const int* active, cudaStream_t s);
