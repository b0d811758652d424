// FP64 kernels for the reduced (m0 x m0) problem of the Rayleigh-Ritz step and
// for the orthonormal bases of the filtered blocks.
#pragma once
#include "common.cuh"
#include "batch.cuh"

// In-place orthonormalisation of the n x m block Q (ld n) by classical
// Gram-Schmidt applied twice, one cooperative launch with bounded grid barriers.
// A column that lies numerically in the span of the earlier ones (Kahan's
// twice-is-enough test) restarts from a unit vector.
// scratch: >= 2 * grid * m double2 + 4 unsigned (see orth_scratch_bytes).
size_t orth_scratch_bytes(int n, int m);
// col0: index of Q's column 0 within a larger basis (a panel of it), so that
// dependent columns of different panels restart from different unit vectors.
// f32dots: coefficients and norms from a complex64 copy of the rows, updates in
// FP64 (the span stays exact, the orthonormality is about 1e-7), for callers
// that form and invert the basis' Gram matrix in FP64 themselves.
cudaError_t orth_cgs2(double2* Q, int n, int m, void* scratch, unsigned* flags, cudaStream_t s, int col0 = 0,
                      bool f32dots = false);

// Single-CTA dense kernels on m x m column-major matrices (ld m) in global memory.
// LU with partial pivoting in place (piv: m ints).
cudaError_t small_lu(double2* M, int m, int* piv, unsigned* flags, cudaStream_t s);
// X (m x nrhs, ld m) <- M^{-1} X (trans = 0) or M^{-H} X (trans = 1) with the factors of small_lu.
cudaError_t small_lu_solve(const double2* LU, const int* piv, int m, double2* X, int nrhs, int trans,
                           cudaStream_t s);
// Schur form of the m x m matrix C (overwritten by the upper triangular T) by
// Householder reduction to Hessenberg form and shifted complex QR iterations;
// Z (m x m) receives the unitary Schur vectors (C = Z T Z^H); lam the diagonal of T.
// log: device scratch of schur_log_bytes(m) for the rotation record.  T is
// float (the fast path, refined afterwards in FP64) or double.
size_t schur_log_bytes(int m);
template <typename T>
cudaError_t small_schur(cplx<T>* C, cplx<T>* Z, cplx<T>* lam, int m, unsigned* flags, void* log, cudaStream_t s);
// Eigenvectors of the upper triangular T (V, m x m, unit diagonal entry, back substitution).
template <typename T>
cudaError_t small_trevc(const cplx<T>* Tm, cplx<T>* V, int m, cudaStream_t s);
// Vi = V^{-1} for an upper triangular m x m V (back substitution, one column per thread).
template <typename T>
cudaError_t small_triu_inv(const cplx<T>* V, cplx<T>* Vi, int m, cudaStream_t s);
cudaError_t small_triu_inv_grp(const float2* V, float2* Vi, const GrpDesc* pd, int np, int mmax, const int* active,
                               cudaStream_t s);
// One refinement sweep of an approximate eigendecomposition C ~ W Lambda W^{-1}:
// from E = W^{-1} C W, lam = diag(E) and D = I + Delta with
// Delta_ij = E_ij / (E_jj - E_ii) (i != j; 0 where |E_jj - E_ii| <= tiny * ||E||),
// so that W D is the first-order corrected eigenvector matrix.
cudaError_t eig_refine_step(const double2* E, double2* D, double2* lam, int m, cudaStream_t s);
// Element-wise precision conversions.
cudaError_t to_c64(const double2* src, float2* dst, size_t count, cudaStream_t s);
cudaError_t to_c128(const float2* src, double2* dst, size_t count, cudaStream_t s);

// ---- grouped forms: one launch for every active pencil of a batch (GrpDesc
// offsets into the n x m, m x m and length-m arenas).
// CTAs [cta0[p], cta0[p+1]) orthonormalise pencil p's block of the n x m arena;
// a cooperative launch of total_ctas = cta0[np] CTAs (at most the resident
// count: orth_grp_ctas_per_sm() per SM).  part: 2 * total_ctas * 256 double2;
// bars: 2 * np unsigned.
int orth_grp_ctas_per_sm();
cudaError_t orth_cgs2_grp(double2* Q, const GrpDesc* pd, const int* cta0, int np, int total_ctas, double2* part,
                          unsigned* bars, const int* active, unsigned* flags, cudaStream_t s);
cudaError_t small_lu_grp(double2* M, const GrpDesc* pd, int np, const int* active, int* piv, unsigned* flags,
                         cudaStream_t s);
// X_p (m x m) <- M_p^{-1} X_p (trans 0) or M_p^{-H} X_p (trans 1)
cudaError_t small_lu_solve_grp(const double2* LU, const int* piv, const GrpDesc* pd, int np, int mmax,
                               const int* active, double2* X, int trans, cudaStream_t s);
// Schur form of C_p (FP32), Schur vectors Z_p, eigenvalues lam_p; rotation logs at olog.
cudaError_t small_schur_grp(float2* C, float2* Z, float2* lam, const GrpDesc* pd, int np, int mmax,
                            const int* active, unsigned* flags, void* logs, cudaStream_t s);
cudaError_t small_trevc_grp(const float2* Tm, float2* V, const GrpDesc* pd, int np, int mmax, const int* active,
                            cudaStream_t s);
cudaError_t eig_refine_step_grp(const double2* E, double2* D, double2* lam, const GrpDesc* pd, int np,
                                const int* active, cudaStream_t s);

// gate = 1 when max |T - I| > tol (or T holds a NaN), else 0 (T = W X checks X ~ W^{-1}).
cudaError_t inverse_check(const double2* T, int m, double tol, int* gate, cudaStream_t s);
// When *gate != 0: X = W^{-1} by LU with partial pivoting (LU, piv: scratch); otherwise
// the kernel returns at once.
cudaError_t small_inverse_gated(const double2* W, double2* LU, int* piv, double2* X, int m, unsigned* flags,
                                const int* gate, cudaStream_t s);
// Grouped forms: gate[p] = active[p] && max |T_p - I| > tol; with X non-null also
// X_p = 2I - T_p (for a near-identity T_p, its inverse to O(|T_p - I|^2)).
cudaError_t inverse_check_grp(const double2* T, const GrpDesc* pd, int np, const int* active, double tol, int* gate,
                              double2* X, cudaStream_t s);
// X_p = W_p^{-1} by LU (LU, piv: arena scratch) for the pencils with gate[p] != 0.
cudaError_t small_inverse_gated_grp(const double2* W, double2* LU, int* piv, double2* X, const GrpDesc* pd, int np,
                                    unsigned* flags, const int* gate, cudaStream_t s);
// X ~ M^{-1} (FP32 accuracy, m <= 160) by Gauss-Jordan elimination with partial
// pivoting on one CTA: the start of a Newton-Schulz refinement.
cudaError_t gj_inverse32(const double2* M, int m, double2* X, cudaStream_t s);
