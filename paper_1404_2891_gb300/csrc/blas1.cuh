// Element-wise and column-wise kernels of the filter and Rayleigh-Ritz steps.
#pragma once
#include "common.cuh"

// S_k = phi_k B - A for k = 0..q-1 (B = I when B == nullptr), written in T.
template <typename T>
cudaError_t form_shifted(const double2* A, long long lda, const double2* B, long long ldb,
                         const double2* z, int q, int n, cplx<T>* S, long long strideS, cudaStream_t s);

// The summation tree of the accumulation: the shifts are split into leaves
// (b[j] .. b[j+1]-1, at most 8), each leaf summed in order of the shift, and
// the leaves combined pairwise level by level ((0+1)+(2+3))+((4+5)+(6+7)).
// A handle that owns an aligned range of the contour's eight leaves computes
// the subtree of that range, so partial sums of several processes combine to
// the same bits as one process (accumulate_tree_combine).
struct AccTree {
  int nleaf = 1;   // 1, 2, 4 or 8
  int b[9] = {0};  // local leaf boundaries, b[nleaf] = q
};
AccTree acc_tree_single(int q);

// Q[r, i] = tree_b(coef[b*m + i] * Xs_b[rowmap_b(r), i]) + c0[i] * Y[r, i]
// (Y and c0 may be null; rowmap may be null = identity).
template <typename T>
cudaError_t accumulate(const cplx<T>* Xs, const AccTree& t, int n, int m, const double2* coef, const double2* c0,
                       const double2* Y, const int32_t* rowmap, double2* Q, cudaStream_t s);

// Real pencils (conjugate node pairs share one factor): X_b is n x 2m, its
// second half solved for conj(R);  Q[r, i] = sum_b (coef[b*m + i] X_b[rr, i] +
// coefc[b*m + i] conj(X_b[rr, m + i])) + c0[i] Y[r, i], b in order.
template <typename T>
cudaError_t accumulate_conj_pairs(const cplx<T>* Xs, int q, int n, int m, const double2* coef, const double2* coefc,
                                  const double2* c0, const double2* Y, const int32_t* rowmap, double2* Q,
                                  cudaStream_t s);

// Q = the top levels of the tree over nparts (1, 2, 4 or 8) partial blocks P_j
// (n x m each, consecutive in P), then + c0 .* Y (c0, Y may be null).
cudaError_t accumulate_tree_combine(const double2* P, int nparts, int n, int m, const double2* c0, const double2* Y,
                                    double2* Q, cudaStream_t s);

// R[:, i] = use_res[i] ? E[:, i] : F[:, i]
cudaError_t select_columns(const double2* E, const double2* F, const int* use_res, int n, int m,
                           double2* R, cudaStream_t s);

// Column 2-norms: nrm[i] = ||X[:, i]||_2
cudaError_t column_norms(const double2* X, int n, int m, double* nrm, cudaStream_t s);

// X[:, i] *= f(i) for up to three blocks sharing the scale: scale[i] = 1 / nrm[i] (mode 0)
// or 1 / conj(d[i]) (mode 1, d complex).
cudaError_t scale_columns_inv(double2* X0, double2* X1, double2* X2, int n, int m, const double* nrm,
                              const double2* d, cudaStream_t s);

// E = AX - BX diag(lam) (conj_lam: diag(conj(lam))), res[i] = ||E[:, i]||_2 / (xn ? xn[i] : 1)
cudaError_t residual_columns(const double2* AX, const double2* BX, const double2* lam, int conj_lam, int n,
                             int m, double2* E, double* res, const double* xn, cudaStream_t s);

// d[i] = X[:, i]^H Y[:, i]
cudaError_t column_dots(const double2* X, const double2* Y, int n, int m, double2* d, cudaStream_t s);


// dst = conj(src) (count complex values)
cudaError_t conj_copy(const double2* src, double2* dst, size_t count, cudaStream_t s);

// Identity m x m
cudaError_t set_identity(double2* M, int m, cudaStream_t s);

// out[:, c] = src[:, idx[c]] for c < k, zero for c >= k (m columns of n rows)
cudaError_t gather_columns(const double2* src, const int* idx, int k, int n, int m, double2* out,
                           cudaStream_t s);

// x <- x / ||x||, *nrm = ||x|| (single vector of length n)
cudaError_t normalize_vector(double2* x, int n, double* nrm, cudaStream_t s);

// d[b] = sum_{i,s} conj(V[i,s]) X_b[i,s] for each of the q solution blocks X_b (n x S),
// summed in a fixed order (one block per shift).
template <typename T>
cudaError_t probe_dots(const double2* V, const cplx<T>* X, int n, int S, int q, double2* d, cudaStream_t s);

// mu[k] = (1/S) sum_b w[b] ((z[b] - c)/R)^k d[b], k = 0..kmax
cudaError_t moments_combine(const double2* d, const double2* z, const double2* w, double2 c, double R, int q,
                            int kmax, int S, double2* mu, cudaStream_t s);

// flags |= NONFINITE if any entry of X (count complex values) is NaN or Inf
cudaError_t check_finite(const double2* X, size_t count, unsigned* flags, cudaStream_t s);
