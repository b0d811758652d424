// Kernels of the classical mixed-precision refinement of the shifted solves:
// X_k += S_k^{-1} (R - S_k X_k), the residual in FP64, the correction solved
// with the complex64 factor of the same shift.
#pragma once
#include "common.cuh"

// X64_b[i, c] (=, or += when add) Xs_b[rowmap_b(i), c] for the q blocks
// (Xs: n x m complex64 per block; rowmap may be null = identity).
cudaError_t refine_widen(const float2* Xs, int q, int n, int m, const int32_t* rowmap, double2* X64, bool add,
                         cudaStream_t s);

// One shift: r = R - z T2 + T1 (n x m, FP64) and norms[c] = ||r[:, c]||_2, where
// T1 = A X and T2 = B X (right: S = z B - A) or T1 = A^H X, T2 = B^H X with
// z = conj(phi) (left: S^H = conj(phi) B^H - A^H).
cudaError_t refine_residual(const double2* R, const double2* T1, const double2* T2, double2 z, int n, int m,
                            double2* r, double* norms, cudaStream_t s);

// Xs_b[i, c] = r_b[perm_b(i), c] in complex64 (right side: permute; left: as is),
// one right-hand side block per shift.
cudaError_t refine_gather(const double2* r, const int32_t* perm, float2* Xs, int q, int n, int m, bool permute,
                          cudaStream_t s);
