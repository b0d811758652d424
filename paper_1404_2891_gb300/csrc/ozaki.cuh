// FP64-accurate complex products on the BF16 tensor cores by exact integer
// slicing (the error-free splitting of Ozaki et al.).
//
// A complex product C = op(A) X (A n x n, X n x m) is taken in its real form
// C~ = L U~: L is the 2n x 2n real matrix that expands each entry a of op(A)
// into [[Re a, -Im a], [Im a, Re a]], U~ stacks Re and Im of X's rows, and
// C~'s rows 2i, 2i+1 are Re and Im of C's row i.
//
// Every row r of L is scaled by 2^-e_r (|L[r, :]| < 2^e_r) and cut into s
// signed integer digits of beta bits: L[r, k] = 2^e_r sum_i d_i[r, k] 2^(-(i+1) beta)
// + remainder (the digits of L are bit fields of the significand shifted to
// s beta bits, rounded at the last one; those of U~ come from repeated
// rounding, t <- 2^beta t - rint(2^beta t)); likewise every column of U~ with
// its own exponent f_c.  With
// K 2^(2 beta) <= 2^24 every digit product P_ij = D_i E_j (a BF16 tensor-core
// GEMM with FP32 accumulation) is exact, and
//     C~[r, c] = 2^(e_r + f_c) sum_{i + j <= s + 1} 2^(-(i + j) beta) P_ij[r, c]
// is summed in FP64.  The dropped terms are below 2^(-(s+1) beta) K of the
// row and column scales; s beta >= 50 keeps C~ at FP64-level accuracy.
//
// The digits of a fixed operator (A, A^H, B, B^H of a handle) are made once;
// the digits of X are made per product.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

struct OzOperator {
  __nv_bfloat16* D = nullptr;  // s x M x Kp digits, rows K-contiguous (Kp = K rounded up to 64)
  int* e = nullptr;            // M row exponents
  int n = 0, M = 0, K = 0, Kp = 0, s = 0, beta = 0;
};

struct OzWork {               // scratch of one product shape (sized by oz_work_bytes)
  __nv_bfloat16* E = nullptr; // s x m x Kp digits of X
  int* f = nullptr;           // m column exponents
  float* P = nullptr;         // s x M x NP digit-pair products (NP = s m rounded up to 32)
};

int oz_beta(int K);
int oz_slices(int beta);
size_t oz_operator_bytes(int n);        // D + e for order n
size_t oz_work_bytes(int n, int m);     // E + f + P for order n and m columns
// Carve an operator / a work area out of one device allocation of the sizes above.
void oz_operator_layout(void* base, int n, OzOperator* L);
void oz_work_layout(void* base, int n, int m, OzWork* w);

// Digits of op(A) (opA = OP_N or OP_C); A complex128 column-major n x n (lda).
cudaError_t oz_make_operator(const double2* A, long long lda, int opA, OzOperator& L, cudaStream_t s);
// C (n x m, ldc) = op(A) X (X n x m, ldx), FP64-accurate.  flags: DEVFLAG_TIMEOUT on a
// bounded-wait expiry in the tensor-core kernel.  gate (device, nullable): when
// *gate == 0 every kernel of the product returns at once (C untouched).
cudaError_t oz_apply(const OzOperator& L, const double2* X, long long ldx, int m, double2* C, long long ldc,
                     const OzWork& w, unsigned* flags, cudaStream_t s, const int* gate = nullptr);
