// Choice of the kernel that performs the LU trailing update A22 -= L21 U12.
#pragma once
#include "lu.cuh"

// Staging for the tensor-core update: bf16 high/low parts of the expanded
// L21 panel (A', 2 * rest rows) and of U12 (rest rows), K-major, 256 B rows.
// Owned by the handle; sized for order n and q shifts by tc_staging_bytes.
struct TcStaging {
  void* Ast = nullptr;       // q x 2 x (2n) x 128 bf16
  void* Bst = nullptr;       // q x 2 x n x 128 bf16
  long long rows_max = 0;    // 2n
  long long cols_max = 0;    // n
  int q = 0;
};
size_t tc_staging_bytes_A(long long n, int q);
size_t tc_staging_bytes_B(long long n, int q);

// complex128: the DMMA batched GEMM (fn = nullptr); complex64: the tcgen05
// kernel, with ctx pointing at the handle's TcStaging.
template <typename T>
void select_trailing_update(TrailingUpdateFn<T>* fn, void** ctx, TcStaging* staging);

// Off-diagonal update of a blocked triangular solve on the tensor cores:
// X[row_out : row_out + M, :] -= op(A) X[row_in : row_in + K, :] for every shift,
// A the factor block at (ar0, ac0) (opA = OP_N) or its conjugate transpose
// (OP_C: A(i,k) = conj(S[ac0 + k, ar0 + i])).  With diag_mode >= 0 the block
// X[row_in : row_in + K, :] is first solved with the diagonal block
// S[row_in : row_in + K, row_in : row_in + K] (0: unit lower L, 1: upper U,
// 2: U^H, 3: unit upper L^H) inside the staging kernel.  Returns false
// (nothing done) when the handle has no staging (lu.tc == nullptr), K > 64, or
// (with a diagonal solve) M == 0.
bool tc_solve_update(const LuBatch<float>& lu, float2* X, int m, int M, int K, int ar0, int ac0, int opA,
                     int row_out, int row_in, int diag_mode, cudaStream_t s, cudaError_t* err);
