// Deep-K trailing update of the two-level LU: C -= L U with K up to 256
// complex columns, for all q shifted matrices, on the tcgen05 tensor cores.
#pragma once
#include "common.cuh"
#include "lu.cuh"

// Split-BF16 staging of the two operands, K-major with rows of DEEP_KP bf16:
//   A' (the interleaved real form of L, 2M rows) : [shift][hi, lo][row][kk]
//   U~ (the columns of U as [Re, Im] pairs, N rows): [shift][hi, lo][col][kk]
constexpr int DEEP_KP = 512;  // 2 x 256 complex K
struct DeepStaging {
  void* Ast = nullptr;
  void* Bst = nullptr;
  long long rows_max = 0;  // 2n
  long long cols_max = 0;  // n
  int q = 0;
};
size_t deep_staging_bytes_A(long long n, int q);
size_t deep_staging_bytes_B(long long n, int q);

// One batched product C_b -= op(L)_b U_b (complex64, column-major, matrix b
// of each operand at its base + b x its batch stride):
//   C (M x N): C_b[(cr + i) + (cc + j) ldc]
//   L (M x K): opL = OP_N: L_b[(lr + i) + (lc + k) ldl];
//              opL = OP_C: conj(L_b[(lc + k) + (lr + i) ldl])  (a block of L^H)
//   U (K x N): U_b[(ur + k) + (uc + j) ldu]
// Both operands are staged before the product runs, so C may overlap U.
struct DeepGemm {
  float2* C = nullptr;
  long long ldc = 0, strc = 0;
  int cr = 0, cc = 0;
  const float2* L = nullptr;
  long long ldl = 0, strl = 0;
  int lr = 0, lc = 0, opL = 0;
  const float2* U = nullptr;
  long long ldu = 0, stru = 0;
  int ur = 0, uc = 0;
  int M = 0, N = 0, K = 0, q = 0;
  bool overwrite = false;  // C = -op(L) U instead of C -= op(L) U (C is not read)
};

// Stage L (rows 0..M; parts & 1) and/or U (columns 0..N; parts & 2) as split
// BF16 (one launch).
cudaError_t deep_stage(const DeepGemm& g, const DeepStaging& st, cudaStream_t s, int parts = 3);
// C[:, c0 : c0 + nc] -= L U[:, c0 : c0 + nc] from the staged operands
// (persistent: one CTA per SM, 128 x 256 tiles, K streamed through a
// two-stage ring, double-buffered TMEM accumulators).
cudaError_t deep_run(const DeepGemm& g, int c0, int nc, const DeepStaging& st, unsigned* flags, cudaStream_t s);
bool deep_fits(const DeepGemm& g, const DeepStaging& st);

// The deep update of the two-level LU after outer block [K0, K0+KB): every
// shifted matrix's S[K0+KB:, K0+KB:] -= S[K0+KB:, K0:K0+KB] S[K0:K0+KB, K0+KB:].
cudaError_t tc_deep_stage(const LuBatch<float>& lu, int K0, int KB, const DeepStaging& st, cudaStream_t s);
cudaError_t tc_deep_run(const LuBatch<float>& lu, int K0, int KB, const DeepStaging& st, cudaStream_t s);
// The far step of outer block [K0, K0+KB) in one product: with
// T = -L11^{-1} (L11 the block's unit lower KB x KB diagonal block, T made by
// block_inverse_negated), the block's rows of the columns beyond it become
// S[K0:K0+KB, K0+KB:] = -T S[K0:K0+KB, K0+KB:] = L11^{-1} S[K0:K0+KB, K0+KB:]
// (the operands are staged before the product, so it may run in place).
// The caller has applied every panel's interchanges to those columns.
cudaError_t tc_far_gemm(const LuBatch<float>& lu, int K0, int KB, const float2* T, const DeepStaging& st,
                        cudaStream_t s);
// Blocked triangular solves with the stored factors of all q shifts, in
// diagonal blocks of KB rows: side 0 overwrites X (q x n x m, ld n, holding
// P R) with S^{-1} R (forward with L, backward with U); side 1 overwrites X
// (holding R) with the solution of S^H X = R before its final P^T (forward
// with U^H, backward with L^H).  Each block step is two deep products: the
// diagonal block by X_I = -T_I X_I with T_I = -D_I^{-1} (TL for the unit lower
// blocks, TU for the upper ones, conjugate-transposed on side 1; made by
// block_inverse_negated), then the rest of the sweep's rows by
// X_rest -= op(S_block) X_I with K = KB.
// pre (or nullptr): the factor operands of every product of this side, staged
// once after the factorisation by tc_solve_prestage; then each product stages
// only its block of X.
cudaError_t tc_solve_deep(const LuBatch<float>& lu, int side, float2* X, int m, int KB, const float2* TL,
                          const float2* TU, const DeepStaging& st, cudaStream_t s, const void* pre = nullptr);
// Bytes of one side's staged factor operands, and the staging itself (the
// products of tc_solve_deep in its order: -T_I and the off-diagonal factor
// blocks, conjugate-transposed on side 1, as split BF16 in the A' form).
size_t tc_solve_prestage_bytes(long long n, int q, int KB);
cudaError_t tc_solve_prestage(const LuBatch<float>& lu, int side, int KB, const float2* TL, const float2* TU,
                              void* pre, cudaStream_t s);
// Algorithmic flops and HBM bytes of one such update (8 flops per complex MAC;
// C read and written once, L and U read once, 8 bytes per complex64 entry).
double tc_deep_flops(long long n, int q, int K0, int KB);
double tc_deep_bytes(long long n, int q, int K0, int KB);
