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

// One batched product C_b -= L_b U_b (complex64, column-major, same ld and
// batch stride for all three):  L = S[lr0 : lr0+M, kc0 : kc0+K],
// U = S[kc0 : kc0+K, uc0 : uc0+N],  C = S[lr0 : lr0+M, uc0 : uc0+N].
// With L set, the L operand is L_b[i + k ldl] (matrix b at L + b strl) instead.
struct DeepGemm {
  float2* S = nullptr;
  long long ld = 0, stride = 0;
  int lr0 = 0, kc0 = 0, uc0 = 0;
  int M = 0, N = 0, K = 0, q = 0;
  const float2* L = nullptr;
  long long ldl = 0, strl = 0;
};

// Stage L (rows 0..M) and U (columns 0..N) as split BF16 (one launch).
cudaError_t deep_stage(const DeepGemm& g, const DeepStaging& st, cudaStream_t s);
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
// T = I - L11^{-1} (L11 the block's unit lower KB x KB diagonal block, T made
// by unit_lower_inverse_complement), the block's rows of the columns beyond it
// become S[K0:K0+KB, K0+KB:] -= T S[K0:K0+KB, K0+KB:] = L11^{-1} S[K0:K0+KB, K0+KB:]
// (the operands are staged before the product, so it may run in place).
// The caller has applied every panel's interchanges to those columns.
cudaError_t tc_far_gemm(const LuBatch<float>& lu, int K0, int KB, const float2* T, const DeepStaging& st,
                        cudaStream_t s);
// Algorithmic flops and HBM bytes of one such update (8 flops per complex MAC;
// C read and written once, L and U read once, 8 bytes per complex64 entry).
double tc_deep_flops(long long n, int q, int K0, int KB);
double tc_deep_bytes(long long n, int q, int K0, int KB);
