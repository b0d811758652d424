// Batched complex GEMM used by every dense contraction of the FP64 path and
// by the FP32 fallback of the mixed path:
//     C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b],   b = 0 .. batch-1
// column-major operands, op in {N, T, C}, per-batch element strides (0 = shared).
#pragma once
#include "common.cuh"

template <typename T>
struct GemmArgs {
  int M = 0, N = 0, K = 0, batch = 1;
  cplx<T> alpha, beta;
  const cplx<T>* A = nullptr;
  long long lda = 0, strideA = 0;
  int opA = OP_N;
  const cplx<T>* B = nullptr;
  long long ldb = 0, strideB = 0;
  int opB = OP_N;
  cplx<T>* C = nullptr;
  long long ldc = 0, strideC = 0;
  // Optional split-K workspace (complex128 path): when M x N spans few tiles and
  // K is long, K is cut into chunks whose partial products land here and are
  // summed in a fixed order by a second kernel (deterministic).
  cplx<T>* ws = nullptr;
  size_t ws_elems = 0;
  int splitk = 1;  // set by gemm_batched; chosen by the caller for gemm_grouped
  int tag = 0;     // gemm_grouped: the problem's index into `active`
};

template <typename T>
cudaError_t gemm_batched(const GemmArgs<T>& g, cudaStream_t s);

// Grouped GEMM: table entry p (tab[p] in device memory, batch = 1) owns grid
// tiles [tstart[p], tstart[p+1]), tstart[p+1] - tstart[p] =
// gemm_tiles(M_p, N_p) * splitk_p; entries with active[tag_p] == 0 are skipped.
// complex128 entries with splitk_p > 1 write K-chunk partials to their ws
// (splitk_p * M_p * N_p elements) and a second kernel sums them in a fixed
// order; split_mn = the largest M_p * N_p among such entries (0: none).
// complex64 entries must have splitk_p = 1.
template <typename T>
cudaError_t gemm_grouped(const GemmArgs<T>* tab, const int* tstart, int np, int total_tiles, const int* active,
                         size_t split_mn, cudaStream_t s);
int gemm_tiles(int M, int N);
