// Trailing-update selection for the batched shifted LU.
#include "tc_update.cuh"

template <>
void select_trailing_update<double>(TrailingUpdateFn<double>* fn, void** ctx) {
  *fn = nullptr;  // default: gemm_batched<double> (mma.sync f64)
  *ctx = nullptr;
}

template <>
void select_trailing_update<float>(TrailingUpdateFn<float>* fn, void** ctx) {
  *fn = nullptr;
  *ctx = nullptr;
}
