// Choice of the kernel that performs the LU trailing update A22 -= L21 U12.
#pragma once
#include "lu.cuh"

// complex128: the DMMA batched GEMM; complex64: the tcgen05 kernel when available.
template <typename T>
void select_trailing_update(TrailingUpdateFn<T>* fn, void** ctx);
