// ||A||_2 estimate by power iteration on A^H A (the normalisation of the
// residual gate ||A x - lambda B x|| / (||A||_2 ||x||)).
#pragma once
#include "common.cuh"

// Scratch needed by norm2_power for order n: x and y (n complex each), one
// partial sum per block and the grid-barrier words.
size_t norm2_scratch_bytes(int n);

// One cooperative launch: x0 = ones / sqrt(n); `iters` times y = A x,
// z = A^H y, s = sqrt(||z||), x = z / ||z||.  *out_dev (device) receives s.
// scratch must hold norm2_scratch_bytes(n) bytes of device memory.
// At (optional, n x n device memory): room for A^T, which makes both products
// read contiguous columns (y = A x then reads rows of A as columns of A^T).
cudaError_t norm2_power(const double2* A, long long lda, int n, int iters, void* scratch, double* out_dev,
                        unsigned* flags, cudaStream_t s, double2* At = nullptr);
