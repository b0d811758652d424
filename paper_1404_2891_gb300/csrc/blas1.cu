// Element-wise and column-wise kernels.  All of them are HBM- or latency-bound;
// the heavy one is the accumulation sum_k sigma_k X_k of Eq. Rasp / Eq. Lasp,
// which streams the q solution blocks once in a fixed order of k.
#include "blas1.cuh"

namespace {

// Columns strided over blockIdx.y, rows over the block.  The complex64
// form computes z b - a in FP32 (the result is rounded to complex64 anyway;
// FP64 arithmetic runs at 1/64 of the FP32 rate on this GPU).
template <typename T>
__global__ void k_form_shifted(const double2* A, long long lda, const double2* B, long long ldb,
                               const double2* z, int q, int n, cplx<T>* S, long long strideS) {
  __shared__ cplx<T> sz[256];
  for (int k = threadIdx.x; k < q && k < 256; k += blockDim.x) sz[k] = cconv<T, double>(z[k]);
  __syncthreads();
  for (int j = blockIdx.y; j < n; j += gridDim.y)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const cplx<T> a = cconv<T, double>(A[(size_t)i + (size_t)j * lda]);
    const cplx<T> b = B ? cconv<T, double>(B[(size_t)i + (size_t)j * ldb]) : mk<T>(i == j ? T(1) : T(0), T(0));
    const size_t idx = (size_t)i + (size_t)j * n;
    for (int k = 0; k < q; ++k) {
      const cplx<T> zk = k < 256 ? sz[k] : cconv<T, double>(z[k]);
      S[(size_t)k * strideS + idx] = csub<T>(cmul<T>(zk, b), a);
    }
  }
}

// complex64 with n even: two consecutive rows per thread, 16-byte stores
// (n even keeps every pair 16-byte aligned in every shifted matrix)
__global__ void k_form_shifted_pairs(const double2* A, long long lda, const double2* B, long long ldb,
                                     const double2* z, int q, int n, float2* S, long long strideS) {
  __shared__ float2 sz[256];
  for (int k = threadIdx.x; k < q && k < 256; k += blockDim.x) sz[k] = make_float2((float)z[k].x, (float)z[k].y);
  __syncthreads();
  const int half = n >> 1;
  for (int j = blockIdx.y; j < n; j += gridDim.y)
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < half; p += gridDim.x * blockDim.x) {
      const int i = 2 * p;
      float2 a[2], b[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const double2 av = A[(size_t)(i + u) + (size_t)j * lda];
        a[u] = make_float2((float)av.x, (float)av.y);
        if (B) {
          const double2 bv = B[(size_t)(i + u) + (size_t)j * ldb];
          b[u] = make_float2((float)bv.x, (float)bv.y);
        } else {
          b[u] = make_float2(i + u == j ? 1.f : 0.f, 0.f);
        }
      }
      const size_t idx = (size_t)i + (size_t)j * n;
      for (int k = 0; k < q; ++k) {
        const float2 zk = k < 256 ? sz[k] : make_float2((float)z[k].x, (float)z[k].y);
        const float2 s0 = csub<float>(cmul<float>(zk, b[0]), a[0]);
        const float2 s1 = csub<float>(cmul<float>(zk, b[1]), a[1]);
        *reinterpret_cast<float4*>(S + (size_t)k * strideS + idx) = make_float4(s0.x, s0.y, s1.x, s1.y);
      }
    }
}

template <typename T>
__global__ void k_accumulate(const cplx<T>* Xs, AccTree t, int n, int m, const double2* coef, const double2* c0,
                             const double2* Y, const int32_t* rowmap, double2* Q) {
  const size_t total = (size_t)n * m;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % n);
    const int i = (int)(idx / n);
    double2 leaf[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      leaf[j] = make_double2(0.0, 0.0);
      if (j < t.nleaf)
        for (int b = t.b[j]; b < t.b[j + 1]; ++b) {
          const int rr = rowmap ? rowmap[(size_t)b * n + r] : r;
          const cplx<T> x = Xs[(size_t)b * total + (size_t)i * n + rr];
          cfma<double>(leaf[j], coef[(size_t)b * m + i], cconv<double, T>(x));
        }
    }
#pragma unroll
    for (int w = 1; w < 8; w *= 2)
#pragma unroll
      for (int j = 0; j + w < 8; j += 2 * w)
        if (j + w < t.nleaf) leaf[j] = cadd<double>(leaf[j], leaf[j + w]);
    double2 acc = leaf[0];
    if (c0 && Y) cfma<double>(acc, c0[i], Y[idx]);
    Q[idx] = acc;
  }
}

template <typename T>
__global__ void k_accumulate_conj(const cplx<T>* Xs, int q, int n, int m, const double2* coef, const double2* coefc,
                                  const double2* c0, const double2* Y, const int32_t* rowmap, double2* Q) {
  const size_t total = (size_t)n * m;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % n);
    const int i = (int)(idx / n);
    double2 acc = make_double2(0.0, 0.0);
    for (int b = 0; b < q; ++b) {
      const int rr = rowmap ? rowmap[(size_t)b * n + r] : r;
      const cplx<T>* Xb = Xs + (size_t)b * 2 * total;
      cfma<double>(acc, coef[(size_t)b * m + i], cconv<double, T>(Xb[(size_t)i * n + rr]));
      cfma<double>(acc, coefc[(size_t)b * m + i], cconj<double>(cconv<double, T>(Xb[total + (size_t)i * n + rr])));
    }
    if (c0 && Y) cfma<double>(acc, c0[i], Y[idx]);
    Q[idx] = acc;
  }
}

__global__ void k_tree_combine(const double2* P, int nparts, int n, int m, const double2* c0, const double2* Y,
                               double2* Q) {
  const size_t total = (size_t)n * m;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n);
    double2 leaf[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) leaf[j] = j < nparts ? P[(size_t)j * total + idx] : make_double2(0.0, 0.0);
#pragma unroll
    for (int w = 1; w < 8; w *= 2)
#pragma unroll
      for (int j = 0; j + w < 8; j += 2 * w)
        if (j + w < nparts) leaf[j] = cadd<double>(leaf[j], leaf[j + w]);
    double2 acc = leaf[0];
    if (c0 && Y) cfma<double>(acc, c0[i], Y[idx]);
    Q[idx] = acc;
  }
}

__global__ void k_select(const double2* E, const double2* F, const int* use_res, int n, int m, double2* R) {
  const size_t total = (size_t)n * m;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n);
    R[idx] = use_res[i] ? E[idx] : F[idx];
  }
}

__device__ double block_sum256(double v) {
  __shared__ double red[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += red[k];
  return t;
}

__device__ double2 block_csum256(double2 v) {
  const double a = block_sum256(v.x);
  const double b = block_sum256(v.y);
  return make_double2(a, b);
}

__global__ void __launch_bounds__(256) k_col_norms(const double2* X, int n, double* nrm) {
  const double2* x = X + (size_t)blockIdx.x * n;
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += 256) s += cnorm2<double>(x[r]);
  s = block_sum256(s);
  if (threadIdx.x == 0) nrm[blockIdx.x] = sqrt(s);
}

__global__ void k_scale_cols(double2* X0, double2* X1, double2* X2, int n, int m, const double* nrm,
                             const double2* d) {
  const size_t total = (size_t)n * m;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n);
    double2 f;
    if (nrm) {
      const double v = nrm[i];
      f = make_double2(v > 0.0 ? 1.0 / v : 0.0, 0.0);
    } else {
      const double2 dv = d[i];
      f = (dv.x == 0.0 && dv.y == 0.0) ? make_double2(1.0, 0.0) : crecip<double>(cconj<double>(dv));
    }
    if (X0) X0[idx] = cmul<double>(X0[idx], f);
    if (X1) X1[idx] = cmul<double>(X1[idx], f);
    if (X2) X2[idx] = cmul<double>(X2[idx], f);
  }
}

__global__ void __launch_bounds__(256)
k_residual(const double2* AX, const double2* BX, const double2* lam, int conj_lam, int n, double2* E,
           double* res, const double* xn) {
  const int i = blockIdx.x;
  double2 l = lam[i];
  if (conj_lam) l.y = -l.y;
  const size_t off = (size_t)i * n;
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += 256) {
    const double2 e = csub<double>(AX[off + r], cmul<double>(BX[off + r], l));
    E[off + r] = e;
    s += cnorm2<double>(e);
  }
  s = block_sum256(s);
  if (threadIdx.x == 0) res[i] = sqrt(s) / (xn ? xn[i] : 1.0);
}

__global__ void __launch_bounds__(256) k_col_dots(const double2* X, const double2* Y, int n, double2* d) {
  const size_t off = (size_t)blockIdx.x * n;
  double2 s = make_double2(0.0, 0.0);
  for (int r = threadIdx.x; r < n; r += 256) s = cadd<double>(s, cmulc<double>(X[off + r], Y[off + r]));
  s = block_csum256(s);
  if (threadIdx.x == 0) d[blockIdx.x] = s;
}


__global__ void k_conj_copy(const double2* src, double2* dst, size_t count) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = cconj<double>(src[e]);
}

__global__ void k_identity(double2* M, int m) {
  const size_t total = (size_t)m * m;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x)
    M[idx] = make_double2((idx % m) == (idx / m) ? 1.0 : 0.0, 0.0);
}

__global__ void k_gather_cols(const double2* src, const int* idx, int k, int n, int m, double2* out) {
  const size_t total = (size_t)n * m;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e % n, c = e / n;
    out[e] = (int)c < k ? src[r + (size_t)idx[c] * n] : make_double2(0.0, 0.0);
  }
}

__global__ void __launch_bounds__(256) k_normalize_vec(double2* x, int n, double* nrm) {
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += 256) s += cnorm2<double>(x[r]);
  s = block_sum256(s);
  const double v = sqrt(s);
  const double inv = v > 0.0 ? 1.0 / v : 0.0;
  for (int r = threadIdx.x; r < n; r += 256) x[r] = cscale<double>(x[r], inv);
  if (threadIdx.x == 0) *nrm = v;
}

__global__ void k_check_finite(const double2* X, size_t count, unsigned* flags) {
  bool bad = false;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const double2 v = X[e];
    if (!isfinite(v.x) || !isfinite(v.y)) bad = true;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, (unsigned)DEVFLAG_NONFINITE);
}

template <typename T>
__global__ void __launch_bounds__(256) k_probe_dots(const double2* V, const cplx<T>* X, int n, int S, double2* d) {
  const size_t total = (size_t)n * S;
  const cplx<T>* Xb = X + (size_t)blockIdx.x * total;
  double2 acc = make_double2(0.0, 0.0);
  for (size_t e = threadIdx.x; e < total; e += 256) acc = cadd<double>(acc, cmulc<double>(V[e], cconv<double, T>(Xb[e])));
  acc = block_csum256(acc);
  if (threadIdx.x == 0) d[blockIdx.x] = acc;
}

__global__ void k_moments_combine(const double2* d, const double2* z, const double2* w, double2 c, double R, int q,
                                  int kmax, int S, double2* mu) {
  const int k = threadIdx.x;
  if (k > kmax) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int b = 0; b < q; ++b) {
    const double2 t = cscale<double>(csub<double>(z[b], c), 1.0 / R);
    double2 tk = make_double2(1.0, 0.0);
    for (int e = 0; e < k; ++e) tk = cmul<double>(tk, t);
    acc = cadd<double>(acc, cmul<double>(cmul<double>(w[b], tk), d[b]));
  }
  mu[k] = cscale<double>(acc, 1.0 / S);
}

unsigned grid_for(size_t total) {
  size_t g = (total + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g ? g : 1);
}

}  // namespace

template <typename T>
cudaError_t form_shifted(const double2* A, long long lda, const double2* B, long long ldb, const double2* z,
                         int q, int n, cplx<T>* S, long long strideS, cudaStream_t s) {
  feast_count_launch();
  dim3 grid((unsigned)((n + 255) / 256 < 8 ? (n + 255) / 256 : 8), (unsigned)(n < 65535 ? n : 65535));
  if constexpr (std::is_same<T, float>::value) {
    if (n % 2 == 0 && strideS % 2 == 0 && (reinterpret_cast<uintptr_t>(S) & 15) == 0) {
      dim3 g2((unsigned)((n / 2 + 255) / 256 < 8 ? (n / 2 + 255) / 256 : 8), grid.y);
      k_form_shifted_pairs<<<g2, 256, 0, s>>>(A, lda, B, ldb, z, q, n, S, strideS);
      return cudaGetLastError();
    }
  }
  k_form_shifted<T><<<grid, 256, 0, s>>>(A, lda, B, ldb, z, q, n, S, strideS);
  return cudaGetLastError();
}
template cudaError_t form_shifted<double>(const double2*, long long, const double2*, long long, const double2*, int, int, double2*, long long, cudaStream_t);
template cudaError_t form_shifted<float>(const double2*, long long, const double2*, long long, const double2*, int, int, float2*, long long, cudaStream_t);

template <typename T>
cudaError_t accumulate(const cplx<T>* Xs, const AccTree& t, int n, int m, const double2* coef, const double2* c0,
                       const double2* Y, const int32_t* rowmap, double2* Q, cudaStream_t s) {
  if (t.nleaf < 1 || t.nleaf > 8 || (t.nleaf & (t.nleaf - 1))) return cudaErrorInvalidValue;
  feast_count_launch();
  k_accumulate<T><<<grid_for((size_t)n * m), 256, 0, s>>>(Xs, t, n, m, coef, c0, Y, rowmap, Q);
  return cudaGetLastError();
}
template cudaError_t accumulate<double>(const double2*, const AccTree&, int, int, const double2*, const double2*, const double2*, const int32_t*, double2*, cudaStream_t);
template cudaError_t accumulate<float>(const float2*, const AccTree&, int, int, const double2*, const double2*, const double2*, const int32_t*, double2*, cudaStream_t);

template <typename T>
cudaError_t accumulate_conj_pairs(const cplx<T>* Xs, int q, int n, int m, const double2* coef, const double2* coefc,
                                  const double2* c0, const double2* Y, const int32_t* rowmap, double2* Q,
                                  cudaStream_t s) {
  feast_count_launch();
  k_accumulate_conj<T><<<grid_for((size_t)n * m), 256, 0, s>>>(Xs, q, n, m, coef, coefc, c0, Y, rowmap, Q);
  return cudaGetLastError();
}
template cudaError_t accumulate_conj_pairs<double>(const double2*, int, int, int, const double2*, const double2*,
                                                   const double2*, const double2*, const int32_t*, double2*,
                                                   cudaStream_t);
template cudaError_t accumulate_conj_pairs<float>(const float2*, int, int, int, const double2*, const double2*,
                                                  const double2*, const double2*, const int32_t*, double2*,
                                                  cudaStream_t);

AccTree acc_tree_single(int q) {
  AccTree t;
  t.nleaf = 1;
  t.b[0] = 0;
  t.b[1] = q;
  return t;
}

cudaError_t accumulate_tree_combine(const double2* P, int nparts, int n, int m, const double2* c0, const double2* Y,
                                    double2* Q, cudaStream_t s) {
  if (nparts < 1 || nparts > 8 || (nparts & (nparts - 1))) return cudaErrorInvalidValue;
  feast_count_launch();
  k_tree_combine<<<grid_for((size_t)n * m), 256, 0, s>>>(P, nparts, n, m, c0, Y, Q);
  return cudaGetLastError();
}

cudaError_t select_columns(const double2* E, const double2* F, const int* use_res, int n, int m, double2* R,
                           cudaStream_t s) {
  feast_count_launch();
  k_select<<<grid_for((size_t)n * m), 256, 0, s>>>(E, F, use_res, n, m, R);
  return cudaGetLastError();
}

cudaError_t column_norms(const double2* X, int n, int m, double* nrm, cudaStream_t s) {
  feast_count_launch();
  k_col_norms<<<m, 256, 0, s>>>(X, n, nrm);
  return cudaGetLastError();
}

cudaError_t scale_columns_inv(double2* X0, double2* X1, double2* X2, int n, int m, const double* nrm,
                              const double2* d, cudaStream_t s) {
  feast_count_launch();
  k_scale_cols<<<grid_for((size_t)n * m), 256, 0, s>>>(X0, X1, X2, n, m, nrm, d);
  return cudaGetLastError();
}

cudaError_t residual_columns(const double2* AX, const double2* BX, const double2* lam, int conj_lam, int n,
                             int m, double2* E, double* res, const double* xn, cudaStream_t s) {
  feast_count_launch();
  k_residual<<<m, 256, 0, s>>>(AX, BX, lam, conj_lam, n, E, res, xn);
  return cudaGetLastError();
}

cudaError_t column_dots(const double2* X, const double2* Y, int n, int m, double2* d, cudaStream_t s) {
  feast_count_launch();
  k_col_dots<<<m, 256, 0, s>>>(X, Y, n, d);
  return cudaGetLastError();
}


cudaError_t conj_copy(const double2* src, double2* dst, size_t count, cudaStream_t s) {
  feast_count_launch();
  k_conj_copy<<<grid_for(count), 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}

cudaError_t set_identity(double2* M, int m, cudaStream_t s) {
  feast_count_launch();
  k_identity<<<grid_for((size_t)m * m), 256, 0, s>>>(M, m);
  return cudaGetLastError();
}

cudaError_t gather_columns(const double2* src, const int* idx, int k, int n, int m, double2* out, cudaStream_t s) {
  feast_count_launch();
  k_gather_cols<<<grid_for((size_t)n * m), 256, 0, s>>>(src, idx, k, n, m, out);
  return cudaGetLastError();
}

cudaError_t normalize_vector(double2* x, int n, double* nrm, cudaStream_t s) {
  feast_count_launch();
  k_normalize_vec<<<1, 256, 0, s>>>(x, n, nrm);
  return cudaGetLastError();
}

template <typename T>
cudaError_t probe_dots(const double2* V, const cplx<T>* X, int n, int S, int q, double2* d, cudaStream_t s) {
  feast_count_launch();
  k_probe_dots<T><<<q, 256, 0, s>>>(V, X, n, S, d);
  return cudaGetLastError();
}
template cudaError_t probe_dots<double>(const double2*, const double2*, int, int, int, double2*, cudaStream_t);
template cudaError_t probe_dots<float>(const double2*, const float2*, int, int, int, double2*, cudaStream_t);

cudaError_t moments_combine(const double2* d, const double2* z, const double2* w, double2 c, double R, int q,
                            int kmax, int S, double2* mu, cudaStream_t s) {
  feast_count_launch();
  k_moments_combine<<<1, 32, 0, s>>>(d, z, w, c, R, q, kmax, S, mu);
  return cudaGetLastError();
}

cudaError_t check_finite(const double2* X, size_t count, unsigned* flags, cudaStream_t s) {
  feast_count_launch();
  k_check_finite<<<grid_for(count), 256, 0, s>>>(X, count, flags);
  return cudaGetLastError();
}
