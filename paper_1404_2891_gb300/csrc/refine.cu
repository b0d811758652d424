// Classical mixed-precision refinement of the shifted solves (the mixed
// path's optional mode, options.max_refine > 0).  The paper solves each
// shifted system once, in the working precision; on this GPU the factors are
// complex64 with split-BF16 tensor-core updates, and FP64 accuracy per system
// is won back by refinement: the residual r_k = R - S_k X_k is formed in FP64
// (its n x n x m products on the emulated-FP64 tensor-core path), the
// correction S_k d_k = r_k is solved with the complex64 factor, and
// X_k += d_k in FP64.  These kernels are the element-wise steps; the loop and
// the stopping rule are in feast.cu.  All are HBM-bound streams.
#include "refine.cuh"

namespace {

unsigned grid_of(size_t total) {
  size_t g = (total + 255) / 256;
  return (unsigned)(g > 152 * 16 ? 152 * 16 : (g ? g : 1));
}

__global__ void k_refine_widen(const float2* Xs, int q, int n, int m, const int32_t* rowmap, double2* X64, bool add) {
  const size_t total = (size_t)n * m;
  const size_t all = total * q;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < all; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t b = idx / total, e = idx % total;
    const int i = (int)(e % n);
    const size_t c = e / n;
    const int src = rowmap ? rowmap[b * n + i] : i;
    const float2 x = Xs[b * total + c * n + src];
    double2 v = make_double2((double)x.x, (double)x.y);
    if (add) v = cadd<double>(X64[idx], v);
    X64[idx] = v;
  }
}

// one block per column
__global__ void k_refine_residual(const double2* R, const double2* T1, const double2* T2, double2 z, int n,
                                  double2* r, double* norms) {
  __shared__ double red[8];
  const int c = blockIdx.x, tid = threadIdx.x;
  const size_t off = (size_t)c * n;
  double acc = 0.0;
  for (int i = tid; i < n; i += 256) {
    double2 v = R[off + i];
    const double2 t2 = cmul<double>(z, T2[off + i]);
    v = cadd<double>(csub<double>(v, t2), T1[off + i]);
    r[off + i] = v;
    acc += cnorm2<double>(v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k];
    norms[c] = sqrt(t);
  }
}

__global__ void k_refine_gather(const double2* r, const int32_t* perm, float2* Xs, int q, int n, int m, bool permute) {
  const size_t total = (size_t)n * m;
  const size_t all = total * q;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < all; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t b = idx / total, e = idx % total;
    const int i = (int)(e % n);
    const size_t c = e / n;
    const int src = permute ? perm[b * n + i] : i;
    const double2 v = r[b * total + c * n + src];
    Xs[idx] = make_float2((float)v.x, (float)v.y);
  }
}

}  // namespace

cudaError_t refine_widen(const float2* Xs, int q, int n, int m, const int32_t* rowmap, double2* X64, bool add,
                         cudaStream_t s) {
  feast_count_launch();
  k_refine_widen<<<grid_of((size_t)n * m * q), 256, 0, s>>>(Xs, q, n, m, rowmap, X64, add);
  return cudaGetLastError();
}

cudaError_t refine_residual(const double2* R, const double2* T1, const double2* T2, double2 z, int n, int m,
                            double2* r, double* norms, cudaStream_t s) {
  feast_count_launch();
  k_refine_residual<<<m, 256, 0, s>>>(R, T1, T2, z, n, r, norms);
  return cudaGetLastError();
}

cudaError_t refine_gather(const double2* r, const int32_t* perm, float2* Xs, int q, int n, int m, bool permute,
                          cudaStream_t s) {
  feast_count_launch();
  k_refine_gather<<<grid_of((size_t)n * m * q), 256, 0, s>>>(r, perm, Xs, q, n, m, permute);
  return cudaGetLastError();
}
