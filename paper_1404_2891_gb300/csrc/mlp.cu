// The eigenvalue-count predictor that chooses the subspace size m0: a
// three-layer perceptron  d_in -> width -> width -> 1  with GELU activations,
// BF16 weights in the forward and backward products, FP32 accumulation, FP32
// master weights and Adam.  Inputs are standardised by stored per-feature
// mean and scale.  All arithmetic is in the kernels below.
#include <cuda_bf16.h>

#include <cstring>
#include <new>
#include <vector>

#include "../../include/feast_gb300.h"
#include "common.cuh"

struct feast_mlp {
  int d_in = 0, width = 0;
  cudaStream_t st = nullptr;
  size_t nparam = 0;
  float* p = nullptr;          // master parameters: W1, b1, W2, b2, W3, b3
  float* g = nullptr;          // gradients (same layout)
  float* m = nullptr;          // Adam first moment
  float* v = nullptr;          // Adam second moment
  __nv_bfloat16* wb = nullptr; // BF16 copies of W1, W2, W3 (same offsets as in p, biases unused)
  float* mean = nullptr;       // d_in
  float* scale = nullptr;      // d_in
  int bmax = 0;
  float *x0 = nullptr, *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *out = nullptr;
  float *d1 = nullptr, *d2 = nullptr, *dout = nullptr, *loss = nullptr;
  int* idx = nullptr;
  int t = 0;                   // Adam step counter
  std::vector<void*> allocs;
};

namespace {

struct Off {
  size_t W1, b1, W2, b2, W3, b3, total;
};
Off offsets(int d_in, int w) {
  Off o;
  o.W1 = 0;
  o.b1 = o.W1 + (size_t)w * d_in;
  o.W2 = o.b1 + w;
  o.b2 = o.W2 + (size_t)w * w;
  o.W3 = o.b2 + w;
  o.b3 = o.W3 + w;
  o.total = o.b3 + 1;
  return o;
}

__device__ __forceinline__ float gelu(float x) {
  const float c = 0.7978845608028654f;  // sqrt(2 / pi)
  return 0.5f * x * (1.f + tanhf(c * (x + 0.044715f * x * x * x)));
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float c = 0.7978845608028654f;
  const float u = c * (x + 0.044715f * x * x * x);
  const float th = tanhf(u);
  return 0.5f * (1.f + th) + 0.5f * x * (1.f - th * th) * c * (1.f + 3.f * 0.044715f * x * x);
}

// x0[b, i] = (X[idx[b], i] - mean[i]) / scale[i]   (row indices clamped to [0, n_rows))
__global__ void k_standardise(const float* X, const int* idx, int B, int n_rows, int d_in, const float* mean,
                              const float* scale, float* x0) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * d_in; e += gridDim.x * blockDim.x) {
    const int b = e / d_in, i = e % d_in;
    int row = idx ? idx[b] : b;
    row = row < 0 ? 0 : (row >= n_rows ? n_rows - 1 : row);
    x0[e] = (X[(size_t)row * d_in + i] - mean[i]) / scale[i];
  }
}

// z[b, o] = sum_i x[b, i] W[o, i] + bias[o];  h = act ? gelu(z) : z   (W bf16, FP32 sums)
__global__ void k_linear_fwd(const float* x, int B, int din, const __nv_bfloat16* W, const float* bias, int dout,
                             float* z, float* h, int act) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * dout; e += gridDim.x * blockDim.x) {
    const int b = e / dout, o = e % dout;
    const float* xr = x + (size_t)b * din;
    const __nv_bfloat16* wr = W + (size_t)o * din;
    float acc = 0.f;
    for (int i = 0; i < din; ++i) acc = fmaf(xr[i], __bfloat162float(wr[i]), acc);
    acc += bias[o];
    z[e] = acc;
    if (h) h[e] = act ? gelu(acc) : acc;
  }
}

// mean squared error on the first B rows: loss = (1/B) sum (out - y)^2, dout = 2 (out - y) / B
__global__ void k_mse(const float* out, const float* y, const int* idx, int B, int n_rows, float* dout, float* loss) {
  __shared__ float red[32];
  float s = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    int row = idx ? idx[b] : b;
    row = row < 0 ? 0 : (row >= n_rows ? n_rows - 1 : row);
    const float r = out[b] - y[row];
    dout[b] = 2.f * r / B;
    s += r * r;
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *loss = t / B;
  }
}

// dx[b, i] = (sum_o dz[b, o] W[o, i]) * (zprev ? gelu'(zprev[b, i]) : 1)
__global__ void k_linear_bwd_data(const float* dz, int B, int dout, const __nv_bfloat16* W, int din, const float* zprev,
                                  float* dx) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * din; e += gridDim.x * blockDim.x) {
    const int b = e / din, i = e % din;
    const float* dr = dz + (size_t)b * dout;
    float acc = 0.f;
    for (int o = 0; o < dout; ++o) acc = fmaf(dr[o], __bfloat162float(W[(size_t)o * din + i]), acc);
    dx[e] = zprev ? acc * gelu_grad(zprev[e]) : acc;
  }
}

// gW[o, i] = sum_b dz[b, o] x[b, i];  gb[o] = sum_b dz[b, o]   (FP32 sums in b order)
__global__ void k_linear_bwd_weight(const float* dz, const float* x, int B, int dout, int din, float* gW, float* gb) {
  const int n = dout * (din + 1);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int o = e / (din + 1), i = e % (din + 1);
    float acc = 0.f;
    if (i < din) {
      for (int b = 0; b < B; ++b) acc = fmaf(dz[(size_t)b * dout + o], x[(size_t)b * din + i], acc);
      gW[(size_t)o * din + i] = acc;
    } else {
      for (int b = 0; b < B; ++b) acc += dz[(size_t)b * dout + o];
      gb[o] = acc;
    }
  }
}

// Adam on the FP32 masters, then the BF16 copies of the weights
__global__ void k_adam(float* p, const float* g, float* m, float* v, __nv_bfloat16* wb, size_t n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    const float pi = p[e] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[e] = pi;
    wb[e] = __float2bfloat16_rn(pi);
  }
}

__global__ void k_to_bf16(const float* p, __nv_bfloat16* wb, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    wb[e] = __float2bfloat16_rn(p[e]);
}

unsigned g1(size_t n) {
  size_t b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 2048 ? 2048 : b));
}

// forward on rows idx[0..B) of X (n_rows rows; idx may be null); leaves out[0..B)
cudaError_t forward(feast_mlp* net, const float* X, const int* idx, int B, int n_rows) {
  const Off o = offsets(net->d_in, net->width);
  const int w = net->width, din = net->d_in;
  feast_count_launch();
  k_standardise<<<g1((size_t)B * din), 256, 0, net->st>>>(X, idx, B, n_rows, din, net->mean, net->scale, net->x0);
  feast_count_launch();
  k_linear_fwd<<<g1((size_t)B * w), 256, 0, net->st>>>(net->x0, B, din, net->wb + o.W1, net->p + o.b1, w, net->z1,
                                                        net->h1, 1);
  feast_count_launch();
  k_linear_fwd<<<g1((size_t)B * w), 256, 0, net->st>>>(net->h1, B, w, net->wb + o.W2, net->p + o.b2, w, net->z2,
                                                        net->h2, 1);
  feast_count_launch();
  k_linear_fwd<<<g1((size_t)B), 256, 0, net->st>>>(net->h2, B, w, net->wb + o.W3, net->p + o.b3, 1, net->out,
                                                    nullptr, 0);
  return cudaGetLastError();
}

cudaError_t backward(feast_mlp* net, const float* y, const int* idx, int B, int n_rows) {
  const Off o = offsets(net->d_in, net->width);
  const int w = net->width, din = net->d_in;
  feast_count_launch();
  k_mse<<<1, 256, 0, net->st>>>(net->out, y, idx, B, n_rows, net->dout, net->loss);
  // layer 3
  feast_count_launch();
  k_linear_bwd_weight<<<g1((size_t)(w + 1)), 256, 0, net->st>>>(net->dout, net->h2, B, 1, w, net->g + o.W3, net->g + o.b3);
  feast_count_launch();
  k_linear_bwd_data<<<g1((size_t)B * w), 256, 0, net->st>>>(net->dout, B, 1, net->wb + o.W3, w, net->z2, net->d2);
  // layer 2
  feast_count_launch();
  k_linear_bwd_weight<<<g1((size_t)w * (w + 1)), 256, 0, net->st>>>(net->d2, net->h1, B, w, w, net->g + o.W2, net->g + o.b2);
  feast_count_launch();
  k_linear_bwd_data<<<g1((size_t)B * w), 256, 0, net->st>>>(net->d2, B, w, net->wb + o.W2, w, net->z1, net->d1);
  // layer 1
  feast_count_launch();
  k_linear_bwd_weight<<<g1((size_t)w * (din + 1)), 256, 0, net->st>>>(net->d1, net->x0, B, w, din, net->g + o.W1,
                                                                       net->g + o.b1);
  return cudaGetLastError();
}

feast_status st_of(cudaError_t e) {
  return e == cudaSuccess ? FEAST_OK : (e == cudaErrorMemoryAllocation ? FEAST_ERR_ALLOC : FEAST_ERR_CUDA);
}

// the kernels read the caller's feature and label arrays directly: device memory only
bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename P>
cudaError_t nalloc(feast_mlp* net, P** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e == cudaSuccess) {
    net->allocs.push_back(q);
    *p = reinterpret_cast<P*>(q);
  }
  return e;
}

}  // namespace

extern "C" {

void feast_mlp_destroy(feast_mlp* net) {
  if (!net) return;
  if (net->st) cudaStreamSynchronize(net->st);
  for (void* p : net->allocs) cudaFree(p);
  delete net;
}

size_t feast_mlp_param_count(int d_in, int width) { return offsets(d_in, width).total; }

feast_status feast_mlp_create(feast_mlp** out, int d_in, int width, int max_batch, const float* params,
                              const float* mean, const float* scale, void* stream) {
  if (!out || d_in < 1 || width < 1 || max_batch < 1 || !params || !mean || !scale) return FEAST_ERR_ARG;
  *out = nullptr;
  feast_mlp* net = new (std::nothrow) feast_mlp();
  if (!net) return FEAST_ERR_ALLOC;
  net->d_in = d_in;
  net->width = width;
  net->bmax = max_batch;
  net->st = reinterpret_cast<cudaStream_t>(stream);
  const Off o = offsets(d_in, width);
  net->nparam = o.total;
  cudaError_t e = cudaSuccess;
  auto fail = [&]() { feast_mlp_destroy(net); return st_of(e); };
  if ((e = nalloc(net, &net->p, o.total * 4)) != cudaSuccess) return fail();
  if ((e = nalloc(net, &net->g, o.total * 4)) != cudaSuccess) return fail();
  if ((e = nalloc(net, &net->m, o.total * 4)) != cudaSuccess) return fail();
  if ((e = nalloc(net, &net->v, o.total * 4)) != cudaSuccess) return fail();
  if ((e = nalloc(net, &net->wb, o.total * 2)) != cudaSuccess) return fail();
  if ((e = nalloc(net, &net->mean, d_in * 4)) != cudaSuccess) return fail();
  if ((e = nalloc(net, &net->scale, d_in * 4)) != cudaSuccess) return fail();
  const size_t B = max_batch;
  float** acts[] = {&net->z1, &net->h1, &net->z2, &net->h2, &net->d1, &net->d2};
  if ((e = nalloc(net, &net->x0, B * d_in * 4)) != cudaSuccess) return fail();
  for (float** a : acts)
    if ((e = nalloc(net, a, B * width * 4)) != cudaSuccess) return fail();
  if ((e = nalloc(net, &net->out, B * 4)) != cudaSuccess) return fail();
  if ((e = nalloc(net, &net->dout, B * 4)) != cudaSuccess) return fail();
  if ((e = nalloc(net, &net->loss, 64)) != cudaSuccess) return fail();
  if ((e = nalloc(net, &net->idx, B * 4)) != cudaSuccess) return fail();
  if ((e = cudaMemcpyAsync(net->p, params, o.total * 4, cudaMemcpyDefault, net->st)) != cudaSuccess) return fail();
  if ((e = cudaMemcpyAsync(net->mean, mean, d_in * 4, cudaMemcpyDefault, net->st)) != cudaSuccess) return fail();
  if ((e = cudaMemcpyAsync(net->scale, scale, d_in * 4, cudaMemcpyDefault, net->st)) != cudaSuccess) return fail();
  if ((e = cudaMemsetAsync(net->m, 0, o.total * 4, net->st)) != cudaSuccess) return fail();
  if ((e = cudaMemsetAsync(net->v, 0, o.total * 4, net->st)) != cudaSuccess) return fail();
  feast_count_launch();
  k_to_bf16<<<g1(o.total), 256, 0, net->st>>>(net->p, net->wb, o.total);
  if ((e = cudaStreamSynchronize(net->st)) != cudaSuccess) return fail();
  *out = net;
  return FEAST_OK;
}

feast_status feast_mlp_get_params(feast_mlp* net, float* params) {
  if (!net || !params) return FEAST_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(params, net->p, net->nparam * 4, cudaMemcpyDefault, net->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->st);
  return st_of(e);
}

feast_status feast_mlp_predict(feast_mlp* net, const float* X, int B, float* y) {
  if (!net || !X || !y || B < 1 || B > net->bmax || !on_device(X)) return FEAST_ERR_ARG;
  cudaError_t e = forward(net, X, nullptr, B, B);
  if (e == cudaSuccess) e = cudaMemcpyAsync(y, net->out, (size_t)B * 4, cudaMemcpyDefault, net->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->st);
  return st_of(e);
}

feast_status feast_mlp_grad(feast_mlp* net, const float* X, const float* y, int B, float* loss, float* grads) {
  if (!net || !X || !y || B < 1 || B > net->bmax || !on_device(X) || !on_device(y)) return FEAST_ERR_ARG;
  cudaError_t e = forward(net, X, nullptr, B, B);
  if (e == cudaSuccess) e = backward(net, y, nullptr, B, B);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, net->loss, 4, cudaMemcpyDefault, net->st);
  if (e == cudaSuccess && grads) e = cudaMemcpyAsync(grads, net->g, net->nparam * 4, cudaMemcpyDefault, net->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->st);
  return st_of(e);
}

feast_status feast_mlp_train(feast_mlp* net, const float* X, const float* y, int n_rows, const int* batches,
                             int steps, int B, float lr, float* last_loss) {
  if (!net || !X || !y || !batches || n_rows < 1 || steps < 1 || B < 1 || B > net->bmax) return FEAST_ERR_ARG;
  if (!on_device(X) || !on_device(y)) return FEAST_ERR_ARG;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < steps && e == cudaSuccess; ++s) {
    e = cudaMemcpyAsync(net->idx, batches + (size_t)s * B, (size_t)B * 4, cudaMemcpyDefault, net->st);
    if (e == cudaSuccess) e = forward(net, X, net->idx, B, n_rows);
    if (e == cudaSuccess) e = backward(net, y, net->idx, B, n_rows);
    if (e != cudaSuccess) break;
    ++net->t;
    const float c1 = 1.f - powf(b1, (float)net->t), c2 = 1.f - powf(b2, (float)net->t);
    feast_count_launch();
    k_adam<<<g1(net->nparam), 256, 0, net->st>>>(net->p, net->g, net->m, net->v, net->wb, net->nparam, lr, b1, b2, eps,
                                                  c1, c2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && last_loss) e = cudaMemcpyAsync(last_loss, net->loss, 4, cudaMemcpyDefault, net->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->st);
  return st_of(e);
}

}  // extern "C"
