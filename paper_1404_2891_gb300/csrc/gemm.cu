// Batched complex GEMM kernels.
//
// complex128: FP64 tensor cores through mma.sync.m16n8k8.f64 (DMMA).  A
//   complex product is four real products (re*re - im*im, re*im + im*re),
//   each an MMA on planar re/im tiles staged in shared memory.
// complex64 : FP32 SIMT (FFMA) register-blocked kernel, the portable fallback
//   of the mixed path; the LU trailing update has its own tcgen05 kernel.
#include "gemm.cuh"

namespace {

constexpr int BM = 64, BN = 64;

// ---------------------------------------------------------------- operand loads
template <typename T>
__device__ __forceinline__ cplx<T> load_op(const cplx<T>* P, long long ld, int op, int r, int c,
                                           int R, int Cn) {
  // element (r, c) of op(P), where op(P) is R x Cn
  if (r >= R || c >= Cn) return czero<T>();
  if (op == OP_N) return P[(size_t)r + (size_t)c * ld];
  cplx<T> v = P[(size_t)c + (size_t)r * ld];
  if (op == OP_C) v.y = -v.y;
  return v;
}

// ---------------------------------------------------------------- FP64 / DMMA
constexpr int BK64 = 8;

__device__ __forceinline__ void dmma16n8k8(double (&c)[4], const double (&a)[4], const double (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(b[0]), "d"(b[1]));
}

// 256 threads = 8 warps as 4 (M) x 2 (N); each warp owns 16 x 32 of the 64 x 64 tile,
// i.e. one m16 row block and four n8 column blocks, with separate re/im accumulators.
__device__ __forceinline__ void zgemm_body(const GemmArgs<double>& g, const int bx, const int by, const int bz) {
  __shared__ double As[2][2][BK64][BM + 1];  // [buf][re/im][k][m]
  __shared__ double Bs[2][2][BK64][BN + 1];  // [buf][re/im][k][n]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 3, wn = warp >> 2;
  const int m0 = bx * BM, n0 = by * BN;
  const int split = bz % g.splitk;
  const size_t b = bz / g.splitk;
  const double2* A = g.A + b * g.strideA;
  const double2* B = g.B + b * g.strideB;
  double2* C = g.C + b * g.strideC;
  // K range of this block (the whole of K unless split-K is on)
  const int kchunk = ((g.K + g.splitk - 1) / g.splitk + BK64 - 1) / BK64 * BK64;
  const int kbeg = split * kchunk;
  const int kend = min(g.K, kbeg + kchunk);

  double acc_re[4][4], acc_im[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc_re[j][e] = acc_im[j][e] = 0.0;

  double2 ra[2], rb[2];
  auto gload = [&](int k0) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      int idx = tid + r * 256;
      int m, k;
      if (g.opA == OP_N) { m = idx & 63; k = idx >> 6; } else { k = idx & 7; m = idx >> 3; }
      ra[r] = load_op<double>(A, g.lda, g.opA, m0 + m, k0 + k, g.M, kend);
      int n, kk;
      if (g.opB == OP_N) { kk = idx & 7; n = idx >> 3; } else { n = idx & 63; kk = idx >> 6; }
      rb[r] = load_op<double>(B, g.ldb, g.opB, k0 + kk, n0 + n, kend, g.N);
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      int idx = tid + r * 256;
      int m, k;
      if (g.opA == OP_N) { m = idx & 63; k = idx >> 6; } else { k = idx & 7; m = idx >> 3; }
      As[buf][0][k][m] = ra[r].x;
      As[buf][1][k][m] = ra[r].y;
      int n, kk;
      if (g.opB == OP_N) { kk = idx & 7; n = idx >> 3; } else { n = idx & 63; kk = idx >> 6; }
      Bs[buf][0][kk][n] = rb[r].x;
      Bs[buf][1][kk][n] = rb[r].y;
    }
  };

  const int nk = kend > kbeg ? (kend - kbeg + BK64 - 1) / BK64 : 0;
  if (nk > 0) {
    gload(kbeg);
    sstore(0);
  }
  __syncthreads();
  const int gq = lane >> 2, tq = lane & 3;
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) gload(kbeg + (kt + 1) * BK64);
    // A fragment (16 x 8): a0 (g, t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4)
    double are[4], aim[4], aimn[4];
    const int mr = wm * 16 + gq;
    are[0] = As[buf][0][tq][mr];     aim[0] = As[buf][1][tq][mr];
    are[1] = As[buf][0][tq][mr + 8]; aim[1] = As[buf][1][tq][mr + 8];
    are[2] = As[buf][0][tq + 4][mr]; aim[2] = As[buf][1][tq + 4][mr];
    are[3] = As[buf][0][tq + 4][mr + 8]; aim[3] = As[buf][1][tq + 4][mr + 8];
#pragma unroll
    for (int e = 0; e < 4; ++e) aimn[e] = -aim[e];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      // B fragment (8 x 8): b0 (t, g), b1 (t+4, g)
      const int nc = wn * 32 + j * 8 + gq;
      double bre[2] = {Bs[buf][0][tq][nc], Bs[buf][0][tq + 4][nc]};
      double bim[2] = {Bs[buf][1][tq][nc], Bs[buf][1][tq + 4][nc]};
      dmma16n8k8(acc_re[j], are, bre);
      dmma16n8k8(acc_re[j], aimn, bim);
      dmma16n8k8(acc_im[j], are, bim);
      dmma16n8k8(acc_im[j], aim, bre);
    }
    if (kt + 1 < nk) sstore(buf ^ 1);
    __syncthreads();
  }
  // epilogue: C fragment c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1)
  const bool beta_zero = (g.beta.x == 0.0 && g.beta.y == 0.0);
  double2* part = g.splitk > 1 ? g.ws + (size_t)bz * g.M * g.N : nullptr;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = m0 + wm * 16 + gq + ((e >> 1) ? 8 : 0);
      const int c = n0 + wn * 32 + j * 8 + tq * 2 + (e & 1);
      if (r < g.M && c < g.N) {
        double2 v = make_double2(acc_re[j][e], acc_im[j][e]);
        if (part) {  // split-K: raw partial sum, reduced later in a fixed order
          part[(size_t)r + (size_t)c * g.M] = v;
          continue;
        }
        double2 out = cmul<double>(g.alpha, v);
        double2* p = C + (size_t)r + (size_t)c * g.ldc;
        if (!beta_zero) out = cadd<double>(out, cmul<double>(g.beta, *p));
        *p = out;
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_zgemm_dmma(GemmArgs<double> g) { zgemm_body(g, blockIdx.x, blockIdx.y, blockIdx.z); }

// Grouped form: tiles [tstart[p], tstart[p+1]) of the grid belong to entry p
// of the table (tm x tn x splitk tiles; split-K partials go to the entry's ws).
__global__ void __launch_bounds__(256)
k_zgemm_dmma_grp(const GemmArgs<double>* tab, const int* tstart, int np, const int* active) {
  const int t = blockIdx.x;
  int p = 0;
  while (p + 1 < np && tstart[p + 1] <= t) ++p;
  const GemmArgs<double> g = tab[p];
  if (!active[g.tag]) return;
  const int local = t - tstart[p], tm = (g.M + BM - 1) / BM, tn = (g.N + BN - 1) / BN;
  const int rest = local / tm;
  zgemm_body(g, local % tm, rest % tn, rest / tn);
}

// C = alpha * sum_s P_s + beta * C for the split entries of a grouped call (fixed order in s).
__global__ void k_splitk_reduce_grp(const GemmArgs<double>* tab, const int* active) {
  const GemmArgs<double> g = tab[blockIdx.y];
  if (g.splitk < 2 || !active[g.tag]) return;
  const size_t mn = (size_t)g.M * g.N;
  const bool beta_zero = (g.beta.x == 0.0 && g.beta.y == 0.0);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < mn; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % g.M), c = (int)(e / g.M);
    double2 acc = make_double2(0.0, 0.0);
    for (int sp = 0; sp < g.splitk; ++sp) acc = cadd<double>(acc, g.ws[sp * mn + e]);
    double2* q = g.C + (size_t)r + (size_t)c * g.ldc;
    double2 out = cmul<double>(g.alpha, acc);
    if (!beta_zero) out = cadd<double>(out, cmul<double>(g.beta, *q));
    *q = out;
  }
}

// ---------------------------------------------------------------- FP32 SIMT
constexpr int BK32 = 16;

// 256 threads, each computing a 4 x 4 block of the 64 x 64 tile.
__device__ __forceinline__ void cgemm_body(const GemmArgs<float>& g, const int bx, const int by, const int bz) {
  __shared__ float2 As[BK32][BM + 1];
  __shared__ float2 Bs[BK32][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = bx * BM, n0 = by * BN;
  const size_t b = bz;
  const float2* A = g.A + b * g.strideA;
  const float2* B = g.B + b * g.strideB;
  float2* C = g.C + b * g.strideC;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

  for (int k0 = 0; k0 < g.K; k0 += BK32) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = tid + r * 256;  // 1024 elements = 64 x 16
      int m, k;
      if (g.opA == OP_N) { m = idx & 63; k = idx >> 6; } else { k = idx & 15; m = idx >> 4; }
      As[k][m] = load_op<float>(A, g.lda, g.opA, m0 + m, k0 + k, g.M, g.K);
      int n, kk;
      if (g.opB == OP_N) { kk = idx & 15; n = idx >> 4; } else { n = idx & 63; kk = idx >> 6; }
      Bs[kk][n] = load_op<float>(B, g.ldb, g.opB, k0 + kk, n0 + n, g.K, g.N);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK32; ++k) {
      float2 a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[k][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma<float>(acc[i][j], a[i], bb[j]);
    }
    __syncthreads();
  }
  const bool beta_zero = (g.beta.x == 0.f && g.beta.y == 0.f);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = m0 + tx + 16 * i, c = n0 + ty + 16 * j;
      if (r < g.M && c < g.N) {
        float2 out = cmul<float>(g.alpha, acc[i][j]);
        float2* p = C + (size_t)r + (size_t)c * g.ldc;
        if (!beta_zero) out = cadd<float>(out, cmul<float>(g.beta, *p));
        *p = out;
      }
    }
}

__global__ void __launch_bounds__(256) k_cgemm_simt(GemmArgs<float> g) { cgemm_body(g, blockIdx.x, blockIdx.y, blockIdx.z); }

__global__ void __launch_bounds__(256)
k_cgemm_simt_grp(const GemmArgs<float>* tab, const int* tstart, int np, const int* active) {
  const int t = blockIdx.x;
  int p = 0;
  while (p + 1 < np && tstart[p + 1] <= t) ++p;
  const GemmArgs<float> g = tab[p];
  if (!active[g.tag]) return;
  const int local = t - tstart[p], tm = (g.M + BM - 1) / BM;
  cgemm_body(g, local % tm, local / tm, 0);
}

}  // namespace

namespace {
// C = alpha * sum_{s < S} P_s + beta * C, the splits summed in increasing s.
__global__ void k_splitk_reduce(GemmArgs<double> g) {
  const size_t mn = (size_t)g.M * g.N;
  const size_t total = mn * g.batch;
  const bool beta_zero = (g.beta.x == 0.0 && g.beta.y == 0.0);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t b = e / mn, rc = e % mn;
    const int r = (int)(rc % g.M), c = (int)(rc / g.M);
    double2 acc = make_double2(0.0, 0.0);
    for (int sp = 0; sp < g.splitk; ++sp) acc = cadd<double>(acc, g.ws[(b * g.splitk + sp) * mn + rc]);
    double2* p = g.C + b * g.strideC + (size_t)r + (size_t)c * g.ldc;
    double2 out = cmul<double>(g.alpha, acc);
    if (!beta_zero) out = cadd<double>(out, cmul<double>(g.beta, *p));
    *p = out;
  }
}
}  // namespace

template <>
cudaError_t gemm_batched<double>(const GemmArgs<double>& g0, cudaStream_t s) {
  if (g0.M <= 0 || g0.N <= 0 || g0.batch <= 0) return cudaSuccess;
  GemmArgs<double> g = g0;
  const size_t tiles = (size_t)ceil_div(g.M, BM) * ceil_div(g.N, BN) * g.batch;
  int S = 1;
  // split only when the tiles fill less than half of the 152 SMs, and keep the
  // split grid within one wave (one 256-thread block per SM)
  if (g.ws && tiles < 76 && g.K >= 4 * BK64 * 2) {
    S = (int)(152 / tiles);
    S = min(S, g.K / (BK64 * 2));  // chunks of at least 16
    while (S > 1 && (size_t)S * g.M * g.N * g.batch > g.ws_elems) --S;
  }
  g.splitk = S;
  dim3 grid(ceil_div(g.M, BM), ceil_div(g.N, BN), g.batch * S);
  feast_count_launch();
  k_zgemm_dmma<<<grid, 256, 0, s>>>(g);
  if (S > 1) {
    const size_t total = (size_t)g.M * g.N * g.batch;
    const size_t want = (total + 255) / 256;
    const unsigned blocks = (unsigned)(want < 152 * 8 ? want : 152 * 8);
    feast_count_launch();
    k_splitk_reduce<<<blocks, 256, 0, s>>>(g);
  }
  return cudaGetLastError();
}

template <>
cudaError_t gemm_batched<float>(const GemmArgs<float>& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  dim3 grid(ceil_div(g.M, BM), ceil_div(g.N, BN), g.batch);
  feast_count_launch();
  k_cgemm_simt<<<grid, 256, 0, s>>>(g);
  return cudaGetLastError();
}

template <>
cudaError_t gemm_grouped<double>(const GemmArgs<double>* tab, const int* tstart, int np, int total_tiles,
                                 const int* active, size_t split_mn, cudaStream_t s) {
  if (np < 1 || total_tiles < 1) return cudaSuccess;
  feast_count_launch();
  k_zgemm_dmma_grp<<<total_tiles, 256, 0, s>>>(tab, tstart, np, active);
  if (split_mn > 0) {
    const size_t want = (split_mn + 255) / 256;
    feast_count_launch();
    k_splitk_reduce_grp<<<dim3((unsigned)(want < 64 ? want : 64), np), 256, 0, s>>>(tab, active);
  }
  return cudaGetLastError();
}

template <>
cudaError_t gemm_grouped<float>(const GemmArgs<float>* tab, const int* tstart, int np, int total_tiles,
                                const int* active, size_t split_mn, cudaStream_t s) {
  (void)split_mn;
  if (np < 1 || total_tiles < 1) return cudaSuccess;
  feast_count_launch();
  k_cgemm_simt_grp<<<total_tiles, 256, 0, s>>>(tab, tstart, np, active);
  return cudaGetLastError();
}

int gemm_tiles(int M, int N) { return (int)(ceil_div(M, BM) * ceil_div(N, BN)); }
