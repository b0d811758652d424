// Power iteration for ||A||_2 as one persistent cooperative kernel.
//
// Phase 1, y = c A x (c = 1 / ||x|| from the previous step): with A^T at hand
// (k_transpose_c128) one warp per row of A, lanes down the contiguous column
// of A^T; else a block owns 16 rows and lane l of a warp reads row l % 16 of
// column 2w + l / 16 (256-byte segments).  Phase 2, x <- A^H y: one warp per
// column, lanes down the contiguous column; one partial sum of |x|^2 per block,
// reduced by every block in the same order.  Two bounded grid barriers per
// iteration.  Each step does 8 n^2 FP64 FMA on 2 n^2 16-byte reads, so on
// GB300 (FP64 at about 1/64 of FP32) the FP64 pipes bound it, not HBM.
#include "norm2.cuh"

namespace {

constexpr int PW_THREADS = 256;
constexpr int PW_ROWS = 16;

struct PowArgs {
  const double2* A;
  const double2* At;  // A^T (ld n) or nullptr
  long long lda;
  int n, iters;
  double2* x;
  double2* y;
  double* part;
  unsigned* bar;
  unsigned* flags;
  double* out;
};

// Bounded sense-counting barrier (about one second per wait at most; on
// timeout DEVFLAG_TIMEOUT is raised and the kernel returns).
__device__ bool pw_barrier(unsigned* bar, unsigned nblocks, unsigned* flags, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    int ok = 1;
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long spins = 0;
      while (*vgen == gen) {
        if (++spins > (1ull << 24)) {
          atomicOr(flags, (unsigned)DEVFLAG_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__global__ void __launch_bounds__(PW_THREADS) k_norm2_power(PowArgs a) {
  __shared__ double2 sacc[2 * PW_THREADS / 32][PW_ROWS];
  __shared__ double red[PW_THREADS / 32];
  __shared__ int s_ok;
  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.n;
  const int nblk = (n + PW_ROWS - 1) / PW_ROWS;
  const double2* A = a.A;
  constexpr int NSTREAM = 2 * PW_THREADS / 32;  // column streams of phase 1
  for (int i = g * PW_THREADS + tid; i < n; i += G * PW_THREADS) a.x[i] = make_double2(1.0, 0.0);
  double xs = 1.0 / sqrt((double)n);  // x = xs * (stored x): the unit start vector
  if (!pw_barrier(a.bar, G, a.flags, &s_ok)) return;
  double s = 0.0;
  for (int it = 0; it < a.iters; ++it) {
    // y = xs A x: with A^T at hand one warp per row, lanes down the contiguous
    // column of A^T; else 16-row blocks of A
    if (a.At) {
      for (int blk = g; blk < nblk; blk += G) {
        for (int rr = warp; rr < PW_ROWS; rr += PW_THREADS / 32) {
          const int r = blk * PW_ROWS + rr;
          if (r >= n) continue;
          const double2* row = a.At + (size_t)r * n;
          double2 acc = make_double2(0.0, 0.0);
#pragma unroll 8
          for (int c = lane; c < n; c += 32) cfma<double>(acc, row[c], a.x[c]);
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
          }
          if (lane == 0) a.y[r] = cscale<double>(acc, xs);
        }
      }
    } else
    for (int blk = g; blk < nblk; blk += G) {
      const int r = blk * PW_ROWS + (lane & 15);
      const int stream = 2 * warp + (lane >> 4);
      double2 acc = make_double2(0.0, 0.0);
      if (r < n) {
#pragma unroll 8
        for (int c = stream; c < n; c += NSTREAM) cfma<double>(acc, A[(size_t)r + (size_t)c * a.lda], a.x[c]);
      }
      sacc[stream][lane & 15] = acc;
      __syncthreads();
      if (tid < PW_ROWS && blk * PW_ROWS + tid < n) {
        double2 t = sacc[0][tid];
        for (int w = 1; w < NSTREAM; ++w) t = cadd<double>(t, sacc[w][tid]);
        a.y[blk * PW_ROWS + tid] = cscale<double>(t, xs);
      }
      __syncthreads();
    }
    if (!pw_barrier(a.bar, G, a.flags, &s_ok)) return;
    // x = A^H y (unnormalised; the next phase 1 applies 1 / ||x||)
    double loc = 0.0;
    for (int blk = g; blk < nblk; blk += G) {
      for (int cc = warp; cc < PW_ROWS; cc += PW_THREADS / 32) {
        const int c = blk * PW_ROWS + cc;
        if (c >= n) continue;
        const double2* col = A + (size_t)c * a.lda;
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll 8
        for (int r = lane; r < n; r += 32) acc = cadd<double>(acc, cmulc<double>(col[r], a.y[r]));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
          acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
        }
        if (lane == 0) {
          a.x[c] = acc;
          loc += cnorm2<double>(acc);
        }
      }
    }
    if (lane == 0) red[warp] = loc;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < PW_THREADS / 32; ++w) t += red[w];
      a.part[g] = t;
    }
    if (!pw_barrier(a.bar, G, a.flags, &s_ok)) return;
    // every block sums the G partials in the same order (one per thread, then a
    // fixed shuffle tree), so all blocks hold the same total
    double tot = 0.0;
    for (int k = tid; k < G; k += PW_THREADS) tot += __ldcg(&a.part[k]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, off);
    __syncthreads();
    if (lane == 0) red[warp] = tot;
    __syncthreads();
    tot = 0.0;
    for (int w = 0; w < PW_THREADS / 32; ++w) tot += red[w];
    const double nz = sqrt(tot);  // ||A^H A u|| for the unit vector u of this step
    s = sqrt(nz);
    xs = nz > 0.0 ? 1.0 / nz : 0.0;
  }
  if (g == 0 && tid == 0) *a.out = s;
}

int pw_grid(int n) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_norm2_power, PW_THREADS, 0);
  const int nblk = (n + PW_ROWS - 1) / PW_ROWS;
  int G = nsm * (per > 0 ? per : 1);
  if (G > 1024) G = 1024;
  return nblk < G ? nblk : G;
}

}  // namespace

size_t norm2_scratch_bytes(int n) {
  return 256 + (size_t)2 * n * sizeof(double2) + 1024 * sizeof(double);
}

// A^T (n x n, ld n) from A (ld lda): 32 x 32 tiles through shared memory.
__global__ void k_transpose_c128(const double2* A, long long lda, int n, double2* At) {
  __shared__ double2 tile[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int i = i0 + threadIdx.x, j = j0 + k;
    if (i < n && j < n) tile[k][threadIdx.x] = A[(size_t)i + (size_t)j * lda];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int j = j0 + threadIdx.x, i = i0 + k;
    if (i < n && j < n) At[(size_t)j + (size_t)i * n] = tile[threadIdx.x][k];
  }
}

cudaError_t norm2_power(const double2* A, long long lda, int n, int iters, void* scratch, double* out_dev,
                        unsigned* flags, cudaStream_t s, double2* At) {
  if (n < 1 || iters < 1 || !A || !scratch || !out_dev) return cudaErrorInvalidValue;
  char* base = reinterpret_cast<char*>(scratch);
  if (At) {
    feast_count_launch();
    k_transpose_c128<<<dim3((n + 31) / 32, (n + 31) / 32), dim3(32, 8), 0, s>>>(A, lda, n, At);
  }
  PowArgs a;
  a.At = At;
  a.A = A;
  a.lda = lda;
  a.n = n;
  a.iters = iters;
  a.bar = reinterpret_cast<unsigned*>(base);
  a.x = reinterpret_cast<double2*>(base + 256);
  a.y = a.x + n;
  a.part = reinterpret_cast<double*>(a.y + n);
  a.flags = flags;
  a.out = out_dev;
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const int G = pw_grid(n);
  void* args[] = {&a};
  feast_count_launch();
  return cudaLaunchCooperativeKernel((void*)k_norm2_power, dim3(G), dim3(PW_THREADS), args, 0, s);
}
