// Power iteration for ||A||_2 as one persistent cooperative kernel.
//
// Phase 1, y = A x: a block owns 32 rows and sweeps all columns (column-major
// A: each warp reads 32 consecutive rows of a column, 512 B).  Phase 2,
// z = A^H y: one warp per column, lanes down the contiguous column.  Phase 3:
// ||z|| from one partial sum per block, x = z / ||z||.  Three bounded grid
// barriers per iteration; A streams from HBM twice per iteration.
#include "norm2.cuh"

namespace {

constexpr int PW_THREADS = 256;
constexpr int PW_ROWS = 32;

struct PowArgs {
  const double2* A;
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
  __shared__ double2 sacc[PW_THREADS / 32][PW_ROWS];
  __shared__ double red[PW_THREADS / 32];
  __shared__ int s_ok;
  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.n;
  const int nblk = (n + PW_ROWS - 1) / PW_ROWS;
  const double2* A = a.A;
  const double inv0 = 1.0 / sqrt((double)n);
  for (int i = g * PW_THREADS + tid; i < n; i += G * PW_THREADS) a.x[i] = make_double2(inv0, 0.0);
  if (!pw_barrier(a.bar, G, a.flags, &s_ok)) return;
  double s = 0.0;
  for (int it = 0; it < a.iters; ++it) {
    // y = A x
    for (int blk = g; blk < nblk; blk += G) {
      const int r = blk * PW_ROWS + lane;
      double2 acc = make_double2(0.0, 0.0);
      if (r < n) {
#pragma unroll 4
        for (int c = warp; c < n; c += PW_THREADS / 32) cfma<double>(acc, A[(size_t)r + (size_t)c * a.lda], a.x[c]);
      }
      sacc[warp][lane] = acc;
      __syncthreads();
      if (warp == 0 && r < n) {
        double2 t = sacc[0][lane];
        for (int w = 1; w < PW_THREADS / 32; ++w) t = cadd<double>(t, sacc[w][lane]);
        a.y[r] = t;
      }
      __syncthreads();
    }
    if (!pw_barrier(a.bar, G, a.flags, &s_ok)) return;
    // z = A^H y, kept in x until normalised
    double loc = 0.0;
    for (int blk = g; blk < nblk; blk += G) {
      for (int cc = warp; cc < PW_ROWS; cc += PW_THREADS / 32) {
        const int c = blk * PW_ROWS + cc;
        if (c >= n) continue;
        const double2* col = A + (size_t)c * a.lda;
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll 4
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
    double tot = 0.0;
    for (int k = 0; k < G; ++k) tot += a.part[k];
    const double nz = sqrt(tot);
    s = sqrt(nz);
    const double inv = nz > 0.0 ? 1.0 / nz : 0.0;
    for (int blk = g; blk < nblk; blk += G) {
      const int c = blk * PW_ROWS + tid;
      if (tid < PW_ROWS && c < n) a.x[c] = cscale<double>(a.x[c], inv);
    }
    if (!pw_barrier(a.bar, G, a.flags, &s_ok)) return;
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

cudaError_t norm2_power(const double2* A, long long lda, int n, int iters, void* scratch, double* out_dev,
                        unsigned* flags, cudaStream_t s) {
  if (n < 1 || iters < 1 || !A || !scratch || !out_dev) return cudaErrorInvalidValue;
  char* base = reinterpret_cast<char*>(scratch);
  PowArgs a;
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
