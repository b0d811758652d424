// FP64 kernels of the Rayleigh-Ritz step (Algorithm R-FEAST steps 4-5,
// Algorithm Bi-FEAST steps 6-7): orthonormal bases of the filtered blocks and
// the dense m0 x m0 eigenproblem.
//
// GB300 executes FP64 at about 1/900 of its BF16 rate, so the m0 x m0 work is
// kept small and on chip where possible: the Hessenberg QR iteration keeps
// the matrix (with room for the bulge) packed in shared memory.
#include "small.cuh"

namespace {

constexpr double ULP = 2.220446049250313e-16;
constexpr double SAFE_MIN = 2.2250738585072014e-308;

// ---------------------------------------------------------------- grid barrier
// Sense-counting barrier for a cooperative launch.  Every wait is bounded: after
// about a second the waiting CTA records DEVFLAG_TIMEOUT and the kernel returns.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned* flags, int* s_ok) {
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

// ---------------------------------------------------------------- CGS2
constexpr int ORTH_THREADS = 256;
constexpr int ORTH_MAX_M = 256;

struct OrthArgs {
  double2* Q;
  int n, m, rows_per;
  double2* part;  // 2 x grid x m
  unsigned* bar;  // 2 unsigned
  unsigned* flags;
};

__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
  return t;
}

__global__ void __launch_bounds__(ORTH_THREADS) k_orth_cgs2(OrthArgs a) {
  __shared__ double2 s_r[ORTH_MAX_M];
  __shared__ double red[ORTH_THREADS / 32];
  __shared__ int s_ok;
  const int g = blockIdx.x, G = gridDim.x, tid = threadIdx.x;
  const int n = a.n, m = a.m;
  const int r0 = min(n, g * a.rows_per), r1 = min(n, r0 + a.rows_per);
  double2* Q = a.Q;
  int use = 0;
  for (int j = 0; j < m; ++j) {
    double2* qj = Q + (size_t)j * n;
    for (int pass = 0; pass < 2 && j > 0; ++pass) {
      double2* part = a.part + (size_t)(use & 1) * G * m;
      for (int i = tid; i < j; i += ORTH_THREADS) {
        const double2* qi = Q + (size_t)i * n;
        double2 acc = make_double2(0.0, 0.0);
        for (int r = r0; r < r1; ++r) acc = cadd<double>(acc, cmulc<double>(qi[r], qj[r]));
        part[(size_t)g * m + i] = acc;
      }
      if (!grid_barrier(a.bar, G, a.flags, &s_ok)) return;
      for (int i = tid; i < j; i += ORTH_THREADS) {
        double2 acc = make_double2(0.0, 0.0);
        for (int gg = 0; gg < G; ++gg) acc = cadd<double>(acc, part[(size_t)gg * m + i]);
        s_r[i] = acc;
      }
      __syncthreads();
      for (int r = r0 + tid; r < r1; r += ORTH_THREADS) {
        double2 acc = qj[r];
        for (int i = 0; i < j; ++i) acc = csub<double>(acc, cmul<double>(Q[(size_t)i * n + r], s_r[i]));
        qj[r] = acc;
      }
      __syncthreads();
      ++use;
    }
    double2* part = a.part + (size_t)(use & 1) * G * m;
    double loc = 0.0;
    for (int r = r0 + tid; r < r1; r += ORTH_THREADS) loc += cnorm2<double>(qj[r]);
    loc = block_sum(loc, red);
    if (tid == 0) part[(size_t)g * m] = make_double2(loc, 0.0);
    if (!grid_barrier(a.bar, G, a.flags, &s_ok)) return;
    double tot = 0.0;
    for (int gg = 0; gg < G; ++gg) tot += part[(size_t)gg * m].x;
    const double inv = tot > 0.0 ? 1.0 / sqrt(tot) : 0.0;
    for (int r = r0 + tid; r < r1; r += ORTH_THREADS) qj[r] = cscale<double>(qj[r], inv);
    __syncthreads();
    ++use;
  }
}

// ---------------------------------------------------------------- small LU
constexpr int SMALL_THREADS = 1024;

__global__ void __launch_bounds__(SMALL_THREADS) k_small_lu(double2* M, int m, int* piv, unsigned* flags) {
  __shared__ int s_p;
  const int tid = threadIdx.x;
  for (int k = 0; k < m; ++k) {
    if (tid < 32) {
      double best = -1.0;
      int bi = m;
      for (int i = k + tid; i < m; i += 32) {
        const double v = cabs1<double>(M[i + (size_t)k * m]);
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double v2 = __shfl_down_sync(0xffffffffu, best, off);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, off);
        if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
      }
      if (tid == 0) {
        if (bi >= m) { bi = k; atomicOr(flags, (unsigned)DEVFLAG_NONFINITE); }
        piv[k] = bi;
        s_p = bi;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p != k)
      for (int j = tid; j < m; j += SMALL_THREADS) {
        const double2 t = M[k + (size_t)j * m];
        M[k + (size_t)j * m] = M[p + (size_t)j * m];
        M[p + (size_t)j * m] = t;
      }
    __syncthreads();
    const double2 d = M[k + (size_t)k * m];
    if (d.x == 0.0 && d.y == 0.0) {
      if (tid == 0) atomicOr(flags, (unsigned)DEVFLAG_SINGULAR);
      __syncthreads();
      continue;
    }
    const double2 rinv = crecip<double>(d);
    for (int i = k + 1 + tid; i < m; i += SMALL_THREADS) M[i + (size_t)k * m] = cmul<double>(M[i + (size_t)k * m], rinv);
    __syncthreads();
    const int w = m - k - 1;
    for (int idx = tid; idx < w * w; idx += SMALL_THREADS) {
      const int i = k + 1 + idx % w, j = k + 1 + idx / w;
      M[i + (size_t)j * m] = csub<double>(M[i + (size_t)j * m], cmul<double>(M[i + (size_t)k * m], M[k + (size_t)j * m]));
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SMALL_THREADS)
k_small_lu_solve(const double2* LU, const int* piv, int m, double2* X, int nrhs, int trans) {
  const int tid = threadIdx.x;
  auto Lx = [&](int i, int j) { return LU[i + (size_t)j * m]; };
  auto Xr = [&](int i, int c) -> double2& { return X[i + (size_t)c * m]; };
  if (trans == 0) {
    for (int c = tid; c < nrhs; c += SMALL_THREADS)
      for (int k = 0; k < m; ++k) {
        const int p = piv[k];
        if (p != k) { double2 t = Xr(k, c); Xr(k, c) = Xr(p, c); Xr(p, c) = t; }
      }
    __syncthreads();
    for (int k = 0; k < m - 1; ++k) {
      const int w = m - k - 1;
      for (int idx = tid; idx < w * nrhs; idx += SMALL_THREADS) {
        const int i = k + 1 + idx % w, c = idx / w;
        Xr(i, c) = csub<double>(Xr(i, c), cmul<double>(Lx(i, k), Xr(k, c)));
      }
      __syncthreads();
    }
    for (int k = m - 1; k >= 0; --k) {
      for (int c = tid; c < nrhs; c += SMALL_THREADS) Xr(k, c) = cdiv<double>(Xr(k, c), Lx(k, k));
      __syncthreads();
      for (int idx = tid; idx < k * nrhs; idx += SMALL_THREADS) {
        const int i = idx % k, c = idx / k;
        Xr(i, c) = csub<double>(Xr(i, c), cmul<double>(Lx(i, k), Xr(k, c)));
      }
      __syncthreads();
    }
  } else {
    for (int k = 0; k < m; ++k) {  // U^H w = x
      for (int c = tid; c < nrhs; c += SMALL_THREADS) Xr(k, c) = cdiv<double>(Xr(k, c), cconj<double>(Lx(k, k)));
      __syncthreads();
      const int w = m - k - 1;
      for (int idx = tid; idx < w * nrhs; idx += SMALL_THREADS) {
        const int i = k + 1 + idx % w, c = idx / w;
        Xr(i, c) = csub<double>(Xr(i, c), cmulc<double>(Lx(k, i), Xr(k, c)));
      }
      __syncthreads();
    }
    for (int k = m - 1; k >= 1; --k) {  // L^H v = w
      for (int idx = tid; idx < k * nrhs; idx += SMALL_THREADS) {
        const int i = idx % k, c = idx / k;
        Xr(i, c) = csub<double>(Xr(i, c), cmulc<double>(Lx(k, i), Xr(k, c)));
      }
      __syncthreads();
    }
    for (int c = tid; c < nrhs; c += SMALL_THREADS)
      for (int k = m - 1; k >= 0; --k) {
        const int p = piv[k];
        if (p != k) { double2 t = Xr(k, c); Xr(k, c) = Xr(p, c); Xr(p, c) = t; }
      }
  }
}

// ---------------------------------------------------------------- Schur form
constexpr int SCHUR_THREADS = 256;
constexpr int SCHUR_MAX_M = 160;

__device__ __forceinline__ double2 csqrt_d(double2 z) {
  const double r = hypot(z.x, z.y);
  if (r == 0.0) return make_double2(0.0, 0.0);
  const double re = sqrt(0.5 * (r + fabs(z.x)));
  const double other = z.y / (2.0 * re);
  if (z.x >= 0.0) return make_double2(re, other);
  return make_double2(fabs(other), z.y >= 0.0 ? re : -re);
}

// packed storage: column j keeps rows 0 .. j+2 (Hessenberg plus the bulge diagonal)
__device__ __forceinline__ int hp_off(int i, int j) { return j * (j + 5) / 2 + i; }

// Givens rotation G = [c s; -conj(s) c] with G [x; y] = [r; 0], c real.
__device__ void givens(double2 x, double2 y, double& c, double2& s) {
  const double ax = hypot(x.x, x.y), ay = hypot(y.x, y.y);
  if (ay == 0.0) { c = 1.0; s = make_double2(0.0, 0.0); return; }
  if (ax == 0.0) { c = 0.0; s = make_double2(1.0, 0.0); return; }
  const double nu = hypot(ax, ay);
  c = ax / nu;
  const double2 ph = make_double2(x.x / ax, x.y / ax);
  s = cscale<double>(cmul<double>(ph, cconj<double>(y)), 1.0 / nu);
}

__global__ void __launch_bounds__(SCHUR_THREADS)
k_small_schur(double2* C, double2* Z, double2* lam, int m, unsigned* flags) {
  extern __shared__ unsigned char smem_raw[];
  double2* H = reinterpret_cast<double2*>(smem_raw);
  __shared__ double2 s_u[SCHUR_MAX_M];
  __shared__ double red[SCHUR_THREADS / 32];
  __shared__ double s_c;
  __shared__ double2 s_s, s_beta;
  __shared__ int s_l, s_skip;
  const int tid = threadIdx.x;
  auto Cg = [&](int i, int j) -> double2& { return C[i + (size_t)j * m]; };
  auto Zg = [&](int i, int j) -> double2& { return Z[i + (size_t)j * m]; };
  for (int idx = tid; idx < m * m; idx += SCHUR_THREADS)
    Z[idx] = make_double2((idx % m) == (idx / m) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  // ---- Householder reduction to upper Hessenberg form, Z <- Z H_k
  for (int k = 0; k + 2 < m; ++k) {
    const int len = m - k - 1;
    double loc = 0.0;
    for (int i = 1 + tid; i < len; i += SCHUR_THREADS) loc += cnorm2<double>(Cg(k + 1 + i, k));
    const double tail = block_sum(loc, red);
    if (tid == 0) {
      const double2 x0 = Cg(k + 1, k);
      const double a0 = hypot(x0.x, x0.y);
      s_skip = (tail == 0.0);
      const double alpha = sqrt(tail + a0 * a0);
      const double2 beta = a0 > 0.0 ? make_double2(-x0.x / a0 * alpha, -x0.y / a0 * alpha) : make_double2(-alpha, 0.0);
      s_beta = beta;
      s_u[0] = csub<double>(x0, beta);
    }
    __syncthreads();
    if (s_skip) { __syncthreads(); continue; }
    for (int i = 1 + tid; i < len; i += SCHUR_THREADS) s_u[i] = Cg(k + 1 + i, k);
    __syncthreads();
    double uu_loc = 0.0;
    for (int i = tid; i < len; i += SCHUR_THREADS) uu_loc += cnorm2<double>(s_u[i]);
    const double uu = block_sum(uu_loc, red);
    const double t = 2.0 / uu;
    // left: columns k .. m-1
    for (int c = k + tid; c < m; c += SCHUR_THREADS) {
      double2 s = make_double2(0.0, 0.0);
      for (int i = 0; i < len; ++i) s = cadd<double>(s, cmulc<double>(s_u[i], Cg(k + 1 + i, c)));
      s = cscale<double>(s, t);
      for (int i = 0; i < len; ++i) Cg(k + 1 + i, c) = csub<double>(Cg(k + 1 + i, c), cmul<double>(s_u[i], s));
    }
    __syncthreads();
    // right: all rows of C and Z, columns k+1 .. m-1
    for (int r = tid; r < 2 * m; r += SCHUR_THREADS) {
      double2* P = r < m ? C : Z;
      const int rr = r < m ? r : r - m;
      double2 s = make_double2(0.0, 0.0);
      for (int i = 0; i < len; ++i) s = cadd<double>(s, cmul<double>(P[rr + (size_t)(k + 1 + i) * m], s_u[i]));
      s = cscale<double>(s, t);
      for (int i = 0; i < len; ++i) {
        double2& e = P[rr + (size_t)(k + 1 + i) * m];
        e = csub<double>(e, cmul<double>(s, cconj<double>(s_u[i])));
      }
    }
    __syncthreads();
    if (tid == 0) Cg(k + 1, k) = s_beta;
    for (int i = 1 + tid; i < len; i += SCHUR_THREADS) Cg(k + 1 + i, k) = make_double2(0.0, 0.0);
    __syncthreads();
  }
  // ---- copy to packed shared memory
  for (int j = 0; j < m; ++j)
    for (int i = tid; i <= j + 2; i += SCHUR_THREADS)
      H[hp_off(i, j)] = (i < m && i <= j + 1) ? Cg(i, j) : make_double2(0.0, 0.0);
  __syncthreads();
  // ---- shifted QR iterations to the complex Schur form
  int ihi = m - 1, its = 0, total = 0;
  const int max_total = 30 * m + 100;
  while (ihi >= 0) {
    if (tid == 0) {
      int l = 0;
      for (int k = ihi; k >= 1; --k) {
        double tst = cabs1<double>(H[hp_off(k - 1, k - 1)]) + cabs1<double>(H[hp_off(k, k)]);
        if (tst == 0.0) tst = 1.0;
        if (cabs1<double>(H[hp_off(k, k - 1)]) <= fmax(ULP * tst, SAFE_MIN * (m / ULP))) {
          H[hp_off(k, k - 1)] = make_double2(0.0, 0.0);
          l = k;
          break;
        }
      }
      s_l = l;
    }
    __syncthreads();
    const int l = s_l;
    if (l == ihi) {
      if (tid == 0) lam[ihi] = H[hp_off(ihi, ihi)];
      --ihi;
      its = 0;
      __syncthreads();
      continue;
    }
    ++its;
    if (++total > max_total) {
      if (tid == 0) {
        atomicOr(flags, (unsigned)DEVFLAG_TIMEOUT);
        for (int i = 0; i <= ihi; ++i) lam[i] = H[hp_off(i, i)];
      }
      break;
    }
    for (int k = l; k < ihi; ++k) {
      if (tid == 0) {
        double2 x, y;
        if (k == l) {
          double2 sh;
          const double2 a = H[hp_off(ihi - 1, ihi - 1)], b = H[hp_off(ihi - 1, ihi)];
          const double2 cc = H[hp_off(ihi, ihi - 1)], d = H[hp_off(ihi, ihi)];
          if (its % 10 == 0) {
            sh = make_double2(d.x + 0.75 * fabs(cc.x), d.y);
          } else {
            const double2 p = cscale<double>(csub<double>(a, d), 0.5);
            const double2 bc = cmul<double>(b, cc);
            const double2 disc = csqrt_d(cadd<double>(cmul<double>(p, p), bc));
            const double2 d1 = cadd<double>(p, disc), d2 = csub<double>(p, disc);
            const double2 den = cabs1<double>(d1) >= cabs1<double>(d2) ? d1 : d2;
            sh = (den.x == 0.0 && den.y == 0.0) ? d : csub<double>(d, cdiv<double>(bc, den));
          }
          x = csub<double>(H[hp_off(l, l)], sh);
          y = H[hp_off(l + 1, l)];
        } else {
          x = H[hp_off(k, k - 1)];
          y = H[hp_off(k + 1, k - 1)];
        }
        double c;
        double2 s;
        givens(x, y, c, s);
        s_c = c;
        s_s = s;
      }
      __syncthreads();
      const double c = s_c;
      const double2 s = s_s;
      const double2 ms = make_double2(-s.x, s.y);  // -conj(s)
      const int j0 = (k == l) ? l : k - 1;
      for (int j = j0 + tid; j < m; j += SCHUR_THREADS) {
        const double2 a = H[hp_off(k, j)], b = H[hp_off(k + 1, j)];
        H[hp_off(k, j)] = cadd<double>(cscale<double>(a, c), cmul<double>(s, b));
        H[hp_off(k + 1, j)] = cadd<double>(cmul<double>(ms, a), cscale<double>(b, c));
      }
      __syncthreads();
      const int imax = min(k + 2, ihi);
      const double2 sc = cconj<double>(s), nsv = make_double2(-s.x, -s.y);
      for (int i = tid; i <= imax; i += SCHUR_THREADS) {
        const double2 a = H[hp_off(i, k)], b = H[hp_off(i, k + 1)];
        H[hp_off(i, k)] = cadd<double>(cscale<double>(a, c), cmul<double>(b, sc));
        H[hp_off(i, k + 1)] = cadd<double>(cmul<double>(a, nsv), cscale<double>(b, c));
      }
      for (int i = tid; i < m; i += SCHUR_THREADS) {
        const double2 a = Zg(i, k), b = Zg(i, k + 1);
        Zg(i, k) = cadd<double>(cscale<double>(a, c), cmul<double>(b, sc));
        Zg(i, k + 1) = cadd<double>(cmul<double>(a, nsv), cscale<double>(b, c));
      }
      __syncthreads();
      if (k > l && tid == 0) H[hp_off(k + 1, k - 1)] = make_double2(0.0, 0.0);
      __syncthreads();
    }
  }
  __syncthreads();
  // ---- T back to global (upper triangle), strictly lower part zero
  for (int idx = tid; idx < m * m; idx += SCHUR_THREADS) {
    const int i = idx % m, j = idx / m;
    C[idx] = (i <= j) ? H[hp_off(i, j)] : make_double2(0.0, 0.0);
  }
}

// ---------------------------------------------------------------- eigenvectors of T
__global__ void k_small_trevc(const double2* T, double2* V, int m) {
  __shared__ double red[32];
  const int k = threadIdx.x;
  double loc = 0.0;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    if (i <= j) loc = fmax(loc, cabs1<double>(T[idx]));
  }
  // block max
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) loc = fmax(loc, __shfl_down_sync(0xffffffffu, loc, off));
  if (lane == 0) red[wid] = loc;
  __syncthreads();
  double tnorm = 0.0;
  for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) tnorm = fmax(tnorm, red[w]);
  const double smin = fmax(ULP * tnorm, SAFE_MIN * (m / ULP));
  if (k >= m) return;
  double2* v = V + (size_t)k * m;
  for (int i = k + 1; i < m; ++i) v[i] = make_double2(0.0, 0.0);
  v[k] = make_double2(1.0, 0.0);
  const double2 lk = T[k + (size_t)k * m];
  for (int i = k - 1; i >= 0; --i) {
    double2 s = make_double2(0.0, 0.0);
    for (int j = i + 1; j <= k; ++j) s = cadd<double>(s, cmul<double>(T[i + (size_t)j * m], v[j]));
    double2 d = csub<double>(T[i + (size_t)i * m], lk);
    if (cabs1<double>(d) < smin) d = make_double2(smin, 0.0);
    double2 vi = cdiv<double>(s, d);
    v[i] = make_double2(-vi.x, -vi.y);
    if (cabs1<double>(v[i]) > 1e150) {  // keep the partial column representable
      for (int j = i; j <= k; ++j) v[j] = cscale<double>(v[j], 1e-150);
    }
  }
}

}  // namespace

size_t orth_scratch_bytes(int n, int m) {
  return (size_t)2 * 160 * m * sizeof(double2) + 64;
}

cudaError_t orth_cgs2(double2* Q, int n, int m, void* scratch, unsigned* flags, cudaStream_t s) {
  if (m > ORTH_MAX_M || m < 1 || n < 1) return cudaErrorInvalidValue;
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_orth_cgs2, ORTH_THREADS, 0);
  int G = min(nsm * max(per, 1), 128);
  G = min(G, max(1, (n + 15) / 16));
  G = min(G, 160);
  OrthArgs a;
  a.Q = Q; a.n = n; a.m = m;
  a.rows_per = (n + G - 1) / G;
  G = (n + a.rows_per - 1) / a.rows_per;
  a.bar = reinterpret_cast<unsigned*>(scratch);
  a.part = reinterpret_cast<double2*>(reinterpret_cast<char*>(scratch) + 64);
  a.flags = flags;
  cudaMemsetAsync(a.bar, 0, 64, s);
  void* args[] = {&a};
  feast_count_launch();
  return cudaLaunchCooperativeKernel((void*)k_orth_cgs2, dim3(G), dim3(ORTH_THREADS), args, 0, s);
}

cudaError_t small_lu(double2* M, int m, int* piv, unsigned* flags, cudaStream_t s) {
  feast_count_launch();
  k_small_lu<<<1, SMALL_THREADS, 0, s>>>(M, m, piv, flags);
  return cudaGetLastError();
}

cudaError_t small_lu_solve(const double2* LU, const int* piv, int m, double2* X, int nrhs, int trans,
                           cudaStream_t s) {
  feast_count_launch();
  k_small_lu_solve<<<1, SMALL_THREADS, 0, s>>>(LU, piv, m, X, nrhs, trans);
  return cudaGetLastError();
}

cudaError_t small_schur(double2* C, double2* Z, double2* lam, int m, unsigned* flags, cudaStream_t s) {
  if (m < 1 || m > SCHUR_MAX_M) return cudaErrorInvalidValue;
  const size_t smem = (size_t)(m * (m + 5) / 2 + 8) * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_small_schur, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  feast_count_launch();
  k_small_schur<<<1, SCHUR_THREADS, smem, s>>>(C, Z, lam, m, flags);
  return cudaGetLastError();
}

cudaError_t small_trevc(const double2* T, double2* V, int m, cudaStream_t s) {
  const int threads = ((m + 31) / 32) * 32;
  feast_count_launch();
  k_small_trevc<<<1, threads, 0, s>>>(T, V, m);
  return cudaGetLastError();
}
