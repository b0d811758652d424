// FP64 kernels of the Rayleigh-Ritz step (Algorithm R-FEAST steps 4-5,
// Algorithm Bi-FEAST steps 6-7): orthonormal bases of the filtered blocks
// (CGS2, with every CTA's rows of Q in shared memory where they fit), the
// small dense LU and its solves, the FP32 Gauss-Jordan start of the
// Newton-Schulz inverses and the device-side checks that guard them, and the
// grouped forms of these for the batched path.
//
// GB300 executes FP64 at about 1/900 of its BF16 rate, so this work is kept
// small and on chip where possible.
#include "small.cuh"

namespace {

constexpr double SAFE_MIN = 2.2250738585072014e-308;

// ---------------------------------------------------------------- grid barriers
// Sense-counting barriers for cooperative launches; every wait is bounded by
// the global timer (the host's wait limit), after which the waiting CTA records
// DEVFLAG_TIMEOUT and the kernel returns.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// The generation word on its own 128-byte line (bar + 32).
__device__ bool grid_barrier_spin(unsigned* bar, unsigned nblocks, unsigned* flags, int* s_ok,
                                  unsigned long long limit_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned* gptr = bar + 32;
    const unsigned gen = ld_acquire_u32(gptr);
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    int ok = 1;
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 32, 1u);
    } else {
      // poll with acquire loads; the global timer is read after the first
      // unsuccessful poll and then once per 64 polls
      const unsigned long long t0 = global_ns();
      for (unsigned polls = 1;; ++polls) {
        if (ld_acquire_u32(gptr) != gen) break;
        if ((polls & 63) == 1 && global_ns() - t0 > limit_ns) {
          atomicOr(flags, (unsigned)DEVFLAG_TIMEOUT);
          ok = 0;
          break;
        }
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
  double2* fin = nullptr;  // 2 x (m + 1): the reduced slots of a phase (shared-memory kernel)
  unsigned* bar;  // 2 unsigned
  unsigned long long wait_ns = 1000000000ull;  // limit of each grid-barrier wait (spin form)
  unsigned* flags;
  int col0 = 0;  // index of column 0 within a larger basis (restart rows differ per panel)
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

// A column that the second projection shrinks below 1/sqrt(2) of what the first
// left (or to zero) lies numerically in the span of the earlier columns
// (Kahan's criterion for 'twice is enough'); it restarts from the unit vector
// e_r, r drawn from the column index and the attempt number.  After
// ORTH_RETRIES attempts the column is kept as it is.
constexpr int ORTH_RETRIES = 3;
__device__ __forceinline__ int orth_restart_row(int c, int attempt, int n) {
  return (int)(((long long)c * 7919 + (long long)(attempt + 1) * 104729) % n);
}

// The sense-counting barrier with acquire-load polling, bounded by the global
// timer (read after the first unsuccessful poll, then once per 64); the
// generation word is bar + 1, as for grid_barrier.
__device__ bool grid_barrier_poll(unsigned* bar, unsigned nblocks, unsigned* flags, int* s_ok,
                                  unsigned long long limit_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned* gptr = bar + 1;
    const unsigned gen = ld_acquire_u32(gptr);
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    int ok = 1;
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      for (unsigned polls = 1;; ++polls) {
        if (ld_acquire_u32(gptr) != gen) break;
        if ((polls & 63) == 1 && global_ns() - t0 > limit_ns) {
          atomicOr(flags, (unsigned)DEVFLAG_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// CTA g of the G that share one block Q.
__device__ __forceinline__ void orth_body(const OrthArgs& a, const int g, const int G) {
  __shared__ double2 s_r[ORTH_MAX_M];
  __shared__ double red[ORTH_THREADS / 32];
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  const int n = a.n, m = a.m;
  const int r0 = min(n, g * a.rows_per), r1 = min(n, r0 + a.rows_per);
  double2* Q = a.Q;
  int use = 0, retries = 0;
  double r1sq = 0.0;  // |q_j|^2 after the first projection
  for (int j = 0; j < m;) {
    double2* qj = Q + (size_t)j * n;
    r1sq = 0.0;
    for (int pass = 0; pass < 2 && j > 0; ++pass) {
      double2* part = a.part + (size_t)(use & 1) * G * m;
      // the second pass also sums |q_j|^2 (slot j)
      const int ns = pass == 1 ? j + 1 : j;
      for (int i = tid; i < ns; i += ORTH_THREADS) {
        const double2* qi = Q + (size_t)i * n;
        double2 acc = make_double2(0.0, 0.0);
        if (i < j) {
#pragma unroll 8
          for (int r = r0; r < r1; ++r) acc = cadd<double>(acc, cmulc<double>(qi[r], qj[r]));
        } else {
          for (int r = r0; r < r1; ++r) acc.x += cnorm2<double>(qj[r]);
        }
        part[(size_t)g * m + i] = acc;
      }
      if (!grid_barrier_poll(a.bar, G, a.flags, &s_ok, a.wait_ns)) return;
      // the G partial dot products of each coefficient: few partials are summed
      // by one thread each; many by one warp (parallel reads, shuffle sums)
      if (G <= 16) {
        for (int i = tid; i < ns; i += ORTH_THREADS) {
          double2 acc = make_double2(0.0, 0.0);
          for (int gg = 0; gg < G; ++gg) acc = cadd<double>(acc, __ldcg(part + (size_t)gg * m + i));
          s_r[i] = acc;
        }
      } else
      for (int i = tid >> 5; i < ns; i += ORTH_THREADS / 32) {
        const int lane = tid & 31;
        double2 acc = make_double2(0.0, 0.0);
        for (int gg = lane; gg < G; gg += 32) acc = cadd<double>(acc, __ldcg(part + (size_t)gg * m + i));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
          acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        }
        if (lane == 0) s_r[i] = acc;
      }
      __syncthreads();
      if (pass == 1) r1sq = s_r[j].x;
      for (int r = r0 + tid; r < r1; r += ORTH_THREADS) {
        double2 acc = qj[r];
#pragma unroll 8
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
    if (!grid_barrier_poll(a.bar, G, a.flags, &s_ok, a.wait_ns)) return;
    double tot = 0.0;
    for (int gg = tid; gg < G; gg += ORTH_THREADS) tot += __ldcg(&part[(size_t)gg * m].x);
    tot = block_sum(tot, red);
    ++use;
    if ((!(tot > SAFE_MIN) || tot < 0.5 * r1sq) && retries < ORTH_RETRIES) {
      const int rr = orth_restart_row(a.col0 + j, retries++, n);
      for (int r = r0 + tid; r < r1; r += ORTH_THREADS) qj[r] = make_double2(r == rr ? 1.0 : 0.0, 0.0);
      __syncthreads();
      continue;
    }
    const double inv = tot > 0.0 ? 1.0 / sqrt(tot) : 0.0;
    for (int r = r0 + tid; r < r1; r += ORTH_THREADS) qj[r] = cscale<double>(qj[r], inv);
    __syncthreads();
    retries = 0;
    ++j;
  }
}

__global__ void __launch_bounds__(ORTH_THREADS) k_orth_cgs2(OrthArgs a) { orth_body(a, blockIdx.x, gridDim.x); }

// Many blocks at once: CTAs [cta0[p], cta0[p+1]) orthonormalise pencil p's
// block, with a grid barrier of their own (bars + 2 p).
__global__ void __launch_bounds__(ORTH_THREADS)
k_orth_cgs2_grp(double2* Q, const GrpDesc* pd, const int* cta0, int np, double2* part, unsigned* bars,
                const int* active, unsigned* flags, unsigned long long wait_ns) {
  int p = 0;
  while (p + 1 < np && cta0[p + 1] <= (int)blockIdx.x) ++p;
  if (!active[p]) return;  // the whole group leaves together
  const GrpDesc d = pd[p];
  const int G = cta0[p + 1] - cta0[p];
  OrthArgs a;
  a.Q = Q + d.onm;
  a.n = d.n;
  a.m = d.m;
  a.rows_per = (d.n + G - 1) / G;
  a.part = part + (size_t)2 * cta0[p] * ORTH_MAX_M;
  a.bar = bars + 2 * p;
  a.flags = flags;
  a.wait_ns = wait_ns;
  orth_body(a, blockIdx.x - cta0[p], G);
}

// CGS2 with every CTA's rows of Q resident in shared memory (rows_per x (m + 1),
// padded so that a warp reading one row of 32 columns and a warp reading one
// column of 32 rows both meet distinct banks).  Two grid barriers per column:
// pass 1 of column j also carries the partial |q_{j-1}|^2, so that q_{j-1} is
// normalised (and its coefficient rescaled) after the same reduction.  The
// partial sums of a phase sit in part[(phase & 1)][g * (m + 1) + slot].
constexpr int ORTH_SM_BYTES_MAX = 200 * 1024;

// F32DOT: the projection coefficients and norms from a complex64 copy of the
// rows (kept beside the FP64 rows in shared memory), the updates in FP64.  Any
// coefficients keep the span exact when the update is FP64; the basis is then
// orthonormal to about 1e-7 instead of 1e-16, which suits a caller that forms
// and inverts the basis' own Gram matrix in FP64 (the Rayleigh-Ritz step) and
// halves the scalar FP64 work (the slow pipe on this GPU).
template <bool F32DOT>
__global__ void __launch_bounds__(ORTH_THREADS) k_orth_cgs2_sm(OrthArgs a) {
  extern __shared__ double2 sQ[];
  __shared__ double2 s_r[ORTH_MAX_M + 1];
  __shared__ double2 s_red[ORTH_THREADS + ORTH_MAX_M + 1];
  __shared__ int s_ok;
  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
  const int n = a.n, m = a.m, ld = m + 1, S = m + 1;
  const int r0 = min(n, g * a.rows_per), R = min(n, r0 + a.rows_per) - r0;
  float2* sQ32 = reinterpret_cast<float2*>(sQ + (size_t)a.rows_per * ld);  // F32DOT only
  auto set = [&](int rl, int c, double2 v) {
    sQ[rl * ld + c] = v;
    if (F32DOT) sQ32[rl * ld + c] = make_float2((float)v.x, (float)v.y);
  };
  for (int idx = tid; idx < R * m; idx += ORTH_THREADS) {
    const int rl = idx % R, c = idx / R;
    set(rl, c, a.Q[(size_t)c * n + r0 + rl]);
  }
  __syncthreads();
  int phase = 0;
  // s_r[0..ns) = the reduced slots of one phase: slot i < nc the coefficient
  // q_i^H q_j; slot nc (when nc_norm >= 0) the squared norm of column nc_norm.
  auto reduce_phase = [&](int j, int nc, int nc_norm) -> bool {
    const int ns = nc + (nc_norm >= 0 ? 1 : 0);
    const int groups = ns <= ORTH_THREADS ? ORTH_THREADS / ns : 1;
    for (int t = tid; t < ns * groups; t += ORTH_THREADS) {
      const int i = t % ns, gr = t / ns;
      double2 acc = make_double2(0.0, 0.0);
      if (F32DOT) {
        float2 a32 = make_float2(0.f, 0.f);
        if (i < nc) {
#pragma unroll 4
          for (int rl = gr; rl < R; rl += groups) cfmac<float>(a32, sQ32[rl * ld + i], sQ32[rl * ld + j]);
        } else {
          for (int rl = gr; rl < R; rl += groups) a32.x += cnorm2<float>(sQ32[rl * ld + nc_norm]);
        }
        acc = make_double2(a32.x, a32.y);
      } else if (i < nc) {
#pragma unroll 4
        for (int rl = gr; rl < R; rl += groups) cfmac<double>(acc, sQ[rl * ld + i], sQ[rl * ld + j]);
      } else {
        for (int rl = gr; rl < R; rl += groups) acc.x += cnorm2<double>(sQ[rl * ld + nc_norm]);
      }
      s_red[t] = acc;
    }
    __syncthreads();
    double2* part = a.part + (size_t)(phase & 1) * G * S;
    for (int i = tid; i < ns; i += ORTH_THREADS) {
      double2 acc = s_red[i];
      for (int gr = 1; gr < groups; ++gr) acc = cadd<double>(acc, s_red[gr * ns + i]);
      part[(size_t)g * S + i] = acc;
    }
    if (!grid_barrier_spin(a.bar, G, a.flags, &s_ok, a.wait_ns)) return false;
    // CTA g sums the G partials of slots g, g + G, ... (scalar FP64 is the
    // slow pipe here, so no CTA sums every slot): thread t takes partial t,
    // then a fixed tree over the threads, the same in every CTA; a second
    // barrier publishes the sums
    double2* fin = a.fin + (size_t)(phase & 1) * S;
    ++phase;
    for (int i = g; i < ns; i += G) {
      double2 acc = make_double2(0.0, 0.0);
      for (int gg = tid; gg < G; gg += ORTH_THREADS) acc = cadd<double>(acc, __ldcg(part + (size_t)gg * S + i));
      s_red[tid] = acc;
      __syncthreads();
      for (int w = ORTH_THREADS / 2; w > 0; w >>= 1) {
        if (tid < w) s_red[tid] = cadd<double>(s_red[tid], s_red[tid + w]);
        __syncthreads();
      }
      if (tid == 0) fin[i] = s_red[0];
      __syncthreads();
    }
    if (!grid_barrier_spin(a.bar, G, a.flags, &s_ok, a.wait_ns)) return false;
    for (int i = tid; i < ns; i += ORTH_THREADS) s_r[i] = __ldcg(fin + i);
    __syncthreads();
    return true;
  };
  // q_j -= sum_{i<j} q_i s_r[i] on this CTA's rows: warp w takes rows w, w+8, ...,
  // its lanes split the i range, a shuffle sums the lanes
  auto update = [&](int j) {
    const int lane = tid & 31, warp = tid >> 5;
    for (int rl = warp; rl < R; rl += ORTH_THREADS / 32) {
      double2 acc = make_double2(0.0, 0.0);
      for (int i = lane; i < j; i += 32) cfma<double>(acc, sQ[rl * ld + i], s_r[i]);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
      }
      if (lane == 0) set(rl, j, csub<double>(sQ[rl * ld + j], acc));
    }
    __syncthreads();
  };
  auto normalise = [&](int c, double nrm2) {
    const double inv = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
    for (int rl = tid; rl < R; rl += ORTH_THREADS) set(rl, c, cscale<double>(sQ[rl * ld + c], inv));
    return inv;
  };
  // column j: pass 1 carries the squared norm of column j - 1, which is then
  // normalised, or restarted from e_r when the second projection took more
  // than half of what the first left (the column lies in the span of the
  // earlier ones: Kahan's criterion for 'twice is enough'); j = m only
  // takes the norm of the last column.  Every CTA reduces the same partials in
  // the same order, so all take the same branch.
  int retries = 0;
  double r1sq = 0.0;  // |q_{j-1}|^2 after its first projection (0 for column 0)
  for (int j = 1; j <= m;) {
    const int nc = j < m ? j : 0;
    if (!reduce_phase(j, nc, j - 1)) return;
    const double nrm2 = s_r[nc].x;
    if ((!(nrm2 > SAFE_MIN) || nrm2 < 0.5 * r1sq) && retries < ORTH_RETRIES) {
      const int c = j - 1, rr = orth_restart_row(a.col0 + c, retries++, n);
      for (int rl = tid; rl < R; rl += ORTH_THREADS) set(rl, c, make_double2(r0 + rl == rr ? 1.0 : 0.0, 0.0));
      __syncthreads();
      if (c == 0) r1sq = 0.0;
      j = c > 0 ? c : 1;  // project the restarted column again (column 0 needs no projection)
      continue;
    }
    retries = 0;
    const double inv = normalise(j - 1, nrm2);
    if (j == m) break;
    if (tid == 0) s_r[j - 1] = cscale<double>(s_r[j - 1], inv);
    __syncthreads();
    update(j);
    if (!reduce_phase(j, j, j)) return;  // pass 2, with |q_j|^2 after pass 1
    r1sq = s_r[j].x;
    update(j);
    ++j;
  }
  __syncthreads();
  for (int idx = tid; idx < R * m; idx += ORTH_THREADS) {
    const int rl = idx % R, c = idx / R;
    a.Q[(size_t)c * n + r0 + rl] = sQ[rl * ld + c];
  }
}

// ---------------------------------------------------------------- small LU
constexpr int SMALL_THREADS = 1024;

__device__ __forceinline__ void small_lu_body(double2* M, int m, int* piv, unsigned* flags) {
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

__global__ void __launch_bounds__(SMALL_THREADS) k_small_lu(double2* M, int m, int* piv, unsigned* flags) {
  small_lu_body(M, m, piv, flags);
}

__global__ void __launch_bounds__(SMALL_THREADS)
k_small_lu_grp(double2* M, const GrpDesc* pd, const int* active, int* piv, unsigned* flags) {
  const int p = blockIdx.x;
  if (!active[p]) return;
  small_lu_body(M + pd[p].omm, pd[p].m, piv + pd[p].om, flags);
}

// One block per group of SOLVE_COLS right-hand sides (the factors are shared).
constexpr int SOLVE_COLS = 8;

__device__ __forceinline__ void small_lu_solve_body(const double2* LU, const int* piv, int m, double2* X, int nrhs,
                                                    int trans, int bx) {
  const int tid = threadIdx.x;
  X += (size_t)bx * SOLVE_COLS * m;
  nrhs = min(SOLVE_COLS, nrhs - bx * SOLVE_COLS);
  if (nrhs <= 0) return;
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

__global__ void __launch_bounds__(SMALL_THREADS)
k_small_lu_solve(const double2* LU, const int* piv, int m, double2* X, int nrhs, int trans) {
  small_lu_solve_body(LU, piv, m, X, nrhs, trans, blockIdx.x);
}

// Square right-hand side per pencil (nrhs = m); grid (chunks of the largest m, pencils).
__global__ void __launch_bounds__(SMALL_THREADS)
k_small_lu_solve_grp(const double2* LU, const int* piv, const GrpDesc* pd, const int* active, double2* X, int trans) {
  const int p = blockIdx.y;
  if (!active[p]) return;
  const GrpDesc d = pd[p];
  small_lu_solve_body(LU + d.omm, piv + d.om, d.m, X + d.omm, d.m, trans, blockIdx.x);
}

// gate = (max_ij |T_ij - delta_ij| > tol): T = W X checks an approximate inverse X of W.
__global__ void __launch_bounds__(256) k_inv_check(const double2* T, int m, double tol, int* gate) {
  __shared__ double red[8];
  double mx = 0.0;
  for (int idx = threadIdx.x; idx < m * m; idx += 256) {
    double2 v = T[idx];
    if (idx % m == idx / m) v.x -= 1.0;
    const double a = cabs1<double>(v);
    mx = (a > mx || a != a) ? a : mx;  // a NaN entry fails the check too
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double o = __shfl_down_sync(0xffffffffu, mx, off);
    mx = (o > mx || o != o) ? o : mx;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) mx = (red[w] > mx || red[w] != red[w]) ? red[w] : mx;
    *gate = (mx > tol || mx != mx) ? 1 : 0;
  }
}

// When *gate != 0: X = W^{-1} by LU with partial pivoting (LU, piv scratch); else nothing.
__global__ void __launch_bounds__(SMALL_THREADS)
k_small_inv_gated(const double2* W, double2* LU, int* piv, double2* X, int m, unsigned* flags, const int* gate) {
  if (*gate == 0) return;
  for (int idx = threadIdx.x; idx < m * m; idx += SMALL_THREADS) LU[idx] = W[idx];
  __syncthreads();
  small_lu_body(LU, m, piv, flags);
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * m; idx += SMALL_THREADS)
    X[idx] = make_double2((idx % m) == (idx / m) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int bx = 0; bx * SOLVE_COLS < m; ++bx) {
    small_lu_solve_body(LU, piv, m, X, m, 0, bx);
    __syncthreads();
  }
}

// Grouped check: gate[p] = active[p] && max_ij |T_ij - delta_ij| > tol (NaN fails);
// with X non-null, X = 2I - T as well (the first-order inverse of a near-identity T).
__global__ void __launch_bounds__(256)
k_inv_check_grp(const double2* T, const GrpDesc* pd, const int* active, double tol, int* gate, double2* X) {
  __shared__ double red[8];
  const int p = blockIdx.x;
  if (!active[p]) {
    if (threadIdx.x == 0) gate[p] = 0;
    return;
  }
  const GrpDesc d = pd[p];
  const int m = d.m;
  double mx = 0.0;
  for (int idx = threadIdx.x; idx < m * m; idx += 256) {
    const double2 t = T[d.omm + idx];
    double2 v = t;
    const bool diag = idx % m == idx / m;
    if (diag) v.x -= 1.0;
    if (X) X[d.omm + idx] = make_double2((diag ? 2.0 : 0.0) - t.x, -t.y);
    const double a = cabs1<double>(v);
    mx = (a > mx || a != a) ? a : mx;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double o = __shfl_down_sync(0xffffffffu, mx, off);
    mx = (o > mx || o != o) ? o : mx;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) mx = (red[w] > mx || red[w] != red[w]) ? red[w] : mx;
    gate[p] = (mx > tol || mx != mx) ? 1 : 0;
  }
}

// Grouped fallback: X_p = W_p^{-1} by LU with partial pivoting where gate[p] != 0.
__global__ void __launch_bounds__(SMALL_THREADS)
k_small_inv_gated_grp(const double2* W, double2* LU, int* piv, double2* X, const GrpDesc* pd, unsigned* flags,
                      const int* gate) {
  const int p = blockIdx.x;
  if (gate[p] == 0) return;
  const GrpDesc d = pd[p];
  const int m = d.m;
  for (int idx = threadIdx.x; idx < m * m; idx += SMALL_THREADS) LU[d.omm + idx] = W[d.omm + idx];
  __syncthreads();
  small_lu_body(LU + d.omm, m, piv + d.om, flags);
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * m; idx += SMALL_THREADS)
    X[d.omm + idx] = make_double2((idx % m) == (idx / m) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int bx = 0; bx * SOLVE_COLS < m; ++bx) {
    small_lu_solve_body(LU + d.omm, piv + d.om, m, X + d.omm, m, 0, bx);
    __syncthreads();
  }
}

// X ~ M^{-1} (m x m, m <= GJ_MAX_M) by Gauss-Jordan elimination with partial
// pivoting in FP32 on one CTA, the matrix in shared memory (ld m + 1): the
// start of a Newton-Schulz refinement in FP64.  Row k is scaled by 1 / A_kk
// (the pivot position then holds 1 / A_kk), column k is eliminated from every
// other row, and the column interchanges undo the row interchanges in reverse
// order at the end.  A zero pivot leaves a non-finite X, which the following
// check rejects.
constexpr int GJ_THREADS = 1024;
constexpr int GJ_MAX_M = 160;

__global__ void __launch_bounds__(GJ_THREADS) k_gj_inverse32(const double2* M, int m, double2* X) {
  extern __shared__ float2 gjA[];  // [i + j * (m + 1)]
  __shared__ float2 f[GJ_MAX_M];
  __shared__ int s_piv[GJ_MAX_M];
  const int tid = threadIdx.x, ld = m + 1;
  for (int idx = tid; idx < m * m; idx += GJ_THREADS) {
    const int i = idx % m, j = idx / m;
    const double2 v = M[idx];
    gjA[i + j * ld] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    if (tid < 32) {
      float best = -1.f;
      int bi = m;
      for (int i = k + tid; i < m; i += 32) {
        const float v = cabs1<float>(gjA[i + k * ld]);
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float v2 = __shfl_down_sync(0xffffffffu, best, off);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, off);
        if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
      }
      if (tid == 0) s_piv[k] = bi < m ? bi : k;
    }
    __syncthreads();
    const int p = s_piv[k];
    if (p != k)
      for (int j = tid; j < m; j += GJ_THREADS) {
        const float2 a = gjA[k + j * ld];
        gjA[k + j * ld] = gjA[p + j * ld];
        gjA[p + j * ld] = a;
      }
    __syncthreads();
    const float2 rd = crecip<float>(gjA[k + k * ld]);
    for (int i = tid; i < m; i += GJ_THREADS) f[i] = i == k ? make_float2(0.f, 0.f) : gjA[i + k * ld];
    __syncthreads();
    for (int j = tid; j < m; j += GJ_THREADS)
      gjA[k + j * ld] = j == k ? rd : cmul<float>(gjA[k + j * ld], rd);
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += GJ_THREADS) {
      const int i = idx % m, j = idx / m;
      if (i != k) {
        const float2 a = j == k ? make_float2(0.f, 0.f) : gjA[i + j * ld];
        gjA[i + j * ld] = csub<float>(a, cmul<float>(f[i], gjA[k + j * ld]));
      }
    }
    __syncthreads();
  }
  for (int k = m - 1; k >= 0; --k) {
    const int p = s_piv[k];
    if (p != k)
      for (int i = tid; i < m; i += GJ_THREADS) {
        const float2 a = gjA[i + k * ld];
        gjA[i + k * ld] = gjA[i + p * ld];
        gjA[i + p * ld] = a;
      }
    __syncthreads();
  }
  for (int idx = tid; idx < m * m; idx += GJ_THREADS) {
    const int i = idx % m, j = idx / m;
    const float2 v = gjA[i + j * ld];
    X[idx] = make_double2((double)v.x, (double)v.y);
  }
}

}  // namespace

size_t orth_scratch_bytes(int n, int m) {
  return (size_t)2 * 160 * (m + 1) * sizeof(double2) + (size_t)2 * (m + 1) * sizeof(double2) + 256;
}

cudaError_t orth_cgs2(double2* Q, int n, int m, void* scratch, unsigned* flags, cudaStream_t s, int col0,
                      bool f32dots) {
  if (m > ORTH_MAX_M || m < 1 || n < 1) return cudaErrorInvalidValue;
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  OrthArgs a;
  a.Q = Q; a.n = n; a.m = m;
  a.col0 = col0;
  a.bar = reinterpret_cast<unsigned*>(scratch);
  a.part = reinterpret_cast<double2*>(reinterpret_cast<char*>(scratch) + 256);
  a.fin = a.part + (size_t)2 * 160 * (m + 1);
  a.flags = flags;
  a.wait_ns = feast_wait_limit_ns(1000000000ull);
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 256, s);
  if (e != cudaSuccess) return e;
  // shared-memory form: one CTA per SM, each holding its rows of Q
  {
    int G = min(nsm, 160);
    G = min(G, max(1, (n + 7) / 8));
    a.rows_per = (n + G - 1) / G;
    G = (n + a.rows_per - 1) / a.rows_per;
    const size_t smem = (size_t)a.rows_per * (m + 1) * (sizeof(double2) + (f32dots ? sizeof(float2) : 0));
    if (m >= 2 && smem <= (size_t)ORTH_SM_BYTES_MAX) {
      static bool attr = false;
      if (!attr) {
        e = cudaFuncSetAttribute(k_orth_cgs2_sm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 ORTH_SM_BYTES_MAX);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(k_orth_cgs2_sm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   ORTH_SM_BYTES_MAX);
        if (e != cudaSuccess) return e;
        attr = true;
      }
      void* args[] = {&a};
      feast_count_launch();
      void* fn = f32dots ? (void*)k_orth_cgs2_sm<true> : (void*)k_orth_cgs2_sm<false>;
      return cudaLaunchCooperativeKernel(fn, dim3(G), dim3(ORTH_THREADS), args, smem, s);
    }
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_orth_cgs2, ORTH_THREADS, 0);
  int G = min(nsm * max(per, 1), 128);
  G = min(G, max(1, (n + 15) / 16));
  G = min(G, 160);
  a.rows_per = (n + G - 1) / G;
  G = (n + a.rows_per - 1) / a.rows_per;
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
  k_small_lu_solve<<<(nrhs + SOLVE_COLS - 1) / SOLVE_COLS, SMALL_THREADS, 0, s>>>(LU, piv, m, X, nrhs, trans);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- grouped forms
int orth_grp_ctas_per_sm() {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_orth_cgs2_grp, ORTH_THREADS, 0);
  return per;
}

cudaError_t orth_cgs2_grp(double2* Q, const GrpDesc* pd, const int* cta0, int np, int total_ctas, double2* part,
                          unsigned* bars, const int* active, unsigned* flags, cudaStream_t s) {
  if (np < 1) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(bars, 0, sizeof(unsigned) * 2 * np, s);
  if (e != cudaSuccess) return e;
  unsigned long long wait_ns = feast_wait_limit_ns(1000000000ull);
  void* args[] = {&Q, &pd, &cta0, &np, &part, &bars, &active, &flags, &wait_ns};
  feast_count_launch();
  return cudaLaunchCooperativeKernel((void*)k_orth_cgs2_grp, dim3(total_ctas), dim3(ORTH_THREADS), args, 0, s);
}

cudaError_t small_lu_grp(double2* M, const GrpDesc* pd, int np, const int* active, int* piv, unsigned* flags,
                         cudaStream_t s) {
  if (np < 1) return cudaSuccess;
  feast_count_launch();
  k_small_lu_grp<<<np, SMALL_THREADS, 0, s>>>(M, pd, active, piv, flags);
  return cudaGetLastError();
}

cudaError_t small_lu_solve_grp(const double2* LU, const int* piv, const GrpDesc* pd, int np, int mmax,
                               const int* active, double2* X, int trans, cudaStream_t s) {
  if (np < 1) return cudaSuccess;
  feast_count_launch();
  k_small_lu_solve_grp<<<dim3((mmax + SOLVE_COLS - 1) / SOLVE_COLS, np), SMALL_THREADS, 0, s>>>(LU, piv, pd, active,
                                                                                                 X, trans);
  return cudaGetLastError();
}


cudaError_t inverse_check(const double2* T, int m, double tol, int* gate, cudaStream_t s) {
  feast_count_launch();
  k_inv_check<<<1, 256, 0, s>>>(T, m, tol, gate);
  return cudaGetLastError();
}

cudaError_t small_inverse_gated(const double2* W, double2* LU, int* piv, double2* X, int m, unsigned* flags,
                                const int* gate, cudaStream_t s) {
  feast_count_launch();
  k_small_inv_gated<<<1, SMALL_THREADS, 0, s>>>(W, LU, piv, X, m, flags, gate);
  return cudaGetLastError();
}

cudaError_t inverse_check_grp(const double2* T, const GrpDesc* pd, int np, const int* active, double tol, int* gate,
                              double2* X, cudaStream_t s) {
  if (np < 1) return cudaSuccess;
  feast_count_launch();
  k_inv_check_grp<<<np, 256, 0, s>>>(T, pd, active, tol, gate, X);
  return cudaGetLastError();
}

cudaError_t small_inverse_gated_grp(const double2* W, double2* LU, int* piv, double2* X, const GrpDesc* pd, int np,
                                    unsigned* flags, const int* gate, cudaStream_t s) {
  if (np < 1) return cudaSuccess;
  feast_count_launch();
  k_small_inv_gated_grp<<<np, SMALL_THREADS, 0, s>>>(W, LU, piv, X, pd, flags, gate);
  return cudaGetLastError();
}

cudaError_t gj_inverse32(const double2* M, int m, double2* X, cudaStream_t s) {
  if (m < 1 || m > GJ_MAX_M) return cudaErrorInvalidValue;
  const int smem = m * (m + 1) * (int)sizeof(float2);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_gj_inverse32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         GJ_MAX_M * (GJ_MAX_M + 1) * (int)sizeof(float2));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  feast_count_launch();
  k_gj_inverse32<<<1, GJ_THREADS, smem, s>>>(M, m, X);
  return cudaGetLastError();
}
