// FP64-accurate complex products on the BF16 tensor cores by exact integer
// slicing; see ozaki.cuh for the arithmetic.
//
// Kernels:
//   k_oz_rowexp    row exponents of L (one per complex row of op(A))
//   k_oz_split_L   digits of L, 32 x 32 complex tiles transposed through
//                  shared memory into K-contiguous rows
//   k_oz_split_X   column exponents and digits of X (K-contiguous already)
//   k_oz_gemm      P_i = D_i [E_0; ...; E_{s-1-i}] on tcgen05 (TMA 4-stage
//                  ring, FP32 accumulator in TMEM, one 128 x 128 tile per CTA)
//   k_oz_combine   C~ = 2^(e_r + f_c) sum 2^(-(i+j+2) beta) P_ij in FP64
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "ozaki.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace tcx;

constexpr int OZ_BM = 128, OZ_BN = 128, OZ_BK = 64;  // BK: 64 bf16 = one 128-byte swizzle row
constexpr int OZ_STAGES = 4;
constexpr int OZ_A_BYTES = OZ_BM * OZ_BK * 2;  // 16 KB
constexpr int OZ_B_BYTES = OZ_BN * OZ_BK * 2;  // 16 KB
constexpr int OZ_THREADS = 192;                // TMA, MMA, 4 epilogue warps
constexpr int OZ_SMEM = 1024 + OZ_STAGES * (OZ_A_BYTES + OZ_B_BYTES) + 256;
constexpr unsigned OZ_IDESC = bf16_idesc(OZ_BM, OZ_BN);

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------- digits
__device__ __forceinline__ int exponent_of(double mx) {
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);  // mx = f 2^ex, 0.5 <= f < 1, so every |x| <= mx < 2^ex
  return ex;
}

// e[2i] = e[2i+1] = exponent of max |Re|, |Im| over row i of op(A).
// OP_N: a block takes 32 rows, its 8 warps stride over the columns (each warp
// reads 32 consecutive entries of a column), the warps' maxima meet in shared
// memory.  OP_C: row i of A^H is column i of A, one block per column.
__global__ void __launch_bounds__(256) k_oz_rowexp(const double2* A, long long lda, int n, int opA, int* e) {
  __shared__ double red[8][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (opA == OP_N) {
    const int i = blockIdx.x * 32 + lane;
    double mx = 0.0;
    if (i < n)
      for (int j = warp; j < n; j += 8) {
        const double2 v = A[(size_t)i + (size_t)j * lda];
        mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
      }
    red[warp][lane] = mx;
    __syncthreads();
    if (warp == 0 && i < n) {
      for (int w = 1; w < 8; ++w) mx = fmax(mx, red[w][lane]);
      e[2 * i] = e[2 * i + 1] = exponent_of(mx);
    }
  } else {
    const int i = blockIdx.x;
    if (i >= n) return;
    double mx = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double2 v = A[(size_t)j + (size_t)i * lda];
      mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
    if (lane == 0) red[warp][0] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < 8; ++w) mx = fmax(mx, red[w][0]);
      e[2 * i] = e[2 * i + 1] = exponent_of(mx);
    }
  }
}

// |v| 2^(sb - ex) rounded to the nearest integer (halves up), with v's sign, for
// |v| < 2^ex and sb = s beta <= 59: the 53-bit significand of v shifted by
// integer operations (a shift left of at most sb - 53 bits, so |N| <= 2^sb).
__device__ __forceinline__ long long scaled_int(double v, int ex, int sb) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const bool neg = (bits >> 63) != 0;
  int E = (int)((bits >> 52) & 0x7ff);
  unsigned long long mant = bits & ((1ULL << 52) - 1);
  if (E == 0) E = 1;  // subnormal: no hidden bit
  else mant |= 1ULL << 52;
  // |v| = mant 2^(E - 1075)
  const int sh = E - 1075 + sb - ex;
  unsigned long long N;
  if (sh >= 0) N = mant << sh;
  else if (sh < -54) N = 0;
  else N = ((mant >> (-sh - 1)) + 1) >> 1;
  return neg ? -(long long)N : (long long)N;
}

// Digit sl of N = sum_i d_i 2^((s-1-i) beta): d_0 = |N| >> (s-1) beta (at most
// 2^beta), the others beta-bit fields; every digit carries N's sign.
__device__ __forceinline__ float int_digit(long long N, int sl, int s, int beta) {
  const unsigned long long u = N < 0 ? (unsigned long long)(-N) : (unsigned long long)N;
  unsigned long long q = u >> ((s - 1 - sl) * beta);
  if (sl > 0) q &= (1ULL << beta) - 1;
  const float f = (float)q;
  return N < 0 ? -f : f;
}

// Two digits streams at once: t <- t 2^beta, d = rint(t), t <- t - d (all exact in FP64).
__device__ __forceinline__ __nv_bfloat162 next_digits(double& t0, double& t1, int beta) {
  t0 = ldexp(t0, beta);
  t1 = ldexp(t1, beta);
  const double d0 = rint(t0), d1 = rint(t1);
  t0 -= d0;
  t1 -= d1;
  __nv_bfloat162 r;
  r.x = __double2bfloat16(d0);  // |d| <= 2^beta <= 256: exact in bfloat16
  r.y = __double2bfloat16(d1);
  return r;
}

// Digits of L for a 32 x 32 tile of op(A): L rows 2i, 2i+1 and K columns 2j, 2j+1.
__global__ void __launch_bounds__(256)
k_oz_split_L(const double2* A, long long lda, int n, int opA, const int* e, int s, int beta, long long M, int Kp,
             __nv_bfloat16* D) {
  __shared__ double2 tile[32][33];  // [i][j] = op(A)(i0 + i, j0 + j)
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32, tid = threadIdx.x;
  for (int idx = tid; idx < 32 * 32; idx += 256) {
    const int a = idx & 31, b = idx >> 5;
    if (opA == OP_N) {  // a = i (contiguous in A), b = j
      const int i = i0 + a, j = j0 + b;
      tile[a][b] = (i < n && j < n) ? A[(size_t)i + (size_t)j * lda] : make_double2(0.0, 0.0);
    } else {  // op(A)(i, j) = conj(A(j, i)); a = j (contiguous), b = i
      const int j = j0 + a, i = i0 + b;
      double2 v = (i < n && j < n) ? A[(size_t)j + (size_t)i * lda] : make_double2(0.0, 0.0);
      v.y = -v.y;
      tile[b][a] = v;
    }
  }
  __syncthreads();
  // thread -> (L row r in 0..63 of the tile, complex column jj in 0..31)
  for (int idx = tid; idx < 64 * 32; idx += 256) {
    const int jj = idx & 31, r = idx >> 5;
    const int i = i0 + (r >> 1), j = j0 + jj;
    if (i >= n || j >= n) continue;
    const double2 a = tile[r >> 1][jj];
    // row 2i: (Re a, -Im a); row 2i+1: (Im a, Re a)
    double t0 = (r & 1) ? a.y : a.x;
    double t1 = (r & 1) ? a.x : -a.y;
    const long long row = 2LL * i + (r & 1);
    const int ex = e[row];
    // t = sum_i d_i 2^(ex - (i+1) beta) + O(2^(ex - s beta)) by integer digits
    const long long N0 = scaled_int(t0, ex, s * beta), N1 = scaled_int(t1, ex, s * beta);
    for (int sl = 0; sl < s; ++sl) {
      __nv_bfloat162 d;
      d.x = __float2bfloat16_rn(int_digit(N0, sl, s, beta));  // |d| <= 2^beta <= 256: exact
      d.y = __float2bfloat16_rn(int_digit(N1, sl, s, beta));
      reinterpret_cast<__nv_bfloat162*>(D + ((size_t)sl * M + row) * Kp)[j] = d;
    }
  }
}

// Column exponents and digits of X (n x m): row c of E_sl holds (Re, Im) of X[:, c].
__global__ void __launch_bounds__(256)
k_oz_split_X(const double2* X, long long ldx, int n, int m, int s, int beta, int Kp, __nv_bfloat16* E, int* f,
             const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ double red[8];
  __shared__ int s_ex;
  const int c = blockIdx.x;
  const double2* x = X + (size_t)c * ldx;
  double mx = 0.0;
  for (int j = threadIdx.x; j < n; j += 256) mx = fmax(mx, fmax(fabs(x[j].x), fabs(x[j].y)));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) mx = fmax(mx, red[w]);
    s_ex = exponent_of(mx);
    f[c] = s_ex;
  }
  __syncthreads();
  const int ex = s_ex;
  for (int j = threadIdx.x; j < Kp / 2; j += 256) {
    double t0 = 0.0, t1 = 0.0;
    if (j < n) {
      t0 = ldexp(x[j].x, -ex);
      t1 = ldexp(x[j].y, -ex);
    }
    for (int sl = 0; sl < s; ++sl) {
      __nv_bfloat162 d = next_digits(t0, t1, beta);
      reinterpret_cast<__nv_bfloat162*>(E + ((size_t)sl * m + c) * Kp)[j] = d;
    }
  }
}

// ---------------------------------------------------------------- digit products
struct OzGemmArgs {
  float* P;       // s x M x NP
  long long M;
  int m, s, NP, nkb;
  unsigned* flags;
  const int* gate;  // nullable: the product is skipped when *gate == 0
};

// CTA (x, y, z): tile x of the stacked columns of slice z's products, 128-row stripe y.
__global__ void __launch_bounds__(OZ_THREADS, 1)
k_oz_gemm(const __grid_constant__ CUtensorMap mapD, const __grid_constant__ CUtensorMap mapE, OzGemmArgs a) {
  const int i = blockIdx.z;
  const int ncols = (a.s - i) * a.m;  // slice i pairs with E_0 .. E_{s-1-i}
  const int col0 = blockIdx.x * OZ_BN;
  if (col0 >= ncols) return;  // whole CTA, before any barrier or allocation
  if (a.gate && *a.gate == 0) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = smem;
  unsigned char* sB = smem + OZ_STAGES * OZ_A_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OZ_STAGES * (OZ_A_BYTES + OZ_B_BYTES));
  uint64_t* full = bars;                // [OZ_STAGES]
  uint64_t* empty = bars + OZ_STAGES;   // [OZ_STAGES]
  uint64_t* d_full = bars + 2 * OZ_STAGES;
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(bars + 2 * OZ_STAGES + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.y * OZ_BM;

  if (threadIdx.x == 0) {
    for (int st = 0; st < OZ_STAGES; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    mbar_init(d_full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(OZ_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const unsigned tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      for (int kb = 0; kb < a.nkb; ++kb) {
        const int st = kb % OZ_STAGES;
        if (kb >= OZ_STAGES && !mbar_wait(&empty[st], ((kb / OZ_STAGES) - 1) & 1)) {
          atomicOr(a.flags, (unsigned)DEVFLAG_TIMEOUT);
          break;
        }
        mbar_expect_tx(&full[st], OZ_A_BYTES + OZ_B_BYTES);
        tma_load_3d(sA + st * OZ_A_BYTES, &mapD, &full[st], kb * OZ_BK, row0, i);
        tma_load_3d(sB + st * OZ_B_BYTES, &mapE, &full[st], kb * OZ_BK, col0, 0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      int issued = 0;
      for (int kb = 0; kb < a.nkb; ++kb) {
        const int st = kb % OZ_STAGES;
        if (!mbar_wait(&full[st], (kb / OZ_STAGES) & 1)) { ok = false; break; }
        fence_after();
        const unsigned aBase = smem_u32(sA + st * OZ_A_BYTES), bBase = smem_u32(sB + st * OZ_B_BYTES);
        for (int kk = 0; kk < 4; ++kk) {
          mma_bf16_idesc(tmem_base, sw128_desc(aBase + kk * 32), sw128_desc(bBase + kk * 32), OZ_IDESC,
                         (kb > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&empty[st]);
        ++issued;
      }
      if (!ok) atomicOr(a.flags, (unsigned)DEVFLAG_TIMEOUT);
      mma_commit(d_full);  // arrives when every MMA issued above has completed
    }
  } else {
    const int quarter = warp & 3;
    const int r = quarter * 32 + lane;
    const long long row = row0 + r;
    const bool ok = __all_sync(0xffffffffu, mbar_wait(d_full, 0));
    if (!ok) {
      if (lane == 0) atomicOr(a.flags, (unsigned)DEVFLAG_TIMEOUT);
    } else {
      fence_after();
      float* out = a.P + ((size_t)i * a.M + (size_t)(row < a.M ? row : 0)) * a.NP + col0;
      for (int c = 0; c < OZ_BN / 32; ++c) {
        float v[32];
        const unsigned taddr = tmem_base + ((unsigned)(quarter * 32) << 16) + (unsigned)(c * 32);
        tmem_ld16(taddr, *reinterpret_cast<float(*)[16]>(&v[0]));
        tmem_ld16(taddr + 16, *reinterpret_cast<float(*)[16]>(&v[16]));
        if (row < a.M && col0 + c * 32 < a.NP) {
          float4* o = reinterpret_cast<float4*>(out + c * 32);
#pragma unroll
          for (int u = 0; u < 8; ++u) o[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    // d_full was committed after the last issued MMA; wait for it (bounded)
    // before the accumulator is freed, whatever the epilogue saw
    if (lane == 0) mbar_wait(d_full, 0);
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(OZ_BN));
  }
}

// ---------------------------------------------------------------- recombination
// C[i, c] = (C~[2i, c], C~[2i+1, c]); pairs summed from the smallest weight up.
__global__ void k_oz_combine(const float* P, const int* e, const int* f, long long M, int m, int s, int NP, int beta,
                             int n, double2* C, long long ldc, const int* gate) {
  if (gate && *gate == 0) return;
  const size_t total = (size_t)n * m;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % m), i = (int)(idx / m);
    double out[2];
    for (int h = 0; h < 2; ++h) {
      const long long r = 2LL * i + h;
      double acc = 0.0;
      for (int d = 2 * s - 2; d >= 0; --d) {  // d = sl + j, pairs with sl + j <= s - 1 only
        if (d > s - 1) continue;
        double part = 0.0;
        for (int sl = 0; sl <= d; ++sl) {
          const int j = d - sl;
          part += (double)P[((size_t)sl * M + r) * NP + (size_t)j * m + c];
        }
        acc += ldexp(part, -(d + 2) * beta);
      }
      out[h] = ldexp(acc, e[r] + f[c]);
    }
    C[(size_t)i + (size_t)c * ldc] = make_double2(out[0], out[1]);
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}

// Digit rows of Kp bf16 (Kp % 64 == 0, so every row is 128-byte aligned), `rows` rows per
// slice, `slices` slices; boxes of 64 x 128.
bool encode_digits(CUtensorMap* map, void* base, int Kp, long long rows, int slices) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)slices};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2};
  cuuint32_t box[3] = {(cuuint32_t)OZ_BK, 128, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int oz_beta(int K) {
  int cl = 0;
  while ((1LL << cl) < K) ++cl;
  const int b = (24 - cl) / 2;
  return b > 8 ? 8 : (b < 1 ? 1 : b);
}

int oz_slices(int beta) { return (52 + beta - 1) / beta; }

namespace {
void oz_shape(int n, int* M, int* K, int* Kp, int* beta, int* s) {
  *M = 2 * n;
  *K = 2 * n;
  *Kp = (int)round_up((size_t)*K, 64);
  *beta = oz_beta(*K);
  *s = oz_slices(*beta);
}
}  // namespace

size_t oz_operator_bytes(int n) {
  int M, K, Kp, beta, s;
  oz_shape(n, &M, &K, &Kp, &beta, &s);
  return round_up((size_t)s * M * Kp * 2, 256) + round_up((size_t)M * 4, 256);
}

void oz_operator_layout(void* base, int n, OzOperator* L) {
  int M, K, Kp, beta, s;
  oz_shape(n, &M, &K, &Kp, &beta, &s);
  L->n = n; L->M = M; L->K = K; L->Kp = Kp; L->beta = beta; L->s = s;
  L->D = reinterpret_cast<__nv_bfloat16*>(base);
  L->e = reinterpret_cast<int*>(reinterpret_cast<char*>(base) + round_up((size_t)s * M * Kp * 2, 256));
}

static int work_np(int s, int m) { return (int)round_up((size_t)s * m, 32); }

size_t oz_work_bytes(int n, int m) {
  int M, K, Kp, beta, s;
  oz_shape(n, &M, &K, &Kp, &beta, &s);
  return round_up((size_t)s * m * Kp * 2, 256) + round_up((size_t)m * 4, 256) + (size_t)s * M * work_np(s, m) * 4;
}

void oz_work_layout(void* base, int n, int m, OzWork* w) {
  int M, K, Kp, beta, s;
  oz_shape(n, &M, &K, &Kp, &beta, &s);
  char* p = reinterpret_cast<char*>(base);
  w->E = reinterpret_cast<__nv_bfloat16*>(p);
  p += round_up((size_t)s * m * Kp * 2, 256);
  w->f = reinterpret_cast<int*>(p);
  p += round_up((size_t)m * 4, 256);
  w->P = reinterpret_cast<float*>(p);
}

cudaError_t oz_make_operator(const double2* A, long long lda, int opA, OzOperator& L, cudaStream_t s) {
  if (L.Kp > L.K) {  // zero the padding columns K..Kp-1 of every digit row (the rest is written below)
    cudaError_t e = cudaMemset2DAsync(L.D + L.K, (size_t)L.Kp * 2, 0, (size_t)(L.Kp - L.K) * 2, (size_t)L.s * L.M, s);
    if (e != cudaSuccess) return e;
  }
  feast_count_launch();
  if (opA == OP_N)
    k_oz_rowexp<<<(L.n + 31) / 32, 256, 0, s>>>(A, lda, L.n, opA, L.e);
  else
    k_oz_rowexp<<<L.n, 256, 0, s>>>(A, lda, L.n, opA, L.e);
  dim3 grid((L.n + 31) / 32, (L.n + 31) / 32);
  feast_count_launch();
  k_oz_split_L<<<grid, 256, 0, s>>>(A, lda, L.n, opA, L.e, L.s, L.beta, L.M, L.Kp, L.D);
  return cudaGetLastError();
}

cudaError_t oz_apply(const OzOperator& L, const double2* X, long long ldx, int m, double2* C, long long ldc,
                     const OzWork& w, unsigned* flags, cudaStream_t s, const int* gate) {
  if (m < 1) return cudaSuccess;
  const int NP = work_np(L.s, m);
  feast_count_launch();
  k_oz_split_X<<<m, 256, 0, s>>>(X, ldx, L.n, m, L.s, L.beta, L.Kp, w.E, w.f, gate);
  CUtensorMap mD, mE;
  if (!encode_digits(&mD, L.D, L.Kp, L.M, L.s)) return cudaErrorInvalidValue;
  if (!encode_digits(&mE, w.E, L.Kp, (long long)L.s * m, 1)) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  OzGemmArgs a;
  a.P = w.P;
  a.M = L.M;
  a.m = m;
  a.s = L.s;
  a.NP = NP;
  a.nkb = L.Kp / OZ_BK;
  a.flags = flags;
  a.gate = gate;
  dim3 grid((unsigned)((L.s * m + OZ_BN - 1) / OZ_BN), (unsigned)((L.M + OZ_BM - 1) / OZ_BM), (unsigned)L.s);
  feast_count_launch();
  k_oz_gemm<<<grid, OZ_THREADS, OZ_SMEM, s>>>(mD, mE, a);
  const size_t total = (size_t)L.n * m;
  const unsigned blocks = (unsigned)((total + 255) / 256 < 152 * 8 ? (total + 255) / 256 : 152 * 8);
  feast_count_launch();
  k_oz_combine<<<blocks, 256, 0, s>>>(w.P, L.e, w.f, L.M, m, L.s, NP, L.beta, L.n, C, ldc, gate);
  return cudaGetLastError();
}
