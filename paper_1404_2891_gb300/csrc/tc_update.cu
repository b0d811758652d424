// LU trailing update A22 -= L21 U12 on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in TMEM, operands staged by TMA), for all q
// shifted matrices of one panel step.
//
// Arithmetic.  The complex64 matrices are stored interleaved, so a column of
// n complex numbers is a column of 2n floats: rows 2i (Re) and 2i+1 (Im).
// Reading the trailing block C and U12 that way, C~ (2M x N) and U~ (2K x N)
// are real matrices, and with the real 2M x 2K operand A' that expands each
// entry l of L21 into [[Re l, -Im l], [Im l, Re l]],
//        C~ -= A' U~          (4 real products per complex product).
// Each real operand is split into bfloat16 high and low parts
// (x = hi + lo, |lo| <= 2^-9 |x|), and the product is taken as
// hi*hi + hi*lo + lo*hi with FP32 accumulation, about 16 significant bits.
//
// Kernel.  One CTA owns a 128-row stripe of C~ (64 complex rows) of one
// shift and loops over the column tiles (BN = 128; 64 in k_tc_update_c):
//   warp 0   TMA producer: the stripe's A' once, then U~ tiles, two stages
//            (k_tc_update_c: also the C~ tiles, into their own two-stage ring)
//   warp 1   TMEM allocation and the MMA issuer (one thread)
//   warps 2-9 epilogue, two per TMEM lane quarter: TMEM -> registers,
//            C~ -= D with coalesced 128-byte accesses (adjacent lanes hold
//            the Re/Im rows of one complex row)
// Two TMEM accumulator buffers let the MMAs of tile t+1 run while the
// epilogue drains tile t.  Every mbarrier wait is bounded; on timeout the CTA
// raises DEVFLAG_TIMEOUT, drains, frees its TMEM and returns.
//
// Staging kernels: k_stage_operands writes A' and U~ as split BF16;
// k_stage_solve first solves the B block with its diagonal block (and, for
// the LU, applies the panel's interchanges to its columns), writes it back to
// the matrix, then stages it.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "tc_ptx.cuh"
#include "tc_update.cuh"

namespace {

constexpr int TC_BM = 128;      // rows of C~ per stripe (= 64 complex rows)
constexpr int TC_BN = 128;      // columns per tile
constexpr int TC_KP = 128;      // staged K width (2 * nb, nb <= 64), bf16 elements
constexpr int TC_BOX_K = 64;    // 64 bf16 = 128 bytes = one swizzle row
constexpr int TC_THREADS = 320; // 10 warps: TMA, MMA, 8 epilogue (two per TMEM lane quarter)
constexpr int A_BYTES = 2 * 2 * TC_BM * TC_BOX_K * 2;        // hi/lo x 2 k-boxes x 128 rows x 128 B = 64 KB
constexpr int B_STAGE_BYTES = 2 * 2 * TC_BN * TC_BOX_K * 2;  // 64 KB
constexpr int TC_SMEM = 1024 + A_BYTES + 2 * B_STAGE_BYTES + 256;  // 197,888 bytes

using namespace tcx;

// kind::f16 instruction descriptor of this kernel: M = 128, N = TC_BN.
constexpr unsigned IDESC = bf16_idesc(TC_BM, TC_BN);
__device__ __forceinline__ void mma_bf16(unsigned tmem_d, uint64_t adesc, uint64_t bdesc, unsigned accumulate) {
  mma_bf16_idesc(tmem_d, adesc, bdesc, IDESC, accumulate);
}

// ---------------------------------------------------------------- operand staging
// A' stage: [shift][hi,lo][row 0..2*rest)[kk 0..TC_KP) bf16; B stage: [shift][hi,lo][col][kk].
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__device__ __forceinline__ __nv_bfloat162 pair(__nv_bfloat16 a, __nv_bfloat16 b) {
  __nv_bfloat162 r;
  r.x = a;
  r.y = b;
  return r;
}

// One block stages 32 complex rows of L21 (blockIdx.z = 0) or 32 columns of
// U12 (blockIdx.z = 1) of one shift: coalesced loads into a shared tile, then
// coalesced 4-byte (bf16 pair) stores of the staged rows.
constexpr int ST_ROWS = 32;

// Operand description of one batched block product C -= A B (all complex64):
//   A (M x K): opA = OP_N: A(i,k) = SA_b[ar0 + i, ac0 + k];  OP_C: A(i,k) = conj(SA_b[ac0 + k, ar0 + i])
//   B (K x N): B(k,j) = SB_b[br0 + k, bc0 + j]
//   C (M x N): C(i,j) = SC_b[cr0 + i, cc0 + j]
struct TcGemm {
  const float2* SA; long long lda, sa; int ar0, ac0, opA;
  const float2* SB; long long ldb, sb; int br0, bc0;
  float2* SC; long long ldc, sc; int cr0, cc0;
  int M, N, K, q;
};

typedef float2 StageTile[TC_KP / 2 + 1];

// Load the block's 32 rows of A (blockIdx.z = 0) or 32 columns of B (z = 1)
// into tile[row or column][k], zero-padded.
__device__ __forceinline__ void stage_load(const TcGemm& g, StageTile* tile, bool isA, int b, int base) {
  const int tid = threadIdx.x;
  const int rest = isA ? g.M : g.N;
  const int w = g.K;
  if (isA && g.opA == OP_N) {
    const float2* Sb = g.SA + (size_t)b * g.sa;
    const int r = tid & 31;
    for (int k = tid >> 5; k < TC_KP / 2; k += 8) {
      const int i = base + r;
      tile[r][k] = (i < rest && k < w) ? Sb[(size_t)(g.ar0 + i) + (size_t)(g.ac0 + k) * g.lda] : make_float2(0.f, 0.f);
    }
  } else if (isA) {
    const float2* Sb = g.SA + (size_t)b * g.sa;
    const int k = tid & 63;
    for (int c = tid >> 6; c < ST_ROWS; c += 4) {
      const int i = base + c;
      float2 v = (i < rest && k < w) ? Sb[(size_t)(g.ac0 + k) + (size_t)(g.ar0 + i) * g.lda] : make_float2(0.f, 0.f);
      v.y = -v.y;
      tile[c][k] = v;
    }
  } else {
    const float2* Sb = g.SB + (size_t)b * g.sb;
    const int k = tid & 63;
    for (int c = tid >> 6; c < ST_ROWS; c += 4) {
      const int j = base + c;
      tile[c][k] = (j < rest && k < w) ? Sb[(size_t)(g.br0 + k) + (size_t)(g.bc0 + j) * g.ldb] : make_float2(0.f, 0.f);
    }
  }
}

// Write the tile as split-BF16 staging rows.
__device__ __forceinline__ void stage_store(const TcGemm& g, StageTile* tile, bool isA, int b, int base,
                                            __nv_bfloat16* Ast, __nv_bfloat16* Bst, long long rows_max,
                                            long long cols_max) {
  const int tid = threadIdx.x;
  const int rest = isA ? g.M : g.N;
  constexpr int WORDS = TC_KP / 2;  // bf16 pairs per staged row
  if (isA) {
    // per complex row i: A' rows 2i ([Re, -Im] pairs) and 2i+1 ([Im, Re] pairs), hi and lo
    for (int e = tid; e < ST_ROWS * 2 * 2 * WORDS; e += 256) {
      const int k = e % WORDS;
      const int rr = (e / WORDS) % (2 * ST_ROWS);  // A' row within the block
      const int h = e / (WORDS * 2 * ST_ROWS);     // 0 = hi, 1 = lo
      const int i = base + (rr >> 1);
      if (i >= rest) continue;
      const float2 l = tile[rr >> 1][k];
      const float x0 = (rr & 1) ? l.y : l.x;
      const float x1 = (rr & 1) ? l.x : -l.y;
      __nv_bfloat16 h0, l0, h1, l1;
      split_bf16(x0, h0, l0);
      split_bf16(x1, h1, l1);
      __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(
          Ast + (((size_t)b * 2 + h) * rows_max + 2 * (size_t)base + rr) * TC_KP);
      dst[k] = h ? pair(l0, l1) : pair(h0, h1);
    }
  } else {
    for (int e = tid; e < ST_ROWS * 2 * WORDS; e += 256) {
      const int k = e % WORDS;
      const int c = (e / WORDS) % ST_ROWS;
      const int h = e / (WORDS * ST_ROWS);
      const int j = base + c;
      if (j >= rest) continue;
      const float2 u = tile[c][k];
      __nv_bfloat16 hr, lr, him, lim;
      split_bf16(u.x, hr, lr);
      split_bf16(u.y, him, lim);
      __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(Bst + (((size_t)b * 2 + h) * cols_max + (size_t)j) * TC_KP);
      dst[k] = h ? pair(lr, lim) : pair(hr, him);
    }
  }
}

__global__ void __launch_bounds__(256)
k_stage_operands(TcGemm g, __nv_bfloat16* Ast, __nv_bfloat16* Bst, long long rows_max, long long cols_max) {
  __shared__ StageTile tile[ST_ROWS];  // [row or column][k]
  const int b = blockIdx.y;
  const int base = blockIdx.x * ST_ROWS;
  const bool isA = blockIdx.z == 0;
  stage_load(g, tile, isA, b, base);
  __syncthreads();
  stage_store(g, tile, isA, b, base, Ast, Bst, rows_max, cols_max);
}

// The staging of one block step of a triangular solve, with the step's
// diagonal solve folded into the B part: B = X[k0 : k0 + w, :] (k0 = br0,
// w = K) is first solved with the w x w diagonal block of the same shift
// (mode: 0 L_kk unit lower, 1 U_kk, 2 U_kk^H, 3 L_kk^H unit upper), written
// back to X, and then staged.  Each warp solves four of the block's 32 columns
// on its own (lanes hold rows lane and lane + 32, pivots broadcast by
// shuffles), so the 64 substitution steps need no block barrier.  D is kept in
// shared memory with the entries a step reads (one column of the triangle)
// contiguous: as stored for modes 0 and 1, transposed for 2 and 3.
__global__ void __launch_bounds__(256)
k_stage_solve(TcGemm g, __nv_bfloat16* Ast, __nv_bfloat16* Bst, long long rows_max, long long cols_max, int mode,
              const int32_t* mv) {
  __shared__ StageTile tile[ST_ROWS];
  __shared__ int s_d[128], s_s[128], s_cnt;
  extern __shared__ __align__(16) unsigned char stage_smem[];
  float2* D = reinterpret_cast<float2*>(stage_smem);  // [s * 64 + r]: the entry that step s applies to row r
  float2* rinv = D + 64 * 64;
  const int b = blockIdx.y, tid = threadIdx.x;
  const int base = blockIdx.x * ST_ROWS;
  const bool isA = blockIdx.z == 0;
  if (!isA && base >= g.N) return;  // no columns of X here (uniform per block)
  if (!isA && mv) {
    // the panel's interchanges on this block's 32 columns of the trailing
    // matrix: moved rows {dst, src} relative to br0, all read (through D's
    // space) before any is written
    const int32_t* m = mv + (size_t)b * LU_MV_STRIDE;
    if (tid == 0) s_cnt = min(max(m[0], 0), 128);
    for (int e = tid; e < 128; e += 256) {
      s_d[e] = m[1 + e];
      s_s[e] = m[129 + e];
    }
    __syncthreads();
    const int cnt = s_cnt;
    float2* Xb = const_cast<float2*>(g.SB) + (size_t)b * g.sb;
    for (int idx = tid; idx < cnt * ST_ROWS; idx += 256) {
      const int e = idx >> 5, j = base + (idx & 31);
      if (j < g.N) D[idx] = Xb[(size_t)(g.br0 + s_s[e]) + (size_t)(g.bc0 + j) * g.ldb];
    }
    __syncthreads();
    for (int idx = tid; idx < cnt * ST_ROWS; idx += 256) {
      const int e = idx >> 5, j = base + (idx & 31);
      if (j < g.N) Xb[(size_t)(g.br0 + s_d[e]) + (size_t)(g.bc0 + j) * g.ldb] = D[idx];
    }
    __syncthreads();
  }
  stage_load(g, tile, isA, b, base);
  if (!isA) {
    const int w = g.K, k0 = g.br0;
    const float2* Sd = g.SA + (size_t)b * g.sa;
    const bool transposed = mode >= 2;
    for (int idx = tid; idx < w * w; idx += 256) {
      const int r = idx % w, s2 = idx / w;
      const float2 v = Sd[(size_t)(k0 + r) + (size_t)(k0 + s2) * g.lda];  // S[k0 + r, k0 + s2]
      if (transposed)
        D[r * 64 + s2] = cconj<float>(v);  // step r, row s2: conj(S[k0 + r, k0 + s2])
      else
        D[s2 * 64 + r] = v;  // step s2, row r
    }
    __syncthreads();
    if (mode == 1 || mode == 2)
      for (int s2 = tid; s2 < w; s2 += 256) rinv[s2] = crecip<float>(D[s2 * 64 + s2]);
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    float2 x[4][2];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      x[j][0] = tile[4 * warp + j][lane];
      x[j][1] = tile[4 * warp + j][lane + 32];
    }
    const bool fwd = mode == 0 || mode == 2, divide = mode == 1 || mode == 2;
    for (int it = 0; it < w; ++it) {
      const int s2 = fwd ? it : w - 1 - it;
      const int owner = s2 & 31, hs = s2 >> 5;
      const float2 d0 = D[s2 * 64 + lane], d1 = D[s2 * 64 + lane + 32];
      const float2 ri = divide ? rinv[s2] : make_float2(1.f, 0.f);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 v = hs ? x[j][1] : x[j][0];
        float2 xs = make_float2(__shfl_sync(0xffffffffu, v.x, owner), __shfl_sync(0xffffffffu, v.y, owner));
        if (divide) xs = cmul<float>(xs, ri);
        if (lane == owner) {
          if (hs) x[j][1] = xs; else x[j][0] = xs;
        }
        const bool a0 = fwd ? lane > s2 : lane < s2;
        const bool a1 = fwd ? lane + 32 > s2 : lane + 32 < s2;
        if (a0 && lane < w) x[j][0] = csub<float>(x[j][0], cmul<float>(d0, xs));
        if (a1 && lane + 32 < w) x[j][1] = csub<float>(x[j][1], cmul<float>(d1, xs));
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      tile[4 * warp + j][lane] = x[j][0];
      tile[4 * warp + j][lane + 32] = x[j][1];
    }
    __syncthreads();
    // the solved rows back to X
    float2* Xb = const_cast<float2*>(g.SB) + (size_t)b * g.sb;
    const int k = tid & 63;
    for (int c = tid >> 6; c < ST_ROWS; c += 4) {
      const int j = base + c;
      if (j < g.N && k < w) Xb[(size_t)(g.br0 + k) + (size_t)(g.bc0 + j) * g.ldb] = tile[c][k];
    }
  }
  __syncthreads();
  stage_store(g, tile, isA, b, base, Ast, Bst, rows_max, cols_max);
}

// ---------------------------------------------------------------- the GEMM
struct TcArgs {
  float* S;            // q output matrices, complex64 interleaved, as floats
  long long ld2;       // 2 * ld (floats per column)
  long long stride2;   // 2 * stride (floats per matrix)
  long long c_off;     // float offset of C~ (its first Re row, first column) inside a matrix
  int M, N;            // complex rows and columns of the C block
  int b_col0;          // first staged B row (column of the B operand) used by this launch
  int kbox;            // number of 64-wide K boxes actually staged (1 or 2)
  unsigned* flags;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
k_tc_update(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = smem;                     // [hi k0, hi k1, lo k0, lo k1] x 16 KB
  unsigned char* sB = smem + A_BYTES;           // 2 stages x [hi k0, hi k1, lo k0, lo k1] x 16 KB
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + A_BYTES + 2 * B_STAGE_BYTES);
  uint64_t* a_full = bars + 0;
  uint64_t* b_full = bars + 1;   // [2]
  uint64_t* b_empty = bars + 3;  // [2]
  uint64_t* d_full = bars + 5;   // [2]
  uint64_t* d_empty = bars + 7;  // [2]
  uint64_t* mma_done = bars + 9;
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(bars + 10);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int stripe = blockIdx.x, shift = blockIdx.y;
  const int ntiles = (a.N + TC_BN - 1) / TC_BN;
  const int row0 = stripe * TC_BM;  // first row of C~ in this stripe

  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
      mbar_init(&d_full[s], 1);
      mbar_init(&d_empty[s], 8);
    }
    mbar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * TC_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const unsigned tmem_base = *tmem_slot;
  const unsigned a_bytes = (unsigned)(2 * a.kbox * TC_BM * TC_BOX_K * 2);
  const unsigned b_bytes = (unsigned)(2 * a.kbox * TC_BN * TC_BOX_K * 2);

  if (warp == 0) {
    if (lane == 0) {
      // A' stripe once
      mbar_expect_tx(a_full, a_bytes);
      for (int h = 0; h < 2; ++h)
        for (int kb = 0; kb < a.kbox; ++kb)
          tma_load_3d(sA + (h * 2 + kb) * (TC_BM * 128), &mapA, a_full, kb * TC_BOX_K, row0, shift * 2 + h);
      int last[2] = {-1, -1};
      for (int t = 0; t < ntiles; ++t) {
        const int s = t & 1;
        if (t >= 2 && !mbar_wait(&b_empty[s], ((t >> 1) - 1) & 1)) {
          atomicOr(a.flags, (unsigned)DEVFLAG_TIMEOUT);
          break;
        }
        mbar_expect_tx(&b_full[s], b_bytes);
        unsigned char* dst = sB + s * B_STAGE_BYTES;
        for (int h = 0; h < 2; ++h)
          for (int kb = 0; kb < a.kbox; ++kb)
            tma_load_3d(dst + (h * 2 + kb) * (TC_BN * 128), &mapB, &b_full[s], kb * TC_BOX_K, a.b_col0 + t * TC_BN,
                        shift * 2 + h);
        last[s] = t;
      }
      // no copy may still be writing shared memory when the block exits
      mbar_wait(a_full, 0);
      for (int s = 0; s < 2; ++s)
        if (last[s] >= 0) mbar_wait(&b_full[s], (last[s] >> 1) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = mbar_wait(a_full, 0);
      fence_after();
      bool issued = false;
      for (int t = 0; ok && t < ntiles; ++t) {
        const int s = t & 1;
        if (!mbar_wait(&b_full[s], (t >> 1) & 1)) { ok = false; break; }
        if (t >= 2 && !mbar_wait(&d_empty[s], ((t >> 1) - 1) & 1)) { ok = false; break; }
        fence_after();
        const unsigned d = tmem_base + (unsigned)(s * TC_BN);
        const unsigned aBase = smem_u32(sA), bBase = smem_u32(sB + s * B_STAGE_BYTES);
        unsigned acc = 0;
        // hi*hi, hi*lo, lo*hi
        for (int term = 0; term < 3; ++term) {
          const int ha = term == 2 ? 1 : 0, hb = term == 1 ? 1 : 0;
          for (int kk = 0; kk < a.kbox * 4; ++kk) {
            const int kb = kk >> 2, ko = (kk & 3) * 32;
            const uint64_t ad = sw128_desc(aBase + (ha * 2 + kb) * (TC_BM * 128) + ko);
            const uint64_t bd = sw128_desc(bBase + (hb * 2 + kb) * (TC_BN * 128) + ko);
            mma_bf16(d, ad, bd, acc);
            acc = 1;
          }
        }
        mma_commit(&b_empty[s]);
        mma_commit(&d_full[s]);
        issued = true;
      }
      if (!ok) atomicOr(a.flags, (unsigned)DEVFLAG_TIMEOUT);
      if (issued) {  // every MMA of this block has completed before TMEM is freed
        mma_commit(mma_done);
        mbar_wait(mma_done, 0);
      }
    }
  } else {
    // epilogue warps 2..5: TMEM lane quarter (warp % 4)
    const int quarter = warp & 3;        // the TMEM lane quarter this warp may read
    const int half = (warp - 2) >> 2;    // which of the tile's 32-column chunks it takes
    const int r = quarter * 32 + lane;  // row within the stripe
    const long long R = row0 + r;       // row of C~
    float* Cb = a.S + (size_t)shift * a.stride2 + a.c_off;
    const bool row_ok = R < 2LL * a.M;
    for (int t = 0; t < ntiles; ++t) {
      const int s = t & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&d_full[s], (t >> 1) & 1));  // warp-uniform
      if (!ok) {
        if (lane == 0) atomicOr(a.flags, (unsigned)DEVFLAG_TIMEOUT);
        break;
      }
      fence_after();
      const int col0 = t * TC_BN;
      for (int c = half; c < TC_BN / 32; c += 2) {
        float cv[32], v[32];
        const int cbase = col0 + c * 32;
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int col = cbase + u;
          cv[u] = (row_ok && col < a.N) ? __ldcs(Cb + R + (size_t)col * a.ld2) : 0.f;
        }
        const unsigned taddr = tmem_base + ((unsigned)(quarter * 32) << 16) + (unsigned)(s * TC_BN + c * 32);
        tmem_ld16(taddr, *reinterpret_cast<float(*)[16]>(&v[0]));
        tmem_ld16(taddr + 16, *reinterpret_cast<float(*)[16]>(&v[16]));
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int col = cbase + u;
          if (row_ok && col < a.N) __stcs(Cb + R + (size_t)col * a.ld2, cv[u] - v[u]);
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&d_empty[s]);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(2 * TC_BN));
  }
}

// The same update with C streamed by TMA: a 64-column variant in which warp 0
// also loads each 128 x 64 tile of C~ into a two-stage shared-memory ring as
// soon as the ring has room (independently of the MMAs), so that the HBM reads
// of C are in flight in bulk while the previous tile is written back; the
// epilogue reads C from shared memory (conflict-free: lane r reads row r).
// Used when the C block's first float row is 16-byte aligned and the column
// stride is a multiple of 16 bytes.
constexpr int TCC_BN = 64;
constexpr int TCC_B_STAGE = 2 * 2 * TCC_BN * TC_BOX_K * 2;      // 32 KB
constexpr int TCC_C_STAGE = TC_BM * TCC_BN * 4;                 // 32 KB
constexpr int TCC_SMEM = 1024 + A_BYTES + 2 * TCC_B_STAGE + 2 * TCC_C_STAGE + 256;
constexpr unsigned IDESC_C = bf16_idesc(TC_BM, TCC_BN);

struct TcCArgs {
  int c_row0;   // float row of the C block's first Re row (multiple of 4)
  int c_col0;   // matrix column of the C block's first column
};

__global__ void __launch_bounds__(TC_THREADS, 1)
k_tc_update_c(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const __grid_constant__ CUtensorMap mapC, TcArgs a, TcCArgs cc) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = smem;                                 // [hi k0, hi k1, lo k0, lo k1] x 16 KB
  unsigned char* sB = smem + A_BYTES;                       // 2 stages x [hi k0, hi k1, lo k0, lo k1] x 8 KB
  float* sC = reinterpret_cast<float*>(smem + A_BYTES + 2 * TCC_B_STAGE);  // 2 stages x [64 cols][128 rows]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + A_BYTES + 2 * TCC_B_STAGE + 2 * TCC_C_STAGE);
  uint64_t* a_full = bars + 0;
  uint64_t* b_full = bars + 1;   // [2]
  uint64_t* b_empty = bars + 3;  // [2]
  uint64_t* d_full = bars + 5;   // [2]
  uint64_t* d_empty = bars + 7;  // [2]
  uint64_t* c_full = bars + 9;   // [2]
  uint64_t* c_empty = bars + 11; // [2]
  uint64_t* mma_done = bars + 13;
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(bars + 14);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int stripe = blockIdx.x, shift = blockIdx.y;
  const int ntiles = (a.N + TCC_BN - 1) / TCC_BN;
  const int row0 = stripe * TC_BM;

  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
      mbar_init(&d_full[s], 1);
      mbar_init(&d_empty[s], 8);
      mbar_init(&c_full[s], 1);
      mbar_init(&c_empty[s], 8);
    }
    mbar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * TCC_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const unsigned tmem_base = *tmem_slot;
  const unsigned a_bytes = (unsigned)(2 * a.kbox * TC_BM * TC_BOX_K * 2);
  const unsigned b_bytes = (unsigned)(2 * a.kbox * TCC_BN * TC_BOX_K * 2);

  if (warp == 0) {
    if (lane == 0) {
      mbar_expect_tx(a_full, a_bytes);
      for (int h = 0; h < 2; ++h)
        for (int kb = 0; kb < a.kbox; ++kb)
          tma_load_3d(sA + (h * 2 + kb) * (TC_BM * 128), &mapA, a_full, kb * TC_BOX_K, row0, shift * 2 + h);
      int lastb[2] = {-1, -1}, lastc[2] = {-1, -1};
      bool ok = true;
      for (int t = 0; t < ntiles && ok; ++t) {
        const int s = t & 1;
        if (t >= 2 && !mbar_wait(&c_empty[s], ((t >> 1) - 1) & 1)) { ok = false; break; }
        mbar_expect_tx(&c_full[s], TCC_C_STAGE);
        tma_load_3d(sC + s * (TC_BM * TCC_BN), &mapC, &c_full[s], cc.c_row0 + row0, cc.c_col0 + t * TCC_BN, shift);
        lastc[s] = t;
        if (t >= 2 && !mbar_wait(&b_empty[s], ((t >> 1) - 1) & 1)) { ok = false; break; }
        mbar_expect_tx(&b_full[s], b_bytes);
        unsigned char* dst = sB + s * TCC_B_STAGE;
        for (int h = 0; h < 2; ++h)
          for (int kb = 0; kb < a.kbox; ++kb)
            tma_load_3d(dst + (h * 2 + kb) * (TCC_BN * 128), &mapB, &b_full[s], kb * TC_BOX_K, a.b_col0 + t * TCC_BN,
                        shift * 2 + h);
        lastb[s] = t;
      }
      if (!ok) atomicOr(a.flags, (unsigned)DEVFLAG_TIMEOUT);
      // no copy may still be writing shared memory when the block exits
      mbar_wait(a_full, 0);
      for (int s = 0; s < 2; ++s) {
        if (lastb[s] >= 0) mbar_wait(&b_full[s], (lastb[s] >> 1) & 1);
        if (lastc[s] >= 0) mbar_wait(&c_full[s], (lastc[s] >> 1) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = mbar_wait(a_full, 0);
      fence_after();
      bool issued = false;
      for (int t = 0; ok && t < ntiles; ++t) {
        const int s = t & 1;
        if (!mbar_wait(&b_full[s], (t >> 1) & 1)) { ok = false; break; }
        if (t >= 2 && !mbar_wait(&d_empty[s], ((t >> 1) - 1) & 1)) { ok = false; break; }
        fence_after();
        const unsigned d = tmem_base + (unsigned)(s * TCC_BN);
        const unsigned aBase = smem_u32(sA), bBase = smem_u32(sB + s * TCC_B_STAGE);
        unsigned acc = 0;
        for (int term = 0; term < 3; ++term) {  // hi*hi, hi*lo, lo*hi
          const int ha = term == 2 ? 1 : 0, hb = term == 1 ? 1 : 0;
          for (int kk = 0; kk < a.kbox * 4; ++kk) {
            const int kb = kk >> 2, ko = (kk & 3) * 32;
            const uint64_t ad = sw128_desc(aBase + (ha * 2 + kb) * (TC_BM * 128) + ko);
            const uint64_t bd = sw128_desc(bBase + (hb * 2 + kb) * (TCC_BN * 128) + ko);
            mma_bf16_idesc(d, ad, bd, IDESC_C, acc);
            acc = 1;
          }
        }
        mma_commit(&b_empty[s]);
        mma_commit(&d_full[s]);
        issued = true;
      }
      if (!ok) atomicOr(a.flags, (unsigned)DEVFLAG_TIMEOUT);
      if (issued) {  // every MMA of this block has completed before TMEM is freed
        mma_commit(mma_done);
        mbar_wait(mma_done, 0);
      }
    }
  } else {
    const int quarter = warp & 3;      // TMEM lane quarter of this warp
    const int c = (warp - 2) >> 2;     // the tile's 32-column chunk it takes
    const int r = quarter * 32 + lane; // row within the stripe
    const long long R = row0 + r;
    float* Cb = a.S + (size_t)shift * a.stride2 + a.c_off;
    const bool row_ok = R < 2LL * a.M;
    for (int t = 0; t < ntiles; ++t) {
      const int s = t & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&c_full[s], (t >> 1) & 1) && mbar_wait(&d_full[s], (t >> 1) & 1));
      if (!ok) {
        if (lane == 0) atomicOr(a.flags, (unsigned)DEVFLAG_TIMEOUT);
        break;
      }
      fence_after();
      const float* tile = sC + s * (TC_BM * TCC_BN);
      const int cbase = t * TCC_BN + c * 32;
      float cv[32], v[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) cv[u] = tile[(c * 32 + u) * TC_BM + r];
      const unsigned taddr = tmem_base + ((unsigned)(quarter * 32) << 16) + (unsigned)(s * TCC_BN + c * 32);
      tmem_ld16(taddr, *reinterpret_cast<float(*)[16]>(&v[0]));
      tmem_ld16(taddr + 16, *reinterpret_cast<float(*)[16]>(&v[16]));
      fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&d_empty[s]);
        mbar_arrive(&c_empty[s]);
      }
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        const int col = cbase + u;
        if (row_ok && col < a.N) __stcs(Cb + R + (size_t)col * a.ld2, cv[u] - v[u]);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(2 * TCC_BN));
  }
}

// ---------------------------------------------------------------- host side
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
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

bool encode_stage_map(CUtensorMap* m, void* base, long long rows, long long rows_max, int q2, int box_rows) {
  EncodeFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)TC_KP, (cuuint64_t)rows, (cuuint64_t)q2};
  cuuint64_t strides[2] = {(cuuint64_t)TC_KP * 2, (cuuint64_t)rows_max * TC_KP * 2};
  cuuint32_t box[3] = {(cuuint32_t)TC_BOX_K, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C -= A B for all q shifts on the tensor cores (K <= 64); false if the staging
// cannot hold the operands (the caller then uses the FP32 GEMM).
bool tc_gemm_fits(const TcGemm& g, const TcStaging* ctx) {
  return ctx && ctx->Ast && g.K >= 1 && g.K <= TC_KP / 2 && 2LL * g.M <= ctx->rows_max && g.N <= ctx->cols_max &&
         g.q <= ctx->q;
}

// Stage the operands of g (all of A and all N columns of B) as split-BF16.
cudaError_t tc_stage(const TcGemm& g, const TcStaging* ctx, cudaStream_t s) {
  const int blocks = (int)ceil_div((size_t)(g.M > g.N ? g.M : g.N), ST_ROWS);
  dim3 grid(blocks, g.q, 2);
  feast_count_launch();
  k_stage_operands<<<grid, 256, 0, s>>>(g, reinterpret_cast<__nv_bfloat16*>(ctx->Ast),
                                        reinterpret_cast<__nv_bfloat16*>(ctx->Bst), ctx->rows_max, ctx->cols_max);
  return cudaGetLastError();
}

// C[:, c0 : c0 + nc] -= A B[:, c0 : c0 + nc] from the staged operands of g.
cudaError_t tc_run(const TcGemm& g, int c0, int nc, const TcStaging* ctx, unsigned* flags, cudaStream_t s) {
  if (g.M <= 0 || nc <= 0) return cudaSuccess;
  CUtensorMap mA, mB;
  if (!encode_stage_map(&mA, ctx->Ast, 2LL * g.M, ctx->rows_max, 2 * g.q, TC_BM)) return cudaErrorInvalidValue;
  if (!encode_stage_map(&mB, ctx->Bst, g.N, ctx->cols_max, 2 * g.q, TC_BN)) return cudaErrorInvalidValue;
  TcArgs a;
  a.S = reinterpret_cast<float*>(g.SC);
  a.ld2 = 2 * g.ldc;
  a.stride2 = 2 * g.sc;
  a.c_off = 2LL * g.cr0 + (long long)(g.cc0 + c0) * a.ld2;
  a.M = g.M;
  a.N = nc;
  a.b_col0 = c0;
  a.kbox = (2 * g.K + TC_BOX_K - 1) / TC_BOX_K;
  a.flags = flags;
  dim3 grid(ceil_div(2 * (size_t)g.M, TC_BM), g.q);
  // C streamed by TMA when its rows start on a 16-byte boundary and the
  // column and matrix strides are multiples of 16 bytes
  const long long c_row0 = 2LL * g.cr0;
  if (c_row0 % 4 == 0 && (2 * g.ldc) % 4 == 0 && (2 * g.sc) % 4 == 0) {
    CUtensorMap mBc, mC;
    EncodeFn enc = get_encode();
    if (enc && encode_stage_map(&mBc, ctx->Bst, g.N, ctx->cols_max, 2 * g.q, TCC_BN)) {
      cuuint64_t dims[3] = {(cuuint64_t)(c_row0 + 2LL * g.M), (cuuint64_t)(g.cc0 + c0 + nc), (cuuint64_t)g.q};
      cuuint64_t strides[2] = {(cuuint64_t)(2 * g.ldc) * 4, (cuuint64_t)(2 * g.sc) * 4};
      cuuint32_t box[3] = {(cuuint32_t)TC_BM, (cuuint32_t)TCC_BN, 1};
      cuuint32_t estr[3] = {1, 1, 1};
      if (enc(&mC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, g.SC, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
          CUDA_SUCCESS) {
        static bool attr_c = false;
        if (!attr_c) {
          cudaError_t e = cudaFuncSetAttribute(k_tc_update_c, cudaFuncAttributeMaxDynamicSharedMemorySize, TCC_SMEM);
          if (e != cudaSuccess) return e;
          attr_c = true;
        }
        TcCArgs cc;
        cc.c_row0 = (int)c_row0;
        cc.c_col0 = g.cc0 + c0;
        feast_count_launch();
        k_tc_update_c<<<grid, TC_THREADS, TCC_SMEM, s>>>(mA, mBc, mC, a, cc);
        return cudaGetLastError();
      }
    }
  }
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_update, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  feast_count_launch();
  k_tc_update<<<grid, TC_THREADS, TC_SMEM, s>>>(mA, mB, a);
  return cudaGetLastError();
}

cudaError_t tc_gemm(const TcGemm& g, const TcStaging* ctx, unsigned* flags, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  cudaError_t e = tc_stage(g, ctx, s);
  if (e != cudaSuccess) return e;
  return tc_run(g, 0, g.N, ctx, flags, s);
}

// Stage g's operands with the B block first solved by its diagonal block (k_stage_solve).
cudaError_t launch_stage_solve(const TcGemm& g, const TcStaging* ctx, int mode, cudaStream_t s,
                               const int32_t* mv = nullptr) {
  constexpr int smem = (64 * 64 + 64) * (int)sizeof(float2);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_stage_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int blocks = (int)ceil_div((size_t)(g.M > g.N ? g.M : g.N), ST_ROWS);
  feast_count_launch();
  k_stage_solve<<<dim3(blocks, g.q, 2), 256, smem, s>>>(g, reinterpret_cast<__nv_bfloat16*>(ctx->Ast),
                                                        reinterpret_cast<__nv_bfloat16*>(ctx->Bst), ctx->rows_max,
                                                        ctx->cols_max, mode, mv);
  return cudaGetLastError();
}

// LU trailing update of step (k0, w): C = S[k0+w:, k0+w:], A = L21 = S[k0+w:, k0:k0+w],
// B = U12 = S[k0:k0+w, k0+w:]; this call updates the columns c0 .. c0+nc-1 of S
// (staging the whole step's operands when `stage`).
cudaError_t tc_trailing_update(const LuBatch<float>& lu, int k0, int w, int c0, int nc, bool stage, void* vctx,
                               cudaStream_t s) {
  const int rest = lu.n - k0 - w;
  if (rest <= 0) return cudaSuccess;
  const TcStaging* ctx = reinterpret_cast<const TcStaging*>(vctx);
  TcGemm g;
  const float2* S = reinterpret_cast<const float2*>(lu.S);
  g.SA = S; g.lda = lu.ld; g.sa = lu.stride; g.ar0 = k0 + w; g.ac0 = k0; g.opA = OP_N;
  g.SB = S; g.ldb = lu.ld; g.sb = lu.stride; g.br0 = k0; g.bc0 = k0 + w;
  g.SC = reinterpret_cast<float2*>(lu.S); g.ldc = lu.ld; g.sc = lu.stride; g.cr0 = k0 + w; g.cc0 = k0 + w;
  // the columns this step sees: all of the trailing matrix, or (two-level LU)
  // those of the current outer block
  const int cend = lu.col_end > 0 ? lu.col_end : lu.n;
  g.M = rest; g.N = cend - (k0 + w); g.K = w; g.q = lu.q;
  if (g.N <= 0) return cudaSuccess;
  if (!tc_gemm_fits(g, ctx)) {
    // the plain update needs U12 solved already, which this path leaves to the staging
    if (lu.u12_in_stage) return cudaErrorInvalidValue;
    return default_trailing_update<float>(lu, k0, w, c0, nc, stage, nullptr, s);
  }
  if (stage) {
    cudaError_t e;
    if (lu.u12_in_stage) {
      // the panel's interchanges on the trailing columns and U12 = L11^{-1} A12
      // (unit lower L11 of this panel), both in the staging kernel's B part,
      // written back to the factor, then staged
      e = launch_stage_solve(g, ctx, 0, s, lu.mv + (size_t)(k0 / 64) * lu.q * LU_MV_STRIDE);
    } else {
      e = tc_stage(g, ctx, s);
    }
    if (e != cudaSuccess) return e;
  }
  if (nc <= 0) return cudaSuccess;  // a staging-only call
  return tc_run(g, c0 - (k0 + w), nc, ctx, lu.flags, s);
}

}  // namespace

size_t tc_staging_bytes_A(long long n, int q) { return (size_t)q * 2 * (2 * (size_t)n) * TC_KP * sizeof(__nv_bfloat16); }
size_t tc_staging_bytes_B(long long n, int q) { return (size_t)q * 2 * (size_t)n * TC_KP * sizeof(__nv_bfloat16); }

template <>
void select_trailing_update<double>(TrailingUpdateFn<double>* fn, void** ctx, TcStaging*) {
  *fn = nullptr;  // complex128: the DMMA batched GEMM (mma.sync f64)
  *ctx = nullptr;
}

template <>
void select_trailing_update<float>(TrailingUpdateFn<float>* fn, void** ctx, TcStaging* staging) {
  *fn = tc_trailing_update;
  *ctx = staging;
}

bool tc_solve_update(const LuBatch<float>& lu, float2* X, int m, int M, int K, int ar0, int ac0, int opA,
                     int row_out, int row_in, int diag_mode, cudaStream_t s, cudaError_t* err) {
  const TcStaging* ctx = reinterpret_cast<const TcStaging*>(lu.tc);
  TcGemm g;
  const float2* S = reinterpret_cast<const float2*>(lu.S);
  const long long n = lu.n, sx = (long long)lu.n * m;
  g.SA = S; g.lda = lu.ld; g.sa = lu.stride; g.ar0 = ar0; g.ac0 = ac0; g.opA = opA;
  g.SB = X; g.ldb = n; g.sb = sx; g.br0 = row_in; g.bc0 = 0;
  g.SC = X; g.ldc = n; g.sc = sx; g.cr0 = row_out; g.cc0 = 0;
  g.M = M; g.N = m; g.K = K; g.q = lu.q;
  if (!tc_gemm_fits(g, ctx)) return false;
  if (diag_mode < 0) {
    *err = tc_gemm(g, ctx, lu.flags, s);
    return true;
  }
  if (M <= 0 || m <= 0) return false;
  cudaError_t e = launch_stage_solve(g, ctx, diag_mode, s);
  *err = e != cudaSuccess ? e : tc_run(g, 0, g.N, ctx, lu.flags, s);
  return true;
}
