// Deep-K trailing update of the two-level LU on the 5th-generation tensor
// cores: C -= L U for all q shifted matrices, K up to 256 complex columns.
//
// Why deep K.  A trailing update with K complex columns reads and writes the
// complex64 block C once (16 B per entry) and does 8 K flops per entry, so its
// arithmetic intensity is K / 2 flop/B: 32 at K = 64, where the update is bound
// by HBM (about 215 TFLOP/s at the measured copy rate), and 128 at K = 256,
// where it is bound by the tensor pipe.  The two-level LU therefore applies the
// far part of the trailing matrix once per 256 columns (this kernel) and only
// the current 256-column block once per 64-column panel.
//
// Arithmetic (as in the K = 64 kernel): complex64 entries stored interleaved,
// so C is a real matrix C~ of 2M rows; L is expanded to the real A' (2M x 2K)
// whose entry l becomes [[Re l, -Im l], [Im l, Re l]], U to U~ (2K x N) with
// each column's [Re, Im] pairs; C~ -= A' U~ is 4 real products per complex one.
// Every real operand is split into bfloat16 hi + lo, and the product is taken
// as hi*hi + hi*lo + lo*hi with FP32 accumulation in TMEM.
//
// Kernel.  Persistent: one CTA per SM takes tiles t = blockIdx.x, + gridDim.x,
// ... of 128 real rows x 256 columns, tiles ordered shift, column stripe,
// row stripe, so that the CTAs running at once share one shift's operands in
// L2.  Warp roles:
//   warp 0    TMA producer: for each tile, the K range in 64-element blocks
//             (A' hi, lo: 128 x 64; U~ hi, lo: 256 x 64; 128-byte swizzle)
//             into a two-stage ring
//   warp 1    TMEM allocation (512 columns: two 256-column accumulators) and
//             the MMA issuer (one thread; M = 128, N = 256, K = 16 per MMA,
//             12 MMAs per 64-element block)
//   warps 2-9 epilogue, two per TMEM lane quarter (each half of the columns):
//             TMEM -> registers, C~ -= D with coalesced 128-byte accesses,
//             while the MMAs of the next tile fill the other accumulator.
// Every mbarrier wait is bounded; on timeout the CTA raises DEVFLAG_TIMEOUT,
// waits for its own copies and MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "tc_deep.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace tcx;

constexpr int DK_BM = 128;
constexpr int DK_BK = 64;                     // bf16 elements per K block (one 128-byte row)
constexpr int DK_A_HALF = DK_BM * 128;        // one of hi / lo: 16 KB
constexpr int DK_THREADS = 320;
// Tile width BN: 256 columns, or 128 for products with at most 128 columns
// (the blocked solves' right-hand sides), which would leave half of a 256-wide
// tile's MMAs and operand loads on padding.
template <int BN>
struct DeepTile {
  static constexpr int B_HALF = BN * 128;                      // 32 KB (BN = 256) / 16 KB
  static constexpr int STAGE = 2 * DK_A_HALF + 2 * B_HALF;     // 96 KB / 64 KB
  static constexpr int SMEM = 1024 + 2 * STAGE + 256;          // 197,888 / 132,352 bytes
  static constexpr unsigned IDESC = bf16_idesc(DK_BM, BN);
};

struct DeepArgs {
  float* S;            // complex64 matrices as floats
  long long ld2;       // floats per column
  long long stride2;   // floats per matrix
  long long c_off;     // float offset of C~ (first Re row, first column) in a matrix
  int M2;              // real rows of C~ (2M)
  int N;               // columns of this launch
  int b_col0;          // first staged U~ row (column of U) of this launch
  int nkb;             // K blocks of 64 bf16
  int row_tiles, col_tiles, q;
  int overwrite;       // C = -D (C not read)
  unsigned* flags;
};

template <int BN>
__global__ void __launch_bounds__(DK_THREADS, 1)
k_tc_deep(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, DeepArgs a) {
  constexpr int DK_BN = BN;
  constexpr int DK_B_HALF = DeepTile<BN>::B_HALF;
  constexpr int DK_STAGE = DeepTile<BN>::STAGE;
  constexpr unsigned DK_IDESC = DeepTile<BN>::IDESC;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * DK_STAGE);
  uint64_t* full = bars + 0;    // [2]
  uint64_t* empty = bars + 2;   // [2]
  uint64_t* tfull = bars + 4;   // [2]
  uint64_t* tempty = bars + 6;  // [2]
  uint64_t* mma_done = bars + 8;
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(bars + 9);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = a.q * a.col_tiles * a.row_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&tfull[s], 1);
      mbar_init(&tempty[s], 8);
    }
    mbar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * DK_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const unsigned tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      long long it = 0;
      int last[2] = {-1, -1};  // parity of the last fill of each stage, -1 = never filled
      bool ok = true;
      for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
        const int rt = t % a.row_tiles, ct = (t / a.row_tiles) % a.col_tiles, shift = t / (a.row_tiles * a.col_tiles);
        for (int kb = 0; kb < a.nkb; ++kb, ++it) {
          const int s = (int)(it & 1);
          if (it >= 2 && !mbar_wait(&empty[s], (unsigned)(((it >> 1) - 1) & 1))) { ok = false; break; }
          unsigned char* st = smem + s * DK_STAGE;
          mbar_expect_tx(&full[s], DK_STAGE);
          for (int h = 0; h < 2; ++h) {
            tma_load_3d(st + h * DK_A_HALF, &mapA, &full[s], kb * DK_BK, rt * DK_BM, shift * 2 + h);
            tma_load_3d(st + 2 * DK_A_HALF + h * DK_B_HALF, &mapB, &full[s], kb * DK_BK, a.b_col0 + ct * DK_BN,
                        shift * 2 + h);
          }
          last[s] = (int)((it >> 1) & 1);
        }
      }
      if (!ok) atomicOr(a.flags, (unsigned)DEVFLAG_TIMEOUT);
      // no copy may still be writing shared memory when the block exits
      for (int s = 0; s < 2; ++s)
        if (last[s] >= 0) mbar_wait(&full[s], (unsigned)last[s]);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long it = 0;
      int tc = 0;
      bool ok = true, issued = false;
      for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++tc) {
        const int b = tc & 1;
        if (tc >= 2 && !mbar_wait(&tempty[b], (unsigned)(((tc >> 1) - 1) & 1))) { ok = false; break; }
        fence_after();
        const unsigned d = tmem_base + (unsigned)(b * DK_BN);
        unsigned acc = 0;
        for (int kb = 0; kb < a.nkb; ++kb, ++it) {
          const int s = (int)(it & 1);
          if (!mbar_wait(&full[s], (unsigned)((it >> 1) & 1))) { ok = false; break; }
          fence_after();
          const unsigned base = smem_u32(smem + s * DK_STAGE);
          for (int term = 0; term < 3; ++term) {  // hi*hi, hi*lo, lo*hi
            const int ha = term == 2 ? 1 : 0, hb = term == 1 ? 1 : 0;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ad = sw128_desc(base + ha * DK_A_HALF + kk * 32);
              const uint64_t bd = sw128_desc(base + 2 * DK_A_HALF + hb * DK_B_HALF + kk * 32);
              mma_bf16_idesc(d, ad, bd, DK_IDESC, acc);
              acc = 1;
            }
          }
          mma_commit(&empty[s]);
          issued = true;
        }
        if (!ok) break;
        mma_commit(&tfull[b]);
      }
      if (!ok) atomicOr(a.flags, (unsigned)DEVFLAG_TIMEOUT);
      if (issued) {  // every MMA of this block has completed before TMEM is freed
        mma_commit(mma_done);
        mbar_wait(mma_done, 0);
      }
    }
  } else {
    const int quarter = warp & 3;        // TMEM lane quarter of this warp
    const int half = (warp - 2) >> 2;    // which 128 of the tile's 256 columns
    const int r = quarter * 32 + lane;   // row within the tile
    int tc = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tc) {
      const int b = tc & 1;
      const int rt = t % a.row_tiles, ct = (t / a.row_tiles) % a.col_tiles, shift = t / (a.row_tiles * a.col_tiles);
      const long long R = (long long)rt * DK_BM + r;
      const bool row_ok = R < a.M2;
      float* Cb = a.S + (size_t)shift * a.stride2 + a.c_off;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull[b], (unsigned)((tc >> 1) & 1)));
      if (!ok) {
        if (lane == 0) atomicOr(a.flags, (unsigned)DEVFLAG_TIMEOUT);
        break;
      }
      fence_after();
      for (int c = 0; c < DK_BN / 64; ++c) {
        const int cl = half * (DK_BN / 2) + c * 32;    // column within the tile
        const int cbase = ct * DK_BN + cl;             // column within this launch
        float cv[32], v[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int col = cbase + u;
          cv[u] = (row_ok && col < a.N && !a.overwrite) ? __ldcs(Cb + R + (size_t)col * a.ld2) : 0.f;
        }
        const unsigned taddr = tmem_base + ((unsigned)(quarter * 32) << 16) + (unsigned)(b * DK_BN + cl);
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
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(2 * DK_BN));
  }
}

// ---------------------------------------------------------------- staging
__device__ __forceinline__ void split2(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}
__device__ __forceinline__ __nv_bfloat162 bpair(__nv_bfloat16 a, __nv_bfloat16 b) {
  __nv_bfloat162 r;
  r.x = a;
  r.y = b;
  return r;
}

// blockIdx.z = 0: 32 rows of L x 32 complex K per block (blockIdx.x: row
// group, blockIdx.y: K group), read down the columns (coalesced), transposed
// through shared memory, written as two A' rows per complex row (one bf16
// pair per complex K).  blockIdx.z = 1: U, one column per warp-row of the block,
// read and written along K (both coalesced, no transpose).
__global__ void __launch_bounds__(256) k_deep_stage(DeepGemm g, __nv_bfloat16* Ast, __nv_bfloat16* Bst,
                                                     long long rows_max, long long cols_max, int part0) {
  const int tid = threadIdx.x;
  const int shift = blockIdx.y / ((g.K + 31) / 32);
  const int kg = blockIdx.y % ((g.K + 31) / 32);
  const float2* Lb = g.L + (size_t)shift * g.strl;
  const float2* Ub = g.U + (size_t)shift * g.stru;
  if (part0 + (int)blockIdx.z == 0) {
    __shared__ float2 tile[32][33];
    const int i0 = blockIdx.x * 32;
    if (i0 >= g.M) return;
    for (int e = tid; e < 32 * 32; e += 256) {
      // the index that runs along the stored columns varies fastest (coalesced):
      // i for L itself, k for a block of L^H
      const bool ct = g.opL == OP_C;
      const int i = ct ? (e >> 5) : (e & 31), k = ct ? (e & 31) : (e >> 5);
      const int gi = i0 + i, gk = kg * 32 + k;
      float2 v = make_float2(0.f, 0.f);
      if (gi < g.M && gk < g.K)
        v = ct ? cconj<float>(Lb[(size_t)(g.lc + gk) + (size_t)(g.lr + gi) * g.ldl])
               : Lb[(size_t)(g.lr + gi) + (size_t)(g.lc + gk) * g.ldl];
      tile[k][i] = v;
    }
    __syncthreads();
    // per complex row i: A' rows 2i ([Re, -Im] pairs) and 2i+1 ([Im, Re]), hi and lo
    for (int e = tid; e < 32 * 2 * 2 * 32; e += 256) {
      const int k = e & 31;
      const int rr = (e >> 5) & 63;   // A' row within the block
      const int h = e >> 11;          // 0 hi, 1 lo
      const int gi = i0 + (rr >> 1);
      if (gi >= g.M) continue;
      const float2 l = tile[k][rr >> 1];
      const float x0 = (rr & 1) ? l.y : l.x;
      const float x1 = (rr & 1) ? l.x : -l.y;
      __nv_bfloat16 h0, l0, h1, l1;
      split2(x0, h0, l0);
      split2(x1, h1, l1);
      __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(
          Ast + (((size_t)shift * 2 + h) * rows_max + 2 * (size_t)i0 + rr) * DEEP_KP);
      dst[kg * 32 + k] = h ? bpair(l0, l1) : bpair(h0, h1);
    }
  } else {
    const int j0 = blockIdx.x * 32;
    if (j0 >= g.N) return;
    for (int e = tid; e < 32 * 32; e += 256) {
      const int k = e & 31, j = e >> 5;
      const int gj = j0 + j, gk = kg * 32 + k;
      if (gj >= g.N) continue;
      const float2 u = gk < g.K ? Ub[(size_t)(g.ur + gk) + (size_t)(g.uc + gj) * g.ldu] : make_float2(0.f, 0.f);
      __nv_bfloat16 hr, lr, him, lim;
      split2(u.x, hr, lr);
      split2(u.y, him, lim);
      __nv_bfloat162* d0 = reinterpret_cast<__nv_bfloat162*>(Bst + (((size_t)shift * 2 + 0) * cols_max + gj) * DEEP_KP);
      __nv_bfloat162* d1 = reinterpret_cast<__nv_bfloat162*>(Bst + (((size_t)shift * 2 + 1) * cols_max + gj) * DEEP_KP);
      d0[gk] = bpair(hr, him);
      d1[gk] = bpair(lr, lim);
    }
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
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

// [2q][rows][DEEP_KP] bf16, box 64 x box_rows, 128-byte swizzle
bool encode_deep_map(CUtensorMap* m, void* base, long long rows, long long rows_max, int q2, int box_rows) {
  EncodeFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)DEEP_KP, (cuuint64_t)rows, (cuuint64_t)q2};
  cuuint64_t strides[2] = {(cuuint64_t)DEEP_KP * 2, (cuuint64_t)rows_max * DEEP_KP * 2};
  cuuint32_t box[3] = {(cuuint32_t)DK_BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n < 1) n = 1;
  }
  return n;
}

}  // namespace

size_t deep_staging_bytes_A(long long n, int q) { return (size_t)q * 2 * (2 * (size_t)n) * DEEP_KP * 2; }
size_t deep_staging_bytes_B(long long n, int q) { return (size_t)q * 2 * (size_t)n * DEEP_KP * 2; }

bool deep_fits(const DeepGemm& g, const DeepStaging& st) {
  return st.Ast && st.Bst && g.K >= 1 && 2 * g.K <= DEEP_KP && 2LL * g.M <= st.rows_max && g.N <= st.cols_max &&
         g.q <= st.q;
}

cudaError_t deep_stage(const DeepGemm& g, const DeepStaging& st, cudaStream_t s, int parts) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (!deep_fits(g, st) || parts < 1 || parts > 3) return cudaErrorInvalidValue;
  const int part0 = parts == 2 ? 1 : 0, nparts = parts == 3 ? 2 : 1;
  const long long span = parts == 1 ? g.M : parts == 2 ? g.N : (g.M > g.N ? g.M : g.N);
  const int groups = (int)ceil_div((size_t)span, 32);
  dim3 grid(groups, g.q * ((g.K + 31) / 32), nparts);
  feast_count_launch();
  k_deep_stage<<<grid, 256, 0, s>>>(g, reinterpret_cast<__nv_bfloat16*>(st.Ast), reinterpret_cast<__nv_bfloat16*>(st.Bst),
                                   st.rows_max, st.cols_max, part0);
  return cudaGetLastError();
}

cudaError_t deep_run(const DeepGemm& g, int c0, int nc, const DeepStaging& st, unsigned* flags, cudaStream_t s) {
  if (g.M <= 0 || nc <= 0) return cudaSuccess;
  if (!deep_fits(g, st) || c0 < 0 || c0 + nc > g.N) return cudaErrorInvalidValue;
  const int BN = nc <= 128 ? 128 : 256;
  CUtensorMap mA, mB;
  if (!encode_deep_map(&mA, st.Ast, 2LL * g.M, st.rows_max, 2 * g.q, DK_BM)) return cudaErrorInvalidValue;
  if (!encode_deep_map(&mB, st.Bst, g.N, st.cols_max, 2 * g.q, BN)) return cudaErrorInvalidValue;
  DeepArgs a;
  a.S = reinterpret_cast<float*>(g.C);
  a.ld2 = 2 * g.ldc;
  a.stride2 = 2 * g.strc;
  a.c_off = 2LL * g.cr + (long long)(g.cc + c0) * a.ld2;
  a.M2 = 2 * g.M;
  a.N = nc;
  a.b_col0 = c0;
  a.nkb = (2 * g.K + DK_BK - 1) / DK_BK;
  a.row_tiles = (int)ceil_div((size_t)a.M2, DK_BM);
  a.col_tiles = (int)ceil_div((size_t)nc, BN);
  a.q = g.q;
  a.overwrite = g.overwrite ? 1 : 0;
  a.flags = flags;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_deep<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         DeepTile<256>::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tc_deep<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, DeepTile<128>::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long tiles = (long long)a.q * a.row_tiles * a.col_tiles;
  const int grid = (int)(tiles < sm_count() ? tiles : sm_count());
  feast_count_launch();
  if (BN == 128)
    k_tc_deep<128><<<grid, DK_THREADS, DeepTile<128>::SMEM, s>>>(mA, mB, a);
  else
    k_tc_deep<256><<<grid, DK_THREADS, DeepTile<256>::SMEM, s>>>(mA, mB, a);
  return cudaGetLastError();
}

namespace {
DeepGemm deep_of(const LuBatch<float>& lu, int K0, int KB) {
  DeepGemm g;
  float2* S = reinterpret_cast<float2*>(lu.S);
  g.C = S; g.ldc = lu.ld; g.strc = lu.stride; g.cr = K0 + KB; g.cc = K0 + KB;
  g.L = S; g.ldl = lu.ld; g.strl = lu.stride; g.lr = K0 + KB; g.lc = K0; g.opL = OP_N;
  g.U = S; g.ldu = lu.ld; g.stru = lu.stride; g.ur = K0; g.uc = K0 + KB;
  g.M = lu.n - K0 - KB;
  g.N = g.M;
  g.K = KB;
  g.q = lu.q;
  return g;
}
}  // namespace

cudaError_t tc_deep_stage(const LuBatch<float>& lu, int K0, int KB, const DeepStaging& st, cudaStream_t s) {
  const DeepGemm g = deep_of(lu, K0, KB);
  if (g.M <= 0) return cudaSuccess;
  return deep_stage(g, st, s, 3);
}

cudaError_t tc_deep_run(const LuBatch<float>& lu, int K0, int KB, const DeepStaging& st, cudaStream_t s) {
  const DeepGemm g = deep_of(lu, K0, KB);
  if (g.M <= 0) return cudaSuccess;
  return deep_run(g, 0, g.N, st, lu.flags, s);
}

cudaError_t tc_far_gemm(const LuBatch<float>& lu, int K0, int KB, const float2* T, const DeepStaging& st,
                        cudaStream_t s) {
  DeepGemm g;
  float2* S = reinterpret_cast<float2*>(lu.S);
  // C and U: the block's rows of the columns beyond it (U staged before the product)
  g.C = S; g.ldc = lu.ld; g.strc = lu.stride; g.cr = K0; g.cc = K0 + KB;
  g.U = S; g.ldu = lu.ld; g.stru = lu.stride; g.ur = K0; g.uc = K0 + KB;
  g.L = T; g.ldl = KB; g.strl = (long long)KB * KB; g.lr = 0; g.lc = 0; g.opL = OP_N;
  g.M = KB;
  g.N = lu.n - K0 - KB;
  g.K = KB;
  g.q = lu.q;
  g.overwrite = true;
  if (g.N <= 0) return cudaSuccess;
  cudaError_t e = deep_stage(g, st, s, 3);
  if (e != cudaSuccess) return e;
  return deep_run(g, 0, g.N, st, lu.flags, s);
}

namespace {
// The products of the blocked solves of one side, in order: for each diagonal
// block I of the sweep, X_I = -T_I X_I (T_I = -D_I^{-1}, overwrite) and then
// the rest of the sweep's rows -= op(S block) X_I.  f(L, ldl, strl, lr, lc,
// M, K, rowC, rowU, overwrite) per product with M, K > 0.
template <typename F>
cudaError_t walk_solve(const LuBatch<float>& lu, int side, int KB, const float2* TL, const float2* TU, F f) {
  const int n = lu.n, q = lu.q, nB = (n + KB - 1) / KB;
  const float2* S = reinterpret_cast<const float2*>(lu.S);
  const long long tstr = (long long)KB * KB;
  auto Tof = [&](const float2* T, int I) { return T ? T + (size_t)I * q * KB * KB : T; };
  const float2* Tfwd = side == 0 ? TL : TU;  // forward sweep: L (right) or U^H (left)
  const float2* Tbwd = side == 0 ? TU : TL;  // backward sweep: U (right) or L^H (left)
  cudaError_t e;
  for (int I = 0; I < nB; ++I) {
    const int r0 = KB * I, nr = std::min(KB, n - r0);
    if ((e = f(Tof(Tfwd, I), (long long)KB, tstr, 0, 0, nr, nr, r0, r0, true)) != cudaSuccess) return e;
    // rows below: right L[r0+nr:, r0:r0+nr]; left (U[r0:r0+nr, r0+nr:])^H
    if (n - r0 - nr > 0 && (e = f(S, lu.ld, lu.stride, r0 + nr, r0, n - r0 - nr, nr, r0 + nr, r0, false)) != cudaSuccess)
      return e;
  }
  for (int I = nB - 1; I >= 0; --I) {
    const int r0 = KB * I, nr = std::min(KB, n - r0);
    if ((e = f(Tof(Tbwd, I), (long long)KB, tstr, 0, 0, nr, nr, r0, r0, true)) != cudaSuccess) return e;
    // rows above: right U[0:r0, r0:r0+nr]; left (L[r0:r0+nr, 0:r0])^H
    if (r0 > 0 && (e = f(S, lu.ld, lu.stride, 0, r0, r0, nr, 0, r0, false)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// bf16 elements of one product's staged factor operand: q x (hi, lo) x 2M x DEEP_KP
size_t prestage_elems(int q, int M) { return (size_t)q * 2 * (2 * (size_t)M) * DEEP_KP; }
}  // namespace

size_t tc_solve_prestage_bytes(long long n, int q, int KB) {
  LuBatch<float> lu;
  lu.n = (int)n;
  lu.q = q;
  size_t elems = 0;
  walk_solve(lu, 0, KB, nullptr, nullptr,
             [&](const float2*, long long, long long, int, int, int M, int, int, int, bool) -> cudaError_t {
               elems += prestage_elems(q, M);
               return cudaSuccess;
             });
  return elems * 2;
}

cudaError_t tc_solve_prestage(const LuBatch<float>& lu, int side, int KB, const float2* TL, const float2* TU,
                              void* pre, cudaStream_t s) {
  if (!pre || KB % 64 || KB > 256) return cudaErrorInvalidValue;
  const int op = side == 0 ? OP_N : OP_C;
  __nv_bfloat16* base = reinterpret_cast<__nv_bfloat16*>(pre);
  size_t off = 0;
  return walk_solve(lu, side, KB, TL, TU,
                    [&](const float2* L, long long ldl, long long strl, int lr, int lc, int M, int K, int, int,
                        bool) -> cudaError_t {
                      DeepGemm g;
                      g.L = L; g.ldl = ldl; g.strl = strl; g.lr = lr; g.lc = lc; g.opL = op;
                      g.M = M; g.N = 1; g.K = K; g.q = lu.q;
                      DeepStaging sa;
                      sa.Ast = base + off;
                      sa.Bst = base;  // not written (A part only)
                      sa.rows_max = 2LL * M;
                      sa.cols_max = 1;
                      sa.q = lu.q;
                      off += prestage_elems(lu.q, M);
                      return deep_stage(g, sa, s, 1);
                    });
}

cudaError_t tc_solve_deep(const LuBatch<float>& lu, int side, float2* X, int m, int KB, const float2* TL,
                          const float2* TU, const DeepStaging& st, cudaStream_t s, const void* pre) {
  if (m < 1 || m > st.cols_max || KB % 64 || KB > 256) return cudaErrorInvalidValue;
  const long long n = lu.n, xs = n * m;
  const int op = side == 0 ? OP_N : OP_C;
  const __nv_bfloat16* base = reinterpret_cast<const __nv_bfloat16*>(pre);
  size_t off = 0;
  return walk_solve(lu, side, KB, TL, TU,
                    [&](const float2* L, long long ldl, long long strl, int lr, int lc, int M, int K, int rowC,
                        int rowU, bool overwrite) -> cudaError_t {
                      DeepGemm g;
                      g.C = X; g.ldc = n; g.strc = xs; g.cr = rowC; g.cc = 0;
                      g.L = L; g.ldl = ldl; g.strl = strl; g.lr = lr; g.lc = lc; g.opL = op;
                      g.U = X; g.ldu = n; g.stru = xs; g.ur = rowU; g.uc = 0;
                      g.M = M; g.N = m; g.K = K; g.q = lu.q;
                      g.overwrite = overwrite;
                      if (!base) {
                        cudaError_t e = deep_stage(g, st, s, 3);
                        if (e != cudaSuccess) return e;
                        return deep_run(g, 0, m, st, lu.flags, s);
                      }
                      // the factor operand was staged after the factorisation: stage X_I only
                      DeepStaging sa = st;
                      sa.Ast = const_cast<__nv_bfloat16*>(base + off);
                      sa.rows_max = 2LL * M;
                      off += prestage_elems(lu.q, M);
                      cudaError_t e = deep_stage(g, sa, s, 2);
                      if (e != cudaSuccess) return e;
                      return deep_run(g, 0, m, sa, lu.flags, s);
                    });
}

double tc_deep_flops(long long n, int q, int K0, int KB) {
  const double r = (double)(n - K0 - KB);
  return r > 0 ? 8.0 * q * r * r * KB : 0.0;
}

double tc_deep_bytes(long long n, int q, int K0, int KB) {
  const double r = (double)(n - K0 - KB);
  return r > 0 ? 8.0 * q * (2.0 * r * r + 2.0 * r * KB) : 0.0;
}
