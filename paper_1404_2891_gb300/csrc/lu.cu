// Batched right-looking blocked LU with partial pivoting (P S = L U) for the
// q shifted matrices phi_k B - A, each factored once and reused for every
// right-hand side and iteration (Sec. 5.5 of the paper), and the blocked
// triangular solves of Eq. Rasp (S X = R) and Eq. Lasp (S^H X = R).
//
// Per panel of width w:  (1) panel factorisation, one CTA per shift, pivot =
// largest |Re|+|Im| with the lowest row on ties; (2) the panel's interchanges
// applied to the other columns and U12 = L11^{-1} A12; (3) the trailing update
// A22 -= L21 U12 as one batched contraction over all shifts.
//
// Schedule (complex64 with the tensor-core update): the next block column is
// updated first and its panel factored on a high-priority side stream beside
// the rest of the update (look-ahead); the panel leaves a list of its moved
// rows, from which the interchanges on the finished L columns run on a third,
// low-priority stream, while those on the trailing columns and the U12 solve
// are done by the update's staging kernel before it stages U12.
#include "lu.cuh"

#include <type_traits>

#include "panel_ll.cuh"
#include "tc_update.cuh"

namespace {

constexpr int PANEL_THREADS = 512;
constexpr int MAX_NB = 128;

template <typename T>
__device__ __forceinline__ void argmax_merge(T& v, int& i, T v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

template <typename T>
__global__ void __launch_bounds__(PANEL_THREADS)
k_panel(cplx<T>* S, long long ld, long long stride, int n, int k0, int w, int32_t* piv, int* info,
        unsigned* flags) {
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  cplx<T>* A = S + (size_t)b * stride;
  int32_t* pv = piv + (size_t)b * n;
  __shared__ T red_v[PANEL_THREADS / 32];
  __shared__ int red_i[PANEL_THREADS / 32];
  __shared__ int s_p;
  __shared__ cplx<T> s_u[MAX_NB];
  const int jend = k0 + w;
  for (int col = k0; col < jend; ++col) {
    // 1. pivot search over rows col .. n-1 (ascending per thread, strict > keeps the lowest)
    T best = T(-1);
    int bi = n;
    for (int i = col + tid; i < n; i += PANEL_THREADS) {
      T v = cabs1<T>(A[(size_t)i + (size_t)col * ld]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      T v2 = __shfl_down_sync(0xffffffffu, best, off);
      int i2 = __shfl_down_sync(0xffffffffu, bi, off);
      argmax_merge<T>(best, bi, v2, i2);
    }
    if (lane == 0) { red_v[wid] = best; red_i[wid] = bi; }
    __syncthreads();
    if (tid == 0) {
      T v = red_v[0];
      int ii = red_i[0];
      for (int k = 1; k < PANEL_THREADS / 32; ++k) argmax_merge<T>(v, ii, red_v[k], red_i[k]);
      if (ii >= n) {  // the column held only NaN: keep the diagonal, flag it
        ii = col;
        atomicOr(flags, (unsigned)DEVFLAG_NONFINITE);
      }
      pv[col] = ii;
      s_p = ii;
    }
    __syncthreads();
    const int p = s_p;
    // 2. interchange rows col and p inside the panel
    if (p != col) {
      for (int j = k0 + tid; j < jend; j += PANEL_THREADS) {
        cplx<T> t1 = A[(size_t)col + (size_t)j * ld];
        A[(size_t)col + (size_t)j * ld] = A[(size_t)p + (size_t)j * ld];
        A[(size_t)p + (size_t)j * ld] = t1;
      }
    }
    __syncthreads();
    // 3. scale the column below the pivot
    const cplx<T> d = A[(size_t)col + (size_t)col * ld];
    const bool zero = (d.x == T(0) && d.y == T(0));
    if (zero && tid == 0) {
      atomicCAS(&info[b], 0, col + 1);
      atomicOr(flags, (unsigned)DEVFLAG_SINGULAR);
    }
    for (int j = col + 1 + tid; j < jend; j += PANEL_THREADS) s_u[j - k0] = A[(size_t)col + (size_t)j * ld];
    __syncthreads();
    // 4. scale the column below the pivot and apply the rank-1 update to the rest
    // of the panel in one pass; each row segment is read in chunks of 8 independent
    // loads before any store, so the L2 latency is paid once per chunk.
    if (!zero) {
      const cplx<T> rinv = crecip<T>(d);
      for (int i = col + 1 + tid; i < n; i += PANEL_THREADS) {
        cplx<T>* row = A + (size_t)i;
        const cplx<T> l = cmul<T>(row[(size_t)col * ld], rinv);
        row[(size_t)col * ld] = l;
        for (int j0 = col + 1; j0 < jend; j0 += 8) {
          cplx<T> v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (j0 + u < jend) v[u] = row[(size_t)(j0 + u) * ld];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (j0 + u < jend) row[(size_t)(j0 + u) * ld] = csub<T>(v[u], cmul<T>(l, s_u[j0 + u - k0]));
        }
      }
    }
    __syncthreads();
  }
}

// Interchanges of one panel applied to 32 "other" columns per CTA, then, for
// columns right of the panel, U12 = L11^{-1} A12 (unit lower, column-oriented).
template <typename T>
__global__ void __launch_bounds__(256)
k_laswp_trsm(cplx<T>* S, long long ld, long long stride, int n, int k0, int w, const int32_t* piv) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* L = reinterpret_cast<cplx<T>*>(smem_raw);  // w x w, [r * w + s]
  cplx<T>* X = L + w * w;                              // w x 32, [r * 32 + cc]
  const int b = blockIdx.y, tid = threadIdx.x;
  cplx<T>* A = S + (size_t)b * stride;
  const int32_t* pv = piv + (size_t)b * n;
  const int nother = n - w;
  const int o = blockIdx.x * 32 + (tid & 31);
  const bool valid = o < nother;
  const int c = valid ? (o < k0 ? o : o + w) : 0;
  const bool right = valid && c >= k0 + w;
  if (tid < 32 && valid) {
    for (int r = 0; r < w; ++r) {
      const int p = pv[k0 + r];
      if (p != k0 + r) {
        cplx<T> t1 = A[(size_t)(k0 + r) + (size_t)c * ld];
        A[(size_t)(k0 + r) + (size_t)c * ld] = A[(size_t)p + (size_t)c * ld];
        A[(size_t)p + (size_t)c * ld] = t1;
      }
    }
  }
  // does any column of this CTA lie right of the panel?
  const int o_last = min(blockIdx.x * 32 + 31, nother - 1);
  const bool any_right = (o_last >= k0);
  if (!any_right) return;
  for (int idx = tid; idx < w * w; idx += 256) {
    const int r = idx % w, s2 = idx / w;
    L[r * w + s2] = A[(size_t)(k0 + r) + (size_t)(k0 + s2) * ld];
  }
  __syncthreads();
  const int cc = tid & 31;
  for (int r = tid >> 5; r < w; r += 8) X[r * 32 + cc] = right ? A[(size_t)(k0 + r) + (size_t)c * ld] : czero<T>();
  __syncthreads();
  for (int s2 = 0; s2 < w - 1; ++s2) {
    const cplx<T> xs = X[s2 * 32 + cc];
    for (int r = s2 + 1 + (tid >> 5); r < w; r += 8)
      X[r * 32 + cc] = csub<T>(X[r * 32 + cc], cmul<T>(L[r * w + s2], xs));
    __syncthreads();
  }
  if (right)
    for (int r = tid >> 5; r < w; r += 8) A[(size_t)(k0 + r) + (size_t)c * ld] = X[r * 32 + cc];
}

// The same from the panel's moved-row list (mv: count, dst[128], src[128], rows
// relative to k0) on the columns right of the panel only (the columns left of
// it go to k_laswp_mv_left): every moved element of a column is read first,
// then written to its new row, so the loads of a column are all in flight at
// once instead of one interchange after another.  Then U12 = L11^{-1} A12.
template <typename T>
__global__ void __launch_bounds__(256)
k_laswp_mv_trsm(cplx<T>* S, long long ld, long long stride, int n, int k0, int w, const int32_t* mv, int do_trsm) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* L = reinterpret_cast<cplx<T>*>(smem_raw);  // w x w, [r * w + s]
  cplx<T>* X = L + w * w;                              // w x 32, [r * 32 + cc]
  __shared__ cplx<T> vals[128 * 32];
  __shared__ int s_d[128], s_s[128], s_cnt;
  const int b = blockIdx.y, tid = threadIdx.x;
  cplx<T>* A = S + (size_t)b * stride;
  const int32_t* m = mv + (size_t)b * LU_MV_STRIDE;
  if (tid == 0) s_cnt = min(max(m[0], 0), 128);
  for (int e = tid; e < 128; e += 256) {
    s_d[e] = m[1 + e];
    s_s[e] = m[129 + e];
  }
  __syncthreads();
  const int cnt = s_cnt;
  const int nright = n - k0 - w;
  for (int idx = tid; idx < cnt * 32; idx += 256) {
    const int e = idx >> 5, o = blockIdx.x * 32 + (idx & 31);
    if (o < nright) vals[idx] = A[(size_t)(k0 + s_s[e]) + (size_t)(k0 + w + o) * ld];
  }
  __syncthreads();
  for (int idx = tid; idx < cnt * 32; idx += 256) {
    const int e = idx >> 5, o = blockIdx.x * 32 + (idx & 31);
    if (o < nright) A[(size_t)(k0 + s_d[e]) + (size_t)(k0 + w + o) * ld] = vals[idx];
  }
  if (!do_trsm) return;  // U12 is solved where it is staged
  const int o = blockIdx.x * 32 + (tid & 31);
  const bool right = o < nright;
  const int c = k0 + w + (right ? o : 0);
  __syncthreads();
  for (int idx = tid; idx < w * w; idx += 256) {
    const int r = idx % w, s2 = idx / w;
    L[r * w + s2] = A[(size_t)(k0 + r) + (size_t)(k0 + s2) * ld];
  }
  const int cc = tid & 31;
  for (int r = tid >> 5; r < w; r += 8) X[r * 32 + cc] = right ? A[(size_t)(k0 + r) + (size_t)c * ld] : czero<T>();
  __syncthreads();
  for (int s2 = 0; s2 < w - 1; ++s2) {
    const cplx<T> xs = X[s2 * 32 + cc];
    for (int r = s2 + 1 + (tid >> 5); r < w; r += 8)
      X[r * 32 + cc] = csub<T>(X[r * 32 + cc], cmul<T>(L[r * w + s2], xs));
    __syncthreads();
  }
  if (right)
    for (int r = tid >> 5; r < w; r += 8) A[(size_t)(k0 + r) + (size_t)c * ld] = X[r * 32 + cc];
}

// The moved rows of one panel (mv as above) on the columns left of it
// (0 .. k0-1, the finished L part): off the factorisation's critical path.
template <typename T>
__global__ void __launch_bounds__(256)
k_laswp_mv_left(cplx<T>* S, long long ld, long long stride, int c_lo, int k0, const int32_t* mv) {
  __shared__ cplx<T> vals[128 * 32];
  __shared__ int s_d[128], s_s[128], s_cnt;
  const int b = blockIdx.y, tid = threadIdx.x;
  cplx<T>* A = S + (size_t)b * stride;
  const int32_t* m = mv + (size_t)b * LU_MV_STRIDE;
  if (tid == 0) s_cnt = min(max(m[0], 0), 128);
  for (int e = tid; e < 128; e += 256) {
    s_d[e] = m[1 + e];
    s_s[e] = m[129 + e];
  }
  __syncthreads();
  const int cnt = s_cnt;
  for (int idx = tid; idx < cnt * 32; idx += 256) {
    const int e = idx >> 5, c = c_lo + blockIdx.x * 32 + (idx & 31);
    if (c < k0) vals[idx] = A[(size_t)(k0 + s_s[e]) + (size_t)c * ld];
  }
  __syncthreads();
  for (int idx = tid; idx < cnt * 32; idx += 256) {
    const int e = idx >> 5, c = c_lo + blockIdx.x * 32 + (idx & 31);
    if (c < k0) A[(size_t)(k0 + s_d[e]) + (size_t)c * ld] = vals[idx];
  }
}

// The interchanges of all panels of the outer block [K0, K1) on the columns
// col0 .. col0+ncols-1: one warp per column applies the panels' moved-row
// lists in order (lanes over the moved rows, so the panel's own top rows are
// read and written contiguously), with no barrier beyond the warp.
__global__ void __launch_bounds__(256)
k_laswp_block_cols(float2* S, long long ld, long long stride, int n, int K0, int K1, int col0, int ncols,
                   const int32_t* mv) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, b = blockIdx.y, q = gridDim.y;
  const int o = blockIdx.x * 8 + warp;
  if (o >= ncols) return;
  float2* col = S + (size_t)b * stride + (size_t)(col0 + o) * ld;
  for (int k0 = K0; k0 < K1; k0 += 64) {
    const int32_t* m = mv + ((size_t)(k0 / 64) * q + b) * LU_MV_STRIDE;
    const int cnt = min(max(__ldcg(m), 0), 128);
    float2 v[4];
    int d[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int e = lane + 32 * j;
      d[j] = -1;
      if (e < cnt) {
        const int sr = k0 + __ldcg(m + 129 + e), dd = k0 + __ldcg(m + 1 + e);
        if (sr >= k0 && sr < n && dd >= k0 && dd < n) {
          v[j] = col[sr];
          d[j] = dd;
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (d[j] >= 0) col[d[j]] = v[j];
    __syncwarp();
  }
}

// Row maps of deferred interchanges, kept per (slot, shift) in one int arena:
// the map itself (row i holds, after the interchanges, the row that was at
// map[i] before), and the compact list of the rows it moves (dst, src pairs in
// increasing dst, and their count).
struct RowMaps {
  int32_t *map = nullptr, *dst = nullptr, *src = nullptr, *cnt = nullptr;
};
__host__ __device__ inline RowMaps rowmaps_view(int32_t* base, long long n, int q, int nblk) {
  const size_t M = (size_t)nblk * q * n;
  RowMaps r;
  r.map = base;
  r.dst = base + M;
  r.src = base + 2 * M;
  r.cnt = base + 3 * M;
  return r;
}

// The rows i in [r0, n) with p[i - r0] != i, compacted in increasing i into
// dst/src (any multiple of 32 threads up to 1024, warp ballots); returns the
// count to every thread.
__device__ int block_compact(const int* p, int r0, int n, int32_t* dst, int32_t* src) {
  __shared__ int wcount[32];
  __shared__ int base;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int c0 = r0; c0 < n; c0 += blockDim.x) {
    const int i = c0 + threadIdx.x;
    const int v = i < n ? p[i - r0] : i;
    const bool moved = v != i;
    const unsigned bal = __ballot_sync(0xffffffffu, moved);
    if (lane == 0) wcount[w] = __popc(bal);
    __syncthreads();
    int off = base;
    for (int k = 0; k < w; ++k) off += wcount[k];
    off += __popc(bal & ((1u << lane) - 1u));
    if (moved) {
      dst[off] = i;
      src[off] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int k = 0; k < nw; ++k) t += wcount[k];
      base += t;
    }
    __syncthreads();
  }
  return base;
}

// Row maps of the interchanges of whole blocks of KB columns: for block
// blk = block0 + blockIdx.x and shift b, the moved-row lists of the block's
// panels (mv, LU_MV_STRIDE ints per panel and shift: count, dst[128],
// src[128], rows relative to the panel's first row) applied in order to an
// index array, so that after them row i (>= blk KB) holds the row that was at
// map[i] before; the map and its own moved-row list go to slot blk.  1024
// threads (one CTA per block and shift).
__global__ void __launch_bounds__(1024)
k_block_rowmaps(const int32_t* mv, int n, int KB, int block0, int32_t* base, int nblk) {
  extern __shared__ int rm_sh[];
  const int blk = block0 + blockIdx.x, b = blockIdx.y, q = gridDim.y;
  const int K0 = blk * KB, K1 = min(K0 + KB, n), len = n - K0;
  if (len <= 0) return;
  const RowMaps rm = rowmaps_view(base, n, q, nblk);
  int* p = rm_sh;  // len
  __shared__ int vals[128];
  for (int i = threadIdx.x; i < len; i += blockDim.x) p[i] = K0 + i;
  __syncthreads();
  for (int k0 = K0; k0 < K1; k0 += 64) {
    const int32_t* m = mv + ((size_t)(k0 / 64) * q + b) * LU_MV_STRIDE;
    const int cnt = min(max(__ldcg(m), 0), 128);
    int d = -1, v = 0;
    if (threadIdx.x < cnt) {
      const int sr = k0 + __ldcg(m + 129 + threadIdx.x);
      d = k0 + __ldcg(m + 1 + threadIdx.x);
      if (sr >= K0 && sr < n && d >= K0 && d < n) v = p[sr - K0]; else d = -1;
    }
    if (threadIdx.x < 128) vals[threadIdx.x] = v;
    __syncthreads();
    if (d >= 0) p[d - K0] = vals[threadIdx.x];
    __syncthreads();
  }
  const size_t li = (size_t)blk * q + b;
  int32_t* mo = rm.map + li * n;
  for (int i = threadIdx.x; i < len; i += blockDim.x) mo[K0 + i] = p[i];
  const int cnt = block_compact(p, K0, n, rm.dst + li * n, rm.src + li * n);
  if (threadIdx.x == 0) rm.cnt[li] = cnt;
}

// The deferred interchanges of the finished L columns: the columns of block
// B - 1 need the interchanges of blocks B .. nblk-1 in order, whose row map is
// t_{B-1}[i] = s_B[t_B[i]] (s_B block B's own map, t_{nblk-1} the identity,
// rows i >= B KB).  One CTA per shift, backward over the blocks; t_{B-1} and
// its moved-row list overwrite slot B.
__global__ void __launch_bounds__(1024) k_compose_tail_maps(int32_t* base, int n, int KB, int nblk) {
  extern __shared__ int cm_sh[];
  int* cur = cm_sh;
  int* nxt = cm_sh + n;
  const int b = blockIdx.x, q = gridDim.x, tid = threadIdx.x;
  const RowMaps rm = rowmaps_view(base, n, q, nblk);
  for (int i = tid; i < n; i += blockDim.x) cur[i] = i;
  __syncthreads();
  for (int B = nblk - 1; B >= 1; --B) {
    const size_t li = (size_t)B * q + b;
    int32_t* sB = rm.map + li * n;
    const int K0 = B * KB;
    for (int i = K0 + tid; i < n; i += blockDim.x) nxt[i] = __ldcg(sB + cur[i]);
    __syncthreads();
    for (int i = K0 + tid; i < n; i += blockDim.x) {
      cur[i] = nxt[i];
      sB[i] = nxt[i];
    }
    const int cnt = block_compact(nxt + K0, K0, n, rm.dst + li * n, rm.src + li * n);
    if (tid == 0) rm.cnt[li] = cnt;
    __syncthreads();
  }
}

// Row permutation of whole columns by a moved-row list: column c
// (col0 <= c < col0 + ncols) of every shift gets new row dst_e = old row src_e.
// When most of the column's rows r0 .. n-1 move, the segment is read once,
// coalesced, into shared memory; otherwise only the moved rows are read.
// tail = false: r0 = R0 and slot `slot` for all columns (the far step);
// tail = true: column c of block B = c / KB takes r0 = (B + 1) KB and slot
// B + 1 (the deferred pass).
template <bool TAIL>
__global__ void __launch_bounds__(256)
k_permute_rows(float2* S, long long ld, long long stride, int n, int col0, int ncols, int32_t* base, int nblk,
               int KB, int R0, int slot) {
  extern __shared__ float2 pr_seg[];
  constexpr int CPB = 16;  // columns per CTA (a divisor of 64: no CTA straddles a block)
  const int b = blockIdx.y, q = gridDim.y;
  const RowMaps rm = rowmaps_view(base, n, q, nblk);
  float2* A = S + (size_t)b * stride;
  for (int j = 0; j < CPB; ++j) {
    const int c = col0 + blockIdx.x * CPB + j;
    if (c >= col0 + ncols) break;
    const int r0 = TAIL ? (c / KB + 1) * KB : R0;
    if (r0 >= n) continue;
    const size_t li = (size_t)(TAIL ? c / KB + 1 : slot) * q + b;
    const int cnt = min(__ldcg(rm.cnt + li), n - r0);
    if (cnt <= 0) continue;
    const int32_t* dl = rm.dst + li * n;
    const int32_t* sl = rm.src + li * n;
    float2* col = A + (size_t)c * ld;
    __syncthreads();  // the previous column's reads of pr_seg are done
    if (4 * cnt >= n - r0) {
      for (int i = r0 + threadIdx.x; i < n; i += blockDim.x) pr_seg[i - r0] = __ldcg(col + i);
      __syncthreads();
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int d = __ldcg(dl + e), sr = __ldcg(sl + e);
        if (d >= r0 && d < n && sr >= r0 && sr < n) col[d] = pr_seg[sr - r0];
      }
    } else {
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int sr = __ldcg(sl + e);
        pr_seg[e] = (sr >= r0 && sr < n) ? __ldcg(col + sr) : make_float2(0.f, 0.f);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int d = __ldcg(dl + e), sr = __ldcg(sl + e);
        if (d >= r0 && d < n && sr >= r0 && sr < n) col[d] = pr_seg[e];
      }
    }
  }
}

// The moved rows of the panel at k0 (mv relative to k0) on the columns
// col0 .. col0+ncols-1: each block gathers its 32 columns' moved entries, then
// writes them to their new rows.
template <typename T>
__global__ void __launch_bounds__(256)
k_laswp_mv_cols(cplx<T>* S, long long ld, long long stride, int k0, int col0, int ncols, const int32_t* mv) {
  __shared__ cplx<T> vals[128 * 32];
  __shared__ int s_d[128], s_s[128], s_cnt;
  const int b = blockIdx.y, tid = threadIdx.x;
  cplx<T>* A = S + (size_t)b * stride;
  const int32_t* m = mv + (size_t)b * LU_MV_STRIDE;
  if (tid == 0) s_cnt = min(max(m[0], 0), 128);
  for (int e = tid; e < 128; e += 256) {
    s_d[e] = m[1 + e];
    s_s[e] = m[129 + e];
  }
  __syncthreads();
  const int cnt = s_cnt;
  for (int idx = tid; idx < cnt * 32; idx += 256) {
    const int e = idx >> 5, o = blockIdx.x * 32 + (idx & 31);
    if (o < ncols) vals[idx] = A[(size_t)(k0 + s_s[e]) + (size_t)(col0 + o) * ld];
  }
  __syncthreads();
  for (int idx = tid; idx < cnt * 32; idx += 256) {
    const int e = idx >> 5, o = blockIdx.x * 32 + (idx & 31);
    if (o < ncols) A[(size_t)(k0 + s_d[e]) + (size_t)(col0 + o) * ld] = vals[idx];
  }
}

// T = -D^{-1} for diagonal blocks D of the factor: D = the unit lower part
// (UPPER = false) or the upper part with its diagonal (UPPER = true) of
// S[r0:r0+KB, r0:r0+KB], r0 = KB * block; rows and columns at or beyond n act as
// the identity (a ragged last block).  One CTA per (CW-column block j of the
// inverse, diagonal block, shift): X = D^{-1} E_j by block substitution -- for
// each 64-row block I reached from the one holding column CW j (downward for
// L, upward for U), the products with the blocks of X already solved (D from
// global memory through shared memory, X in shared memory), then the 64 x 64
// triangular solve (256 / CW threads per column, one barrier per step).  The
// narrow column blocks keep two CTAs on an SM (each about 100 KB of shared
// memory at CW = 32) and halve the work of the CTAs that hold the first
// columns, which set the duration.  With T, a product that overwrites its
// output (C = 0 - T X) gives D^{-1} X without cancelling against X.  T goes to
// T + ((block - block0) q + shift) KB^2, column-major with leading dimension KB.
template <bool UPPER, int CW>
__global__ void __launch_bounds__(256)
k_block_tri_inv(const float2* S, long long ld, long long stride, int n, int KB, int block0, float2* T) {
  constexpr int RG = 256 / CW;  // row groups: thread rows rq, rq + RG, ...
  constexpr int RPT = 64 / RG;  // rows of a 64-row block per thread
  constexpr int XS = CW + 1;    // padded row stride of X
  extern __shared__ __align__(16) unsigned char ti_smem[];
  float2* X = reinterpret_cast<float2*>(ti_smem);  // [KB][XS]
  float2* Db = X + (size_t)KB * XS;                // [64][65]
  const int j = blockIdx.x, blk = block0 + blockIdx.y, b = blockIdx.z, q = gridDim.z;
  const int tid = threadIdx.x, c = tid % CW, rq = tid / CW;
  const int r0 = KB * blk, nr = min(KB, n - r0);
  const float2* A = S + (size_t)b * stride + (size_t)r0 + (size_t)r0 * ld;
  const int nbk = KB / 64, jb = (CW * j) / 64;
  // D(r, t) of the block, identity outside the valid nr x nr part
  auto dval = [&](int r, int t) -> float2 {
    if (r == t && (!UPPER || r >= nr)) return make_float2(1.f, 0.f);
    if (r >= nr || t >= nr) return make_float2(0.f, 0.f);
    if (UPPER ? r > t : r < t) return make_float2(0.f, 0.f);
    return A[(size_t)r + (size_t)t * ld];
  };
  for (int s2 = 0; s2 < nbk; ++s2) {
    const int I = UPPER ? jb - s2 : jb + s2;
    if (I < 0 || I >= nbk) continue;
    float2 acc[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int r = rq + RG * k;
      acc[k] = make_float2(64 * I + r == CW * j + c ? 1.f : 0.f, 0.f);
    }
    for (int s3 = 0; s3 < s2; ++s3) {
      const int J = UPPER ? jb - s3 : jb + s3;  // blocks of X solved before I
      __syncthreads();
      for (int e = tid; e < 64 * 64; e += 256) {
        const int r = e & 63, t = e >> 6;
        Db[r * 65 + t] = dval(64 * I + r, 64 * J + t);
      }
      __syncthreads();
      for (int t = 0; t < 64; ++t) {
        const float2 xv = X[(size_t)(64 * J + t) * XS + c];
#pragma unroll
        for (int k = 0; k < RPT; ++k) acc[k] = csub<float>(acc[k], cmul<float>(Db[(rq + RG * k) * 65 + t], xv));
      }
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) X[(size_t)(64 * I + rq + RG * k) * XS + c] = acc[k];
    __syncthreads();
    for (int e = tid; e < 64 * 64; e += 256) {
      const int r = e & 63, t = e >> 6;
      Db[r * 65 + t] = dval(64 * I + r, 64 * I + t);
    }
    __syncthreads();
    float2* Xc = X + (size_t)(64 * I) * XS + c;
    if (!UPPER) {  // unit lower: forward
      for (int t = 0; t < 63; ++t) {
        const float2 xt = Xc[(size_t)t * XS];
        for (int r = t + 1 + ((rq - (t + 1)) & (RG - 1)); r < 64; r += RG)
          Xc[(size_t)r * XS] = csub<float>(Xc[(size_t)r * XS], cmul<float>(Db[r * 65 + t], xt));
        __syncthreads();
      }
    } else {  // upper with its diagonal: backward, the owner of row t divides first
      for (int t = 63; t >= 0; --t) {
        if ((t & (RG - 1)) == rq) Xc[(size_t)t * XS] = cdiv<float>(Xc[(size_t)t * XS], Db[t * 65 + t]);
        __syncthreads();
        const float2 xt = Xc[(size_t)t * XS];
        for (int r = rq; r < t; r += RG)
          Xc[(size_t)r * XS] = csub<float>(Xc[(size_t)r * XS], cmul<float>(Db[r * 65 + t], xt));
      }
      __syncthreads();
    }
  }
  float2* Tb = T + ((size_t)(blk - block0) * q + b) * KB * KB;
  for (int e = tid; e < KB * CW; e += 256) {
    const int r = e % KB, cc = e / KB, col = CW * j + cc;
    const bool solved = UPPER ? r < 64 * (jb + 1) : r >= 64 * jb;
    const float2 x = solved ? X[(size_t)r * XS + cc] : make_float2(0.f, 0.f);
    Tb[(size_t)r + (size_t)col * KB] = make_float2(-x.x, -x.y);
  }
}

// Row permutation vector from the interchange sequence: perm = P applied to 0..n-1.
__global__ void k_piv_to_perm(const int32_t* piv, int32_t* perm, int32_t* pinv, int n) {
  const int b = blockIdx.x;
  const int32_t* pv = piv + (size_t)b * n;
  int32_t* pm = perm + (size_t)b * n;
  int32_t* pi = pinv + (size_t)b * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) pm[i] = i;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < n; ++k) {
      const int p = pv[k];
      if (p != k && p >= 0 && p < n) { int t = pm[k]; pm[k] = pm[p]; pm[p] = t; }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) pi[pm[i]] = i;
}

}  // namespace

template <typename T>
cudaError_t default_trailing_update(const LuBatch<T>& lu, int k0, int w, int c0, int nc, bool, void*, cudaStream_t s) {
  const int rest = lu.n - k0 - w;
  if (rest <= 0 || nc <= 0) return cudaSuccess;
  GemmArgs<T> g;
  g.M = rest; g.N = nc; g.K = w; g.batch = lu.q;
  g.alpha = mk<T>(T(-1), T(0));
  g.beta = mk<T>(T(1), T(0));
  g.A = lu.S + (size_t)(k0 + w) + (size_t)k0 * lu.ld;  g.lda = lu.ld; g.strideA = lu.stride; g.opA = OP_N;
  g.B = lu.S + (size_t)k0 + (size_t)c0 * lu.ld;        g.ldb = lu.ld; g.strideB = lu.stride; g.opB = OP_N;
  g.C = lu.S + (size_t)(k0 + w) + (size_t)c0 * lu.ld;  g.ldc = lu.ld; g.strideC = lu.stride;
  return gemm_batched<T>(g, s);
}
template cudaError_t default_trailing_update<double>(const LuBatch<double>&, int, int, int, int, bool, void*,
                                                     cudaStream_t);
template cudaError_t default_trailing_update<float>(const LuBatch<float>&, int, int, int, int, bool, void*,
                                                    cudaStream_t);

namespace {

// ---------------------------------------------------------------- solves
enum DiagMode { D_LOWER_UNIT = 0, D_UPPER = 1, D_UPPER_H = 2, D_LOWER_H = 3 };

// Solve with the w x w diagonal block at (k0, k0) for 32 right-hand sides per CTA.
//  D_LOWER_UNIT : L_kk x = b            (forward)
//  D_UPPER      : U_kk x = b            (backward)
//  D_UPPER_H    : U_kk^H x = b          (forward, lower non-unit)
//  D_LOWER_H    : L_kk^H x = b          (backward, upper unit)
template <typename T>
__global__ void __launch_bounds__(256)
k_trsm_diag(const cplx<T>* S, long long ld, long long stride, cplx<T>* Xg, long long ldx,
            long long stridex, int k0, int w, int m, int mode) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* D = reinterpret_cast<cplx<T>*>(smem_raw);  // [r * w + s] = S[k0 + r, k0 + s]
  cplx<T>* X = D + w * w;                              // [r * 32 + cc]
  const int b = blockIdx.y, tid = threadIdx.x, cc = tid & 31, rg = tid >> 5;
  const cplx<T>* A = S + (size_t)b * stride;
  cplx<T>* Xb = Xg + (size_t)b * stridex;
  const int c = blockIdx.x * 32 + cc;
  const bool valid = c < m;
  for (int idx = tid; idx < w * w; idx += 256) {
    const int r = idx % w, s2 = idx / w;
    D[r * w + s2] = A[(size_t)(k0 + r) + (size_t)(k0 + s2) * ld];
  }
  for (int r = rg; r < w; r += 8) X[r * 32 + cc] = valid ? Xb[(size_t)(k0 + r) + (size_t)c * ldx] : czero<T>();
  __syncthreads();
  if (mode == D_LOWER_UNIT || mode == D_UPPER_H) {
    for (int s2 = 0; s2 < w; ++s2) {
      if (mode == D_UPPER_H) {
        if (rg == 0) X[s2 * 32 + cc] = cdiv<T>(X[s2 * 32 + cc], cconj<T>(D[s2 * w + s2]));
        __syncthreads();
      }
      const cplx<T> xs = X[s2 * 32 + cc];
      for (int r = s2 + 1 + rg; r < w; r += 8) {
        const cplx<T> l = (mode == D_LOWER_UNIT) ? D[r * w + s2] : cconj<T>(D[s2 * w + r]);
        X[r * 32 + cc] = csub<T>(X[r * 32 + cc], cmul<T>(l, xs));
      }
      __syncthreads();
    }
  } else {
    for (int s2 = w - 1; s2 >= 0; --s2) {
      if (mode == D_UPPER) {
        if (rg == 0) X[s2 * 32 + cc] = cdiv<T>(X[s2 * 32 + cc], D[s2 * w + s2]);
        __syncthreads();
      }
      const cplx<T> xs = X[s2 * 32 + cc];
      for (int r = rg; r < s2; r += 8) {
        const cplx<T> u = (mode == D_UPPER) ? D[r * w + s2] : cconj<T>(D[s2 * w + r]);
        X[r * 32 + cc] = csub<T>(X[r * 32 + cc], cmul<T>(u, xs));
      }
      __syncthreads();
    }
  }
  if (valid)
    for (int r = rg; r < w; r += 8) Xb[(size_t)(k0 + r) + (size_t)c * ldx] = X[r * 32 + cc];
}

// X_b (n x m_out) from R (n x m): m_out = m, or 2m with the second half conj(R)
template <typename T>
__global__ void k_rows_gather(const double2* R, const int32_t* perm, cplx<T>* X, int n, int m,
                              bool permute, bool conj_dup) {
  const size_t b = blockIdx.y;
  const size_t total = (size_t)n * m * (conj_dup ? 2 : 1);
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n);
    const size_t c = idx / n;
    const int src = permute ? perm[b * n + i] : i;
    double2 v = R[(size_t)src + (c % m) * n];
    if (c >= (size_t)m) v.y = -v.y;
    X[b * total + idx] = cconv<T, double>(v);
  }
}

template <typename T>
__global__ void k_rows_scatter(const cplx<T>* V, const int32_t* perm, cplx<T>* Out, int n, int m) {
  const size_t b = blockIdx.y;
  const size_t total = (size_t)n * m;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n);
    const size_t c = idx / n;
    Out[b * total + (size_t)perm[b * n + i] + c * n] = V[b * total + idx];
  }
}

template <typename T>
size_t diag_smem(int w) { return (size_t)(w * w + w * 32) * sizeof(cplx<T>); }

// complex64 panels: the left-looking group form of panel_ll.cuh, one CTA per shift.
constexpr int PLL_THREADS = 512;
constexpr int PLL_GCAP = 16384;  // group buffer: 128 KB of complex64

template <int GW>
__global__ void __launch_bounds__(PLL_THREADS)
k_panel_ll(float2* S, long long ld, long long stride, int n, int k0, int w, int32_t* piv, int* info, unsigned* flags,
           int gcap, int32_t* mv) {
  extern __shared__ __align__(16) unsigned char pll_smem[];
  __shared__ PanelShared sh;
  const int b = blockIdx.x;
  float2* Lt = reinterpret_cast<float2*>(pll_smem);
  float2* G = Lt + 64 * 64;
  int* pl = reinterpret_cast<int*>(G + gcap);
  panel_ll<GW, PLL_THREADS>(S + (size_t)b * stride, ld, n, k0, w, piv + (size_t)b * n + k0, info + b, flags, Lt, G,
                            pl, sh);
  if (mv) {  // the moved rows, for the interchanges on the other columns
    int32_t* o = mv + (size_t)b * LU_MV_STRIDE;
    const int cnt = sh.cnt;
    if (threadIdx.x == 0) o[0] = cnt;
    for (int e = threadIdx.x; e < cnt; e += PLL_THREADS) {
      o[1 + e] = sh.mvd[e];
      o[129 + e] = sh.mvs[e];
    }
  }
}

size_t pll_smem_bytes(int n, int gcap) { return (size_t)64 * 64 * sizeof(float2) + (size_t)gcap * sizeof(float2) + (size_t)n * sizeof(int); }

template <int GW>
cudaError_t launch_panel_ll(const LuBatch<float>& lu, int k0, int w, int gcap, cudaStream_t s) {
  const size_t smem = pll_smem_bytes(lu.n, gcap);
  cudaError_t e = cudaFuncSetAttribute(k_panel_ll<GW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  feast_count_launch();
  k_panel_ll<GW><<<lu.q, PLL_THREADS, smem, s>>>(reinterpret_cast<float2*>(lu.S), lu.ld, lu.stride, lu.n, k0, w,
                                                 lu.piv, lu.info, lu.flags, gcap,
                                                 lu.mv ? lu.mv + (size_t)(k0 / 64) * lu.q * LU_MV_STRIDE : nullptr);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_panel(const LuBatch<T>& lu, int k0, int w, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (lu.panel_cluster && panel_cluster_applies(lu.n - k0, w, lu.cluster_min_rows) && lu.mv)
      return panel_cluster(lu, k0, w, s);
    if (w <= 64 && lu.n <= PLL_GCAP) {
      const int gcap = min(PLL_GCAP, 8 * lu.n);
      switch (panel_group_width(lu.n - k0, gcap)) {
        case 8: return launch_panel_ll<8>(lu, k0, w, gcap, s);
        case 4: return launch_panel_ll<4>(lu, k0, w, gcap, s);
        case 2: return launch_panel_ll<2>(lu, k0, w, gcap, s);
        default: return launch_panel_ll<1>(lu, k0, w, gcap, s);
      }
    }
  }
  feast_count_launch();
  k_panel<T><<<lu.q, PANEL_THREADS, 0, s>>>(lu.S, lu.ld, lu.stride, lu.n, k0, w, lu.piv, lu.info, lu.flags);
  return cudaGetLastError();
}

}  // namespace

namespace {

cudaError_t smem_attr(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Row maps of the blocks block_from .. nblk-1 (blocks of KB columns), their
// composition from the back, and the one deferred permutation of the finished
// L columns of blocks 0 .. nblk-2 (lu.rowmaps holds nblk x q x n ints).
cudaError_t deferred_left_swaps(const LuBatch<float>& lu, int KB, int block_from, cudaStream_t s) {
  const int n = lu.n, nblk = (n + KB - 1) / KB;
  if (nblk < 2) return cudaSuccess;
  cudaError_t e;
  if (block_from < nblk) {
    const size_t sm = (size_t)n * sizeof(int);
    if ((e = smem_attr((const void*)k_block_rowmaps, sm)) != cudaSuccess) return e;
    feast_count_launch();
    k_block_rowmaps<<<dim3(nblk - block_from, lu.q), 1024, sm, s>>>(lu.mv, n, KB, block_from, lu.rowmaps, nblk);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const size_t smc = 2 * (size_t)n * sizeof(int);
  if ((e = smem_attr((const void*)k_compose_tail_maps, smc)) != cudaSuccess) return e;
  feast_count_launch();
  k_compose_tail_maps<<<lu.q, 1024, smc, s>>>(lu.rowmaps, n, KB, nblk);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int ncols = (nblk - 1) * KB;
  const size_t smp = (size_t)n * sizeof(float2);
  if ((e = smem_attr((const void*)k_permute_rows<true>, smp)) != cudaSuccess) return e;
  feast_count_launch();
  k_permute_rows<true><<<dim3(ceil_div(ncols, 16), lu.q), 256, smp, s>>>(reinterpret_cast<float2*>(lu.S), lu.ld,
                                                                         lu.stride, n, 0, ncols, lu.rowmaps, nblk, KB,
                                                                         0, 0);
  return cudaGetLastError();
}

}  // namespace

size_t lu_rowmap_ints(long long n, int q, int KB) {
  const size_t nblk = (size_t)((n + KB - 1) / KB);
  return 3 * nblk * q * (size_t)n + nblk * q;
}

cudaError_t block_swaps_far(const LuBatch<float>& lu, int K0, int KB, cudaStream_t s) {
  const int far0 = K0 + KB, nfar = lu.n - far0;
  if (nfar <= 0) return cudaSuccess;
  if (!lu.mv || K0 % 64 || KB % 64) return cudaErrorInvalidValue;
  feast_count_launch();
  k_laswp_block_cols<<<dim3(ceil_div(nfar, 8), lu.q), 256, 0, s>>>(reinterpret_cast<float2*>(lu.S), lu.ld,
                                                                  lu.stride, lu.n, K0, far0, far0, nfar, lu.mv);
  return cudaGetLastError();
}

template <typename T>
cudaError_t lu_factor_batched(const LuBatch<T>& lu_in, int nb, TrailingUpdateFn<T> upd, void* ctx,
                              cudaStream_t s) {
  LuBatch<T> lu = lu_in;
  if (nb < 1 || nb > MAX_NB || diag_smem<T>(nb) > 227 * 1024) return cudaErrorInvalidValue;
  if (!upd) upd = default_trailing_update<T>;
  cudaError_t e = cudaFuncSetAttribute(k_laswp_trsm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)diag_smem<T>(nb));
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(lu.info, 0, sizeof(int) * lu.q, s);
  // side stream (highest priority, so that the panel's CTAs are dispatched as
  // soon as SMs free up) and the two events of each step
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  cudaStream_t side = nullptr, lstream = nullptr;  // panels; interchanges on the finished L columns
  cudaEvent_t ev_next = nullptr, ev_panel = nullptr, ev_left = nullptr;
  if ((e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, hi)) != cudaSuccess) return e;
  auto cleanup = [&](cudaError_t r) {
    if (ev_next) cudaEventDestroy(ev_next);
    if (ev_panel) cudaEventDestroy(ev_panel);
    if (ev_left) cudaEventDestroy(ev_left);
    if (lstream) cudaStreamDestroy(lstream);
    cudaStreamDestroy(side);
    return r;
  };
  if ((e = cudaEventCreateWithFlags(&ev_next, cudaEventDisableTiming)) != cudaSuccess) return cleanup(e);
  if ((e = cudaEventCreateWithFlags(&ev_panel, cudaEventDisableTiming)) != cudaSuccess) return cleanup(e);
  if ((e = cudaEventCreateWithFlags(&ev_left, cudaEventDisableTiming)) != cudaSuccess) return cleanup(e);
  if ((e = cudaStreamCreateWithPriority(&lstream, cudaStreamNonBlocking, lo)) != cudaSuccess) return cleanup(e);
  // the complex64 group panel leaves its moved-row list for the interchanges
  const bool use_mv = std::is_same<T, float>::value && lu.mv && nb == 64 && lu.n <= PLL_GCAP &&
                      lu.mv_panels >= (lu.n + 63) / 64;
  // the staging kernel takes over the interchanges on the right columns and
  // U12 = L11^{-1} A12 only together with the moved-row lists
  lu.u12_in_stage = lu.u12_in_stage && use_mv;
  if constexpr (std::is_same<T, float>::value) {
    if (use_mv && (e = cudaFuncSetAttribute(k_laswp_mv_trsm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)diag_smem<float>(nb))) != cudaSuccess)
      return e;
  }
  auto laswp = [&](int k0, int w) -> cudaError_t {
    const int nother = lu.n - w;
    if (nother <= 0) return cudaSuccess;
    dim3 grid(ceil_div(nother, 32), lu.q);
    feast_count_launch();
    if constexpr (std::is_same<T, float>::value) {
      if (use_mv) {
        // right columns here; the left ones on their own stream after this panel
        const int32_t* mvk = lu.mv + (size_t)(k0 / 64) * lu.q * LU_MV_STRIDE;
        const int nright = lu.n - k0 - w;
        if (nright > 0 && !lu.u12_in_stage) {
          k_laswp_mv_trsm<float><<<dim3(ceil_div(nright, 32), lu.q), 256, diag_smem<float>(w), s>>>(
              lu.S, lu.ld, lu.stride, lu.n, k0, w, mvk, lu.u12_in_stage ? 0 : 1);
          cudaError_t r = cudaGetLastError();
          if (r != cudaSuccess) return r;
        }
        if (k0 > 0 && !lu.rowmaps) {  // (with row maps: one deferred pass at the end)
          // s has waited for this panel: the left stream starts from here
          cudaError_t r = cudaEventRecord(ev_left, s);
          if (r == cudaSuccess) r = cudaStreamWaitEvent(lstream, ev_left, 0);
          if (r != cudaSuccess) return r;
          feast_count_launch();
          k_laswp_mv_left<float><<<dim3(ceil_div(k0, 32), lu.q), 256, 0, lstream>>>(lu.S, lu.ld, lu.stride, 0, k0,
                                                                                     mvk);
          return cudaGetLastError();
        }
        return cudaSuccess;
      }
    }
    k_laswp_trsm<T><<<grid, 256, diag_smem<T>(w), s>>>(lu.S, lu.ld, lu.stride, lu.n, k0, w, lu.piv);
    return cudaGetLastError();
  };
  if ((e = launch_panel<T>(lu, 0, min(nb, lu.n), s)) != cudaSuccess) return cleanup(e);
  if ((e = laswp(0, min(nb, lu.n))) != cudaSuccess) return cleanup(e);
  for (int k0 = 0; k0 < lu.n; k0 += nb) {
    const int w = min(nb, lu.n - k0);
    const int rest = lu.n - k0 - w;
    if (rest <= 0) break;
    const int k1 = k0 + w, w1 = min(nb, rest);
    // block column k+1 first, then panel k+1 beside the rest of the update
    if ((e = upd(lu, k0, w, k1, w1, true, ctx, s)) != cudaSuccess) return cleanup(e);
    if ((e = cudaEventRecord(ev_next, s)) != cudaSuccess) return cleanup(e);
    if ((e = cudaStreamWaitEvent(side, ev_next, 0)) != cudaSuccess) return cleanup(e);
    if ((e = launch_panel<T>(lu, k1, w1, side)) != cudaSuccess) return cleanup(e);
    if ((e = cudaEventRecord(ev_panel, side)) != cudaSuccess) return cleanup(e);
    if (rest > w1 && (e = upd(lu, k0, w, k1 + w1, rest - w1, false, ctx, s)) != cudaSuccess) return cleanup(e);
    if ((e = cudaStreamWaitEvent(s, ev_panel, 0)) != cudaSuccess) return cleanup(e);
    if ((e = laswp(k1, w1)) != cudaSuccess) return cleanup(e);
  }
  // the left interchanges are done before anything reads L (the left stream
  // has work only without row maps; an unused stream is not joined, so that a
  // stream capture of this function never waits on an event from outside it)
  const bool deferred = std::is_same<T, float>::value && use_mv && lu.rowmaps;
  if (!deferred) {
    if ((e = cudaEventRecord(ev_left, lstream)) != cudaSuccess) return cleanup(e);
    if ((e = cudaStreamWaitEvent(s, ev_left, 0)) != cudaSuccess) return cleanup(e);
  }
  if constexpr (std::is_same<T, float>::value) {
    if (deferred && (e = deferred_left_swaps(lu, 64, 0, s)) != cudaSuccess) return cleanup(e);
  }
  feast_count_launch();
  k_piv_to_perm<<<lu.q, 256, 0, s>>>(lu.piv, lu.perm, lu.pinv, lu.n);
  return cleanup(cudaGetLastError());
}

template <typename T>
cudaError_t lu_solve_batched(const LuBatch<T>& lu, int side, cplx<T>* X, int m, int nbs, cudaStream_t s) {
  if (nbs < 1 || nbs > MAX_NB || diag_smem<T>(nbs) > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_trsm_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)diag_smem<T>(nbs));
  if (e != cudaSuccess) return e;
  const int n = lu.n;
  const long long ldx = n, sx = (long long)n * m;
  auto diag = [&](int k0, int w, int mode) {
    dim3 grid(ceil_div(m, 32), lu.q);
    feast_count_launch();
    k_trsm_diag<T><<<grid, 256, diag_smem<T>(w), s>>>(lu.S, lu.ld, lu.stride, X, ldx, sx, k0, w, m, mode);
  };
  // X[row_out : row_out+M] -= op(A) X[row_in : row_in+K], A the factor block at
  // (ar0, ac0): op N rows ar0.., columns ac0..; op C the conjugate transpose of
  // the block at rows ac0.., columns ar0..
  auto update = [&](int M, int K, int ar0, int ac0, int opA, int row_out, int row_in) {
    if (M <= 0) return cudaSuccess;
    if constexpr (std::is_same<T, float>::value) {
      if (lu.tc) {
        cudaError_t err = cudaSuccess;
        if (tc_solve_update(lu, X, m, M, K, ar0, ac0, opA, row_out, row_in, -1, s, &err)) return err;
      }
    }
    const cplx<T>* Aop = opA == OP_N ? lu.S + (size_t)ar0 + (size_t)ac0 * lu.ld : lu.S + (size_t)ac0 + (size_t)ar0 * lu.ld;
    GemmArgs<T> g;
    g.M = M; g.N = m; g.K = K; g.batch = lu.q;
    g.alpha = mk<T>(T(-1), T(0));
    g.beta = mk<T>(T(1), T(0));
    g.A = Aop; g.lda = lu.ld; g.strideA = lu.stride; g.opA = opA;
    g.B = X + row_in; g.ldb = ldx; g.strideB = sx; g.opB = OP_N;
    g.C = X + row_out; g.ldc = ldx; g.strideC = sx;
    return gemm_batched<T>(g, s);
  };
  // one block step: the diagonal solve (folded into the tensor-core staging
  // when that path applies) and the update of the rows still to be solved
  auto step = [&](int k0, int w, int mode, int M, int ar0, int ac0, int opA, int row_out) -> cudaError_t {
    if constexpr (std::is_same<T, float>::value) {
      if (lu.tc && M > 0) {
        cudaError_t err = cudaSuccess;
        if (tc_solve_update(lu, X, m, M, w, ar0, ac0, opA, row_out, k0, mode, s, &err)) return err;
      }
    }
    diag(k0, w, mode);
    return update(M, w, ar0, ac0, opA, row_out, k0);
  };
  const int last = ((n - 1) / nbs) * nbs;
  if (side == 0) {
    for (int k0 = 0; k0 < n; k0 += nbs) {  // L y = P r
      const int w = min(nbs, n - k0);
      if ((e = step(k0, w, D_LOWER_UNIT, n - k0 - w, k0 + w, k0, OP_N, k0 + w)) != cudaSuccess) return e;
    }
    for (int k0 = last; k0 >= 0; k0 -= nbs) {  // U x = y
      const int w = min(nbs, n - k0);
      if ((e = step(k0, w, D_UPPER, k0, 0, k0, OP_N, 0)) != cudaSuccess) return e;
    }
  } else {
    for (int k0 = 0; k0 < n; k0 += nbs) {  // U^H w = r; rows k0+w.. of op(A) = (U[k0:k0+w, k0+w:])^H
      const int w = min(nbs, n - k0);
      if ((e = step(k0, w, D_UPPER_H, n - k0 - w, k0 + w, k0, OP_C, k0 + w)) != cudaSuccess) return e;
    }
    for (int k0 = last; k0 >= 0; k0 -= nbs) {  // L^H v = w; rows 0..k0 of op(A) = (L[k0:k0+w, 0:k0])^H
      const int w = min(nbs, n - k0);
      if ((e = step(k0, w, D_LOWER_H, k0, 0, k0, OP_C, 0)) != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t rows_gather(const LuBatch<T>& lu, const double2* R, cplx<T>* X, int m, bool permute,
                        cudaStream_t s, bool conj_dup) {
  dim3 grid(ceil_div((size_t)lu.n * m * (conj_dup ? 2 : 1), 256 * 4), lu.q);
  feast_count_launch();
  k_rows_gather<T><<<grid, 256, 0, s>>>(R, lu.perm, X, lu.n, m, permute, conj_dup);
  return cudaGetLastError();
}

template <typename T>
cudaError_t rows_scatter(const LuBatch<T>& lu, const cplx<T>* V, cplx<T>* Out, int m, cudaStream_t s) {
  dim3 grid(ceil_div((size_t)lu.n * m, 256 * 4), lu.q);
  feast_count_launch();
  k_rows_scatter<T><<<grid, 256, 0, s>>>(V, lu.perm, Out, lu.n, m);
  return cudaGetLastError();
}

template cudaError_t lu_factor_batched<double>(const LuBatch<double>&, int, TrailingUpdateFn<double>, void*, cudaStream_t);
template cudaError_t lu_factor_batched<float>(const LuBatch<float>&, int, TrailingUpdateFn<float>, void*, cudaStream_t);
template cudaError_t lu_solve_batched<double>(const LuBatch<double>&, int, double2*, int, int, cudaStream_t);
template cudaError_t lu_solve_batched<float>(const LuBatch<float>&, int, float2*, int, int, cudaStream_t);
template cudaError_t rows_gather<double>(const LuBatch<double>&, const double2*, double2*, int, bool, cudaStream_t,
                                         bool);
template cudaError_t rows_gather<float>(const LuBatch<float>&, const double2*, float2*, int, bool, cudaStream_t, bool);
template cudaError_t rows_scatter<double>(const LuBatch<double>&, const double2*, double2*, int, cudaStream_t);
template cudaError_t rows_scatter<float>(const LuBatch<float>&, const float2*, float2*, int, cudaStream_t);

cudaError_t laswp_moved_rows(const LuBatch<float>& lu, int k0, int col0, int ncols, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  if (!lu.mv || k0 % 64) return cudaErrorInvalidValue;
  feast_count_launch();
  k_laswp_mv_cols<float><<<dim3(ceil_div(ncols, 32), lu.q), 256, 0, s>>>(
      lu.S, lu.ld, lu.stride, k0, col0, ncols, lu.mv + (size_t)(k0 / 64) * lu.q * LU_MV_STRIDE);
  return cudaGetLastError();
}

// Columns of the inverse per CTA of k_block_tri_inv (16, 32 or 64).
constexpr int kTriInvCols = 32;

cudaError_t block_inverse_negated(const LuBatch<float>& lu, bool upper, int KB, int block0, int nblocks, float2* T,
                                   cudaStream_t s) {
  if (KB % 64 || KB > 256 || KB < 64 || nblocks < 1 || block0 < 0 || (long long)KB * (block0 + nblocks - 1) >= lu.n)
    return cudaErrorInvalidValue;
  constexpr int CW = kTriInvCols;
  const size_t smem = (size_t)KB * (CW + 1) * sizeof(float2) + 64 * 65 * sizeof(float2);
  cudaError_t e = upper
                      ? cudaFuncSetAttribute(k_block_tri_inv<true, CW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                      : cudaFuncSetAttribute(k_block_tri_inv<false, CW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  feast_count_launch();
  const dim3 grid(KB / CW, nblocks, lu.q);
  const float2* S = reinterpret_cast<const float2*>(lu.S);
  if (upper)
    k_block_tri_inv<true, CW><<<grid, 256, smem, s>>>(S, lu.ld, lu.stride, lu.n, KB, block0, T);
  else
    k_block_tri_inv<false, CW><<<grid, 256, smem, s>>>(S, lu.ld, lu.stride, lu.n, KB, block0, T);
  return cudaGetLastError();
}

// Two-level blocked LU (complex64, tensor-core updates).  Inside each outer
// block of KB columns the panels of nb = 64 columns run as in the one-level
// schedule (the next block column updated first, the next panel on the
// high-priority side stream beside the rest of the update), except that every
// step touches only the block's own columns (lu.col_end).  At the end of the
// block `far` applies its panels to the block's rows of the columns beyond it,
// and `deep` subtracts the K = KB product from the rest of the matrix: that
// update carries almost all of the factorisation's flops at four times the
// arithmetic intensity of a K = 64 update.  The interchanges on the finished
// L columns run on a low-priority stream and are joined before `deep` stages L.
cudaError_t lu_factor_two_level(const LuBatch<float>& lu_in, int nb, int KB, TrailingUpdateFn<float> upd, void* ctx,
                                FarFn far, DeepFn deep, void* dctx, cudaStream_t s) {
  LuBatch<float> lu = lu_in;
  if (nb != 64 || KB < nb || KB % nb || !upd || !far || !deep || !lu.mv || lu.n > PLL_GCAP ||
      lu.mv_panels < (lu.n + 63) / 64)
    return cudaErrorInvalidValue;
  lu.u12_in_stage = true;
  cudaMemsetAsync(lu.info, 0, sizeof(int) * lu.q, s);
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  cudaStream_t side = nullptr, lstream = nullptr;
  cudaEvent_t ev_next = nullptr, ev_panel = nullptr, ev_left = nullptr;
  cudaError_t e;
  if ((e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, hi)) != cudaSuccess) return e;
  auto cleanup = [&](cudaError_t r) {
    if (ev_next) cudaEventDestroy(ev_next);
    if (ev_panel) cudaEventDestroy(ev_panel);
    if (ev_left) cudaEventDestroy(ev_left);
    if (lstream) cudaStreamDestroy(lstream);
    cudaStreamDestroy(side);
    return r;
  };
  if ((e = cudaEventCreateWithFlags(&ev_next, cudaEventDisableTiming)) != cudaSuccess) return cleanup(e);
  if ((e = cudaEventCreateWithFlags(&ev_panel, cudaEventDisableTiming)) != cudaSuccess) return cleanup(e);
  if ((e = cudaEventCreateWithFlags(&ev_left, cudaEventDisableTiming)) != cudaSuccess) return cleanup(e);
  if ((e = cudaStreamCreateWithPriority(&lstream, cudaStreamNonBlocking, lo)) != cudaSuccess) return cleanup(e);
  // the panel's moved rows on the finished L columns (0 .. k0-1), off the
  // critical path; with row maps only on the current outer block's columns
  // (the deep update reads them), the earlier blocks' in the deferred pass
  auto left = [&](int k0) -> cudaError_t {
    const int c_lo = lu.rowmaps ? (k0 / KB) * KB : 0;
    if (k0 <= c_lo) return cudaSuccess;
    cudaError_t r = cudaEventRecord(ev_left, s);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(lstream, ev_left, 0);
    if (r != cudaSuccess) return r;
    feast_count_launch();
    k_laswp_mv_left<float><<<dim3(ceil_div(k0 - c_lo, 32), lu.q), 256, 0, lstream>>>(
        lu.S, lu.ld, lu.stride, c_lo, k0, lu.mv + (size_t)(k0 / 64) * lu.q * LU_MV_STRIDE);
    return cudaGetLastError();
  };
  if ((e = launch_panel<float>(lu, 0, min(nb, lu.n), s)) != cudaSuccess) return cleanup(e);
  for (int K0 = 0; K0 < lu.n; K0 += KB) {
    const int cend = min(K0 + KB, lu.n);
    lu.col_end = cend;
    for (int k0 = K0; k0 < cend; k0 += nb) {
      const int w = min(nb, lu.n - k0);
      const int k1 = k0 + w;
      if (k1 >= cend) break;  // the block's last panel: no columns of the block right of it
      const int w1 = min(nb, cend - k1);
      if ((e = upd(lu, k0, w, k1, w1, true, ctx, s)) != cudaSuccess) return cleanup(e);
      if ((e = cudaEventRecord(ev_next, s)) != cudaSuccess) return cleanup(e);
      if ((e = cudaStreamWaitEvent(side, ev_next, 0)) != cudaSuccess) return cleanup(e);
      if ((e = launch_panel<float>(lu, k1, w1, side)) != cudaSuccess) return cleanup(e);
      if ((e = cudaEventRecord(ev_panel, side)) != cudaSuccess) return cleanup(e);
      if (cend > k1 + w1 && (e = upd(lu, k0, w, k1 + w1, cend - k1 - w1, false, ctx, s)) != cudaSuccess)
        return cleanup(e);
      if ((e = cudaStreamWaitEvent(s, ev_panel, 0)) != cudaSuccess) return cleanup(e);
      if ((e = left(k1)) != cudaSuccess) return cleanup(e);
    }
    if (cend >= lu.n) break;
    lu.col_end = 0;
    // the block's L is final once the interchanges of its later panels are on it
    if ((e = cudaEventRecord(ev_left, lstream)) != cudaSuccess) return cleanup(e);
    if ((e = cudaStreamWaitEvent(s, ev_left, 0)) != cudaSuccess) return cleanup(e);
    if ((e = far(lu, K0, cend - K0, dctx, s)) != cudaSuccess) return cleanup(e);
    if ((e = deep(lu, K0, cend - K0, dctx, s)) != cudaSuccess) return cleanup(e);
    if ((e = launch_panel<float>(lu, cend, min(nb, lu.n - cend), s)) != cudaSuccess) return cleanup(e);
    if ((e = left(cend)) != cudaSuccess) return cleanup(e);
  }
  if ((e = cudaEventRecord(ev_left, lstream)) != cudaSuccess) return cleanup(e);
  if ((e = cudaStreamWaitEvent(s, ev_left, 0)) != cudaSuccess) return cleanup(e);
  if (lu.rowmaps && (e = deferred_left_swaps(lu, KB, 0, s)) != cudaSuccess) return cleanup(e);
  feast_count_launch();
  k_piv_to_perm<<<lu.q, 256, 0, s>>>(lu.piv, lu.perm, lu.pinv, lu.n);
  return cleanup(cudaGetLastError());
}
