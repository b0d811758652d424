// Complex64 panel factorisation with partial pivoting, one CTA per panel,
// shared by the single-pencil LU and the batched persistent kernel.
//
// The panel is rows r0 .. N-1 and columns r0 .. r0+w-1 (w <= 64) of a
// column-major matrix.  It is factored left-looking, GW columns at a time:
// the group is gathered into shared memory in logical row order, brought up
// to date with the panel's earlier columns (a unit-lower solve for its rows
// above the group, then a product with the earlier L columns for the rest),
// and factored there with a block-wide pivot search per column (largest
// |Re| + |Im|, lowest row on ties).  Rows never move in memory while the
// panel is factored: `pl` maps logical to physical rows.  At the end the
// moved rows (at most 2w) are written in logical order, so the panel leaves
// memory exactly as a right-looking elimination with row interchanges would.
//
// Compared with a right-looking panel that streams the whole panel through
// L2 for every column (R x w x w / 2 complex read-modify-writes), the group
// form reads the earlier L columns once per group (R x w x w / (2 GW) reads)
// and keeps the rank-1 updates on chip.
#pragma once
#include "common.cuh"

struct PanelShared {
  int piv, cnt;
  float wv[32];
  int wi[32];
  int mvd[128], mvs[128];
};

__device__ __forceinline__ float2 pl_shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Largest group width whose R x GW buffer fits `gcap` elements.
__host__ __device__ __forceinline__ int panel_group_width(int R, int gcap) {
  return R * 8 <= gcap ? 8 : R * 4 <= gcap ? 4 : R * 2 <= gcap ? 2 : 1;
}

// Factor the panel.  Shared memory: Lt (64 x 64 float2), G (gcap float2), pl (R ints).
// piv[c] receives the interchange of column r0 + c as a global row (LAPACK
// style); info gets 1 + the first global column with an exact zero pivot.  On
// return sh.cnt / sh.mvd / sh.mvs hold the moved rows (relative to r0):
// logical row mvd[e] took physical row mvs[e].
template <int GW, int NT>
__device__ void panel_ll(float2* A, long long ld, int N, int r0, int w, int* piv, int* info, unsigned* flags,
                         float2* Lt, float2* G, int* pl, PanelShared& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int R = N - r0;
  for (int r = tid; r < R; r += NT) pl[r] = r;
  __syncthreads();
  for (int g0 = 0; g0 < w; g0 += GW) {
    const int gw = min(GW, w - g0);
    // the group's columns, several loads per thread in flight
    constexpr int GB = NT < 512 ? 4 : 8;
    for (int base = 0; base < R * gw; base += GB * NT) {
      float2 v[GB];
#pragma unroll
      for (int u = 0; u < GB; ++u) {
        const int idx = base + u * NT + tid;
        if (idx < R * gw) {
          const int c = idx / R, r = idx - c * R;
          v[u] = __ldcg(A + (size_t)(r0 + pl[r]) + (size_t)(r0 + g0 + c) * ld);
        }
      }
#pragma unroll
      for (int u = 0; u < GB; ++u) {
        const int idx = base + u * NT + tid;
        if (idx < R * gw) G[idx] = v[u];
      }
    }
    const int lrows = min(64, R);
    for (int idx = tid; idx < 64 * g0; idx += NT) {
      const int t = idx >> 6, r = idx & 63;
      if (r < lrows) Lt[idx] = __ldcg(A + (size_t)(r0 + pl[r]) + (size_t)(r0 + t) * ld);
    }
    __syncthreads();
    if (g0 > 0) {
      // rows above the group: forward substitution with L[0:g0, 0:g0]
      if (warp < gw) {
        float2* Gc = G + warp * R;
        float2 x0 = lane < g0 ? Gc[lane] : make_float2(0.f, 0.f);
        float2 x1 = lane + 32 < g0 ? Gc[lane + 32] : make_float2(0.f, 0.f);
        for (int t = 0; t < g0 - 1; ++t) {
          const float2 xt = pl_shfl2(t < 32 ? x0 : x1, t & 31);
          const float2 l0 = Lt[t * 64 + lane], l1 = Lt[t * 64 + lane + 32];
          if (lane > t && lane < g0) x0 = csub<float>(x0, cmul<float>(l0, xt));
          if (lane + 32 > t && lane + 32 < g0) x1 = csub<float>(x1, cmul<float>(l1, xt));
        }
        if (lane < g0) Gc[lane] = x0;
        if (lane + 32 < g0) Gc[lane + 32] = x1;
      }
      __syncthreads();
      // the remaining rows: G[r, c] -= sum_{t < g0} L[r, t] U[t, c].  The L
      // entries come from L2 and the loop is bound by their latency: each
      // thread takes RR rows and loads PF entries of each before using them,
      // so that RR * PF loads per thread are in flight.
      constexpr int PF = 8;
      // (the 256-thread persistent batch kernel keeps one row per thread: its
      // register budget is shared with its other task types)
      constexpr int RR = NT < 512 ? 1 : (GW >= 8 ? 2 : 4);
      for (int r = g0 + tid; r < R; r += RR * NT) {
        float2 acc[RR][GW];
#pragma unroll
        for (int q = 0; q < RR; ++q)
#pragma unroll
          for (int c = 0; c < GW; ++c) acc[q][c] = make_float2(0.f, 0.f);
        const float2* Lp[RR];
#pragma unroll
        for (int q = 0; q < RR; ++q) {
          const int rq = r + q * NT;
          Lp[q] = A + (size_t)(r0 + pl[rq < R ? rq : r]) + (size_t)r0 * ld;
        }
        for (int t0 = 0; t0 < g0; t0 += PF) {
          float2 lv[RR][PF];
#pragma unroll
          for (int u = 0; u < PF; ++u)
#pragma unroll
            for (int q = 0; q < RR; ++q)
              if (t0 + u < g0) lv[q][u] = __ldcg(Lp[q] + (size_t)(t0 + u) * ld);
#pragma unroll
          for (int u = 0; u < PF; ++u)
            if (t0 + u < g0)
#pragma unroll
              for (int c = 0; c < GW; ++c)
                if (c < gw) {
                  const float2 gv = G[c * R + t0 + u];
#pragma unroll
                  for (int q = 0; q < RR; ++q) cfma<float>(acc[q][c], lv[q][u], gv);
                }
        }
#pragma unroll
        for (int q = 0; q < RR; ++q) {
          const int rq = r + q * NT;
          if (rq < R)
#pragma unroll
            for (int c = 0; c < GW; ++c)
              if (c < gw) G[c * R + rq] = csub<float>(G[c * R + rq], acc[q][c]);
        }
      }
      __syncthreads();
    }
    // factor the group's columns
    for (int c = 0; c < gw; ++c) {
      const int col = g0 + c;
      float2* Gc = G + c * R;
      float best = -1.f;
      int bi = R;
      for (int r = col + tid; r < R; r += NT) {
        const float v = cabs1<float>(Gc[r]);
        if (v > best) { best = v; bi = r; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float v2 = __shfl_down_sync(0xffffffffu, best, off);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, off);
        if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
      }
      if (lane == 0) { sh.wv[warp] = best; sh.wi[warp] = bi; }
      __syncthreads();
      if (tid == 0) {
        float b = sh.wv[0];
        int p = sh.wi[0];
        for (int k = 1; k < NT / 32; ++k)
          if (sh.wv[k] > b || (sh.wv[k] == b && sh.wi[k] < p)) { b = sh.wv[k]; p = sh.wi[k]; }
        if (p >= R) {  // the column held only NaN: keep the diagonal, flag it
          p = col;
          atomicOr(flags, (unsigned)DEVFLAG_NONFINITE);
        }
        sh.piv = p;
        piv[col] = r0 + p;
      }
      __syncthreads();
      const int p = sh.piv;
      if (p != col) {
        if (tid < gw) {
          const float2 t0 = G[tid * R + col];
          G[tid * R + col] = G[tid * R + p];
          G[tid * R + p] = t0;
        }
        if (tid == 0) {
          const int t1 = pl[col];
          pl[col] = pl[p];
          pl[p] = t1;
        }
        __syncthreads();
      }
      const float2 d = Gc[col];
      if (d.x == 0.f && d.y == 0.f) {
        if (tid == 0) {
          atomicCAS(info, 0, r0 + col + 1);
          atomicOr(flags, (unsigned)DEVFLAG_SINGULAR);
        }
      } else {
        const float2 inv = crecip<float>(d);
        for (int r = col + 1 + tid; r < R; r += NT) {
          const float2 l = cmul<float>(Gc[r], inv);
          Gc[r] = l;
#pragma unroll
          for (int c2 = 1; c2 < GW; ++c2)
            if (c + c2 < gw) G[(c + c2) * R + r] = csub<float>(G[(c + c2) * R + r], cmul<float>(l, G[(c + c2) * R + col]));
        }
      }
      __syncthreads();
    }
    for (int idx = tid; idx < R * gw; idx += NT) {
      const int c = idx / R, r = idx - c * R;
      A[(size_t)(r0 + pl[r]) + (size_t)(r0 + g0 + c) * ld] = G[idx];
    }
    __syncthreads();
  }
  // moved rows: logical row dst takes physical row src
  if (tid == 0) sh.cnt = 0;
  __syncthreads();
  for (int r = tid; r < R; r += NT)
    if (pl[r] != r) {
      const int e = atomicAdd(&sh.cnt, 1);
      if (e < 128) { sh.mvd[e] = r; sh.mvs[e] = pl[r]; }
    }
  __syncthreads();
  if (sh.cnt > 128) {  // cannot happen: w <= 64 interchanges move at most 128 rows
    if (tid == 0) {
      atomicOr(flags, (unsigned)DEVFLAG_BADARG);
      sh.cnt = 128;
    }
    __syncthreads();
  }
  const int cnt = sh.cnt;
  // the panel's own columns in logical order, 32 columns at a time through Lt
  for (int c0 = 0; c0 < w; c0 += 32) {
    const int cw = min(32, w - c0);
    for (int idx = tid; idx < cnt * cw; idx += NT) {
      const int e = idx % cnt, c = idx / cnt;
      Lt[idx] = __ldcg(A + (size_t)(r0 + sh.mvs[e]) + (size_t)(r0 + c0 + c) * ld);
    }
    __syncthreads();
    for (int idx = tid; idx < cnt * cw; idx += NT) {
      const int e = idx % cnt, c = idx / cnt;
      A[(size_t)(r0 + sh.mvd[e]) + (size_t)(r0 + c0 + c) * ld] = Lt[idx];
    }
    __syncthreads();
  }
}
