// Complex64 panel factorisation with partial pivoting spread over a
// thread-block cluster: PC_C CTAs per shifted matrix, each owning a
// contiguous range of the panel's logical rows.
//
// The single-CTA panel (panel_ll.cuh) keeps one SM busy per shift and leaves
// the rest of the GPU idle while the factorisation waits for it; with q = 32
// shifts and 152 SMs, four CTAs per shift fit at once.  The algorithm is the
// same left-looking group form (partial pivoting on the largest |Re| + |Im|,
// lowest row on ties, rows tracked by a logical-to-physical map and moved only
// at the end), with the work split by rows:
//   * every CTA brings its rows of the group's columns up to date with the
//     panel's earlier columns (L from global memory, U of the top rows from
//     CTA 0's shared memory);
//   * per column, each CTA finds the largest entry among its rows and posts it
//     with the row's group entries (CTA 0 also posts the entries at the pivot
//     position); after one cluster barrier every CTA reads the posted
//     candidates from distributed shared memory, takes the same decision, and
//     copies the pivot row (and, in the two CTAs involved, the row it
//     replaces) before writing the interchange locally.  The posts are
//     double-buffered by the parity of the column, so a CTA that runs ahead
//     never overwrites what another CTA may still be reading.  Each CTA then
//     applies the rank-1 update to its own rows with its copy of the pivot row.
// CTA 0 owns logical rows 0 .. 63 (every pivot position), so each interchange
// involves CTA 0 and the owner of the pivot row.  Every CTA runs the same
// sequence of cluster barriers (no CTA leaves a loop early), so no barrier can
// be left waiting.
#include <cooperative_groups.h>

#include "common.cuh"
#include "lu.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int PC_C = 4;          // CTAs per shift
constexpr int PC_NT = 512;       // threads per CTA
constexpr int PC_MAXW = 64;      // panel width

struct PcShared {
  float best[PC_NT / 32];
  int bidx[PC_NT / 32];
  // posted for the other CTAs, double-buffered by the parity of the column:
  // this CTA's pivot candidate with its group entries and physical row, and
  // (CTA 0) the entries and physical row of the pivot position itself
  float cand_v[2];
  int cand_i[2];
  float2 cand_row[2][16];
  int cand_pl[2];
  float2 col_row[2][16];
  int col_pl[2];
  int piv, owner;
  int cnt;                       // moved rows of this CTA
  int mvd[128], mvs[128];
  float2 u[16];                  // the pivot row's group entries (local copy)
  float2 oldrow[16];             // the replaced row's entries (owner of the pivot row only)
  int pl_p, pl_col;
};

__device__ __forceinline__ bool better(float v2, int i2, float v, int i) { return v2 > v || (v2 == v && i2 < i); }

// Shared memory: G[GW][chunk] float2 (the group's columns of this CTA's rows),
// pl[chunk] int (logical -> physical row), Lt[64][64] float2 (CTA 0: the top
// rows of the earlier columns), Ut[64][GW] float2 (U of the top rows).
template <int GW>
__global__ void __launch_bounds__(PC_NT, 1)
k_panel_cluster(float2* S, long long ld, long long stride, int n, int r0, int w, int32_t* piv, int* info,
                unsigned* flags, int32_t* mv, int chunk) {
  extern __shared__ __align__(16) unsigned char pc_smem[];
  __shared__ PcShared sh;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int b = blockIdx.x / PC_C;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float2* A = S + (size_t)b * stride;
  int32_t* pv = piv + (size_t)b * n + r0;
  const int R = n - r0;
  const int lo = rank * chunk;
  const int rows = max(0, min(chunk, R - lo));  // this CTA's logical rows lo .. lo+rows-1
  float2* G = reinterpret_cast<float2*>(pc_smem);
  int* pl = reinterpret_cast<int*>(G + (size_t)GW * chunk);
  float2* Lt = reinterpret_cast<float2*>(pl + chunk + (chunk & 1));
  float2* Ut = Lt + 64 * 64;
  for (int r = tid; r < rows; r += PC_NT) pl[r] = lo + r;
  if (tid == 0) sh.cnt = 0;
  cluster.sync();
  for (int g0 = 0; g0 < w; g0 += GW) {
    const int gw = min(GW, w - g0);
    // 1. this CTA's rows of the group's columns
    for (int base = 0; base < rows * gw; base += 8 * PC_NT) {
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * PC_NT + tid;
        if (idx < rows * gw) {
          const int c = idx / rows, r = idx - c * rows;
          v[u] = __ldcg(A + (size_t)(r0 + pl[r]) + (size_t)(r0 + g0 + c) * ld);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * PC_NT + tid;
        if (idx < rows * gw) {
          const int c = idx / rows, r = idx - c * rows;
          G[c * chunk + r] = v[u];
        }
      }
    }
    __syncthreads();
    if (g0 > 0) {
      // 2a. CTA 0: the top rows of the earlier columns, then the forward
      // substitution of the group's top g0 rows (one warp per column)
      if (rank == 0) {
        for (int idx = tid; idx < 64 * g0; idx += PC_NT) {
          const int t = idx >> 6, r = idx & 63;
          if (r < rows) Lt[idx] = __ldcg(A + (size_t)(r0 + pl[r]) + (size_t)(r0 + t) * ld);
        }
        __syncthreads();
        if (warp < gw) {
          float2* Gc = G + warp * chunk;
          float2 x0 = lane < g0 ? Gc[lane] : make_float2(0.f, 0.f);
          float2 x1 = lane + 32 < g0 ? Gc[lane + 32] : make_float2(0.f, 0.f);
          for (int t = 0; t < g0 - 1; ++t) {
            const float2 xv = t < 32 ? x0 : x1;
            const float2 xt = make_float2(__shfl_sync(0xffffffffu, xv.x, t & 31), __shfl_sync(0xffffffffu, xv.y, t & 31));
            const float2 l0 = Lt[t * 64 + lane], l1 = Lt[t * 64 + lane + 32];
            if (lane > t && lane < g0) x0 = csub<float>(x0, cmul<float>(l0, xt));
            if (lane + 32 > t && lane + 32 < g0) x1 = csub<float>(x1, cmul<float>(l1, xt));
          }
          if (lane < g0) Gc[lane] = x0;
          if (lane + 32 < g0) Gc[lane + 32] = x1;
        }
      }
      cluster.sync();  // [S1] U of the top rows is ready in CTA 0
      // 2b. every CTA copies U[0:g0, group] from CTA 0
      {
        const float2* G0 = cluster.map_shared_rank(G, 0);
        for (int idx = tid; idx < g0 * gw; idx += PC_NT) {
          const int t = idx % g0, c = idx / g0;
          Ut[t * GW + c] = G0[c * chunk + t];
        }
      }
      __syncthreads();
      // 2c. G[r, c] -= sum_{t < g0} L[r, t] U[t, c] for this CTA's rows below g0
      constexpr int PF = 8;
      const int rstart = rank == 0 ? g0 : 0;
      for (int r = rstart + tid; r < rows; r += PC_NT) {
        float2 acc[GW];
#pragma unroll
        for (int c = 0; c < GW; ++c) acc[c] = make_float2(0.f, 0.f);
        const float2* Lp = A + (size_t)(r0 + pl[r]) + (size_t)r0 * ld;
        for (int t0 = 0; t0 < g0; t0 += PF) {
          float2 lv[PF];
#pragma unroll
          for (int u = 0; u < PF; ++u)
            if (t0 + u < g0) lv[u] = __ldcg(Lp + (size_t)(t0 + u) * ld);
#pragma unroll
          for (int u = 0; u < PF; ++u)
            if (t0 + u < g0)
#pragma unroll
              for (int c = 0; c < GW; ++c)
                if (c < gw) cfma<float>(acc[c], lv[u], Ut[(t0 + u) * GW + c]);
        }
#pragma unroll
        for (int c = 0; c < GW; ++c)
          if (c < gw) G[c * chunk + r] = csub<float>(G[c * chunk + r], acc[c]);
      }
      __syncthreads();
    }
    // 3. factor the group's columns
    for (int c = 0; c < gw; ++c) {
      const int col = g0 + c;  // logical pivot position (owned by CTA 0)
      float2* Gc = G + c * chunk;
      float best = -1.f;
      int bi = R;
      for (int r = tid; r < rows; r += PC_NT) {
        const int lr = lo + r;
        if (lr >= col) {
          const float v = cabs1<float>(Gc[r]);
          if (v > best) { best = v; bi = lr; }
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float v2 = __shfl_down_sync(0xffffffffu, best, off);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, off);
        if (better(v2, i2, best, bi)) { best = v2; bi = i2; }
      }
      if (lane == 0) { sh.best[warp] = best; sh.bidx[warp] = bi; }
      __syncthreads();
      const int slot = col & 1;
      if (warp == 0) {
        // this CTA's candidate (a shuffle over the warps' results), posted with
        // its group entries; CTA 0 also posts the entries at the pivot position
        float v = lane < PC_NT / 32 ? sh.best[lane] : -1.f;
        int ii = lane < PC_NT / 32 ? sh.bidx[lane] : R;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const float v2 = __shfl_down_sync(0xffffffffu, v, off);
          const int i2 = __shfl_down_sync(0xffffffffu, ii, off);
          if (better(v2, i2, v, ii)) { v = v2; ii = i2; }
        }
        ii = __shfl_sync(0xffffffffu, ii, 0);
        if (lane == 0) {
          sh.cand_v[slot] = v;
          sh.cand_i[slot] = ii;
          sh.cand_pl[slot] = ii < R ? pl[ii - lo] : 0;
          if (rank == 0) sh.col_pl[slot] = pl[col];
        }
        if (lane < gw) {
          sh.cand_row[slot][lane] = ii < R ? G[lane * chunk + (ii - lo)] : make_float2(0.f, 0.f);
          if (rank == 0) sh.col_row[slot][lane] = G[lane * chunk + col];
        }
      }
      cluster.sync();  // [P1] every CTA's candidate (and CTA 0's pivot position) is posted
      if (warp == 0) {
        // the same decision in every CTA: lane k reads CTA k's candidate
        float v = -1.f;
        int ii = R, ow = 0;
        if (lane < PC_C) {
          const PcShared* o = cluster.map_shared_rank(&sh, lane);
          v = o->cand_v[slot];
          ii = o->cand_i[slot];
          ow = lane;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const float v2 = __shfl_down_sync(0xffffffffu, v, off);
          const int i2 = __shfl_down_sync(0xffffffffu, ii, off);
          const int o2 = __shfl_down_sync(0xffffffffu, ow, off);
          if (better(v2, i2, v, ii)) { v = v2; ii = i2; ow = o2; }
        }
        ii = __shfl_sync(0xffffffffu, ii, 0);
        ow = __shfl_sync(0xffffffffu, ow, 0);
        if (ii >= R) {  // the column held only NaN: keep the diagonal, flag it
          ii = col;
          ow = 0;
          if (rank == 0 && lane == 0) atomicOr(flags, (unsigned)DEVFLAG_NONFINITE);
        }
        const PcShared* po = cluster.map_shared_rank(&sh, ow);
        const PcShared* p0 = cluster.map_shared_rank(&sh, 0);
        if (ii == col) {
          if (lane < gw) sh.u[lane] = p0->col_row[slot][lane];
        } else {
          float2 u = make_float2(0.f, 0.f), old = make_float2(0.f, 0.f);
          if (lane < gw) {
            u = po->cand_row[slot][lane];
            if (rank == ow) old = p0->col_row[slot][lane];
          }
          const int plp = lane == 0 ? po->cand_pl[slot] : 0;
          const int plc = (lane == 0 && rank == ow) ? p0->col_pl[slot] : 0;
          if (lane < gw) {
            sh.u[lane] = u;
            if (rank == 0) G[lane * chunk + col] = u;
            if (rank == ow) G[lane * chunk + (ii - ow * chunk)] = old;
          }
          if (lane == 0) {
            if (rank == 0) pl[col] = plp;
            if (rank == ow) pl[ii - ow * chunk] = plc;
          }
        }
        if (lane == 0) sh.piv = ii;
      }
      __syncthreads();  // the interchange and the pivot row are in place
      const int p = sh.piv;
      if (rank == 0 && tid == 0) pv[col] = r0 + p;
      const float2 d = sh.u[c];
      if (d.x == 0.f && d.y == 0.f) {
        if (rank == 0 && tid == 0) {
          atomicCAS(info + b, 0, r0 + col + 1);
          atomicOr(flags, (unsigned)DEVFLAG_SINGULAR);
        }
      } else {
        const float2 inv = crecip<float>(d);
        for (int r = tid; r < rows; r += PC_NT) {
          if (lo + r <= col) continue;
          const float2 l = cmul<float>(Gc[r], inv);
          Gc[r] = l;
#pragma unroll
          for (int c2 = 1; c2 < GW; ++c2)
            if (c + c2 < gw) G[(c + c2) * chunk + r] = csub<float>(G[(c + c2) * chunk + r], cmul<float>(l, sh.u[c + c2]));
        }
      }
      // each thread's next pivot search reads only the rows it has just
      // updated; the next barrier (after the search) orders the rest
    }
    __syncthreads();
    // 4. the group's columns back to their physical rows
    for (int idx = tid; idx < rows * gw; idx += PC_NT) {
      const int c = idx / rows, r = idx - c * rows;
      A[(size_t)(r0 + pl[r]) + (size_t)(r0 + g0 + c) * ld] = G[c * chunk + r];
    }
    __threadfence();
    cluster.sync();  // [S2] the next group reads these columns (any CTA's rows through L) and CTA 0's G
  }
  // 5. moved rows: logical row d took physical row s (relative to r0)
  for (int r = tid; r < rows; r += PC_NT)
    if (pl[r] != lo + r) {
      const int e = atomicAdd(&sh.cnt, 1);
      if (e < 128) { sh.mvd[e] = lo + r; sh.mvs[e] = pl[r]; }
    }
  __threadfence();
  cluster.sync();  // [E1] every CTA's list and every global write of the panel are done
  if (rank == 0) {
    int* tot = reinterpret_cast<int*>(Ut);  // gathered list: count, dst[128], src[128]
    if (tid == 0) {
      int cnt = 0;
      for (int k = 0; k < PC_C; ++k) {
        const PcShared* o = cluster.map_shared_rank(&sh, k);
        const int ck = min(o->cnt, 128);
        for (int e = 0; e < ck && cnt < 128; ++e, ++cnt) {
          tot[1 + cnt] = o->mvd[e];
          tot[129 + cnt] = o->mvs[e];
        }
        if (o->cnt > 128) atomicOr(flags, (unsigned)DEVFLAG_BADARG);
      }
      tot[0] = cnt;
    }
    __syncthreads();
    const int cnt = tot[0];
    // the panel's own columns in logical order, 32 columns at a time through Lt
    for (int c0 = 0; c0 < w; c0 += 32) {
      const int cw = min(32, w - c0);
      for (int idx = tid; idx < cnt * cw; idx += PC_NT) {
        const int e = idx % cnt, c = idx / cnt;
        Lt[idx] = __ldcg(A + (size_t)(r0 + tot[129 + e]) + (size_t)(r0 + c0 + c) * ld);
      }
      __syncthreads();
      for (int idx = tid; idx < cnt * cw; idx += PC_NT) {
        const int e = idx % cnt, c = idx / cnt;
        A[(size_t)(r0 + tot[1 + e]) + (size_t)(r0 + c0 + c) * ld] = Lt[idx];
      }
      __syncthreads();
    }
    if (mv) {
      int32_t* o = mv + (size_t)b * LU_MV_STRIDE;
      if (tid == 0) o[0] = cnt;
      for (int e = tid; e < cnt; e += PC_NT) {
        o[1 + e] = tot[1 + e];
        o[129 + e] = tot[129 + e];
      }
    }
  }
  cluster.sync();  // [E2] no CTA leaves while CTA 0 still reads the others' lists
}

template <int GW>
size_t pc_smem(int chunk) {
  return (size_t)GW * chunk * sizeof(float2) + (size_t)(chunk + (chunk & 1)) * sizeof(int) +
         (size_t)64 * 64 * sizeof(float2) + (size_t)64 * GW * sizeof(float2);
}

template <int GW>
cudaError_t launch_pc(const LuBatch<float>& lu, int k0, int w, int chunk, int32_t* mvk, cudaStream_t s) {
  const size_t smem = pc_smem<GW>(chunk);
  cudaError_t e = cudaFuncSetAttribute(k_panel_cluster<GW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(lu.q * PC_C);
  cfg.blockDim = dim3(PC_NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = PC_C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  feast_count_launch();
  return cudaLaunchKernelEx(&cfg, k_panel_cluster<GW>, reinterpret_cast<float2*>(lu.S), lu.ld, lu.stride, lu.n, k0, w,
                            lu.piv, lu.info, lu.flags, mvk, chunk);
}

}  // namespace

// The cluster panel applies to panels of min_rows (default 1024, at least 256)
// to 8192 rows: below that the per-column cluster barrier costs more than the
// split saves, above it a CTA's rows of an eight-column group no longer fit in
// shared memory.
bool panel_cluster_applies(int rows, int w, int min_rows) {
  return rows >= (min_rows > 0 ? min_rows : 1024) && rows >= 256 && rows <= 8192 && w <= PC_MAXW;
}

cudaError_t panel_cluster(const LuBatch<float>& lu, int k0, int w, cudaStream_t s) {
  const int R = lu.n - k0;
  if (!panel_cluster_applies(R, w, lu.cluster_min_rows)) return cudaErrorInvalidValue;
  const int chunk = ((R + PC_C - 1) / PC_C + 1) & ~1;
  int32_t* mvk = lu.mv ? lu.mv + (size_t)(k0 / 64) * lu.q * LU_MV_STRIDE : nullptr;
  if (chunk * 16 <= 16384) return launch_pc<16>(lu, k0, w, chunk, mvk, s);
  return launch_pc<8>(lu, k0, w, chunk, mvk, s);
}
