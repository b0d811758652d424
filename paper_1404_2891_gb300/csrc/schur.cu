// The dense m0 x m0 eigenproblem of the Rayleigh-Ritz step (Algorithm
// R-FEAST step 5, Algorithm Bi-FEAST step 7).
//
// Scalar FP64 issues at about 1/64 of the FP32 rate on GB300, and the
// Hessenberg QR iteration is a long chain of dependent scalar work (one Givens
// rotation after another).  So the Schur form is computed in FP32 (one block,
// the whole matrix in shared memory, the sweeps run by one warp, the rotations
// logged and applied to Z by a second kernel), and FP64 accuracy is recovered
// afterwards by refinement sweeps built from FP64 tensor-core products
// (eig_refine_step; see feast.cu).  Instantiated for double (the matrix then
// packed, column j holding rows 0 .. j+2) the kernels give a plain FP64 Schur
// form.
#include <float.h>

#include <type_traits>

#include "small.cuh"

namespace {

template <typename T> struct Lim;
template <> struct Lim<float> {
  static constexpr float ulp = FLT_EPSILON * 0.5f;
  static constexpr float safe_min = FLT_MIN;
  static constexpr float big = 1e30f;
  static constexpr float tiny_scale = 1e-30f;
};
template <> struct Lim<double> {
  static constexpr double ulp = DBL_EPSILON * 0.5;
  static constexpr double safe_min = DBL_MIN;
  static constexpr double big = 1e150;
  static constexpr double tiny_scale = 1e-150;
};

constexpr int SCHUR_THREADS = 256;
constexpr int SCHUR_MAX_M = 160;

// One logged rotation (c, Re s, Im s, k) in the working precision.
template <typename T> struct RotRecT;
template <> struct RotRecT<float> { using type = float4; };
template <> struct RotRecT<double> { using type = double4; };
template <typename T> using RotRec = typename RotRecT<T>::type;
__device__ __forceinline__ float4 make_rec(float c, float2 s, int k) { return make_float4(c, s.x, s.y, (float)k); }
__device__ __forceinline__ double4 make_rec(double c, double2 s, int k) { return make_double4(c, s.x, s.y, (double)k); }

template <typename T>
__device__ T block_sum_t(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = T(0);
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
  return t;
}

template <typename T>
__device__ __forceinline__ cplx<T> csqrt_t(cplx<T> z) {
  const T r = hypot(z.x, z.y);
  if (r == T(0)) return mk<T>(T(0), T(0));
  const T re = sqrt(T(0.5) * (r + fabs(z.x)));
  const T other = z.y / (T(2) * re);
  if (z.x >= T(0)) return mk<T>(re, other);
  return mk<T>(fabs(other), z.y >= T(0) ? re : -re);
}

// packed storage: column j keeps rows 0 .. j+2 (Hessenberg plus the bulge diagonal)
__device__ __forceinline__ int hp_off(int i, int j) { return j * (j + 5) / 2 + i; }

// Givens rotation G = [c s; -conj(s) c] with G [x; y] = [r; 0], c real.
template <typename T>
__device__ void givens(cplx<T> x, cplx<T> y, T& c, cplx<T>& s) {
  const T ax = sqrt(cnorm2<T>(x)), ay = sqrt(cnorm2<T>(y));
  if (ay == T(0)) { c = T(1); s = mk<T>(T(0), T(0)); return; }
  if (ax == T(0)) { c = T(0); s = mk<T>(T(1), T(0)); return; }
  const T nu = sqrt(ax * ax + ay * ay);
  c = ax / nu;
  const cplx<T> ph = mk<T>(x.x / ax, x.y / ax);
  s = cscale<T>(cmul<T>(ph, cconj<T>(y)), T(1) / nu);
}

// The same rotation from the squares: c = |x|^2 / (|x| nu), s = x conj(y) / (|x| nu)
// with nu^2 = |x|^2 + |y|^2 (two square roots and one division, all correctly
// rounded); the scaled form above when a square nears the range limits.
template <typename T>
__device__ __forceinline__ void givens_sq(cplx<T> x, cplx<T> y, T& c, cplx<T>& s) {
  const T ax2 = cnorm2<T>(x), ay2 = cnorm2<T>(y);
  if (ay2 == T(0)) { c = T(1); s = mk<T>(T(0), T(0)); return; }
  if (ax2 == T(0)) { c = T(0); s = mk<T>(T(1), T(0)); return; }
  if (!(ax2 > Lim<T>::tiny_scale && ax2 < Lim<T>::big && ay2 < Lim<T>::big)) {
    givens<T>(x, y, c, s);
    return;
  }
  const T ax = sqrt(ax2), nu = sqrt(ax2 + ay2);
  const T inv = T(1) / (ax * nu);
  c = ax2 * inv;
  s = cscale<T>(cmul<T>(x, cconj<T>(y)), inv);
}

// Householder reduction to Hessenberg form (C, Z in global memory), then the
// shifted QR iteration by warp 0 on the packed shared-memory copy.  The
// rotations (c, Re s, Im s, k) go to rot_log; k_apply_rotations folds them into Z.
template <typename T>
__device__ __forceinline__ void small_schur_body(cplx<T>* C, cplx<T>* Z, cplx<T>* lam, int m, unsigned* flags,
                                                 RotRec<T>* rot_log, int rot_cap, int* rot_count) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* H = reinterpret_cast<cplx<T>*>(smem_raw);
  __shared__ cplx<T> s_u[SCHUR_MAX_M];
  __shared__ T red[SCHUR_THREADS / 32];
  __shared__ cplx<T> s_beta;
  __shared__ int s_skip;
  const int tid = threadIdx.x;
  auto Cg = [&](int i, int j) -> cplx<T>& { return C[i + (size_t)j * m]; };
  for (int idx = tid; idx < m * m; idx += SCHUR_THREADS)
    Z[idx] = mk<T>((idx % m) == (idx / m) ? T(1) : T(0), T(0));
  __syncthreads();
  // ---- Householder reduction to upper Hessenberg form, Z <- Z H_k
  for (int k = 0; k + 2 < m; ++k) {
    const int len = m - k - 1;
    T loc = T(0);
    for (int i = 1 + tid; i < len; i += SCHUR_THREADS) loc += cnorm2<T>(Cg(k + 1 + i, k));
    const T tail = block_sum_t<T>(loc, red);
    if (tid == 0) {
      const cplx<T> x0 = Cg(k + 1, k);
      const T a0 = hypot(x0.x, x0.y);
      s_skip = (tail == T(0));
      const T alpha = sqrt(tail + a0 * a0);
      const cplx<T> beta = a0 > T(0) ? mk<T>(-x0.x / a0 * alpha, -x0.y / a0 * alpha) : mk<T>(-alpha, T(0));
      s_beta = beta;
      s_u[0] = csub<T>(x0, beta);
    }
    __syncthreads();
    if (s_skip) { __syncthreads(); continue; }
    for (int i = 1 + tid; i < len; i += SCHUR_THREADS) s_u[i] = Cg(k + 1 + i, k);
    __syncthreads();
    T uu_loc = T(0);
    for (int i = tid; i < len; i += SCHUR_THREADS) uu_loc += cnorm2<T>(s_u[i]);
    const T uu = block_sum_t<T>(uu_loc, red);
    const T t = T(2) / uu;
    for (int c = k + tid; c < m; c += SCHUR_THREADS) {
      cplx<T> s = mk<T>(T(0), T(0));
      for (int i = 0; i < len; ++i) s = cadd<T>(s, cmulc<T>(s_u[i], Cg(k + 1 + i, c)));
      s = cscale<T>(s, t);
      for (int i = 0; i < len; ++i) Cg(k + 1 + i, c) = csub<T>(Cg(k + 1 + i, c), cmul<T>(s_u[i], s));
    }
    __syncthreads();
    for (int r = tid; r < 2 * m; r += SCHUR_THREADS) {
      cplx<T>* P = r < m ? C : Z;
      const int rr = r < m ? r : r - m;
      cplx<T> s = mk<T>(T(0), T(0));
      for (int i = 0; i < len; ++i) s = cadd<T>(s, cmul<T>(P[rr + (size_t)(k + 1 + i) * m], s_u[i]));
      s = cscale<T>(s, t);
      for (int i = 0; i < len; ++i) {
        cplx<T>& e = P[rr + (size_t)(k + 1 + i) * m];
        e = csub<T>(e, cmul<T>(s, cconj<T>(s_u[i])));
      }
    }
    __syncthreads();
    if (tid == 0) Cg(k + 1, k) = s_beta;
    for (int i = 1 + tid; i < len; i += SCHUR_THREADS) Cg(k + 1 + i, k) = mk<T>(T(0), T(0));
    __syncthreads();
  }
  for (int j = 0; j < m; ++j)
    for (int i = tid; i <= j + 2; i += SCHUR_THREADS)
      H[hp_off(i, j)] = (i < m && i <= j + 1) ? Cg(i, j) : mk<T>(T(0), T(0));
  __syncthreads();
  // ---- shifted QR iterations (warp 0)
  if (tid < 32) {
    const int lane = tid;
    int ihi = m - 1, its = 0, total = 0, nrot = 0;
    const int max_total = 30 * m + 100;
    while (ihi >= 0) {
      int l = 0;
      if (lane == 0) {
        for (int k = ihi; k >= 1; --k) {
          T tst = cabs1<T>(H[hp_off(k - 1, k - 1)]) + cabs1<T>(H[hp_off(k, k)]);
          if (tst == T(0)) tst = T(1);
          if (cabs1<T>(H[hp_off(k, k - 1)]) <= fmax(Lim<T>::ulp * tst, Lim<T>::safe_min * (m / Lim<T>::ulp))) {
            H[hp_off(k, k - 1)] = mk<T>(T(0), T(0));
            l = k;
            break;
          }
        }
      }
      l = __shfl_sync(0xffffffffu, l, 0);
      __syncwarp();
      if (l == ihi) {
        if (lane == 0) lam[ihi] = H[hp_off(ihi, ihi)];
        --ihi;
        its = 0;
        __syncwarp();
        continue;
      }
      ++its;
      if (++total > max_total) {
        if (lane == 0) {
          atomicOr(flags, (unsigned)DEVFLAG_TIMEOUT);
          for (int i = 0; i <= ihi; ++i) lam[i] = H[hp_off(i, i)];
        }
        break;
      }
      for (int k = l; k < ihi; ++k) {
        T c = T(0);
        cplx<T> s = mk<T>(T(0), T(0));
        if (lane == 0) {
          cplx<T> x, y;
          if (k == l) {
            cplx<T> sh;
            const cplx<T> a = H[hp_off(ihi - 1, ihi - 1)], b = H[hp_off(ihi - 1, ihi)];
            const cplx<T> cc = H[hp_off(ihi, ihi - 1)], d = H[hp_off(ihi, ihi)];
            if (its % 10 == 0) {
              sh = mk<T>(d.x + T(0.75) * fabs(cc.x), d.y);
            } else {
              const cplx<T> p = cscale<T>(csub<T>(a, d), T(0.5));
              const cplx<T> bc = cmul<T>(b, cc);
              const cplx<T> disc = csqrt_t<T>(cadd<T>(cmul<T>(p, p), bc));
              const cplx<T> d1 = cadd<T>(p, disc), d2 = csub<T>(p, disc);
              const cplx<T> den = cabs1<T>(d1) >= cabs1<T>(d2) ? d1 : d2;
              sh = (den.x == T(0) && den.y == T(0)) ? d : csub<T>(d, cdiv<T>(bc, den));
            }
            x = csub<T>(H[hp_off(l, l)], sh);
            y = H[hp_off(l + 1, l)];
          } else {
            x = H[hp_off(k, k - 1)];
            y = H[hp_off(k + 1, k - 1)];
          }
          givens<T>(x, y, c, s);
          if (nrot < rot_cap) rot_log[nrot] = make_rec(c, s, k);
        }
        ++nrot;
        c = __shfl_sync(0xffffffffu, c, 0);
        s.x = __shfl_sync(0xffffffffu, s.x, 0);
        s.y = __shfl_sync(0xffffffffu, s.y, 0);
        const cplx<T> ms = mk<T>(-s.x, s.y);  // -conj(s)
        const int j0 = (k == l) ? l : k - 1;
        for (int j = j0 + lane; j < m; j += 32) {
          const cplx<T> a = H[hp_off(k, j)], b = H[hp_off(k + 1, j)];
          H[hp_off(k, j)] = cadd<T>(cscale<T>(a, c), cmul<T>(s, b));
          H[hp_off(k + 1, j)] = cadd<T>(cmul<T>(ms, a), cscale<T>(b, c));
        }
        __syncwarp();
        const int imax = min(k + 2, ihi);
        const cplx<T> sc = cconj<T>(s), nsv = mk<T>(-s.x, -s.y);
        for (int i = lane; i <= imax; i += 32) {
          const cplx<T> a = H[hp_off(i, k)], b = H[hp_off(i, k + 1)];
          H[hp_off(i, k)] = cadd<T>(cscale<T>(a, c), cmul<T>(b, sc));
          H[hp_off(i, k + 1)] = cadd<T>(cmul<T>(a, nsv), cscale<T>(b, c));
        }
        __syncwarp();
        if (k > l && lane == 0) H[hp_off(k + 1, k - 1)] = mk<T>(T(0), T(0));
        __syncwarp();
      }
    }
    if (lane == 0) {
      if (nrot > rot_cap) atomicOr(flags, (unsigned)DEVFLAG_TIMEOUT);
      *rot_count = nrot < rot_cap ? nrot : rot_cap;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < m * m; idx += SCHUR_THREADS) {
    const int i = idx % m, j = idx / m;
    C[idx] = (i <= j) ? H[hp_off(i, j)] : mk<T>(T(0), T(0));
  }
}

// The Schur form with the whole matrix in shared memory (full storage, ld m + 1):
// the Householder reduction by all warps on the shared copy (Z accumulated in
// global memory, one row per thread, coalesced), then the shifted QR sweeps by
// warp 0 with every lane forming each rotation itself (no broadcasts), a
// warp-parallel deflation search and the row / column updates unrolled over at
// most five elements per lane.  Rotations are logged as (c, Re s, Im s, k) for
// apply_rotations.  Used for FP32 (m <= 160 fits in shared memory).
template <typename T>
__device__ __forceinline__ void schur_full_body(cplx<T>* C, cplx<T>* Z, cplx<T>* lam, int m, unsigned* flags,
                                                RotRec<T>* rot_log, int rot_cap, int* rot_count) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* H = reinterpret_cast<cplx<T>*>(smem_raw);
  __shared__ cplx<T> s_u[SCHUR_MAX_M];
  __shared__ T red[SCHUR_THREADS / 32];
  __shared__ cplx<T> s_beta;
  __shared__ T s_t;
  __shared__ int s_skip;
  const int tid = threadIdx.x;
  const int ld = m + 1;
  auto h = [&](int i, int j) -> cplx<T>& { return H[i + j * ld]; };
  for (int idx = tid; idx < m * m; idx += SCHUR_THREADS) {
    const int i = idx % m, j = idx / m;
    h(i, j) = C[idx];
    Z[idx] = mk<T>(i == j ? T(1) : T(0), T(0));
  }
  __syncthreads();
  // ---- Householder reduction: H_k = I - t u u^H zeroes column k below row k + 1
  for (int k = 0; k + 2 < m; ++k) {
    const int len = m - k - 1;
    T loc = T(0);
    for (int i = 1 + tid; i < len; i += SCHUR_THREADS) loc += cnorm2<T>(h(k + 1 + i, k));
    const T tail = block_sum_t<T>(loc, red);
    if (tid == 0) {
      const cplx<T> x0 = h(k + 1, k);
      const T a0 = hypot(x0.x, x0.y);
      s_skip = (tail == T(0));
      const T alpha = sqrt(tail + a0 * a0);
      const cplx<T> beta = a0 > T(0) ? mk<T>(-x0.x / a0 * alpha, -x0.y / a0 * alpha) : mk<T>(-alpha, T(0));
      s_beta = beta;
      const cplx<T> u0 = csub<T>(x0, beta);
      s_u[0] = u0;
      s_t = T(2) / (cnorm2<T>(u0) + tail);
    }
    __syncthreads();
    if (s_skip) continue;  // read by all before thread 0 writes it again (block_sum_t synchronises)
    for (int i = 1 + tid; i < len; i += SCHUR_THREADS) s_u[i] = h(k + 1 + i, k);
    __syncthreads();
    const T tt = s_t;
    // left: H(k+1:m, c) -= u (t u^H H(k+1:m, c)) for c > k, two threads per column
    // (the trip count is the same for every thread, so whole warps meet the shuffle)
    for (int base = 0; base < 2 * (m - k - 1); base += SCHUR_THREADS) {
      const int p = base + tid;
      const bool on = p < 2 * (m - k - 1);
      const int c = k + 1 + (p >> 1), half = p & 1;
      cplx<T> s = mk<T>(T(0), T(0));
      if (on)
        for (int i = half; i < len; i += 2) cfmac<T>(s, s_u[i], h(k + 1 + i, c));
      s.x += __shfl_xor_sync(0xffffffffu, s.x, 1);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, 1);
      s = cscale<T>(s, tt);
      if (on)
        for (int i = half; i < len; i += 2) cfms<T>(h(k + 1 + i, c), s_u[i], s);
    }
    __syncthreads();
    // right: rows of H and of Z, (row)(k+1:m) -= ((row)(k+1:m) u) t u^H
    for (int r = tid; r < 2 * m; r += SCHUR_THREADS) {
      if (r < m) {
        cplx<T> s = mk<T>(T(0), T(0));
        for (int i = 0; i < len; ++i) cfma<T>(s, h(r, k + 1 + i), s_u[i]);
        s = cscale<T>(s, tt);
        for (int i = 0; i < len; ++i) cfms<T>(h(r, k + 1 + i), s, cconj<T>(s_u[i]));
      } else {
        cplx<T>* zr = Z + (r - m);
        cplx<T> s = mk<T>(T(0), T(0));
        for (int i = 0; i < len; ++i) cfma<T>(s, zr[(size_t)(k + 1 + i) * m], s_u[i]);
        s = cscale<T>(s, tt);
        for (int i = 0; i < len; ++i) cfms<T>(zr[(size_t)(k + 1 + i) * m], s, cconj<T>(s_u[i]));
      }
    }
    __syncthreads();
    if (tid == 0) h(k + 1, k) = s_beta;
    for (int i = 1 + tid; i < len; i += SCHUR_THREADS) h(k + 1 + i, k) = mk<T>(T(0), T(0));
    __syncthreads();
  }
  // ---- shifted QR sweeps (warp 0)
  if (tid < 32) {
    const int lane = tid;
    int ihi = m - 1, its = 0, total = 0, nrot = 0;
    const int max_total = 30 * m + 100;
    const T smlnum = Lim<T>::safe_min * (T(m) / Lim<T>::ulp);
    RotRec<T> rec;
    while (ihi >= 0) {
      // the largest k <= ihi with a negligible subdiagonal entry (l = 0: none)
      int l = 0;
      for (int base = ihi; base >= 1; base -= 32) {
        const int k = base - lane;
        bool neg = false;
        if (k >= 1) {
          T tst = cabs1<T>(h(k - 1, k - 1)) + cabs1<T>(h(k, k));
          if (tst == T(0)) tst = T(1);
          neg = cabs1<T>(h(k, k - 1)) <= fmax(Lim<T>::ulp * tst, smlnum);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, neg);
        if (bal) {
          l = base - (__ffs(bal) - 1);
          break;
        }
      }
      __syncwarp();
      if (l > 0 && lane == 0) h(l, l - 1) = mk<T>(T(0), T(0));
      __syncwarp();
      if (l == ihi) {
        if (lane == 0) lam[ihi] = h(ihi, ihi);
        --ihi;
        its = 0;
        continue;
      }
      ++its;
      if (++total > max_total) {
        if (lane == 0) {
          atomicOr(flags, (unsigned)DEVFLAG_TIMEOUT);
          for (int i = 0; i <= ihi; ++i) lam[i] = h(i, i);
        }
        break;
      }
      for (int k = l; k < ihi; ++k) {
        cplx<T> x, y;
        if (k == l) {
          cplx<T> sh;
          const cplx<T> a = h(ihi - 1, ihi - 1), b = h(ihi - 1, ihi);
          const cplx<T> cc = h(ihi, ihi - 1), d = h(ihi, ihi);
          if (its % 10 == 0) {
            sh = mk<T>(d.x + T(0.75) * fabs(cc.x), d.y);
          } else {
            const cplx<T> p = cscale<T>(csub<T>(a, d), T(0.5));
            const cplx<T> bc = cmul<T>(b, cc);
            const cplx<T> disc = csqrt_t<T>(cadd<T>(cmul<T>(p, p), bc));
            const cplx<T> d1 = cadd<T>(p, disc), d2 = csub<T>(p, disc);
            const cplx<T> den = cabs1<T>(d1) >= cabs1<T>(d2) ? d1 : d2;
            sh = (den.x == T(0) && den.y == T(0)) ? d : csub<T>(d, cdiv<T>(bc, den));
          }
          x = csub<T>(h(l, l), sh);
          y = h(l + 1, l);
        } else {
          x = h(k, k - 1);
          y = h(k + 1, k - 1);
        }
        T c;
        cplx<T> s;
        givens_sq<T>(x, y, c, s);
        // lane (nrot mod 32) keeps the record; every 32 rotations the warp stores them together
        if (lane == (nrot & 31)) rec = make_rec(c, s, k);
        if ((nrot & 31) == 31 && nrot - 31 + lane < rot_cap) rot_log[nrot - 31 + lane] = rec;
        ++nrot;
        const cplx<T> ms = mk<T>(-s.x, s.y);  // -conj(s)
        const int j0 = (k == l) ? l : k - 1;
        __syncwarp();  // every lane has read x, y before the rows change
        // all loads of a lane before its stores (the stores cannot alias the
        // later loads, but the compiler cannot tell)
        constexpr int NQ = (SCHUR_MAX_M + 31) / 32;
        cplx<T> ra[NQ], rb[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int j = j0 + lane + 32 * q;
          if (j < m) {
            ra[q] = h(k, j);
            rb[q] = h(k + 1, j);
          }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int j = j0 + lane + 32 * q;
          if (j < m) {
            h(k, j) = cadd<T>(cscale<T>(ra[q], c), cmul<T>(s, rb[q]));
            h(k + 1, j) = cadd<T>(cmul<T>(ms, ra[q]), cscale<T>(rb[q], c));
          }
        }
        __syncwarp();
        const int imax = min(k + 2, ihi);
        const cplx<T> sc = cconj<T>(s), nsv = mk<T>(-s.x, -s.y);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int i = lane + 32 * q;
          if (i <= imax) {
            ra[q] = h(i, k);
            rb[q] = h(i, k + 1);
          }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int i = lane + 32 * q;
          if (i <= imax) {
            h(i, k) = cadd<T>(cscale<T>(ra[q], c), cmul<T>(rb[q], sc));
            h(i, k + 1) = cadd<T>(cmul<T>(ra[q], nsv), cscale<T>(rb[q], c));
          }
        }
        if (k > l && lane == 0) h(k + 1, k - 1) = mk<T>(T(0), T(0));
        __syncwarp();
      }
    }
    {  // the records of the last, partial group of 32
      const int base = nrot & ~31;
      if (base + lane < nrot && base + lane < rot_cap) rot_log[base + lane] = rec;
    }
    if (lane == 0) {
      if (nrot > rot_cap) atomicOr(flags, (unsigned)DEVFLAG_TIMEOUT);
      *rot_count = nrot < rot_cap ? nrot : rot_cap;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < m * m; idx += SCHUR_THREADS) {
    const int i = idx % m, j = idx / m;
    C[idx] = (i <= j) ? h(i, j) : mk<T>(T(0), T(0));
  }
}

template <typename T>
__global__ void __launch_bounds__(SCHUR_THREADS)
k_small_schur(cplx<T>* C, cplx<T>* Z, cplx<T>* lam, int m, unsigned* flags, RotRec<T>* rot_log, int rot_cap,
              int* rot_count) {
  if constexpr (std::is_same<T, float>::value)
    schur_full_body<T>(C, Z, lam, m, flags, rot_log, rot_cap, rot_count);
  else
    small_schur_body<T>(C, Z, lam, m, flags, rot_log, rot_cap, rot_count);
}

__global__ void __launch_bounds__(SCHUR_THREADS)
k_small_schur_grp(float2* C, float2* Z, float2* lam, const GrpDesc* pd, const int* active, unsigned* flags,
                  char* logs) {
  const int p = blockIdx.x;
  if (!active[p]) return;
  const GrpDesc d = pd[p];
  char* log = logs + d.olog;
  schur_full_body<float>(C + d.omm, Z + d.omm, lam + d.om, d.m, flags, reinterpret_cast<float4*>(log + 256),
                         (30 * d.m + 100) * d.m, reinterpret_cast<int*>(log));
}

// Z <- Z G_1^H G_2^H ... for the logged rotations, in order.  One warp per block,
// one row of Z per lane, the rows held in shared memory (row-major, padded).
// Consecutive rotations of a sweep act on columns (k, k+1), (k+1, k+2), ...: the
// new column k+1 stays in a register for the next rotation.
template <typename T>
__device__ __forceinline__ void apply_rotations_body(cplx<T>* Z, int m, const RotRec<T>* rot_log, const int* rot_count,
                                                     int bx) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* rows = reinterpret_cast<cplx<T>*>(smem_raw);  // [32][m + 1]
  __shared__ RotRec<T> recs[32];
  const int lane = threadIdx.x;
  const int r = bx * 32 + lane;
  const int ld = m + 1;
  cplx<T>* row = rows + lane * ld;
  for (int j = 0; j < m; ++j) row[j] = r < m ? Z[r + (size_t)j * m] : mk<T>(T(0), T(0));
  const int nrot = *rot_count;
  cplx<T> carry = mk<T>(T(0), T(0));
  int ck = -1;  // the column of this row held in carry (-1: none)
  for (int base = 0; base < nrot; base += 32) {
    __syncwarp();
    if (base + lane < nrot) recs[lane] = rot_log[base + lane];
    __syncwarp();
    const int cnt = min(32, nrot - base);
    for (int q = 0; q < cnt; ++q) {
      const RotRec<T> g = recs[q];
      const int k = (int)g.w;
      const T c = (T)g.x;
      const cplx<T> sc = mk<T>((T)g.y, (T)-g.z), nsv = mk<T>((T)-g.y, (T)-g.z);
      cplx<T> a;
      if (k == ck) {
        a = carry;
      } else {
        if (ck >= 0) row[ck] = carry;
        a = row[k];
      }
      const cplx<T> b = row[k + 1];
      row[k] = cadd<T>(cscale<T>(a, c), cmul<T>(b, sc));
      carry = cadd<T>(cmul<T>(a, nsv), cscale<T>(b, c));
      ck = k + 1;
    }
  }
  if (ck >= 0) row[ck] = carry;
  if (r < m)
    for (int j = 0; j < m; ++j) Z[r + (size_t)j * m] = row[j];
}

template <typename T>
__global__ void __launch_bounds__(32) k_apply_rotations(cplx<T>* Z, int m, const RotRec<T>* rot_log, const int* rot_count) {
  apply_rotations_body<T>(Z, m, rot_log, rot_count, blockIdx.x);
}

__global__ void __launch_bounds__(32)
k_apply_rotations_grp(float2* Z, const GrpDesc* pd, const int* active, const char* logs) {
  const int p = blockIdx.y;
  if (!active[p] || (int)blockIdx.x * 32 >= pd[p].m) return;
  const GrpDesc d = pd[p];
  const char* log = logs + d.olog;
  apply_rotations_body<float>(Z + d.omm, d.m, reinterpret_cast<const float4*>(log + 256),
                              reinterpret_cast<const int*>(log), blockIdx.x);
}

// Eigenvectors of the upper triangular T by back substitution, one per thread.
template <typename T>
__device__ __forceinline__ void small_trevc_body(const cplx<T>* Tm, cplx<T>* V, int m) {
  __shared__ T red[32];
  const int k = threadIdx.x;
  T loc = T(0);
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    if (i <= j) loc = fmax(loc, cabs1<T>(Tm[idx]));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) loc = fmax(loc, __shfl_down_sync(0xffffffffu, loc, off));
  if (lane == 0) red[wid] = loc;
  __syncthreads();
  T tnorm = T(0);
  for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) tnorm = fmax(tnorm, red[w]);
  const T smin = fmax(Lim<T>::ulp * tnorm, Lim<T>::safe_min * (m / Lim<T>::ulp));
  if (k >= m) return;
  cplx<T>* v = V + (size_t)k * m;
  for (int i = k + 1; i < m; ++i) v[i] = mk<T>(T(0), T(0));
  v[k] = mk<T>(T(1), T(0));
  const cplx<T> lk = Tm[k + (size_t)k * m];
  for (int i = k - 1; i >= 0; --i) {
    cplx<T> s = mk<T>(T(0), T(0));
    for (int j = i + 1; j <= k; ++j) s = cadd<T>(s, cmul<T>(Tm[i + (size_t)j * m], v[j]));
    cplx<T> d = csub<T>(Tm[i + (size_t)i * m], lk);
    if (cabs1<T>(d) < smin) d = mk<T>(smin, T(0));
    const cplx<T> vi = cdiv<T>(s, d);
    v[i] = mk<T>(-vi.x, -vi.y);
    if (cabs1<T>(v[i]) > Lim<T>::big)  // keep the partial column representable
      for (int j = i; j <= k; ++j) v[j] = cscale<T>(v[j], Lim<T>::tiny_scale);
  }
}

template <typename T>
__global__ void k_small_trevc(const cplx<T>* Tm, cplx<T>* V, int m) {
  small_trevc_body<T>(Tm, V, m);
}

__global__ void k_small_trevc_grp(const float2* Tm, float2* V, const GrpDesc* pd, const int* active) {
  const int p = blockIdx.x;
  if (!active[p]) return;
  small_trevc_body<float>(Tm + pd[p].omm, V + pd[p].omm, pd[p].m);
}

// lam = diag(E); D = I + Delta, Delta_ij = E_ij / (E_jj - E_ii) for well-separated pairs.
__device__ __forceinline__ void refine_step_body(const double2* E, double2* D, double2* lam, int m) {
  __shared__ double red[32];
  double loc = 0.0;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) loc = fmax(loc, cabs1<double>(E[idx]));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) loc = fmax(loc, __shfl_down_sync(0xffffffffu, loc, off));
  if (lane == 0) red[wid] = loc;
  __syncthreads();
  double enorm = 0.0;
  for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) enorm = fmax(enorm, red[w]);
  const double gap_min = 1e-9 * enorm;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    if (i == j) {
      D[idx] = make_double2(1.0, 0.0);
      lam[i] = E[idx];
    } else {
      // first-order correction only where it is small: pairs inside a cluster
      // (|E_ij| comparable to the gap, e.g. a multiple eigenvalue) keep their
      // common invariant subspace as it is
      const double2 gap = csub<double>(E[j + (size_t)j * m], E[i + (size_t)i * m]);
      const bool sep = cabs1<double>(gap) > gap_min && cabs1<double>(gap) > 10.0 * cabs1<double>(E[idx]);
      D[idx] = sep ? cdiv<double>(E[idx], gap) : make_double2(0.0, 0.0);
    }
  }
}

__global__ void k_refine_step(const double2* E, double2* D, double2* lam, int m) { refine_step_body(E, D, lam, m); }

__global__ void k_refine_step_grp(const double2* E, double2* D, double2* lam, const GrpDesc* pd, const int* active) {
  const int p = blockIdx.x;
  if (!active[p]) return;
  const GrpDesc d = pd[p];
  refine_step_body(E + d.omm, D + d.omm, lam + d.om, d.m);
}

__global__ void k_to_c64(const double2* src, float2* dst, size_t count) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = make_float2((float)src[e].x, (float)src[e].y);
}

__global__ void k_to_c128(const float2* src, double2* dst, size_t count) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = make_double2(src[e].x, src[e].y);
}

unsigned grid1(size_t count) {
  size_t g = (count + 255) / 256;
  return (unsigned)(g < 1 ? 1 : (g > 1216 ? 1216 : g));
}

}  // namespace

size_t schur_log_bytes(int m) { return (size_t)(30 * m + 100) * (size_t)m * sizeof(double4) + 256; }

template <typename T>
cudaError_t small_schur(cplx<T>* C, cplx<T>* Z, cplx<T>* lam, int m, unsigned* flags, void* log, cudaStream_t s) {
  if (m < 1 || m > SCHUR_MAX_M) return cudaErrorInvalidValue;
  const bool full = std::is_same<T, float>::value;  // full storage (FP32) or packed (FP64)
  const size_t smem = full ? (size_t)m * (m + 1) * sizeof(cplx<T>) : (size_t)(m * (m + 5) / 2 + 8) * sizeof(cplx<T>);
  cudaError_t e = cudaFuncSetAttribute(k_small_schur<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int* count = reinterpret_cast<int*>(log);
  RotRec<T>* recs = reinterpret_cast<RotRec<T>*>(reinterpret_cast<char*>(log) + 256);
  const int cap = (30 * m + 100) * m;
  feast_count_launch();
  k_small_schur<T><<<1, SCHUR_THREADS, smem, s>>>(C, Z, lam, m, flags, recs, cap, count);
  const size_t smem2 = (size_t)32 * (m + 1) * sizeof(cplx<T>);
  e = cudaFuncSetAttribute(k_apply_rotations<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
  if (e != cudaSuccess) return e;
  feast_count_launch();
  k_apply_rotations<T><<<(m + 31) / 32, 32, smem2, s>>>(Z, m, recs, count);
  return cudaGetLastError();
}
template cudaError_t small_schur<float>(float2*, float2*, float2*, int, unsigned*, void*, cudaStream_t);
template cudaError_t small_schur<double>(double2*, double2*, double2*, int, unsigned*, void*, cudaStream_t);

template <typename T>
cudaError_t small_trevc(const cplx<T>* Tm, cplx<T>* V, int m, cudaStream_t s) {
  const int threads = ((m + 31) / 32) * 32;
  feast_count_launch();
  k_small_trevc<T><<<1, threads, 0, s>>>(Tm, V, m);
  return cudaGetLastError();
}
template cudaError_t small_trevc<float>(const float2*, float2*, int, cudaStream_t);
template cudaError_t small_trevc<double>(const double2*, double2*, int, cudaStream_t);

namespace {
// Inverse of an upper triangular m x m matrix, one column per thread (back
// substitution for V x = e_j); one block per matrix (grid y = problem index).
template <typename T>
__global__ void k_triu_inv(const cplx<T>* V, cplx<T>* Vi, int m, long long stride, const GrpDesc* pd,
                           const int* active) {
  int mm = m;
  size_t off = (size_t)blockIdx.y * stride;
  if (pd) {
    if (!active[blockIdx.y]) return;
    mm = pd[blockIdx.y].m;
    off = (size_t)pd[blockIdx.y].omm;
  }
  const cplx<T>* Vb = V + off;
  cplx<T>* X = Vi + off;
  for (int j = threadIdx.x; j < mm; j += blockDim.x) {
    cplx<T>* x = X + (size_t)j * mm;
    for (int i = j + 1; i < mm; ++i) x[i] = mk<T>(T(0), T(0));
    x[j] = crecip<T>(Vb[j + (size_t)j * mm]);
    for (int i = j - 1; i >= 0; --i) {
      cplx<T> acc = mk<T>(T(0), T(0));
      for (int k = i + 1; k <= j; ++k) acc = cadd<T>(acc, cmul<T>(Vb[i + (size_t)k * mm], x[k]));
      x[i] = cmul<T>(mk<T>(-acc.x, -acc.y), crecip<T>(Vb[i + (size_t)i * mm]));
    }
  }
}
}  // namespace

template <typename T>
cudaError_t small_triu_inv(const cplx<T>* V, cplx<T>* Vi, int m, cudaStream_t s) {
  feast_count_launch();
  k_triu_inv<T><<<1, ((m + 31) / 32) * 32, 0, s>>>(V, Vi, m, 0, nullptr, nullptr);
  return cudaGetLastError();
}
template cudaError_t small_triu_inv<float>(const float2*, float2*, int, cudaStream_t);

cudaError_t small_triu_inv_grp(const float2* V, float2* Vi, const GrpDesc* pd, int np, int mmax, const int* active,
                               cudaStream_t s) {
  if (np < 1) return cudaSuccess;
  feast_count_launch();
  k_triu_inv<float><<<dim3(1, np), ((mmax + 31) / 32) * 32, 0, s>>>(V, Vi, 0, 0, pd, active);
  return cudaGetLastError();
}

cudaError_t eig_refine_step(const double2* E, double2* D, double2* lam, int m, cudaStream_t s) {
  feast_count_launch();
  k_refine_step<<<1, 1024, 0, s>>>(E, D, lam, m);
  return cudaGetLastError();
}

cudaError_t to_c64(const double2* src, float2* dst, size_t count, cudaStream_t s) {
  feast_count_launch();
  k_to_c64<<<grid1(count), 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}

cudaError_t to_c128(const float2* src, double2* dst, size_t count, cudaStream_t s) {
  feast_count_launch();
  k_to_c128<<<grid1(count), 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- grouped forms
cudaError_t small_schur_grp(float2* C, float2* Z, float2* lam, const GrpDesc* pd, int np, int mmax,
                            const int* active, unsigned* flags, void* logs, cudaStream_t s) {
  if (np < 1) return cudaSuccess;
  if (mmax < 1 || mmax > SCHUR_MAX_M) return cudaErrorInvalidValue;
  const size_t smem = (size_t)mmax * (mmax + 1) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_small_schur_grp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  feast_count_launch();
  k_small_schur_grp<<<np, SCHUR_THREADS, smem, s>>>(C, Z, lam, pd, active, flags, reinterpret_cast<char*>(logs));
  const size_t smem2 = (size_t)32 * (mmax + 1) * sizeof(float2);
  e = cudaFuncSetAttribute(k_apply_rotations_grp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
  if (e != cudaSuccess) return e;
  feast_count_launch();
  k_apply_rotations_grp<<<dim3((mmax + 31) / 32, np), 32, smem2, s>>>(Z, pd, active, reinterpret_cast<const char*>(logs));
  return cudaGetLastError();
}

cudaError_t small_trevc_grp(const float2* Tm, float2* V, const GrpDesc* pd, int np, int mmax, const int* active,
                            cudaStream_t s) {
  if (np < 1) return cudaSuccess;
  feast_count_launch();
  k_small_trevc_grp<<<np, ((mmax + 31) / 32) * 32, 0, s>>>(Tm, V, pd, active);
  return cudaGetLastError();
}

cudaError_t eig_refine_step_grp(const double2* E, double2* D, double2* lam, const GrpDesc* pd, int np,
                                const int* active, cudaStream_t s) {
  if (np < 1) return cudaSuccess;
  feast_count_launch();
  k_refine_step_grp<<<np, 1024, 0, s>>>(E, D, lam, pd, active);
  return cudaGetLastError();
}
