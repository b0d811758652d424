// Shared device helpers: complex arithmetic on double2 / float2, the element
// type traits used by the templated kernels, and launch error plumbing.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#define FEAST_HD __host__ __device__ __forceinline__

template <typename T> struct ctype;
template <> struct ctype<double> { using type = double2; };
template <> struct ctype<float> { using type = float2; };
template <typename T> using cplx = typename ctype<T>::type;

template <typename T> FEAST_HD cplx<T> mk(T re, T im) { cplx<T> r; r.x = re; r.y = im; return r; }
template <typename T> FEAST_HD cplx<T> czero() { return mk<T>(T(0), T(0)); }
template <typename T> FEAST_HD cplx<T> cadd(cplx<T> a, cplx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> FEAST_HD cplx<T> csub(cplx<T> a, cplx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> FEAST_HD cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename T> FEAST_HD cplx<T> cmulc(cplx<T> a, cplx<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename T> FEAST_HD cplx<T> cconj(cplx<T> a) { return mk<T>(a.x, -a.y); }
template <typename T> FEAST_HD cplx<T> cscale(cplx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
template <typename T> FEAST_HD T cabs1(cplx<T> a) { return fabs(a.x) + fabs(a.y); }
template <typename T> FEAST_HD T cnorm2(cplx<T> a) { return a.x * a.x + a.y * a.y; }
// acc += a * b
template <typename T> FEAST_HD void cfma(cplx<T>& acc, cplx<T> a, cplx<T> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename T> FEAST_HD void cfmac(cplx<T>& acc, cplx<T> a, cplx<T> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// acc -= a * b
template <typename T> FEAST_HD void cfms(cplx<T>& acc, cplx<T> a, cplx<T> b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// Division with Smith's scaling (avoids overflow/underflow of |b|^2).
template <typename T> FEAST_HD cplx<T> cdiv(cplx<T> a, cplx<T> b) {
  if (fabs(b.x) >= fabs(b.y)) {
    T r = b.y / b.x, d = b.x + b.y * r;
    return mk<T>((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    T r = b.x / b.y, d = b.y + b.x * r;
    return mk<T>((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}
template <typename T> FEAST_HD cplx<T> crecip(cplx<T> b) { return cdiv<T>(mk<T>(T(1), T(0)), b); }

template <typename To, typename From> FEAST_HD cplx<To> cconv(cplx<From> a) {
  return mk<To>((To)a.x, (To)a.y);
}

// Operation applied to a GEMM operand.
enum GemmOp { OP_N = 0, OP_T = 1, OP_C = 2 };

// Device-side failure flags (bit mask, read by the host after each phase).
enum DevFlag { DEVFLAG_SINGULAR = 1, DEVFLAG_TIMEOUT = 2, DEVFLAG_NONFINITE = 4, DEVFLAG_BADARG = 8 };

inline unsigned ceil_div(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// Process-wide count of kernel launches made by this library (diagnostic;
// read through feast_kernel_launches()).
void feast_count_launch();

// Time limit (ns) of the cross-CTA waits: the value set by feast_set_wait_limit,
// else `dflt` (the kernel's built-in limit).
unsigned long long feast_wait_limit_ns(unsigned long long dflt);
