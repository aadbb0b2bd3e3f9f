// Forward-mode dual numbers with N derivative components (internal).
//
// The adjoint of the step is assembled from local Jacobians: every per-zone or
// per-face function of the step is a template on its scalar type, and
// evaluating it on Dn<N> arguments seeded with unit directions gives N columns
// of its Jacobian at once.  Comparisons act on the value, so branches follow
// the forward evaluation and the derivative is that of the branch taken.
#pragma once
#include <math.h>

#include <type_traits>

namespace hr {

template <int N>
struct Dn {
  double v;
  double d[N];
  __device__ __forceinline__ Dn() : v(0.0) {
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = 0.0;
  }
  __device__ __forceinline__ Dn(double x) : v(x) {
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = 0.0;
  }
  // value with unit derivative in component k (k < 0: constant)
  __device__ __forceinline__ static Dn seed(double x, int k) {
    Dn r(x);
    if (k >= 0 && k < N) r.d[k] = 1.0;
    return r;
  }
  __device__ __forceinline__ Dn& operator+=(const Dn& b) {
    v += b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] += b.d[k];
    return *this;
  }
  __device__ __forceinline__ Dn& operator-=(const Dn& b) {
    v -= b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] -= b.d[k];
    return *this;
  }
  __device__ __forceinline__ Dn& operator*=(const Dn& b) {
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = d[k] * b.v + v * b.d[k];
    v *= b.v;
    return *this;
  }
  __device__ __forceinline__ Dn& operator*=(double c) {
    v *= c;
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] *= c;
    return *this;
  }
  // g(a) with derivative g'(a) = gd applied to every component
  __device__ __forceinline__ static Dn chain(const Dn& a, double gv, double gd) {
    Dn r;
    r.v = gv;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = gd * a.d[k];
    return r;
  }
  // Elementary functions as hidden friends: found by argument-dependent
  // lookup for Dn arguments only, so the math library's overloads for double
  // and float stay visible everywhere.
  friend __device__ __forceinline__ Dn sqrt(const Dn& a) {
    const double s = ::sqrt(a.v);
    return chain(a, s, s > 0.0 ? 0.5 / s : 0.0);
  }
  friend __device__ __forceinline__ Dn rsqrt(const Dn& a) {
    const double s = ::rsqrt(a.v);
    return chain(a, s, -0.5 * s * s * s);
  }
  friend __device__ __forceinline__ Dn log(const Dn& a) { return chain(a, ::log(a.v), 1.0 / a.v); }
  friend __device__ __forceinline__ Dn exp(const Dn& a) {
    const double e = ::exp(a.v);
    return chain(a, e, e);
  }
  friend __device__ __forceinline__ Dn fabs(const Dn& a) {
    Dn r = a;
    if (a.v < 0.0) {
      r.v = -a.v;
#pragma unroll
      for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
    }
    return r;
  }
  friend __device__ __forceinline__ Dn fmax(const Dn& a, const Dn& b) { return a.v >= b.v ? a : b; }
  friend __device__ __forceinline__ Dn fmin(const Dn& a, const Dn& b) { return a.v <= b.v ? a : b; }
  friend __device__ __forceinline__ bool isfinite(const Dn& a) { return ::isfinite(a.v); }
};

template <typename T>
struct is_dual : std::false_type {};
template <int N>
struct is_dual<Dn<N>> : std::true_type {};

// Value of a scalar of any of the step's types.
__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(float x) { return x; }
template <int N>
__device__ __forceinline__ double val(const Dn<N>& x) { return x.v; }

template <int N>
__device__ __forceinline__ Dn<N> operator-(const Dn<N>& a) {
  Dn<N> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator+(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator+(const Dn<N>& a, double b) {
  Dn<N> r = a;
  r.v += b;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator+(double a, const Dn<N>& b) {
  return b + a;
}
template <int N>
__device__ __forceinline__ Dn<N> operator-(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator-(const Dn<N>& a, double b) {
  Dn<N> r = a;
  r.v -= b;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator-(double a, const Dn<N>& b) {
  Dn<N> r = -b;
  r.v += a;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator*(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator*(const Dn<N>& a, double c) {
  Dn<N> r;
  r.v = a.v * c;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * c;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator*(double c, const Dn<N>& a) {
  return a * c;
}
template <int N>
__device__ __forceinline__ Dn<N> operator/(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  const double ib = 1.0 / b.v;
  r.v = a.v / b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator/(const Dn<N>& a, double c) {
  Dn<N> r;
  const double ic = 1.0 / c;
  r.v = a.v / c;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * ic;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator/(double c, const Dn<N>& b) {
  Dn<N> r;
  const double ib = 1.0 / b.v;
  r.v = c / b.v;
  const double f = -r.v * ib;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = f * b.d[k];
  return r;
}

#define HR_DN_CMP(op)                                                                      \
  template <int N>                                                                         \
  __device__ __forceinline__ bool operator op(const Dn<N>& a, const Dn<N>& b) {            \
    return a.v op b.v;                                                                     \
  }                                                                                        \
  template <int N>                                                                         \
  __device__ __forceinline__ bool operator op(const Dn<N>& a, double b) {                  \
    return a.v op b;                                                                       \
  }                                                                                        \
  template <int N>                                                                         \
  __device__ __forceinline__ bool operator op(double a, const Dn<N>& b) {                  \
    return a op b.v;                                                                       \
  }
HR_DN_CMP(<)
HR_DN_CMP(>)
HR_DN_CMP(<=)
HR_DN_CMP(>=)
HR_DN_CMP(==)
HR_DN_CMP(!=)
#undef HR_DN_CMP

}  // namespace hr
