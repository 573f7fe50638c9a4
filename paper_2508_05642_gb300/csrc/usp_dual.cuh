// usp_dual.cuh -- forward-mode derivative numbers for the gradient form of the
// particle update: a value and its derivatives with respect to three
// parameters (Z_rot, the viscosity index omega, the wall temperature).
//
// Every arithmetic operation and elementary function below propagates the
// derivative by the chain rule; comparisons look at the value only, so a
// discrete decision (a level jump, a cell index, a wall hit, a branch) taken
// in the derivative form is the same as in the plain form of the same
// precision and is held fixed in the derivative (the pathwise derivative
// under common random numbers).
//
// Dual<double> (D3) carries FP64 values and derivatives (the FP64 gradient
// form); Dual<float> (F3) carries FP32 values and derivatives for the
// per-particle arithmetic of the FP32 gradient form, whose cell sums and
// cell-level quantities stay D3 (FP64 accumulation).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace usp {
namespace dual {

constexpr int kND = 3;

// elementary functions of the value type
__host__ __device__ inline float vsqrt(float x) { return sqrtf(x); }
__host__ __device__ inline double vsqrt(double x) { return ::sqrt(x); }
__host__ __device__ inline float vlog(float x) { return logf(x); }
__host__ __device__ inline double vlog(double x) { return ::log(x); }
__host__ __device__ inline float vlog1p(float x) { return log1pf(x); }
__host__ __device__ inline double vlog1p(double x) { return ::log1p(x); }
__host__ __device__ inline float vexp(float x) { return expf(x); }
__host__ __device__ inline double vexp(double x) { return ::exp(x); }
__host__ __device__ inline float vexpm1(float x) { return expm1f(x); }
__host__ __device__ inline double vexpm1(double x) { return ::expm1(x); }
__host__ __device__ inline float vsinh(float x) { return sinhf(x); }
__host__ __device__ inline double vsinh(double x) { return ::sinh(x); }
__host__ __device__ inline float vcosh(float x) { return coshf(x); }
__host__ __device__ inline double vcosh(double x) { return ::cosh(x); }
__host__ __device__ inline float vcos(float x) { return cosf(x); }
__host__ __device__ inline double vcos(double x) { return ::cos(x); }
__host__ __device__ inline float vsin(float x) { return sinf(x); }
__host__ __device__ inline double vsin(double x) { return ::sin(x); }
__host__ __device__ inline float vacos(float x) { return acosf(x); }
__host__ __device__ inline double vacos(double x) { return ::acos(x); }
__host__ __device__ inline float vcbrt(float x) { return cbrtf(x); }
__host__ __device__ inline double vcbrt(double x) { return ::cbrt(x); }
__host__ __device__ inline float vpow(float x, float y) { return powf(x, y); }
__host__ __device__ inline double vpow(double x, double y) { return ::pow(x, y); }

template <typename V>
struct Dual {
  V v;
  V d[kND];
  __host__ __device__ Dual() : v(V(0)) { d[0] = d[1] = d[2] = V(0); }
  __host__ __device__ Dual(double x) : v(V(x)) { d[0] = d[1] = d[2] = V(0); }
  __host__ __device__ Dual(double x, double d0, double d1, double d2) : v(V(x)) {
    d[0] = V(d0); d[1] = V(d1); d[2] = V(d2);
  }
  // between precisions (FP32 particle values <-> FP64 cell values)
  template <typename U>
  __host__ __device__ explicit Dual(const Dual<U>& o) : v(V(o.v)) {
    for (int i = 0; i < kND; ++i) d[i] = V(o.d[i]);
  }
  __host__ __device__ explicit operator double() const { return (double)v; }
  __host__ __device__ explicit operator float() const { return (float)v; }
  __host__ __device__ explicit operator int() const { return (int)v; }
  __host__ __device__ Dual& operator+=(const Dual& b) {
    v += b.v;
    for (int i = 0; i < kND; ++i) d[i] += b.d[i];
    return *this;
  }
  __host__ __device__ Dual& operator-=(const Dual& b) {
    v -= b.v;
    for (int i = 0; i < kND; ++i) d[i] -= b.d[i];
    return *this;
  }
  __host__ __device__ Dual& operator*=(const Dual& b) {
    for (int i = 0; i < kND; ++i) d[i] = d[i] * b.v + v * b.d[i];
    v *= b.v;
    return *this;
  }
  __host__ __device__ Dual& operator/=(const Dual& b) {
    const V q = v / b.v;
    for (int i = 0; i < kND; ++i) d[i] = (d[i] - q * b.d[i]) / b.v;
    v = q;
    return *this;
  }
};

using D3 = Dual<double>;
using F3 = Dual<float>;

template <typename V>
__host__ __device__ inline Dual<V> operator+(Dual<V> a, const Dual<V>& b) { return a += b; }
template <typename V>
__host__ __device__ inline Dual<V> operator-(Dual<V> a, const Dual<V>& b) { return a -= b; }
template <typename V>
__host__ __device__ inline Dual<V> operator*(Dual<V> a, const Dual<V>& b) { return a *= b; }
template <typename V>
__host__ __device__ inline Dual<V> operator/(Dual<V> a, const Dual<V>& b) { return a /= b; }
template <typename V>
__host__ __device__ inline Dual<V> operator+(Dual<V> a, double b) { a.v += V(b); return a; }
template <typename V>
__host__ __device__ inline Dual<V> operator+(double b, Dual<V> a) { a.v += V(b); return a; }
template <typename V>
__host__ __device__ inline Dual<V> operator-(Dual<V> a, double b) { a.v -= V(b); return a; }
template <typename V>
__host__ __device__ inline Dual<V> operator-(double b, const Dual<V>& a) {
  Dual<V> r;
  r.v = V(b) - a.v;
  for (int i = 0; i < kND; ++i) r.d[i] = -a.d[i];
  return r;
}
template <typename V>
__host__ __device__ inline Dual<V> operator*(Dual<V> a, double b) {
  const V c = V(b);
  a.v *= c;
  for (int i = 0; i < kND; ++i) a.d[i] *= c;
  return a;
}
template <typename V>
__host__ __device__ inline Dual<V> operator*(double b, Dual<V> a) { return a * b; }
template <typename V>
__host__ __device__ inline Dual<V> operator/(Dual<V> a, double b) {
  const V c = V(b);
  a.v /= c;
  for (int i = 0; i < kND; ++i) a.d[i] /= c;
  return a;
}
template <typename V>
__host__ __device__ inline Dual<V> operator/(double b, const Dual<V>& a) { return Dual<V>(b) / a; }
template <typename V>
__host__ __device__ inline Dual<V> operator-(const Dual<V>& a) {
  Dual<V> r;
  r.v = -a.v;
  for (int i = 0; i < kND; ++i) r.d[i] = -a.d[i];
  return r;
}

#define USP_DUAL_CMP(op)                                                                       \
  template <typename V>                                                                        \
  __host__ __device__ inline bool operator op(const Dual<V>& a, const Dual<V>& b) {            \
    return a.v op b.v;                                                                         \
  }                                                                                            \
  template <typename V>                                                                        \
  __host__ __device__ inline bool operator op(const Dual<V>& a, double b) { return a.v op b; } \
  template <typename V>                                                                        \
  __host__ __device__ inline bool operator op(double a, const Dual<V>& b) { return a op b.v; }
USP_DUAL_CMP(<)
USP_DUAL_CMP(>)
USP_DUAL_CMP(<=)
USP_DUAL_CMP(>=)
USP_DUAL_CMP(==)
USP_DUAL_CMP(!=)
#undef USP_DUAL_CMP

// f(a) with f'(a) = df
template <typename V>
__host__ __device__ inline Dual<V> chain(const Dual<V>& a, V fv, V df) {
  Dual<V> r;
  r.v = fv;
  for (int i = 0; i < kND; ++i) r.d[i] = df * a.d[i];
  return r;
}

template <typename V>
__device__ inline Dual<V> sqrt(const Dual<V>& a) {
  const V s = vsqrt(a.v);
  return chain(a, s, s > V(0) ? V(0.5) / s : V(0));
}
template <typename V>
__device__ inline Dual<V> log(const Dual<V>& a) { return chain(a, vlog(a.v), V(1) / a.v); }
template <typename V>
__device__ inline Dual<V> log1p(const Dual<V>& a) {
  return chain(a, vlog1p(a.v), V(1) / (V(1) + a.v));
}
template <typename V>
__device__ inline Dual<V> exp(const Dual<V>& a) {
  const V e = vexp(a.v);
  return chain(a, e, e);
}
template <typename V>
__device__ inline Dual<V> expm1(const Dual<V>& a) { return chain(a, vexpm1(a.v), vexp(a.v)); }
template <typename V>
__device__ inline Dual<V> sinh(const Dual<V>& a) { return chain(a, vsinh(a.v), vcosh(a.v)); }
template <typename V>
__device__ inline Dual<V> cos(const Dual<V>& a) { return chain(a, vcos(a.v), -vsin(a.v)); }
template <typename V>
__device__ inline Dual<V> acos(const Dual<V>& a) {
  const V den = vsqrt(V(1) - a.v * a.v);
  return chain(a, vacos(a.v), den > V(0) ? V(-1) / den : V(0));
}
template <typename V>
__device__ inline Dual<V> cbrt(const Dual<V>& a) {
  const V c = vcbrt(a.v);
  return chain(a, c, c != V(0) ? c / (V(3) * a.v) : V(0));
}
template <typename V>
__device__ inline Dual<V> fabs(const Dual<V>& a) { return a.v < V(0) ? -a : a; }
template <typename V>
__device__ inline Dual<V> fmin(const Dual<V>& a, const Dual<V>& b) { return b.v < a.v ? b : a; }
template <typename V>
__device__ inline Dual<V> fmax(const Dual<V>& a, const Dual<V>& b) { return b.v > a.v ? b : a; }
// a^b with a > 0 (both carrying derivatives)
template <typename V>
__device__ inline Dual<V> pow(const Dual<V>& a, const Dual<V>& b) {
  const V p = vpow(a.v, b.v);
  Dual<V> r;
  r.v = p;
  const V la = vlog(a.v);
  for (int i = 0; i < kND; ++i) r.d[i] = p * (b.d[i] * la + b.v * a.d[i] / a.v);
  return r;
}
template <typename V>
__device__ inline Dual<V> pow(const Dual<V>& a, double b) {
  const V p = vpow(a.v, V(b));
  return chain(a, p, V(b) * vpow(a.v, V(b - 1.0)));
}
template <typename V>
__device__ inline Dual<V> pow(double a, const Dual<V>& b) {
  const V p = vpow(V(a), b.v);
  return chain(b, p, p * vlog(V(a)));
}
template <typename V>
__device__ inline V value(const Dual<V>& a) { return a.v; }

}  // namespace dual

using dual::D3;
using dual::F3;
using dual::kND;
using dual::value;
__device__ inline double value(double a) { return a; }
__device__ inline float value(float a) { return a; }

// A quantity held at its value in the gradient form: its derivative is
// dropped (the identity in the plain forms).
template <typename V>
__device__ inline dual::Dual<V> held(const dual::Dual<V>& a) { return dual::Dual<V>(a.v); }
__device__ inline double held(double a) { return a; }
__device__ inline float held(float a) { return a; }

}  // namespace usp
