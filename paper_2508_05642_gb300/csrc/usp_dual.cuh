// usp_dual.cuh -- forward-mode derivative numbers for the gradient form of the
// particle update: a value and its derivatives with respect to three
// parameters (Z_rot, the viscosity index omega, the wall temperature).
//
// Every arithmetic operation and elementary function below propagates the
// derivative by the chain rule; comparisons look at the value only, so a
// discrete decision (a level jump, a cell index, a wall hit, a branch) taken
// in the derivative form is the same as in the plain FP64 form and is held
// fixed in the derivative (the pathwise derivative under common random
// numbers).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace usp {
namespace dual {

constexpr int kND = 3;

struct D3 {
  double v;
  double d[kND];
  __host__ __device__ D3() : v(0.0) { d[0] = d[1] = d[2] = 0.0; }
  __host__ __device__ D3(double x) : v(x) { d[0] = d[1] = d[2] = 0.0; }
  __host__ __device__ D3(double x, double d0, double d1, double d2) : v(x) {
    d[0] = d0; d[1] = d1; d[2] = d2;
  }
  __host__ __device__ explicit operator double() const { return v; }
  __host__ __device__ explicit operator float() const { return (float)v; }
  __host__ __device__ explicit operator int() const { return (int)v; }
  __host__ __device__ D3& operator+=(const D3& b) {
    v += b.v;
    for (int i = 0; i < kND; ++i) d[i] += b.d[i];
    return *this;
  }
  __host__ __device__ D3& operator-=(const D3& b) {
    v -= b.v;
    for (int i = 0; i < kND; ++i) d[i] -= b.d[i];
    return *this;
  }
  __host__ __device__ D3& operator*=(const D3& b) {
    for (int i = 0; i < kND; ++i) d[i] = d[i] * b.v + v * b.d[i];
    v *= b.v;
    return *this;
  }
  __host__ __device__ D3& operator/=(const D3& b) {
    const double q = v / b.v;
    for (int i = 0; i < kND; ++i) d[i] = (d[i] - q * b.d[i]) / b.v;
    v = q;
    return *this;
  }
};

__host__ __device__ inline D3 operator+(D3 a, const D3& b) { return a += b; }
__host__ __device__ inline D3 operator-(D3 a, const D3& b) { return a -= b; }
__host__ __device__ inline D3 operator*(D3 a, const D3& b) { return a *= b; }
__host__ __device__ inline D3 operator/(D3 a, const D3& b) { return a /= b; }
__host__ __device__ inline D3 operator+(D3 a, double b) { a.v += b; return a; }
__host__ __device__ inline D3 operator+(double b, D3 a) { a.v += b; return a; }
__host__ __device__ inline D3 operator-(D3 a, double b) { a.v -= b; return a; }
__host__ __device__ inline D3 operator-(double b, const D3& a) {
  D3 r(b - a.v);
  for (int i = 0; i < kND; ++i) r.d[i] = -a.d[i];
  return r;
}
__host__ __device__ inline D3 operator*(D3 a, double b) {
  a.v *= b;
  for (int i = 0; i < kND; ++i) a.d[i] *= b;
  return a;
}
__host__ __device__ inline D3 operator*(double b, D3 a) { return a * b; }
__host__ __device__ inline D3 operator/(D3 a, double b) {
  a.v /= b;
  for (int i = 0; i < kND; ++i) a.d[i] /= b;
  return a;
}
__host__ __device__ inline D3 operator/(double b, const D3& a) { return D3(b) / a; }
__host__ __device__ inline D3 operator-(const D3& a) {
  D3 r(-a.v);
  for (int i = 0; i < kND; ++i) r.d[i] = -a.d[i];
  return r;
}

#define USP_D3_CMP(op)                                                                  \
  __host__ __device__ inline bool operator op(const D3& a, const D3& b) { return a.v op b.v; } \
  __host__ __device__ inline bool operator op(const D3& a, double b) { return a.v op b; }      \
  __host__ __device__ inline bool operator op(double a, const D3& b) { return a op b.v; }
USP_D3_CMP(<)
USP_D3_CMP(>)
USP_D3_CMP(<=)
USP_D3_CMP(>=)
USP_D3_CMP(==)
USP_D3_CMP(!=)
#undef USP_D3_CMP

// f(a) with f'(a) = df
__host__ __device__ inline D3 chain(const D3& a, double fv, double df) {
  D3 r(fv);
  for (int i = 0; i < kND; ++i) r.d[i] = df * a.d[i];
  return r;
}

__device__ inline D3 sqrt(const D3& a) {
  const double s = ::sqrt(a.v);
  return chain(a, s, s > 0.0 ? 0.5 / s : 0.0);
}
__device__ inline D3 log(const D3& a) { return chain(a, ::log(a.v), 1.0 / a.v); }
__device__ inline D3 log1p(const D3& a) { return chain(a, ::log1p(a.v), 1.0 / (1.0 + a.v)); }
__device__ inline D3 exp(const D3& a) {
  const double e = ::exp(a.v);
  return chain(a, e, e);
}
__device__ inline D3 expm1(const D3& a) { return chain(a, ::expm1(a.v), ::exp(a.v)); }
__device__ inline D3 sinh(const D3& a) { return chain(a, ::sinh(a.v), ::cosh(a.v)); }
__device__ inline D3 cos(const D3& a) { return chain(a, ::cos(a.v), -::sin(a.v)); }
__device__ inline D3 acos(const D3& a) {
  const double den = ::sqrt(1.0 - a.v * a.v);
  return chain(a, ::acos(a.v), den > 0.0 ? -1.0 / den : 0.0);
}
__device__ inline D3 cbrt(const D3& a) {
  const double c = ::cbrt(a.v);
  return chain(a, c, c != 0.0 ? c / (3.0 * a.v) : 0.0);
}
__device__ inline D3 fabs(const D3& a) { return a.v < 0.0 ? -a : a; }
__device__ inline D3 fmin(const D3& a, const D3& b) { return b.v < a.v ? b : a; }
__device__ inline D3 fmax(const D3& a, const D3& b) { return b.v > a.v ? b : a; }
// a^b with a > 0 (both carrying derivatives)
__device__ inline D3 pow(const D3& a, const D3& b) {
  const double p = ::pow(a.v, b.v);
  D3 r(p);
  const double la = ::log(a.v);
  for (int i = 0; i < kND; ++i) r.d[i] = p * (b.d[i] * la + b.v * a.d[i] / a.v);
  return r;
}
__device__ inline D3 pow(const D3& a, double b) {
  const double p = ::pow(a.v, b);
  return chain(a, p, b * ::pow(a.v, b - 1.0));
}
__device__ inline D3 pow(double a, const D3& b) {
  const double p = ::pow(a, b.v);
  return chain(b, p, p * ::log(a));
}
__device__ inline double value(const D3& a) { return a.v; }

}  // namespace dual

using dual::D3;
using dual::kND;
using dual::value;
__device__ inline double value(double a) { return a; }
__device__ inline float value(float a) { return a; }

// A quantity held at its value in the gradient form: its derivative is
// dropped (the identity in the plain forms).
__device__ inline D3 held(const D3& a) { return D3(a.v); }
__device__ inline double held(double a) { return a; }
__device__ inline float held(float a) { return a; }

}  // namespace usp
