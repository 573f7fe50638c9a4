// usp_device.cuh -- device building blocks of the USP-FPM particle update on
// sm_103a: the counter-based random stream, the jump samplers, small linear
// algebra and the per-cell closed forms of Kim & Jun (arXiv 2508.05642).
//
// Precision policy: per-cell work (transport coefficients, gamma fixed point,
// conservation factors) is FP64; per-particle work is templated on the state
// type T (float for the FP32-state form, double for the plain FP64 form).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace usp {

constexpr double kB = 1.380649e-23;  // Boltzmann constant [J/K]
constexpr double kPi = 3.14159265358979323846;

// status bits (sticky device word)
enum : uint32_t {
  F_PB_CLAMP = 0x01u,
  F_CHOL_FAIL_AFTER_FIX = 0x02u,
  F_NEG_RADICAND = 0x04u,
  F_VIB_LOOP_CAP = 0x08u,
  F_TREL_CLAMP = 0x10u,
  F_SAMPLER_CAP = 0x20u,
  F_A_NONPOS = 0x40u,
  F_SAMPLER_UNDERFLOW = 0x80u,
  F_WALL_CAP = 0x100u,
  F_BOUNDS = 0x200u,
  F_WAIT_TIMEOUT = 0x400u,
  F_INFLOW_CAP = 0x800u,
  F_CAPACITY = 0x1000u,
};
enum { C_CHOL_FIX = 0, C_PB_CLAMP, C_TREL_CLAMP, C_VIB_DRAWS, C_NEG_RADICAND,
       C_WALL_HITS, C_INTERP_FALLBACK, C_SKIPPED_CELLS, C_INFLOW, C_OUTFLOW, C_NU_ZERO,
       NCOUNTERS };

// Philox stream layout: particle counter (pid, step, tag, 0); cell counter
// (cell, step, 0x80000000 | tag, block).
enum : uint32_t { PTAG_NORMALS = 0u, PTAG_JUMPS = 1u, PTAG_GILLESPIE = 8u };
enum : uint32_t { CTAG_IDELTA = 0x80000000u, CTAG_PICK = 0x80000001u };

struct Species {
  double m, d_ref, omega, T_ref, c_alpha, theta_v, Z_rot, Z_vib;
  int zmodel;
  double Zrot_inf, T_star, C1, C2, sigma_vib;
  // derived on the host: T_ref^omega, pi d_ref^2 / sigma_vib, R = k_B / m,
  // and the VSS mu_ref and tau_c / (mu / p) at this omega
  double Tref_w, zv_ht, R, mu_ref0, tauf0;
  int method;   // 0 USP-FPM (Sec. 3, 4), 1 the plain FPM method (Sec. 2.C)
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds, two 32x32->64 products
// per round, key bumped by the Weyl constants.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c0 = n0; c1 = (uint32_t)p1; c2 = n2; c3 = (uint32_t)p0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// The ten round keys of one key, computed once on the host: kernels take
// them as a by-value parameter, so each round reads its key from the
// parameter bank instead of advancing it per thread.
struct PhiloxRoundKeys {
  uint32_t k0[10], k1[10];
};
inline PhiloxRoundKeys philox_round_keys(uint32_t k0, uint32_t k1) {
  PhiloxRoundKeys rk;
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0;
    rk.k1[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return rk;
}
// Two blocks whose counters differ only in word 2, rounds interleaved so the
// two independent multiply chains overlap.
__device__ __forceinline__ void philox4x32_10_pair(uint32_t c0, uint32_t c1, uint32_t c2a,
                                                   uint32_t c2b, uint32_t c3,
                                                   const PhiloxRoundKeys& rk, U4& a, U4& b) {
  uint32_t a0 = c0, a1 = c1, a2 = c2a, a3 = c3;
  uint32_t b0 = c0, b1 = c1, b2 = c2b, b3 = c3;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t pa0 = (uint64_t)0xD2511F53u * a0, pa1 = (uint64_t)0xCD9E8D57u * a2;
    const uint64_t pb0 = (uint64_t)0xD2511F53u * b0, pb1 = (uint64_t)0xCD9E8D57u * b2;
    const uint32_t na0 = (uint32_t)(pa1 >> 32) ^ a1 ^ rk.k0[r];
    const uint32_t na2 = (uint32_t)(pa0 >> 32) ^ a3 ^ rk.k1[r];
    const uint32_t nb0 = (uint32_t)(pb1 >> 32) ^ b1 ^ rk.k0[r];
    const uint32_t nb2 = (uint32_t)(pb0 >> 32) ^ b3 ^ rk.k1[r];
    a0 = na0; a1 = (uint32_t)pa1; a2 = na2; a3 = (uint32_t)pa0;
    b0 = nb0; b1 = (uint32_t)pb1; b2 = nb2; b3 = (uint32_t)pb0;
  }
  a = U4{a0, a1, a2, a3};
  b = U4{b0, b1, b2, b3};
}
__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            const PhiloxRoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk.k0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk.k1[r];
    c0 = n0; c1 = (uint32_t)p1; c2 = n2; c3 = (uint32_t)p0;
  }
  return U4{c0, c1, c2, c3};
}

// Open-interval uniforms.  double: (x + 0.5) 2^-32 (exact).
// float: (2 (x >> 9) + 1) 2^-24 (exact; 23 random bits).
template <typename T> __device__ __forceinline__ T uniform_open(uint32_t x);
// Both are formed without an integer-to-float conversion: the word goes into
// the mantissa of a number in [1, 2), from which 1 - (half a step) is
// subtracted.  The subtraction is exact (Sterbenz: the operands are within a
// factor of two), so the results are exactly (x + 1/2) 2^-32 and
// (2 (x >> 9) + 1) 2^-24.
template <> __device__ __forceinline__ double uniform_open<double>(uint32_t x) {
  const double a =
      __longlong_as_double((long long)(0x3FF0000000000000ull | ((unsigned long long)x << 20)));
  return __dsub_rn(a, 0.99999999988358467817306518554688);   // 1 - 2^-33
}
template <> __device__ __forceinline__ float uniform_open<float>(uint32_t x) {
  const float a = __int_as_float((int)(0x3F800000u | (x >> 9)));
  return __fsub_rn(a, 0.999999940395355224609375f);          // 1 - 2^-24
}

// Square root in the FP32 particle arithmetic: the hardware approximation
// (relative error about 2^-23), not the correctly rounded square root's longer
// sequence; the double form keeps sqrt.
__device__ __forceinline__ float sqrt_fast(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double sqrt_fast(double x) { return sqrt(x); }

// Box-Muller pair: G_a = sqrt(-2 ln u_a) cos(2 pi u_b), G_b = ... sin(2 pi u_b).
// The float version takes -2 ln u = -2 ln 2 log2 u with the hardware base-2
// logarithm and square root (absolute error of log2 about 2^-22 near u = 1, a
// relative error near 2^-22 elsewhere: far below the 2^-24 resolution of the
// uniforms' effect on the normals' distribution), and evaluates the angle on
// (-pi, pi), where the hardware sine/cosine has an absolute error below 2^-21:
// cos(2 pi u) = -cos(2 pi u - pi), sin(2 pi u) = -sin(2 pi u - pi).  The
// centred form takes uc = u_b - 1/2 directly.
__device__ __forceinline__ void box_muller_centred(float ua, float uc, float& ga, float& gb) {
  float l2;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(ua));
  const float rad = sqrt_fast(fmaxf(-1.38629436111989061883f * l2, 0.0f));
  float s, c;
  __sincosf(6.28318530717958647692f * uc, &s, &c);
  ga = -rad * c;
  gb = -rad * s;
}
__device__ __forceinline__ void box_muller(float ua, float ub, float& ga, float& gb) {
  box_muller_centred(ua, ub - 0.5f, ga, gb);
}
__device__ __forceinline__ void box_muller(double ua, double ub, double& ga, double& gb) {
  const double rad = sqrt(-2.0 * log(ua));
  double s, c;
  sincospi(2.0 * ub, &s, &c);
  ga = rad * c;
  gb = rad * s;
}

// ---------------------------------------------------------------------------
// The collision draws of one particle and step: four standard normals
// g0..g3 (two Box-Muller pairs) and the two words j5, j6 whose uniforms
// drive the jump samplers, all from one Philox block, counter
// (pid, step, 0, 0).  A uniform takes 23 bits of a word,
// (2 (x >> 9) + 1) 2^-24, exact in float and double, so one block carries
// all six: the top 23 bits of words 0 and 1 are the two radius uniforms, those
// of words 2 and 3 the jump uniforms (j5 = word 2, j6 = word 3), and the low
// 9 bits of words 0 and 1, then of words 2 and 3, form the two angle uniforms
// of 18 bits, (2 a + 1) 2^-19 with a = (lo9(word) << 9) | lo9(next word).
// The FP32 and FP64 forms thus draw identical values.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t angle_bits18(uint32_t wa, uint32_t wb) {
  return ((wa & 0x1ffu) << 9) | (wb & 0x1ffu);
}
// the angle uniform minus 1/2: 1 + a 2^-18 minus 3/2 - 2^-19 is exactly
// (2 a + 1) 2^-19 - 1/2 (Sterbenz), the value that (2 a + 1) 2^-19 - 1/2
// rounds to as well, in one subtraction
__device__ __forceinline__ float angle_centred18(uint32_t wa, uint32_t wb) {
  return __fsub_rn(__int_as_float((int)(0x3f800000u | (angle_bits18(wa, wb) << 5))),
                   1.49999809265136718750f);
}
__device__ __forceinline__ double angle_uniform18_d(uint32_t wa, uint32_t wb) {
  return (2.0 * (double)angle_bits18(wa, wb) + 1.0) * 1.9073486328125e-06;   // 2^-19
}
// the 23-bit uniform of a word in double (equal to uniform_open<float>)
__device__ __forceinline__ double uniform23_d(uint32_t x) {
  return (2.0 * (double)(x >> 9) + 1.0) * 5.9604644775390625e-08;             // 2^-24
}

// the jump-sampler uniform of a word, in the working type
template <typename T>
__device__ __forceinline__ T jump_uniform(uint32_t x) { return T(uniform23_d(x)); }
template <>
__device__ __forceinline__ float jump_uniform<float>(uint32_t x) { return uniform_open<float>(x); }

__device__ __forceinline__ void particle_draws(uint32_t pid, uint32_t step,
                                               const PhiloxRoundKeys& rk, float& g0, float& g1,
                                               float& g2, float& g3, uint32_t& j5, uint32_t& j6) {
  const U4 w = philox4x32_10(pid, step, PTAG_NORMALS, 0u, rk);
  box_muller_centred(uniform_open<float>(w.x), angle_centred18(w.x, w.y), g0, g1);
  box_muller_centred(uniform_open<float>(w.y), angle_centred18(w.z, w.w), g2, g3);
  j5 = w.z;
  j6 = w.w;
}

__device__ __forceinline__ void particle_draws(uint32_t pid, uint32_t step,
                                               const PhiloxRoundKeys& rk, double& g0, double& g1,
                                               double& g2, double& g3, uint32_t& j5,
                                               uint32_t& j6) {
  const U4 w = philox4x32_10(pid, step, PTAG_NORMALS, 0u, rk);
  box_muller(uniform23_d(w.x), angle_uniform18_d(w.x, w.y), g0, g1);
  box_muller(uniform23_d(w.y), angle_uniform18_d(w.z, w.w), g2, g3);
  j5 = w.z;
  j6 = w.w;
}

// ---------------------------------------------------------------------------
// Jump samplers of Eq. update_evib: sequential inversion with one uniform,
// pmf stepped by its ratio recursion, P(0) by square-and-multiply; a binomial
// with p > 1/2 is drawn as n - B(n, 1 - p).  Every operation is an explicit
// round-to-nearest intrinsic so the integer outcome is a fixed function of
// (r or n, p, u) in the working precision.  The float search falls back to
// double when P(0) is not a normal float.
// ---------------------------------------------------------------------------
constexpr int kSamplerCap = 4096;

__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rn_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float rn_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rn_i2f(int a, double) { return __int2double_rn(a); }
__device__ __forceinline__ float rn_i2f(int a, float) { return __int2float_rn(a); }

template <typename T>
__device__ __forceinline__ T powi_rn(T x, int e) {
  T r = T(1), b = x;
  while (e > 0) {
    if (e & 1) r = rn_mul(r, b);
    b = rn_mul(b, b);
    e >>= 1;
  }
  return r;
}

static __device__ __noinline__ int nb_inv_d(int r, double p, double u, uint32_t& fl) {
  const double q = rn_sub(1.0, p);
  double P = powi_rn(p, r);
  if (P < 2.2250738585072014e-308) {
    fl |= F_SAMPLER_UNDERFLOW;
    return (int)floor(r * q / p);
  }
  double cdf = P;
  int k = 0;
  while (u >= cdf) {
    if (k >= kSamplerCap) { fl |= F_SAMPLER_CAP; break; }
    const double t = rn_div(rn_i2f(k + r, 0.0), rn_i2f(k + 1, 0.0));
    P = rn_mul(P, t);
    P = rn_mul(P, q);
    k = k + 1;
    const double nc = rn_add(cdf, P);
    if (nc == cdf) break;
    cdf = nc;
  }
  return k;
}

static __device__ __noinline__ int binv_d(int n, double p, double u, uint32_t& fl) {
  const double q = rn_sub(1.0, p);
  double P = powi_rn(q, n);
  if (P < 2.2250738585072014e-308) {
    fl |= F_SAMPLER_UNDERFLOW;
    return (int)floor(n * p);
  }
  const double pq = rn_div(p, q);
  double cdf = P;
  int k = 0;
  while (u >= cdf && k < n) {
    if (k >= kSamplerCap) { fl |= F_SAMPLER_CAP; break; }
    const double t = rn_div(rn_i2f(n - k, 0.0), rn_i2f(k + 1, 0.0));
    P = rn_mul(P, t);
    P = rn_mul(P, pq);
    k = k + 1;
    const double nc = rn_add(cdf, P);
    if (nc == cdf) break;
    cdf = nc;
  }
  return k;
}

__device__ __forceinline__ int nb_inv(int r, float p, float u, uint32_t& fl) {
  const float q = rn_sub(1.0f, p);
  float P = powi_rn(p, r);
  if (P < 1.17549435e-38f) return nb_inv_d(r, (double)p, (double)u, fl);
  float cdf = P;
  int k = 0;
  while (u >= cdf) {
    if (k >= kSamplerCap) { fl |= F_SAMPLER_CAP; break; }
    const float t = rn_div(rn_i2f(k + r, 0.0f), rn_i2f(k + 1, 0.0f));
    P = rn_mul(P, t);
    P = rn_mul(P, q);
    k = k + 1;
    const float nc = rn_add(cdf, P);
    if (nc == cdf) break;
    cdf = nc;
  }
  return k;
}
__device__ __forceinline__ int nb_inv(int r, double p, double u, uint32_t& fl) {
  return nb_inv_d(r, p, u, fl);
}

__device__ __forceinline__ int binv(int n, float p, float u, uint32_t& fl) {
  const float q = rn_sub(1.0f, p);
  float P = powi_rn(q, n);
  if (P < 1.17549435e-38f) return binv_d(n, (double)p, (double)u, fl);
  const float pq = rn_div(p, q);
  float cdf = P;
  int k = 0;
  while (u >= cdf && k < n) {
    if (k >= kSamplerCap) { fl |= F_SAMPLER_CAP; break; }
    const float t = rn_div(rn_i2f(n - k, 0.0f), rn_i2f(k + 1, 0.0f));
    P = rn_mul(P, t);
    P = rn_mul(P, pq);
    k = k + 1;
    const float nc = rn_add(cdf, P);
    if (nc == cdf) break;
    cdf = nc;
  }
  return k;
}
__device__ __forceinline__ int binv(int n, double p, double u, uint32_t& fl) {
  return binv_d(n, p, u, fl);
}

// NB(r, p): failures before the r-th success.
template <typename T>
__device__ __forceinline__ int sample_nb(int r, T p, T u, uint32_t& fl) {
  if (r <= 0 || !(p < T(1))) return 0;
  return nb_inv(r, p, u, fl);
}
// B(n, p); p >= 1 gives n (and flags p > 1).
template <typename T>
__device__ __forceinline__ int sample_b(int n, T p, T u, uint32_t& fl) {
  if (n <= 0) return 0;
  if (p >= T(1)) {
    if (p > T(1)) fl |= F_PB_CLAMP;
    return n;
  }
  if (!(p > T(0))) return 0;
  if (p > T(0.5)) return n - binv(n, rn_sub(T(1), p), u, fl);
  return binv(n, p, u, fl);
}

// ---------------------------------------------------------------------------
// Closed forms (FP64, per cell).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double gasR(const Species& s) { return s.R; }

// The per-cell closed forms below are templates over the scalar S: double
// for the plain forms, a derivative number for the gradient form (with the
// viscosity index omega and the rotational collision number Z_rot passed as
// S so that derivatives with respect to them propagate).

// e_vib(T) = R Theta / (exp(Theta/T) - 1) (Sec. 2.A)
template <typename S>
__device__ __forceinline__ S e_vib_T(const Species& s, const S& T) {
  if (T <= 0.0) return S(0.0);
  return gasR(s) * s.theta_v / expm1(s.theta_v / T);
}
// c_v,vib(T) = R (Theta/2T)^2 / sinh^2(Theta/2T): the derivative of e_vib.
template <typename S>
__device__ __forceinline__ S cv_vib_T(const Species& s, const S& T) {
  if (T <= 0.0) return S(0.0);
  const S h = 0.5 * s.theta_v / T;
  const S sh = sinh(h);
  return gasR(s) * (h * h) / (sh * sh);
}
// temperature whose e_vib is R Theta ebar
template <typename S>
__device__ __forceinline__ S T_vib_of_level(const Species& s, const S& ebar) {
  if (ebar <= 0.0) return S(0.0);
  return s.theta_v / log1p(1.0 / ebar);
}
// VSS viscosity and the factor tau_c = K mu / p (Sec. 4.A)
template <typename S>
__device__ __forceinline__ S mu_of_T_w(const Species& s, const S& T, const S& w) {
  const double ca = s.c_alpha;
  const S mu_ref = 5.0 * (ca + 1.0) * (ca + 2.0) * sqrt(s.m * kB * s.T_ref / kPi) /
                   (4.0 * ca * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) * s.d_ref * s.d_ref);
  return mu_ref * pow(T / s.T_ref, w);
}
template <typename S>
__device__ __forceinline__ S tau_c_factor_w(const Species& s, const S& w) {
  const double ca = s.c_alpha;
  return ca * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) / (5.0 * (ca + 1.0) * (ca + 2.0));
}
__device__ __forceinline__ double mu_of_T(const Species& s, double T) {
  return mu_of_T_w<double>(s, T, s.omega);
}
__device__ __forceinline__ double tau_c_factor(const Species& s) {
  return tau_c_factor_w<double>(s, s.omega);
}
// Eucken Pr (Sec. 4.B), xi_vib evaluated at the cell vibrational temperature
template <typename S>
__device__ __forceinline__ S prandtl_T(const Species& s, const S& Tv) {
  S xi(0.0);
  if (Tv > 0.0) {
    const S x = s.theta_v / Tv;
    xi = x / expm1(x);
  }
  return (14.0 + 2.0 * xi) / (19.0 + 2.0 * xi);
}
// Collision numbers: zmodel 0 the fixed ones, zmodel 1 Parker's Z_rot and
// Millikan-White with the high-temperature term for Z_vib (Sec. 5.C).  xw is
// (T_tr/T_ref)^omega, shared with the viscosity, so that
// T^omega = T_ref^omega xw and (T_ref/T)^(omega - 1/2) = sqrt(T/T_ref) / xw.
template <typename S>
__device__ __forceinline__ void collision_numbers(const Species& s, const S& Ttr, const S& xw,
                                                  const S& zrot0, S& zr, S& zv) {
  if (s.zmodel == 0) { zr = zrot0; zv = S(s.Z_vib); return; }
  const S r = s.T_star / Ttr;
  zr = s.Zrot_inf / (1.0 + 0.5 * kPi * sqrt(kPi) * sqrt(r) + (kPi + 0.25 * kPi * kPi) * r);
  zv = (s.C1 / (s.Tref_w * xw)) * exp(s.C2 / cbrt(Ttr)) + s.zv_ht * sqrt(Ttr / s.T_ref) / xw;
}

// Per-cell coefficients of Sec. 3.A: alpha = A^(1/3) (the real cube root,
// negative when dt >= 2 mu / (p Pr)), nu, the gamma
// coefficients with the implicit c_v,vib(T_1) (fixed point started at
// c_v,vib(T_tr), relative tolerance 1e-14 or the secant's own rounding,
// whichever is larger, at most 50 passes), and the second-order energy
// targets.
template <typename S>
struct CellCoeffsT {
  S mu_p, Pr, A, B, alpha, nu_ref;
  S g_tr_rot, g_tr_vib, g_rot_vib;
  S e_rot_tgt, e_vib_tgt;
  bool ok;
  bool tgt_clamped;   // a negative target was set to 0
};

template <typename S>
__device__ inline CellCoeffsT<S> cell_coeffs_t(const Species& s, const S& omega, const S& zrot,
                                               double n, double dt, const S& Ttr, const S& Trot,
                                               const S& Tvib) {
  CellCoeffsT<S> c;
  const double R = gasR(s);
  const double ctr = 1.5 * R, crot = R;
  const S p = n * kB * Ttr;
  // (T/T_ref)^omega, shared by the viscosity and the collision numbers
  const S xw = exp(omega * log(Ttr / s.T_ref));
  S mu_ref, tauf;
  if constexpr (sizeof(S) == sizeof(double)) {   // plain forms: species constants
    mu_ref = S(s.mu_ref0);
    tauf = S(s.tauf0);
  } else {                                        // derivative form: through omega
    const double ca = s.c_alpha;
    mu_ref = 5.0 * (ca + 1.0) * (ca + 2.0) * sqrt(s.m * kB * s.T_ref / kPi) /
             (4.0 * ca * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega) * s.d_ref * s.d_ref);
    tauf = tau_c_factor_w<S>(s, omega);
  }
  c.mu_p = mu_ref * xw / p;
  const S tau_c = tauf * c.mu_p;
  S zr, zv;
  collision_numbers<S>(s, Ttr, xw, zrot, zr, zv);
  const S tau_rot = zr * tau_c, tau_vib = zv * tau_c;
  c.Pr = prandtl_T<S>(s, Tvib);
  c.A = (2.0 * c.mu_p - c.Pr * dt) / (2.0 * c.mu_p + c.Pr * dt);
  c.B = (2.0 * c.mu_p - dt) / (2.0 * c.mu_p + dt);
  c.ok = c.A > -1.0 && c.A < 1.0;
  c.alpha = c.ok ? cbrt(c.A) : S(0.0);
  const S a2 = c.alpha * c.alpha;
  c.nu_ref = (c.B - a2) / (1.0 - a2);
  const S gr = dt / (dt + 2.0 * tau_rot);
  const S gv = dt / (dt + 2.0 * tau_vib);
  const S evT = e_vib_T<S>(s, Tvib);
  S x = cv_vib_T<S>(s, Ttr);
  for (int it = 0; it < 50; ++it) {
    // T_check = T_tr + (gamma_tr-rot/2 (T_rot - T_tr) + gamma_tr-vib/2 (T_vib - T_tr)) / c_tr
    // with gamma / 2 c_tr = g c / den: one division per pass
    const S idn = 1.0 / (ctr + gr * crot + gv * x);
    const S Tc = Ttr + (gr * crot * (Trot - Ttr) + gv * x * (Tvib - Ttr)) * idn;
    const S scale = fmax(fabs(Tc), fabs(Tvib));
    S xn;
    double noise = 0.0;   // rounding of the secant (its numerator cancels near equilibrium)
    if (fabs(Tc - Tvib) <= 1e-9 * scale) {
      xn = cv_vib_T<S>(s, Tvib);
    } else {
      const S ec = e_vib_T<S>(s, Tc);
      xn = (ec - evT) / (Tc - Tvib);
      noise = 4.0 * 0x1p-52 * (::fabs((double)ec) + ::fabs((double)evT)) /
              ::fabs((double)(Tc - Tvib));
    }
    const S ch = fabs(xn - x);
    x = xn;
    if (ch <= 1e-14 * fabs(xn) || ch <= noise) break;
  }
  const S idn = 1.0 / (ctr + gr * crot + gv * x);
  c.g_tr_rot = 2.0 * gr * ctr * crot * idn;
  c.g_tr_vib = 2.0 * gv * ctr * x * idn;
  c.g_rot_vib = 2.0 * gr * gv * crot * x * idn;
  c.e_rot_tgt = crot * Trot + c.g_tr_rot * (Ttr - Trot) - c.g_rot_vib * (Trot - Tvib);
  c.e_vib_tgt = evT + c.g_tr_vib * (Ttr - Tvib) + c.g_rot_vib * (Trot - Tvib);
  // far above tau_rot the exchange terms can overshoot below zero: such a
  // target is 0 (the velocity rescale still conserves the cell's energy)
  c.tgt_clamped = false;
  if (c.e_rot_tgt < 0.0) { c.e_rot_tgt = S(0.0); c.tgt_clamped = true; }
  if (c.e_vib_tgt < 0.0) { c.e_vib_tgt = S(0.0); c.tgt_clamped = true; }
  return c;
}

typedef CellCoeffsT<double> CellCoeffs;

__device__ inline CellCoeffs cell_coeffs(const Species& s, double n, double dt, double Ttr,
                                         double Trot, double Tvib) {
  return cell_coeffs_t<double>(s, s.omega, s.Z_rot, n, dt, Ttr, Trot, Tvib);
}

// Relaxation temperatures (Eqs. T_tr_USP, T_rot_USP, T_vib_USP) for a given
// alpha; negative values are clamped to 0 and reported.
__device__ __forceinline__ void relax_temps(const Species& s, const CellCoeffs& c, double alpha,
                                            double Ttr, double Trot, double Tvib, double& ttr,
                                            double& trot, double& evr, bool& clamped) {
  const double R = gasR(s);
  const double oma2 = 1.0 - alpha * alpha;
  ttr = Ttr - (c.g_tr_rot * (Ttr - Trot) + c.g_tr_vib * (Ttr - Tvib)) / (oma2 * 1.5 * R);
  trot = Trot + (c.g_tr_rot * (Ttr - Trot) - c.g_rot_vib * (Trot - Tvib)) / (oma2 * R);
  evr = e_vib_T(s, Tvib) + (c.g_tr_vib * (Ttr - Tvib) + c.g_rot_vib * (Trot - Tvib)) / oma2;
  clamped = false;
  if (ttr < 0.0) { ttr = 0.0; clamped = true; }
  if (trot < 0.0) { trot = 0.0; clamped = true; }
  if (evr < 0.0) { evr = 0.0; clamped = true; }
}

// Cholesky factor (l00, l10, l11, l20, l21, l22) of (xx, yy, zz, xy, xz, yz).
template <typename T>
__device__ __forceinline__ bool chol3(const T* M, T* L) {
  if (!(M[0] > T(0))) return false;
  const T l00 = sqrt(M[0]);
  const T l10 = M[3] / l00, l20 = M[4] / l00;
  const T d1 = M[1] - l10 * l10;
  if (!(d1 > T(0))) return false;
  const T l11 = sqrt(d1);
  const T l21 = (M[5] - l20 * l10) / l11;
  const T d2 = M[2] - l20 * l20 - l21 * l21;
  if (!(d2 > T(0))) return false;
  L[0] = l00; L[1] = l10; L[2] = l11; L[3] = l20; L[4] = l21; L[5] = sqrt(d2);
  return true;
}

// extreme eigenvalues of a symmetric 3x3 matrix (trigonometric closed form)
template <typename T>
__device__ __forceinline__ void sym3_minmax(const T* P, T& lmin, T& lmax) {
  const T a = P[0], b = P[1], c = P[2], d = P[3], e = P[4], f = P[5];
  const T p1 = d * d + e * e + f * f;
  if (p1 == T(0)) {
    lmin = fmin(a, fmin(b, c));
    lmax = fmax(a, fmax(b, c));
    return;
  }
  const T q = (a + b + c) / T(3);
  const T p2 = (a - q) * (a - q) + (b - q) * (b - q) + (c - q) * (c - q) + T(2) * p1;
  const T p = sqrt(p2 / T(6));
  const T b11 = (a - q) / p, b22 = (b - q) / p, b33 = (c - q) / p;
  const T b12 = d / p, b13 = e / p, b23 = f / p;
  const T det = b11 * (b22 * b33 - b23 * b23) - b12 * (b12 * b33 - b23 * b13) +
                b13 * (b12 * b23 - b22 * b13);
  T r = det / T(2);
  r = fmin(T(1), fmax(T(-1), r));
  const T phi = acos(r) / T(3);
  lmax = q + T(2) * p * cos(phi);
  lmin = q + T(2) * p * cos(phi + T(2.0943951023931954923));
}

// The per-cell coefficients of cell_coeffs_t evaluated in FP32 (the FP32-state
// form of the 2D path, where 240,000 cells a step would keep the narrow FP64
// pipe busy): the same formulas in the same order, FP32 transcendentals, the
// T_1 fixed point to a relative change of 1e-6, the secant replaced by the
// derivative when T_check is within 2e-3 of T_vib.
struct CellCoeffsF {
  float mu_p, Pr, A, B, alpha, nu_ref, g_tr_rot, g_tr_vib, g_rot_vib, e_rot_tgt, e_vib_tgt;
  bool ok, tgt_clamped;
};

__device__ inline CellCoeffsF cell_coeffs_f32(const Species& s, double n, double dt_d, float Ttr,
                                              float Trot, float Tvib) {
  CellCoeffsF c;
  const float R = (float)s.R, ctr = 1.5f * R, crot = R;
  const float th = (float)s.theta_v, Rth = R * th;
  const float dt = (float)dt_d;
  const float p = (float)(n * kB) * Ttr;
  const float xw = expf((float)s.omega * logf(Ttr / (float)s.T_ref));
  c.mu_p = (float)s.mu_ref0 * xw / p;
  const float tau_c = (float)s.tauf0 * c.mu_p;
  float zr, zv;
  if (s.zmodel == 0) {
    zr = (float)s.Z_rot;
    zv = (float)s.Z_vib;
  } else {
    const float r = (float)s.T_star / Ttr;
    zr = (float)s.Zrot_inf /
         (1.0f + (float)(0.5 * kPi * 1.7724538509055159) * sqrtf(r) +
          (float)(kPi + 0.25 * kPi * kPi) * r);
    zv = ((float)s.C1 / ((float)s.Tref_w * xw)) * expf((float)s.C2 / cbrtf(Ttr)) +
         (float)s.zv_ht * sqrtf(Ttr / (float)s.T_ref) / xw;
  }
  const float tau_rot = zr * tau_c, tau_vib = zv * tau_c;
  float xi = 0.0f;
  if (Tvib > 0.0f) {
    const float x = th / Tvib;
    xi = x / expm1f(x);
  }
  c.Pr = (14.0f + 2.0f * xi) / (19.0f + 2.0f * xi);
  c.A = (2.0f * c.mu_p - c.Pr * dt) / (2.0f * c.mu_p + c.Pr * dt);
  c.B = (2.0f * c.mu_p - dt) / (2.0f * c.mu_p + dt);
  c.ok = c.A > -1.0f && c.A < 1.0f;
  c.alpha = c.ok ? cbrtf(c.A) : 0.0f;
  const float a2 = c.alpha * c.alpha;
  c.nu_ref = (c.B - a2) / (1.0f - a2);
  const float gr = dt / (dt + 2.0f * tau_rot);
  const float gv = dt / (dt + 2.0f * tau_vib);
  auto evib = [&](float T) { return T > 0.0f ? Rth / expm1f(th / T) : 0.0f; };
  auto cv = [&](float T) {
    if (T <= 0.0f) return 0.0f;
    const float h = 0.5f * th / T;
    const float q = h / sinhf(h);
    return R * q * q;
  };
  const float evT = evib(Tvib);
  float x = cv(Ttr);
  for (int it = 0; it < 50; ++it) {
    const float idn = 1.0f / (ctr + gr * crot + gv * x);
    const float Tc = Ttr + (gr * crot * (Trot - Ttr) + gv * x * (Tvib - Ttr)) * idn;
    const float scale = fmaxf(fabsf(Tc), fabsf(Tvib));
    float xn, noise = 0.0f;   // rounding of the secant
    if (fabsf(Tc - Tvib) <= 2e-3f * scale) {
      xn = cv(Tvib);
    } else {
      const float ec = evib(Tc);
      xn = (ec - evT) / (Tc - Tvib);
      noise = 4.0f * 0x1p-23f * (fabsf(ec) + fabsf(evT)) / fabsf(Tc - Tvib);
    }
    const float ch = fabsf(xn - x);
    x = xn;
    if (ch <= 1e-6f * fabsf(xn) || ch <= noise) break;
  }
  const float idn = 1.0f / (ctr + gr * crot + gv * x);
  c.g_tr_rot = 2.0f * gr * ctr * crot * idn;
  c.g_tr_vib = 2.0f * gv * ctr * x * idn;
  c.g_rot_vib = 2.0f * gr * gv * crot * x * idn;
  c.e_rot_tgt = crot * Trot + c.g_tr_rot * (Ttr - Trot) - c.g_rot_vib * (Trot - Tvib);
  c.e_vib_tgt = evT + c.g_tr_vib * (Ttr - Tvib) + c.g_rot_vib * (Trot - Tvib);
  c.tgt_clamped = false;
  if (c.e_rot_tgt < 0.0f) { c.e_rot_tgt = 0.0f; c.tgt_clamped = true; }
  if (c.e_vib_tgt < 0.0f) { c.e_vib_tgt = 0.0f; c.tgt_clamped = true; }
  return c;
}

// Drift-diffusion factor for one set of macroscopic fields: returns the
// alpha actually used and L with L L^T = tau D_tr (Eq. D_tr), applying the
// positivity adjustment of Sec. 3.A.3 when the Cholesky test fails (nu
// clamped by Eq. nu_USP_positivity with the current T_tr^rel and shrunk by
// 1 - 1e-6, alpha^2 from Eq. alpha_USP_positivity_1 clamped to
// [0, 1 - 1e-12], the sign giving the Pr nearest the target, up to four
// passes; then nu = 0 with alpha^2 = B, a failure only if T_tr^rel is 0).  Also returns the relaxation temperatures for that
// alpha.  chol_fix / fail report what happened.
// ---------------------------------------------------------------------------
// The plain FPM method (Sec. 2.B model, Sec. 2.C particle scheme), per cell
// in FP64: nu = 1 - 3/(2 Pr), tau = 2 mu (1 - nu)/p, alpha = exp(-dt/tau);
// relaxation energies of Eqs. T_tr_FPM, T_rot_FPM, T_vib_FPM with
// tau_rot = Z_rot tau_c, tau_vib = Z_vib tau_c (negative ones set to 0);
// the Cholesky factor of tau D_tr = R T_tr^rel I + nu (Pi - R T_tr I), nu
// limited to the admissible bound of Eq. nu_USP_positivity (times 1 - 1e-6)
// when it is not positive definite, then 0; the Gillespie rates per unit
// (I+1) and I times dt: lam_up = 2 dt ebar_rel / tau and
// lam_dn = 2 dt (1 + ebar_rel) / tau with ebar_rel = e_vib_rel / (R Theta);
// the conservation targets: the expected rotational and vibrational energies
// after dt, e_rel + (e^n - e_rel) alpha^2.
// ---------------------------------------------------------------------------
struct FpmCell {
  double alpha, L[6], Trot_rel, lam_up, lam_dn, e_rot_tgt, e_vib_tgt;
  bool ok, fixed, nu_zero, failed, clamped;
};

__device__ inline FpmCell fpm_cell(const Species& s, double n, double dt, const double* Pi,
                                   double Ttr, double Trot, double Tvib) {
  FpmCell o;
  o.fixed = o.nu_zero = o.failed = o.clamped = false;
  const double R = gasR(s);
  const double p = n * kB * Ttr;
  const double xw = exp(s.omega * log(Ttr / s.T_ref));
  const double mu = s.mu_ref0 * xw;
  const double tau_c = s.tauf0 * mu / p;
  double zr, zv;
  collision_numbers<double>(s, Ttr, xw, s.Z_rot, zr, zv);
  const double Pr = prandtl_T<double>(s, Tvib);
  const double nu0 = 1.0 - 3.0 / (2.0 * Pr);
  const double tau = 2.0 * mu * (1.0 - nu0) / p;
  o.ok = tau > 0.0;
  o.alpha = o.ok ? exp(-dt / tau) : 0.0;
  const double grot = tau / (2.0 * zr * tau_c), gvib = tau / (2.0 * zv * tau_c);
  const double ev = e_vib_T<double>(s, Tvib), evt = e_vib_T<double>(s, Ttr);
  double etr = 1.5 * R * Ttr + grot * (R * Trot - R * Ttr) + gvib * (ev - evt);
  double erot = R * Trot + grot * (R * Ttr - R * Trot);
  double evib = ev + gvib * (evt - ev);
  if (etr < 0.0) { etr = 0.0; o.clamped = true; }
  if (erot < 0.0) { erot = 0.0; o.clamped = true; }
  if (evib < 0.0) { evib = 0.0; o.clamped = true; }
  const double RT = R * Ttr, RTrel = etr / 1.5;
  o.Trot_rel = erot / R;
  const double ebar = evib / (R * s.theta_v);
  o.lam_up = 2.0 * dt * ebar / tau;
  o.lam_dn = 2.0 * dt * (1.0 + ebar) / tau;
  const double a2 = o.alpha * o.alpha;
  o.e_rot_tgt = erot + (R * Trot - erot) * a2;
  o.e_vib_tgt = evib + (ev - evib) * a2;
  double nu = nu0, M[6];
  auto fill = [&](double nu_) {
    M[0] = RTrel + nu_ * (Pi[0] - RT);
    M[1] = RTrel + nu_ * (Pi[1] - RT);
    M[2] = RTrel + nu_ * (Pi[2] - RT);
    M[3] = nu_ * Pi[3];
    M[4] = nu_ * Pi[4];
    M[5] = nu_ * Pi[5];
  };
  fill(nu);
  if (chol3(M, o.L)) return o;
  o.fixed = true;
  double lmin, lmax;
  sym3_minmax(Pi, lmin, lmax);
  if (nu <= 0.0) {
    if (lmax - RT > 0.0) nu = fmax(nu, -RTrel / (lmax - RT));
  } else {
    if (RT - lmin > 0.0) nu = fmin(nu, RTrel / (RT - lmin));
  }
  nu = nu * (1.0 - 1e-6);
  fill(nu);
  if (chol3(M, o.L)) return o;
  o.nu_zero = true;
  const double sq = RTrel > 0.0 ? sqrt(RTrel) : 0.0;
  o.failed = !(RTrel > 0.0);
  o.L[0] = sq; o.L[1] = 0.0; o.L[2] = sq; o.L[3] = 0.0; o.L[4] = 0.0; o.L[5] = sq;
  return o;
}

// Gillespie's direct method over one step (Sec. 2.C), time in units of dt:
// waiting time -ln(U1) / rate with rate = lam_up (I+1) + lam_dn I, the step
// ends once the time passes 1, else U2 < lam_up (I+1) / rate raises the
// level and otherwise lowers it.  Counter (pid, step, 8, k) draws the (U1,
// U2) pairs of transitions 2k and 2k+1.  Every operation is an explicit
// round-to-nearest one in the working precision, so the outcome is a fixed
// function of (I, lam_up, lam_dn, the draws) up to the logarithm.
constexpr int kGillespieCap = 4096;
template <typename T>
__device__ __forceinline__ int gillespie(int I, T lu, T ld, uint32_t pid, uint32_t step,
                                         const PhiloxRoundKeys& rk, uint32_t& fl) {
  T t = T(0);
  U4 w = {0u, 0u, 0u, 0u};
#pragma unroll 1
  for (int ev = 0; ev < kGillespieCap; ++ev) {
    if ((ev & 1) == 0) w = philox4x32_10(pid, step, PTAG_GILLESPIE, (uint32_t)(ev >> 1), rk);
    const T u1 = uniform_open<T>((ev & 1) ? w.z : w.x);
    const T u2 = uniform_open<T>((ev & 1) ? w.w : w.y);
    const T up = rn_mul(lu, rn_i2f(I + 1, T(0))), dn = rn_mul(ld, rn_i2f(I, T(0)));
    const T rate = rn_add(up, dn);
    if (!(rate > T(0))) return I;
    t = rn_add(t, rn_div(-log(u1), rate));
    if (t > T(1)) return I;
    I += (u2 < rn_div(up, rate)) ? 1 : -1;
  }
  fl |= F_SAMPLER_CAP;
  return I;
}

struct DriftDiff {
  double alpha, L[6], Ttr_rel, Trot_rel, evib_rel;
  bool fixed, nu_zero, failed, clamped;
};

__device__ inline DriftDiff drift_diffusion(const Species& s, const CellCoeffs& c, double dt,
                                            const double* Pi, double Ttr, double Trot, double Tvib) {
  DriftDiff o;
  const double R = gasR(s);
  o.alpha = c.alpha;
  o.fixed = false;
  o.nu_zero = false;
  o.failed = false;
  relax_temps(s, c, o.alpha, Ttr, Trot, Tvib, o.Ttr_rel, o.Trot_rel, o.evib_rel, o.clamped);
  double nu = c.nu_ref;
  double M[6];
  auto fill = [&](double nu_) {
    M[0] = R * o.Ttr_rel + nu_ * (Pi[0] - R * Ttr);
    M[1] = R * o.Ttr_rel + nu_ * (Pi[1] - R * Ttr);
    M[2] = R * o.Ttr_rel + nu_ * (Pi[2] - R * Ttr);
    M[3] = nu_ * Pi[3];
    M[4] = nu_ * Pi[4];
    M[5] = nu_ * Pi[5];
  };
  fill(nu);
  if (chol3(M, o.L)) return o;
  o.fixed = true;
  double lmin, lmax;
  sym3_minmax(Pi, lmin, lmax);
  bool ok = false;
  for (int pass = 0; pass < 4 && !ok; ++pass) {
    nu = c.nu_ref;
    if (c.nu_ref <= 0.0) {
      if (lmax - R * Ttr > 0.0) nu = fmax(nu, -R * o.Ttr_rel / (lmax - R * Ttr));
    } else {
      if (R * Ttr - lmin > 0.0) nu = fmin(nu, R * o.Ttr_rel / (R * Ttr - lmin));
    }
    nu = nu * (1.0 - 1e-6);
    double a2 = (nu - c.B) / (nu - 1.0);
    a2 = fmin(fmax(a2, 0.0), 1.0 - 1e-12);
    const double ap = sqrt(a2), am = -ap;
    const double prp = 2.0 * c.mu_p * (1.0 - ap * ap * ap) / (dt * (1.0 + ap * ap * ap));
    const double prm = 2.0 * c.mu_p * (1.0 - am * am * am) / (dt * (1.0 + am * am * am));
    o.alpha = (fabs(prm - c.Pr) < fabs(prp - c.Pr)) ? am : ap;
    bool cl;
    relax_temps(s, c, o.alpha, Ttr, Trot, Tvib, o.Ttr_rel, o.Trot_rel, o.evib_rel, cl);
    o.clamped = o.clamped || cl;
    fill(nu);
    ok = chol3(M, o.L);
  }
  if (!ok) {
    // nu = 0 with alpha^2 = B (Eq. alpha_USP_positivity_1 at nu = 0): inside
    // the admissible range whenever T_tr^rel > 0
    o.nu_zero = true;
    const double a2 = fmin(fmax(c.B, 0.0), 1.0 - 1e-12);
    const double ap = sqrt(a2), am = -ap;
    const double prp = 2.0 * c.mu_p * (1.0 - ap * ap * ap) / (dt * (1.0 + ap * ap * ap));
    const double prm = 2.0 * c.mu_p * (1.0 - am * am * am) / (dt * (1.0 + am * am * am));
    o.alpha = (fabs(prm - c.Pr) < fabs(prp - c.Pr)) ? am : ap;
    bool cl;
    relax_temps(s, c, o.alpha, Ttr, Trot, Tvib, o.Ttr_rel, o.Trot_rel, o.evib_rel, cl);
    o.clamped = o.clamped || cl;
    o.failed = !(o.Ttr_rel > 0.0);
    const double sq = o.failed ? 0.0 : sqrt(R * o.Ttr_rel);
    o.L[0] = sq; o.L[1] = 0.0; o.L[2] = sq; o.L[3] = 0.0; o.L[4] = 0.0; o.L[5] = sq;
  }
  return o;
}

}  // namespace usp
