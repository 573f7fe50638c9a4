// usp_spatial.cuh -- pieces shared by the spatial paths (1D channel and 2D
// plane) of the USP-FPM step: per-cell state, warp reductions, the
// per-particle collision of Sec. 4.D with fields at the particle, and the
// per-cell conservation kernels of Sec. 4.C.  Included by one translation
// unit each; everything is internal to it.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "usp_device.cuh"
#include "usp_dual.cuh"

namespace {

using namespace usp;

constexpr int kNF = 13;            // U(3), T_tr, T_rot, T_vib, Pi(6)
constexpr int kRB = 256;           // radix block
constexpr int kRPT = 16;           // keys per thread per radix block
constexpr int kChunk = kRB * kRPT;
constexpr int kNAcc = 12;          // time-average sums per cell
constexpr int kWallHitCap = 16;
constexpr uint32_t PTAG_WALL_A = 2u, PTAG_WALL_B = 3u;

// Per-cell state; S = double (plain forms) or a derivative number.  T_vib
// comes from the mean level alone (levels carry no derivative).
template <typename S>
struct ChCellT {
  S U[3], Pi[6];
  S Ttr, Trot;
  double Tvib, ebar, n;
  S alpha, nu_ref, B, mu_p, Pr, gtr, gtv, grv;
  S e_rot_tgt, e_vib_tgt;
  S Un[3], Us[3], s, r;   // pending rescale: c = Un + s (c* - Us), eps = r eps*
  long long off, N;
  int active, maxI;
  int usable, pad;   // usable as a reconstruction neighbour (plane path)
};


template <typename S>
struct ChSumsT {
  S v[10];
  unsigned long long I;
  long long net;
  int maxI, pad;
};

__device__ __forceinline__ unsigned lane_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename V>
__device__ __forceinline__ dual::Dual<V> wsum(dual::Dual<V> v) {
  v.v = wsum(v.v);
  for (int k = 0; k < kND; ++k) v.d[k] = wsum(v.d[k]);
  return v;
}

// e_vib in the working precision
template <typename T>
__device__ __forceinline__ T evib_t(const T& Rth, const T& theta, const T& Tv) {
  return Tv > T(0) ? Rth / expm1(theta / Tv) : T(0);
}


// add a quantity to block 0 of an accumulator and, for derivative numbers,
// its derivatives to blocks 1..3 (stride blk)
__device__ __forceinline__ void acc_add(double* a, size_t, double q) { atomicAdd(a, q); }
__device__ __forceinline__ void acc_add(double* a, size_t blk, const D3& q) {
  atomicAdd(a, q.v);
  for (int k = 0; k < kND; ++k) atomicAdd(a + (k + 1) * blk, q.d[k]);
}


template <typename T>
__device__ __forceinline__ bool chol3_t(const T* M, T* L) {
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

template <typename T, typename P_>
__device__ __forceinline__ void relax_t(const P_& P, T alpha, const T* f, T& ttr, T& trot,
                                        T& evr, bool& cl) {
  const T oma2 = T(1) - alpha * alpha;
  ttr = f[3] - (P.gtr * (f[3] - f[4]) + P.gtv * (f[3] - f[5])) / (oma2 * T(1.5) * P.R);
  trot = f[4] + (P.gtr * (f[3] - f[4]) - P.grv * (f[4] - f[5])) / (oma2 * P.R);
  evr = evib_t(P.R * P.theta, P.theta, f[5]) + (P.gtv * (f[3] - f[5]) + P.grv * (f[4] - f[5])) / oma2;
  cl = false;
  if (ttr < T(0)) { ttr = T(0); cl = true; }
  if (trot < T(0)) { trot = T(0); cl = true; }
  if (evr < T(0)) { evr = T(0); cl = true; }
}


// FP32 forms of relax_t / chol3_t / the jump parameters with one correctly
// rounded reciprocal (or reciprocal square root) in place of each group of
// divisions.  Used by the FP32 plane path, whose per-particle arithmetic is
// compared with the oracle statistically; the other forms keep the IEEE
// divisions operation for operation.
__device__ __forceinline__ bool chol3_fast(const float* M, float* L) {
  if (!(M[0] > 0.f)) return false;
  const float r0 = rsqrtf(M[0]);
  const float l00 = M[0] * r0;
  const float l10 = M[3] * r0, l20 = M[4] * r0;
  const float d1 = M[1] - l10 * l10;
  if (!(d1 > 0.f)) return false;
  const float r1 = rsqrtf(d1);
  const float l11 = d1 * r1;
  const float l21 = (M[5] - l20 * l10) * r1;
  const float d2 = M[2] - l20 * l20 - l21 * l21;
  if (!(d2 > 0.f)) return false;
  L[0] = l00; L[1] = l10; L[2] = l11; L[3] = l20; L[4] = l21; L[5] = sqrtf(d2);
  return true;
}

template <typename P_>
__device__ __forceinline__ void relax_fast(const P_& P, float alpha, const float* f, float& ttr,
                                           float& trot, float& evr, bool& cl) {
  const float ioR = __frcp_rn((1.f - alpha * alpha) * P.R);   // 1 / ((1 - alpha^2) R)
  ttr = f[3] - (P.gtr * (f[3] - f[4]) + P.gtv * (f[3] - f[5])) * ioR * (2.f / 3.f);
  trot = f[4] + (P.gtr * (f[3] - f[4]) - P.grv * (f[4] - f[5])) * ioR;
  const float ev = f[5] > 0.f ? P.R * P.theta * __frcp_rn(expm1f(P.theta * __frcp_rn(f[5])))
                              : 0.f;
  evr = ev + (P.gtv * (f[3] - f[5]) + P.grv * (f[4] - f[5])) * (ioR * P.R);
  cl = false;
  if (ttr < 0.f) { ttr = 0.f; cl = true; }
  if (trot < 0.f) { trot = 0.f; cl = true; }
  if (evr < 0.f) { evr = 0.f; cl = true; }
}

template <bool kFast, typename T, typename P_>
__device__ __forceinline__ void relax_sel(const P_& P, T alpha, const T* f, T& ttr, T& trot,
                                          T& evr, bool& cl) {
  if constexpr (kFast) relax_fast(P, alpha, f, ttr, trot, evr, cl);
  else relax_t(P, alpha, f, ttr, trot, evr, cl);
}

template <bool kFast, typename T>
__device__ __forceinline__ bool chol3_sel(const T* M, T* L) {
  if constexpr (kFast) return chol3_fast(M, L);
  else return chol3_t(M, L);
}

// Counts kept per thread by the particle collision and reduced per warp.
struct CollideTally {
  uint32_t fl;
  unsigned long long nfix, ncl, npb, nnz;
};

// One particle through the collision step of Sec. 4.D with the fields f at
// its position (U(3), T_tr, T_rot, T_vib, Pi(6)) and the cell coefficients
// of P: relaxation temperatures, M = tau D_tr and its Cholesky factor with
// the Sec. 3.A.3 adjustment (four passes, then nu = 0 with alpha^2 = B),
// Eqs. update_ci / update_erot / update_evib.  Returns the new level.
template <bool kFast = false, typename T, typename P_>
__device__ __forceinline__ int collide_particle_t(const P_& P, const T* f, T& vx, T& vy, T& vz,
                                                  T& e, int I, uint32_t id, uint32_t step,
                                                  const PhiloxRoundKeys& rk, CollideTally& t) {
  static_assert(!kFast || sizeof(T) == 4, "the fast forms are FP32");
  T alpha = P.alpha, nu = P.nu_ref, ttr, trot, evr;
  bool cl;
  relax_sel<kFast>(P, alpha, f, ttr, trot, evr, cl);
  const T RT = P.R * f[3];
  T M[6], L[6];
  auto fill = [&](T nu_) {
    M[0] = P.R * ttr + nu_ * (f[6] - RT);
    M[1] = P.R * ttr + nu_ * (f[7] - RT);
    M[2] = P.R * ttr + nu_ * (f[8] - RT);
    M[3] = nu_ * f[9]; M[4] = nu_ * f[10]; M[5] = nu_ * f[11];
  };
  fill(nu);
  if (!chol3_sel<kFast>(M, L)) {
    ++t.nfix;
    T lmin, lmax;
    sym3_minmax(f + 6, lmin, lmax);
    bool ok = false;
    for (int pass = 0; pass < 4 && !ok; ++pass) {
      nu = P.nu_ref;
      if (P.nu_ref <= T(0)) {
        if (lmax - RT > T(0)) nu = fmax(nu, -P.R * ttr / (lmax - RT));
      } else {
        if (RT - lmin > T(0)) nu = fmin(nu, P.R * ttr / (RT - lmin));
      }
      nu = nu * (T(1) - T(1e-6));
      T a2 = (nu - P.B) / (nu - T(1));
      a2 = fmin(fmax(a2, T(0)), T(1) - (sizeof(T) == 4 ? T(1e-7) : T(1e-12)));
      const T ap = sqrt(a2), am = -ap;
      const T prp = T(2) * P.mu_p * (T(1) - ap * ap * ap) / (P.dt * (T(1) + ap * ap * ap));
      const T prm_ = T(2) * P.mu_p * (T(1) - am * am * am) / (P.dt * (T(1) + am * am * am));
      alpha = (fabs(prm_ - P.Pr) < fabs(prp - P.Pr)) ? am : ap;
      bool cl2;
      relax_sel<kFast>(P, alpha, f, ttr, trot, evr, cl2);
      cl = cl || cl2;
      fill(nu);
      ok = chol3_sel<kFast>(M, L);
    }
    if (!ok) {
      // nu = 0 with alpha^2 = B, admissible whenever T_tr^rel > 0
      ++t.nnz;
      const T a2 = fmin(fmax(P.B, T(0)), T(1) - (sizeof(T) == 4 ? T(1e-7) : T(1e-12)));
      const T ap = sqrt(a2), am = -ap;
      const T prp = T(2) * P.mu_p * (T(1) - ap * ap * ap) / (P.dt * (T(1) + ap * ap * ap));
      const T prm_ = T(2) * P.mu_p * (T(1) - am * am * am) / (P.dt * (T(1) + am * am * am));
      alpha = (fabs(prm_ - P.Pr) < fabs(prp - P.Pr)) ? am : ap;
      bool cl2;
      relax_sel<kFast>(P, alpha, f, ttr, trot, evr, cl2);
      cl = cl || cl2;
      if (!(ttr > T(0))) t.fl |= F_CHOL_FAIL_AFTER_FIX;
      const T sq = ttr > T(0) ? sqrt(P.R * ttr) : T(0);
      L[0] = sq; L[1] = T(0); L[2] = sq; L[3] = T(0); L[4] = T(0); L[5] = sq;
    }
  }
  if (cl) { t.fl |= F_TREL_CLAMP; ++t.ncl; }
  // draws
  T g0, g1, g2, g3;
  uint32_t j5, j6;
  particle_draws(id, step, rk, g0, g1, g2, g3, j5, j6);
  // Eq. update_ci about the interpolated bulk velocity
  const T a2 = alpha * alpha, sq = sqrt(T(1) - a2);
  const T v0 = f[0] + alpha * (vx - f[0]) + sq * (L[0] * g0);
  const T v1 = f[1] + alpha * (vy - f[1]) + sq * (L[1] * g0 + L[2] * g1);
  const T v2 = f[2] + alpha * (vz - f[2]) + sq * (L[3] * g0 + L[4] * g1 + L[5] * g2);
  vx = v0; vy = v1; vz = v2;
  // Eq. update_erot
  const T a = P.R * trot * (T(1) - a2) / T(2);
  const T root = sqrt(e) * alpha + sqrt(a) * g3;
  e = a + root * root;
  // Eq. update_evib
  T eb, p_nb;
  if constexpr (kFast) {
    eb = evr * __frcp_rn(P.R * P.theta);
    p_nb = __frcp_rn(T(1) + eb * (T(1) - a2));
  } else {
    eb = evr / (P.R * P.theta);
    p_nb = T(1) / (T(1) + eb * (T(1) - a2));
  }
  const T p_b = (T(1) + eb) * (T(1) - a2);
  uint32_t f1 = 0;
  const int up = sample_nb<T>(I + 1, p_nb, jump_uniform<T>(j5), f1);
  const int dn = sample_b<T>(I, p_b, jump_uniform<T>(j6), f1);
  if (f1 & F_PB_CLAMP) ++t.npb;
  t.fl |= f1;
  return I + up - dn;
}

// Block-level tally of the status word and counters: kernels over many cells
// add into shared memory and flush once per block, so that a counter bumped
// by a large share of 240,000 cells does not serialise on one global address.
struct BlockTally {
  unsigned long long cnt[NCOUNTERS];
  uint32_t fl;
};
__device__ __forceinline__ void tally_init(BlockTally& t) {
  for (int i = threadIdx.x; i < NCOUNTERS; i += blockDim.x) t.cnt[i] = 0ull;
  if (threadIdx.x == 0) t.fl = 0u;
  __syncthreads();
}
__device__ __forceinline__ void tally_add(BlockTally& t, int k, unsigned long long v) {
  if (v) atomicAdd(&t.cnt[k], v);
}
__device__ __forceinline__ void tally_or(BlockTally& t, uint32_t f) {
  if (f) atomicOr(&t.fl, f);
}
__device__ __forceinline__ void tally_flush(BlockTally& t, uint32_t* flags,
                                            unsigned long long* counters) {
  __syncthreads();
  for (int i = threadIdx.x; i < NCOUNTERS; i += blockDim.x)
    if (t.cnt[i]) atomicAdd(&counters[i], t.cnt[i]);
  if (threadIdx.x == 0 && t.fl) atomicOr(flags, t.fl);
}

// warp-per-cell and thread-per-cell grid-stride indices
__device__ __forceinline__ int warp_global() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int warps_total() { return (gridDim.x * blockDim.x) >> 5; }

// vibrational +-1 correction (Sec. 4.C), one warp per cell; same acceptance
// rule as the one-at-a-time loop (see the homogeneous path)
template <typename S>
__global__ void ch_levelfix(int ny, int cpw, const ChCellT<S>* __restrict__ cells,
                            ChSumsT<S>* __restrict__ sums,
                            int* __restrict__ lev, const long long* __restrict__ dstep, Species sp,
                            uint32_t k0, uint32_t k1, uint32_t* flags,
                            unsigned long long* counters) {
  __shared__ BlockTally tal;
  tally_init(tal);
  const int lane = threadIdx.x & 31;
  const uint32_t step = (uint32_t)*dstep;
  const double Rth = gasR(sp) * sp.theta_v;
  for (long long c0 = (long long)warp_global() * cpw; c0 < ny;
       c0 += (long long)warps_total() * cpw) {
    const int ng = (int)(ny - c0 < cpw ? ny - c0 : cpw);
    // I_Delta of Sec. 4.C for cell c0 + lane (FP64, one cell per lane)
    long long myId = 0;
    if (lane < ng) {
      const long long c = c0 + lane;
      const ChCellT<S>& cs = cells[c];
      if (cs.active) {
        const U4 w = philox4x32_10((uint32_t)c, step, CTAG_IDELTA, 0u, k0, k1);
        const double u = uniform_open<double>(w.x);
        myId = (long long)floor((double)cs.N * value(cs.e_vib_tgt) / Rth -
                                (double)(long long)sums[c].I + u);
      }
    }
    for (int g = 0; g < ng; ++g) {
      const long long Id = __shfl_sync(0xffffffffu, myId, g);
      const long long c = c0 + g;
      const ChCellT<S>& cs = cells[c];
      if (!cs.active) continue;
      const long long N = cs.N;
      long long remaining = Id, draws = 0, net = 0;
      const long long cap = 64 * N;
      int* lv = lev + cs.off;
      while (remaining != 0 && draws < cap) {
        const long long j = draws + lane;
        const U4 w = philox4x32_10((uint32_t)c, step, CTAG_PICK, (uint32_t)(j >> 2), k0, k1);
        const uint32_t word = (j & 3) == 0 ? w.x : (j & 3) == 1 ? w.y : (j & 3) == 2 ? w.z : w.w;
        const long long k = (long long)(((unsigned long long)word * (unsigned long long)N) >> 32);
        const bool valid = j < cap;
        bool accept;
        if (remaining > 0) {
          accept = valid;
        } else {
          const int cur = valid ? __ldcg(&lv[k]) : 0;
          const unsigned grp = __match_any_sync(0xffffffffu, valid ? k : -1ll);
          accept = valid && __popc(grp & lane_lt()) < cur;
        }
        const unsigned am = __ballot_sync(0xffffffffu, accept);
        const long long need = remaining > 0 ? remaining : -remaining;
        const int nacc = __popc(am);
        const int take = (int)(nacc < need ? nacc : need);
        const bool eff = accept && __popc(am & lane_lt()) < take;
        __syncwarp();
        if (eff) atomicAdd(&lv[k], remaining > 0 ? 1 : -1);
        __syncwarp();
        long long used = 32;
        if (take == need && take > 0) {
          unsigned m = am;
          for (int i = 1; i < take; ++i) m &= m - 1;
          used = __ffs((int)m);
        }
        if (draws + used > cap) used = cap - draws;
        draws += used;
        if (remaining > 0) { remaining -= take; net += take; }
        else { remaining += take; net -= take; }
      }
      if (lane == 0) {
        if (remaining != 0) tally_or(tal, (uint32_t)F_VIB_LOOP_CAP);
        tally_add(tal, C_VIB_DRAWS, (unsigned long long)draws);
        sums[c].net = net;
      }
    }
  }
  tally_flush(tal, flags, counters);
}

// rescale factors of Sec. 4.C, kept pending for the next move; the step
// counter advances after the last reader of this step
template <typename S>
__global__ void ch_update(int ny, ChCellT<S>* __restrict__ cells,
                          const ChSumsT<S>* __restrict__ sums, long long* dstep, Species sp,
                          uint32_t* flags, unsigned long long* counters,
                          float* __restrict__ pend) {
  __shared__ BlockTally tal;
  tally_init(tal);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ny; c += gridDim.x * blockDim.x) {
    ChCellT<S>& cs = cells[c];
    if (!cs.active) continue;
    const double R = gasR(sp), Rth = R * sp.theta_v;
    const ChSumsT<S>& sm = sums[c];
    const double invN = 1.0 / (double)cs.N;
    const double sumI = (double)((long long)sm.I + sm.net);
    const S er_star = sm.v[9] * invN;
    const S r = er_star > 0.0 ? cs.e_rot_tgt / er_star : S(1.0);
    const S e_rot_new = r * er_star;
    const double e_vib_new = Rth * sumI * invN;
    const S m0 = sm.v[0] * invN, m1 = sm.v[1] * invN, m2 = sm.v[2] * invN;
    const S etr_star = 0.5 * (sm.v[3] * invN - m0 * m0 + sm.v[4] * invN - m1 * m1 +
                              sm.v[5] * invN - m2 * m2);
    const S e_tr_n = 0.5 * (cs.Pi[0] + cs.Pi[1] + cs.Pi[2]);
    const S rad = (e_tr_n + R * cs.Trot + Rth * cs.ebar - e_rot_new - e_vib_new) / etr_star;
    S Us[3] = {cs.U[0] + m0, cs.U[1] + m1, cs.U[2] + m2};
    if (!(etr_star > 0.0) || !(rad > 0.0)) {
      tally_or(tal, (uint32_t)F_NEG_RADICAND);
      tally_add(tal, C_NEG_RADICAND, 1ull);
      for (int i = 0; i < 3; ++i) { cs.Un[i] = Us[i]; cs.Us[i] = Us[i]; }
      cs.s = S(1.0);
    } else {
      for (int i = 0; i < 3; ++i) { cs.Un[i] = cs.U[i]; cs.Us[i] = Us[i]; }
      cs.s = sqrt(rad);
    }
    cs.r = r;
    cs.maxI = sm.maxI + 1;
    if (pend) {   // FP32 copy for the next move of an FP32 state
      float* pc = pend + (size_t)c * 8;
      for (int i = 0; i < 3; ++i) {
        pc[i] = (float)value(cs.Un[i]);
        pc[3 + i] = (float)value(cs.Us[i]);
      }
      pc[6] = (float)value(cs.s);
      pc[7] = (float)value(cs.r);
    }
  }
  tally_flush(tal, flags, counters);
  if (blockIdx.x == 0 && threadIdx.x == 0) *dstep += 1;
}

// ch_levelfix and ch_update in one pass (FP64 cell records): the warp makes
// the +-1 corrections of its 32 cells one after the other, lane k keeping
// cell k's net change, then every lane computes its cell's rescale factors.
// F32: the factors in FP32 arithmetic (the FP32 state's own precision) from
// the FP64 sums.  dstep[0] is the step counter, dstep[1] counts finished
// blocks: the last block to finish advances the step, after every block has
// read it.
template <bool F32>
__global__ void ch_fix_update(int ncell, ChCellT<double>* __restrict__ cells,
                              const ChSumsT<double>* __restrict__ sums, int* __restrict__ lev,
                              long long* dstep, Species sp, uint32_t k0, uint32_t k1,
                              uint32_t* flags, unsigned long long* counters,
                              float* __restrict__ pend) {
  __shared__ BlockTally tal;
  tally_init(tal);
  const int lane = threadIdx.x & 31;
  const uint32_t step = (uint32_t)dstep[0];
  const double Rth = gasR(sp) * sp.theta_v;
  for (long long c0 = (long long)warp_global() * 32; c0 < ncell;
       c0 += (long long)warps_total() * 32) {
    const int ng = (int)(ncell - c0 < 32 ? ncell - c0 : 32);
    // I_Delta of Sec. 4.C for cell c0 + lane (FP64, one cell per lane)
    long long myId = 0, mynet = 0;
    if (lane < ng) {
      const long long c = c0 + lane;
      const ChCellT<double>& cs = cells[c];
      if (cs.active) {
        const U4 w = philox4x32_10((uint32_t)c, step, CTAG_IDELTA, 0u, k0, k1);
        const double u = uniform_open<double>(w.x);
        myId = (long long)floor((double)cs.N * cs.e_vib_tgt / Rth - (double)(long long)sums[c].I +
                                u);
      }
    }
    for (int g = 0; g < ng; ++g) {
      const long long Id = __shfl_sync(0xffffffffu, myId, g);
      const long long c = c0 + g;
      const ChCellT<double>& cs = cells[c];
      if (!cs.active) continue;
      const long long N = cs.N;
      long long remaining = Id, draws = 0, net = 0;
      const long long cap = 64 * N;
      int* lv = lev + cs.off;
      while (remaining != 0 && draws < cap) {
        const long long j = draws + lane;
        const U4 w = philox4x32_10((uint32_t)c, step, CTAG_PICK, (uint32_t)(j >> 2), k0, k1);
        const uint32_t word = (j & 3) == 0 ? w.x : (j & 3) == 1 ? w.y : (j & 3) == 2 ? w.z : w.w;
        const long long k = (long long)(((unsigned long long)word * (unsigned long long)N) >> 32);
        const bool valid = j < cap;
        bool accept;
        if (remaining > 0) {
          accept = valid;
        } else {
          const int cur = valid ? __ldcg(&lv[k]) : 0;
          const unsigned grp = __match_any_sync(0xffffffffu, valid ? k : -1ll);
          accept = valid && __popc(grp & lane_lt()) < cur;
        }
        const unsigned am = __ballot_sync(0xffffffffu, accept);
        const long long need = remaining > 0 ? remaining : -remaining;
        const int nacc = __popc(am);
        const int take = (int)(nacc < need ? nacc : need);
        const bool eff = accept && __popc(am & lane_lt()) < take;
        __syncwarp();
        if (eff) atomicAdd(&lv[k], remaining > 0 ? 1 : -1);
        __syncwarp();
        long long used = 32;
        if (take == need && take > 0) {
          unsigned m = am;
          for (int i = 1; i < take; ++i) m &= m - 1;
          used = __ffs((int)m);
        }
        if (draws + used > cap) used = cap - draws;
        draws += used;
        if (remaining > 0) { remaining -= take; net += take; }
        else { remaining += take; net -= take; }
      }
      if (lane == g) mynet = net;
      if (lane == 0) {
        if (remaining != 0) tally_or(tal, (uint32_t)F_VIB_LOOP_CAP);
        tally_add(tal, C_VIB_DRAWS, (unsigned long long)draws);
      }
    }
    // the rescale factors of Sec. 4.C for cell c0 + lane
    if (lane >= ng) continue;
    const long long c = c0 + lane;
    ChCellT<double>& cs = cells[c];
    if (!cs.active) continue;
    const ChSumsT<double>& sm = sums[c];
    using V = std::conditional_t<F32, float, double>;
    const V R = (V)gasR(sp), RthV = (V)Rth;
    const V invN = V(1) / (V)cs.N;
    const V sumI = (V)((long long)sm.I + mynet);
    const V er_star = (V)sm.v[9] * invN;
    const V r = er_star > V(0) ? (V)cs.e_rot_tgt / er_star : V(1);
    const V e_rot_new = r * er_star;
    const V e_vib_new = RthV * sumI * invN;
    const V m0 = (V)sm.v[0] * invN, m1 = (V)sm.v[1] * invN, m2 = (V)sm.v[2] * invN;
    const V etr_star = V(0.5) * ((V)sm.v[3] * invN - m0 * m0 + (V)sm.v[4] * invN - m1 * m1 +
                                 (V)sm.v[5] * invN - m2 * m2);
    const V e_tr_n = V(0.5) * ((V)cs.Pi[0] + (V)cs.Pi[1] + (V)cs.Pi[2]);
    const V rad = (e_tr_n + R * (V)cs.Trot + RthV * (V)cs.ebar - e_rot_new - e_vib_new) / etr_star;
    const V U0 = (V)cs.U[0], U1 = (V)cs.U[1], U2 = (V)cs.U[2];
    const V Us[3] = {U0 + m0, U1 + m1, U2 + m2};
    V Un[3] = {U0, U1, U2}, sc = V(1);
    if (!(etr_star > V(0)) || !(rad > V(0))) {
      tally_or(tal, (uint32_t)F_NEG_RADICAND);
      tally_add(tal, C_NEG_RADICAND, 1ull);
      for (int i = 0; i < 3; ++i) Un[i] = Us[i];
    } else {
      sc = sqrt(rad);
    }
    for (int i = 0; i < 3; ++i) { cs.Un[i] = Un[i]; cs.Us[i] = Us[i]; }
    cs.s = sc;
    cs.r = r;
    cs.maxI = sm.maxI + 1;
    if (pend) {   // FP32 copy for the next move of an FP32 state
      float* pc = pend + (size_t)c * 8;
      for (int i = 0; i < 3; ++i) {
        pc[i] = (float)Un[i];
        pc[3 + i] = (float)Us[i];
      }
      pc[6] = (float)sc;
      pc[7] = (float)r;
    }
  }
  tally_flush(tal, flags, counters);
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(reinterpret_cast<unsigned long long*>(dstep + 1), 1ull) ==
        (unsigned long long)gridDim.x - 1) {
      dstep[1] = 0;
      dstep[0] += 1;
    }
  }
}


// ---------------------------------------------------------------------------
// per-cell moments and coefficients
// ---------------------------------------------------------------------------
// A warp takes cpw consecutive cells (1 or 32): the particle sums of each
// cell are warp-wide FP32 (or working-precision) reductions, kept by lane k
// for the k-th cell; the FP64 per-cell arithmetic then runs one cell per lane,
// so each FP64 warp instruction serves up to 32 cells on the narrow FP64 pipe.
template <typename T, typename S>
__global__ void ch_moments(int ny, int cpw, const long long* __restrict__ off,
                           const double* __restrict__ af, const T* __restrict__ cx,
                           const T* __restrict__ cy, const T* __restrict__ cz,
                           const T* __restrict__ er, const int* __restrict__ lev,
                           ChCellT<S>* __restrict__ cells, Species sp,
                           unsigned long long* counters, float* __restrict__ pend,
                           T* __restrict__ fT, int* __restrict__ usable_c) {
  __shared__ BlockTally tal;
  tally_init(tal);
  const int lane = threadIdx.x & 31;
  const double R = gasR(sp);
  constexpr bool f32 = sizeof(T) == 4;
  for (long long c0 = (long long)warp_global() * cpw; c0 < ny;
       c0 += (long long)warps_total() * cpw) {
    const int ng = (int)(ny - c0 < cpw ? ny - c0 : cpw);
    T k0 = T(0), k1 = T(0), k2 = T(0), ke = T(0), kq[6];
    long long kl = 0, kb = 0, kN = 0;
    for (int i = 0; i < 6; ++i) kq[i] = T(0);
    // the task's cell offsets (lane k: start of cell k), and each cell's first
    // 32 particles held one per lane, loaded one cell ahead so that their
    // latency overlaps the previous cell's reductions; the sums keep the
    // order of a plain strided loop
    const long long offl = lane < ng ? off[c0 + lane] : 0;
    const long long offend = off[c0 + ng];
    auto cell_b = [&](int g) { return __shfl_sync(0xffffffffu, offl, g); };
    auto cell_e = [&](int g) { return g + 1 < ng ? __shfl_sync(0xffffffffu, offl, g + 1) : offend; };
    T nx0 = T(0), ny0 = T(0), nz0 = T(0), ne0 = T(0);
    int nl0 = 0;
    auto first = [&](int g) {
      const long long j = cell_b(g) + lane;
      if (j < cell_e(g)) {
        nx0 = cx[j]; ny0 = cy[j]; nz0 = cz[j]; ne0 = er[j]; nl0 = lev[j];
      } else {
        nx0 = ny0 = nz0 = ne0 = T(0); nl0 = 0;
      }
    };
    first(0);
    for (int g = 0; g < ng; ++g) {
      const long long b = cell_b(g), e = cell_e(g), N = e - b;
      const bool has = lane < N;
      const T fx = nx0, fy = ny0, fz = nz0, fe = ne0;
      const int fl = nl0;
      if (g + 1 < ng) first(g + 1);
      T a0 = T(0), a1 = T(0), a2 = T(0), ae = T(0);
      long long al = 0;
      if (has) { a0 += fx; a1 += fy; a2 += fz; ae += fe; al += fl; }
      for (long long j = b + 32 + lane; j < e; j += 32) {
        a0 += cx[j]; a1 += cy[j]; a2 += cz[j]; ae += er[j]; al += lev[j];
      }
      const T t0 = wsum(a0), t1 = wsum(a1), t2 = wsum(a2), te = wsum(ae);
      const long long sl = wsum(al);
      // the reference mean of the second pass (an FP32 state keeps FP32)
      T m0, m1, m2;
      if constexpr (f32) {
        const float fn = N > 0 ? (float)N : 1.0f;
        m0 = t0 / fn; m1 = t1 / fn; m2 = t2 / fn;
      } else {
        const double inv = N > 0 ? 1.0 / (double)N : 0.0;
        m0 = (T)(S(t0) * inv); m1 = (T)(S(t1) * inv); m2 = (T)(S(t2) * inv);
      }
      T p[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
      if (has) {
        const T C0 = fx - m0, C1 = fy - m1, C2 = fz - m2;
        p[0] += C0 * C0; p[1] += C1 * C1; p[2] += C2 * C2;
        p[3] += C0 * C1; p[4] += C0 * C2; p[5] += C1 * C2;
      }
      for (long long j = b + 32 + lane; j < e; j += 32) {
        const T C0 = cx[j] - m0, C1 = cy[j] - m1, C2 = cz[j] - m2;
        p[0] += C0 * C0; p[1] += C1 * C1; p[2] += C2 * C2;
        p[3] += C0 * C1; p[4] += C0 * C2; p[5] += C1 * C2;
      }
      T q[6];
      for (int i = 0; i < 6; ++i) q[i] = wsum(p[i]);
      if (lane == g) {
        k0 = t0; k1 = t1; k2 = t2; ke = te; kl = sl; kb = b; kN = N;
        for (int i = 0; i < 6; ++i) kq[i] = q[i];
      }
    }
    if (lane >= ng) continue;
    const long long c = c0 + lane;
    const long long N = kN;
    const double inv = N > 0 ? 1.0 / (double)N : 0.0;
    const S s0 = S(k0), s1 = S(k1), s2 = S(k2), se = S(ke);
    S P[6];
    for (int i = 0; i < 6; ++i) P[i] = S(kq[i]) * inv;
    if (pend) {   // identity pending rescale (FP32 copy)
      float* pc = pend + (size_t)c * 8;
      pc[0] = pc[1] = pc[2] = pc[3] = pc[4] = pc[5] = 0.0f;
      pc[6] = pc[7] = 1.0f;
    }
    ChCellT<S>& cs = cells[c];
    cs.off = kb;
    cs.N = N;
    cs.active = N >= 2;
    // a neighbour for the reconstruction of Sec. 3.B: two or more particles
    // and not cut by a body (af: fluid fraction, null = every cell whole)
    cs.usable = N >= 2 && (!af || af[c] >= 1.0);
    if (usable_c) usable_c[c] = cs.usable;
    cs.U[0] = s0 * inv; cs.U[1] = s1 * inv; cs.U[2] = s2 * inv;
    // identity pending rescale until the cell is updated
    for (int i = 0; i < 3; ++i) { cs.Un[i] = S(0.0); cs.Us[i] = S(0.0); }
    cs.s = S(1.0);
    cs.r = S(1.0);
    if (!cs.active) {
      tally_add(tal, C_SKIPPED_CELLS, 1ull);
      continue;
    }
    for (int i = 0; i < 6; ++i) cs.Pi[i] = P[i];
    cs.Ttr = (P[0] + P[1] + P[2]) / (3.0 * R);
    cs.Trot = se * inv / R;
    cs.ebar = (double)kl * inv;
    cs.Tvib = T_vib_of_level<double>(sp, cs.ebar);
    if (fT) {   // the 13 fields in the particle precision, for the stencils
      T* o = fT + (size_t)c * kNF;
      for (int i = 0; i < 3; ++i) o[i] = (T)cs.U[i];
      o[3] = (T)cs.Ttr; o[4] = (T)cs.Trot; o[5] = (T)cs.Tvib;
      for (int i = 0; i < 6; ++i) o[6 + i] = (T)cs.Pi[i];
    }
  }
  tally_flush(tal, nullptr, counters);
}

template <typename S>
__global__ void ch_coeffs(int ny, double F_num, double vol, const double* __restrict__ af,
                          double dt, ChCellT<S>* __restrict__ cells, Species sp, S omega, S zrot,
                          uint32_t* flags, unsigned long long* counters) {
  __shared__ BlockTally tal;
  tally_init(tal);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ny; c += gridDim.x * blockDim.x) {
    ChCellT<S>& cs = cells[c];
    if (!cs.active) continue;
    const double v = af ? af[c] * vol : vol;   // fluid volume of a cut cell
    if (!(v > 0.0)) {
      cs.active = 0;
      continue;
    }
    cs.n = (double)cs.N * F_num / v;
    const CellCoeffsT<S> k =
        cell_coeffs_t<S>(sp, omega, zrot, cs.n, dt, cs.Ttr, cs.Trot, S(cs.Tvib));
    if (!k.ok) {
      tally_or(tal, (uint32_t)F_A_NONPOS);
      cs.active = 0;
      continue;
    }
    cs.alpha = k.alpha; cs.nu_ref = k.nu_ref; cs.B = k.B; cs.mu_p = k.mu_p; cs.Pr = k.Pr;
    cs.gtr = k.g_tr_rot; cs.gtv = k.g_tr_vib; cs.grv = k.g_rot_vib;
    cs.e_rot_tgt = k.e_rot_tgt;
    cs.e_vib_tgt = k.e_vib_tgt;
    if (k.tgt_clamped) {
      tally_or(tal, (uint32_t)F_TREL_CLAMP);
      tally_add(tal, C_TREL_CLAMP, 1ull);
    }
  }
  tally_flush(tal, flags, counters);
}

// ---------------------------------------------------------------------------
// FP32 state, USP-FPM: the moments of ch_moments and the coefficients of
// ch_coeffs evaluated in FP32 (cell_coeffs_f32) in one pass, 32 consecutive
// cells per warp.  The warp stages
// its cells' particles in shared memory in chunks of kMC (coalesced loads);
// lane k then sums cell k's particles from there, shifted by the cell's
// first particle (sums of d = c - c_first and of d d^T, so that the central
// second moments need no second pass over the particles), and evaluates
// cell k's fields and coefficients in FP32 from those sums.  Each lane keeps
// its cell's sums in registers, so a cell costs no warp-wide reduction.
// ---------------------------------------------------------------------------
constexpr int kMC = 512;   // particles per warp chunk
constexpr int kMW = 4;     // warps per block

__global__ void __launch_bounds__(kMW * 32)
ch_moments_coeffs_f32(int ncell, const long long* __restrict__ off,
                      const double* __restrict__ af, const double* __restrict__ afv, float nv,
                      double dt,
                      const float* __restrict__ cx, const float* __restrict__ cy,
                      const float* __restrict__ cz, const float* __restrict__ er,
                      const int* __restrict__ lev, ChCellT<double>* __restrict__ cells,
                      Species sp, uint32_t* flags, unsigned long long* counters,
                      float* __restrict__ pend, float* __restrict__ fT,
                      int* __restrict__ usable_c) {
  __shared__ float sv[kMW][4][kMC];
  __shared__ int sl[kMW][kMC];
  __shared__ BlockTally tal;
  tally_init(tal);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float R = (float)gasR(sp), th = (float)sp.theta_v;
  float* S0 = sv[wid][0];
  float* S1 = sv[wid][1];
  float* S2 = sv[wid][2];
  float* S3 = sv[wid][3];
  int* SL = sl[wid];
  const long long stride = (long long)gridDim.x * kMW * 32;
  for (long long c0 = ((long long)blockIdx.x * kMW + wid) * 32; c0 < ncell; c0 += stride) {
    const int ng = (int)(ncell - c0 < 32 ? ncell - c0 : 32);
    const long long b = lane < ng ? off[c0 + lane] : 0;
    const long long e = lane < ng ? off[c0 + lane + 1] : 0;
    const long long P0 = __shfl_sync(0xffffffffu, b, 0);
    const long long P1 = __shfl_sync(0xffffffffu, e, ng - 1);
    float r0 = 0.0f, r1 = 0.0f, r2 = 0.0f;   // the cell's first particle
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, se = 0.0f;
    float q0 = 0.0f, q1 = 0.0f, q2 = 0.0f, q3 = 0.0f, q4 = 0.0f, q5 = 0.0f;
    int sI = 0;
    for (long long q = P0; q < P1; q += kMC) {
      const int len = (int)(P1 - q < kMC ? P1 - q : kMC);
      __syncwarp();   // the previous chunk's readers are done
#pragma unroll 4
      for (int i = lane; i < len; i += 32) {
        S0[i] = cx[q + i]; S1[i] = cy[q + i]; S2[i] = cz[q + i]; S3[i] = er[q + i];
        SL[i] = lev[q + i];
      }
      __syncwarp();
      const long long j0 = b > q ? b : q, j1 = e < q + len ? e : q + len;
      if (j0 < j1) {
        const int i0 = (int)(j0 - q), i1 = (int)(j1 - q);
        if (j0 == b) { r0 = S0[i0]; r1 = S1[i0]; r2 = S2[i0]; }
        for (int i = i0; i < i1; ++i) {
          const float d0 = S0[i] - r0, d1 = S1[i] - r1, d2 = S2[i] - r2;
          s0 += d0; s1 += d1; s2 += d2;
          q0 = fmaf(d0, d0, q0); q1 = fmaf(d1, d1, q1); q2 = fmaf(d2, d2, q2);
          q3 = fmaf(d0, d1, q3); q4 = fmaf(d0, d2, q4); q5 = fmaf(d1, d2, q5);
          se += S3[i];
          sI += SL[i];
        }
      }
    }
    if (lane >= ng) continue;
    const long long c = c0 + lane;
    const long long N = e - b;
    const float inv = N > 0 ? 1.0f / (float)N : 0.0f;
    const float m0 = s0 * inv, m1 = s1 * inv, m2 = s2 * inv;
    const float U0 = r0 + m0, U1 = r1 + m1, U2 = r2 + m2;
    if (pend) {   // identity pending rescale
      float* pc = pend + (size_t)c * 8;
      pc[0] = pc[1] = pc[2] = pc[3] = pc[4] = pc[5] = 0.0f;
      pc[6] = pc[7] = 1.0f;
    }
    ChCellT<double>& cs = cells[c];
    cs.off = b;
    cs.N = N;
    cs.active = N >= 2;
    // a reconstruction neighbour (Sec. 3.B): two or more particles, not cut
    cs.usable = N >= 2 && (!af || af[c] >= 1.0);
    if (usable_c) usable_c[c] = cs.usable;
    cs.U[0] = U0; cs.U[1] = U1; cs.U[2] = U2;
    for (int i = 0; i < 3; ++i) { cs.Un[i] = 0.0; cs.Us[i] = 0.0; }
    cs.s = 1.0;
    cs.r = 1.0;
    if (!cs.active) {
      tally_add(tal, C_SKIPPED_CELLS, 1ull);
      continue;
    }
    float P[6];
    P[0] = fmaf(q0, inv, -m0 * m0); P[1] = fmaf(q1, inv, -m1 * m1); P[2] = fmaf(q2, inv, -m2 * m2);
    P[3] = fmaf(q3, inv, -m0 * m1); P[4] = fmaf(q4, inv, -m0 * m2); P[5] = fmaf(q5, inv, -m1 * m2);
    const float Ttr = (P[0] + P[1] + P[2]) / (3.0f * R);
    const float Trot = se * inv / R;
    const float ebar = (float)sI * inv;
    const float Tvib = ebar > 0.0f ? th / log1pf(1.0f / ebar) : 0.0f;
    for (int i = 0; i < 6; ++i) cs.Pi[i] = P[i];
    cs.Ttr = Ttr;
    cs.Trot = Trot;
    cs.ebar = ebar;
    cs.Tvib = Tvib;
    float* o = fT + (size_t)c * kNF;   // the 13 fields for the stencils
    o[0] = U0; o[1] = U1; o[2] = U2;
    o[3] = Ttr; o[4] = Trot; o[5] = Tvib;
    for (int i = 0; i < 6; ++i) o[6 + i] = P[i];
    // coefficients: the number density from the fluid volume
    // (afv: the cell's volume over the nominal cell volume; nv = F_num over it)
    const float a = afv ? (float)afv[c] : 1.0f;
    if (!(a > 0.0f)) {
      cs.active = 0;
      continue;
    }
    const float n = (float)N * nv / a;
    const CellCoeffsF k = cell_coeffs_f32(sp, (double)n, dt, Ttr, Trot, Tvib);
    if (!k.ok) {
      tally_or(tal, (uint32_t)F_A_NONPOS);
      cs.active = 0;
      continue;
    }
    cs.n = n;
    cs.alpha = k.alpha; cs.nu_ref = k.nu_ref; cs.B = k.B; cs.mu_p = k.mu_p; cs.Pr = k.Pr;
    cs.gtr = k.g_tr_rot; cs.gtv = k.g_tr_vib; cs.grv = k.g_rot_vib;
    cs.e_rot_tgt = k.e_rot_tgt;
    cs.e_vib_tgt = k.e_vib_tgt;
    if (k.tgt_clamped) {
      tally_or(tal, (uint32_t)F_TREL_CLAMP);
      tally_add(tal, C_TREL_CLAMP, 1ull);
    }
  }
  tally_flush(tal, flags, counters);
}

constexpr int kFpmRec = 11;   // doubles per cell of the FPM coefficient pass

// ---------------------------------------------------------------------------
// the plain FPM method (Sec. 2.B-C) per cell, FP64: alpha = exp(-dt / tau),
// the Cholesky factor of tau D_tr from the cell's stress, the rotational
// square-form constants, the Gillespie rates and the conservation targets
// (the first-order method takes the cell values at every particle)
// ---------------------------------------------------------------------------
__global__ void ch_coeffs_fpm(int ncell, double F_num, double vol, const double* __restrict__ afv,
                              double dt, ChCellT<double>* __restrict__ cells,
                              double* __restrict__ rec, Species sp, uint32_t* flags,
                              unsigned long long* counters) {
  __shared__ BlockTally tal;
  tally_init(tal);
  const double R = gasR(sp);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    ChCellT<double>& cs = cells[c];
    if (!cs.active) continue;
    const double v = afv ? afv[c] * vol : vol;   // fluid volume (null: whole cells)
    if (!(v > 0.0)) {
      cs.active = 0;
      continue;
    }
    cs.n = (double)cs.N * F_num / v;
    const FpmCell f = fpm_cell(sp, cs.n, dt, cs.Pi, cs.Ttr, cs.Trot, cs.Tvib);
    if (!f.ok) {
      tally_or(tal, (uint32_t)F_A_NONPOS);
      cs.active = 0;
      continue;
    }
    cs.alpha = f.alpha;
    cs.e_rot_tgt = f.e_rot_tgt;
    cs.e_vib_tgt = f.e_vib_tgt;
    if (f.fixed) tally_add(tal, C_CHOL_FIX, 1ull);
    if (f.nu_zero) tally_add(tal, C_NU_ZERO, 1ull);
    if (f.failed) tally_or(tal, (uint32_t)F_CHOL_FAIL_AFTER_FIX);
    if (f.clamped) {
      tally_or(tal, (uint32_t)F_TREL_CLAMP);
      tally_add(tal, C_TREL_CLAMP, 1ull);
    }
    const double a = f.alpha, oma2 = 1.0 - a * a, sq = sqrt(oma2);
    const double arot = R * f.Trot_rel * oma2 / 2.0;
    double* o = rec + (size_t)c * kFpmRec;
    o[0] = a;
    for (int i = 0; i < 6; ++i) o[1 + i] = sq * f.L[i];
    o[7] = arot;
    o[8] = sqrt(arot);
    o[9] = f.lam_up;
    o[10] = f.lam_dn;
  }
  tally_flush(tal, flags, counters);
}

// the plain FPM method for one particle (Sec. 2.C) with the cell values U:
// Gorji's velocity update c' = U + alpha (c - U) + sqrt(1 - alpha^2) L G, the
// Milstein square form eps' = a + (sqrt(eps) alpha + sqrt(a) G4)^2 and
// Gillespie's direct method for the level
template <typename T>
__device__ __forceinline__ int fpm_particle(const T* U, T a, const T* Lp, T a_rot, T sqrt_a,
                                            T lam_up, T lam_dn, T& v0, T& v1, T& v2, T& en,
                                            int l0, uint32_t id, uint32_t step,
                                            const PhiloxRoundKeys& rk, uint32_t& fl) {
  T g0, g1, g2, g3;
  uint32_t j5, j6;   // unused: Gillespie's method draws from its own stream
  particle_draws(id, step, rk, g0, g1, g2, g3, j5, j6);
  const T d0 = v0 - U[0], d1 = v1 - U[1], d2 = v2 - U[2];
  v0 = U[0] + a * d0 + Lp[0] * g0;
  v1 = U[1] + a * d1 + (Lp[1] * g0 + Lp[2] * g1);
  v2 = U[2] + a * d2 + (Lp[3] * g0 + Lp[4] * g1 + Lp[5] * g2);
  const T root = sqrt(en) * a + sqrt_a * g3;
  en = a_rot + root * root;
  return gillespie<T>(l0, lam_up, lam_dn, id, step, rk, fl);
}

template <typename S>
__device__ __forceinline__ void cell_fields(const ChCellT<S>& c, S* f) {
  f[0] = c.U[0]; f[1] = c.U[1]; f[2] = c.U[2];
  f[3] = c.Ttr; f[4] = c.Trot; f[5] = S(c.Tvib);
  for (int i = 0; i < 6; ++i) f[6 + i] = c.Pi[i];
}

__global__ void ch_mom_out(int ny, const double* __restrict__ a, double* __restrict__ out,
                           Species sp) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ny) return;
  const double* A = a + (size_t)c * 21;
  const double N = A[0];
  if (!(N > 0.0)) {
    for (int f = 0; f < USP_NMOM; ++f) out[(size_t)f * ny + c] = 0.0;
    return;
  }
  const double R = gasR(sp), inv = 1.0 / N;
  out[c] = N;
  for (int i = 0; i < 3; ++i) out[(size_t)(1 + i) * ny + c] = A[1 + i] * inv;
  out[(size_t)4 * ny + c] = (A[6] + A[7] + A[8]) * inv / (3.0 * R);
  out[(size_t)5 * ny + c] = A[4] * inv / R;
  out[(size_t)6 * ny + c] = T_vib_of_level(sp, A[5] * inv);
  for (int i = 0; i < 6; ++i) out[(size_t)(7 + i) * ny + c] = A[6 + i] * inv;
  for (int i = 0; i < 3; ++i) {
    out[(size_t)(13 + i) * ny + c] = A[12 + i] * inv;
    out[(size_t)(16 + i) * ny + c] = A[15 + i] * inv;
    out[(size_t)(19 + i) * ny + c] = A[18 + i] * inv * R * sp.theta_v;
  }
}

}  // namespace
