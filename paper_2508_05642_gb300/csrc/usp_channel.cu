// usp_channel.cu -- the spatial USP-FPM step in a 1D channel between two
// fully diffuse plates (the Poiseuille set-up of Kim & Jun, arXiv 2508.05642,
// Sec. 5.B, force-driven), on sm_103a.
//
// One step, in the order of the particle framework the method is built into
// (move -> sort -> collide per cell, Sec. 4.D):
//   ch_advect      pending conservation rescale of the previous step, ballistic
//                  flight with the body force, diffuse-wall re-emission
//                  (full accommodation at T_wall, flight continued for the
//                  rest of the step), new cell key
//   radix passes   stable LSD radix sort of (cell key, index), 8-bit digits
//   ch_gather      state permuted into cell order
//   ch_offsets     cell segment starts from the sorted keys
//   ch_moments     per-cell moments (Sec. 2.A), one warp per cell
//   ch_coeffs      per-cell coefficients alpha, nu, gamma, targets (Sec. 3.A)
//   ch_recon       first-order reconstruction of Sec. 3.B: per cell the field
//                  values and the slopes used on each side of the centroid
//   ch_collide     per particle: interpolated fields, relaxation temperatures,
//                  tau D_tr and its Cholesky factor with the Sec. 3.A.3 fix,
//                  Eqs. update_ci / update_erot / update_evib; cell sums
//   ch_levelfix    vibrational +-1 correction of Sec. 4.C (warp per cell)
//   ch_update      rescale factors of Sec. 4.C, kept pending for the next move
//   ch_sample      (while sampling) time-average sums of the post-step state
#include <cuda_runtime.h>

#include <type_traits>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "usp_channel.h"
#include "usp_dual.cuh"

using namespace usp;

// The gradient form runs the same kernels on derivative numbers: random
// numbers and discrete outcomes carry no derivative.
namespace usp {
template <>
__device__ __forceinline__ D3 uniform_open<D3>(uint32_t x) {
  return D3(uniform_open<double>(x));
}
__device__ __forceinline__ void box_muller(D3 ua, D3 ub, D3& ga, D3& gb) {
  double a, b;
  box_muller(ua.v, ub.v, a, b);
  ga = D3(a);
  gb = D3(b);
}
__device__ __forceinline__ void particle_draws(uint32_t pid, uint32_t step,
                                               const PhiloxRoundKeys& rk, D3& g0, D3& g1, D3& g2,
                                               D3& g3, uint32_t& j5, uint32_t& j6) {
  double a0, a1, a2, a3;
  particle_draws(pid, step, rk, a0, a1, a2, a3, j5, j6);
  g0 = D3(a0); g1 = D3(a1); g2 = D3(a2); g3 = D3(a3);
}
// the FP32 gradient form: FP32 values and derivatives per particle
template <>
__device__ __forceinline__ F3 uniform_open<F3>(uint32_t x) {
  return F3(uniform_open<float>(x));
}
__device__ __forceinline__ void particle_draws(uint32_t pid, uint32_t step,
                                               const PhiloxRoundKeys& rk, F3& g0, F3& g1, F3& g2,
                                               F3& g3, uint32_t& j5, uint32_t& j6) {
  float a0, a1, a2, a3;
  particle_draws(pid, step, rk, a0, a1, a2, a3, j5, j6);
  g0 = F3(a0); g1 = F3(a1); g2 = F3(a2); g3 = F3(a3);
}
template <>
__device__ __forceinline__ F3 jump_uniform<F3>(uint32_t x) {
  return F3(uniform_open<float>(x));
}
template <>
__device__ __forceinline__ int sample_nb<F3>(int r, F3 p, F3 u, uint32_t& fl) {
  return sample_nb<float>(r, p.v, u.v, fl);
}
template <>
__device__ __forceinline__ int sample_b<F3>(int n, F3 p, F3 u, uint32_t& fl) {
  return sample_b<float>(n, p.v, u.v, fl);
}
template <>
__device__ __forceinline__ int sample_nb<D3>(int r, D3 p, D3 u, uint32_t& fl) {
  return sample_nb<double>(r, p.v, u.v, fl);
}
template <>
__device__ __forceinline__ int sample_b<D3>(int n, D3 p, D3 u, uint32_t& fl) {
  return sample_b<double>(n, p.v, u.v, fl);
}
}  // namespace usp

#include "usp_spatial.cuh"

namespace {


template <typename T>
struct ChParams {
  T alpha, nu_ref, B, mu_p, Pr, gtr, gtv, grv;
  T R, theta, dt, yc;
  T F[kNF], Sm[kNF], Sp[kNF];   // cell values; slopes used below / above the centroid
  int active, pad;
};

// cell index of a position, in the precision of the position
__device__ __forceinline__ int cell_index(float y, double dy) { return (int)floorf(y / (float)dy); }
__device__ __forceinline__ int cell_index(double y, double dy) { return (int)floor(y / dy); }
__device__ __forceinline__ int cell_index(const D3& y, double dy) { return (int)floor(y.v / dy); }
__device__ __forceinline__ int cell_index(const F3& y, double dy) {
  return (int)floorf(y.v / (float)dy);
}

// ---------------------------------------------------------------------------
// move
// ---------------------------------------------------------------------------
// Diffuse re-emission at T_w (double): Rayleigh normal speed into the gas,
// Maxwellian tangential components, exponential eps_rot, geometric level.
template <typename T, typename S>
__device__ void wall_emit(const Species& sp, uint32_t pid, uint32_t step, int hit, const S& Tw,
                          bool into_pos, uint32_t k0, uint32_t k1, S& vx, S& vy, S& vz, S& e,
                          int& l) {
  const double R = gasR(sp);
  const U4 w = philox4x32_10(pid, step, PTAG_WALL_A, (uint32_t)hit, k0, k1);
  const U4 v = philox4x32_10(pid, step, PTAG_WALL_B, (uint32_t)hit, k0, k1);
  const double u0 = (double)value(uniform_open<T>(w.x));
  const double u1 = (double)value(uniform_open<T>(w.y));
  const double u2 = (double)value(uniform_open<T>(w.z));
  const double u3 = (double)value(uniform_open<T>(w.w));
  const double u4 = (double)value(uniform_open<T>(v.x));
  const S vn = sqrt(-2.0 * R * Tw * log(u0));
  vy = into_pos ? vn : -vn;
  double g1, g2;
  box_muller(u1, u2, g1, g2);
  const S s = sqrt(R * Tw);
  vx = s * g1;
  vz = s * g2;
  e = -R * Tw * log(u3);
  l = (int)floor(-log(u4) * value(Tw) / sp.theta_v);
}

template <typename T, typename S>
__global__ void ch_advect(long long n, int ny, double L, double dy, S Tw, double g, double dt,
                          const int* __restrict__ keycell, const ChCellT<S>* __restrict__ cells,
                          T* __restrict__ y, T* __restrict__ cx, T* __restrict__ cy,
                          T* __restrict__ cz, T* __restrict__ er, int* __restrict__ lev,
                          const uint32_t* __restrict__ pid, int* __restrict__ keyout,
                          int* __restrict__ idxout, const long long* __restrict__ dstep, Species sp,
                          uint32_t k0, uint32_t k1, double* wallmom, uint32_t* flags,
                          unsigned long long* counters) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint32_t step = (uint32_t)*dstep;
  const ChCellT<S>& cc = cells[keycell[j]];
  // pending conservation rescale of the previous step
  T vx = (T)cc.Un[0] + (T)cc.s * (cx[j] - (T)cc.Us[0]);
  T vy = (T)cc.Un[1] + (T)cc.s * (cy[j] - (T)cc.Us[1]);
  T vz = (T)cc.Un[2] + (T)cc.s * (cz[j] - (T)cc.Us[2]);
  T e = (T)cc.r * er[j];
  int l = lev[j];
  T yy = y[j];
  T t_left = (T)dt;
  double mom = 0.0;
  int hits = 0;
  for (;;) {
    const T yn = yy + vy * t_left;
    if (yn >= T(0) && yn <= (T)L) {
      yy = yn;
      vx += (T)g * t_left;
      break;
    }
    if (hits >= kWallHitCap) {
      atomicOr(flags, (uint32_t)F_WALL_CAP);
      yy = yn < T(0) ? T(0) : (T)L;
      vx += (T)g * t_left;
      break;
    }
    const T wall = yn < T(0) ? T(0) : (T)L;
    // gradient form: the time of a wall event is held with the event
    T t_hit = held((wall - yy) / vy);
    t_hit = t_hit < T(0) ? T(0) : (t_hit > t_left ? t_left : t_hit);
    vx += (T)g * t_hit;
    mom += (double)vx;
    yy = wall;
    t_left -= t_hit;
    S ox, oy, oz, oe;
    int ol;
    wall_emit<T, S>(sp, pid[j], step, hits, Tw, wall == T(0), k0, k1, ox, oy, oz, oe, ol);
    vx = (T)ox; vy = (T)oy; vz = (T)oz; e = (T)oe; l = ol;
    mom -= (double)vx;
    hits += 1;
  }
  if (hits) {
    atomicAdd(wallmom, mom);
    atomicAdd(&counters[C_WALL_HITS], (unsigned long long)hits);
  }
  // gradient form: the position is held with the cell it selects (through
  // the interpolated fields its derivative would feed a chaotic response)
  yy = held(yy);
  y[j] = yy; cx[j] = vx; cy[j] = vy; cz[j] = vz; er[j] = e; lev[j] = l;
  int k = cell_index(yy, dy);
  k = k < 0 ? 0 : (k >= ny ? ny - 1 : k);
  keyout[j] = k;
  idxout[j] = (int)j;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (key, index), 8-bit digits
// ---------------------------------------------------------------------------
__global__ void rad_hist(const int* __restrict__ key, long long n, int shift, int* __restrict__ bh) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const long long b = (long long)blockIdx.x * kChunk;
  for (int r = 0; r < kRPT; ++r) {
    const long long i = b + (long long)r * kRB + threadIdx.x;
    if (i < n) atomicAdd(&h[(key[i] >> shift) & 255], 1);
  }
  __syncthreads();
  bh[(size_t)blockIdx.x * 256 + threadIdx.x] = h[threadIdx.x];
}

// digit-major exclusive scan of the block histograms, in place (one block)
__global__ void rad_scan(int* __restrict__ bh, int nblk) {
  __shared__ long long base[256];
  const int d = threadIdx.x;
  long long tot = 0;
  for (int b = 0; b < nblk; ++b) tot += bh[(size_t)b * 256 + d];
  base[d] = tot;
  __syncthreads();
  if (d == 0) {
    long long run = 0;
    for (int i = 0; i < 256; ++i) {
      const long long t = base[i];
      base[i] = run;
      run += t;
    }
  }
  __syncthreads();
  long long run = base[d];
  for (int b = 0; b < nblk; ++b) {
    const int v = bh[(size_t)b * 256 + d];
    bh[(size_t)b * 256 + d] = (int)run;
    run += v;
  }
}

__global__ void rad_scatter(const int* __restrict__ kin, const int* __restrict__ iin,
                            int* __restrict__ kout, int* __restrict__ iout, long long n, int shift,
                            const int* __restrict__ bh) {
  __shared__ int cnt[kRB / 32][256];
  __shared__ int run[256];
  const int t = threadIdx.x, w = t >> 5;
  run[t] = bh[(size_t)blockIdx.x * 256 + t];
  const long long b = (long long)blockIdx.x * kChunk;
  for (int r = 0; r < kRPT; ++r) {
    for (int q = 0; q < kRB / 32; ++q) cnt[q][t] = 0;
    __syncthreads();
    const long long i = b + (long long)r * kRB + t;
    const bool valid = i < n;
    const int kk = valid ? kin[i] : 0;
    const int d = valid ? ((kk >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lane_lt());
    if (valid && rank == 0) cnt[w][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int pre = 0;
      for (int q = 0; q < w; ++q) pre += cnt[q][d];
      const int pos = run[d] + pre + rank;
      kout[pos] = kk;
      iout[pos] = iin[i];
    }
    __syncthreads();
    int tot = 0;
    for (int q = 0; q < kRB / 32; ++q) tot += cnt[q][t];
    run[t] += tot;
    __syncthreads();
  }
}

template <typename T>
__global__ void ch_gather(long long n, const int* __restrict__ idx, const T* __restrict__ y0,
                          const T* __restrict__ x0, const T* __restrict__ vy0,
                          const T* __restrict__ z0, const T* __restrict__ e0,
                          const int* __restrict__ l0, const uint32_t* __restrict__ p0,
                          T* __restrict__ y1, T* __restrict__ x1, T* __restrict__ vy1,
                          T* __restrict__ z1, T* __restrict__ e1, int* __restrict__ l1,
                          uint32_t* __restrict__ p1) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int s = idx[j];
  y1[j] = y0[s]; x1[j] = x0[s]; vy1[j] = vy0[s]; z1[j] = z0[s]; e1[j] = e0[s];
  l1[j] = l0[s]; p1[j] = p0[s];
}

__global__ void ch_offsets(long long n, int ny, const int* __restrict__ key,
                           long long* __restrict__ off) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n == 0) {
    if (j <= ny) off[j] = 0;
    return;
  }
  if (j >= n) return;
  const int k = key[j];
  const int prev = j > 0 ? key[j - 1] : -1;
  for (int c = prev + 1; c <= k; ++c) off[c] = j;
  if (j == n - 1)
    for (int c = k + 1; c <= ny; ++c) off[c] = n;
}

// ---------------------------------------------------------------------------
// per-cell moments, coefficients, reconstruction
// ---------------------------------------------------------------------------
// Sec. 3.B in one dimension: the line through the cell average at the
// centroid and the neighbour's average at its centroid, the neighbour on the
// particle's side, or on the other side when that one is a wall or holds
// fewer than two particles.
template <typename T, typename S>
__global__ void ch_recon(int ny, double dy, int recon, double dt,
                         const ChCellT<S>* __restrict__ cells, ChParams<T>* __restrict__ prm,
                         Species sp) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ny) return;
  const ChCellT<S>& cs = cells[c];
  ChParams<T> P;
  P.active = cs.active;
  P.pad = 0;
  P.alpha = (T)cs.alpha; P.nu_ref = (T)cs.nu_ref; P.B = (T)cs.B; P.mu_p = (T)cs.mu_p;
  P.Pr = (T)cs.Pr; P.gtr = (T)cs.gtr; P.gtv = (T)cs.gtv; P.grv = (T)cs.grv;
  P.R = (T)gasR(sp); P.theta = (T)sp.theta_v; P.dt = (T)dt;
  P.yc = (T)((c + 0.5) * dy);
  S f[kNF];
  cell_fields(cs, f);
  auto valid = [&](int k) { return k >= 0 && k < ny && cells[k].active; };
  const int up = valid(c + 1) ? c + 1 : (valid(c - 1) ? c - 1 : -1);
  const int dn = valid(c - 1) ? c - 1 : (valid(c + 1) ? c + 1 : -1);
  S fu[kNF], fd[kNF];
  if (up >= 0) cell_fields(cells[up], fu);
  if (dn >= 0) cell_fields(cells[dn], fd);
  for (int i = 0; i < kNF; ++i) {
    P.F[i] = (T)f[i];
    P.Sp[i] = (recon && up >= 0) ? (T)((fu[i] - f[i]) / ((up - c) * dy)) : T(0);
    P.Sm[i] = (recon && dn >= 0) ? (T)((fd[i] - f[i]) / ((dn - c) * dy)) : T(0);
  }
  prm[c] = P;
}

// ---------------------------------------------------------------------------
// per-particle collision with interpolated fields (working precision T)
// ---------------------------------------------------------------------------
template <typename T, typename S>
__global__ void ch_collide(int ny, const ChCellT<S>* __restrict__ cells,
                           const ChParams<T>* __restrict__ prm,
                           const T* __restrict__ y, T* __restrict__ cx, T* __restrict__ cy,
                           T* __restrict__ cz, T* __restrict__ er, int* __restrict__ lev,
                           const uint32_t* __restrict__ pid, ChSumsT<S>* __restrict__ sums,
                           const long long* __restrict__ dstep, const PhiloxRoundKeys rk,
                           uint32_t* flags, unsigned long long* counters) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= ny) return;
  const ChCellT<S>& cs = cells[c];
  if (!cs.active) return;
  const ChParams<T>& P = prm[c];
  const uint32_t step = (uint32_t)*dstep;
  const T Uc0 = (T)cs.U[0], Uc1 = (T)cs.U[1], Uc2 = (T)cs.U[2];
  T acc[10];
  for (int i = 0; i < 10; ++i) acc[i] = T(0);
  double accI = 0.0;
  int maxI = 0;
  CollideTally tl = {0u, 0ull, 0ull, 0ull, 0ull};
  unsigned long long nfb = 0;
  for (long long j = cs.off + lane; j < cs.off + cs.N; j += 32) {
    // interpolated fields at the particle
    const T dyv = y[j] - P.yc;
    const bool above = dyv >= T(0);
    T f[kNF];
#pragma unroll
    for (int i = 0; i < kNF; ++i) f[i] = P.F[i] + (above ? P.Sp[i] : P.Sm[i]) * dyv;
    if (!(f[3] > T(0)) || !(f[4] > T(0)) || !(f[5] >= T(0))) {
#pragma unroll
      for (int i = 0; i < kNF; ++i) f[i] = P.F[i];
      ++nfb;
    }
    T v0 = cx[j], v1 = cy[j], v2 = cz[j], en = er[j];
    const int ln = collide_particle_t(P, f, v0, v1, v2, en, lev[j], pid[j], step, rk, tl);
    cx[j] = v0; cy[j] = v1; cz[j] = v2; er[j] = en;
    lev[j] = ln;
    maxI = max(maxI, ln);
    const T d0 = v0 - Uc0, d1 = v1 - Uc1, d2 = v2 - Uc2;
    acc[0] += d0; acc[1] += d1; acc[2] += d2;
    acc[3] += d0 * d0; acc[4] += d1 * d1; acc[5] += d2 * d2;
    acc[6] += d0 * d1; acc[7] += d0 * d2; acc[8] += d1 * d2;
    acc[9] += en;
    accI += (double)ln;
  }
  S s[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) s[i] = S(wsum(acc[i]));
  const double sI = wsum(accI);
  const unsigned long long fix = wsum(tl.nfix), fb = wsum(nfb), ncl2 = wsum(tl.ncl),
                           pb = wsum(tl.npb), nz = wsum(tl.nnz);
  const int mI = __reduce_max_sync(0xffffffffu, maxI);
  const uint32_t fla = __reduce_or_sync(0xffffffffu, tl.fl);
  if (lane != 0) return;
  ChSumsT<S>& sm = sums[c];
  for (int i = 0; i < 10; ++i) sm.v[i] = s[i];
  sm.I = (unsigned long long)(long long)llrint(sI);
  sm.net = 0;
  sm.maxI = mI;
  if (fla) atomicOr(flags, fla);
  if (fix) atomicAdd(&counters[C_CHOL_FIX], fix);
  if (fb) atomicAdd(&counters[C_INTERP_FALLBACK], fb);
  if (ncl2) atomicAdd(&counters[C_TREL_CLAMP], ncl2);
  if (pb) atomicAdd(&counters[C_PB_CLAMP], pb);
  if (nz) atomicAdd(&counters[C_NU_ZERO], nz);
}

// the plain FPM method (Sec. 2.C) per particle with the cell values: one warp
// per cell, per-cell sums for the conservation step as in ch_collide
template <typename T>
__global__ void ch_collide_fpm(int ny, const ChCellT<double>* __restrict__ cells,
                               const double* __restrict__ rec, T* __restrict__ cx,
                               T* __restrict__ cy, T* __restrict__ cz, T* __restrict__ er,
                               int* __restrict__ lev, const uint32_t* __restrict__ pid,
                               ChSumsT<double>* __restrict__ sums,
                               const long long* __restrict__ dstep, const PhiloxRoundKeys rk,
                               uint32_t* flags) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= ny) return;
  const ChCellT<double>& cs = cells[c];
  if (!cs.active) return;
  const uint32_t step = (uint32_t)*dstep;
  const double* r = rec + (size_t)c * kFpmRec;
  const T U[3] = {(T)cs.U[0], (T)cs.U[1], (T)cs.U[2]};
  const T Lp[6] = {(T)r[1], (T)r[2], (T)r[3], (T)r[4], (T)r[5], (T)r[6]};
  const T a = (T)r[0], a_rot = (T)r[7], sqrt_a = (T)r[8], lu = (T)r[9], ld = (T)r[10];
  T acc[10];
  for (int i = 0; i < 10; ++i) acc[i] = T(0);
  double accI = 0.0;
  int maxI = 0;
  uint32_t fl = 0;
  for (long long j = cs.off + lane; j < cs.off + cs.N; j += 32) {
    T v0 = cx[j], v1 = cy[j], v2 = cz[j], en = er[j];
    const int ln = fpm_particle<T>(U, a, Lp, a_rot, sqrt_a, lu, ld, v0, v1, v2, en, lev[j],
                                   pid[j], step, rk, fl);
    cx[j] = v0; cy[j] = v1; cz[j] = v2; er[j] = en;
    lev[j] = ln;
    maxI = max(maxI, ln);
    const T d0 = v0 - U[0], d1 = v1 - U[1], d2 = v2 - U[2];
    acc[0] += d0; acc[1] += d1; acc[2] += d2;
    acc[3] += d0 * d0; acc[4] += d1 * d1; acc[5] += d2 * d2;
    acc[6] += d0 * d1; acc[7] += d0 * d2; acc[8] += d1 * d2;
    acc[9] += en;
    accI += (double)ln;
  }
  double s[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) s[i] = (double)wsum(acc[i]);
  const double sI = wsum(accI);
  const int mI = __reduce_max_sync(0xffffffffu, maxI);
  const uint32_t fla = __reduce_or_sync(0xffffffffu, fl);
  if (lane != 0) return;
  ChSumsT<double>& sm = sums[c];
  for (int i = 0; i < 10; ++i) sm.v[i] = s[i];
  sm.I = (unsigned long long)(long long)llrint(sI);
  sm.net = 0;
  sm.maxI = mI;
  if (fla) atomicOr(flags, fla);
}

// time-average sums of the post-step state, one warp per cell (the state is
// in cell order), each sum reduced across the warp in a fixed order and added
// by one lane, so that runs are reproducible bit for bit (gradient form:
// block 0 holds the sums, blocks 1..3 their derivatives)
template <typename T, typename S>
__global__ void ch_sample(int ny, const long long* __restrict__ off,
                          const ChCellT<S>* __restrict__ cells, const T* __restrict__ cx,
                          const T* __restrict__ cy, const T* __restrict__ cz,
                          const T* __restrict__ er, const int* __restrict__ lev,
                          double* __restrict__ acc, const double* __restrict__ wallmom) {
  const int lane = threadIdx.x & 31;
  const size_t blk = (size_t)ny * kNAcc + 2;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    acc[(size_t)ny * kNAcc] += 1.0;
    acc[(size_t)ny * kNAcc + 1] += *wallmom;
  }
  for (int k = warp_global(); k < ny; k += warps_total()) {
    const ChCellT<S>& cc = cells[k];
    S q[10];
    for (int i = 0; i < 10; ++i) q[i] = S(0.0);
    long long sl = 0;
    const long long b = off[k], e = off[k + 1];
    for (long long j = b + lane; j < e; j += 32) {
      const S v0 = cc.Un[0] + cc.s * (S(cx[j]) - cc.Us[0]);
      const S v1 = cc.Un[1] + cc.s * (S(cy[j]) - cc.Us[1]);
      const S v2 = cc.Un[2] + cc.s * (S(cz[j]) - cc.Us[2]);
      q[0] += v0; q[1] += v1; q[2] += v2;
      q[3] += v0 * v0; q[4] += v1 * v1; q[5] += v2 * v2;
      q[6] += v0 * v1; q[7] += v0 * v2; q[8] += v1 * v2;
      q[9] += cc.r * S(er[j]);
      sl += lev[j];
    }
    for (int i = 0; i < 10; ++i) q[i] = wsum(q[i]);
    for (int o = 16; o > 0; o >>= 1) sl += __shfl_xor_sync(0xffffffffu, sl, o);
    if (lane == 0) {
      double* a = acc + (size_t)k * kNAcc;
      a[0] += (double)(e - b);
      for (int i = 0; i < 10; ++i) acc_add(&a[1 + i], blk, q[i]);
      a[11] += (double)sl;
    }
  }
}

// Time-averaged profiles of cell c from the pooled sums: values (b = 0) or
// their derivatives with respect to parameter b - 1 (gradient form), in the
// field order of usp_profiles.  Counts and levels carry no derivative.
__device__ void ch_prof_cell(const double* __restrict__ acc, int ny, int c, int b, double R,
                             double theta, double* P) {
  const size_t blk = (size_t)ny * kNAcc + 2;
  const double* A = acc + (size_t)c * kNAcc;
  const double N = A[0], ns = acc[(size_t)ny * kNAcc];
  for (int f = 0; f < USP_NPROF; ++f) P[f] = 0.0;
  if (!(N > 0.0)) return;
  const double U0 = A[1] / N, U1 = A[2] / N, U2 = A[3] / N;
  if (b == 0) {
    P[0] = ns > 0.0 ? N / ns : 0.0;
    P[1] = U0; P[2] = U1; P[3] = U2;
    P[4] = ((A[4] + A[5] + A[6]) / N - (U0 * U0 + U1 * U1 + U2 * U2)) / (3.0 * R);
    P[5] = A[10] / (N * R);
    const double eb = A[11] / N;
    P[6] = eb > 0.0 ? theta / log1p(1.0 / eb) : 0.0;
    return;
  }
  const double* D = A + (size_t)b * blk;
  const double d0 = D[1] / N, d1 = D[2] / N, d2 = D[3] / N;
  P[1] = d0; P[2] = d1; P[3] = d2;
  P[4] = ((D[4] + D[5] + D[6]) / N - 2.0 * (U0 * d0 + U1 * d1 + U2 * d2)) / (3.0 * R);
  P[5] = D[10] / (N * R);
}

__global__ void ch_profiles(int ny, int blocks, const double* __restrict__ acc, double R,
                            double theta, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ny) return;
  double P[USP_NPROF];
  for (int b = 0; b < blocks; ++b) {
    ch_prof_cell(acc, ny, c, b, R, theta, P);
    for (int f = 0; f < USP_NPROF; ++f) out[((size_t)b * USP_NPROF + f) * ny + c] = P[f];
  }
}

// grad[k] += sum over cells and fields of dL[f * ny + c] d prof[f][c] / d theta_k
// (grad zeroed before the launch)
__global__ void ch_backward(int ny, const double* __restrict__ acc, double R,
                            const double* __restrict__ dL, double* __restrict__ grad) {
  __shared__ double red[kND][256 / 32];
  double g[kND] = {0.0, 0.0, 0.0};
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ny; c += gridDim.x * blockDim.x) {
    double P[USP_NPROF];
    for (int k = 0; k < kND; ++k) {
      ch_prof_cell(acc, ny, c, k + 1, R, 0.0, P);
      for (int f = 0; f < USP_NPROF; ++f) g[k] += dL[(size_t)f * ny + c] * P[f];
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < kND; ++k) {
    double v = g[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < kND) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) v += red[threadIdx.x][w];
    atomicAdd(&grad[threadIdx.x], v);
  }
}

// on-demand moments (USP_NMOM fields) of the current state by cell key:
// pass 0 raw sums, pass 1 central sums (FP64 atomics; not on the step path)
template <typename T, typename S>
__global__ void ch_mom_pass(int pass, long long n, const int* __restrict__ keycell,
                            const ChCellT<S>* __restrict__ cells, const T* __restrict__ cx,
                            const T* __restrict__ cy, const T* __restrict__ cz,
                            const T* __restrict__ er, const int* __restrict__ lev,
                            double* __restrict__ a) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int k = keycell[j];
  const ChCellT<S>& cc = cells[k];
  const double sc = value(cc.s);
  const double v0 = value(cc.Un[0]) + sc * ((double)value(cx[j]) - value(cc.Us[0]));
  const double v1 = value(cc.Un[1]) + sc * ((double)value(cy[j]) - value(cc.Us[1]));
  const double v2 = value(cc.Un[2]) + sc * ((double)value(cz[j]) - value(cc.Us[2]));
  const double ep = value(cc.r) * (double)value(er[j]);
  const double li = (double)lev[j];
  double* A = a + (size_t)k * 21;
  if (pass == 0) {
    atomicAdd(&A[0], 1.0);
    atomicAdd(&A[1], v0); atomicAdd(&A[2], v1); atomicAdd(&A[3], v2);
    atomicAdd(&A[4], ep); atomicAdd(&A[5], li);
    return;
  }
  const double N = A[0];
  const double C0 = v0 - A[1] / N, C1 = v1 - A[2] / N, C2 = v2 - A[3] / N;
  const double q = 0.5 * (C0 * C0 + C1 * C1 + C2 * C2);
  atomicAdd(&A[6], C0 * C0); atomicAdd(&A[7], C1 * C1); atomicAdd(&A[8], C2 * C2);
  atomicAdd(&A[9], C0 * C1); atomicAdd(&A[10], C0 * C2); atomicAdd(&A[11], C1 * C2);
  atomicAdd(&A[12], q * C0); atomicAdd(&A[13], q * C1); atomicAdd(&A[14], q * C2);
  atomicAdd(&A[15], C0 * ep); atomicAdd(&A[16], C1 * ep); atomicAdd(&A[17], C2 * ep);
  atomicAdd(&A[18], C0 * li); atomicAdd(&A[19], C1 * li); atomicAdd(&A[20], C2 * li);
}

template <typename T, typename S>
__global__ void ch_to_host_layout(long long n, const int* __restrict__ keycell,
                                  const ChCellT<S>* __restrict__ cells, const T* __restrict__ y,
                                  const T* __restrict__ cx, const T* __restrict__ cy,
                                  const T* __restrict__ cz, const T* __restrict__ er,
                                  double* __restrict__ out) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const ChCellT<S>& cc = cells[keycell[j]];
  const double sc = value(cc.s);
  out[j] = (double)value(y[j]);
  out[n + j] = value(cc.Un[0]) + sc * ((double)value(cx[j]) - value(cc.Us[0]));
  out[2 * n + j] = value(cc.Un[1]) + sc * ((double)value(cy[j]) - value(cc.Us[1]));
  out[3 * n + j] = value(cc.Un[2]) + sc * ((double)value(cz[j]) - value(cc.Us[2]));
  out[4 * n + j] = value(cc.r) * (double)value(er[j]);
}

template <typename T>
__global__ void ch_from_host_layout(long long n, const double* __restrict__ in, T* __restrict__ y,
                                    T* __restrict__ cx, T* __restrict__ cy, T* __restrict__ cz,
                                    T* __restrict__ er) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  y[j] = (T)in[j]; cx[j] = (T)in[n + j]; cy[j] = (T)in[2 * n + j]; cz[j] = (T)in[3 * n + j];
  er[j] = (T)in[4 * n + j];
}

}  // namespace

// ===========================================================================
// host side
// ===========================================================================
struct ChannelCtx {
  int ny, recon, passes, nblk;
  double L, dy, Tw, g, Fnum, area, dt;
  long long n;
  size_t es;
  void* st[2][5];           // y, cx, cy, cz, eps (ping-pong)
  int* lv[2];
  uint32_t* pd[2];
  int cur;
  int* kbuf[2];
  int* ibuf[2];
  int* keycell;
  int* bh;
  long long* off;
  void* cells;              // ChCellT<S>
  void* prm;                // ChParams<T>
  void* sums;               // ChSumsT<S>
  int blocks;               // accumulator blocks: 1, or 4 in the gradient form
  double* acc;
  double* wallmom;
  double* macc;
  double* mout;
  long long* dstep;
  int sampling;
  double* fpmrec;           // the plain FPM method: kFpmRec per-cell constants (else null)
  double* prof;             // time-averaged profiles (USP_NPROF x ny per block)
  double* grad;             // the objective's gradient (3 doubles, gradient form)
};

namespace {

#define CHK(x)                                 \
  do {                                         \
    if ((x) != cudaSuccess) return USP_ECUDA;  \
  } while (0)

// parameter values of the gradient form: Z_rot, omega, T_wall are the three
// independent variables (derivative slots 0, 1, 2)
template <typename S> S param(double v, int slot);
template <> double param<double>(double v, int) { return v; }
template <> D3 param<D3>(double v, int slot) {
  D3 r(v);
  r.d[slot] = 1.0;
  return r;
}

template <typename T, typename S>
int ch_step_t(ChannelCtx* h, const ChEnv& env, ch_prof_fn prof) {
  cudaStream_t s = env.stream;
  ChCellT<S>* cells = (ChCellT<S>*)h->cells;
  ChSumsT<S>* sums = (ChSumsT<S>*)h->sums;
  const S Tw = param<S>(h->Tw, 2);
  const S omega = param<S>(env.sp.omega, 1);
  const S zrot = param<S>(env.sp.Z_rot, 0);
  const long long n = h->n;
  const int nb = (int)((n + 255) / 256) > 0 ? (int)((n + 255) / 256) : 1;
  const int a = h->cur, b = a ^ 1;
  T* y = (T*)h->st[a][0]; T* cx = (T*)h->st[a][1]; T* cy = (T*)h->st[a][2];
  T* cz = (T*)h->st[a][3]; T* er = (T*)h->st[a][4];
  if (prof) prof(env.owner, 0, 1);
  CHK(cudaMemsetAsync(h->wallmom, 0, sizeof(double), s));
  ch_advect<T, S><<<nb, 256, 0, s>>>(n, h->ny, h->L, h->dy, Tw, h->g, h->dt, h->keycell, cells,
                                   y, cx, cy, cz, er, h->lv[a], h->pd[a], h->kbuf[0], h->ibuf[0],
                                   h->dstep, env.sp, env.k0, env.k1, h->wallmom, env.flags,
                                   env.counters);
  CHK(cudaGetLastError());
  int src = 0;
  for (int p = 0; p < h->passes; ++p) {
    rad_hist<<<h->nblk, kRB, 0, s>>>(h->kbuf[src], n, 8 * p, h->bh);
    rad_scan<<<1, 256, 0, s>>>(h->bh, h->nblk);
    rad_scatter<<<h->nblk, kRB, 0, s>>>(h->kbuf[src], h->ibuf[src], h->kbuf[src ^ 1],
                                        h->ibuf[src ^ 1], n, 8 * p, h->bh);
    CHK(cudaGetLastError());
    src ^= 1;
  }
  ch_gather<T><<<nb, 256, 0, s>>>(n, h->ibuf[src], y, cx, cy, cz, er, h->lv[a], h->pd[a],
                                  (T*)h->st[b][0], (T*)h->st[b][1], (T*)h->st[b][2],
                                  (T*)h->st[b][3], (T*)h->st[b][4], h->lv[b], h->pd[b]);
  CHK(cudaMemcpyAsync(h->keycell, h->kbuf[src], sizeof(int) * (n > 0 ? n : 1),
                      cudaMemcpyDeviceToDevice, s));
  ch_offsets<<<std::max(nb, (h->ny + 256) / 256), 256, 0, s>>>(n, h->ny, h->keycell, h->off);
  CHK(cudaGetLastError());
  h->cur = b;
  y = (T*)h->st[b][0]; cx = (T*)h->st[b][1]; cy = (T*)h->st[b][2]; cz = (T*)h->st[b][3];
  er = (T*)h->st[b][4];
  if (prof) prof(env.owner, 0, 0);
  if (prof) prof(env.owner, 1, 1);
  const int wb = (h->ny * 32 + 127) / 128;
  const int cb = (h->ny + 127) / 128;
  ch_moments<T, S><<<wb, 128, 0, s>>>(h->ny, 1, h->off, nullptr, cx, cy, cz, er, h->lv[b], cells,
                                      env.sp, env.counters, nullptr, (T*)nullptr, nullptr);
  if constexpr (std::is_same<S, double>::value) {
    if (h->fpmrec) {
      // the plain FPM method: cell values at every particle, no reconstruction
      ch_coeffs_fpm<<<cb, 128, 0, s>>>(h->ny, h->Fnum, h->area * h->dy, nullptr, h->dt, cells,
                                       h->fpmrec, env.sp, env.flags, env.counters);
      CHK(cudaGetLastError());
      if (prof) prof(env.owner, 1, 0);
      if (prof) prof(env.owner, 0, 1);
      ch_collide_fpm<T><<<wb, 128, 0, s>>>(h->ny, cells, h->fpmrec, cx, cy, cz, er, h->lv[b],
                                           h->pd[b], sums, h->dstep,
                                           philox_round_keys(env.k0, env.k1), env.flags);
    }
  }
  if (!h->fpmrec) {
  ch_coeffs<S><<<cb, 128, 0, s>>>(h->ny, h->Fnum, h->area * h->dy, nullptr, h->dt, cells, env.sp,
                                  omega, zrot, env.flags, env.counters);
  ch_recon<T, S><<<cb, 128, 0, s>>>(h->ny, h->dy, h->recon, h->dt, cells, (ChParams<T>*)h->prm,
                                    env.sp);
  CHK(cudaGetLastError());
  if (prof) prof(env.owner, 1, 0);
  if (prof) prof(env.owner, 0, 1);
  ch_collide<T, S><<<wb, 128, 0, s>>>(h->ny, cells, (const ChParams<T>*)h->prm, y, cx, cy, cz,
                                      er, h->lv[b], h->pd[b], sums, h->dstep,
                                      philox_round_keys(env.k0, env.k1), env.flags, env.counters);
  }
  CHK(cudaGetLastError());
  if (prof) prof(env.owner, 0, 0);
  if (prof) prof(env.owner, 1, 1);
  ch_levelfix<S><<<wb, 128, 0, s>>>(h->ny, 1, cells, sums, h->lv[b], h->dstep, env.sp, env.k0,
                                    env.k1, env.flags, env.counters);
  ch_update<S><<<cb, 128, 0, s>>>(h->ny, cells, sums, h->dstep, env.sp, env.flags, env.counters,
                                  nullptr);
  CHK(cudaGetLastError());
  if (h->sampling) {
    ch_sample<T, S><<<wb, 128, 0, s>>>(h->ny, h->off, cells, cx, cy, cz, er, h->lv[b], h->acc,
                                       h->wallmom);
    CHK(cudaGetLastError());
  }
  if (prof) prof(env.owner, 1, 0);
  return USP_OK;
}

}  // namespace

int ch_kernels_per_step(const ChannelCtx* h) {
  return 2 + 3 * h->passes + (h->fpmrec ? 7 : 8) + (h->sampling ? 1 : 0);
}

int ch_launch_step(ChannelCtx* h, const ChEnv& env, ch_prof_fn prof) {
  if (env.precision == USP_FP32) return ch_step_t<float, double>(h, env, prof);
  if (env.precision == USP_FP64_TANGENT) return ch_step_t<D3, D3>(h, env, prof);
  if (env.precision == USP_FP32_TANGENT) return ch_step_t<F3, D3>(h, env, prof);
  return ch_step_t<double, double>(h, env, prof);
}

int ch_create(ChannelCtx** out, const ChEnv& env, const usp_channel* chp, double dt, int64_t n,
              int64_t step0, const double* y, const double* cx, const double* cy,
              const double* cz, const double* erot, const int32_t* lev, const uint32_t* pid) {
  if (!chp || chp->ny <= 0 || chp->ny > (1 << 24) || !(chp->L > 0) || !(chp->T_wall > 0) ||
      !(chp->F_num > 0) || !(chp->area > 0) || !(dt > 0) || n < 0 || n > 0x7fffffffll)
    return USP_EINVAL;
  if (n > 0 && (!y || !cx || !cy || !cz || !erot || !lev))
    return USP_EINVAL;
  for (int64_t j = 0; j < n; ++j)
    if (!(y[j] >= 0.0 && y[j] <= chp->L) || lev[j] < 0) return USP_EINVAL;
  ChannelCtx* h = new ChannelCtx();
  h->ny = chp->ny; h->L = chp->L; h->dy = chp->L / chp->ny; h->Tw = chp->T_wall; h->g = chp->g;
  h->Fnum = chp->F_num; h->area = chp->area; h->recon = chp->reconstruct ? 1 : 0; h->dt = dt;
  h->n = n;
  const bool g32 = env.precision == USP_FP32_TANGENT;
  const bool grad = env.precision == USP_FP64_TANGENT || g32;
  h->es = env.precision == USP_FP32 ? 4 : (g32 ? sizeof(F3) : (grad ? sizeof(D3) : 8));
  h->blocks = grad ? 1 + kND : 1;
  const size_t cell_bytes = grad ? sizeof(ChCellT<D3>) : sizeof(ChCellT<double>);
  const size_t sums_bytes = grad ? sizeof(ChSumsT<D3>) : sizeof(ChSumsT<double>);
  const size_t acc_bytes = sizeof(double) * ((size_t)chp->ny * kNAcc + 2) * h->blocks;
  h->cur = 0;
  h->sampling = 0;
  int bits = 1;
  while ((1 << bits) < h->ny) ++bits;
  h->passes = (bits + 7) / 8;
  h->nblk = (int)std::max<long long>(1, (n + kChunk - 1) / kChunk);
  const size_t nn = (size_t)std::max<long long>(n, 1);
  auto A = [&](size_t bytes) { return env.alloc(env.owner, bytes); };
  for (int k = 0; k < 2; ++k) {
    for (int f = 0; f < 5; ++f) h->st[k][f] = A(nn * h->es);
    h->lv[k] = (int*)A(nn * 4);
    h->pd[k] = (uint32_t*)A(nn * 4);
    h->kbuf[k] = (int*)A(nn * 4);
    h->ibuf[k] = (int*)A(nn * 4);
  }
  h->keycell = (int*)A(nn * 4);
  h->bh = (int*)A((size_t)h->nblk * 256 * 4);
  h->off = (long long*)A(sizeof(long long) * (h->ny + 1));
  h->cells = A(cell_bytes * h->ny);
  h->prm = A((env.precision == USP_FP32 ? sizeof(ChParams<float>)
                                        : (g32 ? sizeof(ChParams<F3>)
                                               : (grad ? sizeof(ChParams<D3>)
                                                       : sizeof(ChParams<double>)))) *
             h->ny);
  h->sums = A(sums_bytes * h->ny);
  if (env.sp.method == 1) h->fpmrec = (double*)A(sizeof(double) * kFpmRec * (size_t)h->ny);
  h->acc = (double*)A(acc_bytes);
  h->wallmom = (double*)A(sizeof(double));
  h->macc = (double*)A(sizeof(double) * 21 * h->ny);
  h->mout = (double*)A(sizeof(double) * USP_NMOM * h->ny);
  h->dstep = (long long*)A(sizeof(long long));
  h->prof = (double*)A(sizeof(double) * USP_NPROF * h->ny * h->blocks);
  h->grad = (double*)A(sizeof(double) * kND);
  bool ok = h->keycell && h->bh && h->off && h->cells && h->prm && h->sums && h->acc &&
            h->prof && h->grad &&
            (env.sp.method != 1 || h->fpmrec) &&
            h->wallmom && h->macc && h->mout && h->dstep;
  for (int k = 0; k < 2; ++k) {
    for (int f = 0; f < 5; ++f) ok = ok && h->st[k][f];
    ok = ok && h->lv[k] && h->pd[k] && h->kbuf[k] && h->ibuf[k];
  }
  if (!ok) {
    delete h;
    return USP_ENOMEM;
  }
  cudaStream_t s = env.stream;
  // upload: doubles in host layout, converted on the device
  std::vector<double> hl(5 * nn, 0.0);
  std::vector<int> key(nn, 0);
  std::vector<uint32_t> hp(nn, 0);
  for (int64_t j = 0; j < n; ++j) {
    hl[j] = y[j]; hl[n + j] = cx[j]; hl[2 * n + j] = cy[j]; hl[3 * n + j] = cz[j];
    hl[4 * n + j] = erot[j];
    int k = (int)std::floor(y[j] / h->dy);
    key[j] = std::min(std::max(k, 0), h->ny - 1);
    hp[j] = pid ? pid[j] : (uint32_t)j;
  }
  double* stage = nullptr;
  void* tmp = nullptr;
  if (n > 0) {
    tmp = env.alloc(env.owner, 5 * nn * sizeof(double));
    if (!tmp) {
      delete h;
      return USP_ENOMEM;
    }
    stage = (double*)tmp;
  }
  const long long dstep0 = step0;
  bool cok = n == 0 || cudaMemcpyAsync(h->lv[0], lev, n * 4, cudaMemcpyHostToDevice, s) ==
                           cudaSuccess;
  cok = cok && cudaMemcpyAsync(h->pd[0], hp.data(), nn * 4, cudaMemcpyHostToDevice, s) == cudaSuccess;
  cok = cok && cudaMemcpyAsync(h->keycell, key.data(), nn * 4, cudaMemcpyHostToDevice, s) == cudaSuccess;
  cok = cok && cudaMemsetAsync(h->cells, 0, cell_bytes * h->ny, s) == cudaSuccess;
  cok = cok && cudaMemsetAsync(h->sums, 0, sums_bytes * h->ny, s) == cudaSuccess;
  cok = cok && cudaMemsetAsync(h->acc, 0, acc_bytes, s) == cudaSuccess;
  cok = cok && cudaMemcpyAsync(h->dstep, &dstep0, sizeof(long long), cudaMemcpyHostToDevice, s) == cudaSuccess;
  if (n > 0) {
    cok = cok && cudaMemcpyAsync(stage, hl.data(), 5 * nn * sizeof(double), cudaMemcpyHostToDevice,
                                 s) == cudaSuccess;
    const int nb = (int)((n + 255) / 256);
    if (env.precision == USP_FP32)
      ch_from_host_layout<float><<<nb, 256, 0, s>>>(n, stage, (float*)h->st[0][0],
          (float*)h->st[0][1], (float*)h->st[0][2], (float*)h->st[0][3], (float*)h->st[0][4]);
    else if (g32)
      ch_from_host_layout<F3><<<nb, 256, 0, s>>>(n, stage, (F3*)h->st[0][0], (F3*)h->st[0][1],
          (F3*)h->st[0][2], (F3*)h->st[0][3], (F3*)h->st[0][4]);
    else if (grad)
      ch_from_host_layout<D3><<<nb, 256, 0, s>>>(n, stage, (D3*)h->st[0][0], (D3*)h->st[0][1],
          (D3*)h->st[0][2], (D3*)h->st[0][3], (D3*)h->st[0][4]);
    else
      ch_from_host_layout<double><<<nb, 256, 0, s>>>(n, stage, (double*)h->st[0][0],
          (double*)h->st[0][1], (double*)h->st[0][2], (double*)h->st[0][3], (double*)h->st[0][4]);
    cok = cok && cudaGetLastError() == cudaSuccess;
  }
  // every cell starts with an identity pending rescale (s = r = 1, Un = Us = 0)
  if (grad) {
    std::vector<ChCellT<D3>> hc(h->ny);
    for (auto& c : hc) { c.s = D3(1.0); c.r = D3(1.0); c.active = 0; c.N = 0; c.off = 0; }
    cok = cok && cudaMemcpyAsync(h->cells, hc.data(), cell_bytes * h->ny, cudaMemcpyHostToDevice,
                                 s) == cudaSuccess;
  } else {
    std::vector<ChCellT<double>> hc(h->ny);
    std::memset((void*)hc.data(), 0, cell_bytes * h->ny);
    for (auto& c : hc) { c.s = 1.0; c.r = 1.0; }
    cok = cok && cudaMemcpyAsync(h->cells, hc.data(), cell_bytes * h->ny, cudaMemcpyHostToDevice,
                                 s) == cudaSuccess;
  }
  cok = cok && cudaStreamSynchronize(s) == cudaSuccess;
  if (tmp) env.release(env.owner, tmp);
  if (!cok) {
    delete h;
    return USP_ECUDA;
  }
  *out = h;
  return USP_OK;
}

int ch_sample(ChannelCtx* h, int on) {
  h->sampling = on ? 1 : 0;
  return USP_OK;
}

int ch_read(ChannelCtx* h, const ChEnv& env, double* h_acc, int reset) {
  const size_t bytes = sizeof(double) * ((size_t)h->ny * kNAcc + 2) * h->blocks;
  CHK(cudaMemcpyAsync(h_acc, h->acc, bytes, cudaMemcpyDeviceToHost, env.stream));
  if (reset) CHK(cudaMemsetAsync(h->acc, 0, bytes, env.stream));
  CHK(cudaStreamSynchronize(env.stream));
  return USP_OK;
}

int ch_moments(ChannelCtx* h, const ChEnv& env, double* out, int out_is_device) {
  cudaStream_t s = env.stream;
  const long long n = h->n;
  const int nb = (int)std::max<long long>(1, (n + 255) / 256);
  const int b = h->cur;
  CHK(cudaMemsetAsync(h->macc, 0, sizeof(double) * 21 * h->ny, s));
  for (int pass = 0; pass < 2; ++pass) {
    if (env.precision == USP_FP32)
      ch_mom_pass<float, double><<<nb, 256, 0, s>>>(pass, n, h->keycell,
          (const ChCellT<double>*)h->cells, (float*)h->st[b][1], (float*)h->st[b][2],
          (float*)h->st[b][3], (float*)h->st[b][4], h->lv[b], h->macc);
    else if (env.precision == USP_FP64_TANGENT)
      ch_mom_pass<D3, D3><<<nb, 256, 0, s>>>(pass, n, h->keycell, (const ChCellT<D3>*)h->cells,
          (D3*)h->st[b][1], (D3*)h->st[b][2], (D3*)h->st[b][3], (D3*)h->st[b][4], h->lv[b],
          h->macc);
    else if (env.precision == USP_FP32_TANGENT)
      ch_mom_pass<F3, D3><<<nb, 256, 0, s>>>(pass, n, h->keycell, (const ChCellT<D3>*)h->cells,
          (F3*)h->st[b][1], (F3*)h->st[b][2], (F3*)h->st[b][3], (F3*)h->st[b][4], h->lv[b],
          h->macc);
    else
      ch_mom_pass<double, double><<<nb, 256, 0, s>>>(pass, n, h->keycell,
          (const ChCellT<double>*)h->cells, (double*)h->st[b][1], (double*)h->st[b][2],
          (double*)h->st[b][3], (double*)h->st[b][4], h->lv[b], h->macc);
    CHK(cudaGetLastError());
  }
  ch_mom_out<<<(h->ny + 127) / 128, 128, 0, s>>>(h->ny, h->macc, h->mout, env.sp);
  CHK(cudaGetLastError());
  CHK(cudaMemcpyAsync(out, h->mout, sizeof(double) * USP_NMOM * h->ny,
                      out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (!out_is_device) CHK(cudaStreamSynchronize(s));
  return USP_OK;
}

int ch_get_particles(ChannelCtx* h, const ChEnv& env, double* y, double* cx, double* cy,
                     double* cz, double* erot, int32_t* lev, uint32_t* pid) {
  const long long n = h->n;
  if (n == 0) return USP_OK;
  cudaStream_t s = env.stream;
  double* tmp = (double*)env.alloc(env.owner, 5 * n * sizeof(double));
  if (!tmp) return USP_ENOMEM;
  const int b = h->cur;
  const int nb = (int)((n + 255) / 256);
  if (env.precision == USP_FP32)
    ch_to_host_layout<float, double><<<nb, 256, 0, s>>>(n, h->keycell,
        (const ChCellT<double>*)h->cells, (float*)h->st[b][0], (float*)h->st[b][1],
        (float*)h->st[b][2], (float*)h->st[b][3], (float*)h->st[b][4], tmp);
  else if (env.precision == USP_FP64_TANGENT)
    ch_to_host_layout<D3, D3><<<nb, 256, 0, s>>>(n, h->keycell, (const ChCellT<D3>*)h->cells,
        (D3*)h->st[b][0], (D3*)h->st[b][1], (D3*)h->st[b][2], (D3*)h->st[b][3], (D3*)h->st[b][4],
        tmp);
  else if (env.precision == USP_FP32_TANGENT)
    ch_to_host_layout<F3, D3><<<nb, 256, 0, s>>>(n, h->keycell, (const ChCellT<D3>*)h->cells,
        (F3*)h->st[b][0], (F3*)h->st[b][1], (F3*)h->st[b][2], (F3*)h->st[b][3], (F3*)h->st[b][4],
        tmp);
  else
    ch_to_host_layout<double, double><<<nb, 256, 0, s>>>(n, h->keycell,
        (const ChCellT<double>*)h->cells, (double*)h->st[b][0], (double*)h->st[b][1],
        (double*)h->st[b][2], (double*)h->st[b][3], (double*)h->st[b][4], tmp);
  std::vector<double> hl(5 * n);
  bool ok = cudaGetLastError() == cudaSuccess;
  ok = ok && cudaMemcpyAsync(hl.data(), tmp, 5 * n * sizeof(double), cudaMemcpyDeviceToHost, s) ==
                 cudaSuccess;
  ok = ok && cudaMemcpyAsync(lev, h->lv[b], n * 4, cudaMemcpyDeviceToHost, s) == cudaSuccess;
  if (pid)
    ok = ok && cudaMemcpyAsync(pid, h->pd[b], n * 4, cudaMemcpyDeviceToHost, s) == cudaSuccess;
  ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
  env.release(env.owner, tmp);
  if (!ok) return USP_ECUDA;
  for (long long j = 0; j < n; ++j) {
    if (y) y[j] = hl[j];
    cx[j] = hl[n + j]; cy[j] = hl[2 * n + j]; cz[j] = hl[3 * n + j]; erot[j] = hl[4 * n + j];
  }
  return USP_OK;
}

int ch_profiles(ChannelCtx* h, const ChEnv& env, double* out, int out_is_device) {
  cudaStream_t s = env.stream;
  ch_profiles<<<(h->ny + 127) / 128, 128, 0, s>>>(h->ny, h->blocks, h->acc, env.sp.R,
                                                   env.sp.theta_v, h->prof);
  CHK(cudaGetLastError());
  CHK(cudaMemcpyAsync(out, h->prof, sizeof(double) * USP_NPROF * h->ny * h->blocks,
                      out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (!out_is_device) CHK(cudaStreamSynchronize(s));
  return USP_OK;
}

int ch_backward(ChannelCtx* h, const ChEnv& env, const double* dL, double* grad3,
                int grad_is_device) {
  if (h->blocks != 1 + kND) return USP_ENOTSUP;
  cudaStream_t s = env.stream;
  CHK(cudaMemsetAsync(h->grad, 0, sizeof(double) * kND, s));
  const int nb = std::min(1024, (h->ny + 255) / 256);
  ch_backward<<<nb, 256, 0, s>>>(h->ny, h->acc, env.sp.R, dL, h->grad);
  CHK(cudaGetLastError());
  CHK(cudaMemcpyAsync(grad3, h->grad, sizeof(double) * kND,
                      grad_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (!grad_is_device) CHK(cudaStreamSynchronize(s));
  return USP_OK;
}

// The device buffers a step carries into the next one, in checkpoint order:
// the particle state of the current buffer (y, c, eps, levels, ids, cell
// keys), the per-cell records (pending conservation rescale, step moments),
// the time-average sums and the device step counter.
static int ch_segments(ChannelCtx* h, void** ptr, size_t* bytes) {
  const size_t nn = (size_t)std::max<long long>(h->n, 1);
  const bool grad = h->blocks > 1;
  const size_t cell_bytes = grad ? sizeof(ChCellT<D3>) : sizeof(ChCellT<double>);
  int k = 0;
  for (int f = 0; f < 5; ++f) { ptr[k] = h->st[h->cur][f]; bytes[k++] = nn * h->es; }
  ptr[k] = h->lv[h->cur]; bytes[k++] = nn * 4;
  ptr[k] = h->pd[h->cur]; bytes[k++] = nn * 4;
  ptr[k] = h->keycell; bytes[k++] = nn * 4;
  ptr[k] = h->cells; bytes[k++] = cell_bytes * h->ny;
  ptr[k] = h->acc; bytes[k++] = sizeof(double) * ((size_t)h->ny * kNAcc + 2) * h->blocks;
  ptr[k] = h->dstep; bytes[k++] = sizeof(long long);
  return k;
}

size_t ch_ckpt_bytes(ChannelCtx* h) {
  void* p[16];
  size_t b[16], t = 0;
  const int k = ch_segments(h, p, b);
  for (int i = 0; i < k; ++i) t += b[i];
  return t;
}

int ch_ckpt_copy(ChannelCtx* h, const ChEnv& env, unsigned char* buf, int buf_is_device,
                 int save) {
  void* p[16];
  size_t b[16];
  const int k = ch_segments(h, p, b);
  cudaMemcpyKind kind = buf_is_device ? cudaMemcpyDeviceToDevice
                                      : (save ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
  size_t o = 0;
  for (int i = 0; i < k; ++i) {
    if (save) CHK(cudaMemcpyAsync(buf + o, p[i], b[i], kind, env.stream));
    else CHK(cudaMemcpyAsync(p[i], buf + o, b[i], kind, env.stream));
    o += b[i];
  }
  return USP_OK;
}

int ch_sampling(const ChannelCtx* h) { return h->sampling; }

int ch_ncell(const ChannelCtx* h) { return h->ny; }
int ch_parity(const ChannelCtx* h) { return h->cur; }
long long ch_nparticles(const ChannelCtx* h) { return h->n; }
void ch_destroy(ChannelCtx* h) { delete h; }
