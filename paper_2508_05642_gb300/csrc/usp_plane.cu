// usp_plane.cu -- the spatial USP-FPM step on a uniform 2D Cartesian grid
// with a circular body (the hypersonic cylinder set-up of Kim & Jun, arXiv
// 2508.05642, Sec. 5.C: half body on a specular symmetry plane, fully
// diffuse cylinder, freestream inflow, supersonic outflow), on sm_103a.
//
// The particle count changes every step (inflow, outflow), so it lives on
// the device and every launch reads it there: a step is a fixed launch
// sequence that a CUDA graph can hold.  One step:
//   pl_advect      pending conservation rescale of the previous step, flight
//                  with events (cylinder hit -> diffuse re-emission at
//                  T_wall, sides -> specular / removal), new cell key; a
//                  removed particle gets the key ncell
//   pl_inflow      per inflow face the number of entering particles
//                  floor(flux A dt / F_num + u); exclusive scan over faces,
//                  capacity check, ids for the new particles
//   pl_inject      the entering particles: flux-weighted normal speed,
//                  Maxwellian tangential components, uniform entry point
//                  and entry time, flight for the rest of the step
//   radix passes   stable LSD radix sort of (cell key, index) over the moved
//                  and the new particles, 9-bit digits, removed ones last
//   pl_gather      live state permuted into cell order (other buffer), the
//                  cell segment starts and the new live count
//   ch_moments_coeffs_f32 (FP32 USP-FPM; else ch_moments, ch_coeffs or
//                  ch_coeffs_fpm)  per-cell moments and coefficients (Sec.
//                  2.A, 3.A), cut cells with their fluid volume
//   pl_params      per cell the reconstruction stencil of Sec. 3.B: for each
//                  side of the centroid the neighbour used along x and y and
//                  whether the quadrant's diagonal neighbour is usable
//   pl_collide     per particle: bilinear fields of its quadrant, collision
//                  of Sec. 4.D; per-cell sums
//   ch_fix_update  conservation of Sec. 4.C (rescale kept pending)
//   pl_sample      (while sampling) time-average sums of the post-step state
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "usp_plane.h"
#include "usp_spatial.cuh"

namespace {

constexpr uint32_t PTAG_INFLOW_P = 5u, PTAG_INFLOW_T = 6u, PTAG_INFLOW_V = 7u;
constexpr uint32_t CTAG_INFLOW = 0x80000004u;
constexpr int kInflowTries = 64;
constexpr int kBlk = 256;
constexpr int kNSurf = USP_NSURF;   // cylinder surface bins of the polar angle
constexpr int kParamBlock = 32;   // cells per block of the stencil pass

// Device-resident counts of the current step.
struct PlCount {
  long long n;        // live particles
  long long ntot;     // live + entering (before the sort)
  long long ninj;     // entering this step (0 if the storage was full)
  unsigned int pid0;  // id of the first entering particle
  unsigned int next_pid;
};

struct PlGeom {
  int nx, ny, ncell;
  double x0, x1, y0, y1, dx, dy;
  double cxc, cyc, cr;
  double Tw, dt;
  int bcbits;         // 2 bits per side (USP_BC_*): left, right, bottom, top
};

// The geometry's coordinates in the working precision, converted once on
// the host (an FP32 state would otherwise convert them per particle on the
// narrow FP64 pipe); for T = double the same values as PlGeom's.
template <typename T>
struct PlGeomT {
  T x0, x1, y0, y1, dx, dy, cxc, cyc, cr, dt;
  T RTw, Tw, theta, Rth;   // R T_wall, T_wall, Theta_v, R Theta_v
  T idx, idy;              // 1 / dx, 1 / dy
  T margin;                // 1e-5 of the domain's larger side
};
template <typename T>
PlGeomT<T> geom_t(const PlGeom& g, const Species& sp) {
  return {(T)g.x0, (T)g.x1, (T)g.y0, (T)g.y1, (T)g.dx, (T)g.dy, (T)g.cxc, (T)g.cyc, (T)g.cr,
          (T)g.dt, (T)(sp.R * g.Tw), (T)g.Tw, (T)sp.theta_v, (T)(sp.R * sp.theta_v),
          (T)(1.0 / g.dx), (T)(1.0 / g.dy),
          (T)(1e-5 * std::max(g.x1 - g.x0, g.y1 - g.y0))};
}

// Refined grid (levels 2, 3), in device memory: per level-1 cell its first
// cell, per level-2 child its first cell (-1: the level-1 cell is not split)
// and whether it is split again; per cell its level and integer coordinates
// at that level.  Kept out of PlGeom so that the uniform grid's flight
// kernels take the same parameters as without refinement.
struct PlTree {
  const int* l1_first;
  const int* l2_first;
  const signed char* l2_ref;
  const int* lvl;
  const int* lii;
  const int* ljj;
};

struct PlInflow {
  int nf[4];          // faces per side (0 if the side has no inflow)
  int base[4];        // first face of each side in the face list
  int nfaces;
  double expect[4];   // entering particles per face and step (flux A dt / F_num)
  double u_n[4];      // freestream velocity along the inward normal
  double RT, U, T;    // freestream R T, x velocity, temperature
};

// Per-cell parameters of the particle kernel, working precision T.
template <typename T>
struct PlParams {
  T alpha, nu_ref, B, mu_p, Pr, gtr, gtv, grv;
  T R, theta, dt;
  T xc, yc;
  T F[kNF];
  // the bilinear polynomial of each quadrant (sx, sy = 0 below / 1 at or
  // above the centroid): f = F + gx[sx] dx + gy[sy] dy + gxy[2 sy + sx] dx dy
  T gx[2][kNF], gy[2][kNF];
  union {
    T gxy[4][kNF];
    // the plain FPM method (cell values, no polynomial): alpha, sqrt(1 -
    // alpha^2) L, the rotational square-form constants and the level rates
    struct { T as, Lp[6], a_rot, sqrt_a, lam_up, lam_dn; } fpm;
  };
  int active, pad;
};

__device__ __forceinline__ int grid_threads() { return gridDim.x * blockDim.x; }

// the cell holding (x, y): the level-1 cell, then on a refined grid the
// half (and quarter) of it from the point's offset in units of half a cell
// (round-to-nearest operations: the FP64 form places points exactly as the
// plain definition does)
template <typename T, bool AMR>
__device__ __forceinline__ int plane_cell(const PlGeom& g, const PlGeomT<T>& gt,
                                          const PlTree* __restrict__ tr, T x, T y) {
  int i = (int)floor((x - gt.x0) / gt.dx);
  int j = (int)floor((y - gt.y0) / gt.dy);
  i = i < 0 ? 0 : (i >= g.nx ? g.nx - 1 : i);
  j = j < 0 ? 0 : (j >= g.ny ? g.ny - 1 : j);
  const int c = j * g.nx + i;
  if (!AMR) return c;
  const int first = tr->l2_first[4 * c];
  if (first < 0) return tr->l1_first[c];
  const T ux = rn_div(rn_sub(x, rn_add(gt.x0, rn_mul((T)i, gt.dx))), rn_mul(T(0.5), gt.dx));
  const T uy = rn_div(rn_sub(y, rn_add(gt.y0, rn_mul((T)j, gt.dy))), rn_mul(T(0.5), gt.dy));
  const int ci = ux >= T(1) ? 1 : 0, cj = uy >= T(1) ? 1 : 0;
  const int k = 2 * cj + ci;
  const int l = tr->l2_first[4 * c + k];
  if (!tr->l2_ref[4 * c + k]) return l;
  const T vx = rn_mul(rn_sub(ux, (T)ci), T(2)), vy = rn_mul(rn_sub(uy, (T)cj), T(2));
  return l + 2 * (vy >= T(1) ? 1 : 0) + (vx >= T(1) ? 1 : 0);
}

// Diffuse re-emission at T_w about the inward normal (nx, ny): Rayleigh
// normal speed, Maxwellian in-plane tangential and z components,
// exponential eps_rot, geometric level.  Draws (pid, step, 2, hit) and
// (pid, step, 3, hit).
// (The arithmetic is in the working precision T: the FP32 state's wall
// events and inflow stay off the FP64 pipe.)
template <typename T>
__device__ void plane_emit(const PlGeomT<T>& gt, T nx, T ny, uint32_t pid, uint32_t step, int hit,
                           uint32_t k0, uint32_t k1, T& vx, T& vy, T& vz, T& e, int& l) {
  const T RTw = gt.RTw;
  const U4 w = philox4x32_10(pid, step, PTAG_WALL_A, (uint32_t)hit, k0, k1);
  const U4 v = philox4x32_10(pid, step, PTAG_WALL_B, (uint32_t)hit, k0, k1);
  const T u0 = uniform_open<T>(w.x);
  const T u1 = uniform_open<T>(w.y);
  const T u2 = uniform_open<T>(w.z);
  const T u3 = uniform_open<T>(w.w);
  const T u4 = uniform_open<T>(v.x);
  const T vn = sqrt(T(-2) * RTw * log(u0));
  T g1, g2;
  box_muller(u1, u2, g1, g2);
  const T st = sqrt(RTw);
  const T tx = -ny, ty = nx;
  vx = vn * nx + st * g1 * tx;
  vy = vn * ny + st * g1 * ty;
  vz = st * g2;
  e = -RTw * log(u3);
  l = (int)floor(-log(u4) * gt.Tw / gt.theta);
}

// Flight over t_left with events, earliest first: cylinder (diffuse; a
// particle on or inside the surface moving inward hits it at once), left,
// right, bottom, top (ties to the earlier in that order).  An event
// moves the particle there and applies the side's condition; the flight
// continues for the rest of the time.  Returns false when the particle left
// through an open side.  hits counts the events met (at most 16).
template <typename T>
__device__ bool plane_fly(const PlGeom& g, const PlGeomT<T>& gt, uint32_t pid, uint32_t step,
                          uint32_t k0, uint32_t k1, T t_left, T& x, T& y, T& vx, T& vy, T& vz,
                          T& e, int& l, int& hits, uint32_t& fl, double* surf) {
  for (;;) {
    int ev = -1;
    T te = t_left;
    if (gt.cr > T(0)) {
      const T dx = x - gt.cxc, dy = y - gt.cyc;
      const T a = vx * vx + vy * vy;
      const T b = dx * vx + dy * vy;
      const T c = dx * dx + dy * dy - gt.cr * gt.cr;
      if (c > T(0) && b < T(0) && a > T(0)) {
        const T disc = b * b - a * c;
        if (disc >= T(0)) {
          const T t = (-b - sqrt(disc)) / a;
          if (t >= T(0) && t <= te) { te = t; ev = 0; }
        }
      } else if (c <= T(0) && b < T(0)) {
        // on or (by rounding, e.g. after a specular event at the body's foot
        // on the symmetry plane) inside the surface, moving inward: hit now
        te = T(0);
        ev = 0;
      }
    }
    // a side's time is formed only when the side may be met by te: in FP32
    // a particle whose straight move stops short of the side by more than a
    // margin far above rounding cannot reach it (the FP64 form always forms
    // the time)
    auto may = [&](T pos, T v, T side, bool lower) {
      if constexpr (sizeof(T) == 4) {
        const T end = pos + v * te;
        return lower ? end <= side + gt.margin : end >= side - gt.margin;
      } else {
        return true;
      }
    };
    if (vx < T(0) && may(x, vx, gt.x0, true)) {
      const T t = (gt.x0 - x) / vx;
      if (t <= te && (ev < 0 || t < te)) { te = t < T(0) ? T(0) : t; ev = 1; }
    }
    if (vx > T(0) && may(x, vx, gt.x1, false)) {
      const T t = (gt.x1 - x) / vx;
      if (t <= te && (ev < 0 || t < te)) { te = t < T(0) ? T(0) : t; ev = 2; }
    }
    if (vy < T(0) && may(y, vy, gt.y0, true)) {
      const T t = (gt.y0 - y) / vy;
      if (t <= te && (ev < 0 || t < te)) { te = t < T(0) ? T(0) : t; ev = 3; }
    }
    if (vy > T(0) && may(y, vy, gt.y1, false)) {
      const T t = (gt.y1 - y) / vy;
      if (t <= te && (ev < 0 || t < te)) { te = t < T(0) ? T(0) : t; ev = 4; }
    }
    if (ev < 0) {
      x += vx * t_left;
      y += vy * t_left;
      return true;
    }
    x += vx * te;
    y += vy * te;
    t_left -= te;
    if (hits >= kWallHitCap) {
      fl |= F_WALL_CAP;
      return true;
    }
    T nx = T(0), ny = T(0);
    int kind;
    if (ev == 0) {
      nx = (x - gt.cxc) / gt.cr;
      ny = (y - gt.cyc) / gt.cr;
      kind = USP_BC_DIFFUSE;
    } else {
      const int side = ev - 1;
      kind = (g.bcbits >> (2 * side)) & 3;
      if (side == 0) { nx = T(1); x = gt.x0; }
      if (side == 1) { nx = T(-1); x = gt.x1; }
      if (side == 2) { ny = T(1); y = gt.y0; }
      if (side == 3) { ny = T(-1); y = gt.y1; }
    }
    if (kind == USP_BC_OPEN) return false;
    if (kind == USP_BC_SPECULAR) {
      const T vn = vx * nx + vy * ny;
      vx -= T(2) * vn * nx;
      vy -= T(2) * vn * ny;
    } else {
      const T Rth = gt.Rth;
      const T in_x = vx, in_y = vy;
      const T in_e = T(0.5) * (vx * vx + vy * vy + vz * vz) + e + Rth * (T)l;
      plane_emit<T>(gt, nx, ny, pid, step, hits, k0, k1, vx, vy, vz, e, l);
      if (surf && ev == 0) {
        // surface tally of this wall event (bin of the polar angle)
        const double phi = atan2((double)(y - gt.cyc), (double)(x - gt.cxc));
        int b = (int)floor((phi + kPi) / (2.0 * kPi) * kNSurf);
        b = b < 0 ? 0 : (b > kNSurf - 1 ? kNSurf - 1 : b);
        const T out_e = T(0.5) * (vx * vx + vy * vy + vz * vz) + e + Rth * (T)l;
        atomicAdd(&surf[4 * b + 0], (double)(in_x - vx));
        atomicAdd(&surf[4 * b + 1], (double)(in_y - vy));
        atomicAdd(&surf[4 * b + 2], (double)(in_e - out_e));
        atomicAdd(&surf[4 * b + 3], 1.0);
      }
    }
    hits += 1;
  }
}

template <typename T, bool AMR>
__global__ void __launch_bounds__(kBlk, 3) pl_advect(PlGeom g, PlGeomT<T> gt,
                                                     const PlTree* __restrict__ tr,
                                                     const PlCount* __restrict__ cnt,
                          const int* keycell, const ChCellT<double>* __restrict__ cells,
                          const float* __restrict__ pend,
                          T* __restrict__ x, T* __restrict__ y, T* __restrict__ cx,
                          T* __restrict__ cy, T* __restrict__ cz, T* __restrict__ er,
                          int* __restrict__ lev, const uint32_t* __restrict__ pid,
                          int* keyout, int* __restrict__ idxout,
                          const long long* __restrict__ dstep, Species sp, uint32_t k0,
                          uint32_t k1, uint32_t* flags, unsigned long long* counters,
                          double* surf) {
  __shared__ BlockTally tal;
  tally_init(tal);
  const long long n = cnt->n;
  const uint32_t step = (uint32_t)*dstep;
  uint32_t fl = 0;
  unsigned long long nhit = 0, nout = 0;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += grid_threads()) {
    // pending conservation rescale of the previous step (FP32 state: its
    // FP32 copy, two 16-byte loads, so no FP64 conversion per particle)
    T vx, vy, vz, e;
    if constexpr (sizeof(T) == 4) {
      const float4* pc = reinterpret_cast<const float4*>(pend + (size_t)keycell[j] * 8);
      const float4 p0 = pc[0], p1 = pc[1];   // Un(3), Us(3), s, r
      vx = p0.x + p1.z * (cx[j] - p0.w);
      vy = p0.y + p1.z * (cy[j] - p1.x);
      vz = p0.z + p1.z * (cz[j] - p1.y);
      e = p1.w * er[j];
    } else {
      const ChCellT<double>& cc = cells[keycell[j]];
      vx = (T)cc.Un[0] + (T)cc.s * (cx[j] - (T)cc.Us[0]);
      vy = (T)cc.Un[1] + (T)cc.s * (cy[j] - (T)cc.Us[1]);
      vz = (T)cc.Un[2] + (T)cc.s * (cz[j] - (T)cc.Us[2]);
      e = (T)cc.r * er[j];
    }
    int l = lev[j];
    T px = x[j], py = y[j];
    int hits = 0;
    const bool keep = plane_fly<T>(g, gt, pid[j], step, k0, k1, gt.dt, px, py, vx, vy, vz, e, l,
                                   hits, fl, surf);
    nhit += hits;
    nout += keep ? 0 : 1;
    x[j] = px; y[j] = py; cx[j] = vx; cy[j] = vy; cz[j] = vz; er[j] = e; lev[j] = l;
    keyout[j] = keep ? plane_cell<T, AMR>(g, gt, tr, px, py) : g.ncell;
    idxout[j] = (int)j;
  }
  fl = __reduce_or_sync(0xffffffffu, fl);
  nhit = wsum(nhit);
  nout = wsum(nout);
  if ((threadIdx.x & 31) == 0) {
    tally_or(tal, fl);
    tally_add(tal, C_WALL_HITS, nhit);
    tally_add(tal, C_OUTFLOW, nout);
  }
  tally_flush(tal, flags, counters);
}

// per-side value without a dynamically indexed (local-memory) array
template <typename V>
__device__ __forceinline__ V pick4(const V (&a)[4], int side) {
  return side == 0 ? a[0] : (side == 1 ? a[1] : (side == 2 ? a[2] : a[3]));
}

// face q of the inflow list -> side and face index along the side
__device__ __forceinline__ void face_of(const PlInflow& f, int q, int& side, int& k) {
  side = (f.nf[0] > 0 && q < f.base[0] + f.nf[0]) ? 0
       : (f.nf[1] > 0 && q < f.base[1] + f.nf[1]) ? 1
       : (f.nf[2] > 0 && q < f.base[2] + f.nf[2]) ? 2 : 3;
  k = q - pick4(f.base, side);
}

// One block of 1024 threads: the number of particles entering through each
// face this step, floor(expect + u) with u from the cell stream
// (face id, step, 0x80000004, 0), face id = side << 24 | face; its exclusive
// scan; the capacity check and the ids of the new particles.
__global__ void pl_inflow(PlInflow f, PlCount* __restrict__ cnt, int* __restrict__ face_off,
                          long long cap, const long long* __restrict__ dstep, uint32_t k0,
                          uint32_t k1, uint32_t* flags, unsigned long long* counters) {
  __shared__ int wsums[32];
  __shared__ long long carry;
  const uint32_t step = (uint32_t)*dstep;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (t == 0) carry = 0;
  __syncthreads();
  for (int q0 = 0; q0 < f.nfaces; q0 += blockDim.x) {
    const int q = q0 + t;
    int c = 0;
    if (q < f.nfaces) {
      int side, k;
      face_of(f, q, side, k);
      const uint32_t fid = ((uint32_t)side << 24) | (uint32_t)k;
      const U4 r = philox4x32_10(fid, step, CTAG_INFLOW, 0u, k0, k1);
      c = (int)floor(pick4(f.expect, side) + uniform_open<double>(r.x));
    }
    // block exclusive scan of c
    int v = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) wsums[w] = v;
    __syncthreads();
    if (w == 0) {
      int s = lane < (int)(blockDim.x >> 5) ? wsums[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += u;
      }
      wsums[lane] = s;   // inclusive over warps
    }
    __syncthreads();
    const long long before = carry + (w > 0 ? wsums[w - 1] : 0) + (v - c);
    if (q < f.nfaces) face_off[q] = (int)before;
    __syncthreads();
    if (t == 0) carry += wsums[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (t == 0) {
    const long long total = carry;
    face_off[f.nfaces] = (int)total;
    const long long n = cnt->n;
    long long ninj = total;
    if (n + total > cap) {
      atomicOr(flags, (uint32_t)F_CAPACITY);
      ninj = 0;
    }
    cnt->ninj = ninj;
    cnt->ntot = n + ninj;
    cnt->pid0 = cnt->next_pid;
    cnt->next_pid = cnt->next_pid + (unsigned int)total;
    if (total) atomicAdd(&counters[C_INFLOW], (unsigned long long)total);
  }
}

// Inward normal speed of an entering particle (density proportional to
// w exp(-(w - s)^2) on w > 0, w = v_n / sqrt(2RT), s = u_n / sqrt(2RT)),
// by rejection, attempt k drawing the block (pid, step, 7, k): for s >= 0 a
// mixture proposal (|w - s| + s) exp(-(w - s)^2) (two-sided Rayleigh of
// weight 1, Gaussian of weight s sqrt(pi)), accepted if w > 0 and
// u3 (|w - s| + s) <= w; for s < 0 the Rayleigh proposal 2 w exp(-w^2),
// accepted if u3 <= exp(2 s w).  Double precision on uniforms of the
// working precision.
template <typename T>
__device__ T inflow_speed(T RT, T u_n, uint32_t pid, uint32_t step, uint32_t k0, uint32_t k1,
                          uint32_t& fl) {
  const T sc = sqrt(T(2) * RT);
  const T s = u_n / sc;
  const T p1 = T(1) / (T(1) + s * sqrt(T(kPi)));
  for (int k = 0; k < kInflowTries; ++k) {
    const U4 r = philox4x32_10(pid, step, PTAG_INFLOW_V, (uint32_t)k, k0, k1);
    const T u0 = uniform_open<T>(r.x), u1 = uniform_open<T>(r.y);
    const T u2 = uniform_open<T>(r.z), u3 = uniform_open<T>(r.w);
    if (s < T(0)) {
      const T wn = sqrt(-log(u1));
      if (u3 <= exp(T(2) * s * wn)) return wn * sc;
      continue;
    }
    T t;
    if (u0 < p1) {
      t = sqrt(-log(u1));
      if (u2 < T(0.5)) t = -t;
    } else {
      T g1, g2;
      box_muller(u1, u2, g1, g2);
      t = g1 / sqrt(T(2));
    }
    const T wn = s + t;
    if (!(wn > T(0))) continue;
    if (u3 * (fabs(t) + s) <= wn) return wn * sc;
  }
  fl |= F_INFLOW_CAP;
  return (s > T(0) ? s : T(0.5) * sqrt(T(kPi))) * sc;
}

// one thread per entering particle (grid-stride over the step's count); its
// face by binary search of the face offsets
template <typename T, bool AMR>
__global__ void __launch_bounds__(kBlk, 3) pl_inject(PlGeom g, PlGeomT<T> gt,
                                                     const PlTree* __restrict__ tr,
                                                     PlInflow f, const PlCount* __restrict__ cnt,
                          const int* __restrict__ face_off, T* __restrict__ x, T* __restrict__ y,
                          T* __restrict__ cx, T* __restrict__ cy, T* __restrict__ cz,
                          T* __restrict__ er, int* __restrict__ lev, uint32_t* __restrict__ pid,
                          int* __restrict__ keyout, int* __restrict__ idxout,
                          const long long* __restrict__ dstep, Species sp, uint32_t k0,
                          uint32_t k1, uint32_t* flags, unsigned long long* counters,
                          double* surf) {
  __shared__ BlockTally tal;
  tally_init(tal);
  const long long ninj = cnt->ninj;
  const uint32_t step = (uint32_t)*dstep;
  const long long n = cnt->n;
  // the freestream in the working precision
  struct { T RT, U, Tinf, u_n[4]; } fin = {(T)f.RT, (T)f.U, (T)f.T,
                                          {(T)f.u_n[0], (T)f.u_n[1], (T)f.u_n[2], (T)f.u_n[3]}};
  const T st = sqrt(fin.RT);
  uint32_t fl = 0;
  unsigned long long nhit = 0, nout = 0;
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < ninj;
       m += grid_threads()) {
    // face q: face_off[q] <= m < face_off[q + 1]
    int lo = 0, hi = f.nfaces - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (face_off[mid] <= m) lo = mid; else hi = mid - 1;
    }
    const int q = lo;
    int side, k;
    face_of(f, q, side, k);
    const T nxs = side == 0 ? T(1) : (side == 1 ? T(-1) : T(0));
    const T nys = side == 2 ? T(1) : (side == 3 ? T(-1) : T(0));
    const uint32_t id = cnt->pid0 + (uint32_t)m;
    const U4 a = philox4x32_10(id, step, PTAG_INFLOW_P, 0u, k0, k1);
    const U4 bb = philox4x32_10(id, step, PTAG_INFLOW_T, 0u, k0, k1);
    const T u_pos = uniform_open<T>(a.x), u_t = uniform_open<T>(a.y);
    T g1, g2;
    box_muller(uniform_open<T>(bb.x), uniform_open<T>(bb.y), g1, g2);
    const T vn = inflow_speed<T>(fin.RT, pick4(fin.u_n, side), id, step, k0, k1, fl);
    T X, Y, VX, VY;
    if (side < 2) {
      X = side == 0 ? gt.x0 : gt.x1;
      Y = gt.y0 + ((T)k + u_pos) * gt.dy;
      VX = vn * nxs;
      VY = st * g1;
    } else {
      X = gt.x0 + ((T)k + u_pos) * gt.dx;
      Y = side == 2 ? gt.y0 : gt.y1;
      VX = fin.U + st * g1;
      VY = vn * nys;
    }
    T VZ = st * g2;
    T E = -fin.RT * log(uniform_open<T>(a.z));
    const int l0 = (int)floor(-log(uniform_open<T>(a.w)) * fin.Tinf / gt.theta);
    int L = l0, hits = 0;
    const bool keep = plane_fly<T>(g, gt, id, step, k0, k1, u_t * gt.dt, X, Y, VX, VY, VZ, E, L,
                                   hits, fl, surf);
    nhit += hits;
    nout += keep ? 0 : 1;
    const long long j = n + m;
    x[j] = X; y[j] = Y; cx[j] = VX; cy[j] = VY; cz[j] = VZ; er[j] = E; lev[j] = L; pid[j] = id;
    keyout[j] = keep ? plane_cell<T, AMR>(g, gt, tr, X, Y) : g.ncell;
    idxout[j] = (int)j;
  }
  fl = __reduce_or_sync(0xffffffffu, fl);
  nhit = wsum(nhit);
  nout = wsum(nout);
  if ((threadIdx.x & 31) == 0) {
    tally_or(tal, fl);
    tally_add(tal, C_WALL_HITS, nhit);
    tally_add(tal, C_OUTFLOW, nout);
  }
  tally_flush(tal, flags, counters);
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (key, index) over the device count ntot, kDig-bit
// digits (two passes cover the 240,001 keys of the 600 x 400 grid);
// histograms digit-major (bh[d * nblk + b])
// ---------------------------------------------------------------------------
constexpr int kDig = 9;
constexpr int kNB = 1 << kDig;

__global__ void pl_hist(const int* __restrict__ key, const PlCount* __restrict__ cnt, int shift,
                        int* __restrict__ bh, int nblk) {
  __shared__ int h[kNB];
  for (int d = threadIdx.x; d < kNB; d += kRB) h[d] = 0;
  __syncthreads();
  const long long n = cnt->ntot;
  const long long b = (long long)blockIdx.x * kChunk;
  if (b >= n) return;   // uniform over the block: no keys, a column no one reads
  {
    // every key of the thread loaded first (the loads in flight together)
    int kk[kRPT];
#pragma unroll
    for (int r = 0; r < kRPT; ++r) {
      const long long i = b + (long long)r * kRB + threadIdx.x;
      kk[r] = i < n ? key[i] : -1;
    }
#pragma unroll
    for (int r = 0; r < kRPT; ++r)
      if (kk[r] >= 0) atomicAdd(&h[(kk[r] >> shift) & (kNB - 1)], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kNB; d += kRB) bh[(size_t)d * nblk + blockIdx.x] = h[d];
}

// one block per digit: exclusive scan over the blocks that hold keys (the
// rest of the storage's blocks are empty and read by no one), digit total
__global__ void pl_scan_digits(int* __restrict__ bh, int nblk, const PlCount* __restrict__ cnt,
                               int* __restrict__ tot) {
  __shared__ int ws[kRB / 32];
  __shared__ int carry;
  const int d = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  int* row = bh + (size_t)d * nblk;
  const int nb = (int)min((long long)nblk, (cnt->ntot + kChunk - 1) / kChunk);
  if (t == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += kRB) {
    const int b = b0 + t;
    const int c = b < nb ? row[b] : 0;
    int v = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) ws[w] = v;
    __syncthreads();
    int pre = 0;
    for (int k = 0; k < w; ++k) pre += ws[k];
    if (b < nb) row[b] = carry + pre + v - c;
    __syncthreads();
    if (t == 0) {
      int sum = 0;
      for (int k = 0; k < kRB / 32; ++k) sum += ws[k];
      carry += sum;
    }
    __syncthreads();
  }
  if (t == 0) tot[d] = carry;
}

__global__ void pl_scatter(const int* __restrict__ kin, const int* __restrict__ iin,
                           int* __restrict__ kout, int* __restrict__ iout,
                           const PlCount* __restrict__ cnt, int shift, const int* __restrict__ bh,
                           const int* __restrict__ tot, int nblk) {
  __shared__ int cntw[kRB / 32][kNB];
  __shared__ int run[kNB];
  __shared__ int wsum_[kRB / 32];
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const long long n = cnt->ntot;
  const long long b = (long long)blockIdx.x * kChunk;
  if (b >= n) return;
  // exclusive scan of the digit totals: thread t owns digits t * kPer .. + kPer - 1
  constexpr int kPer = kNB / kRB;
  int loc[kPer];
  int own = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    loc[q] = tot[t * kPer + q];
    own += loc[q];
  }
  int v = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) wsum_[w] = v;
  __syncthreads();
  int pre = v - own;
  for (int k = 0; k < w; ++k) pre += wsum_[k];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int d = t * kPer + q;
    run[d] = pre + bh[(size_t)d * nblk + blockIdx.x];
    pre += loc[q];
  }
  __syncthreads();
  // per round of kRB keys: each warp's count of every digit it holds (set by
  // the digit's first lane, cleared by it after use, so only the touched
  // entries change), the position from the digit's run and the counts of
  // the earlier warps, then the run advanced by each warp's count.  The keys
  // and indices of a round are loaded two rounds ahead.
  for (int q = 0; q < kRB / 32; ++q)
    for (int d = t; d < kNB; d += kRB) cntw[q][d] = 0;
  auto load = [&](int r, int& k_, int& i_) {
    const long long i = b + (long long)r * kRB + t;
    if (r < kRPT && i < n) { k_ = kin[i]; i_ = iin[i]; }
  };
  int k0 = 0, i0 = 0, k1 = 0, i1 = 0;
  load(0, k0, i0);
  load(1, k1, i1);
  __syncthreads();
  for (int r = 0; r < kRPT; ++r) {
    int k2 = 0, i2 = 0;
    load(r + 2, k2, i2);
    const bool valid = b + (long long)r * kRB + t < n;
    const int d = valid ? ((k0 >> shift) & (kNB - 1)) : kNB;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lane_lt());
    const bool lead = valid && rank == 0;
    if (lead) cntw[w][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int p = 0;
      for (int q = 0; q < w; ++q) p += cntw[q][d];
      const int pos = run[d] + p + rank;
      kout[pos] = k0;
      iout[pos] = i0;
    }
    __syncthreads();
    if (lead) {
      atomicAdd(&run[d], cntw[w][d]);
      cntw[w][d] = 0;
    }
    __syncwarp();
    k0 = k1; i0 = i1; k1 = k2; i1 = i2;
  }
}

// The live state permuted into cell order (other buffer), and the cell
// segment starts from the sorted keys (keys in [0, ncell], ncell = removed
// particles, which are not copied): where the key changes between j - 1 and
// j, the cells in between start at j.  The new live count is the start of
// the removed particles' segment.  The sorted keys stay where the sort left
// them and serve as the particles' cells from here on.
template <typename T>
__global__ void pl_gather(PlCount* __restrict__ cnt, int ncell, long long* __restrict__ off,
                          const int* __restrict__ idx, const int* __restrict__ ksorted,
                          const T* __restrict__ x0, const T* __restrict__ y0,
                          const T* __restrict__ vx0, const T* __restrict__ vy0,
                          const T* __restrict__ vz0, const T* __restrict__ e0,
                          const int* __restrict__ l0, const uint32_t* __restrict__ p0,
                          T* __restrict__ x1, T* __restrict__ y1, T* __restrict__ vx1,
                          T* __restrict__ vy1, T* __restrict__ vz1, T* __restrict__ e1,
                          int* __restrict__ l1, uint32_t* __restrict__ p1) {
  const long long n = cnt->ntot;
  const long long j0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n == 0) {
    for (long long c = j0; c <= ncell; c += grid_threads()) off[c] = 0;
    if (j0 == 0) cnt->n = 0;
    return;
  }
  for (long long j = j0; j < n; j += grid_threads()) {
    const int k = ksorted[j];
    const int prev = j > 0 ? ksorted[j - 1] : -1;
    for (int c = prev + 1; c <= k; ++c) off[c] = j;
    if (k == ncell && prev < ncell) cnt->n = j;
    if (j == n - 1 && k < ncell) {
      for (int c = k + 1; c <= ncell; ++c) off[c] = n;
      cnt->n = n;
    }
    if (k < ncell) {
      const int s = idx[j];
      x1[j] = x0[s]; y1[j] = y0[s]; vx1[j] = vx0[s]; vy1[j] = vy0[s]; vz1[j] = vz0[s];
      e1[j] = e0[s]; l1[j] = l0[s]; p1[j] = p0[s];
    }
  }
}

// ---------------------------------------------------------------------------
// reconstruction stencils (Sec. 3.B on the uniform grid): for each side of
// the centroid the x and y neighbour used (that side's if usable, else the
// opposite one, else none) and the quadrant's diagonal when usable
// ---------------------------------------------------------------------------
// cells per block of the uniform grid's stencil pass (its static shared
// memory stays under 48 KB)
template <typename T>
constexpr int kStencilBlock = sizeof(T) == 4 ? 64 : 32;

template <typename T>
__global__ void __launch_bounds__(kStencilBlock<T>)
pl_params(PlGeom g, PlGeomT<T> gt, int recon, const ChCellT<double>* __restrict__ cells,
          const T* __restrict__ fT, const int* __restrict__ usable_c,
          PlParams<T>* __restrict__ prm, Species sp, const double* __restrict__ fpm) {
  // a thread builds its cell's record in shared memory; the block then copies
  // its records out as consecutive 8-byte words (coalesced), where one thread
  // storing a ~0.5 KB record would scatter every store.  The fields and
  // usable flags of the block's cells and their neighbours (three runs of
  // kSpan consecutive cells: the rows below, at and above) are staged first,
  // with coalesced loads.
  constexpr int kB = kStencilBlock<T>;
  constexpr int kSpan = kB + 2;
  __shared__ PlParams<T> buf[kB];
  __shared__ T sf[3][kSpan][kNF];
  __shared__ int su[3][kSpan];
  const int c0 = blockIdx.x * kB;
  const int c = c0 + threadIdx.x;
  const int nb = min(kB, g.ncell - c0);
  // cell of run r (row offset r - 1), place m: c0 - 1 + (r - 1) nx + m
  for (int e = threadIdx.x; e < 3 * kSpan * kNF; e += kB) {
    const int r = e / (kSpan * kNF), m = (e / kNF) % kSpan, k = e % kNF;
    const int cc = c0 - 1 + (r - 1) * g.nx + m;
    sf[r][m][k] = cc >= 0 && cc < g.ncell ? fT[(size_t)cc * kNF + k] : T(0);
  }
  for (int e = threadIdx.x; e < 3 * kSpan; e += kB) {
    const int r = e / kSpan, m = e % kSpan;
    const int cc = c0 - 1 + (r - 1) * g.nx + m;
    su[r][m] = cc >= 0 && cc < g.ncell ? usable_c[cc] : 0;
  }
  __syncthreads();
  if (c < g.ncell) {
    const ChCellT<double>& cs = cells[c];
    PlParams<T>& P = buf[threadIdx.x];
    P.active = cs.active;
    P.pad = 0;
    P.alpha = (T)cs.alpha; P.nu_ref = (T)cs.nu_ref; P.B = (T)cs.B; P.mu_p = (T)cs.mu_p;
    P.Pr = (T)cs.Pr; P.gtr = (T)cs.gtr; P.gtv = (T)cs.gtv; P.grv = (T)cs.grv;
    P.R = (T)gasR(sp); P.theta = gt.theta; P.dt = gt.dt;
    const int i = c % g.nx, j = c / g.nx;
    P.xc = (T)(g.x0 + (i + 0.5) * g.dx);
    P.yc = (T)(g.y0 + (j + 0.5) * g.dy);
    // neighbour (i + di, j + dj): run dj + 1, place threadIdx.x + 1 + di
    const int m0 = threadIdx.x + 1;
    const T* f = sf[1][m0];
    for (int k = 0; k < kNF; ++k) P.F[k] = f[k];
    if (fpm) {
      // the plain FPM method: cell values, its per-cell constants
      for (int k = 0; k < kNF; ++k) { P.gx[0][k] = P.gx[1][k] = P.gy[0][k] = P.gy[1][k] = T(0); }
      const double* r = fpm + (size_t)c * kFpmRec;
      P.fpm.as = (T)r[0];
      for (int k = 0; k < 6; ++k) P.fpm.Lp[k] = (T)r[1 + k];
      P.fpm.a_rot = (T)r[7]; P.fpm.sqrt_a = (T)r[8];
      P.fpm.lam_up = (T)r[9]; P.fpm.lam_dn = (T)r[10];
    } else {
      auto usable = [&](int di, int dj) {
        const int ii = i + di, jj = j + dj;
        return recon && ii >= 0 && ii < g.nx && jj >= 0 && jj < g.ny && su[dj + 1][m0 + di];
      };
      auto field = [&](int di, int dj) { return sf[dj + 1][m0 + di]; };
      // slopes in the working precision from the cell values, times 1/offset
      int ox[2], oy[2];   // the x and y neighbour of each side (offset; 0: none)
      for (int sd = 0; sd < 2; ++sd) {
        const int sg = sd ? 1 : -1;
        ox[sd] = usable(sg, 0) ? sg : (usable(-sg, 0) ? -sg : 0);
        oy[sd] = usable(0, sg) ? sg : (usable(0, -sg) ? -sg : 0);
        if (ox[sd] != 0) {
          const T* fn = field(ox[sd], 0);
          const T ih = ox[sd] > 0 ? gt.idx : -gt.idx;
          for (int k = 0; k < kNF; ++k) P.gx[sd][k] = (fn[k] - f[k]) * ih;
        } else {
          for (int k = 0; k < kNF; ++k) P.gx[sd][k] = T(0);
        }
        if (oy[sd] != 0) {
          const T* fn = field(0, oy[sd]);
          const T ih = oy[sd] > 0 ? gt.idy : -gt.idy;
          for (int k = 0; k < kNF; ++k) P.gy[sd][k] = (fn[k] - f[k]) * ih;
        } else {
          for (int k = 0; k < kNF; ++k) P.gy[sd][k] = T(0);
        }
      }
      for (int q = 0; q < 4; ++q) {
        const int sx = q & 1, sy = q >> 1;
        if (ox[sx] != 0 && oy[sy] != 0 && usable(ox[sx], oy[sy])) {
          const T* fd = field(ox[sx], oy[sy]);
          const T* fx = field(ox[sx], 0);
          const T* fy = field(0, oy[sy]);
          const T ih = ((ox[sx] > 0) == (oy[sy] > 0) ? T(1) : T(-1)) * gt.idx * gt.idy;
          for (int k = 0; k < kNF; ++k) P.gxy[q][k] = (fd[k] - fx[k] - fy[k] + f[k]) * ih;
        } else {
          for (int k = 0; k < kNF; ++k) P.gxy[q][k] = T(0);
        }
      }
    }
  }
  __syncthreads();
  static_assert(sizeof(PlParams<T>) % 8 == 0, "records copied as 8-byte words");
  const int words = nb * (int)(sizeof(PlParams<T>) / 8);
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(buf);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(prm + c0);
  for (int w = threadIdx.x; w < words; w += kB) dst[w] = src[w];
}

// ---------------------------------------------------------------------------
// reconstruction stencils on the refined grid (Sec. 3.B, non-uniform grids):
// the same formula as on the uniform grid, with the average over each
// neighbouring square of the cell's own size taken from the cell of that
// size there, the particle-number weighted mean of the four finer cells
// filling it, or the coarser cell's polynomial at the square's centre (its
// average over the square).  A square is usable when every cell in it is
// (whole, two particles or more).  One launch per level, coarsest first, so that
// a coarser neighbour's record is complete when a finer cell reads it.
// ---------------------------------------------------------------------------
// The cell holding the centre of the level-L square (I, J) (integer
// coordinates at level L, inside the domain): the point location of that
// centre in integer form.  A centre never lies on the edge of a cell of level
// L or coarser; where it is the common corner of finer cells, any of them
// stands for "finer" (here the one the >= rule of the point location takes).
__device__ __forceinline__ int leaf_at(const PlGeom& g, const PlTree* __restrict__ tr, int L, int I,
                                       int J) {
  const int c = (J >> (L - 1)) * g.nx + (I >> (L - 1));
  if (tr->l2_first[4 * c] < 0) return tr->l1_first[c];
  const int k = L == 1 ? 3 : ((((J >> (L - 2)) & 1) << 1) | ((I >> (L - 2)) & 1));
  const int l = tr->l2_first[4 * c + k];
  if (!tr->l2_ref[4 * c + k]) return l;
  return L <= 2 ? l + 3 : l + (((J & 1) << 1) | (I & 1));
}

template <typename T>
__device__ bool pl_region(const PlGeom& g, const PlTree* __restrict__ tr,
                          const PlParams<T>* __restrict__ prm,
                          const T* __restrict__ fT, const int* __restrict__ usable_c,
                          const long long* __restrict__ off, int lvl, int ii, int jj, int di,
                          int dj, double h, double k, T* val) {
  const int I = ii + di, J = jj + dj;
  if (I < 0 || J < 0 || I >= (g.nx << (lvl - 1)) || J >= (g.ny << (lvl - 1))) return false;
  const int l = leaf_at(g, tr, lvl, I, J);
  const int ll = tr->lvl[l];
  if (ll == lvl) {
    if (!usable_c[l]) return false;
    for (int f = 0; f < kNF; ++f) val[f] = fT[(size_t)l * kNF + f];
    return true;
  }
  if (ll > lvl) {
    int q[4];
    long long nq[4], ns = 0;
    for (int a = 0; a < 4; ++a) {
      q[a] = leaf_at(g, tr, lvl + 1, 2 * I + (a & 1), 2 * J + (a >> 1));
      if (tr->lvl[q[a]] != lvl + 1 || !usable_c[q[a]]) return false;
      nq[a] = off[q[a] + 1] - off[q[a]];
      ns += nq[a];
    }
    for (int f = 0; f < kNF; ++f) {
      T sum = T(0);
      for (int a = 0; a < 4; ++a) sum += (T)nq[a] * fT[(size_t)q[a] * kNF + f];
      val[f] = sum / (T)ns;
    }
    return true;
  }
  if (!usable_c[l]) return false;
  const PlParams<T>& C = prm[l];
  const double cx = rn_add(g.x0, rn_mul((double)I + 0.5, h));
  const double cy = rn_add(g.y0, rn_mul((double)J + 0.5, k));
  const T ex = (T)cx - C.xc, ey = (T)cy - C.yc;
  const int sx = ex >= T(0) ? 1 : 0, sy = ey >= T(0) ? 1 : 0;
  for (int f = 0; f < kNF; ++f)
    val[f] = C.F[f] + C.gx[sx][f] * ex + C.gy[sy][f] * ey + C.gxy[2 * sy + sx][f] * ex * ey;
  return true;
}

// blocks: the kParamBlock-cell blocks holding cells of this level
template <typename T>
__global__ void pl_params_amr(PlGeom g, const PlTree* __restrict__ tr, int recon, int level,
                              const int* __restrict__ blocks,
                              const ChCellT<double>* __restrict__ cells, const T* __restrict__ fT,
                              const int* __restrict__ usable_c, const long long* __restrict__ off,
                              PlParams<T>* __restrict__ prm, Species sp) {
  __shared__ PlParams<T> buf[kParamBlock];
  const int c0 = blocks[blockIdx.x] * kParamBlock;
  const int c = c0 + threadIdx.x;
  const int nb = min(kParamBlock, g.ncell - c0);
  if (c < g.ncell && tr->lvl[c] == level) {
    const ChCellT<double>& cs = cells[c];
    PlParams<T>& P = buf[threadIdx.x];
    P.active = cs.active;
    P.pad = 0;
    P.alpha = (T)cs.alpha; P.nu_ref = (T)cs.nu_ref; P.B = (T)cs.B; P.mu_p = (T)cs.mu_p;
    P.Pr = (T)cs.Pr; P.gtr = (T)cs.gtr; P.gtv = (T)cs.gtv; P.grv = (T)cs.grv;
    P.R = (T)gasR(sp); P.theta = (T)sp.theta_v; P.dt = (T)g.dt;
    const double sc = (double)(1 << (level - 1));
    const double h = g.dx / sc, k = g.dy / sc;
    const int ii = tr->lii[c], jj = tr->ljj[c];
    P.xc = (T)rn_add(g.x0, rn_mul((double)ii + 0.5, h));
    P.yc = (T)rn_add(g.y0, rn_mul((double)jj + 0.5, k));
    const T* f = fT + (size_t)c * kNF;
    for (int q = 0; q < kNF; ++q) P.F[q] = f[q];
    const T ih = (T)(1.0 / h), ik = (T)(1.0 / k);
    T PX[2][kNF], PY[2][kNF], PD[kNF];
    int ox[2] = {0, 0}, oy[2] = {0, 0};
    for (int sd = 0; sd < 2; ++sd) {
      const int sg = sd ? 1 : -1;
      if (recon) {
        if (pl_region<T>(g, tr, prm, fT, usable_c, off, level, ii, jj, sg, 0, h, k, PX[sd]))
          ox[sd] = sg;
        else if (pl_region<T>(g, tr, prm, fT, usable_c, off, level, ii, jj, -sg, 0, h, k, PX[sd]))
          ox[sd] = -sg;
        if (pl_region<T>(g, tr, prm, fT, usable_c, off, level, ii, jj, 0, sg, h, k, PY[sd]))
          oy[sd] = sg;
        else if (pl_region<T>(g, tr, prm, fT, usable_c, off, level, ii, jj, 0, -sg, h, k, PY[sd]))
          oy[sd] = -sg;
      }
      const T sx = ox[sd] > 0 ? ih : -ih, sy = oy[sd] > 0 ? ik : -ik;
      for (int q = 0; q < kNF; ++q) {
        P.gx[sd][q] = ox[sd] ? (PX[sd][q] - f[q]) * sx : T(0);
        P.gy[sd][q] = oy[sd] ? (PY[sd][q] - f[q]) * sy : T(0);
      }
    }
    for (int q = 0; q < 4; ++q) {
      const int sx = q & 1, sy = q >> 1;
      const bool d = ox[sx] && oy[sy] &&
                     pl_region<T>(g, tr, prm, fT, usable_c, off, level, ii, jj, ox[sx], oy[sy], h,
                                  k, PD);
      const T s = (ox[sx] * oy[sy] > 0 ? T(1) : T(-1)) * ih * ik;
      for (int m = 0; m < kNF; ++m)
        P.gxy[q][m] = d ? (PD[m] - PX[sx][m] - PY[sy][m] + f[m]) * s : T(0);
    }
  }
  __syncthreads();
  // copy out the records of this level only (the others belong to the other
  // launches)
  constexpr int kW = (int)(sizeof(PlParams<T>) / 8);
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(buf);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(prm + c0);
  for (int w = threadIdx.x; w < nb * kW; w += kParamBlock)
    if (tr->lvl[c0 + w / kW] == level) dst[w] = src[w];
}

// Asynchronous global -> shared copies of 4, 8 or 16 bytes (cp.async): the
// plane collision prefetches the next cell's data while it works on the
// current one.
template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  static_assert(B == 4 || B == 8 || B == 16, "cp.async copies 4, 8 or 16 bytes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "n"(B)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Per-warp staging of one cell for pl_collide: its stencil record, then up to
// kPC particles (x, y, cx, cy, cz, erot in T; level; id).  A cell with more
// particles reads the rest directly.
constexpr int kPC = 64;
template <typename T>
struct PlStage {
  static constexpr size_t arr = (sizeof(PlParams<T>) + 15) / 16 * 16;
  static constexpr size_t bytes = arr + (size_t)kPC * (6 * sizeof(T) + 8);
};
// the cell's place and size, active flag and bulk velocity, staged one cell
// ahead of the particles
struct PlMeta {
  long long off, N;
  double U[3];
  int active, pad;
};
template <typename T>
constexpr size_t pl_collide_smem() {
  return (size_t)(kBlk / 32) * (2 * PlStage<T>::bytes + 3 * sizeof(PlMeta));
}

// per particle: the bilinear polynomial of its quadrant, then the collision
// of Sec. 4.D; one warp per cell, per-cell sums for the conservation step.
// Each warp walks its cells (c, c + W, c + 2W, ...) as a pipeline: while it
// works on cell c out of shared memory, cp.async copies of cell c + W's
// stencil record and particles and of cell c + 2W's place and size are in
// flight, so the DRAM latency of a cell overlaps the previous cell's
// arithmetic.
// METHOD 0: USP-FPM with the reconstructed fields; 1: the plain FPM method
template <typename T, int METHOD>
__global__ void __launch_bounds__(kBlk, 2) pl_collide(int ncell, const ChCellT<double>* __restrict__ cells,
                           const PlParams<T>* __restrict__ prm, const T* __restrict__ x,
                           const T* __restrict__ y, T* __restrict__ cx, T* __restrict__ cy,
                           T* __restrict__ cz, T* __restrict__ er, int* __restrict__ lev,
                           const uint32_t* __restrict__ pid, ChSumsT<double>* __restrict__ sums,
                           const long long* __restrict__ dstep, const PhiloxRoundKeys rk,
                           uint32_t* flags, unsigned long long* counters) {
  extern __shared__ __align__(16) unsigned char pl_smem[];
  __shared__ BlockTally tal;
  using L = PlStage<T>;
  tally_init(tal);
  const int lane = threadIdx.x & 31;
  const uint32_t step = (uint32_t)*dstep;
  unsigned char* wbase =
      pl_smem + (size_t)(threadIdx.x >> 5) * (2 * L::bytes + 3 * sizeof(PlMeta));
  PlMeta* meta = reinterpret_cast<PlMeta*>(wbase + 2 * L::bytes);
  const int W = warps_total();

  // copy cell cc's place, size, flag and velocity into slot m (lanes 0-5)
  auto stage_meta = [&](int cc, PlMeta* m) {
    if (cc < ncell) {
      const ChCellT<double>& cs = cells[cc];
      if (lane == 0) cp_async<8>(&m->off, &cs.off);
      else if (lane == 1) cp_async<8>(&m->N, &cs.N);
      else if (lane < 5) cp_async<8>(&m->U[lane - 2], &cs.U[lane - 2]);
      else if (lane == 5) cp_async<4>(&m->active, &cs.active);
    } else if (lane == 0) {
      m->active = 0;
      m->N = 0;
    }
  };
  // copy cell cc's stencil record and first kPC particles into buffer b
  auto stage_cell = [&](int cc, const PlMeta* m, unsigned char* b) {
    if (cc >= ncell || !m->active) return;
    const unsigned char* src = reinterpret_cast<const unsigned char*>(prm + cc);
    if constexpr (sizeof(PlParams<T>) % 16 == 0) {
      for (int w = lane; w < (int)(sizeof(PlParams<T>) / 16); w += 32)
        cp_async<16>(b + 16 * w, src + 16 * w);
    } else {
      for (int w = lane; w < (int)(sizeof(PlParams<T>) / 8); w += 32)
        cp_async<8>(b + 8 * w, src + 8 * w);
    }
    const long long off = m->off;
    const int n = (int)min(m->N, (long long)kPC);
    T* A = reinterpret_cast<T*>(b + L::arr);
    int* Lv = reinterpret_cast<int*>(A + 6 * kPC);
    uint32_t* Pd = reinterpret_cast<uint32_t*>(Lv + kPC);
    for (int i = lane; i < n; i += 32) {
      const long long j = off + i;
      cp_async<sizeof(T)>(A + i, x + j);
      cp_async<sizeof(T)>(A + kPC + i, y + j);
      cp_async<sizeof(T)>(A + 2 * kPC + i, cx + j);
      cp_async<sizeof(T)>(A + 3 * kPC + i, cy + j);
      cp_async<sizeof(T)>(A + 4 * kPC + i, cz + j);
      cp_async<sizeof(T)>(A + 5 * kPC + i, er + j);
      cp_async<4>(Lv + i, lev + j);
      cp_async<4>(Pd + i, pid + j);
    }
  };

  int c = warp_global();
  // prologue: place of the first cell, then its data and the next one's place
  stage_meta(c, &meta[0]);
  cp_async_commit();
  cp_async_wait_all();
  __syncwarp();
  stage_cell(c, &meta[0], wbase);
  stage_meta(c + W, &meta[1]);
  cp_async_commit();
  int slot = 0, buf = 0;
  // event counts and flags per lane over all of the warp's cells, reduced
  // once at the end
  CollideTally tl = {0u, 0ull, 0ull, 0ull, 0ull};
  unsigned long long nfb = 0;
  for (; c < ncell; c += W) {
    // cell c's data and cell c + W's place are in shared memory once every
    // lane's copies are done; the previous cell's readers are done too
    cp_async_wait_all();
    __syncwarp();
    const int s1 = slot == 2 ? 0 : slot + 1, s2 = s1 == 2 ? 0 : s1 + 1;
    stage_cell(c + W, &meta[s1], wbase + (buf ^ 1) * L::bytes);
    stage_meta(c + 2 * W, &meta[s2]);
    cp_async_commit();
    const PlMeta& m = meta[slot];
    if (m.active) {
      const unsigned char* b = wbase + buf * L::bytes;
      const PlParams<T>& P = *reinterpret_cast<const PlParams<T>*>(b);
      const T* A = reinterpret_cast<const T*>(b + L::arr);
      const int* Lv = reinterpret_cast<const int*>(A + 6 * kPC);
      const uint32_t* Pd = reinterpret_cast<const uint32_t*>(Lv + kPC);
      const long long off = m.off;
      const int n = (int)m.N;
      // cell velocity in T: one conversion per warp (lanes 0-2), then broadcast
      const T uc = (T)(lane < 3 ? m.U[lane < 3 ? lane : 0] : 0.0);
      const T Uc0 = __shfl_sync(0xffffffffu, uc, 0), Uc1 = __shfl_sync(0xffffffffu, uc, 1),
              Uc2 = __shfl_sync(0xffffffffu, uc, 2);
      T acc[10];
#pragma unroll
      for (int i = 0; i < 10; ++i) acc[i] = T(0);
      int accI = 0;
      int maxI = 0;
      for (int i = lane; i < n; i += 32) {
        const long long j = off + i;
        T xv, yv, v0, v1, v2, en;
        int l0;
        uint32_t id;
        if (i < kPC) {
          xv = A[i]; yv = A[kPC + i]; v0 = A[2 * kPC + i]; v1 = A[3 * kPC + i];
          v2 = A[4 * kPC + i]; en = A[5 * kPC + i]; l0 = Lv[i]; id = Pd[i];
        } else {
          xv = x[j]; yv = y[j]; v0 = cx[j]; v1 = cy[j]; v2 = cz[j]; en = er[j];
          l0 = lev[j]; id = pid[j];
        }
        int ln;
        if constexpr (METHOD == 1) {
          ln = fpm_particle<T>(P.F, P.fpm.as, P.fpm.Lp, P.fpm.a_rot, P.fpm.sqrt_a, P.fpm.lam_up,
                               P.fpm.lam_dn, v0, v1, v2, en, l0, id, step, rk, tl.fl);
        } else {
          const T ddx = xv - P.xc, ddy = yv - P.yc;
          const int sx = ddx >= T(0) ? 1 : 0, sy = ddy >= T(0) ? 1 : 0;
          const T dxy = ddx * ddy;
          const T* gx = P.gx[sx];
          const T* gy = P.gy[sy];
          const T* gxy = P.gxy[sy * 2 + sx];
          T f[kNF];
#pragma unroll
          for (int q = 0; q < kNF; ++q) f[q] = P.F[q] + gx[q] * ddx + gy[q] * ddy + gxy[q] * dxy;
          if (!(f[3] > T(0)) || !(f[4] > T(0)) || !(f[5] >= T(0))) {
#pragma unroll
            for (int q = 0; q < kNF; ++q) f[q] = P.F[q];
            ++nfb;
          }
          ln = collide_particle_t<sizeof(T) == 4>(P, f, v0, v1, v2, en, l0, id, step, rk, tl);
        }
        cx[j] = v0; cy[j] = v1; cz[j] = v2; er[j] = en;
        lev[j] = ln;
        maxI = max(maxI, ln);
        const T d0 = v0 - Uc0, d1 = v1 - Uc1, d2 = v2 - Uc2;
        acc[0] += d0; acc[1] += d1; acc[2] += d2;
        acc[3] += d0 * d0; acc[4] += d1 * d1; acc[5] += d2 * d2;
        acc[6] += d0 * d1; acc[7] += d0 * d2; acc[8] += d1 * d2;
        acc[9] += en;
        accI += ln;
      }
      // warp totals; lane i < 10 converts total i (one FP64 conversion per warp)
      T mine = T(0);
#pragma unroll
      for (int i = 0; i < 10; ++i) {
        const T t = wsum(acc[i]);
        mine = lane == i ? t : mine;
      }
      const double sv = (double)mine;
      const long long sI = wsum((long long)accI);
      const int mI = __reduce_max_sync(0xffffffffu, maxI);
      ChSumsT<double>& sm = sums[c];
      if (lane < 10) sm.v[lane] = sv;
      if (lane == 0) {
        sm.I = (unsigned long long)sI;
        sm.net = 0;
        sm.maxI = mI;
      }
    }
    slot = s1;
    buf ^= 1;
  }
  cp_async_wait_all();
  {
    const unsigned long long fix = wsum(tl.nfix), fb = wsum(nfb), ncl2 = wsum(tl.ncl),
                             pb = wsum(tl.npb), nz = wsum(tl.nnz);
    const uint32_t fla = __reduce_or_sync(0xffffffffu, tl.fl);
    if (lane == 0) {
      tally_or(tal, fla);
      tally_add(tal, C_CHOL_FIX, fix);
      tally_add(tal, C_INTERP_FALLBACK, fb);
      tally_add(tal, C_TREL_CLAMP, ncl2);
      tally_add(tal, C_PB_CLAMP, pb);
      tally_add(tal, C_NU_ZERO, nz);
    }
  }
  tally_flush(tal, flags, counters);
}

// time-average sums of the post-step state, binned by cell
template <typename T>
__global__ void pl_sample(const PlCount* __restrict__ cnt, int ncell,
                          const int* __restrict__ keycell,
                          const ChCellT<double>* __restrict__ cells, const T* __restrict__ cx,
                          const T* __restrict__ cy, const T* __restrict__ cz,
                          const T* __restrict__ er, const int* __restrict__ lev,
                          double* __restrict__ acc) {
  const long long n = cnt->n;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&acc[(size_t)ncell * kNAcc], 1.0);
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += grid_threads()) {
    const int k = keycell[j];
    const ChCellT<double>& cc = cells[k];
    const double v0 = cc.Un[0] + cc.s * ((double)cx[j] - cc.Us[0]);
    const double v1 = cc.Un[1] + cc.s * ((double)cy[j] - cc.Us[1]);
    const double v2 = cc.Un[2] + cc.s * ((double)cz[j] - cc.Us[2]);
    const double e = cc.r * (double)er[j];
    double* a = acc + (size_t)k * kNAcc;
    atomicAdd(&a[0], 1.0);
    atomicAdd(&a[1], v0); atomicAdd(&a[2], v1); atomicAdd(&a[3], v2);
    atomicAdd(&a[4], v0 * v0); atomicAdd(&a[5], v1 * v1); atomicAdd(&a[6], v2 * v2);
    atomicAdd(&a[7], v0 * v1); atomicAdd(&a[8], v0 * v2); atomicAdd(&a[9], v1 * v2);
    atomicAdd(&a[10], e);
    atomicAdd(&a[11], (double)lev[j]);
  }
}

// on-demand moments of the current state: pass 0 raw sums, pass 1 central
template <typename T>
__global__ void pl_mom_pass(int pass, const PlCount* __restrict__ cnt,
                            const int* __restrict__ keycell,
                            const ChCellT<double>* __restrict__ cells, const T* __restrict__ cx,
                            const T* __restrict__ cy, const T* __restrict__ cz,
                            const T* __restrict__ er, const int* __restrict__ lev,
                            double* __restrict__ a) {
  const long long n = cnt->n;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += grid_threads()) {
    const int k = keycell[j];
    const ChCellT<double>& cc = cells[k];
    const double v0 = cc.Un[0] + cc.s * ((double)cx[j] - cc.Us[0]);
    const double v1 = cc.Un[1] + cc.s * ((double)cy[j] - cc.Us[1]);
    const double v2 = cc.Un[2] + cc.s * ((double)cz[j] - cc.Us[2]);
    const double ep = cc.r * (double)er[j];
    const double li = (double)lev[j];
    double* A = a + (size_t)k * 21;
    if (pass == 0) {
      atomicAdd(&A[0], 1.0);
      atomicAdd(&A[1], v0); atomicAdd(&A[2], v1); atomicAdd(&A[3], v2);
      atomicAdd(&A[4], ep); atomicAdd(&A[5], li);
      continue;
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
}

template <typename T>
__global__ void pl_to_host_layout(long long n, const int* __restrict__ keycell,
                                  const ChCellT<double>* __restrict__ cells,
                                  const T* __restrict__ x, const T* __restrict__ y,
                                  const T* __restrict__ cx, const T* __restrict__ cy,
                                  const T* __restrict__ cz, const T* __restrict__ er,
                                  double* __restrict__ out) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const ChCellT<double>& cc = cells[keycell[j]];
  out[j] = (double)x[j];
  out[n + j] = (double)y[j];
  out[2 * n + j] = cc.Un[0] + cc.s * ((double)cx[j] - cc.Us[0]);
  out[3 * n + j] = cc.Un[1] + cc.s * ((double)cy[j] - cc.Us[1]);
  out[4 * n + j] = cc.Un[2] + cc.s * ((double)cz[j] - cc.Us[2]);
  out[5 * n + j] = cc.r * (double)er[j];
}

template <typename T>
__global__ void pl_from_host_layout(long long n, const double* __restrict__ in,
                                    T* __restrict__ x, T* __restrict__ y, T* __restrict__ cx,
                                    T* __restrict__ cy, T* __restrict__ cz, T* __restrict__ er) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  x[j] = (T)in[j]; y[j] = (T)in[n + j]; cx[j] = (T)in[2 * n + j]; cy[j] = (T)in[3 * n + j];
  cz[j] = (T)in[4 * n + j]; er[j] = (T)in[5 * n + j];
}

}  // namespace

// ===========================================================================
// host side
// ===========================================================================
struct PlaneCtx {
  PlGeom g;
  PlInflow inf;
  int recon, passes, nblk, grid_p;
  int grid_wc, grid_tc;     // grids of the warp-per-cell and thread-per-cell passes
  int grid_col;             // persistent grid of the collision pass
  int grid_inj;             // grid of the inflow pass (grid-stride over entering particles)
  double Fnum, vol;
  long long cap;
  size_t es;
  void* st[2][6];           // x, y, cx, cy, cz, eps (ping-pong)
  int* lv[2];
  uint32_t* pd[2];
  int cur;
  int* kbuf[2];
  int* ibuf[2];
  int* keycell;
  int* bh;
  int* tot;
  int* face_off;
  long long* off;
  double* af;
  double* afv;              // af / 4^(level-1): the cell volume over dx dy depth
  int* blk_lv;              // refined grid: per level the stencil blocks holding its cells
  double* fpmrec;           // the plain FPM method: kFpmRec per-cell constants (else null)
  int levels;               // 1 uniform, 2 or 3 refined
  PlTree* tree;             // refined grid tables (device; null on the uniform grid)
  PlTree htree;             // the same pointers, host copy
  int blk_off[4], nblk_lv[4];
  PlCount* cnt;
  ChCellT<double>* cells;
  float* pend;              // FP32 copy of the pending rescale (Un, Us, s, r) per cell
  void* fT;                 // cell fields in the particle precision (ncell x 13)
  int* usable_c;            // reconstruction-neighbour flag per cell
  void* prm;                // PlParams<T>
  ChSumsT<double>* sums;
  double* acc;
  double* macc;
  double* mout;
  long long* dstep;
  int sampling;
};

namespace {

#define CHK(x)                                 \
  do {                                         \
    if ((x) != cudaSuccess) return USP_ECUDA;  \
  } while (0)

double inflow_flux(double n, double RT, double u_n) {
  // one-way number flux of a drifting Maxwellian through a surface element
  const double s = u_n / std::sqrt(2.0 * RT);
  return n * std::sqrt(RT / (2.0 * kPi)) * (std::exp(-s * s) + std::sqrt(kPi) * s * (1.0 + std::erf(s)));
}

// Refined grid of a plane (Sec. 5.C): level-1 cells row-major, a split cell
// replaced by its 2 x 2 children in the order (0,0), (1,0), (0,1), (1,1),
// each of which may be split once more.  A cell is split when its centre
// lies within the level's radius of the body centre and not all of it lies
// inside the body.  Plain arithmetic (the host build keeps a * b + c
// unfused), so the layout and point location repeat the plain definition.
struct PlGrid {
  int levels = 1, nleaf = 0;
  bool balanced = true;
  std::vector<int> l1_first, l2_first, lvl, lii, ljj;
  std::vector<signed char> l2_ref;
};

bool pg_centre_in(const usp_plane* p, double xl, double yl, double w, double h, double r) {
  const double ex = xl + 0.5 * w - p->cyl_xc, ey = yl + 0.5 * h - p->cyl_yc;
  return ex * ex + ey * ey < r * r;
}

bool pg_solid(const usp_plane* p, double xl, double yl, double w, double h) {
  if (!(p->cyl_r > 0.0)) return false;
  const double r2 = p->cyl_r * p->cyl_r;
  for (int q = 0; q < 4; ++q) {
    const double ex = xl + (q & 1) * w - p->cyl_xc, ey = yl + (q >> 1) * h - p->cyl_yc;
    if (ex * ex + ey * ey > r2) return false;
  }
  return true;
}

void pg_build(const usp_plane* p, PlGrid& G) {
  const int nx = p->nx, ny = p->ny, n1 = nx * ny;
  const double dx = (p->x1 - p->x0) / nx, dy = (p->y1 - p->y0) / ny;
  G.levels = p->amr_levels >= 2 ? p->amr_levels : 1;
  G.l1_first.assign(n1 + 1, 0);
  G.l2_first.assign((size_t)4 * n1, -1);
  G.l2_ref.assign((size_t)4 * n1, 0);
  G.lvl.clear(); G.lii.clear(); G.ljj.clear();
  for (int c = 0; c < n1; ++c) {
    const int i = c % nx, j = c / nx;
    G.l1_first[c] = (int)G.lvl.size();
    const double xl = p->x0 + i * dx, yl = p->y0 + j * dy;
    if (!(G.levels >= 2 && pg_centre_in(p, xl, yl, dx, dy, p->amr_r2) &&
          !pg_solid(p, xl, yl, dx, dy))) {
      G.lvl.push_back(1); G.lii.push_back(i); G.ljj.push_back(j);
      continue;
    }
    for (int k = 0; k < 4; ++k) {
      const double xk = xl + (k & 1) * 0.5 * dx, yk = yl + (k >> 1) * 0.5 * dy;
      const int i2 = 2 * i + (k & 1), j2 = 2 * j + (k >> 1);
      const bool s3 = G.levels >= 3 && pg_centre_in(p, xk, yk, 0.5 * dx, 0.5 * dy, p->amr_r3) &&
                      !pg_solid(p, xk, yk, 0.5 * dx, 0.5 * dy);
      G.l2_first[(size_t)4 * c + k] = (int)G.lvl.size();
      G.l2_ref[(size_t)4 * c + k] = s3 ? 1 : 0;
      if (!s3) {
        G.lvl.push_back(2); G.lii.push_back(i2); G.ljj.push_back(j2);
        continue;
      }
      for (int q = 0; q < 4; ++q) {
        G.lvl.push_back(3); G.lii.push_back(2 * i2 + (q & 1)); G.ljj.push_back(2 * j2 + (q >> 1));
      }
    }
  }
  G.nleaf = (int)G.lvl.size();
  G.l1_first[n1] = G.nleaf;
  // neighbouring fluid cells differ by one level at most: the eight
  // neighbours of a level-1 cell holding level-3 cells are split or solid
  G.balanced = true;
  for (int c = 0; c < n1 && G.balanced; ++c) {
    bool deep = false;
    for (int k = 0; k < 4; ++k) deep = deep || G.l2_ref[(size_t)4 * c + k];
    if (!deep) continue;
    const int i = c % nx, j = c / nx;
    for (int b = j - 1; b <= j + 1; ++b)
      for (int a = i - 1; a <= i + 1; ++a) {
        if (a < 0 || a >= nx || b < 0 || b >= ny || (a == i && b == j)) continue;
        const int m = b * nx + a;
        if (G.l2_first[(size_t)4 * m] < 0 && !pg_solid(p, p->x0 + a * dx, p->y0 + b * dy, dx, dy))
          G.balanced = false;
      }
  }
}

// the cell holding (x, y), as plane_cell on the device
int pg_leaf(const usp_plane* p, const PlGrid& G, double x, double y) {
  const double dx = (p->x1 - p->x0) / p->nx, dy = (p->y1 - p->y0) / p->ny;
  int i = (int)std::floor((x - p->x0) / dx), j = (int)std::floor((y - p->y0) / dy);
  i = std::min(std::max(i, 0), p->nx - 1);
  j = std::min(std::max(j, 0), p->ny - 1);
  const int c = j * p->nx + i;
  if (G.levels < 2 || G.l2_first[(size_t)4 * c] < 0) return G.l1_first[c];
  const double ux = (x - (p->x0 + i * dx)) / (0.5 * dx), uy = (y - (p->y0 + j * dy)) / (0.5 * dy);
  const int ci = ux >= 1.0 ? 1 : 0, cj = uy >= 1.0 ? 1 : 0;
  const int k = 2 * cj + ci;
  const int l = G.l2_first[(size_t)4 * c + k];
  if (!G.l2_ref[(size_t)4 * c + k]) return l;
  const double vx = (ux - ci) * 2.0, vy = (uy - cj) * 2.0;
  return l + 2 * (vy >= 1.0 ? 1 : 0) + (vx >= 1.0 ? 1 : 0);
}

// sizes and refinement parameters of a plane; 0 or USP_EINVAL
int pg_check(const usp_plane* p) {
  if (!p || p->nx <= 0 || p->ny <= 0 || (long long)p->nx * p->ny >= (1 << 24) ||
      !(p->x1 > p->x0) || !(p->y1 > p->y0))
    return USP_EINVAL;
  if (p->amr_levels < 0 || p->amr_levels > 3) return USP_EINVAL;
  if (p->amr_levels >= 2 && !(p->amr_r2 > 0.0 && std::isfinite(p->amr_r2))) return USP_EINVAL;
  if (p->amr_levels >= 3 && !(p->amr_r3 > 0.0 && std::isfinite(p->amr_r3))) return USP_EINVAL;
  return 0;
}

template <typename T>
int pl_step_t(PlaneCtx* h, const ChEnv& env, ch_prof_fn prof) {
  cudaStream_t s = env.stream;
  const int a = h->cur, b = a ^ 1;
  T* x = (T*)h->st[a][0]; T* y = (T*)h->st[a][1]; T* cx = (T*)h->st[a][2];
  T* cy = (T*)h->st[a][3]; T* cz = (T*)h->st[a][4]; T* er = (T*)h->st[a][5];
  const int ncell = h->g.ncell;
  if (prof) prof(env.owner, 0, 1);
  // surface tallies of the cylinder while sampling
  double* surf = h->sampling ? h->acc + (size_t)ncell * kNAcc + 2 : nullptr;
  // the uniform grid takes the point location without the refined-grid branch
  const bool amr = h->levels >= 2;
  const PlGeomT<T> gt = geom_t<T>(h->g, env.sp);
  (amr ? pl_advect<T, true> : pl_advect<T, false>)<<<h->grid_p, kBlk, 0, s>>>(
      h->g, gt, h->tree, h->cnt, h->keycell, h->cells, h->pend, x, y, cx, cy, cz, er, h->lv[a], h->pd[a],
      h->kbuf[0], h->ibuf[0], h->dstep, env.sp, env.k0, env.k1, env.flags, env.counters, surf);
  pl_inflow<<<1, 1024, 0, s>>>(h->inf, h->cnt, h->face_off, h->cap, h->dstep, env.k0, env.k1,
                               env.flags, env.counters);
  if (h->inf.nfaces > 0)
    (amr ? pl_inject<T, true> : pl_inject<T, false>)<<<h->grid_inj, kBlk, 0, s>>>(
        h->g, gt, h->tree, h->inf, h->cnt, h->face_off, x, y, cx, cy, cz, er, h->lv[a], h->pd[a], h->kbuf[0],
        h->ibuf[0], h->dstep, env.sp, env.k0, env.k1, env.flags, env.counters, surf);
  CHK(cudaGetLastError());
  int src = 0;
  for (int p = 0; p < h->passes; ++p) {
    pl_hist<<<h->nblk, kRB, 0, s>>>(h->kbuf[src], h->cnt, kDig * p, h->bh, h->nblk);
    pl_scan_digits<<<kNB, kRB, 0, s>>>(h->bh, h->nblk, h->cnt, h->tot);
    pl_scatter<<<h->nblk, kRB, 0, s>>>(h->kbuf[src], h->ibuf[src], h->kbuf[src ^ 1],
                                       h->ibuf[src ^ 1], h->cnt, kDig * p, h->bh, h->tot, h->nblk);
    CHK(cudaGetLastError());
    src ^= 1;
  }
  // the sorted keys end in kbuf[passes & 1], which keycell names
  pl_gather<T><<<h->grid_p, kBlk, 0, s>>>(h->cnt, ncell, h->off, h->ibuf[src], h->kbuf[src], x, y,
                                          cx, cy, cz, er, h->lv[a], h->pd[a], (T*)h->st[b][0],
                                          (T*)h->st[b][1], (T*)h->st[b][2], (T*)h->st[b][3],
                                          (T*)h->st[b][4], (T*)h->st[b][5], h->lv[b], h->pd[b]);
  CHK(cudaGetLastError());
  h->cur = b;
  x = (T*)h->st[b][0]; y = (T*)h->st[b][1]; cx = (T*)h->st[b][2]; cy = (T*)h->st[b][3];
  cz = (T*)h->st[b][4]; er = (T*)h->st[b][5];
  if (prof) prof(env.owner, 0, 0);
  if (prof) prof(env.owner, 1, 1);
  const int wb = h->grid_wc, tb = h->grid_tc;
  float* pend = env.precision == USP_FP32 ? h->pend : nullptr;
  const bool fpm = h->fpmrec != nullptr;
  // the FP32 form of USP-FPM takes its moments and FP32 coefficients in one
  // pass; the FP64 form and the plain FPM method in two
  const bool fused = sizeof(T) == 4 && !fpm;
  if (fused)
    ch_moments_coeffs_f32<<<(ncell + 32 * kMW - 1) / (32 * kMW), 32 * kMW, 0, s>>>(
        ncell, h->off, h->af, h->afv, (float)(h->Fnum / h->vol), h->g.dt, (const float*)cx,
        (const float*)cy, (const float*)cz, (const float*)er, h->lv[b], h->cells, env.sp,
        env.flags, env.counters, pend, (float*)h->fT, h->usable_c);
  else
    ch_moments<T, double><<<wb, kBlk, 0, s>>>(ncell, 32, h->off, h->af, cx, cy, cz, er, h->lv[b],
                                              h->cells, env.sp, env.counters, pend, (T*)h->fT,
                                              h->usable_c);
  if (fpm)
    ch_coeffs_fpm<<<tb, kBlk, 0, s>>>(ncell, h->Fnum, h->vol, h->afv, h->g.dt, h->cells,
                                      h->fpmrec, env.sp, env.flags, env.counters);
  else if (!fused)
    ch_coeffs<double><<<tb, kBlk, 0, s>>>(ncell, h->Fnum, h->vol, h->afv, h->g.dt, h->cells,
                                          env.sp, env.sp.omega, env.sp.Z_rot, env.flags,
                                          env.counters);
  if (fpm || h->levels < 2)
    pl_params<T><<<(ncell + kStencilBlock<T> - 1) / kStencilBlock<T>, kStencilBlock<T>, 0, s>>>(
        h->g, gt, fpm ? 0 : h->recon, h->cells, (const T*)h->fT, h->usable_c,
        (PlParams<T>*)h->prm, env.sp, h->fpmrec);
  else
    for (int L = 1; L <= h->levels; ++L)
      if (h->nblk_lv[L] > 0)
        pl_params_amr<T><<<h->nblk_lv[L], kParamBlock, 0, s>>>(
            h->g, h->tree, h->recon, L, h->blk_lv + h->blk_off[L], h->cells, (const T*)h->fT,
            h->usable_c, h->off, (PlParams<T>*)h->prm, env.sp);
  CHK(cudaGetLastError());
  if (prof) prof(env.owner, 1, 0);
  if (prof) prof(env.owner, 0, 1);
  if (fpm)
    pl_collide<T, 1><<<h->grid_col, kBlk, pl_collide_smem<T>(), s>>>(
        ncell, h->cells, (const PlParams<T>*)h->prm, x, y, cx, cy, cz, er, h->lv[b], h->pd[b],
        h->sums, h->dstep, philox_round_keys(env.k0, env.k1), env.flags, env.counters);
  else
    pl_collide<T, 0><<<h->grid_col, kBlk, pl_collide_smem<T>(), s>>>(
        ncell, h->cells, (const PlParams<T>*)h->prm, x, y, cx, cy, cz, er, h->lv[b], h->pd[b],
        h->sums, h->dstep, philox_round_keys(env.k0, env.k1), env.flags, env.counters);
  CHK(cudaGetLastError());
  if (prof) prof(env.owner, 0, 0);
  if (prof) prof(env.owner, 1, 1);
  if (pend)
    ch_fix_update<true><<<wb, kBlk, 0, s>>>(ncell, h->cells, h->sums, h->lv[b], h->dstep, env.sp,
                                             env.k0, env.k1, env.flags, env.counters, pend);
  else
    ch_fix_update<false><<<wb, kBlk, 0, s>>>(ncell, h->cells, h->sums, h->lv[b], h->dstep, env.sp,
                                              env.k0, env.k1, env.flags, env.counters, nullptr);
  CHK(cudaGetLastError());
  if (h->sampling) {
    pl_sample<T><<<h->grid_p, kBlk, 0, s>>>(h->cnt, ncell, h->keycell, h->cells, cx, cy, cz, er,
                                            h->lv[b], h->acc);
    CHK(cudaGetLastError());
  }
  if (prof) prof(env.owner, 1, 0);
  return USP_OK;
}

}  // namespace

int pl_kernels_per_step(const PlaneCtx* h) {
  int params = 1;
  if (h->levels >= 2 && !h->fpmrec) {
    params = 0;
    for (int L = 1; L <= h->levels; ++L) params += h->nblk_lv[L] > 0 ? 1 : 0;
  }
  const int cellpass = h->es == sizeof(float) && !h->fpmrec ? 1 : 2;
  return 2 + (h->inf.nfaces > 0 ? 1 : 0) + 3 * h->passes + 1 + cellpass + params + 1 + 1 +
         (h->sampling ? 1 : 0);
}

int pl_launch_step(PlaneCtx* h, const ChEnv& env, ch_prof_fn prof) {
  if (env.precision == USP_FP32) return pl_step_t<float>(h, env, prof);
  if (env.precision == USP_FP64) return pl_step_t<double>(h, env, prof);
  return USP_ENOTSUP;
}

int pl_create(PlaneCtx** out, const ChEnv& env, const usp_plane* pp, double dt,
              const double* area_frac, int64_t n, int64_t cap, int64_t step0, const double* x,
              const double* y, const double* cx, const double* cy, const double* cz,
              const double* erot, const int32_t* lev, const uint32_t* pid) {
  if (pg_check(pp) || !(pp->F_num > 0) || !(pp->depth > 0) || !(dt > 0) || n < 0 || cap < n ||
      cap < 1 || cap > 0x7fffffffll)
    return USP_EINVAL;
  if (env.precision != USP_FP32 && env.precision != USP_FP64) return USP_ENOTSUP;
  for (int k = 0; k < 4; ++k) {
    if (pp->bc[k] < USP_BC_OPEN || pp->bc[k] > USP_BC_DIFFUSE) return USP_EINVAL;
    if (pp->inflow[k] && pp->bc[k] != USP_BC_OPEN) return USP_EINVAL;
  }
  const bool any_inflow = pp->inflow[0] || pp->inflow[1] || pp->inflow[2] || pp->inflow[3];
  if (any_inflow && !(pp->n_inf > 0 && pp->T_inf > 0)) return USP_EINVAL;
  if ((pp->cyl_r > 0 || pp->bc[0] == USP_BC_DIFFUSE || pp->bc[1] == USP_BC_DIFFUSE ||
       pp->bc[2] == USP_BC_DIFFUSE || pp->bc[3] == USP_BC_DIFFUSE) && !(pp->T_wall > 0))
    return USP_EINVAL;
  if (n > 0 && (!x || !y || !cx || !cy || !cz || !erot || !lev)) return USP_EINVAL;
  if (!area_frac) return USP_EINVAL;
  PlGrid G;
  pg_build(pp, G);
  if (!G.balanced || G.nleaf >= (1 << 24)) return USP_EINVAL;
  const int ncell = G.nleaf;
  for (int c = 0; c < ncell; ++c)
    if (!(area_frac[c] >= 0.0 && area_frac[c] <= 1.0)) return USP_EINVAL;
  for (int64_t j = 0; j < n; ++j)
    if (!(x[j] >= pp->x0 && x[j] <= pp->x1 && y[j] >= pp->y0 && y[j] <= pp->y1) || lev[j] < 0)
      return USP_EINVAL;
  PlaneCtx* h = new PlaneCtx();
  std::memset((void*)h, 0, sizeof(PlaneCtx));
  PlGeom& g = h->g;
  g.nx = pp->nx; g.ny = pp->ny; g.ncell = ncell;
  g.x0 = pp->x0; g.x1 = pp->x1; g.y0 = pp->y0; g.y1 = pp->y1;
  g.dx = (pp->x1 - pp->x0) / pp->nx; g.dy = (pp->y1 - pp->y0) / pp->ny;
  g.cxc = pp->cyl_xc; g.cyc = pp->cyl_yc; g.cr = pp->cyl_r > 0 ? pp->cyl_r : 0.0;
  g.Tw = pp->T_wall; g.dt = dt;
  h->levels = G.levels;
  g.bcbits = 0;
  for (int k = 0; k < 4; ++k) g.bcbits |= (pp->bc[k] & 3) << (2 * k);
  h->recon = pp->reconstruct ? 1 : 0;
  h->Fnum = pp->F_num;
  h->vol = g.dx * g.dy * pp->depth;
  h->cap = cap;
  // inflow faces, sides in the order left, right, bottom, top
  PlInflow& f = h->inf;
  const double R = env.sp.m > 0 ? kB / env.sp.m : 0.0;
  f.RT = R * pp->T_inf; f.U = pp->U_inf; f.T = pp->T_inf;
  f.nfaces = 0;
  for (int k = 0; k < 4; ++k) {
    f.nf[k] = pp->inflow[k] ? (k < 2 ? pp->ny : pp->nx) : 0;
    f.base[k] = f.nfaces;
    f.nfaces += f.nf[k];
    const double nxs = k == 0 ? 1.0 : (k == 1 ? -1.0 : 0.0);
    f.u_n[k] = pp->U_inf * nxs;
    f.expect[k] = 0.0;
    if (pp->inflow[k]) {
      const double flen = k < 2 ? g.dy : g.dx;
      f.expect[k] = inflow_flux(pp->n_inf, f.RT, f.u_n[k]) * flen * pp->depth * dt / pp->F_num;
    }
  }
  h->es = env.precision == USP_FP32 ? 4 : 8;
  int bits = 1;
  while ((1 << bits) < ncell + 1) ++bits;
  h->passes = (bits + kDig - 1) / kDig;
  h->nblk = (int)std::max<long long>(1, (cap + kChunk - 1) / kChunk);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (nsm <= 0) nsm = 1;
  h->grid_p = (int)std::min<long long>(std::max<long long>(1, (cap + kBlk - 1) / kBlk), nsm * 16);
  h->grid_wc = (int)std::min<long long>(((long long)ncell * 32 + kBlk - 1) / kBlk, nsm * 8);
  h->grid_tc = (int)std::min<long long>((ncell + kBlk - 1) / kBlk, nsm * 8);
  {
    // the collision pass keeps one block per resident slot, each warp a
    // pipeline over its cells
    const bool f32 = env.precision == USP_FP32;
    const bool m1 = env.sp.method == 1;
    const void* fn = f32 ? (m1 ? (const void*)pl_collide<float, 1> : (const void*)pl_collide<float, 0>)
                         : (m1 ? (const void*)pl_collide<double, 1> : (const void*)pl_collide<double, 0>);
    const int smem = (int)(f32 ? pl_collide_smem<float>() : pl_collide_smem<double>());
    int per_sm = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlk, smem) != cudaSuccess)
      per_sm = 0;
    if (per_sm <= 0) { pl_destroy(h); return USP_ECUDA; }
    h->grid_col = (int)std::min<long long>(((long long)ncell * 32 + kBlk - 1) / kBlk,
                                           (long long)nsm * per_sm);
  }
  h->grid_inj = nsm * 4;
  auto A = [&](size_t bytes) { return env.alloc(env.owner, bytes); };
  const size_t nn = (size_t)cap;
  for (int k = 0; k < 2; ++k) {
    for (int q = 0; q < 6; ++q) h->st[k][q] = A(nn * h->es);
    h->lv[k] = (int*)A(nn * 4);
    h->pd[k] = (uint32_t*)A(nn * 4);
    h->kbuf[k] = (int*)A(nn * 4);
    h->ibuf[k] = (int*)A(nn * 4);
  }
  // the particles' cells: the sorted keys, where the last radix pass leaves them
  h->keycell = h->kbuf[h->passes & 1];

  h->bh = (int*)A((size_t)h->nblk * kNB * 4);
  h->tot = (int*)A(kNB * 4);
  h->face_off = (int*)A(sizeof(int) * (f.nfaces + 1));
  h->off = (long long*)A(sizeof(long long) * (ncell + 1));
  h->af = (double*)A(sizeof(double) * ncell);
  h->afv = h->af;
  if (env.sp.method == 1) h->fpmrec = (double*)A(sizeof(double) * kFpmRec * (size_t)ncell);
  const int n1 = pp->nx * pp->ny;
  if (G.levels >= 2) {
    h->afv = (double*)A(sizeof(double) * ncell);
    PlTree& t = h->htree;
    t.l1_first = (const int*)A(sizeof(int) * (n1 + 1));
    t.l2_first = (const int*)A(sizeof(int) * 4 * (size_t)n1);
    t.l2_ref = (const signed char*)A(4 * (size_t)n1);
    t.lvl = (const int*)A(sizeof(int) * ncell);
    t.lii = (const int*)A(sizeof(int) * ncell);
    t.ljj = (const int*)A(sizeof(int) * ncell);
    h->tree = (PlTree*)A(sizeof(PlTree));
  }
  // per level the stencil blocks (kParamBlock consecutive cells) holding its cells
  std::vector<int> blk;
  if (G.levels >= 2) {
    const int nb = (ncell + kParamBlock - 1) / kParamBlock;
    for (int L = 1; L <= 3; ++L) {
      h->blk_off[L] = (int)blk.size();
      if (L <= G.levels)
        for (int b = 0; b < nb; ++b) {
          bool has = false;
          for (int c = b * kParamBlock; c < std::min(ncell, (b + 1) * kParamBlock) && !has; ++c)
            has = G.lvl[c] == L;
          if (has) blk.push_back(b);
        }
      h->nblk_lv[L] = (int)blk.size() - h->blk_off[L];
    }
    h->blk_lv = (int*)A(sizeof(int) * std::max<size_t>(1, blk.size()));
  }
  h->cnt = (PlCount*)A(sizeof(PlCount));
  h->cells = (ChCellT<double>*)A(sizeof(ChCellT<double>) * ncell);
  h->pend = (float*)A(sizeof(float) * 8 * ncell);
  h->fT = A(h->es * kNF * ncell);
  h->usable_c = (int*)A(sizeof(int) * ncell);
  h->prm = A((env.precision == USP_FP32 ? sizeof(PlParams<float>) : sizeof(PlParams<double>)) *
             ncell);
  h->sums = (ChSumsT<double>*)A(sizeof(ChSumsT<double>) * ncell);
  const size_t acc_bytes = sizeof(double) * ((size_t)ncell * kNAcc + 2 + 4 * kNSurf);
  h->acc = (double*)A(acc_bytes);
  h->macc = (double*)A(sizeof(double) * 21 * ncell);
  h->mout = (double*)A(sizeof(double) * USP_NMOM * ncell);
  h->dstep = (long long*)A(2 * sizeof(long long));   // step, finished blocks
  bool ok = h->keycell && h->bh && h->tot && h->face_off && h->off && h->af && h->afv && h->cnt &&
            (env.sp.method != 1 || h->fpmrec) &&
            (G.levels < 2 || (h->htree.l1_first && h->htree.l2_first && h->htree.l2_ref &&
                               h->htree.lvl && h->htree.lii && h->htree.ljj && h->blk_lv &&
                               h->tree)) &&
            h->cells && h->pend && h->fT && h->usable_c && h->prm && h->sums && h->acc && h->macc && h->mout && h->dstep;
  for (int k = 0; k < 2; ++k) {
    for (int q = 0; q < 6; ++q) ok = ok && h->st[k][q];
    ok = ok && h->lv[k] && h->pd[k] && h->kbuf[k] && h->ibuf[k];
  }
  if (!ok) {
    delete h;
    return USP_ENOMEM;
  }
  cudaStream_t s = env.stream;
  const size_t nh = (size_t)std::max<int64_t>(n, 1);
  std::vector<double> hl(6 * nh, 0.0);
  std::vector<int> key(nh, 0);
  std::vector<uint32_t> hp(nh, 0);
  uint32_t next = 0;
  for (int64_t j = 0; j < n; ++j) {
    hl[j] = x[j]; hl[n + j] = y[j]; hl[2 * n + j] = cx[j]; hl[3 * n + j] = cy[j];
    hl[4 * n + j] = cz[j]; hl[5 * n + j] = erot[j];
    key[j] = pg_leaf(pp, G, x[j], y[j]);
    hp[j] = pid ? pid[j] : (uint32_t)j;
    next = std::max(next, hp[j] + 1u);
  }
  PlCount c0;
  c0.n = n; c0.ntot = n; c0.ninj = 0; c0.pid0 = next; c0.next_pid = next;
  std::vector<ChCellT<double>> hc(ncell);
  std::memset((void*)hc.data(), 0, sizeof(ChCellT<double>) * ncell);
  for (auto& cc : hc) { cc.s = 1.0; cc.r = 1.0; }
  void* tmp = n > 0 ? env.alloc(env.owner, 6 * nh * sizeof(double)) : nullptr;
  if (n > 0 && !tmp) {
    delete h;
    return USP_ENOMEM;
  }
  const long long dstep0 = step0;
  bool cok = true;
  if (n > 0) {
    cok = cok && cudaMemcpyAsync(h->lv[0], lev, n * 4, cudaMemcpyHostToDevice, s) == cudaSuccess;
    cok = cok && cudaMemcpyAsync(h->pd[0], hp.data(), n * 4, cudaMemcpyHostToDevice, s) == cudaSuccess;
    cok = cok && cudaMemcpyAsync(h->keycell, key.data(), n * 4, cudaMemcpyHostToDevice, s) == cudaSuccess;
    cok = cok && cudaMemcpyAsync(tmp, hl.data(), 6 * n * sizeof(double), cudaMemcpyHostToDevice,
                                 s) == cudaSuccess;
    const int nb = (int)((n + 255) / 256);
    if (env.precision == USP_FP32)
      pl_from_host_layout<float><<<nb, 256, 0, s>>>(n, (const double*)tmp, (float*)h->st[0][0],
          (float*)h->st[0][1], (float*)h->st[0][2], (float*)h->st[0][3], (float*)h->st[0][4],
          (float*)h->st[0][5]);
    else
      pl_from_host_layout<double><<<nb, 256, 0, s>>>(n, (const double*)tmp, (double*)h->st[0][0],
          (double*)h->st[0][1], (double*)h->st[0][2], (double*)h->st[0][3], (double*)h->st[0][4],
          (double*)h->st[0][5]);
    cok = cok && cudaGetLastError() == cudaSuccess;
  }
  cok = cok && cudaMemcpyAsync(h->af, area_frac, sizeof(double) * ncell, cudaMemcpyHostToDevice,
                               s) == cudaSuccess;
  std::vector<double> afv;
  if (G.levels >= 2) {
    // the grid tables and the volume factor af / 4^(level-1) of every cell
    afv.resize(ncell);
    for (int c = 0; c < ncell; ++c) {
      const double sc = (double)(1 << (G.lvl[c] - 1));
      afv[c] = area_frac[c] / (sc * sc);
    }
    auto up = [&](const void* dst, const void* src, size_t bytes) {
      return cudaMemcpyAsync(const_cast<void*>(dst), src, bytes, cudaMemcpyHostToDevice, s) ==
             cudaSuccess;
    };
    cok = cok && up(h->afv, afv.data(), sizeof(double) * ncell);
    const PlTree& t = h->htree;
    cok = cok && up(t.l1_first, G.l1_first.data(), sizeof(int) * (n1 + 1));
    cok = cok && up(t.l2_first, G.l2_first.data(), sizeof(int) * 4 * (size_t)n1);
    cok = cok && up(t.l2_ref, G.l2_ref.data(), 4 * (size_t)n1);
    cok = cok && up(t.lvl, G.lvl.data(), sizeof(int) * ncell);
    cok = cok && up(t.lii, G.lii.data(), sizeof(int) * ncell);
    cok = cok && up(t.ljj, G.ljj.data(), sizeof(int) * ncell);
    cok = cok && up(h->tree, &h->htree, sizeof(PlTree));
    if (!blk.empty()) cok = cok && up(h->blk_lv, blk.data(), sizeof(int) * blk.size());
  }
  cok = cok && cudaMemcpyAsync(h->cnt, &c0, sizeof(PlCount), cudaMemcpyHostToDevice, s) == cudaSuccess;
  cok = cok && cudaMemcpyAsync(h->cells, hc.data(), sizeof(ChCellT<double>) * ncell,
                               cudaMemcpyHostToDevice, s) == cudaSuccess;
  cok = cok && cudaMemsetAsync(h->sums, 0, sizeof(ChSumsT<double>) * ncell, s) == cudaSuccess;
  {
    std::vector<float> pe((size_t)ncell * 8, 0.0f);
    for (int c = 0; c < ncell; ++c) pe[(size_t)c * 8 + 6] = pe[(size_t)c * 8 + 7] = 1.0f;
    cok = cok && cudaMemcpyAsync(h->pend, pe.data(), sizeof(float) * 8 * ncell,
                                 cudaMemcpyHostToDevice, s) == cudaSuccess;
    cok = cok && cudaStreamSynchronize(s) == cudaSuccess;
  }
  cok = cok && cudaMemsetAsync(h->acc, 0, acc_bytes, s) == cudaSuccess;
  cok = cok && cudaMemcpyAsync(h->dstep, &dstep0, sizeof(long long), cudaMemcpyHostToDevice, s) == cudaSuccess;
  cok = cok && cudaMemsetAsync(h->dstep + 1, 0, sizeof(long long), s) == cudaSuccess;
  cok = cok && cudaStreamSynchronize(s) == cudaSuccess;
  if (tmp) env.release(env.owner, tmp);
  if (!cok) {
    delete h;
    return USP_ECUDA;
  }
  *out = h;
  return USP_OK;
}

int pl_sample(PlaneCtx* h, int on) {
  h->sampling = on ? 1 : 0;
  return USP_OK;
}

int pl_read(PlaneCtx* h, const ChEnv& env, double* h_acc, int reset) {
  const size_t bytes = sizeof(double) * ((size_t)h->g.ncell * kNAcc + 2 + 4 * kNSurf);
  CHK(cudaMemcpyAsync(h_acc, h->acc, bytes, cudaMemcpyDeviceToHost, env.stream));
  if (reset) CHK(cudaMemsetAsync(h->acc, 0, bytes, env.stream));
  CHK(cudaStreamSynchronize(env.stream));
  return USP_OK;
}

int pl_count(PlaneCtx* h, const ChEnv& env, int64_t* n, uint32_t* next_pid) {
  PlCount c;
  CHK(cudaMemcpyAsync(&c, h->cnt, sizeof(PlCount), cudaMemcpyDeviceToHost, env.stream));
  CHK(cudaStreamSynchronize(env.stream));
  if (n) *n = c.n;
  if (next_pid) *next_pid = c.next_pid;
  return USP_OK;
}

int pl_moments(PlaneCtx* h, const ChEnv& env, double* out, int out_is_device) {
  cudaStream_t s = env.stream;
  const int b = h->cur, ncell = h->g.ncell;
  CHK(cudaMemsetAsync(h->macc, 0, sizeof(double) * 21 * ncell, s));
  for (int pass = 0; pass < 2; ++pass) {
    if (env.precision == USP_FP32)
      pl_mom_pass<float><<<h->grid_p, kBlk, 0, s>>>(pass, h->cnt, h->keycell, h->cells,
          (float*)h->st[b][2], (float*)h->st[b][3], (float*)h->st[b][4], (float*)h->st[b][5],
          h->lv[b], h->macc);
    else
      pl_mom_pass<double><<<h->grid_p, kBlk, 0, s>>>(pass, h->cnt, h->keycell, h->cells,
          (double*)h->st[b][2], (double*)h->st[b][3], (double*)h->st[b][4], (double*)h->st[b][5],
          h->lv[b], h->macc);
    CHK(cudaGetLastError());
  }
  ch_mom_out<<<(ncell + 127) / 128, 128, 0, s>>>(ncell, h->macc, h->mout, env.sp);
  CHK(cudaGetLastError());
  CHK(cudaMemcpyAsync(out, h->mout, sizeof(double) * USP_NMOM * ncell,
                      out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (!out_is_device) CHK(cudaStreamSynchronize(s));
  return USP_OK;
}

int pl_get_particles(PlaneCtx* h, const ChEnv& env, int64_t cap, int64_t* n_out, double* x,
                     double* y, double* cx, double* cy, double* cz, double* erot, int32_t* lev,
                     uint32_t* pid) {
  int64_t n = 0;
  int rc = pl_count(h, env, &n, nullptr);
  if (rc) return rc;
  if (n_out) *n_out = n;
  if (n > cap) return USP_EINVAL;
  if (n == 0) return USP_OK;
  cudaStream_t s = env.stream;
  double* tmp = (double*)env.alloc(env.owner, 6 * n * sizeof(double));
  if (!tmp) return USP_ENOMEM;
  const int b = h->cur;
  const int nb = (int)((n + 255) / 256);
  if (env.precision == USP_FP32)
    pl_to_host_layout<float><<<nb, 256, 0, s>>>(n, h->keycell, h->cells, (float*)h->st[b][0],
        (float*)h->st[b][1], (float*)h->st[b][2], (float*)h->st[b][3], (float*)h->st[b][4],
        (float*)h->st[b][5], tmp);
  else
    pl_to_host_layout<double><<<nb, 256, 0, s>>>(n, h->keycell, h->cells, (double*)h->st[b][0],
        (double*)h->st[b][1], (double*)h->st[b][2], (double*)h->st[b][3], (double*)h->st[b][4],
        (double*)h->st[b][5], tmp);
  std::vector<double> hl(6 * n);
  bool ok = cudaGetLastError() == cudaSuccess;
  ok = ok && cudaMemcpyAsync(hl.data(), tmp, 6 * n * sizeof(double), cudaMemcpyDeviceToHost, s) ==
                 cudaSuccess;
  if (lev) ok = ok && cudaMemcpyAsync(lev, h->lv[b], n * 4, cudaMemcpyDeviceToHost, s) == cudaSuccess;
  if (pid) ok = ok && cudaMemcpyAsync(pid, h->pd[b], n * 4, cudaMemcpyDeviceToHost, s) == cudaSuccess;
  ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
  env.release(env.owner, tmp);
  if (!ok) return USP_ECUDA;
  for (int64_t j = 0; j < n; ++j) {
    if (x) x[j] = hl[j];
    if (y) y[j] = hl[n + j];
    if (cx) cx[j] = hl[2 * n + j];
    if (cy) cy[j] = hl[3 * n + j];
    if (cz) cz[j] = hl[4 * n + j];
    if (erot) erot[j] = hl[5 * n + j];
  }
  return USP_OK;
}

int pl_leaves(const usp_plane* pp, int32_t* level, int32_t* ii, int32_t* jj) {
  if (pg_check(pp)) return USP_EINVAL;
  PlGrid G;
  pg_build(pp, G);
  if (!G.balanced || G.nleaf >= (1 << 24)) return USP_EINVAL;
  for (int c = 0; c < G.nleaf; ++c) {
    if (level) level[c] = G.lvl[c];
    if (ii) ii[c] = G.lii[c];
    if (jj) jj[c] = G.ljj[c];
  }
  return G.nleaf;
}

int pl_ncell(const PlaneCtx* h) { return h->g.ncell; }
int pl_parity(const PlaneCtx* h) { return h->cur; }
void pl_destroy(PlaneCtx* h) { delete h; }
