// usp_homog.cu -- kernels and C ABI of the homogeneous (batched-cell) USP-FPM
// step on sm_103a.
//
// Data layout in HBM
//   particles: SoA arrays cx, cy, cz, erot (T = float or double) and lev
//   (int32).  Each cell's particles are a contiguous segment whose start is
//   padded to a multiple of 4 elements, so every 16-byte vector lies inside
//   one cell and vector loads are aligned.
//   cells: FP64 CellState (moments of the current step, targets, the pending
//   conservation rescale), CollideParams<T> (everything the particle kernel
//   needs, precomputed per cell), CellSums (FP64 post-collision sums).
//
// One step = one particle pass and three per-cell kernels:
//   collide (warp- or block-tiled, chosen by the autotuner)
//                    one pass over the particles (read 1x, write 1x).  It
//                    applies the previous step's pending conservation rescale
//                    on load (c = U + s (c* - U*), eps = r eps*), performs the
//                    particle updates of Eqs. update_ci, update_erot and
//                    update_evib with per-cell coefficients, stores the
//                    post-collision state and accumulates per-cell sums.
//   levelfix_kernel  one warp per cell: the vibrational +-1 correction of
//                    Sec. 4.C (warp-parallel with the sequential semantics).
//   cellupdate_kernel one thread per cell: the rotational and velocity
//                    rescale factors, the moments of the next step (exact
//                    under the affine rescale: U' = U, Pi' = s^2 Pi*,
//                    e_rot' = r e_rot*), and the next step's coefficients
//                    (Sec. 3.A) in FP64.
//   jumptable_kernel (FP32 form) the per-cell inversion tables of the
//                    vibrational jump samplers for the next step.
// The rescale is never written back as a separate pass: it rides along with
// the next collide pass, or with usp_moments / usp_get_particles.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/usp.h"
#include "usp_channel.h"
#include "usp_plane.h"
#include "usp_device.cuh"

using namespace usp;

namespace {

constexpr int kBlock = 256;       // threads of the particle kernels
constexpr int kAlign = 4;         // segment alignment (elements)

struct CellState {
  double U[3], Pi[6];        // bulk velocity and temperature tensor of the step
  double Ttr, Trot, ebar;    // temperatures (T_vib through ebar = <I>)
  double e_rot_tgt, e_vib_tgt;
  double Us[3], s, r;        // pending rescale of the stored state
  double ndens, dt;
  long long off, N;          // padded segment start, particle count
  unsigned int pid0, step;   // id of the first particle, step index
  int active;
  int maxI;                  // bound on the levels entering the step (jump-table rows)
};

// 16-byte aligned and sized: the block-tiled particle pass bulk-copies a
// cell's record into shared memory with its particles
template <typename T>
struct alignas(16) CollideParams {
  T U[3], Us[3];
  T as, ar;                  // alpha * s, alpha * sqrt(r)
  T Lp[6];                   // sqrt(1 - alpha^2) L, L L^T = tau D_tr
  T a_rot, sqrt_a;           // R T_rot^rel (1 - alpha^2) / 2 and its root
  T p_nb, p_b;               // USP-FPM: jump parameters; FPM: lam_up, lam_dn
  unsigned int step, pid0;
  long long off;
  int count, active;
  int method, pad_;          // Species::method of the context
};

struct CellSums {
  double v[10];              // sum d (3), sum d d^T (6), sum eps
  unsigned long long I;      // sum of levels after the collision
  long long net;             // net change of the level sum by the +-1 correction
  int maxI;                  // largest level after the collision
  int pad_;
};

struct Tile {
  int cell, start, count, pad_;
};

// ---------------------------------------------------------------------------
// Jump tables of the FP32 form.  In a homogeneous cell p_NB and p_B are cell
// constants, so the cumulative values the sequential inversion would compute
// for a given r = I + 1 (or n = I) are the same for every particle of the
// cell.  jumptable_kernel computes them once per cell and step with exactly
// the operations of nb_inv / binv; a particle then scans its row.  The result
// is identical, bit for bit, to the sequential search: a stall of the
// cumulative sum and the end of the binomial support become +inf entries, an
// underflowed P(0) marks the row (-1) and sends the particle to the
// sequential search, as does a search running past the row.
// ---------------------------------------------------------------------------
constexpr int kJR = 32;   // rows: NB r = 1..32, B n = 0..31
constexpr int kJK = 48;   // cumulative values per row (rows 16-byte aligned)

// The pmf ratios of the rows, the same for every cell: (k + r) / (k + 1) of
// the NB row r (index r - 1) and (n - k) / (k + 1) of the binomial row n,
// each the correctly rounded float quotient that the sequential inversion
// forms; filled once per context by jratio_kernel.
__device__ float g_jratio[2][kJR][kJK];

__global__ void jratio_kernel() {
  for (int e = threadIdx.x; e < kJR * kJK; e += blockDim.x) {
    const int a = e / kJK, k = e % kJK;
    g_jratio[0][a][k] = rn_div(rn_i2f(k + a + 1, 0.0f), rn_i2f(k + 1, 0.0f));
    g_jratio[1][a][k] = k < a ? rn_div(rn_i2f(a - k, 0.0f), rn_i2f(k + 1, 0.0f)) : 0.0f;
  }
}

__device__ void nb_row(int r, float p, float* T) {
  const float q = rn_sub(1.0f, p);
  float P = powi_rn(p, r);
  if (P < 1.17549435e-38f) { T[0] = -1.0f; return; }
  float cdf = P;
  T[0] = cdf;
  bool stop = false;
  for (int j = 1; j < kJK; ++j) {
    if (!stop) {
      const int k = j - 1;
      const float t = g_jratio[0][r - 1][k];   // (k + r) / (k + 1)
      P = rn_mul(P, t);
      P = rn_mul(P, q);
      const float nc = rn_add(cdf, P);
      if (nc == cdf) stop = true;
      else cdf = nc;
    }
    T[j] = stop ? __int_as_float(0x7f800000) : cdf;
  }
}

// p here is the binomial parameter after the p > 1/2 flip
__device__ void b_row(int n, float p, float* T) {
  const float q = rn_sub(1.0f, p);
  float P = powi_rn(q, n);
  if (P < 1.17549435e-38f) { T[0] = -1.0f; return; }
  const float pq = rn_div(p, q);
  float cdf = P;
  T[0] = cdf;
  bool stop = false;
  for (int j = 1; j < kJK; ++j) {
    if (!stop) {
      if (j >= n) {
        stop = true;   // the search ends at k = n whatever u is
      } else {
        const int k = j - 1;
        const float t = g_jratio[1][n][k];       // (n - k) / (k + 1)
        P = rn_mul(P, t);
        P = rn_mul(P, pq);
        const float nc = rn_add(cdf, P);
        if (nc == cdf) stop = true;
        else cdf = nc;
      }
    }
    T[j] = stop ? __int_as_float(0x7f800000) : cdf;
  }
}

// Guide tables (the indexed search of Chen & Asau): per row, one byte for
// each of the 256 bins of the uniform's top eight bits.  A float uniform
// (2 (x >> 9) + 1) 2^-24 lies in bin m = x >> 24, between
// umin(m) = (2 (m << 15) + 1) 2^-24 and umax(m) = (2 ((m << 15) + 32767) + 1) 2^-24.
// With k = the number of row entries <= umin(m): when no entry lies in
// (umin(m), umax(m)], every uniform of the bin gives k, and the byte holds
// bit 7 and the sampler's outcome for that k (k; n - k for a binomial row
// taken at 1 - p_B, p_B > 1/2); otherwise it holds k, from which the search
// continues.  An outcome k = kJK (past the row) or a row whose P(0)
// underflowed (0xff bytes) sends the particle to the sequential search.  The
// rows a cell's parameters make trivial hold their outcome in every byte:
// 0 for an NB row at p_NB >= 1 and for the binomial rows n = 0 and p_B <= 0,
// n at p_B = 1, and 0x7f (the general path, which flags the clamp) at
// p_B > 1.  The outcome is the row search's, so still the sequential
// inversion's, bit for bit.
constexpr int kGBits = 8;             // guide bins per row: 2^kGBits
constexpr int kGB = 1 << kGBits;      // guide bytes per row
constexpr int kGS = 23 - kGBits;      // 23-bit uniform index -> bin: >> kGS

// the guide byte of the word x's bin in the guide g of a row
__device__ __forceinline__ unsigned guide_byte(const uint8_t* __restrict__ g, uint32_t x) {
  return __ldg(g + (x >> (32 - kGBits)));
}
// the outcome an exact guide byte holds (>= kJK: none)
__device__ __forceinline__ unsigned guide_outcome(unsigned gv) { return gv - 0x80u; }

// number of leading row entries <= u for a guide byte without an outcome
// below kJK (an exact byte here sends the particle to the sequential search)
__device__ __forceinline__ int guided_search(const float* __restrict__ T, unsigned gv, float u) {
  int k = (int)(gv & 0x7fu);
  if (!(gv & 0x80u)) {
#pragma unroll 1
    while (k < kJK && T[k] <= u) ++k;
  }
  return k;
}

// The general path of the two samplers (the guide byte of u's bin gv)
__device__ __forceinline__ int nb_tab(const float* __restrict__ T, unsigned gv, int r, float p,
                                      float u, uint32_t& fl) {
  if (r <= 0 || !(p < 1.0f)) return 0;
  if (r > kJR) return nb_inv(r, p, u, fl);
  if (guide_outcome(gv) < (unsigned)kJK) return (int)guide_outcome(gv);
  const int k = guided_search(T, gv, u);
  return k < kJK ? k : nb_inv(r, p, u, fl);
}

// npb counts the draws clamped at p_B > 1
__device__ __forceinline__ int b_tab(const float* __restrict__ T, unsigned gv, int n, float p,
                                     float u, uint32_t& fl, int& npb) {
  if (n <= 0) return 0;
  if (p >= 1.0f) {
    if (p > 1.0f) {
      fl |= F_PB_CLAMP;
      ++npb;
    }
    return n;
  }
  if (!(p > 0.0f)) return 0;
  const bool flip = p > 0.5f;
  if (n < kJR) {
    if (guide_outcome(gv) < (unsigned)kJK) return (int)guide_outcome(gv);
    const int k = guided_search(T, gv, u);   // T[n] = +inf: k <= n < kJK
    if (k < kJK) return flip ? n - k : k;
  }
  const int k = binv(n, flip ? rn_sub(1.0f, p) : p, u, fl);
  return flip ? n - k : k;
}

// the per-cell jump tables and their guides (FP32 form)
struct JumpTabs {
  const float* nb;
  const float* b;
  const uint8_t* gnb;
  const uint8_t* gb;
};

// ---------------------------------------------------------------------------
// One particle: pending rescale, velocity, rotation, vibration.  Flags go
// into fl, draws clamped at p_B > 1 are counted in npb.
// ---------------------------------------------------------------------------
template <typename T, int METHOD>
__device__ __forceinline__ void collide_one(const CollideParams<T>& P, uint32_t pid,
                                            const PhiloxRoundKeys& rk, T& cx, T& cy, T& cz, T& er,
                                            int& lv,
                                            T* acc, int& accI, int& maxI, uint32_t& fl, int& npb,
                                            const JumpTabs& jt) {
  // levels are non-negative; a negative one (invalid input) is taken as 0,
  // which also keeps the particle's table row in range
  const int I = max(lv, 0);
  T g0, g1, g2, g3;
  uint32_t j5, j6;
  particle_draws(pid, P.step, rk, g0, g1, g2, g3, j5, j6);
  // FP32 form: the guide bytes of the particle's two rows (NB r = I + 1 is
  // row I, binomial n = I is row I) are loaded here, so that their latency
  // passes under the arithmetic below
  size_t row = 0;
  unsigned gv5 = 0, gv6 = 0;
  if constexpr (sizeof(T) == 4 && METHOD == 0) {
    row = (size_t)(I < kJR ? I : 0);
    gv5 = guide_byte(jt.gnb + row * kGB, j5);
    gv6 = guide_byte(jt.gb + row * kGB, j6);
  }
  // c^n - U = s (c* - U*);  C' = alpha C^n + sqrt(1 - alpha^2) L G
  const T d0 = cx - P.Us[0], d1 = cy - P.Us[1], d2 = cz - P.Us[2];
  const T r0 = P.as * d0 + P.Lp[0] * g0;
  const T r1 = P.as * d1 + (P.Lp[1] * g0 + P.Lp[2] * g1);
  const T r2 = P.as * d2 + (P.Lp[3] * g0 + P.Lp[4] * g1 + P.Lp[5] * g2);
  cx = P.U[0] + r0;
  cy = P.U[1] + r1;
  cz = P.U[2] + r2;
  // eps' = a + (sqrt(eps^n) alpha + sqrt(a) G)^2, eps^n = r eps*
  const T root = sqrt_fast(er) * P.ar + P.sqrt_a * g3;
  er = P.a_rot + root * root;
  // I' = I + NB(I + 1, p_NB) - B(I, p_B)
  const T u5 = jump_uniform<T>(j5), u6 = jump_uniform<T>(j6);
  if constexpr (METHOD == 1) {
    // plain FPM method: Gillespie's direct method (Sec. 2.C)
    uint32_t f1 = 0;
    lv = gillespie<T>(I, P.p_nb, P.p_b, pid, P.step, rk, f1);
    npb += (f1 & F_PB_CLAMP) ? 1 : 0;
    fl |= f1;
  } else {
    int up, dn;
    if constexpr (sizeof(T) == 4) {
      // both guide bytes hold their outcome (every cell case included):
      // one test decides the jump
      const unsigned o5 = guide_outcome(gv5), o6 = guide_outcome(gv6);
      if ((I < kJR) & (o5 < (unsigned)kJK) & (o6 < (unsigned)kJK)) {
        up = (int)o5;
        dn = (int)o6;
      } else {
        up = nb_tab(jt.nb + row * kJK, gv5, I + 1, P.p_nb, u5, fl);
        dn = b_tab(jt.b + row * kJK, gv6, I, P.p_b, u6, fl, npb);
      }
    } else {
      uint32_t f1 = 0;
      up = sample_nb<T>(I + 1, P.p_nb, u5, f1);
      dn = sample_b<T>(I, P.p_b, u6, f1);
      npb += (f1 & F_PB_CLAMP) ? 1 : 0;
      fl |= f1;
    }
    lv = I + up - dn;
  }
  maxI = max(maxI, lv);
  acc[0] += r0; acc[1] += r1; acc[2] += r2;
  acc[3] += r0 * r0; acc[4] += r1 * r1; acc[5] += r2 * r2;
  acc[6] += r0 * r1; acc[7] += r0 * r2; acc[8] += r1 * r2;
  acc[9] += er;
  accI += lv;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block reduction of the tile sums and one FP64 atomic per sum.  Partial sums
// stay in T inside a thread and a warp; warps combine in FP64.
template <typename T>
__device__ __forceinline__ void flush_sums(const T* acc, int accI, int maxI, CellSums* dst) {
  __shared__ double red[kBlock / 32][11];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const T s = warp_sum(acc[i]);
    if (lane == 0) red[wid][i] = (double)s;
  }
  const int sI = warp_sum(accI);
  if (lane == 0) red[wid][10] = (double)sI;
  const int mI = __reduce_max_sync(0xffffffffu, maxI);
  if (lane == 0 && mI > 0) atomicMax(&dst->maxI, mI);
  __syncthreads();
  if (threadIdx.x < 11) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w) t += red[w][threadIdx.x];
    if (threadIdx.x < 10)
      atomicAdd(&dst->v[threadIdx.x], t);
    else
      atomicAdd(&dst->I, (unsigned long long)(long long)t);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Bulk-copy (TMA) staging helpers: shared-memory mbarrier, cp.async.bulk
// global<->shared copies, proxy fences.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
      ::"r"(smem_u32(bar)), "r"(bytes)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared, completion counted on the mbarrier (bytes % 16 == 0,
// both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// shared -> global in the current bulk group
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
               ::"l"(dst), "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait on an mbarrier phase: gives up after `limit` SM cycles and
// reports false.  The waits of the particle pass take the context's limit
// (usp_set_wait_limit; by default kWaitCycles, about a second); the waits of
// a block that is leaving after a timeout, for its own copies still in
// flight, always take kWaitCycles.
constexpr long long kWaitCycles = 2000000000ll;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// Check of the timeout path: one block waits, with the bounded wait of the
// particle pass, on an mbarrier phase that nothing completes (no thread
// arrives on it, no copy is aimed at it), records USP_F_WAIT_TIMEOUT when
// the limit runs out and returns.
__global__ void wait_check_kernel(long long limit, uint32_t* flags) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0u, limit);
  if (!ok && threadIdx.x == 0) atomicOr(flags, (uint32_t)F_WAIT_TIMEOUT);
}

constexpr int kTileMax = 1536;   // particles per staged tile
constexpr int kBS = 2;           // staging buffers of the block-tiled pass

// One staging buffer: x, y, z, eps (kTileMax T each) then levels (kTileMax int).
template <typename T>
constexpr size_t stage_bytes() {
  return (size_t)kTileMax * (4 * sizeof(T) + sizeof(int));
}
template <typename T>
__device__ __forceinline__ T* sb_x(unsigned char* b) { return reinterpret_cast<T*>(b); }
template <typename T>
__device__ __forceinline__ int* sb_l(unsigned char* b) {
  return reinterpret_cast<int*>(b + 4 * kTileMax * sizeof(T));
}

// bytes of one staged copy of `count` particles (rounded up to the 4-element
// segment padding, so every copy is a multiple of 16 bytes)
__device__ __forceinline__ int round4(int n) { return (n + 3) & ~3; }

// ---------------------------------------------------------------------------
// Warp-tiled particle pass.  Every warp runs its own pipeline over a
// contiguous range of small tiles (<= kWT particles of one cell): kWS staging
// buffers, bulk loads issued by lane 0 up to two tiles ahead, bulk stores of
// the updated tile, cell sums reduced across the warp when its cell changes.
// There is no block-wide barrier, so a warp never waits for the slowest
// thread of its block.
// ---------------------------------------------------------------------------
constexpr int kWT = 128;            // particles per warp tile
constexpr int kWS = 3;              // staging buffers per warp
constexpr int kWarps = kBlock / 32;

template <typename T>
constexpr size_t wstage_bytes() {
  return (size_t)kWT * (4 * sizeof(T) + sizeof(int));
}
template <typename T>
constexpr size_t wsmem_bytes() {
  return (size_t)kWarps * kWS * wstage_bytes<T>();
}

// all but the most recent bulk group have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}

template <typename T>
__device__ __forceinline__ void wstage_load(const Tile& tl, long long off, unsigned char* b,
                                            uint64_t* bar, const T* cx, const T* cy, const T* cz,
                                            const T* er, const int* lev) {
  const int n4 = round4(tl.count);
  const long long base = off + tl.start;
  const uint32_t bt = (uint32_t)(n4 * sizeof(T)), bl = (uint32_t)(n4 * sizeof(int));
  T* X = reinterpret_cast<T*>(b);
  mbar_expect_tx(bar, 4 * bt + bl);
  if (n4 > 0) {
    bulk_g2s(X, cx + base, bt, bar);
    bulk_g2s(X + kWT, cy + base, bt, bar);
    bulk_g2s(X + 2 * kWT, cz + base, bt, bar);
    bulk_g2s(X + 3 * kWT, er + base, bt, bar);
    bulk_g2s(reinterpret_cast<int*>(b + 4 * kWT * sizeof(T)), lev + base, bl, bar);
  }
}

// Warp reduction of the cell sums and one FP64 atomic per sum.
template <typename T>
__device__ __forceinline__ void flush_sums_warp(const T* acc, int accI, int maxI,
                                                CellSums* dst) {
  const int lane = threadIdx.x & 31;
  double mine = 0.0;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const T s = warp_sum(acc[i]);
    if (lane == i) mine = (double)s;
  }
  const int sI = warp_sum(accI);
  const int mI = __reduce_max_sync(0xffffffffu, maxI);
  if (lane < 10) atomicAdd(&dst->v[lane], mine);
  if (lane == 10) atomicAdd(&dst->I, (unsigned long long)(long long)sI);
  if (lane == 11 && mI > 0) atomicMax(&dst->maxI, mI);
}

template <typename T, int MINB, int METHOD>
__global__ void __launch_bounds__(kBlock, MINB)
collide_warp_kernel(const Tile* __restrict__ tiles, int ntiles,
                    const CollideParams<T>* __restrict__ prm, T* __restrict__ cx,
                    T* __restrict__ cy, T* __restrict__ cz, T* __restrict__ er,
                    int* __restrict__ lev, CellSums* __restrict__ sums, uint32_t* flags,
                    unsigned long long* counters, const PhiloxRoundKeys rk,
                    const JumpTabs tabs, long long wait_cycles) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_all[kWarps][kWS];
  __shared__ __align__(16) CollideParams<T> Pw[kWarps];   // the warp's current cell
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long W = (long long)gridDim.x * kWarps;
  const long long gw = (long long)blockIdx.x * kWarps + wid;
  const int t_begin = (int)(((long long)ntiles * gw) / W);
  const int t_end = (int)(((long long)ntiles * (gw + 1)) / W);
  if (t_begin >= t_end) return;
  unsigned char* wbuf = smem + (size_t)wid * kWS * wstage_bytes<T>();
  uint64_t* bar = bar_all[wid];
  CollideParams<T>& P = Pw[wid];
  if (lane == 0) {
#pragma unroll
    for (int s = 0; s < kWS; ++s) mbar_init(&bar[s], 1);
    mbar_init_fence();
  }
  __syncwarp();
  uint32_t inflight = 0;   // lane 0: buffers with a load in flight
  if (lane == 0) {
    for (int s = 0; s < kWS - 1 && t_begin + s < t_end; ++s) {
      const Tile tl = tiles[t_begin + s];
      wstage_load<T>(tl, prm[tl.cell].off, wbuf + s * wstage_bytes<T>(), &bar[s], cx, cy, cz, er,
                     lev);
      inflight |= 1u << s;
    }
  }
  uint32_t phase = 0;      // bit s: parity of buffer s's next completion
  T acc[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) acc[i] = T(0);
  int accI = 0, maxI = 0;
  uint32_t fl = 0;
  int npb = 0;
  int cell = -1;
  int s = 0;
  for (int t = t_begin; t < t_end; ++t) {
    const Tile tl = tiles[t];
    if (tl.cell != cell) {
      constexpr int nw = (int)(sizeof(CollideParams<T>) / 4);
      __syncwarp();
      for (int i = lane; i < nw; i += 32)
        reinterpret_cast<uint32_t*>(&P)[i] = reinterpret_cast<const uint32_t*>(&prm[tl.cell])[i];
      __syncwarp();
      cell = tl.cell;
    }
    const bool ok = mbar_wait_bounded(&bar[s], (phase >> s) & 1u, wait_cycles);
    if (__any_sync(0xffffffffu, !ok)) {
      if (lane == 0) atomicOr(flags, (uint32_t)F_WAIT_TIMEOUT);
      break;
    }
    phase ^= 1u << s;
    if (lane == 0) inflight &= ~(1u << s);
    unsigned char* b = wbuf + s * wstage_bytes<T>();
    if (P.active) {
      T* X = reinterpret_cast<T*>(b);
      int* Lv = reinterpret_cast<int*>(b + 4 * kWT * sizeof(T));
      const uint32_t pid0 = P.pid0 + (uint32_t)tl.start;
      const size_t tc = (size_t)tl.cell * kJR;
      const JumpTabs jt{tabs.nb + tc * kJK, tabs.b + tc * kJK, tabs.gnb + tc * kGB,
                        tabs.gb + tc * kGB};
#pragma unroll 1
      for (int k = lane; k < tl.count; k += 32) {
        T x = X[k], y = X[k + kWT], z = X[k + 2 * kWT], e = X[k + 3 * kWT];
        int l = Lv[k];
        collide_one<T, METHOD>(P, pid0 + (uint32_t)k, rk, x, y, z, e, l, acc, accI, maxI, fl, npb,
                               jt);
        X[k] = x; X[k + kWT] = y; X[k + 2 * kWT] = z; X[k + 3 * kWT] = e;
        Lv[k] = l;
      }
      // results in shared memory -> visible to the bulk-copy engine
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        const int n4 = round4(tl.count);
        const long long base = P.off + tl.start;
        const uint32_t bt = (uint32_t)(n4 * sizeof(T)), bl = (uint32_t)(n4 * sizeof(int));
        if (n4 > 0) {
          bulk_s2g(cx + base, X, bt);
          bulk_s2g(cy + base, X + kWT, bt);
          bulk_s2g(cz + base, X + 2 * kWT, bt);
          bulk_s2g(er + base, X + 3 * kWT, bt);
          bulk_s2g(lev + base, Lv, bl);
        }
      }
      if (t + 1 >= t_end || tiles[t + 1].cell != tl.cell) {
        flush_sums_warp<T>(acc, accI, maxI, &sums[tl.cell]);
#pragma unroll
        for (int i = 0; i < 10; ++i) acc[i] = T(0);
        accI = 0;
        maxI = 0;
      }
    }
    if (lane == 0) {
      // one bulk group per tile (empty for an inactive cell), so that the
      // group before the newest is always the previous tile's store
      bulk_commit();
      const int tn = t + kWS - 1;
      if (tn < t_end) {
        // the buffer of tile t - 1 takes tile t + kWS - 1 once its store has
        // read it
        const int sn = s == 0 ? kWS - 1 : s - 1;
        bulk_wait_read_1();
        const Tile tn_l = tiles[tn];
        wstage_load<T>(tn_l, prm[tn_l.cell].off, wbuf + sn * wstage_bytes<T>(), &bar[sn], cx, cy,
                       cz, er, lev);
        inflight |= 1u << sn;
      }
    }
    s = s == kWS - 1 ? 0 : s + 1;
  }
  fl = __reduce_or_sync(0xffffffffu, fl);
  npb = __reduce_add_sync(0xffffffffu, npb);
  if (lane == 0) {
    if (fl) {
      atomicOr(flags, fl);
      if (npb) atomicAdd(&counters[C_PB_CLAMP], (unsigned long long)npb);
    }
    // loads still in flight after a timeout: wait for them (bounded) before
    // the block's shared memory is released
    for (int q = 0; q < kWS; ++q)
      if (inflight & (1u << q)) (void)mbar_wait_bounded(&bar[q], (phase >> q) & 1u, kWaitCycles);
    bulk_wait_all();
  }
}

// ---------------------------------------------------------------------------
// Block-tiled particle pass.  Each persistent block owns a contiguous range
// of the tile list (tiles of one cell are adjacent, so a block meets few cell
// boundaries); each tile (<= kTileMax particles of one cell) and its cell's
// CollideParams are brought into shared memory by bulk copies while the
// previous tile is being processed (kBS buffers), updated in place, and
// written back by bulk copies.  The block's warps share each tile but never
// wait for one another: a warp that finishes its part of a tile counts itself
// done; the last one issues the tile's bulk store and, once the store has
// read the buffer, releases it to the producer (thread 0), which refills it
// with the tile after next.  Cell sums are reduced per warp when the cell
// changes.
// ---------------------------------------------------------------------------
template <typename T>
constexpr size_t bstage_bytes() {
  return stage_bytes<T>() + sizeof(CollideParams<T>);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}

// the five state loads of a tile and its cell's record (one thread)
template <typename T>
__device__ __forceinline__ void stage_load_p(const Tile& tl, const CollideParams<T>* prm,
                                             unsigned char* b, uint64_t* bar, const T* cx,
                                             const T* cy, const T* cz, const T* er,
                                             const int* lev) {
  const CollideParams<T>* pc = prm + tl.cell;
  const int n4 = round4(tl.count);
  const long long base = pc->off + tl.start;
  const uint32_t bt = (uint32_t)(n4 * sizeof(T)), bl = (uint32_t)(n4 * sizeof(int));
  T* X = sb_x<T>(b);
  mbar_expect_tx(bar, 4 * bt + bl + (uint32_t)sizeof(CollideParams<T>));
  bulk_g2s(b + stage_bytes<T>(), pc, (uint32_t)sizeof(CollideParams<T>), bar);
  if (n4 > 0) {
    bulk_g2s(X, cx + base, bt, bar);
    bulk_g2s(X + kTileMax, cy + base, bt, bar);
    bulk_g2s(X + 2 * kTileMax, cz + base, bt, bar);
    bulk_g2s(X + 3 * kTileMax, er + base, bt, bar);
    bulk_g2s(sb_l<T>(b), lev + base, bl, bar);
  }
}

template <typename T, int MINB, int METHOD>
__global__ void __launch_bounds__(kBlock, MINB)
collide_kernel(const Tile* __restrict__ tiles, int ntiles,
               const CollideParams<T>* __restrict__ prm, T* __restrict__ cx,
               T* __restrict__ cy, T* __restrict__ cz, T* __restrict__ er,
               int* __restrict__ lev, CellSums* __restrict__ sums, uint32_t* flags,
               unsigned long long* counters, const PhiloxRoundKeys rk,
               const JumpTabs tabs, long long wait_cycles) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kBS], empty[kBS];
  __shared__ int done[kBS];
  const int tid = threadIdx.x, lane = tid & 31;
  const int G = gridDim.x;
  const int t_begin = (int)(((long long)ntiles * blockIdx.x) / G);
  const int t_end = (int)(((long long)ntiles * (blockIdx.x + 1)) / G);
  if (t_begin >= t_end) return;
  if (tid == 0) {
    for (int q = 0; q < kBS; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
      done[q] = 0;
    }
    mbar_init_fence();
  }
  __syncthreads();
  uint32_t inflight = 0;   // thread 0: buffers with a load in flight
  if (tid == 0) {
    // the first kBS - 1 tiles
    for (int q = 0; q < kBS - 1 && t_begin + q < t_end; ++q) {
      stage_load_p<T>(tiles[t_begin + q], prm, smem + q * bstage_bytes<T>(), &full[q], cx, cy, cz,
                      er, lev);
      inflight |= 1u << q;
    }
  }
  uint32_t fph = 0, eph = 0;   // parities of the next full / empty completion per buffer
  T acc[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) acc[i] = T(0);
  int accI = 0, maxI = 0;
  uint32_t fl = 0;
  int npb = 0;
  int it = 0;
  int b = 0;   // buffer of tile t: it % kBS
  for (int t = t_begin; t < t_end; ++t, ++it, b = b == kBS - 1 ? 0 : b + 1) {
    unsigned char* buf = smem + b * bstage_bytes<T>();
    const int bn = b == 0 ? kBS - 1 : b - 1;   // the buffer of tile t - 1
    if (tid == 0 && t + kBS - 1 < t_end) {
      // tile t - 1's buffer takes tile t + kBS - 1 once every warp is done
      // with tile t - 1 there and its store has read it
      bool ok = true;
      if (it >= 1) {
        ok = mbar_wait_bounded(&empty[bn], (eph >> bn) & 1u, wait_cycles);
        eph ^= 1u << bn;
      }
      if (ok) {
        stage_load_p<T>(tiles[t + kBS - 1], prm, smem + bn * bstage_bytes<T>(), &full[bn], cx, cy,
                        cz, er, lev);
        inflight |= 1u << bn;
      } else {
        atomicOr(flags, (uint32_t)F_WAIT_TIMEOUT);
      }
    }
    const Tile tl = tiles[t];
    const bool ok = mbar_wait_bounded(&full[b], (fph >> b) & 1u, wait_cycles);
    if (__any_sync(0xffffffffu, !ok)) {
      if (lane == 0) atomicOr(flags, (uint32_t)F_WAIT_TIMEOUT);
      break;
    }
    fph ^= 1u << b;
    if (tid == 0) inflight &= ~(1u << b);
    const CollideParams<T>& P = *reinterpret_cast<const CollideParams<T>*>(buf + stage_bytes<T>());
    const bool active = P.active != 0;
    if (active) {
      T* X = sb_x<T>(buf);
      int* Lv = sb_l<T>(buf);
      const uint32_t pid0 = P.pid0 + (uint32_t)tl.start;
      const size_t tc = (size_t)tl.cell * kJR;
      const JumpTabs jt{tabs.nb + tc * kJK, tabs.b + tc * kJK, tabs.gnb + tc * kGB,
                        tabs.gb + tc * kGB};
#pragma unroll 1
      for (int k = tid; k < tl.count; k += kBlock) {
        T x = X[k], y = X[k + kTileMax], z = X[k + 2 * kTileMax], e = X[k + 3 * kTileMax];
        int l = Lv[k];
        collide_one<T, METHOD>(P, pid0 + (uint32_t)k, rk, x, y, z, e, l, acc, accI, maxI, fl, npb,
                               jt);
        X[k] = x; X[k + kTileMax] = y; X[k + 2 * kTileMax] = z; X[k + 3 * kTileMax] = e;
        Lv[k] = l;
      }
    }
    // this warp's results -> visible to the bulk-copy engine; count it done
    fence_async_smem();
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      if (atomicAdd(&done[b], 1) == kBlock / 32 - 1) {
        // last warp of the tile: store it, wait until the store has read the
        // buffer, release the buffer
        __threadfence_block();
        done[b] = 0;
        const int n4 = round4(tl.count);
        if (active && n4 > 0) {
          const long long base = P.off + tl.start;
          const uint32_t bt = (uint32_t)(n4 * sizeof(T)), bl = (uint32_t)(n4 * sizeof(int));
          T* X = sb_x<T>(buf);
          bulk_s2g(cx + base, X, bt);
          bulk_s2g(cy + base, X + kTileMax, bt);
          bulk_s2g(cz + base, X + 2 * kTileMax, bt);
          bulk_s2g(er + base, X + 3 * kTileMax, bt);
          bulk_s2g(lev + base, sb_l<T>(buf), bl);
        }
        bulk_commit();
        bulk_wait_read_all();
        mbar_arrive(&empty[b]);
      }
    }
    // sums of a cell are flushed once its last tile in this range is done
    if (t + 1 >= t_end || tiles[t + 1].cell != tl.cell) {
      if (active) flush_sums_warp<T>(acc, accI, maxI, &sums[tl.cell]);
#pragma unroll
      for (int i = 0; i < 10; ++i) acc[i] = T(0);
      accI = 0;
      maxI = 0;
    }
  }
  fl = __reduce_or_sync(0xffffffffu, fl);
  npb = __reduce_add_sync(0xffffffffu, npb);
  if (lane == 0) {
    if (fl) {
      atomicOr(flags, fl);
      if (npb) atomicAdd(&counters[C_PB_CLAMP], (unsigned long long)npb);
    }
    bulk_wait_all();
  }
  if (tid == 0) {
    // loads still in flight after a timeout: wait for them (bounded) before
    // the block's shared memory is released
    for (int q = 0; q < kBS; ++q)
      if (inflight & (1u << q)) (void)mbar_wait_bounded(&full[q], (fph >> q) & 1u, kWaitCycles);
  }
}


// Jump-table rows of every cell for the coming step (FP32 form), one block of
// kJT threads per cell: thread j < kJR builds the NB row r = j + 1, thread
// kJR + n the binomial row n, for the rows the cell's levels can reach; then
// every row's guide is built by kGP threads.
constexpr int kJT = 8 * kJR;

__device__ __forceinline__ bool nb_row_used(int j, int rows, float p_nb) {
  return j + 1 <= rows && p_nb < 1.0f;
}
__device__ __forceinline__ bool b_row_used(int n, int rows, float p_b) {
  return n >= 1 && n <= rows - 1 && p_b < 1.0f && p_b > 0.0f;
}

// bins [q kQ, (q + 1) kQ) of the guide of row T (the guide tables above),
// kQ = kGB / kGP; nflip = n for a binomial row taken at 1 - p_B (exact bytes
// hold n - k), else -1.  The bounds of bin m are exact floats formed by one
// fused multiply-add each: umin(m) = m 2^-kGBits + 2^-24 and
// umax(m) = (m + 1) 2^-kGBits - 2^-24.  Four bins that no row entry reaches
// (the next entry above umin lies above the fourth bin's umax) are exact at
// the same count and written as one word.
constexpr int kGP = 4;   // threads per guide row
constexpr int kGQ = kGB / kGP;   // bins per guide part
__host__ __device__ inline void guide_fill(uint8_t* __restrict__ g, int q, uint32_t byte) {
  uint32_t* g4 = reinterpret_cast<uint32_t*>(g);
  const uint32_t word = byte * 0x01010101u;
  for (int w = q * kGQ / 4; w < (q + 1) * kGQ / 4; ++w) g4[w] = word;
}
__host__ __device__ inline float guide_umin(int m) {
  return fmaf((float)m, 1.0f / (float)kGB, 5.9604644775390625e-8f);
}
__host__ __device__ inline float guide_umax(int m) {
  return fmaf((float)(m + 1), 1.0f / (float)kGB, -5.9604644775390625e-8f);
}
__host__ __device__ inline void guide_part(const float* T, uint8_t* __restrict__ g, int q,
                                           int nflip) {
  uint32_t* g4 = reinterpret_cast<uint32_t*>(g);
  if (T[0] < 0.0f) {
    guide_fill(g, q, 0xffu);
    return;
  }
  const float inf = INFINITY;
  int k = 0;
  const float u0 = guide_umin(q * kGQ);
  while (k < kJK && T[k] <= u0) ++k;
  float tk = k < kJK ? T[k] : inf;   // the first entry above the current umin
  for (int w = q * kGQ / 4; w < (q + 1) * kGQ / 4; ++w) {
    uint32_t word;
    if (tk > guide_umax(4 * w + 3)) {
      const int o = k < kJK && nflip >= 0 ? nflip - k : k;
      word = (uint32_t)(o | 0x80) * 0x01010101u;
    } else {
      word = 0;
      for (int b = 0; b < 4; ++b) {
        const int m = 4 * w + b;
        const float umin = guide_umin(m), umax = guide_umax(m);
        while (k < kJK && T[k] <= umin) ++k;
        const bool exact = k >= kJK || T[k] > umax;
        const int o = exact && k < kJK && nflip >= 0 ? nflip - k : k;
        word |= (uint32_t)(o | (exact ? 0x80 : 0)) << (8 * b);
      }
      tk = k < kJK ? T[k] : inf;
    }
    g4[w] = word;
  }
}

__global__ void __launch_bounds__(kJT)
jumptable_kernel(int c0, int c1, const CollideParams<float>* __restrict__ prm,
                 const CellState* __restrict__ cells, float* __restrict__ tab_nb,
                 float* __restrict__ tab_b, uint8_t* __restrict__ gd_nb,
                 uint8_t* __restrict__ gd_b) {
  const int c = c0 + blockIdx.x;
  const int j = threadIdx.x;
  if (c >= c1) return;                       // uniform over the block
  const CollideParams<float>& P = prm[c];
  if (!P.active) return;                     // uniform over the block
  // the rows are built in shared memory, copied out coalesced, and the
  // guides read them there
  __shared__ float rs[2][kJR][kJK];
  const int rows = min(kJR, cells[c].maxI + 1);
  float pb = P.p_b;
  if (pb > 0.5f && pb < 1.0f) pb = rn_sub(1.0f, pb);
  if (j < kJR) {
    if (nb_row_used(j, rows, P.p_nb)) nb_row(j + 1, P.p_nb, rs[0][j]);
  } else if (j < 2 * kJR) {
    const int n = j - kJR;
    if (b_row_used(n, rows, P.p_b)) b_row(n, pb, rs[1][n]);
  }
  __syncthreads();
  for (int e = j; e < 2 * kJR * kJK; e += kJT) {
    const int t = e / (kJR * kJK), row = (e / kJK) % kJR, k = e % kJK;
    if (t == 0 ? nb_row_used(row, rows, P.p_nb) : b_row_used(row, rows, P.p_b))
      (t == 0 ? tab_nb : tab_b)[((size_t)c * kJR + row) * kJK + k] = rs[t][row][k];
  }
  static_assert(2 * kJR * kGP == kJT, "one guide part per thread");
  const int row = j / kGP, q = j % kGP;      // 2 kJR rows, kGP parts each
  if (row < kJR) {
    uint8_t* g = gd_nb + ((size_t)c * kJR + row) * kGB;
    if (nb_row_used(row, rows, P.p_nb))
      guide_part(rs[0][row], g, q, -1);
    else if (row < rows)
      guide_fill(g, q, 0x80u);              // p_NB >= 1: no jump up
  } else {
    const int n = row - kJR;
    uint8_t* g = gd_b + ((size_t)c * kJR + n) * kGB;
    const float p = P.p_b;
    if (b_row_used(n, rows, p))
      guide_part(rs[1][n], g, q, p > 0.5f ? n : -1);
    else if (n < rows)
      // n = 0 or p_B <= 0: no jump down; p_B = 1: n; p_B > 1: the general
      // path, which flags the clamp
      guide_fill(g, q, n >= 1 && p >= 1.0f ? (p > 1.0f ? 0x7fu : 0x80u | (uint32_t)n) : 0x80u);
  }
}

// ---------------------------------------------------------------------------
// Per-cell coefficient block: from the step's moments to CollideParams.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void write_params(const Species& sp, CellState& cs, CollideParams<T>& P, uint32_t* flags,
                             unsigned long long* counters) {
  const double R = gasR(sp);
  P.step = cs.step;
  P.pid0 = cs.pid0;
  P.off = cs.off;
  P.count = (int)cs.N;
  P.active = cs.active;
  for (int i = 0; i < 3; ++i) { P.U[i] = (T)cs.U[i]; P.Us[i] = (T)cs.Us[i]; }
  P.method = sp.method;
  P.pad_ = 0;
  if (!cs.active) return;
  const double Tvib = T_vib_of_level(sp, cs.ebar);
  if (sp.method == 1) {
    // the plain FPM method (Sec. 2.C): Gorji's velocity update and the
    // Milstein square form with alpha = exp(-dt/tau), Gillespie levels
    const FpmCell f = fpm_cell(sp, cs.ndens, cs.dt, cs.Pi, cs.Ttr, cs.Trot, Tvib);
    if (!f.ok) {
      atomicOr(flags, (uint32_t)F_A_NONPOS);
      cs.active = 0;
      P.active = 0;
      return;
    }
    cs.e_rot_tgt = f.e_rot_tgt;
    cs.e_vib_tgt = f.e_vib_tgt;
    if (f.fixed) atomicAdd(&counters[C_CHOL_FIX], 1ull);
    if (f.nu_zero) atomicAdd(&counters[C_NU_ZERO], 1ull);
    if (f.failed) atomicOr(flags, (uint32_t)F_CHOL_FAIL_AFTER_FIX);
    if (f.clamped) {
      atomicOr(flags, (uint32_t)F_TREL_CLAMP);
      atomicAdd(&counters[C_TREL_CLAMP], 1ull);
    }
    const double a = f.alpha, oma2 = 1.0 - a * a, sq = sqrt(oma2);
    P.as = (T)(a * cs.s);
    P.ar = (T)(a * sqrt(cs.r));
    for (int i = 0; i < 6; ++i) P.Lp[i] = (T)(sq * f.L[i]);
    const double arot = R * f.Trot_rel * oma2 / 2.0;
    P.a_rot = (T)arot;
    P.sqrt_a = (T)sqrt(arot);
    P.p_nb = (T)f.lam_up;
    P.p_b = (T)f.lam_dn;
    return;
  }
  const CellCoeffs c = cell_coeffs(sp, cs.ndens, cs.dt, cs.Ttr, cs.Trot, Tvib);
  if (!c.ok) {
    atomicOr(flags, (uint32_t)F_A_NONPOS);
    cs.active = 0;
    P.active = 0;
    return;
  }
  cs.e_rot_tgt = c.e_rot_tgt;
  cs.e_vib_tgt = c.e_vib_tgt;
  if (c.tgt_clamped) {
    atomicOr(flags, (uint32_t)F_TREL_CLAMP);
    atomicAdd(&counters[C_TREL_CLAMP], 1ull);
  }
  // homogeneous cell: the fields at every particle are the cell values, so
  // D_tr, its Cholesky factor and the relaxation temperatures are per cell
  const DriftDiff dd = drift_diffusion(sp, c, cs.dt, cs.Pi, cs.Ttr, cs.Trot, Tvib);
  if (dd.fixed) atomicAdd(&counters[C_CHOL_FIX], 1ull);
  if (dd.nu_zero) atomicAdd(&counters[C_NU_ZERO], 1ull);
  if (dd.failed) atomicOr(flags, (uint32_t)F_CHOL_FAIL_AFTER_FIX);
  if (dd.clamped) {
    atomicOr(flags, (uint32_t)F_TREL_CLAMP);
    atomicAdd(&counters[C_TREL_CLAMP], 1ull);
  }
  const double a = dd.alpha, oma2 = 1.0 - a * a, sq = sqrt(oma2);
  P.as = (T)(a * cs.s);
  P.ar = (T)(a * sqrt(cs.r));
  for (int i = 0; i < 6; ++i) P.Lp[i] = (T)(sq * dd.L[i]);
  const double arot = R * dd.Trot_rel * oma2 / 2.0;
  P.a_rot = (T)arot;
  P.sqrt_a = (T)sqrt(arot);
  const double eb = dd.evib_rel / (R * sp.theta_v);
  P.p_nb = (T)(1.0 / (1.0 + eb * oma2));
  P.p_b = (T)((1.0 + eb) * oma2);
}

// Initial coefficients from freshly reduced moments (identity pending rescale).
// mom: field-major USP_NMOM x ncell as written by assemble_moments.
template <typename T>
__global__ void init_params_kernel(Species sp, int ncell, int c0, int c1,
                                   const double* __restrict__ mom, CellState* cells,
                                   CollideParams<T>* prm, uint32_t* flags,
                                   unsigned long long* counters) {
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c1) return;
  CellState cs = cells[c];
  const double R = gasR(sp);
  for (int i = 0; i < 3; ++i) { cs.U[i] = mom[(1 + i) * ncell + c]; cs.Us[i] = cs.U[i]; }
  for (int i = 0; i < 6; ++i) cs.Pi[i] = mom[(7 + i) * ncell + c];
  cs.Ttr = mom[4 * ncell + c];
  cs.Trot = mom[5 * ncell + c];
  cs.ebar = 0.0;
  cs.s = 1.0;
  cs.r = 1.0;
  cs.maxI = 1 << 30;   // unknown: build every jump-table row
  cs.active = cs.N >= 2;
  if (!cs.active) atomicAdd(&counters[C_SKIPPED_CELLS], 1ull);
  cells[c] = cs;  // ebar is filled by the level-sum pass below
  (void)R;
  (void)prm;
  (void)flags;
}

template <typename T>
__global__ void init_params_finish(Species sp, int c0, int c1, const double* __restrict__ levsum,
                                   CellState* cells, CollideParams<T>* prm, uint32_t* flags,
                                   unsigned long long* counters) {
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c1) return;
  CellState cs = cells[c];
  cs.ebar = cs.N > 0 ? levsum[c] / (double)cs.N : 0.0;
  CollideParams<T> P;
  write_params<T>(sp, cs, P, flags, counters);
  cells[c] = cs;
  prm[c] = P;
}

// ---------------------------------------------------------------------------
// finalize: +-1 level correction, rescale factors, next moments and params.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Vibrational summation correction of Sec. 4.C, one warp per cell:
// I_Delta = floor(N e_vib^{n+1} / (R Theta) - sum I* + U), then random +-1
// picks with replacement at position k = floor(w N / 2^32), at most 64 N
// draws, a decrement meeting level 0 drawing again.  32 draws per round; the
// acceptance of draw j is decided exactly as in the one-at-a-time loop: a
// decrement on particle k is accepted iff fewer than lev[k] earlier accepted
// decrements in the round hit k.  The net level change goes to sums[c].net.
__global__ void __launch_bounds__(128, 8)
levelfix_kernel(Species sp, int c0, int c1, const CellState* __restrict__ cells,
                                CellSums* __restrict__ sums, int* __restrict__ lev,
                                uint32_t* flags, unsigned long long* counters, uint32_t k0,
                                uint32_t k1) {
  const int lane = threadIdx.x & 31;
  const int c = c0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (c >= c1) return;
  const CellState& cs = cells[c];
  if (!cs.active) return;
  const double Rth = gasR(sp) * sp.theta_v;
  const long long N = cs.N;
  const unsigned int step = cs.step;
  long long Id = 0;
  if (lane == 0) {
    const U4 w = philox4x32_10((uint32_t)c, step, CTAG_IDELTA, 0u, k0, k1);
    const double u = uniform_open<double>(w.x);
    Id = (long long)floor((double)N * cs.e_vib_tgt / Rth - (double)(long long)sums[c].I + u);
  }
  Id = __shfl_sync(0xffffffffu, Id, 0);
  long long remaining = Id, draws = 0;
  const long long cap = 64 * N;
  long long net = 0;
  int* lv = lev + cs.off;
  const bool down = remaining < 0;   // decrements need the current level
  // Draw j picks particle k = floor(word_j N / 2^32), word j % 4 of the
  // Philox block (c, step, CTAG_PICK, j / 4), and the draws are decided one
  // after another.  The warp takes them 128 at a time: lane l computes the
  // block of draws 4 l .. 4 l + 3 and the lanes exchange words so that
  // sub-batch s holds draws 32 s + lane; the levels of all four sub-batches
  // are read before the first is decided, so their latencies overlap.  A
  // sub-batch is cut short only where the correction completes (or at the
  // cap), which ends the loop, so every round starts on a multiple of 128.
  // A level read before an earlier sub-batch's decrements is read again when
  // that sub-batch decremented its particle (every level of the later
  // sub-batches, after more than two decrements).
  constexpr int kSub = 4;
  while (remaining != 0 && draws < cap) {
    const U4 w = philox4x32_10((uint32_t)c, step, CTAG_PICK, (uint32_t)((draws >> 2) + lane),
                               k0, k1);
    long long kk[kSub];
    bool vd[kSub];
    int cur[kSub];
#pragma unroll
    for (int s = 0; s < kSub; ++s) {
      const int src = 8 * s + (lane >> 2);
      const uint32_t x = __shfl_sync(0xffffffffu, w.x, src), y = __shfl_sync(0xffffffffu, w.y, src);
      const uint32_t z = __shfl_sync(0xffffffffu, w.z, src), v = __shfl_sync(0xffffffffu, w.w, src);
      const int q = lane & 3;
      const uint32_t word = q == 0 ? x : q == 1 ? y : q == 2 ? z : v;
      kk[s] = (long long)(((unsigned long long)word * (unsigned long long)N) >> 32);
      vd[s] = draws + 32 * s + lane < cap;
      cur[s] = down && vd[s] ? __ldcg(&lv[kk[s]]) : 0;
    }
#pragma unroll
    for (int s = 0; s < kSub; ++s) {
      if (remaining == 0 || draws >= cap) break;
      const long long k = kk[s];
      const bool valid = vd[s];
      bool accept;
      if (!down) {
        accept = valid;
      } else {
        const unsigned grp = __match_any_sync(0xffffffffu, valid ? k : -1ll);
        const int rank = __popc(grp & lanemask_lt());
        accept = valid && rank < cur[s];
      }
      const unsigned am = __ballot_sync(0xffffffffu, accept);
      const long long need = remaining > 0 ? remaining : -remaining;
      const int nacc = __popc(am);
      const int take = (int)(nacc < need ? nacc : need);
      const int order = __popc(am & lanemask_lt());
      const bool eff = accept && order < take;
      __syncwarp();
      if (eff) atomicAdd(&lv[k], down ? -1 : 1);
      __syncwarp();
      long long used = 32;
      if (take == need && take > 0) {
        // the loop stops at the take-th accepted draw
        unsigned m = am;
        for (int i = 1; i < take; ++i) m &= m - 1;
        used = __ffs((int)m);  // lane index + 1
      }
      if (draws + used > cap) used = cap - draws;
      draws += used;
      if (!down) { remaining -= take; net += take; }
      else { remaining += take; net -= take; }
      if (down && remaining != 0 && s + 1 < kSub) {
        unsigned em = __ballot_sync(0xffffffffu, eff);
        if (em) {
          bool st[kSub];
#pragma unroll
          for (int t = 0; t < kSub; ++t) st[t] = __popc(em) > 2;
          if (__popc(em) <= 2) {
            while (em) {
              const int l = __ffs((int)em) - 1;
              em &= em - 1;
              const long long kd = __shfl_sync(0xffffffffu, k, l);
#pragma unroll
              for (int t = s + 1; t < kSub; ++t) st[t] |= kk[t] == kd;
            }
          }
#pragma unroll
          for (int t = s + 1; t < kSub; ++t)
            if (st[t] && vd[t]) cur[t] = __ldcg(&lv[kk[t]]);
        }
      }
    }
  }
  if (lane != 0) return;
  if (remaining != 0) atomicOr(flags, (uint32_t)F_VIB_LOOP_CAP);
  if (draws) atomicAdd(&counters[C_VIB_DRAWS], (unsigned long long)draws);
  sums[c].net = net;
}

// Rotational and velocity rescale factors of Sec. 4.C, the moments of the
// next step (exact under the affine rescale) and the next step's per-cell
// coefficients; one thread per cell so that the FP64 work of 32 cells shares
// each warp instruction.
template <typename T>
__global__ void cellupdate_kernel(Species sp, int c0, int c1, CellState* __restrict__ cells,
                                  CollideParams<T>* __restrict__ prm,
                                  CellSums* __restrict__ sums, uint32_t* flags,
                                  unsigned long long* counters) {
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c1) return;
  CellState cs = cells[c];
  if (!cs.active) return;
  const double R = gasR(sp);
  const double Rth = R * sp.theta_v;
  const CellSums S = sums[c];
  const double invN = 1.0 / (double)cs.N;
  const double sumI = (double)((long long)S.I + S.net);
  // rotational scaling
  const double er_star = S.v[9] * invN;
  const double r = er_star > 0.0 ? cs.e_rot_tgt / er_star : 1.0;
  const double e_rot_new = r * er_star;
  const double e_vib_new = Rth * sumI * invN;
  // velocity scaling about the post-collision mean
  const double m0 = S.v[0] * invN, m1 = S.v[1] * invN, m2 = S.v[2] * invN;
  double Ps[6];
  Ps[0] = S.v[3] * invN - m0 * m0;
  Ps[1] = S.v[4] * invN - m1 * m1;
  Ps[2] = S.v[5] * invN - m2 * m2;
  Ps[3] = S.v[6] * invN - m0 * m1;
  Ps[4] = S.v[7] * invN - m0 * m2;
  Ps[5] = S.v[8] * invN - m1 * m2;
  const double etr_star = 0.5 * (Ps[0] + Ps[1] + Ps[2]);
  const double e_tr_n = 0.5 * (cs.Pi[0] + cs.Pi[1] + cs.Pi[2]);
  const double e_rot_n = R * cs.Trot;
  const double e_vib_n = Rth * cs.ebar;
  const double rad = (e_tr_n + e_rot_n + e_vib_n - e_rot_new - e_vib_new) / etr_star;
  double s;
  double Un[3] = {cs.U[0], cs.U[1], cs.U[2]};
  double Us[3] = {cs.U[0] + m0, cs.U[1] + m1, cs.U[2] + m2};
  if (!(etr_star > 0.0) || !(rad > 0.0)) {
    atomicOr(flags, (uint32_t)F_NEG_RADICAND);
    atomicAdd(&counters[C_NEG_RADICAND], 1ull);
    s = 1.0;  // velocities stay as collided: c = U* + (c* - U*)
    for (int i = 0; i < 3; ++i) Un[i] = Us[i];
  } else {
    s = sqrt(rad);
  }
  for (int i = 0; i < 3; ++i) { cs.U[i] = Un[i]; cs.Us[i] = Us[i]; }
  for (int i = 0; i < 6; ++i) cs.Pi[i] = s * s * Ps[i];
  cs.Ttr = (cs.Pi[0] + cs.Pi[1] + cs.Pi[2]) / (3.0 * R);
  cs.Trot = e_rot_new / R;
  cs.ebar = sumI * invN;
  cs.s = s;
  cs.r = r;
  cs.step += 1;
  cs.maxI = S.maxI + 1;   // the +-1 correction can raise the largest level by one
  CollideParams<T> P;
  write_params<T>(sp, cs, P, flags, counters);
  cells[c] = cs;
  prm[c] = P;
  CellSums z;
  memset(&z, 0, sizeof(z));
  sums[c] = z;
}

// ---------------------------------------------------------------------------
// Moments of the current state (pending rescale applied), FP64 accumulation.
// pass 0: sum c, sum eps, sum I;  pass 1: central sums about the mean.
// acc layout per cell: [0..2] sum c, [3] sum eps, [4] sum I,
// [5..10] sum CC, [11..13] sum C^2 C / 2, [14..16] sum C eps, [17..19] sum C I
// ---------------------------------------------------------------------------
constexpr int kMomAcc = 20;

// Per-particle arithmetic in the state precision T; partial sums stay in T
// within a thread (a few particles) and a warp, then combine in FP64.
template <typename T>
__global__ void __launch_bounds__(kBlock)
moments_kernel(int pass, const Tile* __restrict__ tiles, int ntiles,
               const CellState* __restrict__ cells, const T* __restrict__ cx,
               const T* __restrict__ cy, const T* __restrict__ cz, const T* __restrict__ er,
               const int* __restrict__ lev, double* __restrict__ acc_out) {
  // each block owns a contiguous range of the tile list; per-thread sums run
  // over all its tiles of one cell and are reduced and added to the cell's
  // accumulators once per (block, cell)
  __shared__ double red[kBlock / 32][15];
  __shared__ T cp[11];   // U (3), U* (3), s, r, pass-0 mean (3) in T
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int G = gridDim.x;
  const int t_begin = (int)(((long long)ntiles * blockIdx.x) / G);
  const int t_end = (int)(((long long)ntiles * (blockIdx.x + 1)) / G);
  const int na = pass == 0 ? 5 : 15;
  T a[15];
  for (int i = 0; i < 15; ++i) a[i] = T(0);
  for (int t = t_begin; t < t_end; ++t) {
    const Tile tl = tiles[t];
    const CellState& cs = cells[tl.cell];
    const bool first = t == t_begin || tiles[t - 1].cell != tl.cell;
    if (first) {
      // the cell's constants, converted once (one value per thread)
      __syncthreads();
      if (threadIdx.x < 11) {
        const int i = threadIdx.x;
        double v;
        if (i < 3) v = cs.U[i];
        else if (i < 6) v = cs.Us[i - 3];
        else if (i == 6) v = cs.s;
        else if (i == 7) v = cs.r;
        else v = (pass == 1 && cs.N > 0)
                     ? acc_out[(size_t)tl.cell * kMomAcc + (i - 8)] / (double)cs.N : 0.0;
        cp[i] = (T)v;
      }
      __syncthreads();
    }
    const long long base = cs.off + tl.start;
    const T U0 = cp[0], U1 = cp[1], U2 = cp[2];
    const T S0 = cp[3], S1 = cp[4], S2 = cp[5];
    const T sc = cp[6], rc = cp[7];
    const T mean0 = cp[8], mean1 = cp[9], mean2 = cp[10];
    for (int k = threadIdx.x; k < tl.count; k += kBlock) {
      const long long e = base + k;
      const T c0 = U0 + sc * (cx[e] - S0);
      const T c1 = U1 + sc * (cy[e] - S1);
      const T c2 = U2 + sc * (cz[e] - S2);
      const T ep = rc * er[e];
      const T li = (T)lev[e];
      if (pass == 0) {
        a[0] += c0; a[1] += c1; a[2] += c2; a[3] += ep; a[4] += li;
      } else {
        const T C0 = c0 - mean0, C1 = c1 - mean1, C2 = c2 - mean2;
        const T q = T(0.5) * (C0 * C0 + C1 * C1 + C2 * C2);
        a[0] += C0 * C0; a[1] += C1 * C1; a[2] += C2 * C2;
        a[3] += C0 * C1; a[4] += C0 * C2; a[5] += C1 * C2;
        a[6] += q * C0; a[7] += q * C1; a[8] += q * C2;
        a[9] += C0 * ep; a[10] += C1 * ep; a[11] += C2 * ep;
        a[12] += C0 * li; a[13] += C1 * li; a[14] += C2 * li;
      }
    }
    const bool last = t + 1 >= t_end || tiles[t + 1].cell != tl.cell;
    if (last) {
      // warp totals; lane i < na converts total i (one conversion per warp)
      T mine = T(0);
      for (int i = 0; i < na; ++i) {
        const T sm = warp_sum(a[i]);
        mine = lane == i ? sm : mine;
      }
      if (lane < na) red[wid][lane] = (double)mine;
      __syncthreads();
      if (threadIdx.x < na) {
        double sm = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) sm += red[w][threadIdx.x];
        atomicAdd(&acc_out[(size_t)tl.cell * kMomAcc + (pass == 0 ? 0 : 5) + threadIdx.x], sm);
      }
      for (int i = 0; i < 15; ++i) a[i] = T(0);
    }
  }
}

__global__ void assemble_moments(Species sp, int ncell, int c0, int c1,
                                 const CellState* __restrict__ cells,
                                 const double* __restrict__ acc, double* __restrict__ out,
                                 double* __restrict__ levsum) {
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c1) return;
  const double R = gasR(sp);
  const double N = (double)cells[c].N;
  const double* a = acc + (size_t)c * kMomAcc;
  if (levsum) levsum[c] = a[4];
  if (N <= 0.0) {
    for (int f = 0; f < USP_NMOM; ++f) out[(size_t)f * ncell + c] = 0.0;
    return;
  }
  const double inv = 1.0 / N;
  out[c] = N;
  for (int i = 0; i < 3; ++i) out[(size_t)(1 + i) * ncell + c] = a[i] * inv;
  const double Pxx = a[5] * inv, Pyy = a[6] * inv, Pzz = a[7] * inv;
  out[(size_t)4 * ncell + c] = (Pxx + Pyy + Pzz) / (3.0 * R);
  out[(size_t)5 * ncell + c] = a[3] * inv / R;
  out[(size_t)6 * ncell + c] = T_vib_of_level(sp, a[4] * inv);
  for (int i = 0; i < 6; ++i) out[(size_t)(7 + i) * ncell + c] = a[5 + i] * inv;
  for (int i = 0; i < 3; ++i) {
    out[(size_t)(13 + i) * ncell + c] = a[11 + i] * inv;
    out[(size_t)(16 + i) * ncell + c] = a[14 + i] * inv;
    out[(size_t)(19 + i) * ncell + c] = a[17 + i] * inv * R * sp.theta_v;
  }
}

// A freshly uploaded state has no pending rescale.
__global__ void reset_pending(int ncell, CellState* cells, CellSums* sums) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  for (int i = 0; i < 3; ++i) { cells[c].U[i] = 0.0; cells[c].Us[i] = 0.0; }
  cells[c].s = 1.0;
  cells[c].r = 1.0;
  for (int i = 0; i < 10; ++i) sums[c].v[i] = 0.0;
  sums[c].I = 0ull;
}

// Scatter an unpadded host-layout state (type S) into the padded device
// layout (type T), or gather back with the pending rescale applied.
template <typename S, typename T>
__global__ void scatter_state(int c_begin, int ncell, const CellState* __restrict__ cells,
                              const long long* __restrict__ uoff, const S* __restrict__ ix,
                              const S* __restrict__ iy, const S* __restrict__ iz,
                              const S* __restrict__ ie, const int* __restrict__ il,
                              T* __restrict__ cx, T* __restrict__ cy, T* __restrict__ cz,
                              T* __restrict__ er, int* __restrict__ lev) {
  for (int c = c_begin + blockIdx.y; c < ncell; c += gridDim.y) {
  const long long b = uoff[c], n = uoff[c + 1] - b, o = cells[c].off;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    cx[o + k] = (T)ix[b + k];
    cy[o + k] = (T)iy[b + k];
    cz[o + k] = (T)iz[b + k];
    er[o + k] = (T)ie[b + k];
    lev[o + k] = il[b + k];
  }
  }
}

template <typename T>
__global__ void gather_state(int ncell, const CellState* __restrict__ cells,
                             const long long* __restrict__ uoff, const T* __restrict__ cx,
                             const T* __restrict__ cy, const T* __restrict__ cz,
                             const T* __restrict__ er, const int* __restrict__ lev,
                             double* __restrict__ ox, double* __restrict__ oy,
                             double* __restrict__ oz, double* __restrict__ oe,
                             int* __restrict__ ol) {
  for (int c = blockIdx.y; c < ncell; c += gridDim.y) {
  const CellState cs = cells[c];
  const long long b = uoff[c], n = uoff[c + 1] - b, o = cs.off;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    ox[b + k] = cs.U[0] + cs.s * ((double)cx[o + k] - cs.Us[0]);
    oy[b + k] = cs.U[1] + cs.s * ((double)cy[o + k] - cs.Us[1]);
    oz[b + k] = cs.U[2] + cs.s * ((double)cz[o + k] - cs.Us[2]);
    oe[b + k] = cs.r * (double)er[o + k];
    ol[b + k] = lev[o + k];
  }
  }
}

template <typename T>
__global__ void gather_state_native(int ncell, const CellState* __restrict__ cells,
                                    const long long* __restrict__ uoff, const T* __restrict__ cx,
                                    const T* __restrict__ cy, const T* __restrict__ cz,
                                    const T* __restrict__ er, const int* __restrict__ lev,
                                    T* __restrict__ ox, T* __restrict__ oy, T* __restrict__ oz,
                                    T* __restrict__ oe, int* __restrict__ ol) {
  for (int c = blockIdx.y; c < ncell; c += gridDim.y) {
  const CellState cs = cells[c];
  const long long b = uoff[c], n = uoff[c + 1] - b, o = cs.off;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    ox[b + k] = (T)(cs.U[0] + cs.s * ((double)cx[o + k] - cs.Us[0]));
    oy[b + k] = (T)(cs.U[1] + cs.s * ((double)cy[o + k] - cs.Us[1]));
    oz[b + k] = (T)(cs.U[2] + cs.s * ((double)cz[o + k] - cs.Us[2]));
    oe[b + k] = (T)(cs.r * (double)er[o + k]);
    ol[b + k] = lev[o + k];
  }
  }
}

}  // namespace

// ===========================================================================
// Host side
// ===========================================================================
// runs of cells of the host-buffer step: each run's upload overlaps the
// previous run's arithmetic, and only the last run's arithmetic is exposed
constexpr int kHostRuns = 16;

struct usp_ctx {
  int kind;                 // 0 homogeneous cells, 1 channel, 2 plane
  ChannelCtx* ch;
  PlaneCtx* pl;
  cudaEvent_t prof_pending;
  Species sp;
  usp_config cfg;
  int precision;
  int ncell;
  long long nparticles;     // real particles
  long long nstore;         // padded storage length
  cudaStream_t stream;
  bool own_stream;
  // device buffers
  void* cx; void* cy; void* cz; void* er;
  int* lev;
  CellState* cells;
  void* prm;
  CellSums* sums;
  Tile* tiles;              // tiles of <= tile particles (block-tiled kernels)
  int ntiles;
  Tile* wtiles;             // tiles of <= kWT particles (warp-tiled particle pass)
  int nwtiles;
  std::vector<int> h_tfirst, h_wfirst;   // first tile of each cell in either list (ncell + 1)
  long long* uoff;          // unpadded offsets (device)
  double* macc;             // moment accumulators
  double* mout;             // moment output (device)
  double* levsum;
  long long wait_cycles;    // limit of the particle pass's waits (SM cycles)
  float* tab_nb;            // jump tables (FP32 form)
  float* tab_b;
  uint8_t* gd_nb;           // their guide tables
  uint8_t* gd_b;
  uint32_t* flags;
  unsigned long long* counters;
  std::vector<long long> h_uoff;
  std::vector<long long> h_poff;   // padded segment starts
  std::vector<float> tune_ms;      // autotuner timings: block-tiled 2, 3, 4, warp-tiled 2, 3, 4
  bool jratio_ready = false;       // the rows' pmf ratio table filled on the device
  int tile;
  int grid_collide;
  int minb;                 // register-budget variant of the particle pass
  int warp_tiles;           // 1: warp-tiled particle pass, 0: block-tiled
  int grid_by_minb[2][5];   // persistent grid per (design, variant)
  long long step;
  long long launches;
  cudaGraphExec_t graph_exec;
  int graph_steps;
  int graph_parity;          // channel buffer parity the graph was captured at
  cudaGraph_t graph;
  long long device_bytes;
  std::vector<void*> owned;
  void* stage;              // host-path staging buffer, kept between calls
  size_t stage_bytes;
  cudaStream_t copy_stream; // host-path uploads, overlapped with the scatter
  cudaEvent_t up_ev[kHostRuns + 1];   // upload pipeline: start + one per run of cells
  // per-kernel event timing
  int profiling;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_kind;   // kind of pair i (events 2i, 2i+1)
  size_t ev_used;
};

namespace {

int g_last_cuda_error = 0;

#define CK(x)                                            \
  do {                                                   \
    cudaError_t e_ = (x);                                \
    if (e_ != cudaSuccess) {                             \
      g_last_cuda_error = (int)e_;                       \
      return USP_ECUDA;                                  \
    }                                                    \
  } while (0)

void* dev_alloc(usp_ctx* c, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (c->cfg.alloc) {
    p = c->cfg.alloc(bytes, c->cfg.alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) {
    c->owned.push_back(p);
    c->device_bytes += (long long)bytes;
  }
  return p;
}

void dev_free_all(usp_ctx* c) {
  for (void* p : c->owned) {
    if (c->cfg.alloc && c->cfg.free_) c->cfg.free_(p, c->cfg.alloc_user);
    else if (!c->cfg.alloc) cudaFree(p);
  }
  c->owned.clear();
}

Species to_dev(const usp_species* s) {
  Species d;
  d.m = s->m; d.d_ref = s->d_ref; d.omega = s->omega; d.T_ref = s->T_ref;
  d.c_alpha = s->c_alpha; d.theta_v = s->theta_v; d.Z_rot = s->Z_rot; d.Z_vib = s->Z_vib;
  d.zmodel = s->zmodel; d.Zrot_inf = s->Zrot_inf; d.T_star = s->T_star; d.C1 = s->C1;
  d.C2 = s->C2; d.sigma_vib = s->sigma_vib;
  d.Tref_w = std::pow(s->T_ref, s->omega);
  d.zv_ht = s->sigma_vib > 0 ? kPi * s->d_ref * s->d_ref / s->sigma_vib : 0.0;
  d.R = kB / s->m;
  const double ca = s->c_alpha, w = s->omega;
  d.mu_ref0 = 5.0 * (ca + 1.0) * (ca + 2.0) * std::sqrt(s->m * kB * s->T_ref / kPi) /
              (4.0 * ca * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) * s->d_ref * s->d_ref);
  d.tauf0 = ca * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) / (5.0 * (ca + 1.0) * (ca + 2.0));
  d.method = 0;
  return d;
}

uint32_t key0(const usp_ctx* c) { return (uint32_t)(c->cfg.seed & 0xffffffffull); }
uint32_t key1(const usp_ctx* c) { return (uint32_t)(c->cfg.seed >> 32); }

void dev_release(usp_ctx* c, void* p) {
  auto it = std::find(c->owned.begin(), c->owned.end(), p);
  if (it == c->owned.end()) return;
  c->owned.erase(it);
  if (c->cfg.alloc && c->cfg.free_) c->cfg.free_(p, c->cfg.alloc_user);
  else if (!c->cfg.alloc) cudaFree(p);
}

void* env_alloc(void* owner, size_t bytes) { return dev_alloc((usp_ctx*)owner, bytes); }
void env_release(void* owner, void* p) { dev_release((usp_ctx*)owner, p); }

ChEnv make_env(usp_ctx* c) {
  ChEnv e;
  e.stream = c->stream;
  e.flags = c->flags;
  e.counters = c->counters;
  e.sp = c->sp;
  e.k0 = key0(c);
  e.k1 = key1(c);
  e.precision = c->precision;
  e.alloc = env_alloc;
  e.release = env_release;
  e.owner = c;
  return e;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// Cells split into tiles of at most `tile` particles, in cell order; first[i]
// is the index of cell i's first tile (first[ncell] = the number of tiles).
int make_tiles(usp_ctx* c, int tile, Tile** out, int* nout, std::vector<int>& first) {
  std::vector<Tile> t;
  first.assign(c->ncell + 1, 0);
  for (int i = 0; i < c->ncell; ++i) {
    first[i] = (int)t.size();
    const long long n = c->h_uoff[i + 1] - c->h_uoff[i];
    for (long long s = 0; s < n; s += tile) {
      Tile x;
      x.cell = i;
      x.start = (int)s;
      x.count = (int)std::min<long long>(tile, n - s);
      x.pad_ = 0;
      t.push_back(x);
    }
  }
  first[c->ncell] = (int)t.size();
  if (t.empty()) {
    Tile x = {0, 0, 0, 0};
    t.push_back(x);
  }
  Tile* d = (Tile*)dev_alloc(c, t.size() * sizeof(Tile));
  if (!d) return USP_ENOMEM;
  CK(cudaMemcpyAsync(d, t.data(), t.size() * sizeof(Tile), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *out = d;
  *nout = (int)t.size();
  return USP_OK;
}

int build_tiles(usp_ctx* c, int tile) {
  int rc = make_tiles(c, tile, &c->tiles, &c->ntiles, c->h_tfirst);
  if (rc) return rc;
  rc = make_tiles(c, std::min(tile, kWT), &c->wtiles, &c->nwtiles, c->h_wfirst);
  if (rc) return rc;
  c->tile = tile;
  return USP_OK;
}

// Event pair for one timed launch (profiling mode only).
int prof_begin(usp_ctx* c, int kind, cudaEvent_t* e1) {
  if (!c->profiling) return USP_OK;
  if (c->ev_used + 2 > c->ev_pool.size()) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      c->ev_pool.push_back(e);
    }
  }
  CK(cudaEventRecord(c->ev_pool[c->ev_used], c->stream));
  *e1 = c->ev_pool[c->ev_used + 1];
  c->ev_kind.push_back(kind);
  c->ev_used += 2;
  return USP_OK;
}
int prof_end(usp_ctx* c, cudaEvent_t e1) {
  if (!c->profiling) return USP_OK;
  CK(cudaEventRecord(e1, c->stream));
  return USP_OK;
}

int prof_cb(void* owner, int kind, int begin) {
  usp_ctx* c = (usp_ctx*)owner;
  if (begin) return prof_begin(c, kind, &c->prof_pending);
  return prof_end(c, c->prof_pending);
}

template <typename T, int MINB, int METHOD>
void* collide_fn(int warp_tiles) {
  return warp_tiles ? (void*)collide_warp_kernel<T, MINB, METHOD>
                    : (void*)collide_kernel<T, MINB, METHOD>;
}

template <typename T, int METHOD>
void* collide_variant_m(int warp_tiles, int minb) {
  return minb == 2 ? collide_fn<T, 2, METHOD>(warp_tiles)
                   : minb == 3 ? collide_fn<T, 3, METHOD>(warp_tiles)
                               : collide_fn<T, 4, METHOD>(warp_tiles);
}

template <typename T>
void* collide_variant(int warp_tiles, int minb, int method) {
  return method == 1 ? collide_variant_m<T, 1>(warp_tiles, minb)
                     : collide_variant_m<T, 0>(warp_tiles, minb);
}

template <typename T>
size_t collide_smem(int warp_tiles) {
  return warp_tiles ? wsmem_bytes<T>() : kBS * bstage_bytes<T>();
}

// A run of consecutive cells [c0, c1) and its tiles in either tile list.
struct CellRange {
  int c0, c1;
  int t0, t1;   // block tiles
  int w0, w1;   // warp tiles
};
CellRange cell_range(const usp_ctx* c, int c0, int c1) {
  return CellRange{c0, c1, c->h_tfirst[c0], c->h_tfirst[c1], c->h_wfirst[c0], c->h_wfirst[c1]};
}
CellRange all_cells(const usp_ctx* c) { return cell_range(c, 0, c->ncell); }

// Launch the particle pass (design warp_tiles, register-budget variant minb,
// the context's particle method) over the tiles of the cell range r, on the
// given state / sums buffers.
template <typename T, int METHOD>
int launch_collide_m(usp_ctx* c, int warp_tiles, int minb, int grid, void* cx, void* cy,
                     void* cz, void* er, int* lev, CellSums* sums, uint32_t* flags,
                     unsigned long long* counters, const CellRange& r) {
  const size_t smem = collide_smem<T>(warp_tiles);
  const CollideParams<T>* prm = (const CollideParams<T>*)c->prm;
  T* x = (T*)cx; T* y = (T*)cy; T* z = (T*)cz; T* e = (T*)er;
  const PhiloxRoundKeys rk = philox_round_keys(key0(c), key1(c));
  const JumpTabs tb{c->tab_nb, c->tab_b, c->gd_nb, c->gd_b};
  if (warp_tiles) {
    const Tile* tiles = c->wtiles + r.w0;
    const int ntiles = r.w1 - r.w0;
    if (minb == 2)
      collide_warp_kernel<T, 2, METHOD><<<grid, kBlock, smem, c->stream>>>(
          tiles, ntiles, prm, x, y, z, e, lev, sums, flags, counters, rk, tb, c->wait_cycles);
    else if (minb == 3)
      collide_warp_kernel<T, 3, METHOD><<<grid, kBlock, smem, c->stream>>>(
          tiles, ntiles, prm, x, y, z, e, lev, sums, flags, counters, rk, tb, c->wait_cycles);
    else
      collide_warp_kernel<T, 4, METHOD><<<grid, kBlock, smem, c->stream>>>(
          tiles, ntiles, prm, x, y, z, e, lev, sums, flags, counters, rk, tb, c->wait_cycles);
    CK(cudaGetLastError());
    return USP_OK;
  }
  const Tile* tiles = c->tiles + r.t0;
  const int ntiles = r.t1 - r.t0;
  if (minb == 2)
    collide_kernel<T, 2, METHOD><<<grid, kBlock, smem, c->stream>>>(
        tiles, ntiles, prm, x, y, z, e, lev, sums, flags, counters, rk, tb, c->wait_cycles);
  else if (minb == 3)
    collide_kernel<T, 3, METHOD><<<grid, kBlock, smem, c->stream>>>(
        tiles, ntiles, prm, x, y, z, e, lev, sums, flags, counters, rk, tb, c->wait_cycles);
  else
    collide_kernel<T, 4, METHOD><<<grid, kBlock, smem, c->stream>>>(
        tiles, ntiles, prm, x, y, z, e, lev, sums, flags, counters, rk, tb, c->wait_cycles);
  CK(cudaGetLastError());
  return USP_OK;
}
template <typename T>
int launch_collide(usp_ctx* c, int warp_tiles, int minb, int grid, void* cx, void* cy, void* cz,
                   void* er, int* lev, CellSums* sums, uint32_t* flags,
                   unsigned long long* counters, const CellRange& r) {
  return c->sp.method == 1
             ? launch_collide_m<T, 1>(c, warp_tiles, minb, grid, cx, cy, cz, er, lev, sums, flags,
                                      counters, r)
             : launch_collide_m<T, 0>(c, warp_tiles, minb, grid, cx, cy, cz, er, lev, sums, flags,
                                      counters, r);
}

// jump tables for the coming step (FP32 form only)
int launch_tables(usp_ctx* c, const CellRange& r) {
  if (c->precision != USP_FP32 || c->sp.method != 0 || r.c1 <= r.c0) return USP_OK;
  if (!c->jratio_ready) {
    jratio_kernel<<<1, 256, 0, c->stream>>>();
    CK(cudaGetLastError());
    c->jratio_ready = true;
  }
  jumptable_kernel<<<r.c1 - r.c0, kJT, 0, c->stream>>>(
      r.c0, r.c1, (const CollideParams<float>*)c->prm, c->cells, c->tab_nb, c->tab_b, c->gd_nb,
      c->gd_b);
  CK(cudaGetLastError());
  return USP_OK;
}

// one step of the cells of r
template <typename T>
int launch_step(usp_ctx* c, const CellRange& r) {
  if (r.c1 <= r.c0) return USP_OK;
  cudaEvent_t e1 = nullptr;
  int rc = prof_begin(c, 0, &e1);
  if (rc) return rc;
  rc = launch_collide<T>(c, c->warp_tiles, c->minb, c->grid_collide, c->cx, c->cy, c->cz, c->er,
                         c->lev, c->sums, c->flags, c->counters, r);
  if (rc) return rc;
  if ((rc = prof_end(c, e1))) return rc;
  if ((rc = prof_begin(c, 1, &e1))) return rc;
  const int n = r.c1 - r.c0;
  const int warps_per_block = 4;
  const int blocks = (n + warps_per_block - 1) / warps_per_block;
  levelfix_kernel<<<blocks, 32 * warps_per_block, 0, c->stream>>>(
      c->sp, r.c0, r.c1, c->cells, c->sums, c->lev, c->flags, c->counters, key0(c), key1(c));
  CK(cudaGetLastError());
  // one warp per block: the cells' FP64 work spreads over all SMs' FP64 pipes
  cellupdate_kernel<T><<<(n + 31) / 32, 32, 0, c->stream>>>(
      c->sp, r.c0, r.c1, c->cells, (CollideParams<T>*)c->prm, c->sums, c->flags, c->counters);
  CK(cudaGetLastError());
  if ((rc = launch_tables(c, r))) return rc;
  return prof_end(c, e1);
}

int kernels_per_step(const usp_ctx* c) {
  if (c->kind == 1) return ch_kernels_per_step(c->ch);
  if (c->kind == 2) return pl_kernels_per_step(c->pl);
  return c->precision == USP_FP32 && c->sp.method == 0 ? 4 : 3;
}

int step_once(usp_ctx* c) {
  if (c->kind == 1) return ch_launch_step(c->ch, make_env(c), c->profiling ? prof_cb : nullptr);
  if (c->kind == 2) return pl_launch_step(c->pl, make_env(c), c->profiling ? prof_cb : nullptr);
  return c->precision == USP_FP32 ? launch_step<float>(c, all_cells(c))
                                  : launch_step<double>(c, all_cells(c));
}

// moments of the cells of r (pending rescale applied) into mout
template <typename T>
int compute_moments(usp_ctx* c, double* levsum, const CellRange& r) {
  if (r.c1 <= r.c0) return USP_OK;
  CK(cudaMemsetAsync(c->macc + (size_t)r.c0 * kMomAcc, 0,
                     sizeof(double) * kMomAcc * (r.c1 - r.c0), c->stream));
  if (r.t1 > r.t0) {
    for (int pass = 0; pass < 2; ++pass) {
      moments_kernel<T><<<c->grid_collide, kBlock, 0, c->stream>>>(
          pass, c->tiles + r.t0, r.t1 - r.t0, c->cells, (const T*)c->cx, (const T*)c->cy,
          (const T*)c->cz, (const T*)c->er, c->lev, c->macc);
      CK(cudaGetLastError());
    }
    c->launches += 2;
  }
  assemble_moments<<<(r.c1 - r.c0 + 127) / 128, 128, 0, c->stream>>>(
      c->sp, c->ncell, r.c0, r.c1, c->cells, c->macc, c->mout, levsum);
  CK(cudaGetLastError());
  c->launches += 1;
  return USP_OK;
}
template <typename T>
int compute_moments(usp_ctx* c, double* levsum) {
  return compute_moments<T>(c, levsum, all_cells(c));
}

// coefficients of the cells of r from freshly uploaded particles
template <typename T>
int init_params(usp_ctx* c, const CellRange& r) {
  if (r.c1 <= r.c0) return USP_OK;
  int rc = compute_moments<T>(c, c->levsum, r);
  if (rc) return rc;
  const int b = (r.c1 - r.c0 + 127) / 128;
  init_params_kernel<T><<<b, 128, 0, c->stream>>>(c->sp, c->ncell, r.c0, r.c1, c->mout,
                                                  c->cells, (CollideParams<T>*)c->prm, c->flags,
                                                  c->counters);
  CK(cudaGetLastError());
  init_params_finish<T><<<b, 128, 0, c->stream>>>(c->sp, r.c0, r.c1, c->levsum, c->cells,
                                                  (CollideParams<T>*)c->prm, c->flags, c->counters);
  CK(cudaGetLastError());
  c->launches += 2;
  if ((rc = launch_tables(c, r))) return rc;
  c->launches += c->precision == USP_FP32 && c->sp.method == 0 ? 1 : 0;
  return USP_OK;
}
template <typename T>
int init_params(usp_ctx* c) {
  return init_params<T>(c, all_cells(c));
}

// The host paths stage the state in one device buffer, allocated on first use
// and kept (the largest request so far), so a call makes no allocation.
void* staging(usp_ctx* c, size_t bytes) {
  if (c->stage && c->stage_bytes >= bytes) return c->stage;
  if (c->stage) {
    // queued copies and kernels may still read the old buffer, and a caller's
    // free callback is not stream-ordered: let them finish first
    cudaStreamSynchronize(c->stream);
    if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
    dev_release(c, c->stage);
  }
  c->stage = dev_alloc(c, bytes);
  c->stage_bytes = c->stage ? bytes : 0;
  return c->stage;
}

int upload_state(usp_ctx* c, const void* hx, const void* hy, const void* hz, const void* he,
                 const int32_t* hl, bool host_is_native) {
  const long long n = c->nparticles;
  const size_t es = host_is_native ? (c->precision == USP_FP32 ? 4 : 8) : 8;
  static_assert(sizeof(int) == 4, "int32");
  void* st = staging(c, (size_t)n * (4 * es + 4) + 64);
  if (!st) return USP_ENOMEM;
  char* p = (char*)st;
  void* sx = p; void* sy = p + n * es; void* sz = p + 2 * n * es; void* se = p + 3 * n * es;
  int* sl = (int*)(p + 4 * n * es);
  CK(cudaMemcpyAsync(sx, hx, n * es, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(sy, hy, n * es, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(sz, hz, n * es, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(se, he, n * es, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(sl, hl, n * 4, cudaMemcpyHostToDevice, c->stream));
  reset_pending<<<(c->ncell + 127) / 128, 128, 0, c->stream>>>(c->ncell, c->cells, c->sums);
  CK(cudaGetLastError());
  c->launches += 1;
  dim3 grid(64, std::min(c->ncell, 65535));
  if (c->precision == USP_FP32) {
    if (es == 4)
      scatter_state<float, float><<<grid, 256, 0, c->stream>>>(
          0, c->ncell, c->cells, c->uoff, (const float*)sx, (const float*)sy, (const float*)sz,
          (const float*)se, sl, (float*)c->cx, (float*)c->cy, (float*)c->cz, (float*)c->er, c->lev);
    else
      scatter_state<double, float><<<grid, 256, 0, c->stream>>>(
          0, c->ncell, c->cells, c->uoff, (const double*)sx, (const double*)sy, (const double*)sz,
          (const double*)se, sl, (float*)c->cx, (float*)c->cy, (float*)c->cz, (float*)c->er, c->lev);
  } else {
    scatter_state<double, double><<<grid, 256, 0, c->stream>>>(
        0, c->ncell, c->cells, c->uoff, (const double*)sx, (const double*)sy, (const double*)sz,
        (const double*)se, sl, (double*)c->cx, (double*)c->cy, (double*)c->cz, (double*)c->er,
        c->lev);
  }
  CK(cudaGetLastError());
  c->launches += 1;
  return USP_OK;
}

// Host-buffer step of a homogeneous context.  Cells are independent, so the
// state goes up in kUpChunks runs of whole cells on the copy stream, and each
// run is scattered, set up, stepped nsteps times and reduced to its moments
// (into mout) on the context stream while the next run is still in transit:
// the transfer hides the arithmetic instead of preceding it.
template <typename T>
int step_host_chunked(usp_ctx* c, const void* hx, const void* hy, const void* hz,
                      const void* he, const int32_t* hl, int nsteps) {
  constexpr int K = kHostRuns;
  const long long n = c->nparticles;
  const size_t es = sizeof(T);
  void* st = staging(c, (size_t)n * (4 * es + 4) + 64);
  if (!st) return USP_ENOMEM;
  if (!c->copy_stream) {
    CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    for (int k = 0; k <= K; ++k) CK(cudaEventCreateWithFlags(&c->up_ev[k], cudaEventDisableTiming));
  }
  char* p = (char*)st;
  char* dst[5] = {p, p + n * es, p + 2 * n * es, p + 3 * n * es, p + 4 * n * es};
  const char* src[5] = {(const char*)hx, (const char*)hy, (const char*)hz, (const char*)he,
                        (const char*)hl};
  const size_t sz[5] = {es, es, es, es, 4};
  // after the first copy is queued, an error return first waits for the
  // copies from the caller's buffers still in flight
  auto body = [&]() -> int {
  // the staging buffer is free once the context stream has passed this point
  CK(cudaEventRecord(c->up_ev[0], c->stream));
  CK(cudaStreamWaitEvent(c->copy_stream, c->up_ev[0], 0));
  reset_pending<<<(c->ncell + 127) / 128, 128, 0, c->stream>>>(c->ncell, c->cells, c->sums);
  CK(cudaGetLastError());
  c->launches += 1;
  int cb = 0;
  for (int k = 0; k < K; ++k) {
    const int ca = cb;
    const long long target = n * (k + 1) / K;
    while (cb < c->ncell && (c->h_uoff[cb + 1] <= target || k == K - 1)) ++cb;
    if (cb == ca) continue;
    const long long b = c->h_uoff[ca], e = c->h_uoff[cb];
    for (int f = 0; f < 5; ++f)
      CK(cudaMemcpyAsync(dst[f] + b * sz[f], src[f] + b * sz[f], (e - b) * sz[f],
                         cudaMemcpyHostToDevice, c->copy_stream));
    CK(cudaEventRecord(c->up_ev[k + 1], c->copy_stream));
    CK(cudaStreamWaitEvent(c->stream, c->up_ev[k + 1], 0));
    dim3 grid(64, std::min(cb - ca, 65535));
    scatter_state<T, T><<<grid, 256, 0, c->stream>>>(
        ca, cb, c->cells, c->uoff, (const T*)dst[0], (const T*)dst[1], (const T*)dst[2],
        (const T*)dst[3], (const int*)dst[4], (T*)c->cx, (T*)c->cy, (T*)c->cz, (T*)c->er, c->lev);
    CK(cudaGetLastError());
    c->launches += 1;
    const CellRange r = cell_range(c, ca, cb);
    int rc = init_params<T>(c, r);
    if (rc) return rc;
    for (int s = 0; s < nsteps; ++s) {
      if ((rc = launch_step<T>(c, r))) return rc;
      c->launches += kernels_per_step(c);
    }
    if ((rc = compute_moments<T>(c, nullptr, r))) return rc;
  }
  return USP_OK;
  };
  const int rc = body();
  if (rc) {
    cudaStreamSynchronize(c->copy_stream);
    return rc;
  }
  c->step += nsteps;
  return USP_OK;
}

int build_graph(usp_ctx* c, int steps) {
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
  }
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  int rc = USP_OK;
  for (int i = 0; i < steps && rc == USP_OK; ++i) rc = step_once(c);
  cudaGraph_t g;
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (rc != USP_OK) return rc;
  CK(e);
  CK(cudaGraphInstantiate(&c->graph_exec, g, 0));
  c->graph = g;
  c->graph_steps = steps;
  return USP_OK;
}

// Autotuner of the particle pass: times each design (block-tiled, warp-tiled)
// and register-budget variant (2, 3 or 4 resident blocks per SM) on a scratch
// copy of the whole state (each variant starts from the same copy; one
// untimed and two timed launches) and keeps the fastest; within 3 % the
// earlier candidate wins (warp-tiled before block-tiled, fewer resident
// blocks before more).  The state it is timed on is the initial one; as the
// levels spread over more jump-table rows, the tables' share of the unified
// L1 grows, and fewer resident blocks (less shared memory, more registers)
// keep the pass faster: on the 4096-instance workload 3 and 4 blocks per SM
// tie within 1 % at the start, while from step 250 on 3 take 1.69 ms per
// launch and 4 take 1.82 ms.
template <typename T>
int autotune(usp_ctx* c) {
  const size_t es = sizeof(T);
  const int last_cell = c->ncell - 1;
  const long long end = c->h_poff[last_cell] +
      ((c->h_uoff[last_cell + 1] - c->h_uoff[last_cell]) + kAlign - 1) / kAlign * kAlign;
  const size_t bytes = (size_t)end * (4 * es + 4);
  unsigned char* scratch = (unsigned char*)dev_alloc(c, bytes + sizeof(CellSums) * c->ncell + 512);
  if (!scratch) return USP_ENOMEM;
  void* sx = scratch; void* sy = scratch + end * es; void* sz = scratch + 2 * end * es;
  void* se = scratch + 3 * end * es;
  int* sl = (int*)(scratch + 4 * end * es);
  CellSums* ssum = (CellSums*)(scratch + ((bytes + 255) & ~(size_t)255));
  uint32_t* sflags = (uint32_t*)((unsigned char*)ssum + sizeof(CellSums) * c->ncell);
  unsigned long long* scnt = (unsigned long long*)((unsigned char*)sflags + 256);
  auto fresh = [&]() -> int {
    CK(cudaMemcpyAsync(sx, c->cx, end * es, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(sy, c->cy, end * es, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(sz, c->cz, end * es, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(se, c->er, end * es, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(sl, c->lev, end * 4, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemsetAsync(ssum, 0, sizeof(CellSums) * c->ncell + 512, c->stream));
    return USP_OK;
  };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_mb = 3, best_wt = 1;
  c->tune_ms.assign(6, 0.f);
  for (int wt = 1; wt >= 0; --wt) {
    for (int mb = 2; mb <= 4; ++mb) {
      int rc = fresh();
      if (rc) return rc;
      const int grid = c->grid_by_minb[wt][mb];
      for (int r = 0; r < 3; ++r) {
        if (r == 1) CK(cudaEventRecord(e0, c->stream));
        rc = launch_collide<T>(c, wt, mb, grid, sx, sy, sz, se, sl, ssum, sflags, scnt,
                             all_cells(c));
        if (rc) return rc;
      }
      CK(cudaEventRecord(e1, c->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      c->tune_ms[3 * wt + mb - 2] = ms / 2.f;
      if (ms < 0.97f * best) { best = ms; best_mb = mb; best_wt = wt; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->launches += 18;
  c->minb = best_mb;
  c->warp_tiles = best_wt;
  c->grid_collide = c->grid_by_minb[best_wt][best_mb];
  CK(cudaStreamSynchronize(c->stream));
  if (!c->cfg.alloc) cudaFree(scratch);
  else if (c->cfg.free_) c->cfg.free_(scratch, c->cfg.alloc_user);
  c->owned.erase(std::find(c->owned.begin(), c->owned.end(), (void*)scratch));
  c->device_bytes -= (long long)(((bytes + sizeof(CellSums) * c->ncell + 512) + 255) & ~(size_t)255);
  return USP_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int usp_select_device(int dev) {
  int n = 0;
  CK(cudaGetDeviceCount(&n));
  if (dev < 0 || dev >= n) return USP_EINVAL;
  CK(cudaSetDevice(dev));
  return USP_OK;
}

double usp_tau_c(const usp_species* s, double n, double T) {
  if (!s) return 0.0;
  const double kPiH = 3.14159265358979323846;
  const double kBH = 1.380649e-23;
  const double ca = s->c_alpha, w = s->omega;
  const double mu_ref = 5.0 * (ca + 1.0) * (ca + 2.0) * std::sqrt(s->m * kBH * s->T_ref / kPiH) /
                        (4.0 * ca * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) * s->d_ref * s->d_ref);
  const double mu = mu_ref * std::pow(T / s->T_ref, w);
  return ca * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) / (5.0 * (ca + 1.0) * (ca + 2.0)) * mu /
         (n * kBH * T);
}

const char* usp_strerror(int err) {
  switch (err) {
    case USP_OK: return "ok";
    case USP_EINVAL: return "invalid argument";
    case USP_ENOMEM: return "device allocation failed";
    case USP_ECUDA: return "CUDA runtime error";
    case USP_EDEVICE: return "device status word reports an error";
    case USP_ENOTSUP: return "not supported";
    default: return "unknown error";
  }
}

int usp_init_homogeneous(usp_ctx** out, const usp_species* sp, const usp_config* cfg, int n_cells,
                         const int64_t* h_offsets, const double* h_ndens, const double* h_dt,
                         const double* h_cx, const double* h_cy, const double* h_cz,
                         const double* h_erot, const int32_t* h_lev) {
  if (!out || !sp || !cfg || n_cells <= 0 || !h_offsets || !h_ndens || !h_dt) return USP_EINVAL;
  if (cfg->precision != USP_FP32 && cfg->precision != USP_FP64) return USP_EINVAL;
  if (h_offsets[0] != 0) return USP_EINVAL;
  for (int i = 0; i < n_cells; ++i) {
    if (h_offsets[i + 1] < h_offsets[i]) return USP_EINVAL;
    if (!(h_ndens[i] > 0.0) || !(h_dt[i] > 0.0)) return USP_EINVAL;
  }
  const long long n = h_offsets[n_cells];
  if (n > 0x7fffffffll) return USP_EINVAL;
  if (n > 0 && (!h_cx || !h_cy || !h_cz || !h_erot || !h_lev)) return USP_EINVAL;
  if (!(sp->m > 0) || !(sp->d_ref > 0) || !(sp->T_ref > 0) || !(sp->c_alpha > 0) ||
      !(sp->theta_v > 0))
    return USP_EINVAL;
  *out = nullptr;
  if (cfg->method != USP_METHOD_USP_FPM && cfg->method != USP_METHOD_FPM) return USP_EINVAL;
  usp_ctx* c = new usp_ctx();
  c->kind = 0;
  c->ch = nullptr;
  c->pl = nullptr;
  std::memset((void*)&c->sp, 0, sizeof(c->sp));
  c->cfg = *cfg;
  c->sp = to_dev(sp);
  c->sp.method = cfg->method;
  c->precision = cfg->precision;
  c->ncell = n_cells;
  c->nparticles = n;
  c->graph_exec = nullptr;
  c->graph = nullptr;
  c->graph_steps = 0;
  c->graph_parity = 0;
  c->step = cfg->step0;
  c->launches = 0;
  c->device_bytes = 0;
  c->profiling = 0;
  c->ev_used = 0;
  // the stream is made after the allocations, so that a failing allocator
  // callback is reported (USP_ENOMEM) before any CUDA call
  c->stream = nullptr;
  c->own_stream = false;
  auto fail = [&](int rc) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    dev_free_all(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return rc;
  };
  c->h_uoff.assign(h_offsets, h_offsets + n_cells + 1);
  std::vector<CellState> hc(n_cells);
  long long off = 0;
  for (int i = 0; i < n_cells; ++i) {
    CellState& s = hc[i];
    std::memset(&s, 0, sizeof(s));
    s.off = off;
    c->h_poff.push_back(off);
    s.N = h_offsets[i + 1] - h_offsets[i];
    s.pid0 = (unsigned int)h_offsets[i];
    s.step = (unsigned int)cfg->step0;
    s.ndens = h_ndens[i];
    s.dt = h_dt[i];
    s.s = 1.0;
    s.r = 1.0;
    off += (s.N + kAlign - 1) / kAlign * kAlign;
  }
  c->nstore = std::max<long long>(off, kAlign);
  const size_t es = c->precision == USP_FP32 ? 4 : 8;
  c->cx = dev_alloc(c, c->nstore * es);
  c->cy = dev_alloc(c, c->nstore * es);
  c->cz = dev_alloc(c, c->nstore * es);
  c->er = dev_alloc(c, c->nstore * es);
  c->lev = (int*)dev_alloc(c, c->nstore * 4);
  c->cells = (CellState*)dev_alloc(c, sizeof(CellState) * n_cells);
  c->prm = dev_alloc(c, (c->precision == USP_FP32 ? sizeof(CollideParams<float>)
                                                  : sizeof(CollideParams<double>)) * n_cells);
  c->sums = (CellSums*)dev_alloc(c, sizeof(CellSums) * n_cells);
  c->uoff = (long long*)dev_alloc(c, sizeof(long long) * (n_cells + 1));
  c->macc = (double*)dev_alloc(c, sizeof(double) * kMomAcc * n_cells);
  c->mout = (double*)dev_alloc(c, sizeof(double) * USP_NMOM * n_cells);
  c->levsum = (double*)dev_alloc(c, sizeof(double) * n_cells);
  c->wait_cycles = kWaitCycles;
  c->tab_nb = nullptr;
  c->tab_b = nullptr;
  c->gd_nb = nullptr;
  c->gd_b = nullptr;
  if (c->precision == USP_FP32) {
    c->tab_nb = (float*)dev_alloc(c, sizeof(float) * (size_t)n_cells * kJR * kJK);
    c->tab_b = (float*)dev_alloc(c, sizeof(float) * (size_t)n_cells * kJR * kJK);
    c->gd_nb = (uint8_t*)dev_alloc(c, (size_t)n_cells * kJR * kGB);
    c->gd_b = (uint8_t*)dev_alloc(c, (size_t)n_cells * kJR * kGB);
    if (!c->tab_nb || !c->tab_b || !c->gd_nb || !c->gd_b) return fail(USP_ENOMEM);
  }
  c->flags = (uint32_t*)dev_alloc(c, 256);
  c->counters = (unsigned long long*)dev_alloc(c, 256);
  if (!c->cx || !c->cy || !c->cz || !c->er || !c->lev || !c->cells || !c->prm || !c->sums ||
      !c->uoff || !c->macc || !c->mout || !c->levsum || !c->flags || !c->counters)
    return fail(USP_ENOMEM);
  if (cfg->stream) {
    c->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      c->stream = nullptr;
      return fail(USP_ECUDA);
    }
    c->own_stream = true;
  }
  if (cudaMemsetAsync(c->cx, 0, c->nstore * es, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->cy, 0, c->nstore * es, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->cz, 0, c->nstore * es, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->er, 0, c->nstore * es, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->lev, 0, c->nstore * 4, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->sums, 0, sizeof(CellSums) * n_cells, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->flags, 0, 256, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->counters, 0, 256, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->cells, hc.data(), sizeof(CellState) * n_cells, cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->uoff, c->h_uoff.data(), sizeof(long long) * (n_cells + 1),
                      cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    return fail(USP_ECUDA);
  // the particle pass stages fixed tiles of kTileMax; smaller tiles (tests)
  // split cells more finely but use the same staging buffers
  const int tile = cfg->tile > 0 ? std::min(kTileMax, (cfg->tile + kAlign - 1) / kAlign * kAlign)
                                  : kTileMax;
  int rc = build_tiles(c, tile);
  if (rc) return fail(rc);
  {
    // persistent grid per design and register-budget variant: as many
    // resident blocks as the SMs hold (warp-tiled: no more warps than tiles)
    const bool f32 = c->precision == USP_FP32;
    for (int wt = 0; wt < 2; ++wt) {
      const size_t smem = f32 ? collide_smem<float>(wt) : collide_smem<double>(wt);
      for (int mb = 2; mb <= 4; ++mb) {
        void* fn = f32 ? collide_variant<float>(wt, mb, c->sp.method)
                       : collide_variant<double>(wt, mb, c->sp.method);
        int per_sm = 1;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, smem) != cudaSuccess)
          return fail(USP_ECUDA);
        const int units = wt ? (c->nwtiles + kWarps - 1) / kWarps : c->ntiles;
        c->grid_by_minb[wt][mb] = std::max(1, std::min(units, sm_count() * std::max(1, per_sm)));
      }
    }
    c->minb = 3;
    c->warp_tiles = 1;
    c->grid_collide = c->grid_by_minb[1][3];
  }
  if (n > 0) {
    rc = upload_state(c, h_cx, h_cy, h_cz, h_erot, h_lev, false);
    if (rc) return fail(rc);
    // the FP64 host layout of the initial upload is staged once only
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(USP_ECUDA);
    dev_release(c, c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
  }
  rc = c->precision == USP_FP32 ? init_params<float>(c) : init_params<double>(c);
  if (rc) return fail(rc);
  if (cfg->tile == 0 && n >= (1ll << 20)) {
    rc = c->precision == USP_FP32 ? autotune<float>(c) : autotune<double>(c);
    if (rc) return fail(rc);
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(USP_ECUDA);
  *out = c;
  return USP_OK;
}

int usp_init_channel(usp_ctx** out, const usp_species* sp, const usp_config* cfg,
                     const usp_channel* ch, double dt, int64_t n, const double* h_y,
                     const double* h_cx, const double* h_cy, const double* h_cz,
                     const double* h_erot, const int32_t* h_lev, const uint32_t* h_pid) {
  if (!out || !sp || !cfg || !ch) return USP_EINVAL;
  if (cfg->method != USP_METHOD_USP_FPM && cfg->method != USP_METHOD_FPM) return USP_EINVAL;
  const bool tangent = cfg->precision == USP_FP64_TANGENT || cfg->precision == USP_FP32_TANGENT;
  if (cfg->method == USP_METHOD_FPM && tangent) return USP_ENOTSUP;
  if (cfg->precision != USP_FP32 && cfg->precision != USP_FP64 && !tangent) return USP_EINVAL;
  if (!(sp->m > 0) || !(sp->d_ref > 0) || !(sp->T_ref > 0) || !(sp->c_alpha > 0) ||
      !(sp->theta_v > 0))
    return USP_EINVAL;
  *out = nullptr;
  usp_ctx* c = new usp_ctx();
  c->kind = 1;
  c->ch = nullptr;
  c->pl = nullptr;
  c->cfg = *cfg;
  c->sp = to_dev(sp);
  c->sp.method = cfg->method;
  c->precision = cfg->precision;
  c->ncell = 0;
  c->nparticles = 0;
  c->graph_exec = nullptr;
  c->graph = nullptr;
  c->graph_steps = 0;
  c->graph_parity = 0;
  c->step = cfg->step0;
  c->launches = 0;
  c->device_bytes = 0;
  c->profiling = 0;
  c->ev_used = 0;
  c->minb = 0;
  c->stage = nullptr;
  c->stage_bytes = 0;
  if (cfg->stream) {
    c->stream = (cudaStream_t)cfg->stream;
    c->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return USP_ECUDA;
    }
    c->own_stream = true;
  }
  auto fail = [&](int rc) {
    cudaStreamSynchronize(c->stream);
    if (c->ch) ch_destroy(c->ch);
    dev_free_all(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return rc;
  };
  c->flags = (uint32_t*)dev_alloc(c, 256);
  c->counters = (unsigned long long*)dev_alloc(c, 256);
  if (!c->flags || !c->counters) return fail(USP_ENOMEM);
  if (cudaMemsetAsync(c->flags, 0, 256, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->counters, 0, 256, c->stream) != cudaSuccess)
    return fail(USP_ECUDA);
  const int rc = ch_create(&c->ch, make_env(c), ch, dt, n, cfg->step0, h_y, h_cx, h_cy, h_cz,
                           h_erot, h_lev, h_pid);
  if (rc != USP_OK) return fail(rc);
  c->nparticles = ch_nparticles(c->ch);
  c->ncell = ch_ncell(c->ch);
  *out = c;
  return USP_OK;
}

int usp_init_plane(usp_ctx** out, const usp_species* sp, const usp_config* cfg,
                   const usp_plane* pl, double dt, const double* area_frac, int64_t n,
                   int64_t capacity, const double* h_x, const double* h_y, const double* h_cx,
                   const double* h_cy, const double* h_cz, const double* h_erot,
                   const int32_t* h_lev, const uint32_t* h_pid) {
  if (!out || !sp || !cfg || !pl) return USP_EINVAL;
  if (cfg->method != USP_METHOD_USP_FPM && cfg->method != USP_METHOD_FPM) return USP_EINVAL;
  if (cfg->precision != USP_FP32 && cfg->precision != USP_FP64) return USP_EINVAL;
  if (!(sp->m > 0) || !(sp->d_ref > 0) || !(sp->T_ref > 0) || !(sp->c_alpha > 0) ||
      !(sp->theta_v > 0))
    return USP_EINVAL;
  *out = nullptr;
  usp_ctx* c = new usp_ctx();
  c->kind = 2;
  c->ch = nullptr;
  c->pl = nullptr;
  c->cfg = *cfg;
  c->sp = to_dev(sp);
  c->sp.method = cfg->method;
  c->precision = cfg->precision;
  c->ncell = 0;
  c->nparticles = 0;
  c->graph_exec = nullptr;
  c->graph = nullptr;
  c->graph_steps = 0;
  c->graph_parity = 0;
  c->step = cfg->step0;
  c->launches = 0;
  c->device_bytes = 0;
  c->profiling = 0;
  c->ev_used = 0;
  c->minb = 0;
  c->stage = nullptr;
  c->stage_bytes = 0;
  if (cfg->stream) {
    c->stream = (cudaStream_t)cfg->stream;
    c->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return USP_ECUDA;
    }
    c->own_stream = true;
  }
  auto fail = [&](int rc) {
    cudaStreamSynchronize(c->stream);
    if (c->pl) pl_destroy(c->pl);
    dev_free_all(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return rc;
  };
  c->flags = (uint32_t*)dev_alloc(c, 256);
  c->counters = (unsigned long long*)dev_alloc(c, 256);
  if (!c->flags || !c->counters) return fail(USP_ENOMEM);
  if (cudaMemsetAsync(c->flags, 0, 256, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->counters, 0, 256, c->stream) != cudaSuccess)
    return fail(USP_ECUDA);
  const int rc = pl_create(&c->pl, make_env(c), pl, dt, area_frac, n, capacity, cfg->step0, h_x,
                           h_y, h_cx, h_cy, h_cz, h_erot, h_lev, h_pid);
  if (rc != USP_OK) return fail(rc);
  c->nparticles = n;
  c->ncell = pl_ncell(c->pl);
  *out = c;
  return USP_OK;
}

int usp_plane_leaves(const usp_plane* pl, int32_t* level, int32_t* ii, int32_t* jj) {
  return pl_leaves(pl, level, ii, jj);
}

int usp_plane_count(usp_ctx* c, int64_t* n, uint32_t* next_pid) {
  if (!c || c->kind != 2) return USP_EINVAL;
  return pl_count(c->pl, make_env(c), n, next_pid);
}

int usp_plane_get_particles(usp_ctx* c, int64_t cap, int64_t* n, double* x, double* y,
                            double* cx, double* cy, double* cz, double* erot, int32_t* lev,
                            uint32_t* pid) {
  if (!c || c->kind != 2) return USP_EINVAL;
  return pl_get_particles(c->pl, make_env(c), cap, n, x, y, cx, cy, cz, erot, lev, pid);
}

int usp_sample(usp_ctx* c, int on) {
  if (!c || (c->kind != 1 && c->kind != 2)) return USP_EINVAL;
  if (c->graph_exec) {  // the captured step depends on the sampling switch
    cudaGraphExecDestroy(c->graph_exec);
    cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
  }
  return c->kind == 1 ? ch_sample(c->ch, on) : pl_sample(c->pl, on);
}

int usp_channel_sample(usp_ctx* c, int on) { return usp_sample(c, on); }

int usp_sample_read(usp_ctx* c, double* h_acc, int reset) {
  if (!c || (c->kind != 1 && c->kind != 2) || !h_acc) return USP_EINVAL;
  return c->kind == 1 ? ch_read(c->ch, make_env(c), h_acc, reset)
                      : pl_read(c->pl, make_env(c), h_acc, reset);
}

int usp_channel_read(usp_ctx* c, double* h_acc, int reset) {
  return usp_sample_read(c, h_acc, reset);
}

int usp_channel_get_particles(usp_ctx* c, double* y, double* cx, double* cy, double* cz,
                              double* erot, int32_t* lev, uint32_t* pid) {
  if (!c || c->kind != 1 || !cx || !cy || !cz || !erot || !lev) return USP_EINVAL;
  return ch_get_particles(c->ch, make_env(c), y, cx, cy, cz, erot, lev, pid);
}

int usp_step(usp_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return USP_EINVAL;
  if (nsteps == 0) return USP_OK;
  if (!c->cfg.use_graph || c->profiling) {
    for (int i = 0; i < nsteps; ++i) {
      int rc = step_once(c);
      if (rc) return rc;
      c->launches += kernels_per_step(c);
    }
    c->step += nsteps;
    return USP_OK;
  }
  // The channel path alternates two particle buffers chosen on the host, so
  // its graphs hold an even number of steps and are captured at the current
  // buffer parity; an odd remainder runs eagerly.
  int G = nsteps >= 16 ? 16 : 1;
  if (c->kind != 0) G = nsteps >= 16 ? 16 : (nsteps >= 2 ? 2 : 0);
  if (G == 0) {
    int rc = step_once(c);
    if (rc) return rc;
    c->launches += kernels_per_step(c);
    c->step += nsteps;
    return USP_OK;
  }
  const int parity = c->kind == 1 ? ch_parity(c->ch) : (c->kind == 2 ? pl_parity(c->pl) : 0);
  if (!c->graph_exec || c->graph_steps != G || c->graph_parity != parity) {
    int rc = build_graph(c, G);
    if (rc) return rc;
    c->graph_parity = parity;
  }
  int done = 0;
  while (nsteps - done >= c->graph_steps) {
    CK(cudaGraphLaunch(c->graph_exec, c->stream));
    c->launches += kernels_per_step(c) * c->graph_steps;
    done += c->graph_steps;
  }
  for (; done < nsteps; ++done) {
    int rc = step_once(c);
    if (rc) return rc;
    c->launches += kernels_per_step(c);
  }
  c->step += nsteps;
  return USP_OK;
}

int usp_moments(usp_ctx* c, double* out, int out_is_device) {
  if (!c || !out) return USP_EINVAL;
  if (c->kind == 1) return ch_moments(c->ch, make_env(c), out, out_is_device);
  if (c->kind == 2) return pl_moments(c->pl, make_env(c), out, out_is_device);
  int rc = c->precision == USP_FP32 ? compute_moments<float>(c, nullptr)
                                    : compute_moments<double>(c, nullptr);
  if (rc) return rc;
  if (out_is_device) {
    CK(cudaMemcpyAsync(out, c->mout, sizeof(double) * USP_NMOM * c->ncell,
                       cudaMemcpyDeviceToDevice, c->stream));
  } else {
    CK(cudaMemcpyAsync(out, c->mout, sizeof(double) * USP_NMOM * c->ncell,
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return USP_OK;
}

int usp_get_particles(usp_ctx* c, double* hx, double* hy, double* hz, double* he, int32_t* hl) {
  if (!c || !hx || !hy || !hz || !he || !hl) return USP_EINVAL;
  if (c->kind != 0) return USP_ENOTSUP;
  const long long n = c->nparticles;
  if (n == 0) return USP_OK;
  double* st = (double*)dev_alloc(c, (size_t)n * 36 + 64);
  if (!st) return USP_ENOMEM;
  double* ox = st; double* oy = st + n; double* oz = st + 2 * n; double* oe = st + 3 * n;
  int* ol = (int*)(st + 4 * n);
  dim3 grid(64, std::min(c->ncell, 65535));
  if (c->precision == USP_FP32)
    gather_state<float><<<grid, 256, 0, c->stream>>>(c->ncell, c->cells, c->uoff,
        (const float*)c->cx, (const float*)c->cy, (const float*)c->cz, (const float*)c->er,
        c->lev, ox, oy, oz, oe, ol);
  else
    gather_state<double><<<grid, 256, 0, c->stream>>>(c->ncell, c->cells, c->uoff,
        (const double*)c->cx, (const double*)c->cy, (const double*)c->cz, (const double*)c->er,
        c->lev, ox, oy, oz, oe, ol);
  CK(cudaGetLastError());
  c->launches += 1;
  CK(cudaMemcpyAsync(hx, ox, n * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(hy, oy, n * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(hz, oz, n * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(he, oe, n * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(hl, ol, n * 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (c->cfg.alloc && c->cfg.free_) c->cfg.free_(st, c->cfg.alloc_user);
  else if (!c->cfg.alloc) cudaFree(st);
  c->owned.erase(std::find(c->owned.begin(), c->owned.end(), (void*)st));
  c->device_bytes -= (long long)(((size_t)n * 36 + 64 + 255) & ~(size_t)255);
  return USP_OK;
}

int usp_set_particles(usp_ctx* c, const double* hx, const double* hy, const double* hz,
                      const double* he, const int32_t* hl) {
  if (!c || !hx || !hy || !hz || !he || !hl) return USP_EINVAL;
  if (c->kind != 0) return USP_ENOTSUP;
  int rc = upload_state(c, hx, hy, hz, he, hl, false);
  if (rc) return rc;
  return c->precision == USP_FP32 ? init_params<float>(c) : init_params<double>(c);
}

int usp_step_host(usp_ctx* c, const void* hx, const void* hy, const void* hz, const void* he,
                  const int32_t* hl, int nsteps, double* h_moments, void* ox, void* oy, void* oz,
                  void* oe, int32_t* ol) {
  if (!c || !hx || !hy || !hz || !he || !hl || !h_moments || nsteps < 0) return USP_EINVAL;
  if (c->kind != 0) return USP_ENOTSUP;
  int rc = c->precision == USP_FP32 ? step_host_chunked<float>(c, hx, hy, hz, he, hl, nsteps)
                                    : step_host_chunked<double>(c, hx, hy, hz, he, hl, nsteps);
  if (rc) return rc;
  CK(cudaMemcpyAsync(h_moments, c->mout, sizeof(double) * USP_NMOM * c->ncell,
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (ox && oy && oz && oe && ol) {
    const long long n = c->nparticles;
    const size_t es = c->precision == USP_FP32 ? 4 : 8;
    void* st = staging(c, (size_t)n * (4 * es + 4) + 64);
    if (!st) return USP_ENOMEM;
    char* p = (char*)st;
    dim3 grid(64, std::min(c->ncell, 65535));
    if (c->precision == USP_FP32)
      gather_state_native<float><<<grid, 256, 0, c->stream>>>(c->ncell, c->cells, c->uoff,
          (const float*)c->cx, (const float*)c->cy, (const float*)c->cz, (const float*)c->er,
          c->lev, (float*)p, (float*)(p + n * es), (float*)(p + 2 * n * es),
          (float*)(p + 3 * n * es), (int*)(p + 4 * n * es));
    else
      gather_state_native<double><<<grid, 256, 0, c->stream>>>(c->ncell, c->cells, c->uoff,
          (const double*)c->cx, (const double*)c->cy, (const double*)c->cz, (const double*)c->er,
          c->lev, (double*)p, (double*)(p + n * es), (double*)(p + 2 * n * es),
          (double*)(p + 3 * n * es), (int*)(p + 4 * n * es));
    CK(cudaGetLastError());
    c->launches += 1;
    CK(cudaMemcpyAsync(ox, p, n * es, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(oy, p + n * es, n * es, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(oz, p + 2 * n * es, n * es, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(oe, p + 3 * n * es, n * es, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(ol, p + 4 * n * es, n * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return USP_OK;
}

int usp_profiles(usp_ctx* c, double* out, int out_is_device) {
  if (!c || c->kind != 1 || !out) return USP_EINVAL;
  return ch_profiles(c->ch, make_env(c), out, out_is_device);
}

int usp_backward(usp_ctx* c, const double* d_dL, double* grad3, int grad_is_device) {
  if (!c || !d_dL || !grad3) return USP_EINVAL;
  if (c->kind != 1 || (c->precision != USP_FP64_TANGENT && c->precision != USP_FP32_TANGENT))
    return USP_ENOTSUP;
  return ch_backward(c->ch, make_env(c), d_dL, grad3, grad_is_device);
}

// ---------------------------------------------------------------------------
// Checkpoints: a header that identifies the context, the status word and
// counters, then the kind's own device buffers in a fixed order.
// ---------------------------------------------------------------------------
struct CkptHeader {
  uint32_t magic, version;
  int32_t kind, precision, method, sampling;
  int64_t n, ncell, step;
  uint64_t seed, payload;
};
constexpr uint32_t kCkptMagic = 0x43505355u;   // "USPC"
constexpr size_t kCkptStatus = 4 + 8 * NCOUNTERS;

// homogeneous contexts: particles (storage order), cell records, the
// parameters and jump tables of the coming step, the cell sums
int homog_segments(usp_ctx* c, void** ptr, size_t* bytes) {
  const size_t es = c->precision == USP_FP32 ? 4 : 8;
  const size_t pb = c->precision == USP_FP32 ? sizeof(CollideParams<float>)
                                             : sizeof(CollideParams<double>);
  int k = 0;
  ptr[k] = c->cx; bytes[k++] = c->nstore * es;
  ptr[k] = c->cy; bytes[k++] = c->nstore * es;
  ptr[k] = c->cz; bytes[k++] = c->nstore * es;
  ptr[k] = c->er; bytes[k++] = c->nstore * es;
  ptr[k] = c->lev; bytes[k++] = c->nstore * 4;
  ptr[k] = c->cells; bytes[k++] = sizeof(CellState) * c->ncell;
  ptr[k] = c->prm; bytes[k++] = pb * c->ncell;
  ptr[k] = c->sums; bytes[k++] = sizeof(CellSums) * c->ncell;
  if (c->tab_nb) {
    ptr[k] = c->tab_nb; bytes[k++] = sizeof(float) * (size_t)c->ncell * kJR * kJK;
    ptr[k] = c->tab_b; bytes[k++] = sizeof(float) * (size_t)c->ncell * kJR * kJK;
    ptr[k] = c->gd_nb; bytes[k++] = (size_t)c->ncell * kJR * kGB;
    ptr[k] = c->gd_b; bytes[k++] = (size_t)c->ncell * kJR * kGB;
  }
  return k;
}

size_t ckpt_payload(usp_ctx* c) {
  if (c->kind == 1) return ch_ckpt_bytes(c->ch);
  void* p[16];
  size_t b[16], t = 0;
  const int k = homog_segments(c, p, b);
  for (int i = 0; i < k; ++i) t += b[i];
  return t;
}

CkptHeader ckpt_header(usp_ctx* c) {
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  h.magic = kCkptMagic;
  h.version = 1;
  h.kind = c->kind;
  h.precision = c->precision;
  h.method = c->sp.method;
  h.sampling = c->kind == 1 ? ch_sampling(c->ch) : 0;
  h.n = c->kind == 1 ? ch_nparticles(c->ch) : c->nparticles;
  h.ncell = c->kind == 1 ? ch_ncell(c->ch) : c->ncell;
  h.step = c->step;
  h.seed = c->cfg.seed;
  h.payload = ckpt_payload(c);
  return h;
}

int usp_checkpoint_bytes(usp_ctx* c, size_t* bytes) {
  if (!c || !bytes) return USP_EINVAL;
  if (c->kind == 2) return USP_ENOTSUP;
  *bytes = sizeof(CkptHeader) + kCkptStatus + ckpt_payload(c);
  return USP_OK;
}

int usp_save(usp_ctx* c, void* buf, int buf_is_device) {
  if (!c || !buf) return USP_EINVAL;
  if (c->kind == 2) return USP_ENOTSUP;
  const CkptHeader h = ckpt_header(c);
  unsigned char* b = (unsigned char*)buf;
  const cudaMemcpyKind d2b = buf_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (buf_is_device) {
    CK(cudaMemcpyAsync(b, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
    // the header lives on the host stack: complete its copy before returning
    CK(cudaStreamSynchronize(c->stream));
  } else {
    std::memcpy(b, &h, sizeof(h));
  }
  b += sizeof(h);
  CK(cudaMemcpyAsync(b, c->flags, 4, d2b, c->stream));
  CK(cudaMemcpyAsync(b + 4, c->counters, 8 * NCOUNTERS, d2b, c->stream));
  b += kCkptStatus;
  if (c->kind == 1) {
    const int rc = ch_ckpt_copy(c->ch, make_env(c), b, buf_is_device, 1);
    if (rc) return rc;
  } else {
    void* p[16];
    size_t sz[16];
    const int k = homog_segments(c, p, sz);
    for (int i = 0; i < k; ++i) {
      CK(cudaMemcpyAsync(b, p[i], sz[i], d2b, c->stream));
      b += sz[i];
    }
  }
  if (!buf_is_device) CK(cudaStreamSynchronize(c->stream));
  return USP_OK;
}

int usp_load(usp_ctx* c, const void* buf, int buf_is_device) {
  if (!c || !buf) return USP_EINVAL;
  if (c->kind == 2) return USP_ENOTSUP;
  CkptHeader h;
  const unsigned char* b = (const unsigned char*)buf;
  if (buf_is_device) {
    CK(cudaMemcpyAsync(&h, b, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  } else {
    std::memcpy(&h, b, sizeof(h));
  }
  const CkptHeader mine = ckpt_header(c);
  if (h.magic != kCkptMagic || h.version != mine.version || h.kind != mine.kind ||
      h.precision != mine.precision || h.method != mine.method || h.n != mine.n ||
      h.ncell != mine.ncell || h.seed != mine.seed || h.payload != mine.payload)
    return USP_EINVAL;
  // a captured graph replays the step of the state it was captured with
  CK(cudaStreamSynchronize(c->stream));
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
  }
  const cudaMemcpyKind b2d = buf_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  b += sizeof(h);
  CK(cudaMemcpyAsync(c->flags, b, 4, b2d, c->stream));
  CK(cudaMemcpyAsync(c->counters, b + 4, 8 * NCOUNTERS, b2d, c->stream));
  b += kCkptStatus;
  if (c->kind == 1) {
    const int rc = ch_ckpt_copy(c->ch, make_env(c), const_cast<unsigned char*>(b),
                                buf_is_device, 0);
    if (rc) return rc;
    ch_sample(c->ch, h.sampling);
  } else {
    void* p[16];
    size_t sz[16];
    const int k = homog_segments(c, p, sz);
    for (int i = 0; i < k; ++i) {
      CK(cudaMemcpyAsync(p[i], b, sz[i], b2d, c->stream));
      b += sz[i];
    }
  }
  c->step = h.step;
  CK(cudaStreamSynchronize(c->stream));
  return USP_OK;
}

int usp_status(usp_ctx* c, uint32_t* flags, int64_t* counters, int reset) {
  if (!c) return USP_EINVAL;
  uint32_t f = 0;
  unsigned long long cnt[NCOUNTERS];
  CK(cudaMemcpyAsync(&f, c->flags, 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (flags) *flags = f;
  if (counters)
    for (int i = 0; i < NCOUNTERS; ++i) counters[i] = (int64_t)cnt[i];
  if (reset) {
    CK(cudaMemsetAsync(c->flags, 0, 256, c->stream));
    CK(cudaMemsetAsync(c->counters, 0, 256, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  const uint32_t err = F_A_NONPOS | F_SAMPLER_UNDERFLOW | F_BOUNDS | F_CAPACITY | F_WAIT_TIMEOUT;
  return (f & err) ? USP_EDEVICE : USP_OK;
}

int usp_guide_row(const float* row, int n_flip, uint8_t* guide) {
  if (!row || !guide || n_flip < -1 || n_flip >= kJR) return USP_EINVAL;
  if (n_flip >= 0 && !(row[n_flip] == INFINITY)) return USP_EINVAL;
  uint32_t w[kGB / 4];
  for (int q = 0; q < kGP; ++q) guide_part(row, reinterpret_cast<uint8_t*>(w), q, n_flip);
  std::memcpy(guide, w, kGB);
  return USP_OK;
}

int usp_set_wait_limit(usp_ctx* c, int64_t cycles) {
  if (!c || cycles < 0) return USP_EINVAL;
  if (c->kind != 0) return USP_ENOTSUP;
  CK(cudaStreamSynchronize(c->stream));
  if (c->graph_exec) {  // the captured launches carry the old limit
    cudaGraphExecDestroy(c->graph_exec);
    cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
  }
  c->wait_cycles = cycles == 0 ? kWaitCycles : (long long)cycles;
  return USP_OK;
}

int usp_wait_check(usp_ctx* c, int64_t cycles) {
  if (!c || cycles <= 0 || cycles > kWaitCycles) return USP_EINVAL;
  wait_check_kernel<<<1, 32, 0, c->stream>>>((long long)cycles, c->flags);
  CK(cudaGetLastError());
  c->launches += 1;
  return USP_OK;
}

int usp_sync(usp_ctx* c) {
  if (!c) return USP_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  return USP_OK;
}

int usp_info(usp_ctx* c, int64_t* np, int* nc, int* prec, int64_t* step, int* tile,
             int64_t* bytes) {
  if (!c) return USP_EINVAL;
  if (np) {
    if (c->kind == 2) {
      const int rc = pl_count(c->pl, make_env(c), np, nullptr);
      if (rc) return rc;
    } else {
      *np = c->kind == 1 ? ch_nparticles(c->ch) : c->nparticles;
    }
  }
  if (nc) *nc = c->kind == 1 ? ch_ncell(c->ch) : (c->kind == 2 ? pl_ncell(c->pl) : c->ncell);
  if (prec) *prec = c->precision;
  if (step) *step = c->step;
  if (tile) *tile = c->tile;
  if (bytes) *bytes = c->device_bytes;
  return USP_OK;
}

int64_t usp_launch_count(usp_ctx* c) { return c ? c->launches : -1; }

int usp_tuning(usp_ctx* c, int* warp_tiles, int* blocks_per_sm, double* ms) {
  if (!c) return USP_EINVAL;
  const bool homog = c->kind == 0;
  if (warp_tiles) *warp_tiles = homog ? c->warp_tiles : 0;
  if (blocks_per_sm) *blocks_per_sm = homog ? c->minb : 0;
  if (ms)
    for (int i = 0; i < 6; ++i) ms[i] = homog && i < (int)c->tune_ms.size() ? c->tune_ms[i] : 0.0;
  return USP_OK;
}

int usp_set_variant(usp_ctx* c, int warp_tiles, int blocks_per_sm) {
  if (!c || c->kind != 0 || (warp_tiles != 0 && warp_tiles != 1) || blocks_per_sm < 2 ||
      blocks_per_sm > 4)
    return USP_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  if (c->graph_exec) {  // the captured step launches the previous variant
    cudaGraphExecDestroy(c->graph_exec);
    cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
  }
  c->warp_tiles = warp_tiles;
  c->minb = blocks_per_sm;
  c->grid_collide = c->grid_by_minb[warp_tiles][blocks_per_sm];
  return USP_OK;
}

int usp_profile_enable(usp_ctx* c, int on) {
  if (!c) return USP_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  c->profiling = on ? 1 : 0;
  c->ev_used = 0;
  c->ev_kind.clear();
  return USP_OK;
}

int usp_profile_read(usp_ctx* c, double* ms, int64_t* launches) {
  if (!c || !ms || !launches) return USP_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  ms[0] = ms[1] = 0.0;
  launches[0] = launches[1] = 0;
  for (size_t i = 0; i < c->ev_kind.size(); ++i) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]));
    const int k = c->ev_kind[i];
    if (k >= 0 && k < 2) {
      ms[k] += t;
      launches[k] += 1;
    }
  }
  return USP_OK;
}

void usp_destroy(usp_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    cudaGraphDestroy(c->graph);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->ch) ch_destroy(c->ch);
  if (c->pl) pl_destroy(c->pl);
  if (c->copy_stream) {
    cudaStreamDestroy(c->copy_stream);
    for (cudaEvent_t e : c->up_ev) cudaEventDestroy(e);
  }
  dev_free_all(c);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // extern "C"
