// usp_noalloc.cu -- per-cell moments of a caller-owned particle state with no
// device allocation at all.
//
// Some callers cannot let a library allocate device memory: frameworks that
// carve all device memory out of their own pool at start-up and forbid any
// later cudaMalloc, code that must not trigger the implicit device
// synchronisation cudaMalloc/cudaFree can cause in the middle of a time step,
// or hosts running under a hard device-memory budget.  usp_moments_noalloc
// serves them: it computes the same per-cell moments as usp_moments, but its
// working space (the FP64 per-cell accumulators) lives in the file-scope
// device array below, of fixed size, kept on each device until the process
// exits.  With CUDA's lazy module loading (the default), the array is
// reserved on a device when the library's module is first loaded there,
// which is at the first call on that device at the latest (that call also
// looks up the array's address): a caller that must not see any reservation
// inside its time loop makes one warm-up call at start-up, or sets
// CUDA_MODULE_LOADING=EAGER.  The address looked up at a device's first call
// is kept, so a cudaDeviceReset between calls is not supported.  The caller
// passes the inputs and the output buffer.
//
// Every call shares that one array and leaves its last contents there: each
// call clears it first on the caller's stream.  Two calls whose work overlaps
// on the GPU (for instance on two streams at once) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/usp.h"

// Scratch: 20 FP64 sums for each of up to USP_NOALLOC_MAX_CELLS cells
// (20 x 8192 x 8 B = 1.25 MiB on every device that loads the library).
static __device__ __align__(256) double g_na_scratch[20 * USP_NOALLOC_MAX_CELLS];

namespace {

constexpr int kNaAcc = 20;     // accumulators per cell
constexpr int kNaBlock = 256;
constexpr double kNaKB = 1.380649e-23;  // Boltzmann constant [J/K]

// what the moments need of the species: R = k_B / m and Theta_vib
struct NaGas {
  double R, theta_v;
};

// temperature whose e_vib = R Theta / (exp(Theta/T) - 1) equals R Theta ebar
__device__ __forceinline__ double na_T_vib(const NaGas& g, double ebar) {
  if (ebar <= 0.0) return 0.0;
  return g.theta_v / log1p(1.0 / ebar);
}

// Device address of g_na_scratch, looked up once per device (host code may
// not use the symbol itself as a device pointer).
constexpr int kMaxDevices = 64;
double* g_na_ptr[kMaxDevices] = {nullptr};
std::mutex g_na_mutex;

__global__ void na_clear(double* acc, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    acc[i] = 0.0;
}

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// pass 0: sum c, sum eps, sum I; pass 1: central sums about the cell mean.
// acc layout per cell: [0..2] sum c, [3] sum eps, [4] sum I, [5..10] sum CC,
// [11..13] sum C^2 C / 2, [14..16] sum C eps, [17..19] sum C I.
__global__ void __launch_bounds__(kNaBlock)
na_pass(int pass, int ncell, const int64_t* __restrict__ off, const double* __restrict__ cx,
        const double* __restrict__ cy, const double* __restrict__ cz,
        const double* __restrict__ er, const int32_t* __restrict__ lev, double* __restrict__ acc) {
  __shared__ double red[kNaBlock / 32][15];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = blockIdx.y; c < ncell; c += gridDim.y) {
    const long long b = off[c], e = off[c + 1];
    const double N = (double)(e - b);
    double mean[3] = {0.0, 0.0, 0.0};
    if (pass == 1 && N > 0.0)
      for (int i = 0; i < 3; ++i) mean[i] = acc[(size_t)c * kNaAcc + i] / N;
    double a[15];
    for (int i = 0; i < 15; ++i) a[i] = 0.0;
    for (long long k = b + (long long)blockIdx.x * blockDim.x + threadIdx.x; k < e;
         k += (long long)gridDim.x * blockDim.x) {
      const double ep = er[k], li = (double)lev[k];
      if (pass == 0) {
        a[0] += cx[k]; a[1] += cy[k]; a[2] += cz[k]; a[3] += ep; a[4] += li;
      } else {
        const double C0 = cx[k] - mean[0], C1 = cy[k] - mean[1], C2 = cz[k] - mean[2];
        const double q = 0.5 * (C0 * C0 + C1 * C1 + C2 * C2);
        a[0] += C0 * C0; a[1] += C1 * C1; a[2] += C2 * C2;
        a[3] += C0 * C1; a[4] += C0 * C2; a[5] += C1 * C2;
        a[6] += q * C0; a[7] += q * C1; a[8] += q * C2;
        a[9] += C0 * ep; a[10] += C1 * ep; a[11] += C2 * ep;
        a[12] += C0 * li; a[13] += C1 * li; a[14] += C2 * li;
      }
    }
    const int na = pass == 0 ? 5 : 15;
    for (int i = 0; i < na; ++i) {
      const double s = na_warp_sum(a[i]);
      if (lane == 0) red[wid][i] = s;
    }
    __syncthreads();
    if (threadIdx.x < na) {
      double s = 0.0;
      for (int w = 0; w < kNaBlock / 32; ++w) s += red[w][threadIdx.x];
      atomicAdd(&acc[(size_t)c * kNaAcc + (pass == 0 ? 0 : 5) + threadIdx.x], s);
    }
    __syncthreads();
  }
}

__global__ void na_assemble(NaGas gas, int ncell, const int64_t* __restrict__ off,
                            const double* __restrict__ acc, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const double R = gas.R;
  const double N = (double)(off[c + 1] - off[c]);
  const double* a = acc + (size_t)c * kNaAcc;
  if (N <= 0.0) {
    for (int f = 0; f < USP_NMOM; ++f) out[(size_t)f * ncell + c] = 0.0;
    return;
  }
  const double inv = 1.0 / N;
  out[c] = N;
  for (int i = 0; i < 3; ++i) out[(size_t)(1 + i) * ncell + c] = a[i] * inv;
  out[(size_t)4 * ncell + c] = (a[5] + a[6] + a[7]) * inv / (3.0 * R);
  out[(size_t)5 * ncell + c] = a[3] * inv / R;
  out[(size_t)6 * ncell + c] = na_T_vib(gas, a[4] * inv);
  for (int i = 0; i < 6; ++i) out[(size_t)(7 + i) * ncell + c] = a[5 + i] * inv;
  for (int i = 0; i < 3; ++i) {
    out[(size_t)(13 + i) * ncell + c] = a[11 + i] * inv;
    out[(size_t)(16 + i) * ncell + c] = a[14 + i] * inv;
    out[(size_t)(19 + i) * ncell + c] = a[17 + i] * inv * R * gas.theta_v;
  }
}

// Look up the device address of the scratch array for the current device,
// once per device.
int na_scratch_for_current_device(double** ptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return USP_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return USP_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return USP_ECUDA;
    g_na_ptr[dev] = (double*)p;
  }
  *ptr = g_na_ptr[dev];
  return USP_OK;
}

}  // namespace

extern "C" int usp_moments_noalloc(const usp_species* sp, int n_cells, const int64_t* d_offsets,
                                   const double* d_cx, const double* d_cy, const double* d_cz,
                                   const double* d_erot, const int32_t* d_lev, double* d_out,
                                   void* stream) {
  if (!sp || !d_offsets || !d_out || n_cells <= 0) return USP_EINVAL;
  if (n_cells > USP_NOALLOC_MAX_CELLS) return USP_EINVAL;
  if (!d_cx || !d_cy || !d_cz || !d_erot || !d_lev) return USP_EINVAL;
  if (!(sp->m > 0.0) || !(sp->theta_v > 0.0)) return USP_EINVAL;
  double* acc = nullptr;
  const int rc = na_scratch_for_current_device(&acc);
  if (rc != USP_OK) return rc;
  NaGas gas;
  gas.R = kNaKB / sp->m;
  gas.theta_v = sp->theta_v;
  cudaStream_t st = (cudaStream_t)stream;
  // an error left by the caller's earlier work is not this call's: report it
  // without launching (and without clearing it)
  if (cudaPeekAtLastError() != cudaSuccess) return USP_ECUDA;
  const int nacc = kNaAcc * n_cells;
  na_clear<<<(nacc + 255) / 256, 256, 0, st>>>(acc, nacc);
  if (cudaGetLastError() != cudaSuccess) return USP_ECUDA;
  const dim3 grid(8, n_cells < 65535 ? n_cells : 65535);
  for (int pass = 0; pass < 2; ++pass) {
    na_pass<<<grid, kNaBlock, 0, st>>>(pass, n_cells, d_offsets, d_cx, d_cy, d_cz, d_erot,
                                       d_lev, acc);
    if (cudaGetLastError() != cudaSuccess) return USP_ECUDA;
  }
  na_assemble<<<(n_cells + 127) / 128, 128, 0, st>>>(gas, n_cells, d_offsets, acc, d_out);
  if (cudaGetLastError() != cudaSuccess) return USP_ECUDA;
  return USP_OK;
}
