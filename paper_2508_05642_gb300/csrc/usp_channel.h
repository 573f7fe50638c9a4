// usp_channel.h -- internal interface between the C ABI (usp_homog.cu) and
// the 1D channel (spatial) path (usp_channel.cu).  Not installed.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/usp.h"
#include "usp_device.cuh"

// What the channel path needs from its owning context.
struct ChEnv {
  cudaStream_t stream;
  uint32_t* flags;
  unsigned long long* counters;
  usp::Species sp;
  uint32_t k0, k1;            // Philox key
  int precision;              // USP_FP32 or USP_FP64
  void* (*alloc)(void* owner, size_t bytes);   // owner-tracked device allocation
  void (*release)(void* owner, void* p);       // give an allocation back early
  void* owner;
};

struct ChannelCtx;

int ch_create(ChannelCtx** out, const ChEnv& env, const usp_channel* chp, double dt, int64_t n,
              int64_t step0, const double* y, const double* cx, const double* cy,
              const double* cz, const double* erot, const int32_t* lev, const uint32_t* pid);
// enqueue one step (capturable in a CUDA graph); kind = kernel kind for
// profiling (0 particle passes, 1 per-cell passes) is reported through prof()
typedef int (*ch_prof_fn)(void* owner, int kind, int begin);
int ch_launch_step(ChannelCtx* ch, const ChEnv& env, ch_prof_fn prof);
int ch_kernels_per_step(const ChannelCtx* ch);
int ch_moments(ChannelCtx* ch, const ChEnv& env, double* out, int out_is_device);
int ch_sample(ChannelCtx* ch, int on);
int ch_read(ChannelCtx* ch, const ChEnv& env, double* h_acc, int reset);
int ch_get_particles(ChannelCtx* ch, const ChEnv& env, double* y, double* cx, double* cy,
                     double* cz, double* erot, int32_t* lev, uint32_t* pid);
// time-averaged profiles (and their derivatives in the gradient form) and the
// device-side contraction of their derivatives with an objective's gradient
int ch_profiles(ChannelCtx* ch, const ChEnv& env, double* out, int out_is_device);
int ch_backward(ChannelCtx* ch, const ChEnv& env, const double* dL, double* grad3,
                int grad_is_device);
// checkpoint payload: size, and copy to (save = 1) or from (save = 0) buf
size_t ch_ckpt_bytes(ChannelCtx* ch);
int ch_ckpt_copy(ChannelCtx* ch, const ChEnv& env, unsigned char* buf, int buf_is_device,
                 int save);
int ch_sampling(const ChannelCtx* ch);
int ch_ncell(const ChannelCtx* ch);
// which of the two particle buffers holds the state (steps alternate them)
int ch_parity(const ChannelCtx* ch);
long long ch_nparticles(const ChannelCtx* ch);
void ch_destroy(ChannelCtx* ch);
