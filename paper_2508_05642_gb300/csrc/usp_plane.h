// usp_plane.h -- internal interface between the C ABI (usp_homog.cu) and the
// 2D plane path (usp_plane.cu): flow past a circular cylinder with freestream
// inflow.  Not installed.
#pragma once

#include <cstdint>

#include "usp_channel.h"

struct PlaneCtx;

int pl_create(PlaneCtx** out, const ChEnv& env, const usp_plane* pp, double dt,
              const double* area_frac, int64_t n, int64_t cap, int64_t step0, const double* x,
              const double* y, const double* cx, const double* cy, const double* cz,
              const double* erot, const int32_t* lev, const uint32_t* pid);
// enqueue one step (capturable in a CUDA graph: the particle count lives on
// the device)
int pl_launch_step(PlaneCtx* pl, const ChEnv& env, ch_prof_fn prof);
int pl_kernels_per_step(const PlaneCtx* pl);
int pl_moments(PlaneCtx* pl, const ChEnv& env, double* out, int out_is_device);
int pl_sample(PlaneCtx* pl, int on);
int pl_read(PlaneCtx* pl, const ChEnv& env, double* h_acc, int reset);
// live particle count and the id the next injected particle gets (syncs)
int pl_count(PlaneCtx* pl, const ChEnv& env, int64_t* n, uint32_t* next_pid);
int pl_get_particles(PlaneCtx* pl, const ChEnv& env, int64_t cap, int64_t* n, double* x,
                     double* y, double* cx, double* cy, double* cz, double* erot, int32_t* lev,
                     uint32_t* pid);
int pl_ncell(const PlaneCtx* pl);
// cells of a plane's grid (count or USP_EINVAL; arrays may be NULL); host only
int pl_leaves(const usp_plane* pp, int32_t* level, int32_t* ii, int32_t* jj);
int pl_parity(const PlaneCtx* pl);
void pl_destroy(PlaneCtx* pl);
