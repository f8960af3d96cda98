// Host-side entry points of the device passes (step, geometry, reductions).
#pragma once

#include <cuda_runtime.h>

#include "context.hpp"

namespace lbm {

// One time step: the seven passes of step.cu on stream s. `macros` also
// stores rho and u of this step.
void launch_step(int Q, int storage, const Dom &d, cudaStream_t s,
                 bool macros);

// The same step with an event recorded before each of its kernels and after
// the last (ev[0..7], the slots of lbm_step_timed); kernels that do not run
// (no Zou-He planes, no solid-boundary nodes) get back-to-back events.
void launch_step_events(int Q, int storage, const Dom &d, cudaStream_t s,
                        bool macros, cudaEvent_t *ev);

// The passes of a step before the collision (stream, Zou-He fix-up, Eq. 34,
// gradient and wetting, Eq. 35) on the current state: fills U, R, the
// phase fields and the normals without changing the state.
void launch_fields(int Q, int storage, const Dom &d, cudaStream_t s);

// Geometry set-up (geometry.cu): classes, the compact lists and the map,
// Eq. (25) smoothing, Eq. (26) normals and the counts.
cudaError_t build_geometry(lbm_ctx *c, cudaStream_t s);

// f^s_i = w_i rho^s at fluid nodes, phi and the macros of the initial
// state (geometry.cu).
void launch_init_state(int Q, int storage, const Dom &d, const float *phi0,
                       cudaStream_t s);

// Eqs. (37)-(38) at the inlet plane's fluid nodes: the stored state becomes
// pure colour b (blue) or r (geometry.cu).
void launch_swap_inlet(const Dom &d, bool blue, cudaStream_t s);

// Dense float32 export/import of the stored populations (geometry.cu).
void launch_export_pops(int Q, int storage, const Dom &d, float *dst,
                        cudaStream_t s);
void launch_import_pops(int Q, int storage, const Dom &d, const float *src,
                        cudaStream_t s);

// Wall normals as float32 [3][N] (geometry.cu).
void launch_export_nw(const Dom &d, float *out, cudaStream_t s);

// Dense rho [N], phi [N], u [3][N] of the last macro step (geometry.cu);
// any pointer may be null.
void launch_export_macros(const Dom &d, float *rho, float *phi, float *u,
                          cudaStream_t s);

// FP64 reductions (reduce.cu): the result lands in *out_dev.
void launch_reduce(int Q, int storage, const Dom &d, int kind, double *partials,
                   int slots, double *out_dev, cudaStream_t s);

}  // namespace lbm
