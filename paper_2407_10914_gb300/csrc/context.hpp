// Internal state of one domain and the kernel-argument block shared by the
// step, geometry and reduction translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/lbmgb.h"

namespace lbm {

enum : uint8_t {
  CLS_SOLID = LBM_CLS_SOLID,
  CLS_SOLID_BND = LBM_CLS_SOLID_BND,
  CLS_FLUID = LBM_CLS_FLUID,
  CLS_FLUID_BND = LBM_CLS_FLUID_BND
};

// Constants of the step as the kernels use them (float, precomputed).
struct StepConst {
  float nu_r, nu_b;        // kinematic viscosities
  float gamma, beta, rho0;
  float cos_t, sin_t, theta;
  int wetting, zou_he, axis;
  float rho_in_r, rho_in_b, rho_out;  // rho_in zeta^s, rho_out
  float phi_in;                       // zeta^r - zeta^b
  float g[3];
};

// Everything a kernel needs, passed by value.
struct Dom {
  int nx, ny, nz;
  long long N;         // nodes
  long long Np;        // padded stride of one population plane
  unsigned periodic;
  // populations: fp32 [2][Q][Np] or, for 16-bit storage, two planes of
  // [Q][Np] 16-bit values (T, D)
  void *f_src;
  void *f_dst;
  float *phi;          // [N]
  float4 *nc;          // [N] (n_c, |C|); at solid-boundary nodes (Eq. 35, 0)
  const uint8_t *cls;  // [N]
  const float4 *nw;    // [N] wall normal at fluid-boundary nodes
  const int *sbnd;     // solid-boundary node list
  int n_sbnd;
  float *rho_m;        // [N] macros of the last step
  float *u_m;          // [3][N]
  StepConst c;
};

}  // namespace lbm

struct lbm_ctx {
  int Q = 0;
  int nx = 0, ny = 0, nz = 0;
  long long N = 0, Np = 0;
  unsigned periodic = 0;
  int storage = 0;
  long long n_fluid = 0, n_sbnd = 0, n_fbnd = 0;
  bool params_set = false;
  bool state_set = false;
  lbm_params p{};
  lbm::Dom d{};
  void *fA = nullptr, *fB = nullptr;  // population buffers (current = fA)
  uint8_t *mask = nullptr;            // device copy of the solid image
  double *g0 = nullptr, *g1 = nullptr;  // smoothing ping-pong (init only)
  double *red = nullptr;              // reduction partials
  double *red_out = nullptr;          // 4 doubles: the combined partials
  int red_slots = 0;
  unsigned long long *counters = nullptr;  // device counters
  char err[256] = {0};
};
