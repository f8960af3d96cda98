// Internal state of one domain and the kernel-argument block shared by the
// step, geometry and reduction translation units.
//
// Memory layout (all inside the caller's workspace):
//  * the box is cut into tiles (tiles.cuh); a uint16 map over the box holds,
//    per node, its class (bits 14-15) and its rank among the nodes of the
//    same kind (fluid, or solid-boundary) in its tile (bits 0-13); per-tile
//    bases turn (tile, rank) into an index of the compact fluid list
//    ("F-space", tile by tile) or solid-boundary list ("S-space");
//  * populations live in F-space only, in the post-recolouring form that
//    Eqs. (20)-(21) give them: f''_i = f^r'_i + f^b'_i per direction (Q
//    planes) plus one float4 per node (q, v): q the encoded colour split
//    (as the phase field below) and v = beta rho^r rho^b / rho n,
//    from which f^r'_i and f^b'_i are rebuilt exactly;
//  * the phase field is stored "encoded": m = min(rho^r,rho^b)/rho (signed:
//    a colour density can overshoot slightly below zero) with the majority
//    colour in the lowest mantissa bit, so that phi - sign(phi) keeps
//    float32 relative accuracy near the pure phases (the colour gradient of
//    Eq. 6 is built from it).
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
  float nu_r, nu_b;  // kinematic viscosities
  float h_r, h_b;    // 1 / (2 nu^r), 1 / (2 nu^b) (Eq. 14's halves)
  float gamma, beta, rho0;
  float cos_t, sin_t;
  int wetting, zou_he, axis;
  float rho_in_r, rho_in_b, rho_out;  // rho_in zeta^s, rho_out
  float m_in;                          // encoded inlet phase field
  float g[3];
  int mrt;  // 1: Eq. 2 with the rates of Eqs. 4, 15-16 (D3Q19)
};

// Everything a kernel needs, passed by value.
struct Dom {
  int nx, ny, nz;
  long long N;      // nodes of the box
  unsigned periodic;
  int ntx, nty, ntz;  // tiles per axis
  int ntiles;
  int NF, NS;       // fluid nodes, solid-boundary nodes
  long long NFp;    // stride of one population plane (NF rounded up)
  const uint16_t *map;  // [N]
  const int *fbase;     // [ntiles + 1]
  const int *sbase;     // [ntiles + 1]
  const int *fg;        // [NF] box index of fluid node k
  const int *sg;        // [NS] box index of solid-boundary node j
  const uint8_t *cls;   // [N]
  // lattice-neighbour entries over the padded box (strides px, py): the
  // cell at padded position x + 1 holds class << 30 | OUT << 29 | index of
  // the node x reaches, after wrapping the periodic axes and clamping the
  // others (OUT set where it clamped); a fluid node reads its neighbours at
  // its padded index plus a fixed offset per direction (see tiles.cuh)
  const uint32_t *nbd;  // [(nx + 2)(ny + 2)(nz + 2)]
  // fluid lattice neighbours of the solid-boundary nodes (the terms of
  // Eqs. 34-35), node j's at [soff[j], soff[j+1]): F-index, bit 31 set for
  // a diagonal direction (weight w_diag instead of w_axis)
  const int *soff;         // [NS + 1]
  const uint32_t *slink;
  const uint8_t *fflag; // [NF] bit 0 fluid-boundary; bit 1+2a / 2+2a: on the
                        // first / last plane along axis a
  const int *zh_list;   // fluid nodes of the two Zou-He planes of the axis
  int n_zh;
  const float4 *nw;     // [NF] wall normal (fluid-boundary nodes), else 0
  const void *T_src;    // [Q][NFp] f'' (float32, or 16-bit offsets)
  void *T_dst;
  void *U;              // [Q][NFp] f^t after streaming and App. B (as T)
  float2 *R;            // [NF] (rho^r, rho^b) after streaming and App. B
  const float4 *S_src;  // [NF] (q, v)
  float4 *S_dst;
  float *mf;            // [NF] encoded phase field
  float *ms;            // [NS] encoded phase field (Eq. 34)
  float4 *ncf;          // [NF] (n_c, |C|)
  float *kap;           // [NF] curvature of Eq. (12), for the collision
  float4 *ncs;          // [NS] (n_c of Eq. 35, 0)
  float4 *macro;        // [NF] (u_x, u_y, u_z, rho) of the last macro step
  // the phase field again as a dense box with a one-node halo (padded
  // strides px = nx + 2, py = ny + 2): the gradient stencil reads it at the
  // node's padded index plus a fixed offset per direction, with no
  // neighbour-table entry (dense_store keeps the halo)
  float *phib;          // [(nx + 2)(ny + 2)(nz + 2)]
  const int *fgp;       // [NF] padded box index of fluid node k
  const int *sgp;       // [NS] padded box index of solid-boundary node j
  const uint8_t *sflag; // [NS] face bits as fflag (bits 1 + 2a, 2 + 2a)
  // [NS] bit i set when x + e_i of solid-boundary node j is a fluid node:
  // the directions of its links, so that Eq. 34 reads the dense box
  const uint32_t *sdir;
  int px, py;
  unsigned *err;        // error word of the bounds-checked build (guard())
  StepConst c;
  int tlx, tly, tlz;    // log2 of the tile extents (set-up kernels only)
  // [NS] 1: a fluid neighbour with an interface reads this node's n_c in
  // the curvature stencil; set by the step's gradient pass, cleared by its
  // Eq. 35 pass (zero between steps)
  uint8_t *smark;
};

}  // namespace lbm

struct lbm_ctx {
  int Q = 0;
  int nx = 0, ny = 0, nz = 0;
  long long N = 0;
  unsigned periodic = 0;
  int storage = 0;
  long long ntiles = 0;
  long long n_fluid = 0, n_sbnd = 0, n_fbnd = 0;
  bool params_set = false;
  bool state_set = false;
  lbm_params p{};
  lbm::Dom d{};
  void *TA = nullptr, *TB = nullptr;      // population planes (current = A)
  float4 *SA = nullptr, *SB = nullptr;
  uint8_t *mask = nullptr;                // device copy of the solid image
  double *g0 = nullptr, *g1 = nullptr;    // smoothing ping-pong (set-up)
  int *cnt_f = nullptr, *cnt_s = nullptr; // per-tile counts (set-up)
  double *red = nullptr;                  // reduction partials
  double *red_out = nullptr;              // 4 doubles: the combined partials
  int red_slots = 0;
  unsigned long long *counters = nullptr;
  int *zh_lists = nullptr;                // [3][NFp]: plane nodes per axis
  long long zh_count[3] = {0, 0, 0};
  // bumped by every call that changes the parameters or the state outside a
  // batch (set_params, init_state, set_populations, step): a batch holding
  // this domain refreshes its copy of the kernel arguments when it changes
  unsigned long long gen = 0;
  // lbm_step replays two steps at a time from a CUDA graph recorded on the
  // handle's own stream: one graph per orientation of the state buffers
  // (index 0: state in TA), valid while the parameters are those of pgen
  unsigned long long pgen = 0;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t g2[2] = {nullptr, nullptr};
  unsigned long long g2_pgen[2] = {0, 0};
  char err[256] = {0};
  ~lbm_ctx() {
    for (auto &x : g2)
      if (x) cudaGraphExecDestroy(x);
    if (cap) cudaStreamDestroy(cap);
  }
};

namespace lbm {
// After a step the destination buffers hold the current state.
inline void swap_state(lbm_ctx *c) {
  const void *t = c->d.T_src;
  c->d.T_src = c->d.T_dst;
  c->d.T_dst = const_cast<void *>(t);
  const float4 *u = c->d.S_src;
  c->d.S_src = c->d.S_dst;
  c->d.S_dst = const_cast<float4 *>(u);
}
}  // namespace lbm
