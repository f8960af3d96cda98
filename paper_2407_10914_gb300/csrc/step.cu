// The time step as five dependent passes over the box. Each pass needs the
// previous one's values at lattice neighbours:
//   1 k_phase      pull + Zou-He + Eqs. (7)-(9), inlet/outlet phi -> phi
//   2 k_phi_solid  Eq. (34) at solid-boundary nodes                -> phi
//   3 k_gradient   Eqs. (6), (27), wetting (28-33) at fluid nodes  -> nc
//   4 k_nc_solid   Eq. (35) at solid-boundary nodes                -> nc
//   5 k_collide    Eq. (12), (5), (36), pull again, Zou-He, Eq. (2)
//                  single-rate, recolouring (20)-(21)              -> f_dst
#include <cuda_runtime.h>

#include "stencil.cuh"
#include "step.hpp"

namespace lbm {

constexpr int BLOCK = 256;

// Phase field of one fluid node from its streamed populations, with the
// Zou-He overrides: phi = zeta^r - zeta^b on the inlet plane, and on the
// outlet plane phi(x - a) (Eq. 39) from the streamed populations of that
// node (the node's own value if that node is solid).
template <int Q, int ST>
__global__ void __launch_bounds__(BLOCK) k_phase(Dom d) {
  const long long n = (long long)blockIdx.x * BLOCK + threadIdx.x;
  if (n >= d.N) return;
  if (!is_fluid_cls(d.cls[n])) return;
  int x, y, z;
  node_coords(d, n, x, y, z);
  const PopIO<Q, ST> io(d);
  if (d.c.zou_he) {
    const int a = d.c.axis;
    const int ca = axis_coord(x, y, z, a);
    if (ca == 0) {
      d.phi[n] = d.c.phi_in;
      return;
    }
    if (ca == axis_extent(d, a) - 1) {
      bool out = false;
      const long long m = nb_index(d, x, y, z, a == 0 ? -1 : 0,
                                   a == 1 ? -1 : 0, a == 2 ? -1 : 0, false, out);
      int mx = x, my = y, mz = z;
      long long src = n;
      if (!out && is_fluid_cls(d.cls[m])) {
        src = m;
        if (a == 0) mx -= 1;
        if (a == 1) my -= 1;
        if (a == 2) mz -= 1;
      }
      float fr[Q], fb[Q], rr, rb;
      pull<Q, ST>(d, io, src, mx, my, mz, fr, fb);
      sum_colours<Q>(fr, fb, rr, rb);
      d.phi[n] = (rr - rb) / (rr + rb);
      return;
    }
  }
  float fr[Q], fb[Q], rr, rb;
  pull<Q, ST>(d, io, n, x, y, z, fr, fb);
  sum_colours<Q>(fr, fb, rr, rb);
  d.phi[n] = (rr - rb) / (rr + rb);
}

// Eq. (34): phi at a solid-boundary node = w-weighted mean over its fluid
// lattice neighbours.
template <int Q>
__global__ void __launch_bounds__(BLOCK) k_phi_solid(Dom d) {
  const int k = blockIdx.x * BLOCK + threadIdx.x;
  if (k >= d.n_sbnd) return;
  const long long n = d.sbnd[k];
  int x, y, z;
  node_coords(d, n, x, y, z);
  float num = 0.f, den = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    bool out = false;
    const long long m = nb_index(d, x, y, z, Lattice<Q>::e(i, 0),
                                 Lattice<Q>::e(i, 1), Lattice<Q>::e(i, 2),
                                 false, out);
    if (out || !is_fluid_cls(d.cls[m])) continue;
    num += Lattice<Q>::w(i) * d.phi[m];
    den += Lattice<Q>::w(i);
  }
  d.phi[n] = num / den;
}

// Eq. (6) (c = dt = 1) and Eq. (27); at fluid-boundary nodes the wetting
// scheme turns n_c, keeping |C|. Stored: (n_c, |C|), or zero where
// |C| <= EPS_C (no interface).
template <int Q>
__global__ void __launch_bounds__(BLOCK) k_gradient(Dom d) {
  const long long n = (long long)blockIdx.x * BLOCK + threadIdx.x;
  if (n >= d.N) return;
  const uint8_t cl = d.cls[n];
  if (!is_fluid_cls(cl)) return;
  int x, y, z;
  node_coords(d, n, x, y, z);
  float G[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    bool out = false;
    const long long m = nb_index(d, x, y, z, Lattice<Q>::e(i, 0),
                                 Lattice<Q>::e(i, 1), Lattice<Q>::e(i, 2),
                                 true, out);
    const float p = 3.f * Lattice<Q>::w(i) * d.phi[m];
#pragma unroll
    for (int a = 0; a < 3; ++a) G[a] += (float)Lattice<Q>::e(i, a) * p;
  }
  const float mag = sqrtf(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
  if (!(mag > EPS_C)) {
    d.nc[n] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const float im = 1.f / mag;
  float nc[3] = {G[0] * im, G[1] * im, G[2] * im};
  if (cl == CLS_FLUID_BND && d.c.wetting) {
    const float4 w4 = d.nw[n];
    const float nw[3] = {w4.x, w4.y, w4.z};
    if (nw[0] != 0.f || nw[1] != 0.f || nw[2] != 0.f) {
      if (d.c.wetting == 1)
        scheme1(nc, nw, d.c.cos_t);
      else
        scheme2(nc, nw, d.c.cos_t, d.c.sin_t);
    }
  }
  d.nc[n] = make_float4(nc[0], nc[1], nc[2], mag);
}

// Eq. (35): n_c at a solid-boundary node = w-weighted mean of the fluid
// neighbours' (post-wetting) n_c, not renormalised.
template <int Q>
__global__ void __launch_bounds__(BLOCK) k_nc_solid(Dom d) {
  const int k = blockIdx.x * BLOCK + threadIdx.x;
  if (k >= d.n_sbnd) return;
  const long long n = d.sbnd[k];
  int x, y, z;
  node_coords(d, n, x, y, z);
  float num[3] = {0.f, 0.f, 0.f}, den = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    bool out = false;
    const long long m = nb_index(d, x, y, z, Lattice<Q>::e(i, 0),
                                 Lattice<Q>::e(i, 1), Lattice<Q>::e(i, 2),
                                 false, out);
    if (out || !is_fluid_cls(d.cls[m])) continue;
    const float4 v = d.nc[m];
    const float w = Lattice<Q>::w(i);
    num[0] += w * v.x;
    num[1] += w * v.y;
    num[2] += w * v.z;
    den += w;
  }
  const float id = 1.f / den;
  d.nc[n] = make_float4(num[0] * id, num[1] * id, num[2] * id, 0.f);
}

// Eq. (12) with d_b n_a by the Eq. (6) stencil on each component, Eq. (5)
// F = 1/2 gamma kappa C (C = |C| n_c) plus rho g (Eq. 36); then the streamed
// populations again (pull + Zou-He), the collision and the recolouring, and
// the write to the other buffer. MACROS also stores rho and u (Eq. 22).
template <int Q, int ST, bool MACROS>
__global__ void __launch_bounds__(BLOCK) k_collide(Dom d) {
  const long long n = (long long)blockIdx.x * BLOCK + threadIdx.x;
  if (n >= d.N) return;
  if (!is_fluid_cls(d.cls[n])) return;
  int x, y, z;
  node_coords(d, n, x, y, z);
  float dn[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    bool out = false;
    const long long m = nb_index(d, x, y, z, Lattice<Q>::e(i, 0),
                                 Lattice<Q>::e(i, 1), Lattice<Q>::e(i, 2),
                                 true, out);
    const float4 v = d.nc[m];
    const float w3 = 3.f * Lattice<Q>::w(i);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float eb = (float)Lattice<Q>::e(i, b);
      if (eb == 0.f) continue;
      dn[0][b] += w3 * eb * v.x;
      dn[1][b] += w3 * eb * v.y;
      dn[2][b] += w3 * eb * v.z;
    }
  }
  const float4 c4 = d.nc[n];
  const float nx_ = c4.x, ny_ = c4.y, nz_ = c4.z;
  const float kappa = (nx_ * nx_ - 1.f) * dn[0][0] +
                      (ny_ * ny_ - 1.f) * dn[1][1] +
                      (nz_ * nz_ - 1.f) * dn[2][2] +
                      (dn[0][1] + dn[1][0]) * nx_ * ny_ +
                      (dn[0][2] + dn[2][0]) * nx_ * nz_ +
                      (dn[2][1] + dn[1][2]) * nz_ * ny_;
  const PopIO<Q, ST> io(d);
  float fr[Q], fb[Q];
  pull<Q, ST>(d, io, n, x, y, z, fr, fb);
  const float phi = d.phi[n];
  if (d.c.zou_he) {
    const int a = d.c.axis;
    const int ca = axis_coord(x, y, z, a);
    if (ca == 0) {
      zou_he_inlet<Q>(fr, d.c.rho_in_r, a);
      zou_he_inlet<Q>(fb, d.c.rho_in_b, a);
    } else if (ca == axis_extent(d, a) - 1) {
      zou_he_outlet<Q>(fr, fb, d.c.rho_out, phi, a);
    }
  }
  float rr, rb;
  sum_colours<Q>(fr, fb, rr, rb);
  const float rho = rr + rb;
  const float hk = 0.5f * d.c.gamma * kappa * c4.w;
  const float F[3] = {hk * nx_ + rho * d.c.g[0], hk * ny_ + rho * d.c.g[1],
                      hk * nz_ + rho * d.c.g[2]};
  const float nrm[3] = {nx_, ny_, nz_};
  float u[3];
  collide_recolour<Q>(d.c, fr, fb, phi, F, nrm, u);
#pragma unroll
  for (int i = 0; i < Q; ++i) io.store(i, n, fr[i], fb[i]);
  if (MACROS) {
    d.rho_m[n] = rho;
    d.u_m[n] = u[0];
    d.u_m[d.N + n] = u[1];
    d.u_m[2 * d.N + n] = u[2];
  }
}

static inline unsigned blocks_for(long long n) {
  return (unsigned)((n + BLOCK - 1) / BLOCK);
}

template <int Q, int ST>
static void launch_step_t(const Dom &d, cudaStream_t s, bool macros,
                          cudaEvent_t *ev) {
  const unsigned gN = blocks_for(d.N);
  if (ev) cudaEventRecord(ev[0], s);
  k_phase<Q, ST><<<gN, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[1], s);
  if (d.n_sbnd > 0)
    k_phi_solid<Q><<<blocks_for(d.n_sbnd), BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[2], s);
  k_gradient<Q><<<gN, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[3], s);
  if (d.n_sbnd > 0)
    k_nc_solid<Q><<<blocks_for(d.n_sbnd), BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[4], s);
  if (macros)
    k_collide<Q, ST, true><<<gN, BLOCK, 0, s>>>(d);
  else
    k_collide<Q, ST, false><<<gN, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[5], s);
}

static void dispatch(int Q, int storage, const Dom &d, cudaStream_t s,
                     bool macros, cudaEvent_t *ev) {
  if (Q == 19) {
    if (storage == LBM_STORAGE_FP32) launch_step_t<19, LBM_STORAGE_FP32>(d, s, macros, ev);
    if (storage == LBM_STORAGE_FP16) launch_step_t<19, LBM_STORAGE_FP16>(d, s, macros, ev);
    if (storage == LBM_STORAGE_BF16) launch_step_t<19, LBM_STORAGE_BF16>(d, s, macros, ev);
  } else {
    if (storage == LBM_STORAGE_FP32) launch_step_t<9, LBM_STORAGE_FP32>(d, s, macros, ev);
    if (storage == LBM_STORAGE_FP16) launch_step_t<9, LBM_STORAGE_FP16>(d, s, macros, ev);
    if (storage == LBM_STORAGE_BF16) launch_step_t<9, LBM_STORAGE_BF16>(d, s, macros, ev);
  }
}

void launch_step(int Q, int storage, const Dom &d, cudaStream_t s,
                 bool macros) {
  dispatch(Q, storage, d, s, macros, nullptr);
}

void launch_step_events(int Q, int storage, const Dom &d, cudaStream_t s,
                        bool macros, cudaEvent_t *ev) {
  dispatch(Q, storage, d, s, macros, ev);
}

}  // namespace lbm
