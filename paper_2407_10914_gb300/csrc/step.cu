// The time step as five dependent passes. Each pass needs the previous one's
// values at lattice neighbours:
//   1 k_phase      (fluid)  pull + Zou-He + Eqs. (7)-(9), inlet/outlet phi
//   2 k_phi_solid  (solid-boundary) Eq. (34)
//   3 k_gradient   (fluid)  Eqs. (6), (27) and wetting, Eqs. (28)-(33)
//   4 k_nc_solid   (solid-boundary) Eq. (35)
//   5 k_collide    (fluid)  Eq. (12), (5), (36); pull + Zou-He again;
//                  Eq. (2) single-rate; store f'' and (q, v), i.e. the
//                  recoloured state of Eqs. (20)-(21)
// One thread per node of the compact fluid (F) or solid-boundary (S) list.
#include <cuda_runtime.h>

#include "stencil.cuh"
#include "step.hpp"

namespace lbm {

constexpr int BLOCK = 256;

template <int Q, int ST>
__device__ __forceinline__ float phase_of_node(const Dom &d, int k, int x,
                                               int y, int z) {
  const float4 S = __ldg(d.S_src + k);
  float fr[Q], fb[Q], rr, rb;
  pull<Q, ST>(d, k, x, y, z, S, fr, fb);
  sum_colours<Q>(fr, fb, rr, rb);
  return m_of(rr, rb);
}

// Encoded phase field of a fluid node from its streamed populations, with
// the Zou-He overrides: zeta^r - zeta^b on the inlet plane; on the outlet
// plane phi(x - a), Eq. (39), from the streamed populations of that node
// (the node's own value if that node is solid).
template <int Q, int ST>
__global__ void __launch_bounds__(BLOCK) k_phase(Dom d) {
  const int k = blockIdx.x * BLOCK + threadIdx.x;
  if (k >= d.NF) return;
  int x, y, z;
  box_coords(d, __ldg(d.fg + k), x, y, z);
  if (d.c.zou_he) {
    const int a = d.c.axis;
    const int ca = axis_coord(x, y, z, a);
    if (ca == 0) {
      d.mf[k] = d.c.m_in;
      return;
    }
    if (ca == axis_extent(d, a) - 1) {
      const int mx = x - (a == 0), my = y - (a == 1), mz = z - (a == 2);
      const Loc L = locate(d, mx, my, mz);
      d.mf[k] = is_fluid_cls(L.cls) ? phase_of_node<Q, ST>(d, L.idx, mx, my, mz)
                                    : phase_of_node<Q, ST>(d, k, x, y, z);
      return;
    }
  }
  d.mf[k] = phase_of_node<Q, ST>(d, k, x, y, z);
}

// Eq. (34): phi at a solid-boundary node = w-weighted mean over its fluid
// lattice neighbours, kept in the encoded form: the mean of phi - s for the
// sign s of the mean.
template <int Q>
__global__ void __launch_bounds__(BLOCK) k_phi_solid(Dom d) {
  const int j = blockIdx.x * BLOCK + threadIdx.x;
  if (j >= d.NS) return;
  int x, y, z;
  box_coords(d, __ldg(d.sg + j), x, y, z);
  float den = 0.f, sphi = 0.f, ex_pos = 0.f, ex_neg = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    bool out = false;
    const Loc L = neighbour(d, x, y, z, Lattice<Q>::ex(i), Lattice<Q>::ey(i),
                            Lattice<Q>::ez(i), false, out);
    if (!is_fluid_cls(L.cls)) continue;
    const float w = Lattice<Q>::w(i);
    const float m = d.mf[L.idx];
    den += w;
    sphi += w * m_phi(m);
    ex_pos += w * m_excess(m, false);
    ex_neg += w * m_excess(m, true);
  }
  const bool blue = sphi < 0.f;
  const float ex = (blue ? ex_neg : ex_pos) / den;  // phi_s - s
  d.ms[j] = m_pack(blue, blue ? 0.5f * ex : -0.5f * ex);
}

// Eq. (6) (c = dt = 1) and Eq. (27), with phi(x + e_i) - s(x) in place of
// phi(x + e_i) (the same sum since sum_i w_i e_i = 0); at fluid-boundary
// nodes the wetting scheme turns n_c, keeping |C|. Stored: (n_c, |C|), or
// zero where |C| <= EPS_C (no interface).
template <int Q>
__global__ void __launch_bounds__(BLOCK) k_gradient(Dom d) {
  const int k = blockIdx.x * BLOCK + threadIdx.x;
  if (k >= d.NF) return;
  const int g = __ldg(d.fg + k);
  int x, y, z;
  box_coords(d, g, x, y, z);
  const bool own_blue = m_blue(d.mf[k]);
  float G[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    bool out = false;
    const Loc L = neighbour(d, x, y, z, Lattice<Q>::ex(i), Lattice<Q>::ey(i),
                            Lattice<Q>::ez(i), true, out);
    const float m = is_fluid_cls(L.cls) ? d.mf[L.idx] : d.ms[L.idx];
    const float p = 3.f * Lattice<Q>::w(i) * m_excess(m, own_blue);
    G[0] += (float)Lattice<Q>::ex(i) * p;
    G[1] += (float)Lattice<Q>::ey(i) * p;
    G[2] += (float)Lattice<Q>::ez(i) * p;
  }
  const float mag = sqrtf(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
  if (!(mag > EPS_C)) {
    d.ncf[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const float im = 1.f / mag;
  float nc[3] = {G[0] * im, G[1] * im, G[2] * im};
  if (d.c.wetting && __ldg(d.cls + g) == CLS_FLUID_BND) {
    const float4 w4 = __ldg(d.nw + k);
    const float nw[3] = {w4.x, w4.y, w4.z};
    if (nw[0] != 0.f || nw[1] != 0.f || nw[2] != 0.f) {
      if (d.c.wetting == 1)
        scheme1(nc, nw, d.c.cos_t);
      else
        scheme2(nc, nw, d.c.cos_t, d.c.sin_t);
    }
  }
  d.ncf[k] = make_float4(nc[0], nc[1], nc[2], mag);
}

// Eq. (35): n_c at a solid-boundary node = w-weighted mean of the fluid
// neighbours' (post-wetting) n_c, not renormalised.
template <int Q>
__global__ void __launch_bounds__(BLOCK) k_nc_solid(Dom d) {
  const int j = blockIdx.x * BLOCK + threadIdx.x;
  if (j >= d.NS) return;
  int x, y, z;
  box_coords(d, __ldg(d.sg + j), x, y, z);
  float num[3] = {0.f, 0.f, 0.f}, den = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    bool out = false;
    const Loc L = neighbour(d, x, y, z, Lattice<Q>::ex(i), Lattice<Q>::ey(i),
                            Lattice<Q>::ez(i), false, out);
    if (!is_fluid_cls(L.cls)) continue;
    const float4 v = d.ncf[L.idx];
    const float w = Lattice<Q>::w(i);
    num[0] += w * v.x;
    num[1] += w * v.y;
    num[2] += w * v.z;
    den += w;
  }
  const float id = 1.f / den;
  d.ncs[j] = make_float4(num[0] * id, num[1] * id, num[2] * id, 0.f);
}

// Eq. (12) with d_b n_a by the Eq. (6) stencil on each component, Eq. (5)
// F = 1/2 gamma kappa C (C = |C| n_c) plus rho g (Eq. 36); then the streamed
// populations again (pull + Zou-He), the collision, and the store of the
// recoloured state: f''_i and (q, v) with q the encoded rho^r/rho and
// v = beta rho^r rho^b / rho n (Eqs. 20-21). MACROS also stores (u, rho).
template <int Q, int ST, bool MACROS>
__global__ void __launch_bounds__(BLOCK) k_collide(Dom d) {
  const int k = blockIdx.x * BLOCK + threadIdx.x;
  if (k >= d.NF) return;
  int x, y, z;
  box_coords(d, __ldg(d.fg + k), x, y, z);
  float dn[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    bool out = false;
    const Loc L = neighbour(d, x, y, z, Lattice<Q>::ex(i), Lattice<Q>::ey(i),
                            Lattice<Q>::ez(i), true, out);
    const float4 v = is_fluid_cls(L.cls) ? d.ncf[L.idx] : d.ncs[L.idx];
    const float w3 = 3.f * Lattice<Q>::w(i);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int eb = Lattice<Q>::e(i, b);
      if (eb == 0) continue;
      dn[0][b] += w3 * (float)eb * v.x;
      dn[1][b] += w3 * (float)eb * v.y;
      dn[2][b] += w3 * (float)eb * v.z;
    }
  }
  const float4 c4 = d.ncf[k];
  const float nx_ = c4.x, ny_ = c4.y, nz_ = c4.z;
  const float kappa = (nx_ * nx_ - 1.f) * dn[0][0] +
                      (ny_ * ny_ - 1.f) * dn[1][1] +
                      (nz_ * nz_ - 1.f) * dn[2][2] +
                      (dn[0][1] + dn[1][0]) * nx_ * ny_ +
                      (dn[0][2] + dn[2][0]) * nx_ * nz_ +
                      (dn[2][1] + dn[1][2]) * nz_ * ny_;
  const float4 Sown = __ldg(d.S_src + k);
  float fr[Q], fb[Q];
  pull<Q, ST>(d, k, x, y, z, Sown, fr, fb);
  const float phi = m_phi(d.mf[k]);
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
#pragma unroll
  for (int i = 0; i < Q; ++i) fr[i] += fb[i];  // f^t
  float u[3];
  collide<Q>(d.c, fr, rho, F, phi, u);
#pragma unroll
  for (int i = 0; i < Q; ++i) TIO<Q, ST>::store(d, d.T_dst, i, k, fr[i]);
  const float seg = d.c.beta * rr * rb / rho;
  d.S_dst[k] = make_float4(m_of(rr, rb), seg * nx_, seg * ny_, seg * nz_);
  if (MACROS) d.macro[k] = make_float4(u[0], u[1], u[2], rho);
}

static inline unsigned blocks_for(long long n) {
  return (unsigned)((n + BLOCK - 1) / BLOCK);
}

template <int Q, int ST>
static void launch_step_t(const Dom &d, cudaStream_t s, bool macros,
                          cudaEvent_t *ev) {
  const unsigned gF = blocks_for(d.NF);
  const unsigned gS = blocks_for(d.NS);
  if (ev) cudaEventRecord(ev[0], s);
  k_phase<Q, ST><<<gF, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[1], s);
  if (d.NS > 0) k_phi_solid<Q><<<gS, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[2], s);
  k_gradient<Q><<<gF, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[3], s);
  if (d.NS > 0) k_nc_solid<Q><<<gS, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[4], s);
  if (macros)
    k_collide<Q, ST, true><<<gF, BLOCK, 0, s>>>(d);
  else
    k_collide<Q, ST, false><<<gF, BLOCK, 0, s>>>(d);
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
