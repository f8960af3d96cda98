// The time step as five dependent passes. Each pass needs the previous one's
// values at lattice neighbours:
//   1 k_phase      (fluid)  pull + Zou-He + Eqs. (7)-(9), inlet/outlet phi
//   2 k_phi_solid  (solid-boundary) Eq. (34)
//   3 k_gradient   (fluid)  Eqs. (6), (27) and wetting, Eqs. (28)-(33)
//   4 k_nc_solid   (solid-boundary) Eq. (35)
//   5 k_collide    (fluid)  Eq. (12), (5), (36); pull + Zou-He again;
//                  Eq. (2) single-rate; store f'' and (q, v), i.e. the
//                  recoloured state of Eqs. (20)-(21)
// One CTA per tile: it stages the tile's neighbour table in shared memory
// (tiles.cuh), then its threads walk the tile's fluid (or solid-boundary)
// nodes.
#include <cuda_runtime.h>

#include "step.hpp"
#include "tiles.cuh"

namespace lbm {

constexpr int BLOCK = 256;

#define LBM_TILE_SMEM(Q)                                  \
  __shared__ uint32_t tab[TileGeo<Q>::HN];                \
  __shared__ uint16_t fpos[TileGeo<Q>::TN];               \
  __shared__ uint16_t spos[TileGeo<Q>::TN];               \
  int X0, Y0, Z0

// ---------------------------------------------------- global-lookup path
// Neighbour entry through the map (used only for the outlet plane, whose
// Eq. (39) value needs the populations streamed into the node behind it).
template <int Q>
__device__ __forceinline__ uint32_t entry_global(const Dom &d, int x, int y,
                                                 int z, int dx, int dy,
                                                 int dz) {
  bool out = false;
  const int X = axis_step(x + dx, d.nx, d.periodic & 1u, false, out);
  const int Y = axis_step(y + dy, d.ny, d.periodic & 2u, false, out);
  const int Z = axis_step(z + dz, d.nz, d.periodic & 4u, false, out);
  return out ? ENTRY_OUT : box_entry<Q>(d, X, Y, Z);
}

template <int Q, int ST>
__device__ float phase_global(const Dom &d, int k, int x, int y, int z) {
  const float4 Sown = __ldg(d.S_src + k);
  float rr = 0.f, rb = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float fr, fb;
    if (i == 0) {
      rebuild<Q>(TIO<Q, ST>::load(d, 0, k), Sown, 0, fr, fb);
    } else {
      const uint32_t e = entry_global<Q>(d, x, y, z, -Lattice<Q>::ex(i),
                                         -Lattice<Q>::ey(i), -Lattice<Q>::ez(i));
      const bool fl = entry_cls(e) & 2;
      const int src = fl ? entry_idx(e) : k;
      const float T = TIO<Q, ST>::load_dyn(d, fl ? i : Lattice<Q>::opp(i), src);
      const float4 S = fl ? __ldg(d.S_src + src) : Sown;
      const float ev = (float)Lattice<Q>::ex(i) * S.y +
                       (float)Lattice<Q>::ey(i) * S.z +
                       (float)Lattice<Q>::ez(i) * S.w;
      rebuild_ev<Q>(T, S.x, fl ? ev : -ev, i, fr, fb);
    }
    rr += fr;
    rb += fb;
  }
  return m_of(rr, rb);
}

// --------------------------------------------------------------- passes
// Encoded phase field of a fluid node from its streamed populations, with
// the Zou-He overrides: zeta^r - zeta^b on the inlet plane; on the outlet
// plane phi(x - a), Eq. (39), from the streamed populations of that node
// (the node's own value if that node is solid).
template <int Q, int ST>
__global__ void __launch_bounds__(BLOCK) k_phase(Dom d) {
  LBM_TILE_SMEM(Q);
  const int t = blockIdx.x;
  const int fb0 = __ldg(d.fbase + t);
  const int nf = __ldg(d.fbase + t + 1) - fb0;
  if (nf == 0) return;
  stage_tile<Q>(d, t, tab, fpos, spos, X0, Y0, Z0);
  for (int j = threadIdx.x; j < nf; j += BLOCK) {
    int x, y, z, p0;
    local_node<Q>(fpos[j], X0, Y0, Z0, x, y, z, p0);
    const int k = fb0 + j;
    if (d.c.zou_he) {
      const int a = d.c.axis;
      const int ca = axis_coord(x, y, z, a);
      if (ca == 0) {
        d.mf[k] = d.c.m_in;
        continue;
      }
      if (ca == axis_extent(d, a) - 1) {
        const int mx = x - (a == 0), my = y - (a == 1), mz = z - (a == 2);
        const uint32_t e = entry_global<Q>(d, mx, my, mz, 0, 0, 0);
        d.mf[k] = (entry_cls(e) & 2)
                      ? phase_global<Q, ST>(d, entry_idx(e), mx, my, mz)
                      : phase_global<Q, ST>(d, k, x, y, z);
        continue;
      }
    }
    float fr[Q], fb[Q], rr, rb;
    pull_tab<Q, ST>(d, tab, p0, k, __ldg(d.S_src + k), fr, fb);
    sum_colours<Q>(fr, fb, rr, rb);
    d.mf[k] = m_of(rr, rb);
  }
}

// Eq. (34): phi at a solid-boundary node = w-weighted mean over its fluid
// lattice neighbours, kept in the encoded form: the mean of phi - s for the
// sign s of the mean.
template <int Q>
__global__ void __launch_bounds__(BLOCK) k_phi_solid(Dom d) {
  LBM_TILE_SMEM(Q);
  using G = TileGeo<Q>;
  const int t = blockIdx.x;
  const int sb0 = __ldg(d.sbase + t);
  const int ns = __ldg(d.sbase + t + 1) - sb0;
  if (ns == 0) return;
  stage_tile<Q>(d, t, tab, fpos, spos, X0, Y0, Z0);
  for (int j = threadIdx.x; j < ns; j += BLOCK) {
    int x, y, z, p0;
    local_node<Q>(spos[j], X0, Y0, Z0, x, y, z, p0);
    float den = 0.f, sphi = 0.f, ex_pos = 0.f, ex_neg = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t e = tab[p0 + G::off(Lattice<Q>::ex(i), Lattice<Q>::ey(i),
                                         Lattice<Q>::ez(i))];
      if (!(entry_cls(e) & 2)) continue;
      const float w = Lattice<Q>::w(i);
      const float m = d.mf[entry_idx(e)];
      den += w;
      sphi += w * m_phi(m);
      ex_pos += w * m_excess(m, false);
      ex_neg += w * m_excess(m, true);
    }
    const bool blue = sphi < 0.f;
    const float ex = (blue ? ex_neg : ex_pos) / den;  // phi_s - s
    d.ms[sb0 + j] = m_pack(blue, blue ? 0.5f * ex : -0.5f * ex);
  }
}

// Eq. (6) (c = dt = 1) and Eq. (27), with phi(x + e_i) - s(x) in place of
// phi(x + e_i) (the same sum since sum_i w_i e_i = 0); at fluid-boundary
// nodes the wetting scheme turns n_c, keeping |C|. Stored: (n_c, |C|), or
// zero where |C| <= EPS_C (no interface).
template <int Q>
__global__ void __launch_bounds__(BLOCK) k_gradient(Dom d) {
  LBM_TILE_SMEM(Q);
  const int t = blockIdx.x;
  const int fb0 = __ldg(d.fbase + t);
  const int nf = __ldg(d.fbase + t + 1) - fb0;
  if (nf == 0) return;
  stage_tile<Q>(d, t, tab, fpos, spos, X0, Y0, Z0);
  for (int j = threadIdx.x; j < nf; j += BLOCK) {
    int x, y, z, p0;
    local_node<Q>(fpos[j], X0, Y0, Z0, x, y, z, p0);
    const int k = fb0 + j;
    const bool own_blue = m_blue(d.mf[k]);
    float G[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t e =
          clamped_entry<Q>(d, tab, p0, x, y, z, Lattice<Q>::ex(i),
                           Lattice<Q>::ey(i), Lattice<Q>::ez(i));
      const int idx = entry_idx(e);
      const float m = (entry_cls(e) & 2) ? d.mf[idx] : d.ms[idx];
      const float p = 3.f * Lattice<Q>::w(i) * m_excess(m, own_blue);
      G[0] += (float)Lattice<Q>::ex(i) * p;
      G[1] += (float)Lattice<Q>::ey(i) * p;
      G[2] += (float)Lattice<Q>::ez(i) * p;
    }
    const float mag = sqrtf(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
    if (!(mag > EPS_C)) {
      d.ncf[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const float im = 1.f / mag;
    float nc[3] = {G[0] * im, G[1] * im, G[2] * im};
    if (d.c.wetting && entry_cls(tab[p0]) == CLS_FLUID_BND) {
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
}

// Eq. (35): n_c at a solid-boundary node = w-weighted mean of the fluid
// neighbours' (post-wetting) n_c, not renormalised.
template <int Q>
__global__ void __launch_bounds__(BLOCK) k_nc_solid(Dom d) {
  LBM_TILE_SMEM(Q);
  using G = TileGeo<Q>;
  const int t = blockIdx.x;
  const int sb0 = __ldg(d.sbase + t);
  const int ns = __ldg(d.sbase + t + 1) - sb0;
  if (ns == 0) return;
  stage_tile<Q>(d, t, tab, fpos, spos, X0, Y0, Z0);
  for (int j = threadIdx.x; j < ns; j += BLOCK) {
    int x, y, z, p0;
    local_node<Q>(spos[j], X0, Y0, Z0, x, y, z, p0);
    float num[3] = {0.f, 0.f, 0.f}, den = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t e = tab[p0 + G::off(Lattice<Q>::ex(i), Lattice<Q>::ey(i),
                                         Lattice<Q>::ez(i))];
      if (!(entry_cls(e) & 2)) continue;
      const float4 v = d.ncf[entry_idx(e)];
      const float w = Lattice<Q>::w(i);
      num[0] += w * v.x;
      num[1] += w * v.y;
      num[2] += w * v.z;
      den += w;
    }
    const float id = 1.f / den;
    d.ncs[sb0 + j] = make_float4(num[0] * id, num[1] * id, num[2] * id, 0.f);
  }
}

// Eq. (12) with d_b n_a by the Eq. (6) stencil on each component, Eq. (5)
// F = 1/2 gamma kappa C (C = |C| n_c) plus rho g (Eq. 36); then the streamed
// populations again (pull + Zou-He), the collision, and the store of the
// recoloured state: f''_i and (q, v) with q the encoded rho^r/rho and
// v = beta rho^r rho^b / rho n (Eqs. 20-21). MACROS also stores (u, rho).
template <int Q, int ST, bool MACROS>
__global__ void __launch_bounds__(BLOCK) k_collide(Dom d) {
  LBM_TILE_SMEM(Q);
  const int t = blockIdx.x;
  const int fb0 = __ldg(d.fbase + t);
  const int nf = __ldg(d.fbase + t + 1) - fb0;
  if (nf == 0) return;
  stage_tile<Q>(d, t, tab, fpos, spos, X0, Y0, Z0);
  for (int j = threadIdx.x; j < nf; j += BLOCK) {
    int x, y, z, p0;
    local_node<Q>(fpos[j], X0, Y0, Z0, x, y, z, p0);
    const int k = fb0 + j;
    float dn[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t e =
          clamped_entry<Q>(d, tab, p0, x, y, z, Lattice<Q>::ex(i),
                           Lattice<Q>::ey(i), Lattice<Q>::ez(i));
      const int idx = entry_idx(e);
      const float4 v = (entry_cls(e) & 2) ? d.ncf[idx] : d.ncs[idx];
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
    float fr[Q], fb[Q];
    pull_tab<Q, ST>(d, tab, p0, k, __ldg(d.S_src + k), fr, fb);
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
}

template <int Q, int ST>
static void launch_step_t(const Dom &d, cudaStream_t s, bool macros,
                          cudaEvent_t *ev) {
  const unsigned g = (unsigned)d.ntiles;
  if (ev) cudaEventRecord(ev[0], s);
  k_phase<Q, ST><<<g, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[1], s);
  if (d.NS > 0) k_phi_solid<Q><<<g, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[2], s);
  k_gradient<Q><<<g, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[3], s);
  if (d.NS > 0) k_nc_solid<Q><<<g, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[4], s);
  if (macros)
    k_collide<Q, ST, true><<<g, BLOCK, 0, s>>>(d);
  else
    k_collide<Q, ST, false><<<g, BLOCK, 0, s>>>(d);
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
