// The time step as five dependent passes. Each pass needs the previous one's
// values at lattice neighbours:
//   1 k_stream     (fluid)  pull of Eq. (1), Eqs. (7)-(9): stores f^t,
//                  (rho^r, rho^b) and the phase field; k_zh_fix then applies
//                  App. B on the Zou-He planes
//   2 k_phi_solid  (solid-boundary) Eq. (34)
//   3 k_gradient   (fluid)  Eqs. (6), (27) and wetting, Eqs. (28)-(33)
//   4 k_nc_solid   (solid-boundary) Eq. (35)
//   5 k_collide    (fluid)  Eq. (12), (5), (36); Eq. (2) single-rate on the
//                  stored f^t; store f'' and (q, v), i.e. the recoloured
//                  state of Eqs. (20)-(21)
// One thread per node of the compact fluid (F) or solid-boundary (S) list;
// every lattice neighbour is one entry of the node's precomputed neighbour
// table (built at set-up, geometry.cu).
#include <cuda_runtime.h>

#include "step.hpp"
#include "tiles.cuh"

namespace lbm {

constexpr int BLOCK = 256;

__device__ __forceinline__ uint32_t nb_f(const Dom &d, int dir, int k) {
  return __ldg(d.nbf + (long long)(dir - 1) * d.NFp + k);
}
// Weight of a solid-boundary link (bit 31: diagonal direction).
template <int Q>
__device__ __forceinline__ float link_w(uint32_t l) {
  return (l >> 31) ? Lattice<Q>::w(Q - 1) : Lattice<Q>::w(1);
}

template <int Q, int ST>
__device__ __forceinline__ void store_streamed(const Dom &d, int k,
                                               const float *ft, float rr,
                                               float rb, float m) {
#pragma unroll
  for (int i = 0; i < Q; ++i) TIO<Q, ST>::store(d, d.U, i, k, ft[i]);
  d.R[k] = make_float2(rr, rb);
  d.mf[k] = m;
}

// Streamed populations of a fluid node (Eq. 1), their colour densities and
// the encoded phase field (Eqs. 7-9). On the Zou-He planes the populations
// from outside the box are placeholders until k_zh_fix.
template <int Q, int ST>
__global__ void __launch_bounds__(BLOCK) k_stream(Dom d) {
  const int k = blockIdx.x * BLOCK + threadIdx.x;
  if (k >= d.NF) return;
  float ft[Q], rr, rb;
  pull_sums<Q, ST>(d, k, __ldg(d.S_src + k), ft, rr, rb);
  store_streamed<Q, ST>(d, k, ft, rr, rb, m_of(rr, rb));
}

// App. B on the Zou-He planes (one thread per node of their list), after
// k_stream. Its per-colour rules are linear in the populations, and the
// collision needs only f^t = f^r + f^b and rho^r, rho^b, so the unknown
// populations are rebuilt in totals: with K0 the sum of the known f^t with
// e.a = 0, Kin that of the known ones with e.a pointing into the box, and
// N_t = 1/2 sum_{e.a=0} (e.t) f^t (t != a),
//   inlet  (B.1-B.8):  j = rho_in - (K0 + 2 Kin),
//                      f_i = f_opp(i) + 6 w_i j - sum_t (e_i.t) N_t, e_i.a = +1;
//   outlet (B.9-B.18): j = (K0 + 2 Kin) - rho_out,
//                      f_i = f_opp(i) - 6 w_i j - sum_t (e_i.t) N_t, e_i.a = -1
// (chi^r + chi^b = 1). Summing the per-colour rules over i gives the colour
// densities: rho^s = rho_in zeta^s at the inlet, and at the outlet
// rho^s = K0^s + 2 Kin^s - j chi^s with chi^r = (1 + phi_out)/2, where the
// red sums K0^r, Kin^r come from the pull's colour split. The phase field
// is zeta^r - zeta^b at the inlet and phi(x - a), Eq. (39), at the outlet
// (the node's own value if that node is solid).
template <int Q, int ST>
__global__ void __launch_bounds__(BLOCK) k_zh_fix(Dom d) {
  const int jz = blockIdx.x * BLOCK + threadIdx.x;
  if (jz >= d.n_zh) return;
  const int k = __ldg(d.zh_list + jz);
  const int a = d.c.axis;
  const bool inlet = __ldg(d.fflag + k) & (2u << (2 * a));
  const int in_dir = inlet ? -1 : 1;  // e.a of the known, inward populations
  float ft[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) ft[i] = TIO<Q, ST>::load_from(d, d.U, i, k);
  float K0 = 0.f, Kin = 0.f, N[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int ea = Lattice<Q>::e(i, a);
    if (ea == 0) {
      K0 += ft[i];
#pragma unroll
      for (int t = 0; t < 3; ++t)
        if (t != a) N[t] += 0.5f * (float)Lattice<Q>::e(i, t) * ft[i];
    } else if (ea == in_dir) {
      Kin += ft[i];
    }
  }
  float rr, rb, m, jt;
  if (inlet) {
    jt = d.c.rho_in_r + d.c.rho_in_b - (K0 + 2.f * Kin);
    rr = d.c.rho_in_r;
    rb = d.c.rho_in_b;
    m = d.c.m_in;
  } else {
    jt = (K0 + 2.f * Kin) - d.c.rho_out;
    const uint32_t e = nb_f(d, 2 * a + 2, k);  // the node at x - a
    const float2 Rk = d.R[k];
    m = ((entry_cls(e) & 2) && !entry_out(e)) ? d.mf[entry_idx(e)]
                                               : m_of(Rk.x, Rk.y);
    // red parts of the known populations (e.a >= 0), as the pull split them
    const float4 Sown = __ldg(d.S_src + k);
    float K0r = 0.f, Kinr = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int ea = Lattice<Q>::e(i, a);
      if (ea < 0) continue;
      float fr, fb;
      if (i == 0) {
        rebuild<Q>(ft[0], Sown, 0, fr, fb);
      } else {
        const uint32_t es = nb_f(d, Lattice<Q>::opp(i), k);
        const bool fl = (entry_cls(es) & 2) && !entry_out(es);
        const float4 S = fl ? __ldg(d.S_src + entry_idx(es)) : Sown;
        const float ev = (float)Lattice<Q>::ex(i) * S.y +
                         (float)Lattice<Q>::ey(i) * S.z +
                         (float)Lattice<Q>::ez(i) * S.w;
        rebuild_ev<Q>(ft[i], S.x, fl ? ev : -ev, i, fr, fb);
      }
      if (ea == 0) K0r += fr;
      else Kinr += fr;
    }
    const float chi_r = 0.5f * (1.f + m_phi(m));
    rr = K0r + 2.f * Kinr - jt * chi_r;
    rb = (K0 - K0r) + 2.f * (Kin - Kinr) - jt * (1.f - chi_r);
    jt = -jt;  // the outlet rule subtracts 6 w_i j
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (Lattice<Q>::e(i, a) != -in_dir) continue;
    float corr = 0.f;
#pragma unroll
    for (int t = 0; t < 3; ++t)
      if (t != a) corr += (float)Lattice<Q>::e(i, t) * N[t];
    TIO<Q, ST>::store(d, d.U, i, k,
                      ft[Lattice<Q>::opp(i)] + 6.f * Lattice<Q>::w(i) * jt - corr);
  }
  d.R[k] = make_float2(rr, rb);
  d.mf[k] = m;
}

// Eq. (34): phi at a solid-boundary node = w-weighted mean over its fluid
// lattice neighbours, kept in the encoded form: the mean of phi - s for the
// sign s of the mean.
template <int Q>
__global__ void __launch_bounds__(BLOCK) k_phi_solid(Dom d) {
  const int j = blockIdx.x * BLOCK + threadIdx.x;
  if (j >= d.NS) return;
  float den = 0.f, sphi = 0.f, ex_pos = 0.f, ex_neg = 0.f;
  const int e = __ldg(d.soff + j + 1);
  for (int p = __ldg(d.soff + j); p < e; ++p) {
    const uint32_t l = __ldg(d.slink + p);
    const float w = link_w<Q>(l);
    const float m = d.mf[l & 0x7FFFFFFFu];
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
// phi(x + e_i) (the same sum since sum_i w_i e_i = 0), off-box neighbours
// clamped; at fluid-boundary nodes the wetting scheme turns n_c, keeping
// |C|. Stored: (n_c, |C|), or zero where |C| <= EPS_C (no interface).
template <int Q>
__global__ void __launch_bounds__(BLOCK) k_gradient(Dom d) {
  const int k = blockIdx.x * BLOCK + threadIdx.x;
  if (k >= d.NF) return;
  const bool own_blue = m_blue(d.mf[k]);
  float G[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const uint32_t e = nb_f(d, i, k);
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
    return;
  }
  const float im = 1.f / mag;
  float nc[3] = {G[0] * im, G[1] * im, G[2] * im};
  if (d.c.wetting && (__ldg(d.fflag + k) & 1u)) {
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
  float num[3] = {0.f, 0.f, 0.f}, den = 0.f;
  const int e = __ldg(d.soff + j + 1);
  for (int p = __ldg(d.soff + j); p < e; ++p) {
    const uint32_t l = __ldg(d.slink + p);
    const float w = link_w<Q>(l);
    const float4 v = d.ncf[l & 0x7FFFFFFFu];
    num[0] += w * v.x;
    num[1] += w * v.y;
    num[2] += w * v.z;
    den += w;
  }
  const float id = 1.f / den;
  d.ncs[j] = make_float4(num[0] * id, num[1] * id, num[2] * id, 0.f);
}

// Eq. (12) with d_b n_a by the Eq. (6) stencil on each component (off-box
// neighbours clamped); returns kappa and the node's (n_c, |C|).
template <int Q>
__device__ __forceinline__ float curvature(const Dom &d, int k, float4 &c4) {
  float dn[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const uint32_t e = nb_f(d, i, k);
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
  c4 = d.ncf[k];
  const float nx_ = c4.x, ny_ = c4.y, nz_ = c4.z;
  return (nx_ * nx_ - 1.f) * dn[0][0] + (ny_ * ny_ - 1.f) * dn[1][1] +
         (nz_ * nz_ - 1.f) * dn[2][2] + (dn[0][1] + dn[1][0]) * nx_ * ny_ +
         (dn[0][2] + dn[2][0]) * nx_ * nz_ + (dn[2][1] + dn[1][2]) * nz_ * ny_;
}

// Eq. (5) F = 1/2 gamma kappa C (C = |C| n_c) plus rho g (Eq. 36), the
// collision (Eq. 2) of the stored f^t, and the store of the recoloured
// state: f''_i and (q, v) with q the encoded rho^r/rho and
// v = beta rho^r rho^b / rho n (Eqs. 20-21). The relaxation rate follows
// the node's phase field (Eq. 39's value on the outlet plane).
template <int Q, int ST, bool MACROS>
__global__ void __launch_bounds__(BLOCK, 4) k_collide(Dom d) {
  const int k = blockIdx.x * BLOCK + threadIdx.x;
  if (k >= d.NF) return;
  float4 c4;
  const float kappa = curvature<Q>(d, k, c4);
  float ft[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) ft[i] = TIO<Q, ST>::load_from(d, d.U, i, k);
  const float2 R = d.R[k];
  const float rr = R.x, rb = R.y;
  const float rho = rr + rb;
  const float hk = 0.5f * d.c.gamma * kappa * c4.w;
  const float F[3] = {hk * c4.x + rho * d.c.g[0], hk * c4.y + rho * d.c.g[1],
                      hk * c4.z + rho * d.c.g[2]};
  float u[3];
  collide<Q>(d.c, ft, rho, F, m_phi(d.mf[k]), u);
#pragma unroll
  for (int i = 0; i < Q; ++i) TIO<Q, ST>::store(d, d.T_dst, i, k, ft[i]);
  const float seg = d.c.beta * rr * rb / rho;
  d.S_dst[k] = make_float4(m_of(rr, rb), seg * c4.x, seg * c4.y, seg * c4.z);
  if (MACROS) d.macro[k] = make_float4(u[0], u[1], u[2], rho);
}

template <int Q, int ST>
static void launch_step_t(const Dom &d, cudaStream_t s, bool macros,
                          cudaEvent_t *ev) {
  const unsigned g = (unsigned)((d.NF + BLOCK - 1) / BLOCK);
  const unsigned gs = (unsigned)((d.NS + BLOCK - 1) / BLOCK);
  const unsigned gz = (unsigned)((d.n_zh + BLOCK - 1) / BLOCK);
  if (ev) cudaEventRecord(ev[0], s);
  k_stream<Q, ST><<<g, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[1], s);
  if (d.n_zh > 0) k_zh_fix<Q, ST><<<gz, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[2], s);
  if (d.NS > 0) k_phi_solid<Q><<<gs, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[3], s);
  k_gradient<Q><<<g, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[4], s);
  if (d.NS > 0) k_nc_solid<Q><<<gs, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[5], s);
  if (macros)
    k_collide<Q, ST, true><<<g, BLOCK, 0, s>>>(d);
  else
    k_collide<Q, ST, false><<<g, BLOCK, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[6], s);
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
