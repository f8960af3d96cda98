// Hand-written adjoint (reverse mode) of one time step, for gradients of a
// scalar of the final state with respect to the contact angle theta and the
// body acceleration g (Eqs. 32-33, 36).
//
// The state of a fluid node is x = (T_i, r, v): T_i = f''_i the total
// post-recolouring populations, r = rho^r/rho the red fraction and
// v = beta rho^r rho^b / rho n, so that the red part of population i after
// recolouring is r T_i + w_i e_i.v (Eqs. 20-21). The stored encoding of r
// (the minority fraction with the majority colour in its lowest bit) is a
// precision device only. The adjoint state lambda = (lT_i, lr, lv) has the
// same shape. Reversing the step x_t -> x_{t+1} maps lambda(x_{t+1}) to
// lambda(x_t) and adds the step's contribution to dJ/dtheta and dJ/dg.
//
// The forward fields of the step (f^t, rho^r, rho^b, phi, n_c, |C| and
// their solid-boundary extrapolations) are recomputed from x_t by the
// forward kernels, then the passes run in reverse:
//   A1 collision, force and curvature (Eqs. 2, 5, 12, 20-21, 36): per node;
//      the curvature stencil transposes to the neighbours' n (atomics);
//   A2 Eq. (35) transposed: solid-boundary n to the fluid links (atomics);
//   A3 normalisation (Eq. 11), Scheme-II (Eqs. 32-33) and the gradient
//      stencil (Eq. 6) transposed to the neighbours' phi (atomics);
//   A4 Eq. (34) transposed: solid-boundary phi to the fluid links;
//   A5 the phase field (Eq. 7) and the colour densities per node;
//   A6 streaming (Eq. 1) transposed: every (node, direction) of x_t sends
//      its population to exactly one place, so this is a gather.
// The adjoint covers float32 storage, the single-rate collision, no wetting
// or Scheme-II, and ends without Zou-He planes (periodic axes or bounce-back
// walls); Scheme-I's secant iterations, App. B and the MRT rates are not
// differentiated here.
//
// Regularised linearisation. Where n_c is almost along n_w, Scheme-II's
// result direction around n_w is undefined and its derivative grows as
// 1/sin(theta'); over a few hundred steps such nodes make the exact
// derivative of the discrete step grow without bound (the FP64 tangent-
// linear run of the oracle shows it), while the response to a finite
// change of theta or g stays smooth. The interface normal n_c = C/|C| has
// the same kind of Jacobian (1/|C|) in the interface tails. By default the
// adjoint drops the derivative of Scheme-II's direction around n_w where
// sin(theta') < 0.05 and of n_c's direction where |C| < 1e-3, and keeps
// everything else exact; lbm_adj_set_freeze(a, 0) and lbm_adj_set_cmin(a,
// 0) restore the exact derivative.
#include <cuda_runtime.h>

#include <cstdio>
#include <new>

#include "passes.cuh"
#include "step.hpp"

namespace lbm {

constexpr int ABLOCK = 256;

// Adjoint buffers (inside the caller's adjoint workspace).
struct Adj {
  float *lt_in, *lt_out;    // [Q][NFp] lambda of T: of x_t / of x_{t+1}
  float4 *ls_in, *ls_out;   // [NF] (lambda r, lambda v)
  float *lft;               // [Q][NFp] lambda of f^t after streaming
  float2 *lr;               // [NF] lambda of (rho^r, rho^b)
  float *lphi;              // [NF] lambda of phi
  float *lphis;             // [NS] lambda of the Eq. 34 phi
  float4 *ln;               // [NF] (lambda n, lambda |C|)
  float4 *lns;              // [NS] lambda of the Eq. 35 n
  float2 *ab;               // [NF] coefficients of the stream transpose
  double *acc;              // [4] dJ/dtheta, dJ/dg
  float freeze_sin;         // Scheme-II linearisation: see scheme2_adj
  float c_min;              // normalisation linearisation: see k_adj_gradient
};

__device__ __forceinline__ void atomic_add3(float4 *p, float x, float y,
                                            float z) {
  atomicAdd(&p->x, x);
  atomicAdd(&p->y, y);
  atomicAdd(&p->z, z);
}

// Sum over the warp, then one double atomic per warp.
__device__ __forceinline__ void warp_acc(double *dst, float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.f) atomicAdd(dst, (double)v);
}

// Red fraction r of the stored state of node k (from the encoding).
__device__ __forceinline__ float red_fraction(float q) {
  return m_blue(q) ? q : 1.f - q;
}

// A1: collision, force, curvature and recolouring reversed at fluid node
// k. Outputs lft, lr, lphi (own values), ln.w (lambda |C|), and adds the
// node's lambda n and the curvature transposes to ln / lns.
template <int Q>
__global__ void __launch_bounds__(ABLOCK) k_adj_collide(Dom d, Adj a) {
  const int k = blockIdx.x * ABLOCK + threadIdx.x;
  const bool live = k < d.NF;
  float lg[3] = {0.f, 0.f, 0.f};
  if (live) {
    using IO = TIO<Q, LBM_STORAGE_FP32>;
    // forward values of the step. The curvature stencil only where the
    // node has an interface: elsewhere |C| = 0, so kappa enters neither F
    // nor, through lambda kappa = gamma |C| lambda_hk / 2, any neighbour;
    // its lambda |C| is read only at nodes with an interface
    // (k_adj_gradient)
    const float4 c4 = d.ncf[k];
    float dn[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    if (c4.w != 0.f) {
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const uint32_t e = nb_f<Q>(d, i, k);
        const int idx = entry_idx(e);
        const float4 v = (entry_cls(e) & 2) ? d.ncf[idx] : d.ncs[idx];
        const float w3 = 3.f * Lattice<Q>::w(i);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const float eb = (float)Lattice<Q>::e(i, b);
          dn[0][b] += w3 * eb * v.x;
          dn[1][b] += w3 * eb * v.y;
          dn[2][b] += w3 * eb * v.z;
        }
      }
    }
    const float n[3] = {c4.x, c4.y, c4.z};
    const float Cm = c4.w;
    float kappa = 0.f;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        kappa += (n[p] * n[b] - (p == b ? 1.f : 0.f)) * dn[p][b];
    float ft[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) ft[i] = IO::load_from(d, d.U, i, k);
    const float2 R = d.R[k];
    const float rr = R.x, rb = R.y, rho = rr + rb;
    const float phi = m_phi(d.mf[k]);
    const float hk = 0.5f * d.c.gamma * kappa * Cm;
    float F[3], j[3] = {0.f, 0.f, 0.f}, u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) F[c] = hk * n[c] + rho * d.c.g[c];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      j[0] += (float)Lattice<Q>::ex(i) * ft[i];
      j[1] += (float)Lattice<Q>::ey(i) * ft[i];
      j[2] += (float)Lattice<Q>::ez(i) * ft[i];
    }
    const float irho = 1.f / rho;
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = (j[c] + 0.5f * F[c]) * irho;
    const float S = relaxation_rate(d.c, phi);
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    const float kf = 1.f - 0.5f * S;
    const float iE2 = 1.f / Lattice<Q>::E2;
    float B[3];  // b = S B
#pragma unroll
    for (int c = 0; c < 3; ++c)
      B[c] = (j[c] - d.c.rho0 * u[c] + 0.5f * F[c]) * iE2;
    // adjoints of the outputs
    const float4 lS = a.ls_out[k];  // (lambda r', lambda v')
    float lft[Q], lS_ = 0.f, lb[3] = {0.f, 0.f, 0.f}, lu[3] = {0.f, 0.f, 0.f},
          lF[3] = {0.f, 0.f, 0.f}, lrho = 0.f, luu = 0.f, luF = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float lT = a.lt_out[(long long)i * d.NFp + k];
      const float e3[3] = {(float)Lattice<Q>::ex(i), (float)Lattice<Q>::ey(i),
                           (float)Lattice<Q>::ez(i)};
      const float w = Lattice<Q>::w(i);
      const float eu = e3[0] * u[0] + e3[1] * u[1] + e3[2] * u[2];
      const float eF = e3[0] * F[0] + e3[1] * F[1] + e3[2] * F[2];
      const float feq = w * (rho + d.c.rho0 * (3.f * eu + 4.5f * eu * eu - 1.5f * uu));
      const float G = w * (3.f * (eF - uF) + 9.f * eu * eF);
      const float eB = e3[0] * B[0] + e3[1] * B[1] + e3[2] * B[2];
      // T'_i = ft_i - S (ft_i - feq_i) + (1 - S/2) G_i + S e_i.B
      lft[i] = lT * (1.f - S);
      lS_ += lT * (feq - ft[i] - 0.5f * G + eB);
      const float lfeq = lT * S, lG = lT * kf;
#pragma unroll
      for (int c = 0; c < 3; ++c) lb[c] += lT * S * e3[c];  // lambda of B
      lrho += lfeq * w;
      const float leu = lfeq * w * d.c.rho0 * (3.f + 9.f * eu) + lG * w * 9.f * eF;
      const float leF = lG * w * (3.f + 9.f * eu);
      luu += -1.5f * d.c.rho0 * lfeq * w;
      luF += -3.f * lG * w;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        lu[c] += leu * e3[c];
        lF[c] += leF * e3[c];
      }
    }
    // B = (j - rho0 u + F/2) / E2
    float lj[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      lu[c] += 2.f * u[c] * luu + F[c] * luF - d.c.rho0 * iE2 * lb[c];
      lF[c] += u[c] * luF + 0.5f * iE2 * lb[c];
      lj[c] = iE2 * lb[c];
    }
    // u = (j + F/2) / rho
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      lj[c] += lu[c] * irho;
      lF[c] += 0.5f * lu[c] * irho;
      lrho -= lu[c] * u[c] * irho;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i)
      lft[i] += (float)Lattice<Q>::ex(i) * lj[0] + (float)Lattice<Q>::ey(i) * lj[1] +
                (float)Lattice<Q>::ez(i) * lj[2];
    // S(phi), Eqs. (13)-(14): S = 1 / (3 / inv + 1/2)
    float lphi = 0.f;
    if (phi > -1.f && phi < 1.f) {
      const float inv = (1.f + phi) / (2.f * d.c.nu_r) + (1.f - phi) / (2.f * d.c.nu_b);
      const float dS_dinv = 3.f * S * S / (inv * inv);
      lphi = lS_ * dS_dinv * (0.5f / d.c.nu_r - 0.5f / d.c.nu_b);
    }
    // F = hk n + rho g, hk = gamma kappa |C| / 2
    const float lhk = n[0] * lF[0] + n[1] * lF[1] + n[2] * lF[2];
    float ln[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ln[c] = hk * lF[c];
      lrho += d.c.g[c] * lF[c];
      lg[c] = rho * lF[c];
    }
    const float lkappa = 0.5f * d.c.gamma * Cm * lhk;
    const float lCm = 0.5f * d.c.gamma * kappa * lhk;
    // recolouring outputs: r' = rr / rho, v' = beta rr rb / rho n
    const float seg = d.c.beta * rr * rb * irho;
    const float lseg = n[0] * lS.y + n[1] * lS.z + n[2] * lS.w;
    ln[0] += seg * lS.y;
    ln[1] += seg * lS.z;
    ln[2] += seg * lS.w;
    float lrr = lrho + lS.x * rb * irho * irho + lseg * d.c.beta * rb * rb * irho * irho;
    float lrb = lrho - lS.x * rr * irho * irho + lseg * d.c.beta * rr * rr * irho * irho;
    // kappa = sum_ab (n_a n_b - delta_ab) D_ab: own n, then the stencil
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float s = 0.f;
#pragma unroll
      for (int b = 0; b < 3; ++b) s += (dn[c][b] + dn[b][c]) * n[b];
      ln[c] += lkappa * s;
    }
    atomic_add3(a.ln + k, ln[0], ln[1], ln[2]);
    a.ln[k].w = lCm;  // only this thread writes the w component
    if (lkappa != 0.f) {
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const float e3[3] = {(float)Lattice<Q>::ex(i), (float)Lattice<Q>::ey(i),
                             (float)Lattice<Q>::ez(i)};
        const float en = e3[0] * n[0] + e3[1] * n[1] + e3[2] * n[2];
        const float c3 = 3.f * Lattice<Q>::w(i) * lkappa;
        const uint32_t e = nb_f<Q>(d, i, k);
        const int idx = entry_idx(e);
        float4 *dst = (entry_cls(e) & 2) ? a.ln + idx : a.lns + idx;
        atomic_add3(dst, c3 * (n[0] * en - e3[0]), c3 * (n[1] * en - e3[1]),
                    c3 * (n[2] * en - e3[2]));
      }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) a.lft[(long long)i * d.NFp + k] = lft[i];
    a.lr[k] = make_float2(lrr, lrb);
    a.lphi[k] = lphi;
  }
  warp_acc(a.acc + 1, lg[0]);
  warp_acc(a.acc + 2, lg[1]);
  warp_acc(a.acc + 3, lg[2]);
}

// A2: Eq. (35) reversed, n_s = sum_l w_l n(x_l) / sum_l w_l.
template <int Q>
__global__ void __launch_bounds__(ABLOCK) k_adj_nc_solid(Dom d, Adj a) {
  const int j = blockIdx.x * ABLOCK + threadIdx.x;
  if (j >= d.NS) return;
  const float4 l = a.lns[j];
  // nothing read this node's n_c (no fluid neighbour with an interface)
  if (l.x == 0.f && l.y == 0.f && l.z == 0.f) return;
  const int e = d.soff[j + 1];
  float W = 0.f;
  for (int p = d.soff[j]; p < e; ++p) W += link_w<Q>(d.slink[p]);
  const float iW = 1.f / W;
  for (int p = d.soff[j]; p < e; ++p) {
    const uint32_t lk = d.slink[p];
    const float c = link_w<Q>(lk) * iW;
    atomic_add3(a.ln + (lk & 0x7FFFFFFFu), c * l.x, c * l.y, c * l.z);
  }
}

// Scheme-II (Eqs. 32-33) reversed: given lambda of its output n, adds
// lambda of its input n_c to lnc and of theta (radians) to *lth. The
// forward choice between n+ and n- is kept (a discrete, locally constant
// decision); below EPS_SIN the scheme is the identity. The output is
// cos(theta) n_w +- sin(theta) t^ with t^ the direction of n_c's part
// across n_w; where sin(theta') = |n_c - cos(theta') n_w| < freeze_sin the
// derivative of t^ (which grows as 1/sin(theta')) is dropped and only the
// theta dependence is kept: the regularised linearisation (see Adj).
__device__ __forceinline__ void scheme2_adj(const float *nc, const float *nw,
                                            float cth, float sth,
                                            float freeze_sin,
                                            const float *lout, float *lnc,
                                            float *lth) {
  const float c0 = dot3(nw, nc);
  const float c = fminf(1.f, fmaxf(-1.f, c0));
  float t[3] = {nc[0] - c * nw[0], nc[1] - c * nw[1], nc[2] - c * nw[2]};
  const float sp = sqrtf(dot3(t, t));
  if (sp < EPS_SIN) {
    for (int q = 0; q < 3; ++q) lnc[q] += lout[q];
    return;
  }
  const float k = sth / sp;
  float dp = 0.f, dm = 0.f;
  for (int q = 0; q < 3; ++q) {
    const float np_ = cth * nw[q] + k * t[q], nm_ = cth * nw[q] - k * t[q];
    dp += (np_ - nc[q]) * (np_ - nc[q]);
    dm += (nm_ - nc[q]) * (nm_ - nc[q]);
  }
  const float s = dp <= dm ? 1.f : -1.f;
  const float th[3] = {t[0] / sp, t[1] / sp, t[2] / sp};
  // out = cos(theta) n_w + s sin(theta) t^, t^ = t / |t|, t = n_c - c n_w
  *lth += dot3(lout, nw) * (-sth) + s * cth * dot3(lout, th);
  if (sp < freeze_sin) return;
  float lt[3];
  const float lth_dot = s * sth * dot3(lout, th);
  for (int q = 0; q < 3; ++q) lt[q] = (s * sth * lout[q] - th[q] * lth_dot) / sp;
  const float lc = (c0 > -1.f && c0 < 1.f) ? -dot3(lt, nw) : 0.f;
  for (int q = 0; q < 3; ++q) lnc[q] += lt[q] + lc * nw[q];
}

// A3: normalisation (Eq. 11), wetting (Scheme-II) and the gradient stencil
// (Eq. 6) reversed at fluid node k; the stencil transposes to the phase
// field of the neighbours (fluid: lphi, solid-boundary: lphis).
template <int Q>
__global__ void __launch_bounds__(ABLOCK) k_adj_gradient(Dom d, Adj a) {
  const int k = blockIdx.x * ABLOCK + threadIdx.x;
  float lth = 0.f;
  // where the forward step found no interface (stored |C| = 0) n_c was held
  // at zero, so nothing flows back through the stencil
  if (k < d.NF && d.ncf[k].w != 0.f) {
    const bool own_blue = m_blue(d.mf[k]);
    float G[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t e = nb_f<Q>(d, i, k);
      const int idx = entry_idx(e);
      const float m = (entry_cls(e) & 2) ? d.mf[idx] : d.ms[idx];
      const float p = 3.f * Lattice<Q>::w(i) * m_excess(m, own_blue);
      G[0] += (float)Lattice<Q>::ex(i) * p;
      G[1] += (float)Lattice<Q>::ey(i) * p;
      G[2] += (float)Lattice<Q>::ez(i) * p;
    }
    const float Cm = sqrtf(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
    if (Cm > EPS_C) {
      const float4 l4 = a.ln[k];
      const float lout[3] = {l4.x, l4.y, l4.z};
      const float nc[3] = {G[0] / Cm, G[1] / Cm, G[2] / Cm};
      float lnc[3] = {0.f, 0.f, 0.f};
      bool wet = false;
      if (d.c.wetting == 2 && (d.fflag[k] & 1u)) {
        const float4 w4 = d.nw[k];
        const float nw[3] = {w4.x, w4.y, w4.z};
        if (nw[0] != 0.f || nw[1] != 0.f || nw[2] != 0.f) {
          scheme2_adj(nc, nw, d.c.cos_t, d.c.sin_t, a.freeze_sin, lout, lnc,
                      &lth);
          wet = true;
        }
      }
      if (!wet)
        for (int q = 0; q < 3; ++q) lnc[q] = lout[q];
      // n_c = C / |C|: its derivative grows as 1 / |C|; below c_min the
      // direction is held constant (regularised linearisation)
      const float nl = dot3(nc, lnc);
      const float kn = Cm < a.c_min ? 0.f : 1.f / Cm;
      float lC[3];
      for (int q = 0; q < 3; ++q) lC[q] = (lnc[q] - nc[q] * nl) * kn + nc[q] * l4.w;
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const float v = 3.f * Lattice<Q>::w(i) *
                        ((float)Lattice<Q>::ex(i) * lC[0] + (float)Lattice<Q>::ey(i) * lC[1] +
                         (float)Lattice<Q>::ez(i) * lC[2]);
        const uint32_t e = nb_f<Q>(d, i, k);
        const int idx = entry_idx(e);
        atomicAdd((entry_cls(e) & 2) ? a.lphi + idx : a.lphis + idx, v);
      }
    }
  }
  warp_acc(a.acc + 0, lth);
}

// A4: Eq. (34) reversed, phi_s = sum_l w_l phi(x_l) / sum_l w_l.
template <int Q>
__global__ void __launch_bounds__(ABLOCK) k_adj_phi_solid(Dom d, Adj a) {
  const int j = blockIdx.x * ABLOCK + threadIdx.x;
  if (j >= d.NS) return;
  const float l = a.lphis[j];
  if (l == 0.f) return;
  const int e = d.soff[j + 1];
  float W = 0.f;
  for (int p = d.soff[j]; p < e; ++p) W += link_w<Q>(d.slink[p]);
  const float iW = 1.f / W;
  for (int p = d.soff[j]; p < e; ++p) {
    const uint32_t lk = d.slink[p];
    atomicAdd(a.lphi + (lk & 0x7FFFFFFFu), link_w<Q>(lk) * iW * l);
  }
}

// A5: phi = (rho^r - rho^b) / (rho^r + rho^b) (Eq. 7) folded into the
// colour-density adjoints; ab = (lambda of every red part f^r_i,
// lambda added to every f^t_i), since rho^r = sum f^r_i and
// rho^b = sum f^t_i - rho^r.
__global__ void __launch_bounds__(ABLOCK) k_adj_prep(Dom d, Adj a) {
  const int k = blockIdx.x * ABLOCK + threadIdx.x;
  if (k >= d.NF) return;
  const float2 R = d.R[k];
  const float rho = R.x + R.y, i2 = 2.f / (rho * rho);
  const float lphi = a.lphi[k];
  const float2 lr = a.lr[k];
  const float lrr = lr.x + lphi * R.y * i2;
  const float lrb = lr.y - lphi * R.x * i2;
  a.ab[k] = make_float2(lrr - lrb, lrb);
}

// A6: streaming (Eq. 1) reversed at fluid node y. Its stored population k
// went to exactly one place: population k of y + e_k when that node is a
// fluid node inside the box, else population opp(k) of y itself (halfway
// bounce-back); there its red part was r(y) T_k(y) + w_k e_k.v(y).
template <int Q>
__global__ void __launch_bounds__(ABLOCK) k_adj_stream(Dom d, Adj a) {
  const int y = blockIdx.x * ABLOCK + threadIdx.x;
  if (y >= d.NF) return;
  using IO = TIO<Q, LBM_STORAGE_FP32>;
  const float4 S = d.S_src[y];
  const float r = red_fraction(S.x);
  float lr = 0.f, lv[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    int x = y, i = 0;
    if (k > 0) {
      const uint32_t e = nb_f<Q>(d, k, y);
      const bool fl = (entry_cls(e) & 2) && !entry_out(e);
      x = fl ? entry_idx(e) : y;
      i = fl ? k : Lattice<Q>::opp(k);
    }
    const float2 ab = a.ab[x];
    const float lft = a.lft[(long long)i * d.NFp + x];
    a.lt_in[(long long)k * d.NFp + y] = lft + ab.y + r * ab.x;
    lr += IO::load(d, k, y) * ab.x;
    const float wa = Lattice<Q>::w(k) * ab.x;
    lv[0] += wa * (float)Lattice<Q>::ex(k);
    lv[1] += wa * (float)Lattice<Q>::ey(k);
    lv[2] += wa * (float)Lattice<Q>::ez(k);
  }
  // the stored q is the minority fraction; lambda is taken w.r.t. r
  a.ls_in[y] = make_float4(lr, lv[0], lv[1], lv[2]);
}

// Seed of J = mean over the fluid nodes of (1 - phi)/2 with phi from the
// streamed populations (LBM_SW_SMOOTH): lambda phi = -1 / (2 N_f).
__global__ void __launch_bounds__(ABLOCK) k_adj_seed_sw(Dom d, Adj a, int Q) {
  const int k = blockIdx.x * ABLOCK + threadIdx.x;
  if (k >= d.NF) return;
  for (int i = 0; i < Q; ++i) a.lft[(long long)i * d.NFp + k] = 0.f;
  a.lr[k] = make_float2(0.f, 0.f);
  a.lphi[k] = -0.5f / (float)d.NF;
}

}  // namespace lbm

// ---------------------------------------------------------------- host
struct lbm_adj_s {
  lbm_ctx *c = nullptr;
  lbm::Adj a{};
  size_t ln_bytes = 0, lns_bytes = 0, lphis_bytes = 0;
  bool seeded = false;
  char err[256] = {0};
};

namespace {

struct AdjLayout {
  size_t lt_in, lt_out, ls_in, ls_out, lft, lr, lphi, lphis, ln, lns, ab, acc,
      total;
};

AdjLayout adj_layout(int Q, long long NFp, long long NS) {
  AdjLayout L{};
  const size_t nfp = (size_t)NFp, nsp = (size_t)(NS > 0 ? NS : 1);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = (o + bytes + 255) / 256 * 256;
    return at;
  };
  L.lt_in = take((size_t)Q * nfp * 4);
  L.lt_out = take((size_t)Q * nfp * 4);
  L.ls_in = take(nfp * 16);
  L.ls_out = take(nfp * 16);
  L.lft = take((size_t)Q * nfp * 4);
  L.lr = take(nfp * 8);
  L.lphi = take(nfp * 4);
  L.lphis = take(nsp * 4);
  L.ln = take(nfp * 16);
  L.lns = take(nsp * 16);
  L.ab = take(nfp * 8);
  L.acc = take(8 * 8);
  L.total = o;
  return L;
}

lbm_status afail(lbm_adj a, lbm_status st, const char *msg) {
  if (a) snprintf(a->err, sizeof(a->err), "%s", msg);
  return st;
}

void swap_lambda(lbm::Adj &a) {
  float *t = a.lt_in;
  a.lt_in = a.lt_out;
  a.lt_out = t;
  float4 *s = a.ls_in;
  a.ls_in = a.ls_out;
  a.ls_out = s;
}

unsigned blocks(long long n) { return (unsigned)((n + lbm::ABLOCK - 1) / lbm::ABLOCK); }

// A5 and A6: lambda(x_t) into lt_in / ls_in, then made the "out" side.
template <int Q>
void finish_t(lbm_adj a, cudaStream_t s) {
  const lbm::Dom &d = a->c->d;
  lbm::k_adj_prep<<<blocks(d.NF), lbm::ABLOCK, 0, s>>>(d, a->a);
  lbm::k_adj_stream<Q><<<blocks(d.NF), lbm::ABLOCK, 0, s>>>(d, a->a);
  swap_lambda(a->a);
}

template <int Q>
void step_t(lbm_adj a, cudaStream_t s) {
  const lbm::Dom &d = a->c->d;
  lbm::k_adj_collide<Q><<<blocks(d.NF), lbm::ABLOCK, 0, s>>>(d, a->a);
  if (d.NS > 0)
    lbm::k_adj_nc_solid<Q><<<blocks(d.NS), lbm::ABLOCK, 0, s>>>(d, a->a);
  lbm::k_adj_gradient<Q><<<blocks(d.NF), lbm::ABLOCK, 0, s>>>(d, a->a);
  if (d.NS > 0)
    lbm::k_adj_phi_solid<Q><<<blocks(d.NS), lbm::ABLOCK, 0, s>>>(d, a->a);
  finish_t<Q>(a, s);
}

}  // namespace

extern "C" {

size_t lbm_adj_workspace_bytes(lbm_handle h) {
  if (!h) return 0;
  return adj_layout(h->Q, h->d.NFp, h->d.NS).total;
}

lbm_status lbm_adj_create(lbm_adj *out, lbm_handle h, void *dev_workspace,
                          size_t ws_bytes) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  if (!h || !dev_workspace) return LBM_ERR_ARG;
  if (((uintptr_t)dev_workspace) % 256) return LBM_ERR_ARG;
  if (h->storage != LBM_STORAGE_FP32) return LBM_ERR_ARG;
  if (!h->params_set) return LBM_ERR_STATE;
  if (h->p.zou_he || h->p.wetting == 1 || h->p.collision) return LBM_ERR_ARG;
  const AdjLayout L = adj_layout(h->Q, h->d.NFp, h->d.NS);
  if (ws_bytes < L.total) return LBM_ERR_NOMEM;
  lbm_adj a = new (std::nothrow) lbm_adj_s();
  if (!a) return LBM_ERR_NOMEM;
  char *b = (char *)dev_workspace;
  a->c = h;
  a->a.lt_in = (float *)(b + L.lt_in);
  a->a.lt_out = (float *)(b + L.lt_out);
  a->a.ls_in = (float4 *)(b + L.ls_in);
  a->a.ls_out = (float4 *)(b + L.ls_out);
  a->a.lft = (float *)(b + L.lft);
  a->a.lr = (float2 *)(b + L.lr);
  a->a.lphi = (float *)(b + L.lphi);
  a->a.lphis = (float *)(b + L.lphis);
  a->a.ln = (float4 *)(b + L.ln);
  a->a.lns = (float4 *)(b + L.lns);
  a->a.ab = (float2 *)(b + L.ab);
  a->a.acc = (double *)(b + L.acc);
  a->a.freeze_sin = 0.05f;
  a->a.c_min = 1e-3f;
  a->ln_bytes = L.lns - L.ln;
  a->lns_bytes = L.ab - L.lns;
  a->lphis_bytes = L.ln - L.lphis;
  *out = a;
  return LBM_OK;
}

lbm_status lbm_adj_seed_sw(lbm_adj a, void *stream) {
  if (!a) return LBM_ERR_ARG;
  lbm_ctx *c = a->c;
  if (!c->state_set) return afail(a, LBM_ERR_STATE, "the handle has no state");
  if (c->p.zou_he || c->p.wetting == 1 || c->p.collision ||
      c->storage != LBM_STORAGE_FP32)
    return afail(a, LBM_ERR_ARG, "parameters outside the adjoint's scope");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(a->a.acc, 0, 8 * sizeof(double), s);
  if (e != cudaSuccess) return afail(a, LBM_ERR_CUDA, cudaGetErrorString(e));
  lbm::launch_fields(c->Q, c->storage, c->d, s);
  lbm::k_adj_seed_sw<<<blocks(c->d.NF), lbm::ABLOCK, 0, s>>>(c->d, a->a, c->Q);
  if (c->Q == 19) finish_t<19>(a, s);
  else finish_t<9>(a, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return afail(a, LBM_ERR_CUDA, cudaGetErrorString(e));
  a->seeded = true;
  return LBM_OK;
}

lbm_status lbm_adj_step(lbm_adj a, void *stream) {
  if (!a) return LBM_ERR_ARG;
  if (!a->seeded) return afail(a, LBM_ERR_STATE, "seed the adjoint first");
  lbm_ctx *c = a->c;
  if (c->p.zou_he || c->p.wetting == 1 || c->p.collision ||
      c->storage != LBM_STORAGE_FP32)
    return afail(a, LBM_ERR_ARG, "parameters outside the adjoint's scope");
  cudaStream_t s = (cudaStream_t)stream;
  lbm::launch_fields(c->Q, c->storage, c->d, s);
  cudaError_t e = cudaMemsetAsync(a->a.ln, 0, a->ln_bytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a->a.lns, 0, a->lns_bytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a->a.lphis, 0, a->lphis_bytes, s);
  if (e != cudaSuccess) return afail(a, LBM_ERR_CUDA, cudaGetErrorString(e));
  if (c->Q == 19) step_t<19>(a, s);
  else step_t<9>(a, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return afail(a, LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_adj_gradients(lbm_adj a, double *out4, void *stream) {
  if (!a || !out4) return LBM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(out4, a->a.acc, 4 * sizeof(double),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return afail(a, LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_adj_get_lambda(lbm_adj a, float *lt_dev, float *ls_dev,
                              void *stream) {
  if (!a || !lt_dev || !ls_dev) return LBM_ERR_ARG;
  const lbm::Dom &d = a->c->d;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(lt_dev, a->a.lt_out,
                                  sizeof(float) * a->c->Q * (size_t)d.NFp,
                                  cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ls_dev, a->a.ls_out, sizeof(float4) * (size_t)d.NF,
                        cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return afail(a, LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_adj_set_freeze(lbm_adj a, double freeze_sin) {
  if (!a || !(freeze_sin >= 0.0) || freeze_sin > 1.0) return LBM_ERR_ARG;
  a->a.freeze_sin = (float)freeze_sin;
  return LBM_OK;
}

lbm_status lbm_adj_set_cmin(lbm_adj a, double c_min) {
  if (!a || !(c_min >= 0.0) || c_min > 10.0) return LBM_ERR_ARG;
  a->a.c_min = (float)c_min;
  return LBM_OK;
}

const char *lbm_adj_last_error(lbm_adj a) { return a ? a->err : "null adjoint"; }

void lbm_adj_destroy(lbm_adj a) { delete a; }

}  // extern "C"
