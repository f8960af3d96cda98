// The work of one node in each pass of the time step, shared by the
// per-domain kernels (step.cu) and the batched kernels (batch.cu). The
// passes, in order; each needs the previous one's values at lattice
// neighbours:
//   stream_node     (fluid)  pull of Eq. (1), Eqs. (7)-(9): stores f^t,
//                   (rho^r, rho^b) and the phase field;
//   zh_fix_node     (Zou-He plane nodes) App. B in totals;
//   phi_solid_node  (solid-boundary) Eq. (34);
//   gradient_node   (fluid)  Eqs. (6), (27) and wetting, Eqs. (28)-(33);
//   nc_solid_node   (solid-boundary) Eq. (35);
//   collide_node    (fluid)  Eq. (12), (5), (36); Eq. (2) single-rate on
//                   the stored f^t; stores f'' and (q, v), the recoloured
//                   state of Eqs. (20)-(21).
// Every lattice neighbour of a fluid node is one read of the dense entry box
// (geometry.cu) at the node's padded index plus a fixed offset. COH selects
// loads that bypass L1 for the values that change within a step (see ldv).
#pragma once

#include "tiles.cuh"

namespace lbm {

// Entry of the lattice neighbour x + e_dir of fluid node k.
template <int Q>
__device__ __forceinline__ uint32_t nb_f(const Dom &d, int dir, int k) {
  return nb_entry<Q>(d, __ldg(d.fgp + k), dir);
}

// Weight of a solid-boundary link (bit 31: diagonal direction).
template <int Q>
__device__ __forceinline__ float link_w(uint32_t l) {
  return (l >> 31) ? Lattice<Q>::w(Q - 1) : Lattice<Q>::w(1);
}

// Streamed populations of fluid node k (Eq. 1), their colour densities and
// the encoded phase field (Eqs. 7-9). On the Zou-He planes the populations
// from outside the box are placeholders until zh_fix_node.
template <int Q, int ST, bool COH>
__device__ __forceinline__ void stream_node(const Dom &d, int k) {
  float ft[Q], rr, rb;
  const int gp = __ldg(d.fgp + k);
  pull_sums<Q, ST, COH>(d, k, gp, ldv<COH>(d.S_src + k), ft, rr, rb);
#pragma unroll
  for (int i = 0; i < Q; ++i) TIO<Q, ST>::store(d, d.U, i, k, ft[i]);
  d.R[k] = make_float2(rr, rb);
  const float m = m_of(rr, rb);
  d.mf[k] = m;
  dense_store<Q>(d, d.phib, gp, __ldg(d.fflag + k), m);
}

// App. B in totals on the pulled f^t of a Zou-He plane node, shared by both
// step schedules. Its per-colour rules are linear in the populations, and
// the collision needs only f^t = f^r + f^b and rho^r, rho^b, so the unknown
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
// red sums K0^r, Kin^r come from the pull's colour split. m: the node's
// phase field (Eq. 39's value at the outlet); Sown its (q, v). srcS(i, fl),
// for a known direction i > 0 with e_i.a >= 0, returns the (q, v) of the node
// the pull took f_i from and sets fl when that node is a fluid source (else
// it is the node itself, by bounce-back). ft is updated in place (the
// unknowns only).
template <int Q, class SrcS>
__device__ __forceinline__ void zou_he_totals(const StepConst &cc, float *ft,
                                              bool inlet, float m, float4 Sown,
                                              SrcS srcS, float &rr, float &rb) {
  const int a = cc.axis;
  const int in_dir = inlet ? -1 : 1;  // e.a of the known, inward populations
  // K0, Kin and N_t from the deviations f_i - w_i rho0 (exact in float32,
  // and small): the weights of the known populations add up to
  // sum_{e.a=0} w + 2 sum_{e.a=in} w = 1 and sum_{e.a=0} (e.t) w = 0, so
  // j = (rho_in - rho0) - (K0d + 2 Kind) keeps the precision of the
  // deviations instead of cancelling two numbers near one.
  float K0 = 0.f, Kin = 0.f, K0d = 0.f, Kind = 0.f, N[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int ea = Lattice<Q>::e(i, a);
    const float dv = __fsub_rn(ft[i], __fmul_rn(Lattice<Q>::w(i), cc.rho0));
    if (ea == 0) {
      K0 = __fadd_rn(K0, ft[i]);
      K0d = __fadd_rn(K0d, dv);
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const int et = Lattice<Q>::e(i, t);
        if (t != a && et) N[t] = __fadd_rn(N[t], __fmul_rn(et > 0 ? 0.5f : -0.5f, dv));
      }
    } else if (ea == in_dir) {
      Kin = __fadd_rn(Kin, ft[i]);
      Kind = __fadd_rn(Kind, dv);
    }
  }
  float jt;
  if (inlet) {
    jt = __fsub_rn(__fsub_rn(__fadd_rn(cc.rho_in_r, cc.rho_in_b), cc.rho0),
                   __fmaf_rn(2.f, Kind, K0d));
    rr = cc.rho_in_r;
    rb = cc.rho_in_b;
  } else {
    jt = __fsub_rn(__fmaf_rn(2.f, Kind, K0d), __fsub_rn(cc.rho_out, cc.rho0));
    // red parts of the known populations (e.a >= 0), as the pull split them
    float K0r = 0.f, Kinr = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int ea = Lattice<Q>::e(i, a);
      if (ea < 0) continue;
      float fr, fb;
      if (i == 0) {
        rebuild<Q>(ft[0], Sown, 0, fr, fb);
      } else {
        bool fl;
        const float4 S = srcS(i, fl);
        const float ev = edot<Q>(i, S.y, S.z, S.w);
        rebuild_ev<Q>(ft[i], S.x, fl ? ev : -ev, i, fr, fb);
      }
      if (ea == 0) K0r = __fadd_rn(K0r, fr);
      else Kinr = __fadd_rn(Kinr, fr);
    }
    const float chi_r = __fmul_rn(0.5f, __fadd_rn(1.f, m_phi(m)));
    rr = __fsub_rn(__fmaf_rn(2.f, Kinr, K0r), __fmul_rn(jt, chi_r));
    rb = __fsub_rn(__fmaf_rn(2.f, __fsub_rn(Kin, Kinr), __fsub_rn(K0, K0r)),
                   __fmul_rn(jt, __fsub_rn(1.f, chi_r)));
    jt = -jt;  // the outlet rule subtracts 6 w_i j
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (Lattice<Q>::e(i, a) != -in_dir) continue;
    float corr = 0.f;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int et = Lattice<Q>::e(i, t);
      if (t != a && et) corr = __fadd_rn(corr, et > 0 ? N[t] : -N[t]);
    }
    ft[i] = __fsub_rn(__fmaf_rn(6.f * Lattice<Q>::w(i), jt, ft[Lattice<Q>::opp(i)]),
                      corr);
  }
}

// App. B on the Zou-He planes (node jz of their list), after stream_node:
// the unknown populations and the colour densities stored back into U and
// R, and the planes' phase field: zeta^r - zeta^b at the inlet, phi(x - a)
// (Eq. 39) at the outlet (the node's own value if that node is solid).
template <int Q, int ST, bool COH>
__device__ __forceinline__ void zh_fix_node(const Dom &d, int jz) {
  // U and R of the node are read and then rewritten by this thread: never
  // through the read-only path
  using IO = TIO<Q, ST, true>;
  const int k = guard(d, __ldg(d.zh_list + jz), d.NF, GUARD_ZOU_HE);
  const int gp = __ldg(d.fgp + k);
  const int a = d.c.axis;
  const bool inlet = __ldg(d.fflag + k) & (2u << (2 * a));
  float ft[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) ft[i] = IO::load_from(d, d.U, i, k);
  float m;
  if (inlet) {
    m = d.c.m_in;
  } else {
    const int sa = a == 0 ? 1 : (a == 1 ? d.px : d.px * d.py);
    const uint32_t e = __ldg(
        d.nbd + guard(d, gp - sa, d.px * d.py * (d.nz + 2), GUARD_ZOU_HE));
    const float2 Rk = ldv<true>(d.R + k);
    m = ((entry_cls(e) & 2) && !entry_out(e))
            ? ldv<COH>(d.mf + guard(d, entry_idx(e), d.NF, GUARD_ZOU_HE))
            : m_of(Rk.x, Rk.y);
  }
  const float4 Sown = ldv<COH>(d.S_src + k);
  auto srcS = [&](int i, bool &fl) {
    const uint32_t es = nb_entry<Q>(d, gp, Lattice<Q>::opp(i));
    fl = (entry_cls(es) & 2) && !entry_out(es);
    return fl ? ldv<COH>(d.S_src + guard(d, entry_idx(es), d.NF, GUARD_ZOU_HE))
              : Sown;
  };
  float rr, rb;
  zou_he_totals<Q>(d.c, ft, inlet, m, Sown, srcS, rr, rb);
  const int in_dir = inlet ? -1 : 1;
#pragma unroll
  for (int i = 0; i < Q; ++i)
    if (Lattice<Q>::e(i, a) == -in_dir) IO::store(d, d.U, i, k, ft[i]);
  d.R[k] = make_float2(rr, rb);
  d.mf[k] = m;
  dense_store<Q>(d, d.phib, gp, __ldg(d.fflag + k), m);
}

// Eq. (34): phi at solid-boundary node j = w-weighted mean over its fluid
// lattice neighbours, kept in the encoded form: the mean of phi - s for the
// sign s of the mean.
template <int Q, bool COH>
__device__ __forceinline__ void phi_solid_node(const Dom &d, int j) {
  // the fluid neighbours' phase from the dense box at fixed offsets, in
  // the order of the node's links (ascending direction): one round of
  // independent loads instead of a walk over the link list
  const uint32_t dirs = __ldg(d.sdir + j);
  const int gp = __ldg(d.sgp + j);
  Eq34 acc;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    if (!(dirs & (1u << i))) continue;
    acc.add(Lattice<Q>::w(i),
            ldv<COH>(d.phib + guard(d, gp + dense_off<Q>(d, i),
                                    d.px * d.py * (d.nz + 2), GUARD_STENCIL)));
  }
  const float ms = acc.finish();
  d.ms[j] = ms;
  dense_store<Q>(d, d.phib, __ldg(d.sgp + j), __ldg(d.sflag + j), ms);
}

// Eq. (6) (c = dt = 1) and Eq. (27) at fluid node k, with phi(x + e_i) -
// s(x) in place of phi(x + e_i) (the same sum since sum_i w_i e_i = 0),
// off-box neighbours clamped; at fluid-boundary nodes the wetting scheme
// turns n_c, keeping |C|. Stored: (n_c, |C|), or zero where |C| <= EPS_C
// (no interface). MARK: a fluid-boundary node with an interface marks its
// solid-boundary neighbours (smark), whose Eq. (35) n_c its curvature
// stencil will read.
template <int Q, bool COH, bool MARK = false>
__device__ __forceinline__ void gradient_node(const Dom &d, int k) {
  // the neighbours' phase from the dense box at fixed offsets (the nodes the
  // dense entry box names: fluid, solid-boundary, or the halo cell of a
  // wrapped or clamped neighbour)
  const int gp = __ldg(d.fgp + k);
  const bool own_blue = m_blue(ldv<COH>(d.mf + k));
  Grad<Q> g;
#pragma unroll
  for (int i = 1; i < Q; ++i)
    g.add(i,
          ldv<COH>(d.phib + guard(d, gp + dense_off<Q>(d, i),
                                  d.px * d.py * (d.nz + 2), GUARD_STENCIL)),
          own_blue);
  const bool fbnd = (__ldg(d.fflag + k) & 1u) != 0;
  const float4 c4 = normal_and_wetting(d.c, g, fbnd, d.nw + k);
  d.ncf[k] = c4;
  if (MARK && fbnd && c4.w != 0.f) {
    // all entry loads issued together (one round trip)
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t e = nb_entry<Q>(d, gp, i);
      if (entry_cls(e) == CLS_SOLID_BND)
        d.smark[guard(d, entry_idx(e), d.NS, GUARD_STENCIL)] = 1;
    }
  }
}

// Eq. (35): n_c at solid-boundary node j = w-weighted mean of the fluid
// neighbours' (post-wetting) n_c, not renormalised.
template <int Q, bool COH>
__device__ __forceinline__ float4 eq35_at(const Dom &d, int j) {
  Eq35 acc;
  const int e = __ldg(d.soff + j + 1);
  for (int p = __ldg(d.soff + j); p < e; ++p) {
    const uint32_t l =
        __ldg(d.slink + guard(d, p, (Q - 1) * d.NS, GUARD_LINK));
    const float4 v =
        ldv<COH>(d.ncf + guard(d, (int)(l & 0x7FFFFFFFu), d.NF, GUARD_LINK));
    acc.add(link_w<Q>(l), v.x, v.y, v.z);
  }
  return acc.finish();
}

template <int Q, bool COH>
__device__ __forceinline__ void nc_solid_node(const Dom &d, int j) {
  d.ncs[j] = eq35_at<Q, COH>(d, j);
}

// Eq. (35) only where the step's curvature stencil will read it: at the
// solid-boundary nodes the gradient pass marked (the neighbours of
// fluid-boundary nodes with an interface; the curvature runs at no other
// node, and Eq. 35 of a node whose fluid neighbours all lack an interface
// is zero). The mark is cleared for the next step.
template <int Q>
__device__ __forceinline__ void nc_solid_marked_node(const Dom &d, int j) {
  if (!d.smark[j]) return;
  d.smark[j] = 0;
  d.ncs[j] = eq35_at<Q, false>(d, j);
}

// Eq. (12) with d_b n_a by the Eq. (6) stencil on each component (off-box
// neighbours clamped); returns kappa and the node's (n_c, |C|).
template <int Q, bool COH>
__device__ __forceinline__ float curvature(const Dom &d, int k, float4 &c4) {
  // kappa enters the step only through F = 1/2 gamma kappa |C| n_c (Eq. 5).
  // A node with no interface (|C| <= EPS_C) stores (n_c, |C|) = 0, so its
  // surface force is zero whatever kappa is: the stencil is skipped there
  // and kappa = 0 stored (the force, hence every population, is the same
  // bit for bit).
  c4 = ldv<COH>(d.ncf + k);
  if (c4.w == 0.f) return 0.f;
  Curv<Q> cv;
  // n_c from the compact lists through the dense entry box: a dense copy of
  // n_c (as the phase field has) was measured slower, 0.293 against 0.265 ms
  // for the collision: a 16-byte gather from the dense box touches about 3.7
  // times more sectors than from the compact fluid list on the 256^3 rock
  const int gp = __ldg(d.fgp + k);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const uint32_t e = nb_entry<Q>(d, gp, i);
    const bool fl = entry_cls(e) & 2;
    const int idx = guard(d, entry_idx(e), fl ? d.NF : d.NS, GUARD_STENCIL);
    const float4 v = fl ? ldv<COH>(d.ncf + idx) : ldv<COH>(d.ncs + idx);
    cv.add(i, v.x, v.y, v.z);
  }
  return cv.kappa(c4.x, c4.y, c4.z);
}

// Eq. (12) at fluid node k, stored for the collision pass.
template <int Q, bool COH>
__device__ __forceinline__ void curvature_node(const Dom &d, int k) {
  float4 c4;
  const float kappa = curvature<Q, COH>(d, k, c4);
  // stored only where the collision reads it back (a node with an interface)
  if (c4.w != 0.f) d.kap[k] = kappa;
}

// Eq. (5) F = 1/2 gamma kappa C (C = |C| n_c) plus rho g (Eq. 36), the
// collision (Eq. 2) of the stored f^t, and the store of the recoloured
// state of fluid node k: f''_i and (q, v) with q the encoded rho^r/rho and
// v = beta rho^r rho^b / rho n (Eqs. 20-21). The relaxation rate follows
// the node's phase field (Eq. 39's value on the outlet plane).
// KAP: the curvature was stored by curvature_node (the same float, so both
// forms agree bit for bit); else it is computed here.
template <int Q, int ST, bool MACROS, bool COH, int MRT = -1, bool KAP = false>
__device__ __forceinline__ void collide_node(const Dom &d, int k) {
  using IO = TIO<Q, ST, COH>;
  float4 c4;
  float kappa;
  if (KAP) {
    // kappa is stored only at nodes with an interface; elsewhere the
    // surface force is zero (c4 = 0) and kappa = 0 as curvature() gives it.
    // Both loads are issued together and the select discards the stale
    // value (a load that waited for c4 made the pass 4 % slower).
    c4 = ldv<COH>(d.ncf + k);
    const float stored = ldv<COH>(d.kap + k);
    kappa = c4.w == 0.f ? 0.f : stored;
  } else {
    kappa = curvature<Q, COH>(d, k, c4);
  }
  float ft[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) ft[i] = IO::load_from(d, d.U, i, k);
  const float2 R = ldv<COH>(d.R + k);
  const float rr = R.x, rb = R.y;
  float F[3], u[3];
  const float rho = force(d.c, rr, rb, kappa, c4, F);
  collide<Q, MRT>(d.c, ft, rho, F, m_phi(ldv<COH>(d.mf + k)), u);
#pragma unroll
  for (int i = 0; i < Q; ++i) IO::store(d, d.T_dst, i, k, ft[i]);
  d.S_dst[k] = recoloured_split(d.c, rr, rb, rho, c4);
  if (MACROS) d.macro[k] = make_float4(u[0], u[1], u[2], rho);
}

}  // namespace lbm
