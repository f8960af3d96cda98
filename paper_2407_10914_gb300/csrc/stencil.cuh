// Device building blocks of the step: coordinates, the encoded phase field,
// the storage of the post-recolouring populations and their rebuild, Zou-He
// (App. B), the wetting schemes (Eqs. 28-33) and the collision (Eq. 2,
// single-rate form). All arithmetic is FP32. The neighbour lookup and the
// pull of Eq. (1) are in tiles.cuh.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "context.hpp"
#include "lattice.cuh"

namespace lbm {

constexpr float EPS_C = 1e-8f;        // |C| at or below: no interface
constexpr float EPS_SIN = 1e-6f;      // Scheme-II: n_c parallel to n_w
constexpr float EPS_SECANT = 1e-12f;  // Scheme-I: secant denominator

// ------------------------------------------------------ coordinates
// Box sizes stay below 2^31 nodes, so index arithmetic is 32-bit.
__device__ __forceinline__ void box_coords(const Dom &d, int g, int &x,
                                           int &y, int &z) {
  const unsigned q = (unsigned)g / (unsigned)d.nx;
  x = g - (int)q * d.nx;
  z = (int)(q / (unsigned)d.ny);
  y = (int)q - z * d.ny;
}

// Coordinate v + dv (|dv| <= 1) on an axis of extent m. Periodic axes wrap;
// otherwise an out-of-box value sets `out` (clamp = false) or is clamped.
__device__ __forceinline__ int axis_step(int v, int m, bool per, bool clamp,
                                         bool &out) {
  if (v < 0) {
    if (per) return v + m;
    if (!clamp) out = true;
    return 0;
  }
  if (v >= m) {
    if (per) return v - m;
    if (!clamp) out = true;
    return m - 1;
  }
  return v;
}

// ------------------------------------------------------ index guards
// Every gathered index goes through guard(). In a build with
// LBM_BOUNDS_CHECK defined (build.build(check=True): liblbmgb_check.so) an
// index outside [0, bound) sets `code` in the domain's error word
// (lbm_debug_flags) and is replaced by 0, so that the access stays inside
// its array; in the normal build guard() is the identity. This stands in
// for a memory checker, which this GPU pool does not offer.
enum : unsigned {
  GUARD_PULL = 1u,      // a pull source (F-space)
  GUARD_STENCIL = 2u,   // a stencil neighbour (F- or S-space)
  GUARD_ZOU_HE = 4u,    // a Zou-He plane node or its x - a neighbour
  GUARD_LINK = 8u,      // a solid-boundary link or its CSR offsets
};
__device__ __forceinline__ int guard(const Dom &d, int idx, int bound,
                                     unsigned code) {
#ifdef LBM_BOUNDS_CHECK
  if ((unsigned)idx >= (unsigned)bound) {
    atomicOr(d.err, code);
    return 0;
  }
#else
  (void)d;
  (void)bound;
  (void)code;
#endif
  return idx;
}

// ------------------------------------------------------ dense fields
// A node's value v in a dense box with a one-node halo (padded index gp),
// and in the halo cells that stand for it: on a periodic axis a node of the
// first plane is also the cell past the last plane and a node of the last
// plane the cell before the first; on a non-periodic axis the stencils use
// the clamped node, so each face node also fills the halo cell beside it.
// Edge and corner nodes fill every combination. flags: face bits as fflag
// (bit 1 + 2a first plane, 2 + 2a last plane of axis a). D2Q9 never reads
// across z, so its z halo is left alone.
template <int Q, class T>
__device__ __forceinline__ void dense_store(const Dom &d, T *arr, int gp,
                                            unsigned flags, T v) {
  arr[gp] = v;
  if (!(flags & 0x7Eu)) return;
  const int stride[3] = {1, d.px, d.px * d.py};
  const int ext[3] = {d.nx, d.ny, d.nz};
  int off[3][3], n[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    n[a] = 1;
    off[a][0] = 0;
    if (Q == 9 && a == 2) continue;
    const bool per = d.periodic & (1u << a);
    if (flags & (2u << (2 * a))) off[a][n[a]++] = per ? ext[a] * stride[a] : -stride[a];
    if (flags & (4u << (2 * a))) off[a][n[a]++] = per ? -ext[a] * stride[a] : stride[a];
  }
  // fixed bounds, fully unrolled: the offsets stay in registers
#pragma unroll
  for (int ia = 0; ia < 3; ++ia)
#pragma unroll
    for (int ib = 0; ib < 3; ++ib)
#pragma unroll
      for (int ic = 0; ic < 3; ++ic)
        if ((ia | ib | ic) && ia < n[0] && ib < n[1] && ic < n[2])
          arr[gp + off[0][ia] + off[1][ib] + off[2][ic]] = v;
}

// Offset of the neighbour x + e_i in the padded box.
template <int Q>
__device__ __forceinline__ int dense_off(const Dom &d, int i) {
  return Lattice<Q>::ex(i) + d.px * (Lattice<Q>::ey(i) + d.py * Lattice<Q>::ez(i));
}

// ------------------------------------------------------ phase encoding
// A node's colour split is kept as one float m: the minority fraction
// mu = min(rho^r, rho^b)/rho with its own sign (it can be slightly negative,
// like the colour density it comes from), and, in the lowest mantissa bit,
// which colour is the majority (1 = blue, i.e. phi < 0). Then
// phi = 1 - 2 mu (red majority) or 2 mu - 1 (blue majority), and
// phi - sign(phi) keeps float32 relative accuracy near the pure phases.
// Stealing the bit costs one unit in the last place of mu.
__device__ __forceinline__ float m_pack(bool blue, float mu) {
  return __uint_as_float((__float_as_uint(mu) & ~1u) | (blue ? 1u : 0u));
}
__device__ __forceinline__ bool m_blue(float m) {
  return __float_as_uint(m) & 1u;
}
__device__ __forceinline__ float m_of(float rr, float rb) {
  return m_pack(rr < rb, fminf(rr, rb) / (rr + rb));
}
__device__ __forceinline__ float m_phi(float m) {
  return m_blue(m) ? 2.f * m - 1.f : 1.f - 2.f * m;
}
// phi(nb) - s, s = -1 if own_blue else +1, to full relative accuracy.
__device__ __forceinline__ float m_excess(float m_nb, bool own_blue) {
  const float mag = (m_blue(m_nb) == own_blue) ? m_nb : 1.f - m_nb;
  return own_blue ? 2.f * mag : -2.f * mag;
}

// ------------------------------------------------------------ storage
// Weight of a run-time direction index (a select on the three shells).
template <int Q>
__device__ __forceinline__ float weight_of(int p) {
  return p == 0 ? Lattice<Q>::w(0)
                : (p <= (Q == 19 ? 6 : 4) ? Lattice<Q>::w(1) : Lattice<Q>::w(Q - 1));
}

// Loads of values that change from step to step. A kernel that never
// writes what it reads takes them through the read-only path (__ldg). The
// persistent batch kernel runs several passes in one launch, so it reads
// values that other blocks wrote earlier in the same launch: COH = true,
// plain coherent loads (ld.global.ca), never the read-only path. Each of
// its work items starts after an acquire (and a fence) by one thread and a
// block barrier, which order these loads after the writes they depend on.
template <bool COH, class T>
__device__ __forceinline__ T ldv(const T *p) {
  if constexpr (COH)
    return __ldca(p);
  else
    return __ldg(p);
}

// f''_i planes: float32, or 16-bit (f''_i/w_i - rho0) so that the stored
// numbers are O(1e-2) deviations; arithmetic stays FP32.
template <int Q, int ST, bool COH = false>
struct TIO;

template <int Q, bool COH>
struct TIO<Q, LBM_STORAGE_FP32, COH> {
  __device__ __forceinline__ static float load_from(const Dom &d,
                                                   const void *buf, int i,
                                                   int k) {
    return ldv<COH>((const float *)buf + (long long)i * d.NFp + k);
  }
  __device__ __forceinline__ static float load(const Dom &d, int i, int k) {
    return load_from(d, d.T_src, i, k);
  }
  // plane p chosen at run time, p in {i, opp(i)} (equal weights)
  __device__ __forceinline__ static float load_dyn(const Dom &d, int p, int k) {
    return ldv<COH>((const float *)d.T_src + (long long)p * d.NFp + k);
  }
  __device__ __forceinline__ static void store(const Dom &d, void *T, int i,
                                               int k, float v) {
    ((float *)T)[(long long)i * d.NFp + k] = v;
  }
};

template <int Q, bool COH>
struct TIO<Q, LBM_STORAGE_FP16, COH> {
  __device__ __forceinline__ static float load_from(const Dom &d,
                                                   const void *buf, int i,
                                                   int k) {
    const __half h = ldv<COH>((const __half *)buf + (long long)i * d.NFp + k);
    return Lattice<Q>::w(i) * (__half2float(h) + d.c.rho0);
  }
  __device__ __forceinline__ static float load(const Dom &d, int i, int k) {
    return load_from(d, d.T_src, i, k);
  }
  // plane p at run time with the weight of w(p) = w(i) supplied by caller's i
  __device__ __forceinline__ static float load_dyn(const Dom &d, int p, int k) {
    const __half h = ldv<COH>((const __half *)d.T_src + (long long)p * d.NFp + k);
    return weight_of<Q>(p) * (__half2float(h) + d.c.rho0);
  }
  __device__ __forceinline__ static void store(const Dom &d, void *T, int i,
                                               int k, float v) {
    ((__half *)T)[(long long)i * d.NFp + k] =
        __float2half_rn(v * (1.f / Lattice<Q>::w(i)) - d.c.rho0);
  }
};

template <int Q, bool COH>
struct TIO<Q, LBM_STORAGE_BF16, COH> {
  __device__ __forceinline__ static float load_from(const Dom &d,
                                                   const void *buf, int i,
                                                   int k) {
    const __nv_bfloat16 h =
        ldv<COH>((const __nv_bfloat16 *)buf + (long long)i * d.NFp + k);
    return Lattice<Q>::w(i) * (__bfloat162float(h) + d.c.rho0);
  }
  __device__ __forceinline__ static float load(const Dom &d, int i, int k) {
    return load_from(d, d.T_src, i, k);
  }
  __device__ __forceinline__ static float load_dyn(const Dom &d, int p, int k) {
    const __nv_bfloat16 h =
        ldv<COH>((const __nv_bfloat16 *)d.T_src + (long long)p * d.NFp + k);
    return weight_of<Q>(p) * (__bfloat162float(h) + d.c.rho0);
  }
  __device__ __forceinline__ static void store(const Dom &d, void *T, int i,
                                               int k, float v) {
    ((__nv_bfloat16 *)T)[(long long)i * d.NFp + k] =
        __float2bfloat16_rn(v * (1.f / Lattice<Q>::w(i)) - d.c.rho0);
  }
};

// Rebuild f^r'_i, f^b'_i of a node from its f''_i and (q, v), Eqs. (20)-(21):
// with ev = e_i.v, the minority colour is mu f''_i -+ w_i ev (exact up to
// rounding, and to full relative accuracy when that colour is scarce), the
// majority the rest.
// Every helper from here on fixes its rounding: each product and sum is one
// explicit IEEE operation (__fmul_rn, __fadd_rn, __fsub_rn and __fmaf_rn are
// never fused or reassociated by the compiler). The kernels of both step
// schedules, the batch and the set-up inline them, so they all compute the
// same float32 numbers bit for bit; left to the compiler, a*b + c may be
// fused in one kernel and not in another.
//
// e_i . (a, b, c): the components of e_i are 0 or +-1, so the dot product
// is a signed sum of at most three of a, b, c, in axis order.
template <int Q>
__device__ __forceinline__ float edot(int i, float a, float b, float c) {
  const int ex = Lattice<Q>::ex(i), ey = Lattice<Q>::ey(i), ez = Lattice<Q>::ez(i);
  float s = ex ? (ex > 0 ? a : -a) : 0.f;
  if (ey) s = ex ? __fadd_rn(s, ey > 0 ? b : -b) : (ey > 0 ? b : -b);
  if (ez) s = (ex || ey) ? __fadd_rn(s, ez > 0 ? c : -c) : (ez > 0 ? c : -c);
  return s;
}

template <int Q>
__device__ __forceinline__ void rebuild_ev(float T, float q, float ev, int i,
                                           float &fr, float &fb) {
  const bool blue = m_blue(q);  // blue majority: red is the minority
  const float minor = __fmaf_rn(
      q, T, __fmul_rn(blue ? Lattice<Q>::w(i) : -Lattice<Q>::w(i), ev));
  const float major = __fsub_rn(T, minor);  // the minority keeps its accuracy
  fr = blue ? minor : major;
  fb = blue ? major : minor;
}

template <int Q>
__device__ __forceinline__ void rebuild(float T, float4 S, int i, float &fr,
                                        float &fb) {
  rebuild_ev<Q>(T, S.x, edot<Q>(i, S.y, S.z, S.w), i, fr, fb);
}

__device__ __forceinline__ int axis_coord(int x, int y, int z, int a) {
  return a == 0 ? x : (a == 1 ? y : z);
}
__device__ __forceinline__ int axis_extent(const Dom &d, int a) {
  return a == 0 ? d.nx : (a == 1 ? d.ny : d.nz);
}

// ------------------------------------------------------------ wetting
__device__ __forceinline__ float dot3(const float *a, const float *b) {
  return __fmaf_rn(a[2], b[2], __fmaf_rn(a[1], b[1], __fmul_rn(a[0], b[0])));
}

// Eq. (28): f(v) = v.n_w - |v| cos(theta)
__device__ __forceinline__ float secant_f(const float *v, const float *nw,
                                          float cth) {
  return __fsub_rn(dot3(v, nw), __fmul_rn(sqrtf(dot3(v, v)), cth));
}

// Scheme-I, Eqs. (29)-(31): v0 = n_c, v1 = n_c - (n_c + n_w)/2, three secant
// updates (n = 2, 3, 4), early stop on a vanishing denominator, then
// normalise; a zero-length result leaves n_c unchanged.
__device__ __forceinline__ void scheme1(float *nc, const float *nw, float cth) {
  float vm2[3], vm1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    vm2[a] = nc[a];
    vm1[a] = __fsub_rn(nc[a], __fmul_rn(0.5f, __fadd_rn(nc[a], nw[a])));
  }
#pragma unroll
  for (int it = 2; it <= 4; ++it) {
    const float f1 = secant_f(vm1, nw, cth);
    const float f2 = secant_f(vm2, nw, cth);
    const float den = __fsub_rn(f1, f2);
    if (fabsf(den) < EPS_SECANT) break;
    const float inv = 1.f / den;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float vn =
          __fmul_rn(__fsub_rn(__fmul_rn(vm2[a], f1), __fmul_rn(vm1[a], f2)), inv);
      vm2[a] = vm1[a];
      vm1[a] = vn;
    }
  }
  const float m = sqrtf(dot3(vm1, vm1));
  if (m > 0.f) {
    const float im = 1.f / m;
#pragma unroll
    for (int a = 0; a < 3; ++a) nc[a] = __fmul_rn(vm1[a], im);
  }
}

// Scheme-II, Eqs. (32)-(33): with c = n_w.n_c = cos(theta') and
// s' = sin(theta'), n_+- = (cos(theta) -+ sin(theta) c/s') n_w
// +- (sin(theta)/s') n_c; keep the one nearer to n_c (n_+ on a tie);
// unchanged when s' < EPS_SIN. Regrouped as n_+- = cos(theta) n_w
// +- (sin(theta)/s') t with t = n_c - c n_w and s' = |t| (the same numbers
// for unit vectors), which stays accurate when n_c and n_w are nearly
// parallel.
__device__ __forceinline__ void scheme2(float *nc, const float *nw, float cth,
                                        float sth) {
  const float c = fminf(1.f, fmaxf(-1.f, dot3(nw, nc)));
  float t[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) t[a] = __fsub_rn(nc[a], __fmul_rn(c, nw[a]));
  const float sp = sqrtf(dot3(t, t));
  if (sp < EPS_SIN) return;
  const float k = sth / sp;
  float np_[3], nm_[3], dp = 0.f, dm = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float cw = __fmul_rn(cth, nw[a]), kt = __fmul_rn(k, t[a]);
    np_[a] = __fadd_rn(cw, kt);
    nm_[a] = __fsub_rn(cw, kt);
    const float ep = __fsub_rn(np_[a], nc[a]), em = __fsub_rn(nm_[a], nc[a]);
    dp = __fmaf_rn(ep, ep, dp);
    dm = __fmaf_rn(em, em, dm);
  }
  const bool plus = dp <= dm;
#pragma unroll
  for (int a = 0; a < 3; ++a) nc[a] = plus ? np_[a] : nm_[a];
}

// ------------------------------------------------- stencil accumulators
// Eq. (34): phi at a solid-boundary node, the w-weighted mean over its
// in-box fluid neighbours, kept in the encoded form (the mean of phi - s for
// the sign s of the mean). add() once per neighbour in direction order.
struct Eq34 {
  float den = 0.f, sphi = 0.f, ex_pos = 0.f, ex_neg = 0.f;
  __device__ __forceinline__ void add(float w, float m) {
    den = __fadd_rn(den, w);
    sphi = __fmaf_rn(w, m_phi(m), sphi);
    ex_pos = __fmaf_rn(w, m_excess(m, false), ex_pos);
    ex_neg = __fmaf_rn(w, m_excess(m, true), ex_neg);
  }
  __device__ __forceinline__ float finish() const {
    const bool blue = sphi < 0.f;
    const float ex = (blue ? ex_neg : ex_pos) / den;  // phi_s - s
    return m_pack(blue, __fmul_rn(blue ? 0.5f : -0.5f, ex));
  }
};

// Eq. (6) (c = dt = 1) as 3 sum_i w_i e_i (phi(x + e_i) - s(x)), the same sum
// since sum_i w_i e_i = 0, from the encoded neighbour values.
template <int Q>
struct Grad {
  float G[3] = {0.f, 0.f, 0.f};
  __device__ __forceinline__ void add(int i, float m_nb, bool own_blue) {
    const float p = __fmul_rn(3.f * Lattice<Q>::w(i), m_excess(m_nb, own_blue));
    const int e[3] = {Lattice<Q>::ex(i), Lattice<Q>::ey(i), Lattice<Q>::ez(i)};
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (e[a]) G[a] = __fadd_rn(G[a], e[a] > 0 ? p : -p);
  }
  __device__ __forceinline__ float mag() const { return sqrtf(dot3(G, G)); }
};

// Eq. (35): n_c at a solid-boundary node, the w-weighted mean of its in-box
// fluid neighbours' n_c, not renormalised.
struct Eq35 {
  float num[3] = {0.f, 0.f, 0.f}, den = 0.f;
  __device__ __forceinline__ void add(float w, float vx, float vy, float vz) {
    num[0] = __fmaf_rn(w, vx, num[0]);
    num[1] = __fmaf_rn(w, vy, num[1]);
    num[2] = __fmaf_rn(w, vz, num[2]);
    den = __fadd_rn(den, w);
  }
  __device__ __forceinline__ float4 finish() const {
    const float id = 1.f / den;
    return make_float4(__fmul_rn(num[0], id), __fmul_rn(num[1], id),
                       __fmul_rn(num[2], id), 0.f);
  }
};

// Eq. (12) with d_b n_a by the Eq. (6) stencil on each component:
// dn[a][b] = 3 sum_i w_i e_ib n_a(x + e_i).
template <int Q>
struct Curv {
  float dn[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  __device__ __forceinline__ void add(int i, float vx, float vy, float vz) {
    const float w3 = 3.f * Lattice<Q>::w(i);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int eb = Lattice<Q>::e(i, b);
      if (eb == 0) continue;
      const float c = eb > 0 ? w3 : -w3;
      dn[0][b] = __fmaf_rn(c, vx, dn[0][b]);
      dn[1][b] = __fmaf_rn(c, vy, dn[1][b]);
      dn[2][b] = __fmaf_rn(c, vz, dn[2][b]);
    }
  }
  // kappa = sum_ab (n_a n_b - delta_ab) d_b n_a for the node's n_c
  __device__ __forceinline__ float kappa(float x, float y, float z) const {
    float k = __fmul_rn(__fmaf_rn(x, x, -1.f), dn[0][0]);
    k = __fmaf_rn(__fmaf_rn(y, y, -1.f), dn[1][1], k);
    k = __fmaf_rn(__fmaf_rn(z, z, -1.f), dn[2][2], k);
    k = __fmaf_rn(__fmul_rn(__fadd_rn(dn[0][1], dn[1][0]), x), y, k);
    k = __fmaf_rn(__fmul_rn(__fadd_rn(dn[0][2], dn[2][0]), x), z, k);
    return __fmaf_rn(__fmul_rn(__fadd_rn(dn[2][1], dn[1][2]), z), y, k);
  }
};

// Eq. (11) n_c = C/|C| (zero where |C| <= EPS_C: no interface) and, at a
// fluid-boundary node with wetting on, Scheme-I or Scheme-II turning n_c
// with |C| kept (Eq. 27); returns (n_c, |C|).
template <int Q>
__device__ __forceinline__ float4 normal_and_wetting(const StepConst &c,
                                                     const Grad<Q> &g,
                                                     bool fluid_bnd,
                                                     const float4 *nw_at) {
  const float mag = g.mag();
  if (!(mag > EPS_C)) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float im = 1.f / mag;
  float nc[3] = {__fmul_rn(g.G[0], im), __fmul_rn(g.G[1], im),
                 __fmul_rn(g.G[2], im)};
  if (c.wetting && fluid_bnd) {
    const float4 w4 = __ldg(nw_at);
    const float nw[3] = {w4.x, w4.y, w4.z};
    if (nw[0] != 0.f || nw[1] != 0.f || nw[2] != 0.f) {
      if (c.wetting == 1)
        scheme1(nc, nw, c.cos_t);
      else
        scheme2(nc, nw, c.cos_t, c.sin_t);
    }
  }
  return make_float4(nc[0], nc[1], nc[2], mag);
}

// Eq. (5) F = 1/2 gamma kappa C with C = |C| n_c (c4 = (n_c, |C|)), plus the
// body force rho g (Eq. 36); returns rho = rho^r + rho^b.
__device__ __forceinline__ float force(const StepConst &c, float rr, float rb,
                                       float kappa, float4 c4, float *F) {
  const float rho = __fadd_rn(rr, rb);
  const float hk = __fmul_rn(__fmul_rn(__fmul_rn(0.5f, c.gamma), kappa), c4.w);
  F[0] = __fmaf_rn(rho, c.g[0], __fmul_rn(hk, c4.x));
  F[1] = __fmaf_rn(rho, c.g[1], __fmul_rn(hk, c4.y));
  F[2] = __fmaf_rn(rho, c.g[2], __fmul_rn(hk, c4.z));
  return rho;
}

// The stored colour split of the recoloured state (Eqs. 20-21): q, the
// encoded rho^r/rho, and v = beta rho^r rho^b / rho n_c.
__device__ __forceinline__ float4 recoloured_split(const StepConst &c, float rr,
                                                   float rb, float rho,
                                                   float4 c4) {
  const float seg = __fmul_rn(__fmul_rn(c.beta, rr), rb) / rho;
  return make_float4(m_of(rr, rb), __fmul_rn(seg, c4.x), __fmul_rn(seg, c4.y),
                     __fmul_rn(seg, c4.z));
}

// ----------------------------------------------------------- collision
// Eqs. (13)-(14): S_nu from the harmonic-mean viscosity (phi clamped).
__device__ __forceinline__ float relaxation_rate(const StepConst &c,
                                                 float phi) {
  // 1/nu = (1 + phi)/(2 nu^r) + (1 - phi)/(2 nu^b); 1/S = 3 nu + 1/2, so
  // S = (1/nu) / (3 + (1/nu)/2): one division
  const float pc = fminf(1.f, fmaxf(-1.f, phi));
  const float inv_nu =
      __fmaf_rn(__fadd_rn(1.f, pc), c.h_r, __fmul_rn(__fsub_rn(1.f, pc), c.h_b));
  return inv_nu / __fmaf_rn(0.5f, inv_nu, 3.f);
}

// Eq. (2) with one rate S for all non-conserved moments and rate 0 for rho
// and j, in velocity space:
//   f''_i = f_i - S (f_i - feq_i) + (1 - S/2) G_i + e_i . b,
//   b = S (j - rho0 u + F/2) / E2,
// feq of Eq. (A.4), G_i = w_i [3 (e_i - u) + 9 (e_i.u) e_i].F (A.5), u of
// Eq. (22). ft holds f^t on entry and f''^t on exit. MRT: 1 the MRT rates
// below, 0 the single rate, -1 as c.mrt says at run time.
template <int Q, int MRT = -1>
__device__ __forceinline__ void collide(const StepConst &c, float *ft,
                                        float rho, const float *F, float phi,
                                        float *u) {
  const bool mrt = MRT < 0 ? c.mrt != 0 : MRT == 1;
  // Moments from the deviations d_i = f_i - w_i rho0: each d_i is exact in
  // float32 (f_i and w_i rho0 are within a factor two of each other) and
  // small, so rho = rho0 + sum d_i and j = sum e_i d_i carry the rounding of
  // the deviations, not of the populations. With the colour sums of the
  // pull as rho (the argument, the same number up to rounding), the
  // collision changed the mass by S (rho - sum f) per node and step, with a
  // bias: a Zou-He tube drifted 0.08 % in flux against the FP64 oracle.
  // The equilibrium's density is now this sum, so the collision keeps the
  // mass it is given, and f - feq is formed from the deviations as well.
  // w_i rho0 is an explicit rounded product (__fmul_rn is never fused into
  // an FMA), so every kernel that inlines this function computes the same
  // d_i bit for bit.
  (void)rho;
  // Directions come in opposite pairs (i, opp(i)) with e_opp = -e_i and equal
  // weights: per pair, e.u, e.F and e.b change sign, the rest is shared, and
  // the two populations are updated with packed two-lane float32 operations
  // (FFMA2 / FADD2 / FMUL2; each lane rounds as its scalar op).
  constexpr int NP = (Q - 1) / 2;
  float d[Q], drho, j[3] = {0.f, 0.f, 0.f};
  {
    d[0] = __fsub_rn(ft[0], __fmul_rn(Lattice<Q>::w(0), c.rho0));
    drho = d[0];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int i = Lattice<Q>::pair(p), o = Lattice<Q>::opp(i);
      const float wr = __fmul_rn(Lattice<Q>::w(i), c.rho0);
      const float2 dd = __fadd2_rn(make_float2(ft[i], ft[o]), make_float2(-wr, -wr));
      d[i] = dd.x;
      d[o] = dd.y;
      // s = d_i + d_o (mass), t = d_i - d_o (momentum along e_i)
      const float2 st = __fadd2_rn(make_float2(dd.x, dd.x), make_float2(dd.y, -dd.y));
      drho = __fadd_rn(drho, st.x);
      const int e[3] = {Lattice<Q>::ex(i), Lattice<Q>::ey(i), Lattice<Q>::ez(i)};
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (e[a]) j[a] = __fadd_rn(j[a], e[a] > 0 ? st.y : -st.y);
    }
  }
  rho = __fadd_rn(c.rho0, drho);
  const float irho = 1.f / rho;
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = __fmul_rn(__fmaf_rn(0.5f, F[a], j[a]), irho);
  const float S = relaxation_rate(c, phi);
  const float uu = dot3(u, u);
  float b[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    b[a] = __fmul_rn(__fmul_rn(S, __fmaf_rn(0.5f, F[a], __fmaf_rn(-c.rho0, u[a], j[a]))),
                     1.f / Lattice<Q>::E2);
  const float kf = __fsub_rn(1.f, __fmul_rn(0.5f, S));
  const float uF = dot3(u, F);
  // MRT (D3Q19): Eq. (2) with the rates of Eq. (4), S_e = S_eps = S_pi =
  // S_nu (Eq. 15) and S_q = S_m from Eq. (16). It differs from the
  // single-rate form only in the rows of q (4, 6, 8) and m (16-18) of M
  // (Eq. A.3), which relax at S_q instead of S_nu. The rows of M are
  // orthogonal, so M^-1 = M^T diag(1/|row_k|^2), and the difference is
  //   f''_i += sum_k M_ki dm_k / |row_k|^2,
  //   dm_k = -(S_q - S_nu) (m_k - m_k^eq + h_k / 2)
  // with m^eq_q = -2/3 rho0 u, h_q = -2/3 F (A.4, A.5), m^eq_m = h_m = 0,
  // |row_q|^2 = 40 and |row_m|^2 = 8.
  float aq[3] = {0.f, 0.f, 0.f}, am[3] = {0.f, 0.f, 0.f};
  if constexpr (Q == 19 && MRT != 0) {
    if (mrt) {
      float q[3] = {0.f, 0.f, 0.f}, m[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int ex = Lattice<Q>::ex(i), ey = Lattice<Q>::ey(i),
                  ez = Lattice<Q>::ez(i);
        const int c5 = 5 * (ex * ex + ey * ey + ez * ez) - 9;
        const int e[3] = {ex, ey, ez};
        const int mm[3] = {ex * (ey * ey - ez * ez), ey * (ez * ez - ex * ex),
                           ez * (ex * ex - ey * ey)};
        const float di = d[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (e[a]) q[a] = __fmaf_rn((float)(c5 * e[a]), di, q[a]);
          if (mm[a]) m[a] = __fadd_rn(m[a], mm[a] > 0 ? di : -di);
        }
      }
      const float Sq = 8.f * __fsub_rn(2.f, S) / __fsub_rn(8.f, S);  // Eq. (16)
      const float dS = __fsub_rn(Sq, S);
      const float r23 = __fmul_rn(2.f / 3.f, c.rho0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float t = __fmaf_rn(-(1.f / 3.f), F[a], __fmaf_rn(r23, u[a], q[a]));
        aq[a] = __fmul_rn(__fmul_rn(-dS, t), 1.f / 40.f);
        am[a] = __fmul_rn(__fmul_rn(-dS, m[a]), 0.125f);
      }
    }
  }
  // f''_i = f_i + upd_i + e_i.b with, in deviations,
  //   f - feq = d_i - w_i (drho + rho0 P_i),  P_i = 3 e.u + 4.5 (e.u)^2 - 1.5 u.u,
  //   upd_i = -S (f - feq) + (1 - S/2) w_i (3 (e.F - u.F) + 9 (e.u)(e.F));
  // the update is summed apart from f_i and added last (it keeps the
  // precision of the deviations: the full droplet and tube runs stay within
  // 1e-4 of the FP64 oracle in phi this way, and not when f_i is updated
  // term by term)
  const float m15uu = __fmul_rn(-1.5f, uu), m3uF = __fmul_rn(-3.f, uF);
  auto pair_update = [&](int i, int o) {
    const float w = Lattice<Q>::w(i);
    const float eu = edot<Q>(i, u[0], u[1], u[2]);
    const float eF = edot<Q>(i, F[0], F[1], F[2]);
    const float eb = edot<Q>(i, b[0], b[1], b[2]);
    const float A = __fmaf_rn(__fmul_rn(4.5f, eu), eu, m15uu);  // shared part of P
    const float t3 = __fmul_rn(3.f, eu);
    const float G0 = __fmaf_rn(__fmul_rn(9.f, eu), eF, m3uF);  // shared part of G/w
    const float t4 = __fmul_rn(3.f, eF);
    const float2 P = __fadd2_rn(make_float2(A, A), make_float2(t3, -t3));
    const float2 X = __ffma2_rn(make_float2(c.rho0, c.rho0), P, make_float2(drho, drho));
    const float2 dneq = __ffma2_rn(make_float2(-w, -w), X, make_float2(d[i], d[o]));
    const float2 g = __fmul2_rn(make_float2(w, w),
                                __fadd2_rn(make_float2(G0, G0), make_float2(t4, -t4)));
    const float2 upd = __ffma2_rn(make_float2(-S, -S), dneq,
                                  __fmul2_rn(make_float2(kf, kf), g));
    const float2 nf = __fadd2_rn(make_float2(ft[i], ft[o]),
                                 __fadd2_rn(upd, make_float2(eb, -eb)));
    ft[i] = nf.x;
    ft[o] = nf.y;
  };
  {
    // rest population: e_0 = 0
    const float X0 = __fmaf_rn(c.rho0, m15uu, drho);
    const float dneq0 = __fmaf_rn(-Lattice<Q>::w(0), X0, d[0]);
    const float g0 = __fmul_rn(Lattice<Q>::w(0), m3uF);
    ft[0] = __fadd_rn(ft[0], __fmaf_rn(-S, dneq0, __fmul_rn(kf, g0)));
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int i = Lattice<Q>::pair(p);
    pair_update(i, Lattice<Q>::opp(i));
  }
  if constexpr (Q == 19 && MRT != 0) {
    if (mrt) {
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int ix = Lattice<Q>::ex(i), iy = Lattice<Q>::ey(i),
                  iz = Lattice<Q>::ez(i);
        const float c5 = (float)(5 * (ix * ix + iy * iy + iz * iz) - 9);
        const int mm[3] = {ix * (iy * iy - iz * iz), iy * (iz * iz - ix * ix),
                           iz * (ix * ix - iy * iy)};
        float cm = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a)
          if (mm[a]) cm = __fadd_rn(cm, mm[a] > 0 ? am[a] : -am[a]);
        ft[i] = __fadd_rn(ft[i], __fmaf_rn(c5, edot<Q>(i, aq[0], aq[1], aq[2]), cm));
      }
    }
  }
}

}  // namespace lbm
