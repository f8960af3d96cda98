// The time step as four tile passes (schedule LBM_SCHED_TILES, the
// default). Each pass needs the previous one's values at lattice neighbours:
//   1 kt_pull       (fluid)  pull of Eq. (1), Eqs. (7)-(9): the colour
//                   densities (rho^r, rho^b) and the encoded phase field;
//     kt_planes     the Zou-He planes' phase field: zeta^r - zeta^b at the
//                   inlet, Eq. (39) at the outlet
//   2 kt_gradient   Eq. (34) at the solid-boundary nodes in and around the
//                   tile, then Eqs. (6), (27) and wetting (Eqs. 28-33) at
//                   the tile's fluid nodes: (n_c, |C|)
//   3 kt_curvature  Eq. (35) at the solid-boundary nodes in and around the
//                   tile, then Eq. (12) at its fluid nodes: kappa
//   4 kt_collide    the pull again (the streamed populations are never
//                   stored), App. B on the Zou-He planes, Eqs. (5), (36),
//                   Eq. (2) single-rate or MRT, and the store of the
//                   recoloured state of Eqs. (20)-(21)
// A block works on one tile of the box (tiles.cuh), or a z-slab of one. It
// first stages the entries of its cells and of a halo of one or two nodes in
// shared memory: for each cell, the F-index of the node it stands for
// (periodic axes wrapped; other axes clamped to the face, with the OUT
// flag), or its class if solid. Entries come from the row words (Dom::rows,
// 16 B per 32 box cells), so a pass reads about 0.5 B of index data per box
// cell; the gathers of a node then depend on one level of loads only. The
// stencil passes also stage the values their stencils read (the phase
// field, n_c) and evaluate Eqs. (34)-(35) in shared memory for the
// solid-boundary nodes they need, so the solid-boundary values are never
// stored. Every sum runs in the order of the node passes of passes.cuh, so
// both schedules give the same float32 numbers bit for bit.
#include <cuda_runtime.h>

#include "step.hpp"
#include "tiles.cuh"

namespace lbm {
namespace tp {

constexpr int TB = 256;  // threads per block

// Entry of a staged cell: bits 0-28 the F-index (fluid), bit 29 the class's
// boundary bit (fluid-boundary or solid-boundary), bit 30 OUT (the cell is
// off the box on a non-periodic axis and stands for the clamped node),
// bit 31 solid.
constexpr uint32_t E_BND = 1u << 29;
constexpr uint32_t E_OUT = 1u << 30;
constexpr uint32_t E_SOLID = 1u << 31;
constexpr uint32_t E_IDX = E_BND - 1u;

__device__ __forceinline__ bool e_fluid(uint32_t e) { return !(e & E_SOLID); }
// fluid and on the box (or wrapped): a pull source, a term of Eqs. 34-35
__device__ __forceinline__ bool e_link(uint32_t e) { return (e >> 30) == 0u; }
__device__ __forceinline__ int e_idx(uint32_t e) { return (int)(e & E_IDX); }

// The staged region of a block: the TX x TY x SZ cells of its (sub)tile and
// a halo of H cells (none along z in D2Q9).
template <int Q, int H, int SZ>
struct Reg {
  static constexpr int TX = Tile<Q>::TX, TY = Tile<Q>::TY, TZ = Tile<Q>::TZ;
  static constexpr int LY = Tile<Q>::LY;
  static constexpr int SZZ = Q == 19 ? SZ : 1;
  static constexpr int HZ = Q == 19 ? H : 0;
  static constexpr int RX = TX + 2 * H, RY = TY + 2 * H, RZ = SZZ + 2 * HZ;
  static constexpr int NC = RX * RY * RZ;
  static constexpr int NROW = RY * RZ;
  static constexpr int NOWN = TX * TY * SZZ;
  static constexpr int NSUB = TZ / SZZ;
  static constexpr int RPT = TY * TZ;  // rows per tile
  static_assert(TX == 32, "a tile row is one 32-bit mask");
  static_assert(TZ % SZZ == 0, "slabs divide the tile");
  // offset of direction i in the region
  __device__ static constexpr int off(int i) {
    return Lattice<Q>::ex(i) + RX * (Lattice<Q>::ey(i) + RY * Lattice<Q>::ez(i));
  }
  // region cell of the (sub)tile's local node lp (x fastest)
  __device__ static constexpr int own(int lp) {
    return (lp % TX + H) + RX * ((lp / TX) % TY + H + RY * ((lp / (TX * TY)) + HZ));
  }
};

// Coordinate v on an axis of extent n: wrapped if periodic, else clamped
// to the face with `out` set.
__device__ __forceinline__ int canon(int v, int n, bool per, bool &out) {
  if (v >= 0 && v < n) return v;
  if (per) {
    v %= n;
    return v < 0 ? v + n : v;
  }
  out = true;
  return v < 0 ? 0 : n - 1;
}

// Block b of a pass over slabs of SZ planes: its origin, the F-index of its
// first fluid node and their number.
template <class R>
__device__ __forceinline__ void slab_of(const Dom &d, int b, int &X0, int &Y0,
                                        int &Z0, int &base, int &n) {
  const int t = b / R::NSUB, sub = b % R::NSUB;
  X0 = (t % d.ntx) * R::TX;
  const int q = t / d.ntx;
  Y0 = (q % d.nty) * R::TY;
  Z0 = (q / d.nty) * R::TZ + sub * R::SZZ;
  const int r0 = sub * R::SZZ * R::TY;
  base = (int)__ldg(&d.rows[(size_t)t * R::RPT + r0].z);
  const int end = sub + 1 == R::NSUB
                      ? __ldg(d.fbase + t + 1)
                      : (int)__ldg(&d.rows[(size_t)t * R::RPT + r0 + R::SZZ * R::TY].z);
  n = end - base;
}

// Entries of every region cell, one warp per region row.
template <int Q, int H, int SZ>
__device__ __forceinline__ void stage(const Dom &d, int X0, int Y0, int Z0,
                                      uint32_t *E) {
  using R = Reg<Q, H, SZ>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int row = warp; row < R::NROW; row += TB / 32) {
    const int ry = row % R::RY, rz = row / R::RY;
    bool out = false;
    const int y = canon(Y0 - H + ry, d.ny, d.periodic & 2u, out);
    const int z = Q == 19 ? canon(Z0 - R::HZ + rz, d.nz, d.periodic & 4u, out) : 0;
    const int tyz = d.ntx * ((y >> R::LY) + d.nty * (z >> Tile<Q>::LZ));
    const int rw = (y & (R::TY - 1)) + R::TY * (z & (R::TZ - 1));
#pragma unroll
    for (int rx0 = 0; rx0 < R::RX; rx0 += 32) {
      const int rx = rx0 + lane;
      if (rx < R::RX) {
        bool o = out;
        const int x = canon(X0 - H + rx, d.nx, d.periodic & 1u, o);
        const uint4 w = __ldg(d.rows + (size_t)((x >> 5) + tyz) * R::RPT + rw);
        const uint32_t bit = 1u << (x & 31);
        uint32_t e = (w.x & bit) ? w.z + (uint32_t)__popc(w.x & (bit - 1u))
                                 : E_SOLID;
        if (w.y & bit) e |= E_BND;
        if (o) e |= E_OUT;
        E[rx + R::RX * row] = e;
      }
    }
  }
}

// list[j] = local index of the (sub)tile's j-th fluid node (F order, so
// node j is F-index base + j). Cells past the box's end are not the
// block's (on a periodic axis they wrap to other nodes).
template <int Q, int H, int SZ>
__device__ __forceinline__ void own_list(const Dom &d, int X0, int Y0, int Z0,
                                         int base, const uint32_t *E,
                                         uint16_t *list) {
  using R = Reg<Q, H, SZ>;
  for (int lp = threadIdx.x; lp < R::NOWN; lp += TB) {
    const int lx = lp % R::TX, ly = (lp / R::TX) % R::TY, lz = lp / (R::TX * R::TY);
    if (X0 + lx >= d.nx || Y0 + ly >= d.ny || Z0 + lz >= d.nz) continue;
    const uint32_t e = E[R::own(lp)];
    if (e_fluid(e)) list[e_idx(e) - base] = (uint16_t)lp;
  }
}

// Region cell of the node an OUT cell stands for: every non-periodic
// coordinate clamped to the box (the periodic ones keep the wrapped cell,
// which holds the same node).
template <int Q, int H, int SZ>
__device__ __forceinline__ int clamp_cell(const Dom &d, int X0, int Y0, int Z0,
                                          int c) {
  using R = Reg<Q, H, SZ>;
  int rx = c % R::RX, ry = (c / R::RX) % R::RY, rz = c / (R::RX * R::RY);
  const int o[3] = {X0 - H, Y0 - H, Z0 - R::HZ};
  const int n[3] = {d.nx, d.ny, d.nz};
  int r[3] = {rx, ry, rz};
#pragma unroll
  for (int a = 0; a < (Q == 19 ? 3 : 2); ++a) {
    if (d.periodic & (1u << a)) continue;
    const int v = o[a] + r[a];
    if (v < 0) r[a] = -o[a];
    if (v >= n[a]) r[a] = n[a] - 1 - o[a];
  }
  return r[0] + R::RX * (r[1] + R::RY * r[2]);
}

// The node's coordinate along axis a from its local index.
template <class R>
__device__ __forceinline__ int axis_pos(int X0, int Y0, int Z0, int lp, int a) {
  return a == 0 ? X0 + lp % R::TX
                : (a == 1 ? Y0 + (lp / R::TX) % R::TY : Z0 + lp / (R::TX * R::TY));
}

// ------------------------------------------------------------------ pass 1
// Eq. (1) pull of the colour densities and the encoded phase field of every
// fluid node (stream_node's sums, nothing stored but R and mf).
template <int Q, int ST>
__global__ void __launch_bounds__(TB, 6) kt_pull(Dom d) {
  using R = Reg<Q, 1, Tile<Q>::TZ>;
  using IO = TIO<Q, ST>;
  __shared__ uint32_t E[R::NC];
  __shared__ uint16_t list[R::NOWN];
  int X0, Y0, Z0, base, n;
  slab_of<R>(d, blockIdx.x, X0, Y0, Z0, base, n);
  if (n == 0) return;
  stage<Q, 1, Tile<Q>::TZ>(d, X0, Y0, Z0, E);
  __syncthreads();
  own_list<Q, 1, Tile<Q>::TZ>(d, X0, Y0, Z0, base, E, list);
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += TB) {
    const int c = R::own(list[j]), k = base + j;
    const float4 Sown = __ldg(d.S_src + k);
    float rr = 0.f, rb = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float fr, fb;
      if (i == 0) {
        rebuild<Q>(IO::load(d, 0, k), Sown, 0, fr, fb);
      } else {
        const uint32_t e = E[c + R::off(Lattice<Q>::opp(i))];
        const bool fl = e_link(e);
        const int src = guard(d, fl ? e_idx(e) : k, d.NF, GUARD_PULL);
        const float t = IO::load_dyn(d, fl ? i : Lattice<Q>::opp(i), src);
        const float4 S = fl ? __ldg(d.S_src + src) : Sown;
        const float ev = (float)Lattice<Q>::ex(i) * S.y +
                         (float)Lattice<Q>::ey(i) * S.z +
                         (float)Lattice<Q>::ez(i) * S.w;
        rebuild_ev<Q>(t, S.x, fl ? ev : -ev, i, fr, fb);
      }
      rr += fr;
      rb += fb;
    }
    d.R[k] = make_float2(rr, rb);
    d.mf[k] = m_of(rr, rb);
  }
}

// The phase field of the Zou-He planes' nodes: zeta^r - zeta^b at the
// inlet; at the outlet phi(x - a) (Eq. 39), or the node's own value where
// x - a is solid.
__global__ void __launch_bounds__(TB) kt_planes(Dom d) {
  const int j = blockIdx.x * TB + threadIdx.x;
  if (j >= d.n_zh) return;
  const int k = guard(d, __ldg(d.zh_list + j), d.NF, GUARD_ZOU_HE);
  const int a = d.c.axis;
  if (__ldg(d.fflag + k) & (2u << (2 * a))) {
    d.mf[k] = d.c.m_in;
    return;
  }
  const int sa = a == 0 ? 1 : (a == 1 ? d.px : d.px * d.py);
  const uint32_t e = __ldg(
      d.nbd + guard(d, __ldg(d.fgp + k) - sa, d.px * d.py * (d.nz + 2), GUARD_ZOU_HE));
  const float2 Rk = d.R[k];
  d.mf[k] = ((entry_cls(e) & 2) && !entry_out(e))
                ? d.mf[guard(d, entry_idx(e), d.NF, GUARD_ZOU_HE)]
                : m_of(Rk.x, Rk.y);
}

// ------------------------------------------------------------------ pass 2
// Eq. (34) at the solid-boundary cells within one node of the slab, then
// the colour gradient (Eq. 6, as gradient_node) and wetting at its fluid
// nodes.
template <int Q, int SZ>
__global__ void __launch_bounds__(TB) kt_gradient(Dom d) {
  using R = Reg<Q, 2, SZ>;
  __shared__ uint32_t E[R::NC];
  __shared__ float P[R::NC];
  __shared__ uint16_t list[R::NOWN];
  int X0, Y0, Z0, base, n;
  slab_of<R>(d, blockIdx.x, X0, Y0, Z0, base, n);
  if (n == 0) return;
  stage<Q, 2, SZ>(d, X0, Y0, Z0, E);
  __syncthreads();
  own_list<Q, 2, SZ>(d, X0, Y0, Z0, base, E, list);
  for (int c = threadIdx.x; c < R::NC; c += TB) {
    const uint32_t e = E[c];
    if (e_fluid(e)) P[c] = __ldg(d.mf + guard(d, e_idx(e), d.NF, GUARD_STENCIL));
  }
  __syncthreads();
  // Eq. (34) over the in-box fluid neighbours, in direction order
  constexpr int IX = R::RX - 2, IY = R::RY - 2, IZ = R::RZ - 2 * (R::HZ / 2);
  constexpr int HZ1 = R::HZ / 2;
  for (int q = threadIdx.x; q < IX * IY * IZ; q += TB) {
    const int c = (q % IX + 1) + R::RX * ((q / IX) % IY + 1 + R::RY * (q / (IX * IY) + HZ1));
    const uint32_t e = E[c];
    if ((e & (E_SOLID | E_BND | E_OUT)) != (E_SOLID | E_BND)) continue;
    float den = 0.f, sphi = 0.f, ex_pos = 0.f, ex_neg = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (!e_link(E[c + R::off(i)])) continue;
      const float w = Lattice<Q>::w(i);
      const float m = P[c + R::off(i)];
      den += w;
      sphi += w * m_phi(m);
      ex_pos += w * m_excess(m, false);
      ex_neg += w * m_excess(m, true);
    }
    const bool blue = sphi < 0.f;
    const float ex = (blue ? ex_neg : ex_pos) / den;
    P[c] = m_pack(blue, blue ? 0.5f * ex : -0.5f * ex);
  }
  __syncthreads();
  // a solid cell off a non-periodic face holds the node it stands for
  if (d.periodic != 7u) {
    for (int q = threadIdx.x; q < IX * IY * IZ; q += TB) {
      const int c = (q % IX + 1) + R::RX * ((q / IX) % IY + 1 + R::RY * (q / (IX * IY) + HZ1));
      const uint32_t e = E[c];
      if ((e & (E_SOLID | E_OUT)) == (E_SOLID | E_OUT))
        P[c] = P[clamp_cell<Q, 2, SZ>(d, X0, Y0, Z0, c)];
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < n; j += TB) {
    const int c = R::own(list[j]), k = base + j;
    const bool own_blue = m_blue(P[c]);
    float G[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const float p = 3.f * Lattice<Q>::w(i) * m_excess(P[c + R::off(i)], own_blue);
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
    if (d.c.wetting && (E[c] & E_BND)) {
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

// ------------------------------------------------------------------ pass 3
// Eq. (35) at the solid-boundary cells within one node of the slab, then
// the curvature of Eq. (12) (as curvature()) at its fluid nodes. n_c is
// staged for the cells within one node; Eq. (35) reads its terms, up to two
// nodes out, from the compact list.
template <int Q, int SZ>
__global__ void __launch_bounds__(TB) kt_curvature(Dom d) {
  using R = Reg<Q, 2, SZ>;
  using R1 = Reg<Q, 1, SZ>;
  __shared__ uint32_t E[R::NC];
  __shared__ float NX[R1::NC], NY[R1::NC], NZ[R1::NC];
  __shared__ uint16_t list[R::NOWN];
  int X0, Y0, Z0, base, n;
  slab_of<R>(d, blockIdx.x, X0, Y0, Z0, base, n);
  if (n == 0) return;
  stage<Q, 2, SZ>(d, X0, Y0, Z0, E);
  __syncthreads();
  own_list<Q, 2, SZ>(d, X0, Y0, Z0, base, E, list);
  // cell q of the one-node region is cell c2(q) of the two-node one
  auto c2 = [](int q) {
    return (q % R1::RX + 1) +
           R::RX * ((q / R1::RX) % R1::RY + 1 + R::RY * (q / (R1::RX * R1::RY) + (R::HZ - R1::HZ)));
  };
  for (int q = threadIdx.x; q < R1::NC; q += TB) {
    const uint32_t e = E[c2(q)];
    if (e_fluid(e)) {
      const float4 v = __ldg(d.ncf + guard(d, e_idx(e), d.NF, GUARD_STENCIL));
      NX[q] = v.x;
      NY[q] = v.y;
      NZ[q] = v.z;
    }
  }
  __syncthreads();
  // Eq. (35): w-weighted mean of the in-box fluid neighbours' n_c, not
  // renormalised, in direction order
  for (int q = threadIdx.x; q < R1::NC; q += TB) {
    const int c = c2(q);
    const uint32_t e = E[c];
    if ((e & (E_SOLID | E_BND | E_OUT)) != (E_SOLID | E_BND)) continue;
    float num[3] = {0.f, 0.f, 0.f}, den = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t en = E[c + R::off(i)];
      if (!e_link(en)) continue;
      const float w = Lattice<Q>::w(i);
      const float4 v = __ldg(d.ncf + guard(d, e_idx(en), d.NF, GUARD_LINK));
      num[0] += w * v.x;
      num[1] += w * v.y;
      num[2] += w * v.z;
      den += w;
    }
    const float id = 1.f / den;
    NX[q] = num[0] * id;
    NY[q] = num[1] * id;
    NZ[q] = num[2] * id;
  }
  __syncthreads();
  if (d.periodic != 7u) {
    for (int q = threadIdx.x; q < R1::NC; q += TB) {
      const uint32_t e = E[c2(q)];
      if ((e & (E_SOLID | E_OUT)) == (E_SOLID | E_OUT)) {
        const int cc = clamp_cell<Q, 1, SZ>(d, X0, Y0, Z0, q);
        NX[q] = NX[cc];
        NY[q] = NY[cc];
        NZ[q] = NZ[cc];
      }
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < n; j += TB) {
    const int c = R1::own(list[j]), k = base + j;
    float dn[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int cn = c + R1::off(i);
      const float vx = NX[cn], vy = NY[cn], vz = NZ[cn];
      const float w3 = 3.f * Lattice<Q>::w(i);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int eb = Lattice<Q>::e(i, b);
        if (eb == 0) continue;
        dn[0][b] += w3 * (float)eb * vx;
        dn[1][b] += w3 * (float)eb * vy;
        dn[2][b] += w3 * (float)eb * vz;
      }
    }
    const float nx_ = NX[c], ny_ = NY[c], nz_ = NZ[c];
    d.kap[k] = (nx_ * nx_ - 1.f) * dn[0][0] + (ny_ * ny_ - 1.f) * dn[1][1] +
               (nz_ * nz_ - 1.f) * dn[2][2] + (dn[0][1] + dn[1][0]) * nx_ * ny_ +
               (dn[0][2] + dn[2][0]) * nx_ * nz_ + (dn[2][1] + dn[1][2]) * nz_ * ny_;
  }
}

// ------------------------------------------------------------------ pass 4
// App. B on a Zou-He plane node, in totals on the pulled f^t (the
// arithmetic of zh_fix_node): the unknown populations, and the colour
// densities rho^r, rho^b. m: the node's phase field (Eq. 39's value at the
// outlet). c: the node's region cell, E the staged entries.
template <int Q, class R>
__device__ __forceinline__ void zou_he(const Dom &d, float *ft, bool inlet,
                                       int k, int c, const uint32_t *E,
                                       float m, float &rr, float &rb) {
  const int a = d.c.axis;
  const int in_dir = inlet ? -1 : 1;
  float K0 = 0.f, Kin = 0.f, K0d = 0.f, Kind = 0.f, N[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int ea = Lattice<Q>::e(i, a);
    const float dv = ft[i] - __fmul_rn(Lattice<Q>::w(i), d.c.rho0);
    if (ea == 0) {
      K0 += ft[i];
      K0d += dv;
#pragma unroll
      for (int t = 0; t < 3; ++t)
        if (t != a) N[t] += 0.5f * (float)Lattice<Q>::e(i, t) * dv;
    } else if (ea == in_dir) {
      Kin += ft[i];
      Kind += dv;
    }
  }
  float jt;
  if (inlet) {
    jt = (d.c.rho_in_r + d.c.rho_in_b - d.c.rho0) - (K0d + 2.f * Kind);
    rr = d.c.rho_in_r;
    rb = d.c.rho_in_b;
  } else {
    jt = (K0d + 2.f * Kind) - (d.c.rho_out - d.c.rho0);
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
        const uint32_t es = E[c + R::off(Lattice<Q>::opp(i))];
        const bool fl = e_link(es);
        const float4 S =
            fl ? __ldg(d.S_src + guard(d, e_idx(es), d.NF, GUARD_ZOU_HE)) : Sown;
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
    jt = -jt;
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (Lattice<Q>::e(i, a) != -in_dir) continue;
    float corr = 0.f;
#pragma unroll
    for (int t = 0; t < 3; ++t)
      if (t != a) corr += (float)Lattice<Q>::e(i, t) * N[t];
    ft[i] = ft[Lattice<Q>::opp(i)] + 6.f * Lattice<Q>::w(i) * jt - corr;
  }
}

// The pull of f^t again, App. B on the Zou-He planes, Eq. (5) F = 1/2
// gamma kappa C + rho g (Eq. 36), the collision (Eq. 2) and the store of the
// recoloured state (f''_i; q and v = beta rho^r rho^b / rho n of Eqs.
// 20-21), as collide_node.
template <int Q, int ST, bool MACROS, int MRT>
__global__ void __launch_bounds__(TB, MRT ? 3 : 4) kt_collide(Dom d) {
  using R = Reg<Q, 1, Tile<Q>::TZ>;
  using IO = TIO<Q, ST>;
  __shared__ uint32_t E[R::NC];
  __shared__ uint16_t list[R::NOWN];
  int X0, Y0, Z0, base, n;
  slab_of<R>(d, blockIdx.x, X0, Y0, Z0, base, n);
  if (n == 0) return;
  stage<Q, 1, Tile<Q>::TZ>(d, X0, Y0, Z0, E);
  __syncthreads();
  own_list<Q, 1, Tile<Q>::TZ>(d, X0, Y0, Z0, base, E, list);
  __syncthreads();
  const int a = d.c.axis;
  const int ext = a == 0 ? d.nx : (a == 1 ? d.ny : d.nz);
  for (int j = threadIdx.x; j < n; j += TB) {
    const int lp = list[j];
    const int c = R::own(lp), k = base + j;
    float ft[Q];
    ft[0] = IO::load(d, 0, k);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t e = E[c + R::off(Lattice<Q>::opp(i))];
      const bool fl = e_link(e);
      const int src = guard(d, fl ? e_idx(e) : k, d.NF, GUARD_PULL);
      ft[i] = IO::load_dyn(d, fl ? i : Lattice<Q>::opp(i), src);
    }
    float rr, rb, m;
    const int ac = axis_pos<R>(X0, Y0, Z0, lp, a);
    if (d.c.zou_he && (ac == 0 || ac == ext - 1)) {
      m = __ldg(d.mf + k);
      zou_he<Q, R>(d, ft, ac == 0, k, c, E, m, rr, rb);
    } else {
      const float2 Rk = __ldg(d.R + k);
      rr = Rk.x;
      rb = Rk.y;
      m = m_of(rr, rb);
    }
    const float kappa = __ldg(d.kap + k);
    const float4 c4 = __ldg(d.ncf + k);
    const float rho = rr + rb;
    const float hk = 0.5f * d.c.gamma * kappa * c4.w;
    const float F[3] = {hk * c4.x + rho * d.c.g[0], hk * c4.y + rho * d.c.g[1],
                        hk * c4.z + rho * d.c.g[2]};
    float u[3];
    collide<Q, MRT>(d.c, ft, rho, F, m_phi(m), u);
#pragma unroll
    for (int i = 0; i < Q; ++i) IO::store(d, d.T_dst, i, k, ft[i]);
    const float seg = d.c.beta * rr * rb / rho;
    d.S_dst[k] = make_float4(m_of(rr, rb), seg * c4.x, seg * c4.y, seg * c4.z);
    if (MACROS) d.macro[k] = make_float4(u[0], u[1], u[2], rho);
  }
}

// ------------------------------------------------------------- launches
constexpr int SZ_GRAD = 8;  // slab depth of the stencil passes (D3Q19)
constexpr int SZ_CURV = 4;

template <int Q, int ST>
void launch_t(const Dom &d, cudaStream_t s, bool macros, cudaEvent_t *ev) {
  using R1 = Reg<Q, 1, Tile<Q>::TZ>;
  using RG = Reg<Q, 2, Q == 19 ? SZ_GRAD : 1>;
  using RC = Reg<Q, 2, Q == 19 ? SZ_CURV : 1>;
  const unsigned g1 = (unsigned)(d.ntiles * R1::NSUB);
  const unsigned gg = (unsigned)(d.ntiles * RG::NSUB);
  const unsigned gc = (unsigned)(d.ntiles * RC::NSUB);
  if (ev) cudaEventRecord(ev[0], s);
  kt_pull<Q, ST><<<g1, TB, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[1], s);
  if (d.n_zh > 0) kt_planes<<<(d.n_zh + TB - 1) / TB, TB, 0, s>>>(d);
  if (ev) {
    cudaEventRecord(ev[2], s);
    cudaEventRecord(ev[3], s);
  }
  kt_gradient<Q, Q == 19 ? SZ_GRAD : 1><<<gg, TB, 0, s>>>(d);
  if (ev) {
    cudaEventRecord(ev[4], s);
    cudaEventRecord(ev[5], s);
  }
  kt_curvature<Q, Q == 19 ? SZ_CURV : 1><<<gc, TB, 0, s>>>(d);
  if (ev) cudaEventRecord(ev[6], s);
  const bool mrt = Q == 19 && d.c.mrt;
  if (macros) {
    if (mrt) kt_collide<Q, ST, true, 1><<<g1, TB, 0, s>>>(d);
    else kt_collide<Q, ST, true, 0><<<g1, TB, 0, s>>>(d);
  } else {
    if (mrt) kt_collide<Q, ST, false, 1><<<g1, TB, 0, s>>>(d);
    else kt_collide<Q, ST, false, 0><<<g1, TB, 0, s>>>(d);
  }
  if (ev) cudaEventRecord(ev[7], s);
}

}  // namespace tp

void launch_step_tiles(int Q, int storage, const Dom &d, cudaStream_t s,
                       bool macros, cudaEvent_t *ev) {
  if (Q == 19) {
    if (storage == LBM_STORAGE_FP32) tp::launch_t<19, LBM_STORAGE_FP32>(d, s, macros, ev);
    if (storage == LBM_STORAGE_FP16) tp::launch_t<19, LBM_STORAGE_FP16>(d, s, macros, ev);
    if (storage == LBM_STORAGE_BF16) tp::launch_t<19, LBM_STORAGE_BF16>(d, s, macros, ev);
  } else {
    if (storage == LBM_STORAGE_FP32) tp::launch_t<9, LBM_STORAGE_FP32>(d, s, macros, ev);
    if (storage == LBM_STORAGE_FP16) tp::launch_t<9, LBM_STORAGE_FP16>(d, s, macros, ev);
    if (storage == LBM_STORAGE_BF16) tp::launch_t<9, LBM_STORAGE_BF16>(d, s, macros, ev);
  }
}

}  // namespace lbm
