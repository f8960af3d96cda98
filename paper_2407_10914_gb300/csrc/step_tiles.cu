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

#include "passes.cuh"
#include "step.hpp"

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

// Entry of bit b of a row word, with the OUT flag.
__device__ __forceinline__ uint32_t entry_of(uint4 w, int b, bool out) {
  const uint32_t bit = 1u << b;
  uint32_t e = (w.x & bit) ? w.z + (uint32_t)__popc(w.x & (bit - 1u)) : E_SOLID;
  if (w.y & bit) e |= E_BND;
  if (out) e |= E_OUT;
  return e;
}

// Canonical position of region row `row`: the tile-row offset of its (y, z)
// and whether y or z was clamped.
template <int Q, class R, int H>
__device__ __forceinline__ void row_of(const Dom &d, int Y0, int Z0, int row,
                                       int &tyz, int &rw, bool &out) {
  const int ry = row % R::RY, rz = row / R::RY;
  out = false;
  const int y = canon(Y0 - H + ry, d.ny, d.periodic & 2u, out);
  const int z = Q == 19 ? canon(Z0 - R::HZ + rz, d.nz, d.periodic & 4u, out) : 0;
  tyz = d.ntx * ((y >> R::LY) + d.nty * (z >> Tile<Q>::LZ));
  rw = (y & (R::TY - 1)) + R::TY * (z & (R::TZ - 1));
}

// Entries of every region cell. All global loads are issued together: one
// thread per region row loads the row word of the block's own x-range, and
// the halo cells of every row (H on each side) load their own words; the
// interior cells are then filled from the staged words (W, one per row).
// The caller synchronises before reading E.
template <int Q, int H, int SZ>
__device__ __forceinline__ void stage(const Dom &d, int X0, int Y0, int Z0,
                                      uint32_t *E, uint4 *W) {
  using R = Reg<Q, H, SZ>;
  constexpr int NH = 2 * H * R::NROW;
  constexpr int IT = (NH + TB - 1) / TB;
  static_assert(R::NROW <= TB, "one row word per thread");
  const int tid = threadIdx.x;
  uint4 wo = make_uint4(0u, 0u, 0u, 0u);
  bool oo = false;
  if (tid < R::NROW) {
    int tyz, rw;
    row_of<Q, R, H>(d, Y0, Z0, tid, tyz, rw, oo);
    wo = __ldg(d.rows + (size_t)((X0 >> 5) + tyz) * R::RPT + rw);
  }
  uint32_t eh[IT];
  int ch[IT];
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int t = tid + it * TB;
    ch[it] = -1;
    eh[it] = 0u;
    if (t < NH) {
      const int row = t / (2 * H), p = t % (2 * H);
      const int rx = p < H ? p : R::RX - 2 * H + p;
      int tyz, rw;
      bool o;
      row_of<Q, R, H>(d, Y0, Z0, row, tyz, rw, o);
      const int x = canon(X0 - H + rx, d.nx, d.periodic & 1u, o);
      const uint4 w = __ldg(d.rows + (size_t)((x >> 5) + tyz) * R::RPT + rw);
      eh[it] = entry_of(w, x & 31, o);
      ch[it] = rx + R::RX * row;
    }
  }
  if (tid < R::NROW) {
    wo.w = oo ? 1u : 0u;
    W[tid] = wo;
  }
#pragma unroll
  for (int it = 0; it < IT; ++it)
    if (ch[it] >= 0) E[ch[it]] = eh[it];
  __syncthreads();
  for (int c = tid; c < R::NROW * 32; c += TB) {
    const int row = c >> 5, lx = c & 31;
    const uint4 w = W[row];
    const int x = X0 + lx;
    uint32_t e;
    if (x < d.nx) {
      e = entry_of(w, lx, w.w != 0u);
    } else {  // past the box's end: wrapped or clamped like a halo cell
      int tyz, rw;
      bool o;
      row_of<Q, R, H>(d, Y0, Z0, row, tyz, rw, o);
      const int xc = canon(x, d.nx, d.periodic & 1u, o);
      const uint4 w2 = __ldg(d.rows + (size_t)((xc >> 5) + tyz) * R::RPT + rw);
      e = entry_of(w2, xc & 31, o);
    }
    E[lx + H + R::RX * row] = e;
  }
}

// Region cells q of the one-node box (the cells within one node of the
// slab) of a two-node region.
template <class R>
struct Box1 {
  static constexpr int HZ1 = R::HZ / 2;
  static constexpr int IX = R::RX - 2, IY = R::RY - 2, IZ = R::RZ - 2 * HZ1;
  static constexpr int N = IX * IY * IZ;
  __device__ static constexpr int cell(int q) {
    return (q % IX + 1) + R::RX * ((q / IX) % IY + 1 + R::RY * (q / (IX * IY) + HZ1));
  }
};

// sl[0..*ns) = the one-node box's solid-boundary cells that lie on the box
// (not OUT): where Eqs. (34)-(35) are evaluated. Warp-aggregated append.
template <class R>
__device__ __forceinline__ void solid_list(const uint32_t *E, uint16_t *sl,
                                           int *ns) {
  using B = Box1<R>;
  const int lane = threadIdx.x & 31;
  for (int q0 = threadIdx.x - lane; q0 < B::N; q0 += TB) {
    const int q = q0 + lane;
    const int c = B::cell(q < B::N ? q : 0);
    const bool want = q < B::N &&
                      (E[c] & (E_SOLID | E_BND | E_OUT)) == (E_SOLID | E_BND);
    const unsigned m = __ballot_sync(0xffffffffu, want);
    int at = 0;
    if (lane == 0 && m) at = atomicAdd(ns, __popc(m));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (want) sl[at + __popc(m & ((1u << lane) - 1u))] = (uint16_t)c;
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
  __shared__ uint4 W[R::NROW];
  __shared__ uint16_t list[R::NOWN];
  int X0, Y0, Z0, base, n;
  slab_of<R>(d, blockIdx.x, X0, Y0, Z0, base, n);
  if (n == 0) return;
  stage<Q, 1, Tile<Q>::TZ>(d, X0, Y0, Z0, E, W);
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
        const float ev = edot<Q>(i, S.y, S.z, S.w);
        rebuild_ev<Q>(t, S.x, fl ? ev : -ev, i, fr, fb);
      }
      rr = __fadd_rn(rr, fr);
      rb = __fadd_rn(rb, fb);
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
  using B = Box1<R>;
  __shared__ uint32_t E[R::NC];
  __shared__ float P[R::NC];
  __shared__ uint4 W[R::NROW];
  __shared__ uint16_t list[R::NOWN];
  __shared__ uint16_t sl[B::N];
  __shared__ int ns;
  int X0, Y0, Z0, base, n;
  slab_of<R>(d, blockIdx.x, X0, Y0, Z0, base, n);
  if (n == 0) return;
  if (threadIdx.x == 0) ns = 0;
  stage<Q, 2, SZ>(d, X0, Y0, Z0, E, W);
  __syncthreads();
  own_list<Q, 2, SZ>(d, X0, Y0, Z0, base, E, list);
  solid_list<R>(E, sl, &ns);
  // the fluid cells' phase field, FU loads in flight per thread
  constexpr int FU = 8;
  for (int c0 = threadIdx.x; c0 < R::NC; c0 += TB * FU) {
    float v[FU];
#pragma unroll
    for (int u = 0; u < FU; ++u) {
      const int c = c0 + u * TB;
      v[u] = 0.f;
      if (c < R::NC) {
        const uint32_t e = E[c];
        if (e_fluid(e)) v[u] = __ldg(d.mf + guard(d, e_idx(e), d.NF, GUARD_STENCIL));
      }
    }
#pragma unroll
    for (int u = 0; u < FU; ++u)
      if (c0 + u * TB < R::NC) P[c0 + u * TB] = v[u];
  }
  __syncthreads();
  // Eq. (34) over the in-box fluid neighbours, in direction order
  for (int j = threadIdx.x; j < ns; j += TB) {
    const int c = sl[j];
    Eq34 acc;
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (e_link(E[c + R::off(i)])) acc.add(Lattice<Q>::w(i), P[c + R::off(i)]);
    P[c] = acc.finish();
  }
  __syncthreads();
  // a solid cell off a non-periodic face holds the node it stands for
  if (d.periodic != 7u) {
    for (int q = threadIdx.x; q < B::N; q += TB) {
      const int c = B::cell(q);
      const uint32_t e = E[c];
      if ((e & (E_SOLID | E_OUT)) == (E_SOLID | E_OUT))
        P[c] = P[clamp_cell<Q, 2, SZ>(d, X0, Y0, Z0, c)];
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < n; j += TB) {
    const int c = R::own(list[j]), k = base + j;
    const bool own_blue = m_blue(P[c]);
    Grad<Q> g;
#pragma unroll
    for (int i = 1; i < Q; ++i) g.add(i, P[c + R::off(i)], own_blue);
    d.ncf[k] = normal_and_wetting(d.c, g, (E[c] & E_BND) != 0u, d.nw + k);
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
  using B = Box1<R>;
  static_assert(B::N == R1::NC, "the one-node box is the one-node region");
  __shared__ uint32_t E[R::NC];
  __shared__ float NX[R1::NC], NY[R1::NC], NZ[R1::NC];
  __shared__ uint4 W[R::NROW];
  __shared__ uint16_t list[R::NOWN];
  __shared__ uint16_t sl[B::N];
  __shared__ int ns;
  int X0, Y0, Z0, base, n;
  slab_of<R>(d, blockIdx.x, X0, Y0, Z0, base, n);
  if (n == 0) return;
  if (threadIdx.x == 0) ns = 0;
  stage<Q, 2, SZ>(d, X0, Y0, Z0, E, W);
  __syncthreads();
  own_list<Q, 2, SZ>(d, X0, Y0, Z0, base, E, list);
  solid_list<R>(E, sl, &ns);
  // the fluid cells' n_c within one node of the slab, FU loads in flight
  constexpr int FU = 4;
  for (int q0 = threadIdx.x; q0 < R1::NC; q0 += TB * FU) {
    float4 v[FU];
#pragma unroll
    for (int u = 0; u < FU; ++u) {
      const int q = q0 + u * TB;
      v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (q < R1::NC) {
        const uint32_t e = E[B::cell(q)];
        if (e_fluid(e)) v[u] = __ldg(d.ncf + guard(d, e_idx(e), d.NF, GUARD_STENCIL));
      }
    }
#pragma unroll
    for (int u = 0; u < FU; ++u) {
      const int q = q0 + u * TB;
      if (q < R1::NC) {
        NX[q] = v[u].x;
        NY[q] = v[u].y;
        NZ[q] = v[u].z;
      }
    }
  }
  __syncthreads();
  // Eq. (35): w-weighted mean of the in-box fluid neighbours' n_c, not
  // renormalised, in direction order (terms up to two nodes out are read
  // from the compact list)
  for (int j = threadIdx.x; j < ns; j += TB) {
    const int c = sl[j];
    Eq35 acc;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t en = E[c + R::off(i)];
      if (!e_link(en)) continue;
      const float4 v = __ldg(d.ncf + guard(d, e_idx(en), d.NF, GUARD_LINK));
      acc.add(Lattice<Q>::w(i), v.x, v.y, v.z);
    }
    const float4 nv = acc.finish();
    // the region cell c is one-node cell q of the same position
    const int rx = c % R::RX - 1, ry = (c / R::RX) % R::RY - 1,
              rz = c / (R::RX * R::RY) - B::HZ1;
    const int q = rx + R1::RX * (ry + R1::RY * rz);
    NX[q] = nv.x;
    NY[q] = nv.y;
    NZ[q] = nv.z;
  }
  __syncthreads();
  if (d.periodic != 7u) {
    for (int q = threadIdx.x; q < R1::NC; q += TB) {
      const uint32_t e = E[B::cell(q)];
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
    Curv<Q> cv;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int cn = c + R1::off(i);
      cv.add(i, NX[cn], NY[cn], NZ[cn]);
    }
    d.kap[k] = cv.kappa(NX[c], NY[c], NZ[c]);
  }
}

// ------------------------------------------------------------------ pass 4
// The pull of f^t again, App. B on the Zou-He planes, Eq. (5) F = 1/2
// gamma kappa C + rho g (Eq. 36), the collision (Eq. 2) and the store of the
// recoloured state (f''_i; q and v = beta rho^r rho^b / rho n of Eqs.
// 20-21), as collide_node.
template <int Q, int ST, bool MACROS, int MRT>
__global__ void __launch_bounds__(TB, MRT ? 3 : 4) kt_collide(Dom d) {
  using R = Reg<Q, 1, Tile<Q>::TZ>;
  using IO = TIO<Q, ST>;
  __shared__ uint32_t E[R::NC];
  __shared__ uint4 W[R::NROW];
  __shared__ uint16_t list[R::NOWN];
  int X0, Y0, Z0, base, n;
  slab_of<R>(d, blockIdx.x, X0, Y0, Z0, base, n);
  if (n == 0) return;
  stage<Q, 1, Tile<Q>::TZ>(d, X0, Y0, Z0, E, W);
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
      const float4 Sown = __ldg(d.S_src + k);
      auto srcS = [&](int i, bool &fl) {
        const uint32_t es = E[c + R::off(Lattice<Q>::opp(i))];
        fl = e_link(es);
        return fl ? __ldg(d.S_src + guard(d, e_idx(es), d.NF, GUARD_ZOU_HE)) : Sown;
      };
      zou_he_totals<Q>(d.c, ft, ac == 0, m, Sown, srcS, rr, rb);
    } else {
      const float2 Rk = __ldg(d.R + k);
      rr = Rk.x;
      rb = Rk.y;
      m = m_of(rr, rb);
    }
    const float kappa = __ldg(d.kap + k);
    const float4 c4 = __ldg(d.ncf + k);
    float F[3], u[3];
    const float rho = force(d.c, rr, rb, kappa, c4, F);
    collide<Q, MRT>(d.c, ft, rho, F, m_phi(m), u);
#pragma unroll
    for (int i = 0; i < Q; ++i) IO::store(d, d.T_dst, i, k, ft[i]);
    d.S_dst[k] = recoloured_split(d.c, rr, rb, rho, c4);
    if (MACROS) d.macro[k] = make_float4(u[0], u[1], u[2], rho);
  }
}

// ------------------------------------------------------------- launches
constexpr int SZ_GRAD = 4;  // slab depth of the stencil passes (D3Q19)
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
