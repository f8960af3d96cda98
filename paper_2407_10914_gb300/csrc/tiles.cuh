// Tiles of the box, the entries that name a box position's node, and the
// pull of Eq. (1).
//
// The box is cut into tiles of TX x TY x TZ nodes (by default 32 x 8 x 8
// for D3Q19, 64 x 32 x 1 for D2Q9; the shape is chosen when the geometry is
// built: powers of two, TX from 32 to 1024, at most 16384 nodes). Fluid
// nodes are numbered tile by tile (F-space), and within a tile the fluid
// nodes on the box's x faces first, then the others in (z, y, x) order;
// solid-boundary nodes in (z, y, x) order (S-space). The shape changes
// only where a node's values sit in memory, never what is computed. The uint16 map over the box holds a node's class (bits 14-15)
// and its rank among the nodes of its kind in its tile (bits 0-13); with the
// per-tile bases fbase/sbase this gives its F- or S-index.
//
// An entry (class << 30 | OUT << 29 | index) names the node at a box
// position. In the step, a fluid node finds its lattice neighbours in the
// dense entry box (one entry per cell of the box padded by one node;
// geometry.cu), at its padded index plus a compile-time offset per
// direction.
#pragma once

#include "stencil.cuh"

namespace lbm {

// Limits of a tile shape (log2 of the extents): the x extent from a warp's
// run of nodes to 1024, at most 2^14 nodes (the rank field of the map).
constexpr int TILE_MIN_LX = 5, TILE_MAX_LX = 10, TILE_MAX_LN = 14;

// Entries: class << 30 | index (index < 2^29). In the dense entry box a halo
// cell off a non-periodic axis holds the entry of the clamped position (the
// stencils' zero-gradient rule; periodic axes wrap) with the OUT bit set
// (the pull bounces back, the extrapolations skip it).
constexpr uint32_t OUT_BIT = 1u << 29;
__device__ __forceinline__ int entry_cls(uint32_t e) { return (int)(e >> 30); }
__device__ __forceinline__ int entry_idx(uint32_t e) {
  return (int)(e & 0x1FFFFFFFu);
}
__device__ __forceinline__ bool entry_out(uint32_t e) { return e & OUT_BIT; }

// Tile number of box node (X, Y, Z).
__device__ __forceinline__ int tile_of(const Dom &d, int X, int Y, int Z) {
  return (X >> d.tlx) + d.ntx * ((Y >> d.tly) + d.nty * (Z >> d.tlz));
}

// Entry of box node (X, Y, Z) (inside the box).
__device__ __forceinline__ uint32_t box_entry(const Dom &d, int X, int Y,
                                              int Z) {
  const uint16_t m = __ldg(d.map + (X + d.nx * (Y + d.ny * Z)));
  const int cls = m >> 14;
  const int t = tile_of(d, X, Y, Z);
  const int base = __ldg(((cls & 2) ? d.fbase : d.sbase) + t);
  return ((uint32_t)cls << 30) | (uint32_t)(base + (m & 0x3FFF));
}

// Origin of tile t.
__device__ __forceinline__ void tile_origin(const Dom &d, int t, int &X0,
                                            int &Y0, int &Z0) {
  const int q = t / d.ntx;
  X0 = (t % d.ntx) << d.tlx;
  Y0 = (q % d.nty) << d.tly;
  Z0 = (q / d.nty) << d.tlz;
}

// Box coordinates of the tile-local node lp of the tile at (X0, Y0, Z0).
__device__ __forceinline__ void local_node(const Dom &d, int lp, int X0,
                                           int Y0, int Z0, int &x, int &y,
                                           int &z) {
  x = X0 + (lp & ((1 << d.tlx) - 1));
  y = Y0 + ((lp >> d.tlx) & ((1 << d.tly) - 1));
  z = Z0 + (lp >> (d.tlx + d.tly));
}

// Entry of the lattice neighbour x + e_dir of the fluid node at padded box
// index gp (the dense entry box: the same cell for every node that reaches
// that position, so the reads of neighbouring nodes share cache lines).
template <int Q>
__device__ __forceinline__ uint32_t nb_entry(const Dom &d, int gp, int dir) {
  return __ldg(d.nbd + guard(d, gp + dense_off<Q>(d, dir),
                             d.px * d.py * (d.nz + 2), GUARD_STENCIL));
}

// Eq. (1) propagation of fluid node k (padded index gp): f^s_i(x) =
// f^s_i'(x - e_i) from a fluid source (the entry of direction opp(i), which
// points to x - e_i), else the halfway bounce-back f^s_opp(i)'(x). Kept is
// what the collision needs: f^t_i = f^r_i + f^b_i (which is f''_i of the
// source, no colour rebuild) and the colour densities rho^r, rho^b (the
// rebuilt colours summed as they arrive), so no per-colour arrays stay live.
template <int Q, int ST, bool COH = false>
__device__ __forceinline__ void pull_sums(const Dom &d, int k, int gp,
                                          float4 Sown, float *ft, float &rr,
                                          float &rb) {
  using IO = TIO<Q, ST, COH>;
  rr = 0.f;
  rb = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float fr, fb;
    if (i == 0) {
      ft[0] = IO::load(d, 0, k);
      rebuild<Q>(ft[0], Sown, 0, fr, fb);
    } else {
      const uint32_t e = nb_entry<Q>(d, gp, Lattice<Q>::opp(i));
      // a fluid class (bit 31) not clamped off the box (OUT)
      const bool fl = (e & (0x80000000u | OUT_BIT)) == 0x80000000u;
      const int src = guard(d, fl ? entry_idx(e) : k, d.NF, GUARD_PULL);
      ft[i] = IO::load_dyn(d, fl ? i : Lattice<Q>::opp(i), src);
      // bounce-back reads the node's own (q, v): src = k
      const float4 S = ldv<COH>(d.S_src + src);
      const float ev = edot<Q>(i, S.y, S.z, S.w);
      rebuild_ev<Q>(ft[i], S.x, fl ? ev : -ev, i, fr, fb);
    }
    rr = __fadd_rn(rr, fr);
    rb = __fadd_rn(rb, fb);
  }
}

}  // namespace lbm
