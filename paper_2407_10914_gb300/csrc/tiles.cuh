// Tiles of the box, the entries that name a box position's node, and the
// pull of Eq. (1).
//
// The box is cut into tiles of TX x TY x TZ nodes (32 x 8 x 8 for D3Q19,
// 64 x 32 x 1 for D2Q9). Fluid nodes are numbered tile by tile (F-space),
// and within a tile the fluid nodes on the box's x faces first, then the
// others in (z, y, x) order; solid-boundary nodes in (z, y, x) order
// (S-space). The uint16 map over the box holds a node's class (bits 14-15)
// and its rank among the nodes of its kind in its tile (bits 0-13); with the
// per-tile bases fbase/sbase this gives its F- or S-index.
//
// At set-up one CTA works on one tile: it stages, for the tile and a
// one-node halo, an entry (class << 30 | index) per box position in shared
// memory (OUT for a position off a non-periodic axis). In the step, a fluid
// node finds its lattice neighbours in the dense entry box (one entry per
// cell of the box padded by one node; geometry.cu), at its padded index
// plus a compile-time offset per direction.
#pragma once

#include "stencil.cuh"

namespace lbm {

template <int Q>
struct Tile;

template <>
struct Tile<19> {
  static constexpr int TX = 32, TY = 8, TZ = 8, LX = 5, LY = 3, LZ = 3;
  static constexpr int RZ = 1;  // halo depth along z
};

template <>
struct Tile<9> {
  static constexpr int TX = 64, TY = 32, TZ = 1, LX = 6, LY = 5, LZ = 0;
  static constexpr int RZ = 0;
};

template <int Q>
struct TileGeo {
  static constexpr int TX = Tile<Q>::TX, TY = Tile<Q>::TY, TZ = Tile<Q>::TZ;
  static constexpr int RZ = Tile<Q>::RZ;
  static constexpr int TN = TX * TY * TZ;
  static constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2 * RZ;
  static constexpr int HN = HX * HY * HZ;
  // offset of the neighbour (dx, dy, dz) in the staged table
  __host__ __device__ static constexpr int off(int dx, int dy, int dz) {
    return dx + HX * (dy + HY * dz);
  }
  // staged position of the tile-local node (lx, ly, lz)
  __device__ __forceinline__ static int pos(int lx, int ly, int lz) {
    return (lx + 1) + HX * ((ly + 1) + HY * (lz + RZ));
  }
};

// Entries: class << 30 | index (index < 2^29). A staged position off a
// non-periodic axis holds ENTRY_OUT. In the dense entry box a halo cell off
// a non-periodic axis holds the entry of the clamped position (the stencils'
// zero-gradient rule; periodic axes wrap) with the OUT bit set (the pull
// bounces back, the extrapolations skip it).
constexpr uint32_t ENTRY_OUT = 0x3FFFFFFFu;  // class 0, staging only
constexpr uint32_t OUT_BIT = 1u << 29;
__device__ __forceinline__ int entry_cls(uint32_t e) { return (int)(e >> 30); }
__device__ __forceinline__ int entry_idx(uint32_t e) {
  return (int)(e & 0x1FFFFFFFu);
}
__device__ __forceinline__ bool entry_out(uint32_t e) { return e & OUT_BIT; }

// Tile number of box node (X, Y, Z).
template <int Q>
__device__ __forceinline__ int tile_of(const Dom &d, int X, int Y, int Z) {
  return (X >> Tile<Q>::LX) +
         d.ntx * ((Y >> Tile<Q>::LY) + d.nty * (Z >> Tile<Q>::LZ));
}

// Entry of box node (X, Y, Z) (inside the box).
template <int Q>
__device__ __forceinline__ uint32_t box_entry(const Dom &d, int X, int Y,
                                              int Z) {
  const uint16_t m = __ldg(d.map + (X + d.nx * (Y + d.ny * Z)));
  const int cls = m >> 14;
  const int t = tile_of<Q>(d, X, Y, Z);
  const int base = __ldg(((cls & 2) ? d.fbase : d.sbase) + t);
  return ((uint32_t)cls << 30) | (uint32_t)(base + (m & 0x3FFF));
}

// Stage the table of tile t into tab[HN]; list the tile's fluid and
// solid-boundary nodes (tile-local linear positions) in fpos / spos by rank.
// Returns the tile origin. Ends with __syncthreads().
template <int Q>
__device__ __forceinline__ void stage_tile(const Dom &d, int t, uint32_t *tab,
                                           uint16_t *fpos, uint16_t *spos,
                                           int &X0, int &Y0, int &Z0) {
  using G = TileGeo<Q>;
  const int ttx = t % d.ntx;
  const int q = t / d.ntx;
  const int tty = q % d.nty;
  const int ttz = q / d.nty;
  X0 = ttx * G::TX;
  Y0 = tty * G::TY;
  Z0 = ttz * G::TZ;
  for (int p = threadIdx.x; p < G::HN; p += blockDim.x) {
    const int hx = p % G::HX;
    const int r = p / G::HX;
    const int hy = r % G::HY;
    const int hz = r / G::HY;
    bool out = false;
    const int xr = X0 + hx - 1, yr = Y0 + hy - 1, zr = Z0 + hz - G::RZ;
    const int X = axis_step(xr, d.nx, d.periodic & 1u, false, out);
    const int Y = axis_step(yr, d.ny, d.periodic & 2u, false, out);
    const int Z = axis_step(zr, d.nz, d.periodic & 4u, false, out);
    uint32_t e = ENTRY_OUT;
    if (!out) e = box_entry<Q>(d, X, Y, Z);
    tab[p] = e;
    // members of this tile: interior positions inside the box, no wrap
    const bool interior = hx >= 1 && hx <= G::TX && hy >= 1 && hy <= G::TY &&
                          hz >= G::RZ && hz < G::TZ + G::RZ;
    if (interior && !out && X == xr && Y == yr && Z == zr) {
      const int c = entry_cls(e);
      const uint16_t lp =
          (uint16_t)((hx - 1) + G::TX * ((hy - 1) + G::TY * (hz - G::RZ)));
      if (c & 2) {
        fpos[entry_idx(e) - __ldg(d.fbase + t)] = lp;
      } else if (c == CLS_SOLID_BND) {
        spos[entry_idx(e) - __ldg(d.sbase + t)] = lp;
      }
    }
  }
  __syncthreads();
}

// Box coordinates and staged position of the tile-local node lp.
template <int Q>
__device__ __forceinline__ void local_node(int lp, int X0, int Y0, int Z0,
                                           int &x, int &y, int &z, int &p0) {
  using G = TileGeo<Q>;
  const int lx = lp & (G::TX - 1);
  const int ly = (lp >> Tile<Q>::LX) & (G::TY - 1);
  const int lz = lp >> (Tile<Q>::LX + Tile<Q>::LY);
  x = X0 + lx;
  y = Y0 + ly;
  z = Z0 + lz;
  p0 = G::pos(lx, ly, lz);
}

// Entry of the neighbour x + e with off-box coordinates clamped to the box
// (the zero-gradient rule of the stencils): the staged entry, or, where it
// is OUT, the entry of the clamped position (also staged).
template <int Q>
__device__ __forceinline__ uint32_t clamped_entry(const Dom &d,
                                                  const uint32_t *tab, int p0,
                                                  int x, int y, int z, int dx,
                                                  int dy, int dz) {
  using G = TileGeo<Q>;
  uint32_t e = tab[p0 + G::off(dx, dy, dz)];
  if (e == ENTRY_OUT) {
    const int cx = (x + dx < 0 || x + dx >= d.nx) ? 0 : dx;
    const int cy = (y + dy < 0 || y + dy >= d.ny) ? 0 : dy;
    const int cz = (z + dz < 0 || z + dz >= d.nz) ? 0 : dz;
    e = tab[p0 + G::off(cx, cy, cz)];
  }
  return e;
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
      const bool fl = (entry_cls(e) & 2) && !entry_out(e);
      const int src = guard(d, fl ? entry_idx(e) : k, d.NF, GUARD_PULL);
      ft[i] = IO::load_dyn(d, fl ? i : Lattice<Q>::opp(i), src);
      const float4 S = fl ? ldv<COH>(d.S_src + src) : Sown;
      const float ev = (float)Lattice<Q>::ex(i) * S.y +
                       (float)Lattice<Q>::ey(i) * S.z +
                       (float)Lattice<Q>::ez(i) * S.w;
      rebuild_ev<Q>(ft[i], S.x, fl ? ev : -ev, i, fr, fb);
    }
    rr += fr;
    rb += fb;
  }
}

}  // namespace lbm
