// Set-up passes: node classes; the compact fluid (F) and solid-boundary (S)
// lists, tile by tile, with the per-tile map; the smoothing of Eq. (25) and the wall
// normal of Eq. (26); the initial state; dense export/import of the state and
// fields. These run once or on request, not in the time loop.
#include <cuda_runtime.h>

#include "step.hpp"
#include "tiles.cuh"

namespace lbm {

constexpr int GBLOCK = 256;

static inline unsigned gblocks(long long n) {
  return (unsigned)((n + GBLOCK - 1) / GBLOCK);
}

// A fluid node with a solid lattice neighbour is fluid-boundary; a solid node
// with a fluid lattice neighbour is solid-boundary. Off-box neighbours on a
// non-periodic axis do not count.
template <int Q>
__global__ void k_classify(Dom d, const uint8_t *__restrict__ mask,
                           uint8_t *__restrict__ cls) {
  const long long g = (long long)blockIdx.x * GBLOCK + threadIdx.x;
  if (g >= d.N) return;
  int x, y, z;
  box_coords(d, g, x, y, z);
  const bool solid = mask[g] != 0;
  bool bnd = false;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    bool out = false;
    const int X = axis_step(x + Lattice<Q>::ex(i), d.nx, d.periodic & 1u, false, out);
    const int Y = axis_step(y + Lattice<Q>::ey(i), d.ny, d.periodic & 2u, false, out);
    const int Z = axis_step(z + Lattice<Q>::ez(i), d.nz, d.periodic & 4u, false, out);
    if (out) continue;
    const long long m = X + (long long)d.nx * (Y + (long long)d.ny * Z);
    if ((mask[m] != 0) != solid) bnd = true;
  }
  cls[g] = solid ? (bnd ? CLS_SOLID_BND : CLS_SOLID)
                 : (bnd ? CLS_FLUID_BND : CLS_FLUID);
}

// One block per tile: fluid and solid-boundary counts of the tile.
__global__ void k_tile_count(Dom d, int *__restrict__ cf, int *__restrict__ cs) {
  __shared__ int sf, ss;
  if (threadIdx.x == 0) {
    sf = 0;
    ss = 0;
  }
  __syncthreads();
  const int t = blockIdx.x;
  int X0, Y0, Z0;
  tile_origin(d, t, X0, Y0, Z0);
  const int TN = 1 << (d.tlx + d.tly + d.tlz);
  int nf = 0, ns = 0;
  for (int lp = threadIdx.x; lp < TN; lp += GBLOCK) {
    int x, y, z;
    local_node(d, lp, X0, Y0, Z0, x, y, z);
    if (x >= d.nx || y >= d.ny || z >= d.nz) continue;
    const int c = d.cls[x + d.nx * (y + d.ny * z)];
    nf += (c & 2) ? 1 : 0;
    ns += c == CLS_SOLID_BND ? 1 : 0;
  }
  atomicAdd(&sf, nf);
  atomicAdd(&ss, ns);
  __syncthreads();
  if (threadIdx.x == 0) {
    cf[t] = sf;
    cs[t] = ss;
  }
}

// Exclusive prefix sum of n counts into base[0..n] (base[n] = total), one
// block of 1024 threads walking the array in chunks of 1024.
__global__ void k_scan(const int *__restrict__ cnt, long long n,
                       int *__restrict__ base) {
  __shared__ int warp_tot[32];
  __shared__ int carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (long long off = 0; off < n; off += 1024) {
    const long long i = off + threadIdx.x;
    const int v = i < n ? cnt[i] : 0;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      int t = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += u;
      }
      warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const int before = (warp > 0 ? warp_tot[warp - 1] : 0) + carry;
    if (i < n) base[i] = before + inc - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = before + inc;
    __syncthreads();
  }
  if (threadIdx.x == 0) base[n] = carry;
}

// Device-wide exclusive prefix sum in three launches: per 1024-element
// block a local scan and its total; the single-block scan of the totals;
// the block offsets added back. out has n + 1 entries (out[n] = total),
// bsum ceil(n / 1024) + 1.
__global__ void k_scan_local(const int *__restrict__ in, long long n,
                             int *__restrict__ out, int *__restrict__ bsum) {
  __shared__ int warp_tot[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
  const int v = i < n ? in[i] : 0;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int t = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  const int before = warp > 0 ? warp_tot[warp - 1] : 0;
  if (i < n) out[i] = before + inc - v;
  if (threadIdx.x == 1023) bsum[blockIdx.x] = before + inc;
}

__global__ void k_scan_add(int *__restrict__ out, long long n,
                           const int *__restrict__ bsum, long long nb) {
  const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
  if (i < n) out[i] += bsum[blockIdx.x];
  if (i == 0) out[n] = bsum[nb];
}

static void scan_exclusive(const int *in, int *out, long long n, int *bsum,
                           cudaStream_t s) {
  const long long nb = (n + 1023) / 1024;
  if (nb == 0) {
    cudaMemsetAsync(out, 0, sizeof(int), s);
    return;
  }
  k_scan_local<<<(unsigned)nb, 1024, 0, s>>>(in, n, out, bsum);
  k_scan<<<1, 1024, 0, s>>>(bsum, nb, bsum);  // in place
  k_scan_add<<<(unsigned)nb, 1024, 0, s>>>(out, n, bsum, nb);
}

// One block per tile: rank of each node among the nodes of its kind in the
// tile; map = (class << 14) | rank; the F and S lists hold box indices.
// Fluid nodes on the two x faces of the box (x = 0, x = nx - 1) come first
// in their tile, then the tile's other fluid nodes in (z, y, x) order;
// solid-boundary nodes in (z, y, x) order. With the x faces leading, the
// Zou-He planes of an x-axis flow are runs of consecutive F indices (the
// fix-up pass reads and writes them coalesced) instead of nodes a tile row
// apart; for every other node the order is the plain tile order.
__global__ void k_tile_map(Dom d, uint16_t *__restrict__ map,
                           int *__restrict__ fg, int *__restrict__ sg) {
  __shared__ int wf[GBLOCK / 32], ws[GBLOCK / 32];
  __shared__ int carry_f, carry_s;
  const int t = blockIdx.x;
  int X0, Y0, Z0;
  tile_origin(d, t, X0, Y0, Z0);
  const int TN = 1 << (d.tlx + d.tly + d.tlz);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  if (threadIdx.x == 0) {
    carry_f = 0;
    carry_s = 0;
  }
  __syncthreads();
  // pass 0: the x-face fluid nodes (tiles on an x face only); pass 1: the rest
  const bool face_tile = X0 == 0 || X0 + (1 << d.tlx) >= d.nx;
  for (int pass = face_tile ? 0 : 1; pass < 2; ++pass) {
    for (int c0 = 0; c0 < TN; c0 += GBLOCK) {
      const int lp = c0 + threadIdx.x;
      int x, y, z;
      local_node(d, lp, X0, Y0, Z0, x, y, z);
      // a tile smaller than the block leaves the block's last threads idle
      const bool valid = lp < TN && x < d.nx && y < d.ny && z < d.nz;
      const int g = valid ? x + d.nx * (y + d.ny * z) : 0;
      const int c = valid ? d.cls[g] : CLS_SOLID;
      const bool face = x == 0 || x == d.nx - 1;
      const bool fluid = valid && (c & 2);
      const bool isf = fluid && (pass == 0 ? face : !(face && face_tile));
      const bool iss = pass == 1 && valid && c == CLS_SOLID_BND;
      const unsigned bf = __ballot_sync(0xffffffffu, isf);
      const unsigned bs = __ballot_sync(0xffffffffu, iss);
      if (lane == 0) {
        wf[warp] = __popc(bf);
        ws[warp] = __popc(bs);
      }
      __syncthreads();
      int of = carry_f, os = carry_s;
      for (int w = 0; w < warp; ++w) {
        of += wf[w];
        os += ws[w];
      }
      // the node's map entry is written in the pass that ranks it (every
      // node that is not fluid in pass 1)
      if (valid && (isf || (pass == 1 && !fluid))) {
        int rank = 0;
        if (isf) {
          rank = of + __popc(bf & lt);
          fg[d.fbase[t] + rank] = g;
        } else if (iss) {
          rank = os + __popc(bs & lt);
          sg[d.sbase[t] + rank] = g;
        }
        map[g] = (uint16_t)((c << 14) | rank);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int w = 0; w < GBLOCK / 32; ++w) {
          carry_f += wf[w];
          carry_s += ws[w];
        }
      }
      __syncthreads();
    }
  }
}

// Flags of fluid node k: bit 0 fluid-boundary; bit 1 + 2a / 2 + 2a on the
// first / last plane along axis a.
__global__ void k_fluid_flags(Dom d, uint8_t *__restrict__ fflag) {
  const int k = blockIdx.x * GBLOCK + threadIdx.x;
  if (k >= d.NF) return;
  const int g = d.fg[k];
  int x, y, z;
  box_coords(d, g, x, y, z);
  uint8_t f = d.cls[g] == CLS_FLUID_BND ? 1u : 0u;
  const int c[3] = {x, y, z}, n[3] = {d.nx, d.ny, d.nz};
  for (int a = 0; a < 3; ++a) {
    if (c[a] == 0) f |= (uint8_t)(2u << (2 * a));
    if (c[a] == n[a] - 1) f |= (uint8_t)(4u << (2 * a));
  }
  fflag[k] = f;
}

// One thread per cell of the padded box: the entry of the node that the
// lattice position x (padded position x + 1) stands for. A periodic axis
// wraps; on a non-periodic one an off-box coordinate is clamped to the face
// (the stencils' zero-gradient rule) and the OUT bit is set (the pull
// bounces back, the extrapolations skip it). Since x + e_i, clamped, is x
// or one of its lattice neighbours, a fluid node only ever reaches fluid
// or solid-boundary entries.
template <int Q>
__global__ void k_dense_entries(Dom d, uint32_t *__restrict__ nbd) {
  const long long p = (long long)blockIdx.x * GBLOCK + threadIdx.x;
  if (p >= (long long)d.px * d.py * (d.nz + 2)) return;
  const int hx = (int)(p % d.px);
  const long long r = p / d.px;
  const int hy = (int)(r % d.py);
  const int hz = (int)(r / d.py);
  int c[3] = {hx - 1, hy - 1, hz - 1};
  const int n[3] = {d.nx, d.ny, d.nz};
  bool out = false;
  for (int a = 0; a < 3; ++a) {
    if (c[a] >= 0 && c[a] < n[a]) continue;
    if (d.periodic & (1u << a)) {
      c[a] = c[a] < 0 ? n[a] - 1 : 0;
    } else {
      c[a] = c[a] < 0 ? 0 : n[a] - 1;
      out = true;
    }
  }
  const uint32_t e = box_entry(d, c[0], c[1], c[2]);
  nbd[p] = out ? (e | OUT_BIT) : e;
}

// One thread per solid-boundary node: its fluid lattice neighbours that are
// inside the box (the terms of Eqs. 34-35), in direction order. With
// links == nullptr only their number goes to cnt[j]; otherwise they are
// written from off[j] on as F-index | (diagonal direction) << 31.
template <int Q>
__global__ void k_s_links(Dom d, const int *__restrict__ off,
                          uint32_t *__restrict__ links, int *__restrict__ cnt,
                          uint32_t *__restrict__ dirs) {
  const int j = blockIdx.x * GBLOCK + threadIdx.x;
  if (j >= d.NS) return;
  int x, y, z;
  box_coords(d, d.sg[j], x, y, z);
  const int at = links ? off[j] : 0;
  int n = 0;
  uint32_t mask = 0;
  for (int i = 1; i < Q; ++i) {
    bool out = false;
    const int X = axis_step(x + Lattice<Q>::ex(i), d.nx, d.periodic & 1u, false, out);
    const int Y = axis_step(y + Lattice<Q>::ey(i), d.ny, d.periodic & 2u, false, out);
    const int Z = axis_step(z + Lattice<Q>::ez(i), d.nz, d.periodic & 4u, false, out);
    if (out) continue;
    const uint32_t e = box_entry(d, X, Y, Z);
    if (!(entry_cls(e) & 2)) continue;
    if (links)
      links[at + n] = (uint32_t)entry_idx(e) |
                      (Lattice<Q>::w(i) < Lattice<Q>::w(1) ? 0x80000000u : 0u);
    mask |= 1u << i;
    ++n;
  }
  if (links)
    dirs[j] = mask;
  else
    cnt[j] = n;
}

// Fluid node k on the first or last plane of axis a (a Zou-He plane).
__device__ __forceinline__ int on_planes(const Dom &d, int k, int a) {
  return (d.fflag[k] & (6u << (2 * a))) ? 1 : 0;
}

__global__ void k_zh_mark(Dom d, int a, int *__restrict__ cnt) {
  const int k = blockIdx.x * GBLOCK + threadIdx.x;
  if (k < d.NF) cnt[k] = on_planes(d, k, a);
}

// The Zou-He planes' fluid nodes of axis a in F order: node k goes to
// list[off[k]].
__global__ void k_zh_fill(Dom d, int a, const int *__restrict__ off,
                          int *__restrict__ list) {
  const int k = blockIdx.x * GBLOCK + threadIdx.x;
  if (k < d.NF && on_planes(d, k, a)) list[off[k]] = k;
}

__global__ void k_indicator(long long N, const uint8_t *__restrict__ mask,
                            double *__restrict__ g) {
  const long long n = (long long)blockIdx.x * GBLOCK + threadIdx.x;
  if (n < N) g[n] = mask[n] ? 0.0 : 1.0;
}

// Eq. (25): g^(itr) = sum over the 3x3x3 neighbourhood of
// w_s(i^2+j^2+k^2) g^(itr-1), w_s = 8/27, 2/27, 1/54, 1/216 (3-D) or the
// 3x3 analogue 4/9, 1/9, 1/36 (2-D). Off the box: wrap or clamp.
template <int DIM>
__global__ void k_smooth(Dom d, const double *__restrict__ gin,
                         double *__restrict__ gout) {
  const long long n = (long long)blockIdx.x * GBLOCK + threadIdx.x;
  if (n >= d.N) return;
  int x, y, z;
  box_coords(d, n, x, y, z);
  const double w3[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
  const double w2[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
  constexpr int KR = DIM == 3 ? 1 : 0;
  double acc = 0.0;
#pragma unroll
  for (int k = -KR; k <= KR; ++k)
#pragma unroll
    for (int j = -1; j <= 1; ++j)
#pragma unroll
      for (int i = -1; i <= 1; ++i) {
        bool out = false;
        const int X = axis_step(x + i, d.nx, d.periodic & 1u, true, out);
        const int Y = axis_step(y + j, d.ny, d.periodic & 2u, true, out);
        const int Z = axis_step(z + k, d.nz, d.periodic & 4u, true, out);
        const int r2 = i * i + j * j + k * k;
        acc += (DIM == 3 ? w3[r2] : w2[r2]) *
               gin[X + (long long)d.nx * (Y + (long long)d.ny * Z)];
      }
  gout[n] = acc;
}

// Eq. (26): n_w = grad g^(3) by the Eq. (6) stencil, normalised, at
// fluid-boundary nodes (F-space); zero elsewhere and where it vanishes.
template <int Q>
__global__ void k_wall_normal(Dom d, const double *__restrict__ g3,
                              float4 *__restrict__ nw) {
  const int k = blockIdx.x * GBLOCK + threadIdx.x;
  if (k >= d.NF) return;
  const int g = d.fg[k];
  float4 out4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (d.cls[g] == CLS_FLUID_BND) {
    int x, y, z;
    box_coords(d, g, x, y, z);
    double G[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      bool out = false;
      const int X = axis_step(x + Lattice<Q>::ex(i), d.nx, d.periodic & 1u, true, out);
      const int Y = axis_step(y + Lattice<Q>::ey(i), d.ny, d.periodic & 2u, true, out);
      const int Z = axis_step(z + Lattice<Q>::ez(i), d.nz, d.periodic & 4u, true, out);
      const double p = 3.0 * Lattice<Q>::wd(i) *
                       g3[X + (long long)d.nx * (Y + (long long)d.ny * Z)];
      G[0] += Lattice<Q>::ex(i) * p;
      G[1] += Lattice<Q>::ey(i) * p;
      G[2] += Lattice<Q>::ez(i) * p;
    }
    const double mag = sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
    if (mag > 1e-12)
      out4 = make_float4((float)(G[0] / mag), (float)(G[1] / mag),
                         (float)(G[2] / mag), 0.f);
  }
  nw[k] = out4;
}

__global__ void k_count_fbnd(Dom d, unsigned long long *__restrict__ c) {
  const int k = blockIdx.x * GBLOCK + threadIdx.x;
  const bool b = k < d.NF && d.cls[d.fg[k]] == CLS_FLUID_BND;
  const int n = __syncthreads_count(b);
  if (threadIdx.x == 0 && n) atomicAdd(c, (unsigned long long)n);
}

// Padded box index (one-node halo on every side) of each fluid and
// solid-boundary node, and the face bits of the solid-boundary nodes (as
// fflag: bit 1 + 2a on the first plane of axis a, bit 2 + 2a on the last).
__global__ void k_padded_index(Dom d, int *__restrict__ fgp,
                               int *__restrict__ sgp,
                               uint8_t *__restrict__ sflag) {
  const int k = blockIdx.x * GBLOCK + threadIdx.x;
  const bool fluid = k < d.NF;
  if (!fluid && k >= d.NF + d.NS) return;
  const int g = fluid ? d.fg[k] : d.sg[k - d.NF];
  int x, y, z;
  box_coords(d, g, x, y, z);
  const int gp = (x + 1) + d.px * ((y + 1) + d.py * (z + 1));
  if (fluid) {
    fgp[k] = gp;
    return;
  }
  const int c[3] = {x, y, z}, n[3] = {d.nx, d.ny, d.nz};
  uint8_t f = 0;
  for (int a = 0; a < 3; ++a) {
    if (c[a] == 0) f |= (uint8_t)(2u << (2 * a));
    if (c[a] == n[a] - 1) f |= (uint8_t)(4u << (2 * a));
  }
  sgp[k - d.NF] = gp;
  sflag[k - d.NF] = f;
}

cudaError_t build_geometry(lbm_ctx *c, cudaStream_t s) {
  Dom &d = c->d;
  const unsigned gN = gblocks(d.N);
  uint8_t *cls = const_cast<uint8_t *>(d.cls);
  if (c->Q == 19)
    k_classify<19><<<gN, GBLOCK, 0, s>>>(d, c->mask, cls);
  else
    k_classify<9><<<gN, GBLOCK, 0, s>>>(d, c->mask, cls);
  const unsigned nt = (unsigned)c->ntiles;
  k_tile_count<<<nt, GBLOCK, 0, s>>>(d, c->cnt_f, c->cnt_s);
  k_scan<<<1, 1024, 0, s>>>(c->cnt_f, c->ntiles, const_cast<int *>(d.fbase));
  k_scan<<<1, 1024, 0, s>>>(c->cnt_s, c->ntiles, const_cast<int *>(d.sbase));
  uint16_t *map = const_cast<uint16_t *>(d.map);
  int *fg = const_cast<int *>(d.fg), *sg = const_cast<int *>(d.sg);
  k_tile_map<<<nt, GBLOCK, 0, s>>>(d, map, fg, sg);
  int tot[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(&tot[0], d.fbase + c->ntiles, sizeof(int),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&tot[1], d.sbase + c->ntiles, sizeof(int),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  if (tot[0] != d.NF || tot[1] > d.NS) return cudaErrorInvalidValue;
  d.NS = tot[1];
  c->n_fluid = tot[0];
  c->n_sbnd = tot[1];
  {
    uint32_t *nbd = const_cast<uint32_t *>(d.nbd);
    const long long P = (long long)d.px * d.py * (d.nz + 2);
    k_fluid_flags<<<gblocks(d.NF), GBLOCK, 0, s>>>(
        d, const_cast<uint8_t *>(d.fflag));
    if (c->Q == 19)
      k_dense_entries<19><<<gblocks(P), GBLOCK, 0, s>>>(d, nbd);
    else
      k_dense_entries<9><<<gblocks(P), GBLOCK, 0, s>>>(d, nbd);
  }
  // Eq. (25) three times, then Eq. (26) at the fluid-boundary nodes
  k_indicator<<<gN, GBLOCK, 0, s>>>(d.N, c->mask, c->g0);
  double *gi = c->g0, *go = c->g1;
  for (int itr = 0; itr < 3; ++itr) {
    if (c->Q == 19)
      k_smooth<3><<<gN, GBLOCK, 0, s>>>(d, gi, go);
    else
      k_smooth<2><<<gN, GBLOCK, 0, s>>>(d, gi, go);
    double *t = gi;
    gi = go;
    go = t;
  }
  const unsigned gF = gblocks(d.NF);
  float4 *nw = const_cast<float4 *>(d.nw);
  if (c->Q == 19)
    k_wall_normal<19><<<gF, GBLOCK, 0, s>>>(d, gi, nw);
  else
    k_wall_normal<9><<<gF, GBLOCK, 0, s>>>(d, gi, nw);
  // the smoothing buffers are free from here on: scan scratch
  int *cnt = (int *)c->g0;
  int *bsum = (int *)c->g1;
  int *pos = bsum + ((d.N + 1023) / 1024 + 2);
  // links of the solid-boundary nodes (Eqs. 34-35)
  const unsigned gS = gblocks(d.NS);
  int *soff = const_cast<int *>(d.soff);
  uint32_t *slink = const_cast<uint32_t *>(d.slink);
  uint32_t *sdir = const_cast<uint32_t *>(d.sdir);
  if (d.NS > 0) {
    if (c->Q == 19)
      k_s_links<19><<<gS, GBLOCK, 0, s>>>(d, nullptr, nullptr, cnt, nullptr);
    else
      k_s_links<9><<<gS, GBLOCK, 0, s>>>(d, nullptr, nullptr, cnt, nullptr);
  }
  scan_exclusive(cnt, soff, d.NS, bsum, s);
  if (d.NS > 0) {
    if (c->Q == 19)
      k_s_links<19><<<gS, GBLOCK, 0, s>>>(d, soff, slink, nullptr, sdir);
    else
      k_s_links<9><<<gS, GBLOCK, 0, s>>>(d, soff, slink, nullptr, sdir);
  }
  // the Zou-He planes' fluid nodes per axis, in F order
  int zh_n[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a) {
    k_zh_mark<<<gF, GBLOCK, 0, s>>>(d, a, cnt);
    scan_exclusive(cnt, pos, d.NF, bsum, s);
    k_zh_fill<<<gF, GBLOCK, 0, s>>>(d, a, pos, c->zh_lists + (size_t)a * d.NFp);
    e = cudaMemcpyAsync(&zh_n[a], pos + d.NF, sizeof(int),
                        cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(c->counters, 0, 4 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_count_fbnd<<<gF, GBLOCK, 0, s>>>(d, c->counters);
  k_padded_index<<<gblocks((long long)d.NF + d.NS), GBLOCK, 0, s>>>(
      d, const_cast<int *>(d.fgp), const_cast<int *>(d.sgp),
      const_cast<uint8_t *>(d.sflag));
  unsigned long long nfb = 0;
  e = cudaMemcpyAsync(&nfb, c->counters, sizeof(nfb), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  c->n_fbnd = (long long)nfb;
  for (int a = 0; a < 3; ++a) c->zh_count[a] = zh_n[a];
  return cudaGetLastError();
}

// ------------------------------------------------ injected-fluid swap
// Sec. II.D.1, Eqs. (37)-(38) on the stored state: at every fluid node of
// the inlet plane (coordinate 0 of the flow axis, first half of the Zou-He
// list) the populations of the other colour join colour `blue ? b : r`:
// f^s_i += f^sbar_i, f^sbar_i = 0. In the stored form (f''_i, q, v) that is
// f''_i unchanged, the minority fraction q = 0 with colour s the majority,
// and v = 0 (the minority part of every population is zero).
__global__ void k_swap_inlet(Dom d, bool blue) {
  const int j = blockIdx.x * GBLOCK + threadIdx.x;
  if (j >= d.n_zh) return;
  const int k = d.zh_list[j];
  if (!(d.fflag[k] & (2u << (2 * d.c.axis)))) return;  // outlet node
  const_cast<float4 *>(d.S_src)[k] = make_float4(m_pack(blue, 0.f), 0.f, 0.f, 0.f);
}

void launch_swap_inlet(const Dom &d, bool blue, cudaStream_t s) {
  if (d.n_zh > 0) k_swap_inlet<<<gblocks(d.n_zh), GBLOCK, 0, s>>>(d, blue);
}

// ------------------------------------------------------------ state I/O
// Fluid at rest: f^s_i = w_i rho^s, i.e. f''_i = w_i rho0, q from phi0, v = 0.
template <int Q, int ST>
__global__ void k_init_state(Dom d, const float *__restrict__ phi0) {
  const int k = blockIdx.x * GBLOCK + threadIdx.x;
  if (k < d.NF) {
    const float p = phi0[d.fg[k]];
    const float m = m_pack(p < 0.f, 0.5f * (1.f - fabsf(p)));
#pragma unroll
    for (int i = 0; i < Q; ++i)
      TIO<Q, ST>::store(d, d.T_dst, i, k, Lattice<Q>::w(i) * d.c.rho0);
    d.S_dst[k] = make_float4(m, 0.f, 0.f, 0.f);
    d.mf[k] = m;
    d.ncf[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    d.macro[k] = make_float4(0.f, 0.f, 0.f, d.c.rho0);
  }
  if (k < d.NS) {
    d.ms[k] = 0.5f;  // phi = 0 until the first step fills Eq. (34)
    d.ncs[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

template <int Q, int ST>
__global__ void k_export(Dom d, float *__restrict__ dst) {
  const int k = blockIdx.x * GBLOCK + threadIdx.x;
  if (k >= d.NF) return;
  const int g = d.fg[k];
  const float4 S = d.S_src[k];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float r, b;
    rebuild<Q>(TIO<Q, ST>::load(d, i, k), S, i, r, b);
    dst[(long long)i * d.N + g] = r;
    dst[(long long)(Q + i) * d.N + g] = b;
  }
}

// Import of arbitrary f^r, f^b: f''_i = f^r_i + f^b_i, q from the colour
// densities, v from the minority colour's momentum (sum_i w_i e_i e_i = I/3):
// v = 3 (sum_i e_i f^r_i - mu j) where red is the minority, else
// v = 3 (mu j - sum_i e_i f^b_i). Exact for a post-recolouring state.
template <int Q, int ST>
__global__ void k_import(Dom d, const float *__restrict__ src) {
  const int k = blockIdx.x * GBLOCK + threadIdx.x;
  if (k >= d.NF) return;
  const int g = d.fg[k];
  float rr = 0.f, rb = 0.f, j[3] = {0.f, 0.f, 0.f}, jr[3] = {0.f, 0.f, 0.f},
        jb[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float r = src[(long long)i * d.N + g];
    const float b = src[(long long)(Q + i) * d.N + g];
    rr += r;
    rb += b;
    const float e3[3] = {(float)Lattice<Q>::ex(i), (float)Lattice<Q>::ey(i),
                         (float)Lattice<Q>::ez(i)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      jr[a] += e3[a] * r;
      jb[a] += e3[a] * b;
      j[a] += e3[a] * (r + b);
    }
    TIO<Q, ST>::store(d, d.T_dst, i, k, r + b);
  }
  const bool blue = rr < rb;
  const float mu = fminf(rr, rb) / (rr + rb);
  float v[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    v[a] = blue ? 3.f * (jr[a] - mu * j[a]) : 3.f * (mu * j[a] - jb[a]);
  d.S_dst[k] = make_float4(m_pack(blue, mu), v[0], v[1], v[2]);
}

template <int Q, int ST>
static void init_t(const Dom &d, const float *phi0, cudaStream_t s) {
  const long long n = d.NF > d.NS ? d.NF : d.NS;
  k_init_state<Q, ST><<<gblocks(n), GBLOCK, 0, s>>>(d, phi0);
}

// The state kernels write the current buffers: a copy of d whose T_dst and
// S_dst point at them.
void launch_init_state(int Q, int st, const Dom &d0, const float *phi0,
                       cudaStream_t s) {
  Dom d = d0;
  d.T_dst = const_cast<void *>(d.T_src);
  d.S_dst = const_cast<float4 *>(d.S_src);
  if (Q == 19) {
    if (st == 0) init_t<19, 0>(d, phi0, s);
    if (st == 1) init_t<19, 1>(d, phi0, s);
    if (st == 2) init_t<19, 2>(d, phi0, s);
  } else {
    if (st == 0) init_t<9, 0>(d, phi0, s);
    if (st == 1) init_t<9, 1>(d, phi0, s);
    if (st == 2) init_t<9, 2>(d, phi0, s);
  }
}

void launch_export_pops(int Q, int st, const Dom &d, float *dst,
                        cudaStream_t s) {
  cudaMemsetAsync(dst, 0, sizeof(float) * 2 * Q * (size_t)d.N, s);
  const unsigned g = gblocks(d.NF);
#define LBM_EXP(QQ, SS) k_export<QQ, SS><<<g, GBLOCK, 0, s>>>(d, dst)
  if (Q == 19) {
    if (st == 0) LBM_EXP(19, 0);
    if (st == 1) LBM_EXP(19, 1);
    if (st == 2) LBM_EXP(19, 2);
  } else {
    if (st == 0) LBM_EXP(9, 0);
    if (st == 1) LBM_EXP(9, 1);
    if (st == 2) LBM_EXP(9, 2);
  }
#undef LBM_EXP
}

void launch_import_pops(int Q, int st, const Dom &d0, const float *src,
                        cudaStream_t s) {
  Dom d = d0;
  d.T_dst = const_cast<void *>(d.T_src);
  d.S_dst = const_cast<float4 *>(d.S_src);
  const unsigned g = gblocks(d.NF);
#define LBM_IMP(QQ, SS) k_import<QQ, SS><<<g, GBLOCK, 0, s>>>(d, src)
  if (Q == 19) {
    if (st == 0) LBM_IMP(19, 0);
    if (st == 1) LBM_IMP(19, 1);
    if (st == 2) LBM_IMP(19, 2);
  } else {
    if (st == 0) LBM_IMP(9, 0);
    if (st == 1) LBM_IMP(9, 1);
    if (st == 2) LBM_IMP(9, 2);
  }
#undef LBM_IMP
}

// Dense fields of the last macro step: rho, phi (solid-boundary nodes:
// Eq. 34), u; zero elsewhere.
__global__ void k_export_macros(Dom d, float *__restrict__ rho,
                                float *__restrict__ phi, float *__restrict__ u) {
  const int k = blockIdx.x * GBLOCK + threadIdx.x;
  if (k < d.NF) {
    const int g = d.fg[k];
    const float4 m = d.macro[k];
    if (rho) rho[g] = m.w;
    if (phi) phi[g] = m_phi(d.mf[k]);
    if (u) {
      u[g] = m.x;
      u[d.N + g] = m.y;
      u[2 * d.N + g] = m.z;
    }
  }
  if (k < d.NS && phi) phi[d.sg[k]] = m_phi(d.ms[k]);
}

void launch_export_macros(const Dom &d, float *rho, float *phi, float *u,
                          cudaStream_t s) {
  if (rho) cudaMemsetAsync(rho, 0, sizeof(float) * (size_t)d.N, s);
  if (phi) cudaMemsetAsync(phi, 0, sizeof(float) * (size_t)d.N, s);
  if (u) cudaMemsetAsync(u, 0, sizeof(float) * 3 * (size_t)d.N, s);
  const long long n = d.NF > d.NS ? d.NF : d.NS;
  k_export_macros<<<gblocks(n), GBLOCK, 0, s>>>(d, rho, phi, u);
}

__global__ void k_export_nw(Dom d, float *__restrict__ out) {
  const int k = blockIdx.x * GBLOCK + threadIdx.x;
  if (k >= d.NF) return;
  const int g = d.fg[k];
  const float4 v = d.nw[k];
  out[g] = v.x;
  out[d.N + g] = v.y;
  out[2 * d.N + g] = v.z;
}

void launch_export_nw(const Dom &d, float *out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(float) * 3 * (size_t)d.N, s);
  k_export_nw<<<gblocks(d.NF), GBLOCK, 0, s>>>(d, out);
}

}  // namespace lbm
