// Set-up passes: node classes, the smoothing of Eq. (25), the wall normal of
// Eq. (26), the solid-boundary list; the initial state; dense population
// export/import. These run once (or on request), not in the time loop.
#include <cuda_runtime.h>

#include "stencil.cuh"
#include "step.hpp"

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
  const long long n = (long long)blockIdx.x * GBLOCK + threadIdx.x;
  if (n >= d.N) return;
  int x, y, z;
  node_coords(d, n, x, y, z);
  const bool solid = mask[n] != 0;
  bool bnd = false;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    bool out = false;
    const long long m = nb_index(d, x, y, z, Lattice<Q>::e(i, 0),
                                 Lattice<Q>::e(i, 1), Lattice<Q>::e(i, 2),
                                 false, out);
    if (!out && ((mask[m] != 0) != solid)) bnd = true;
  }
  cls[n] = solid ? (bnd ? CLS_SOLID_BND : CLS_SOLID)
                 : (bnd ? CLS_FLUID_BND : CLS_FLUID);
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
  node_coords(d, n, x, y, z);
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
        const long long m = nb_index(d, x, y, z, i, j, k, true, out);
        const int r2 = i * i + j * j + k * k;
        acc += (DIM == 3 ? w3[r2] : w2[r2]) * gin[m];
      }
  gout[n] = acc;
}

// Eq. (26): n_w = grad g^(3) by the Eq. (6) stencil, normalised, at
// fluid-boundary nodes; zero elsewhere (and where the gradient vanishes).
template <int Q>
__global__ void k_wall_normal(Dom d, const double *__restrict__ g,
                              float4 *__restrict__ nw) {
  const long long n = (long long)blockIdx.x * GBLOCK + threadIdx.x;
  if (n >= d.N) return;
  float4 out4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (d.cls[n] == CLS_FLUID_BND) {
    int x, y, z;
    node_coords(d, n, x, y, z);
    double G[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      bool out = false;
      const long long m = nb_index(d, x, y, z, Lattice<Q>::e(i, 0),
                                   Lattice<Q>::e(i, 1), Lattice<Q>::e(i, 2),
                                   true, out);
      const double p = 3.0 * Lattice<Q>::wd(i) * g[m];
#pragma unroll
      for (int a = 0; a < 3; ++a) G[a] += Lattice<Q>::e(i, a) * p;
    }
    const double mag = sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
    if (mag > 1e-12)
      out4 = make_float4((float)(G[0] / mag), (float)(G[1] / mag),
                         (float)(G[2] / mag), 0.f);
  }
  nw[n] = out4;
}

// Compact list of solid-boundary nodes and the counts (fluid, solid-bnd,
// fluid-bnd) in counters[0..2]. The list order is irrelevant to the results.
__global__ void k_lists(Dom d, int *__restrict__ sbnd,
                        unsigned long long *__restrict__ counters) {
  const long long n = (long long)blockIdx.x * GBLOCK + threadIdx.x;
  if (n >= d.N) return;
  const uint8_t c = d.cls[n];
  if (c & 2) atomicAdd(&counters[0], 1ull);
  if (c == CLS_FLUID_BND) atomicAdd(&counters[2], 1ull);
  if (c == CLS_SOLID_BND) {
    const unsigned long long k = atomicAdd(&counters[1], 1ull);
    sbnd[k] = (int)n;
  }
}

cudaError_t build_geometry(lbm_ctx *c, cudaStream_t s) {
  Dom &d = c->d;
  const unsigned g = gblocks(d.N);
  uint8_t *cls = const_cast<uint8_t *>(d.cls);
  if (c->Q == 19)
    k_classify<19><<<g, GBLOCK, 0, s>>>(d, c->mask, cls);
  else
    k_classify<9><<<g, GBLOCK, 0, s>>>(d, c->mask, cls);
  k_indicator<<<g, GBLOCK, 0, s>>>(d.N, c->mask, c->g0);
  double *gi = c->g0, *go = c->g1;
  for (int itr = 0; itr < 3; ++itr) {
    if (c->Q == 19)
      k_smooth<3><<<g, GBLOCK, 0, s>>>(d, gi, go);
    else
      k_smooth<2><<<g, GBLOCK, 0, s>>>(d, gi, go);
    double *t = gi;
    gi = go;
    go = t;
  }
  float4 *nw = const_cast<float4 *>(d.nw);
  if (c->Q == 19)
    k_wall_normal<19><<<g, GBLOCK, 0, s>>>(d, gi, nw);
  else
    k_wall_normal<9><<<g, GBLOCK, 0, s>>>(d, gi, nw);
  cudaError_t e = cudaMemsetAsync(c->counters, 0, 4 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_lists<<<g, GBLOCK, 0, s>>>(d, const_cast<int *>(d.sbnd), c->counters);
  unsigned long long h[4] = {0, 0, 0, 0};
  e = cudaMemcpyAsync(h, c->counters, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  c->n_fluid = (long long)h[0];
  c->n_sbnd = (long long)h[1];
  c->n_fbnd = (long long)h[2];
  d.n_sbnd = (int)h[1];
  return cudaGetLastError();
}

// ------------------------------------------------------------ state I/O
template <int Q, int ST>
__global__ void k_init_state(Dom d, const float *__restrict__ phi0) {
  const long long n = (long long)blockIdx.x * GBLOCK + threadIdx.x;
  if (n >= d.N) return;
  const PopIO<Q, ST> io(d);
  const bool fluid = is_fluid_cls(d.cls[n]);
  float r = 0.f, b = 0.f;
  if (fluid) {
    const float p = phi0[n];
    r = d.c.rho0 * 0.5f * (1.f + p);
    b = d.c.rho0 * 0.5f * (1.f - p);
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float w = Lattice<Q>::w(i);
    if (fluid)
      io.store(i, n, w * r, w * b);
    else
      io.store(i, n, 0.f, 0.f);
  }
  d.phi[n] = fluid ? (r - b) / (r + b) : 0.f;
  d.nc[n] = make_float4(0.f, 0.f, 0.f, 0.f);
  d.rho_m[n] = fluid ? r + b : 0.f;
  d.u_m[n] = 0.f;
  d.u_m[d.N + n] = 0.f;
  d.u_m[2 * d.N + n] = 0.f;
}

template <int Q, int ST>
__global__ void k_export(Dom d, float *__restrict__ dst) {
  const long long n = (long long)blockIdx.x * GBLOCK + threadIdx.x;
  if (n >= d.N) return;
  const PopIO<Q, ST> io(d);
  const bool fluid = is_fluid_cls(d.cls[n]);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float r = 0.f, b = 0.f;
    if (fluid) io.load(i, n, r, b);
    dst[(long long)i * d.N + n] = r;
    dst[(long long)(Q + i) * d.N + n] = b;
  }
}

template <int Q, int ST>
__global__ void k_import(Dom d, const float *__restrict__ src) {
  const long long n = (long long)blockIdx.x * GBLOCK + threadIdx.x;
  if (n >= d.N) return;
  const PopIO<Q, ST> io(d);
  const bool fluid = is_fluid_cls(d.cls[n]);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float r = 0.f, b = 0.f;
    if (fluid) {
      r = src[(long long)i * d.N + n];
      b = src[(long long)(Q + i) * d.N + n];
    }
    io.store(i, n, r, b);
  }
}

// The state kernels write the current buffer: a copy of d with f_dst
// pointing at it.
void launch_init_state(int Q, int st, const Dom &d0, const float *phi0,
                       cudaStream_t s) {
  Dom d = d0;
  d.f_dst = d.f_src;
  const unsigned g = gblocks(d.N);
#define LBM_INIT(QQ, SS) k_init_state<QQ, SS><<<g, GBLOCK, 0, s>>>(d, phi0)
  if (Q == 19) {
    if (st == 0) LBM_INIT(19, 0);
    if (st == 1) LBM_INIT(19, 1);
    if (st == 2) LBM_INIT(19, 2);
  } else {
    if (st == 0) LBM_INIT(9, 0);
    if (st == 1) LBM_INIT(9, 1);
    if (st == 2) LBM_INIT(9, 2);
  }
#undef LBM_INIT
}

void launch_export_pops(int Q, int st, const Dom &d, float *dst,
                        cudaStream_t s) {
  const unsigned g = gblocks(d.N);
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
  d.f_dst = d.f_src;
  const unsigned g = gblocks(d.N);
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

}  // namespace lbm

namespace lbm {

__global__ void k_export_nw(Dom d, float *__restrict__ out) {
  const long long n = (long long)blockIdx.x * GBLOCK + threadIdx.x;
  if (n >= d.N) return;
  const float4 v = d.nw[n];
  out[n] = v.x;
  out[d.N + n] = v.y;
  out[2 * d.N + n] = v.z;
}

void launch_export_nw(const Dom &d, float *out, cudaStream_t s) {
  k_export_nw<<<gblocks(d.N), GBLOCK, 0, s>>>(d, out);
}

}  // namespace lbm
