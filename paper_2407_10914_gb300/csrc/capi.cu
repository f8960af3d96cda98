// The C-ABI of include/lbmgb.h: argument checks, workspace layout, launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "step.hpp"
#include "tiles.cuh"

using lbm::Dom;

namespace {

constexpr size_t ALIGN = 256;
constexpr int RED_SLOTS = 1024;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

long long pad64(long long n) { return (n + 63) / 64 * 64; }

lbm_status fail(lbm_ctx *c, lbm_status st, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

lbm_status cuda_fail(lbm_ctx *c, cudaError_t e, const char *where) {
  return fail(c, LBM_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

long long count_solid(const uint8_t *solid, long long N) {
  if (!solid) return 0;
  long long k = 0;
  for (long long n = 0; n < N; ++n) k += solid[n] != 0;
  return k;
}

// Byte offsets of every buffer inside the caller's workspace.
struct Layout {
  size_t TA, TB, U, R, SA, SB, mf, ncf, kap, nw, fg, macro;  // F-space
  size_t ms, ncs, sg, sgp, sflag, sdir, smark;    // S-space
  size_t phib, fgp;                               // dense phase field
  size_t nbd, soff, slink, fflag, zh;             // neighbour lookup
  size_t map, cls, mask, fbase, sbase, cntf, cnts, g0, g1;
  size_t red, out, cnt, total;
  long long NF, NFp, NS, ntiles;
  int ntx, nty, ntz;
};

// NF is the number of fluid nodes; NS an upper bound of the solid-boundary
// nodes (the number of solid nodes).
// Tile extents as log2 (lx, ly, lz): the caller's tile[3] (powers of two,
// x extent 32..1024, at most 2^14 nodes, z extent 1 for D2Q9) or, for a
// null tile, 32 x 8 x 8 (D3Q19) / 64 x 32 x 1 (D2Q9). False if invalid.
bool tile_shape(int Q, const int *tile, int lg[3]) {
  if (!tile) {
    lg[0] = Q == 19 ? 5 : 6;
    lg[1] = Q == 19 ? 3 : 5;
    lg[2] = Q == 19 ? 3 : 0;
    return true;
  }
  for (int a = 0; a < 3; ++a) {
    const int t = tile[a];
    if (t < 1 || t > 1024 || (t & (t - 1))) return false;
    lg[a] = 0;
    while ((1 << lg[a]) < t) ++lg[a];
  }
  if (lg[0] < lbm::TILE_MIN_LX || lg[0] > lbm::TILE_MAX_LX) return false;
  if (lg[0] + lg[1] + lg[2] > lbm::TILE_MAX_LN) return false;
  return Q == 19 || lg[2] == 0;
}

Layout make_layout(int Q, int nx, int ny, int nz, int storage, long long NF,
                   long long NS, const int lg[3]) {
  Layout L{};
  const long long N = (long long)nx * ny * nz;
  L.NF = NF;
  L.NFp = pad64(NF > 0 ? NF : 1);
  L.NS = NS;
  const int TX = 1 << lg[0], TY = 1 << lg[1], TZ = 1 << lg[2];
  L.ntx = (nx + TX - 1) / TX;
  L.nty = (ny + TY - 1) / TY;
  L.ntz = (nz + TZ - 1) / TZ;
  L.ntiles = (long long)L.ntx * L.nty * L.ntz;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + (bytes > 0 ? bytes : 1));
    return at;
  };
  const size_t tb = (size_t)Q * L.NFp * (storage == LBM_STORAGE_FP32 ? 4 : 2);
  const size_t nfp = (size_t)L.NFp, nsp = (size_t)pad64(NS > 0 ? NS : 1);
  L.TA = take(tb);
  L.TB = take(tb);
  L.U = take(tb);
  L.R = take(nfp * 8);
  L.SA = take(nfp * 16);
  L.SB = take(nfp * 16);
  L.mf = take(nfp * 4);
  L.ncf = take(nfp * 16);
  L.kap = take(nfp * 4);
  L.nw = take(nfp * 16);
  L.fg = take(nfp * 4);
  L.macro = take(nfp * 16);
  L.ms = take(nsp * 4);
  L.ncs = take(nsp * 16);
  L.sg = take(nsp * 4);
  L.sgp = take(nsp * 4);
  L.sflag = take(nsp);
  L.sdir = take(nsp * 4);
  L.smark = take(nsp);
  L.fgp = take(nfp * 4);
  L.phib = take((size_t)(nx + 2) * (ny + 2) * (nz + 2) * 4);
  L.nbd = take((size_t)(nx + 2) * (ny + 2) * (nz + 2) * 4);
  L.soff = take((nsp + 1) * 4);
  // Links of the solid-boundary nodes: at most Q - 1 per node, and, since
  // each link reversed is a distinct (fluid node, direction) pair, at most
  // Q - 1 per fluid node too
  L.slink = take((size_t)(Q - 1) * (nsp < nfp ? nsp : nfp) * 4);
  L.fflag = take(nfp);
  L.zh = take(3 * nfp * 4);
  L.map = take((size_t)N * 2);
  L.cls = take((size_t)N);
  L.mask = take((size_t)N);
  L.fbase = take((size_t)(L.ntiles + 1) * 4);
  L.sbase = take((size_t)(L.ntiles + 1) * 4);
  L.cntf = take((size_t)L.ntiles * 4);
  L.cnts = take((size_t)L.ntiles * 4);
  L.g0 = take((size_t)N * 8);
  L.g1 = take((size_t)N * 8);
  L.red = take((size_t)RED_SLOTS * 4 * 8);
  L.out = take(4 * 8);
  L.cnt = take(4 * 8);
  L.total = o;
  return L;
}

bool valid_shape(int lattice, int nx, int ny, int nz) {
  if (lattice != 9 && lattice != 19) return false;
  if (nx < 1 || ny < 1 || nz < 1) return false;
  if (lattice == 9 && nz != 1) return false;
  const long long N = (long long)nx * ny * nz;
  const long long P = (long long)(nx + 2) * (ny + 2) * (nz + 2);
  return N < (1LL << 31) && P < (1LL << 31);  // box indices are int32
}

void swap_buffers(lbm_ctx *c) { lbm::swap_state(c); }

}  // namespace

extern "C" {

size_t lbm_workspace_bytes_tiled(int lattice, int nx, int ny, int nz,
                                 const uint8_t *solid_host, int storage,
                                 const int *tile) {
  int lg[3];
  if (!valid_shape(lattice, nx, ny, nz)) return 0;
  if (storage < 0 || storage > 2 || !tile_shape(lattice, tile, lg)) return 0;
  const long long N = (long long)nx * ny * nz;
  const long long ns = solid_host ? count_solid(solid_host, N) : N;
  const long long nf = solid_host ? N - ns : N;
  return make_layout(lattice, nx, ny, nz, storage, nf, ns, lg).total;
}

size_t lbm_workspace_bytes(int lattice, int nx, int ny, int nz,
                           const uint8_t *solid_host, int storage) {
  return lbm_workspace_bytes_tiled(lattice, nx, ny, nz, solid_host, storage,
                                   nullptr);
}

lbm_status lbm_init_geometry(lbm_handle *out, int lattice, int nx, int ny,
                             int nz, const uint8_t *solid_host,
                             unsigned periodic_mask, int storage,
                             void *ws, size_t ws_bytes, void *stream) {
  return lbm_init_geometry_tiled(out, lattice, nx, ny, nz, solid_host,
                                 periodic_mask, storage, nullptr, ws,
                                 ws_bytes, stream);
}

lbm_status lbm_init_geometry_tiled(lbm_handle *out, int lattice, int nx,
                                   int ny, int nz, const uint8_t *solid_host,
                                   unsigned periodic_mask, int storage,
                                   const int *tile, void *ws, size_t ws_bytes,
                                   void *stream) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  int lg[3];
  if (!valid_shape(lattice, nx, ny, nz) || !solid_host || !ws ||
      storage < 0 || storage > 2 || periodic_mask > 7u ||
      !tile_shape(lattice, tile, lg))
    return LBM_ERR_ARG;
  if (((uintptr_t)ws) % ALIGN) return LBM_ERR_ARG;
  const long long N = (long long)nx * ny * nz;
  const long long n_solid = count_solid(solid_host, N);
  if (n_solid == N) return LBM_ERR_ARG;  // no fluid node
  // node indices travel in 29 bits of a neighbour entry
  if (N - n_solid >= (1LL << 29) || n_solid >= (1LL << 29)) return LBM_ERR_ARG;
  const Layout L = make_layout(lattice, nx, ny, nz, storage, N - n_solid,
                               n_solid, lg);
  if (ws_bytes < L.total) return LBM_ERR_NOMEM;
  lbm_ctx *c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ERR_NOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  char *base = (char *)ws;
  c->Q = lattice;
  c->nx = nx;
  c->ny = ny;
  c->nz = nz;
  c->N = N;
  c->periodic = periodic_mask;
  c->storage = storage;
  c->ntiles = L.ntiles;
  c->TA = base + L.TA;
  c->TB = base + L.TB;
  c->SA = (float4 *)(base + L.SA);
  c->SB = (float4 *)(base + L.SB);
  c->mask = (uint8_t *)(base + L.mask);
  c->g0 = (double *)(base + L.g0);
  c->g1 = (double *)(base + L.g1);
  c->cnt_f = (int *)(base + L.cntf);
  c->cnt_s = (int *)(base + L.cnts);
  c->red = (double *)(base + L.red);
  c->red_slots = RED_SLOTS;
  c->red_out = (double *)(base + L.out);
  c->counters = (unsigned long long *)(base + L.cnt);
  Dom &d = c->d;
  d.nx = nx;
  d.ny = ny;
  d.nz = nz;
  d.N = N;
  d.periodic = periodic_mask;
  d.ntx = L.ntx;
  d.nty = L.nty;
  d.ntz = L.ntz;
  d.tlx = lg[0];
  d.tly = lg[1];
  d.tlz = lg[2];
  d.ntiles = (int)L.ntiles;
  d.NF = (int)L.NF;
  d.NS = (int)L.NS;  // upper bound until the lists are built
  d.NFp = L.NFp;
  d.map = (const uint16_t *)(base + L.map);
  d.fbase = (const int *)(base + L.fbase);
  d.sbase = (const int *)(base + L.sbase);
  d.fg = (const int *)(base + L.fg);
  d.sg = (const int *)(base + L.sg);
  d.cls = (const uint8_t *)(base + L.cls);
  d.nbd = (const uint32_t *)(base + L.nbd);
  d.soff = (const int *)(base + L.soff);
  d.slink = (const uint32_t *)(base + L.slink);
  d.fflag = (const uint8_t *)(base + L.fflag);
  c->zh_lists = (int *)(base + L.zh);
  d.zh_list = c->zh_lists;
  d.n_zh = 0;
  d.nw = (const float4 *)(base + L.nw);
  d.U = base + L.U;
  d.R = (float2 *)(base + L.R);
  d.T_src = c->TA;
  d.T_dst = c->TB;
  d.S_src = c->SA;
  d.S_dst = c->SB;
  d.mf = (float *)(base + L.mf);
  d.ms = (float *)(base + L.ms);
  d.ncf = (float4 *)(base + L.ncf);
  d.kap = (float *)(base + L.kap);
  d.ncs = (float4 *)(base + L.ncs);
  d.macro = (float4 *)(base + L.macro);
  d.phib = (float *)(base + L.phib);
  d.fgp = (const int *)(base + L.fgp);
  d.sgp = (const int *)(base + L.sgp);
  d.sflag = (const uint8_t *)(base + L.sflag);
  d.sdir = (const uint32_t *)(base + L.sdir);
  d.smark = (uint8_t *)(base + L.smark);
  d.px = nx + 2;
  d.py = ny + 2;
  d.err = (unsigned *)(c->counters + 3);  // zeroed with the counters at set-up
  cudaError_t e = cudaMemcpyAsync(c->mask, solid_host, (size_t)N,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.smark, 0, (size_t)(L.NS > 0 ? L.NS : 1), s);
  if (e == cudaSuccess) e = lbm::build_geometry(c, s);
  if (e != cudaSuccess) {
    delete c;
    return LBM_ERR_CUDA;
  }
  *out = c;
  return LBM_OK;
}

lbm_status lbm_set_params(lbm_handle c, const lbm_params *p) {
  if (!c || !p) return LBM_ERR_ARG;
  if (!(p->tau_r > 0.5) || !(p->tau_b > 0.5))
    return fail(c, LBM_ERR_ARG, "tau must exceed 1/2");
  if (!(p->beta >= 0.0 && p->beta <= 1.0))
    return fail(c, LBM_ERR_ARG, "beta outside [0,1]");
  if (!(p->gamma >= 0.0)) return fail(c, LBM_ERR_ARG, "gamma < 0");
  if (!(p->rho0 > 0.0)) return fail(c, LBM_ERR_ARG, "rho0 <= 0");
  if (!(p->theta_deg > 0.0 && p->theta_deg < 180.0))
    return fail(c, LBM_ERR_ARG, "theta outside (0,180)");
  if (p->wetting < 0 || p->wetting > 2)
    return fail(c, LBM_ERR_ARG, "wetting must be 0, 1 or 2");
  if (p->flow_axis < 0 || p->flow_axis > 2)
    return fail(c, LBM_ERR_ARG, "flow_axis must be 0, 1 or 2");
  if (p->zou_he != 0 && p->zou_he != 1)
    return fail(c, LBM_ERR_ARG, "zou_he must be 0 or 1");
  if (p->collision != 0 && p->collision != 1)
    return fail(c, LBM_ERR_ARG, "collision must be 0 or 1");
  if (p->collision == 1 && c->Q != 19)
    return fail(c, LBM_ERR_ARG, "MRT collision is defined for D3Q19 only");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(p->g[a])) return fail(c, LBM_ERR_ARG, "g not finite");
  if (p->zou_he) {
    const int ext = p->flow_axis == 0 ? c->nx : (p->flow_axis == 1 ? c->ny : c->nz);
    if (c->periodic & (1u << p->flow_axis))
      return fail(c, LBM_ERR_ARG, "Zou-He needs a non-periodic flow axis");
    if (ext < 3) return fail(c, LBM_ERR_ARG, "Zou-He needs >= 3 planes");
    if (!(p->rho_in > 0.0) || !(p->rho_out > 0.0))
      return fail(c, LBM_ERR_ARG, "Zou-He densities must be > 0");
    if (!(p->zeta_r >= 0.0 && p->zeta_r <= 1.0))
      return fail(c, LBM_ERR_ARG, "zeta_r outside [0,1]");
  }
  c->p = *p;
  lbm::StepConst &k = c->d.c;
  k.nu_r = (float)((p->tau_r - 0.5) / 3.0);
  k.nu_b = (float)((p->tau_b - 0.5) / 3.0);
  k.h_r = (float)(1.5 / (p->tau_r - 0.5));
  k.h_b = (float)(1.5 / (p->tau_b - 0.5));
  k.gamma = (float)p->gamma;
  k.beta = (float)p->beta;
  k.rho0 = (float)p->rho0;
  const double th = p->theta_deg * 3.14159265358979323846 / 180.0;
  k.cos_t = (float)std::cos(th);
  k.sin_t = (float)std::sin(th);
  k.wetting = p->wetting;
  k.zou_he = p->zou_he;
  k.axis = p->flow_axis;
  c->d.zh_list = c->zh_lists + (size_t)p->flow_axis * c->d.NFp;
  c->d.n_zh = p->zou_he ? (int)c->zh_count[p->flow_axis] : 0;
  k.rho_in_r = (float)(p->rho_in * p->zeta_r);
  k.rho_in_b = (float)(p->rho_in * (1.0 - p->zeta_r));
  k.rho_out = (float)p->rho_out;
  {
    // encoded inlet phase field: minority fraction, majority flag in the
    // lowest mantissa bit (1 = blue)
    const double phi_in = p->zeta_r - (1.0 - p->zeta_r);
    const float mu = (float)(0.5 * (1.0 - std::fabs(phi_in)));
    uint32_t bits;
    std::memcpy(&bits, &mu, 4);
    bits = (bits & ~1u) | (phi_in < 0.0 ? 1u : 0u);
    std::memcpy(&k.m_in, &bits, 4);
  }
  for (int a = 0; a < 3; ++a) k.g[a] = (float)p->g[a];
  k.mrt = p->collision;
  c->params_set = true;
  ++c->pgen;  // recorded step graphs hold the old parameters
  ++c->gen;
  return LBM_OK;
}

lbm_status lbm_init_state(lbm_handle c, const float *phi0, void *stream) {
  if (!c || !phi0) return LBM_ERR_ARG;
  if (!c->params_set) return fail(c, LBM_ERR_STATE, "set params first");
  lbm::launch_init_state(c->Q, c->storage, c->d, phi0, (cudaStream_t)stream);
  // the stored curvature is read (and discarded) at nodes without an
  // interface too: keep it defined
  cudaError_t e = cudaMemsetAsync(c->d.kap, 0, (size_t)c->d.NFp * sizeof(float),
                                  (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "init_state");
  c->state_set = true;
  ++c->gen;
  return LBM_OK;
}

// The graph of two steps without macros for the current orientation of the
// state buffers, recorded on first use (or after lbm_set_params); null if
// the stream cannot be captured (lbm_step then launches step by step).
static cudaGraphExec_t step_pair_graph(lbm_ctx *c) {
  const int o = c->d.T_src == c->TA ? 0 : 1;
  if (c->g2[o] && c->g2_pgen[o] == c->pgen) return c->g2[o];
  if (c->g2[o]) {
    cudaGraphExecDestroy(c->g2[o]);
    c->g2[o] = nullptr;
  }
  cudaError_t e = cudaSuccess;
  if (!c->cap) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return nullptr;
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int k = 0; k < 2; ++k) {  // two swaps: the orientation comes back
      lbm::launch_step(c->Q, c->storage, c->d, c->cap, false);
      swap_buffers(c);
    }
    e = cudaStreamEndCapture(c->cap, &g);
  }
  cudaGraphExec_t x = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear a capture error; step without a graph
    return nullptr;
  }
  c->g2[o] = x;
  c->g2_pgen[o] = c->pgen;
  return x;
}

lbm_status lbm_step(lbm_handle c, int nsteps, void *stream) {
  if (!c || nsteps < 0) return LBM_ERR_ARG;
  if (!c->state_set) return fail(c, LBM_ERR_STATE, "init the state first");
  cudaStream_t s = (cudaStream_t)stream;
  // all steps but the last (which also stores the macros) in pairs from
  // the recorded graph, then the odd one and the last by plain launches;
  // the kernels and their arguments are the same either way
  int k = 0;
  const int pairs = (nsteps - 1) / 2;
  cudaGraphExec_t g = pairs > 0 ? step_pair_graph(c) : nullptr;
  if (g) {
    for (int p = 0; p < pairs; ++p) {
      const cudaError_t e = cudaGraphLaunch(g, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "step graph");
    }
    k = 2 * pairs;
  }
  for (; k < nsteps; ++k) {
    lbm::launch_step(c->Q, c->storage, c->d, s, k == nsteps - 1);
    swap_buffers(c);
  }
  ++c->gen;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "step");
  return LBM_OK;
}

lbm_status lbm_step_timed(lbm_handle c, int nsteps, void *stream,
                          double *pass_ms) {
  if (!c || nsteps < 0 || !pass_ms) return LBM_ERR_ARG;
  if (!c->state_set) return fail(c, LBM_ERR_STATE, "init the state first");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t ev[LBM_N_PASSES + 1];
  int made = 0;
  cudaError_t e = cudaSuccess;
  for (; made < LBM_N_PASSES + 1 && e == cudaSuccess; ++made)
    e = cudaEventCreate(&ev[made]);
  if (e != cudaSuccess) {
    for (int k = 0; k + 1 < made; ++k) cudaEventDestroy(ev[k]);
    return cuda_fail(c, e, "step_timed events");
  }
  ++c->gen;
  for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
    lbm::launch_step_events(c->Q, c->storage, c->d, s, k == nsteps - 1, ev);
    swap_buffers(c);
    e = cudaEventSynchronize(ev[LBM_N_PASSES]);
    for (int p = 0; p < LBM_N_PASSES && e == cudaSuccess; ++p) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[p], ev[p + 1]);
      pass_ms[p] += ms;
    }
  }
  for (int k = 0; k < LBM_N_PASSES + 1; ++k) cudaEventDestroy(ev[k]);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "step_timed");
  return LBM_OK;
}

lbm_status lbm_macros(lbm_handle c, float *rho, float *phi, float *u,
                      void *stream) {
  if (!c) return LBM_ERR_ARG;
  if (!c->state_set) return fail(c, LBM_ERR_STATE, "init the state first");
  lbm::launch_export_macros(c->d, rho, phi, u, (cudaStream_t)stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "macros");
  return LBM_OK;
}

lbm_status lbm_reduce_async(lbm_handle c, int kind, double *raw4,
                            void *stream) {
  if (!c || !raw4 || kind < 0 || kind > LBM_CA_B) return LBM_ERR_ARG;
  if (!c->state_set) return fail(c, LBM_ERR_STATE, "init the state first");
  cudaStream_t s = (cudaStream_t)stream;
  lbm::launch_reduce(c->Q, c->storage, c->d, kind, c->red, c->red_slots,
                     c->red_out, s);
  cudaError_t e = cudaMemcpyAsync(raw4, c->red_out, 4 * sizeof(double),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "reduce");
  return LBM_OK;
}

lbm_status lbm_reduce(lbm_handle c, int kind, double *out, void *stream) {
  if (!c || !out || kind < 0 || kind > LBM_CA_B) return LBM_ERR_ARG;
  double h[4];
  const lbm_status st = lbm_reduce_async(c, kind, h, stream);
  if (st != LBM_OK) return st;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "reduce");
  return lbm_reduce_value(c, kind, h, out);
}

lbm_status lbm_reduce_value(lbm_handle c, int kind, const double *h,
                            double *out) {
  if (!c || !h || !out || kind < 0 || kind > LBM_CA_B) return LBM_ERR_ARG;
  double v = 0.0;
  const double nf = (double)c->n_fluid;
  switch (kind) {
    case LBM_MASS_R:
    case LBM_MASS_B:
      v = h[0];
      break;
    case LBM_SW_COUNT:
    case LBM_SW_SMOOTH:
      v = h[0] / nf;
      break;
    case LBM_DP:
      v = ((h[1] > 0 ? h[0] / h[1] : 0.0) - (h[3] > 0 ? h[2] / h[3] : 0.0)) / 3.0;
      break;
    default: {
      const double tau = kind == LBM_CA_R ? c->p.tau_r : c->p.tau_b;
      const double mu = c->p.rho0 * (tau - 0.5) / 3.0;
      v = h[1] > 0 ? mu * (h[0] / h[1]) / c->p.gamma : 0.0;
    }
  }
  *out = v;
  if (!std::isfinite(v)) return fail(c, LBM_ERR_NONFINITE, "reduction not finite");
  return LBM_OK;
}

lbm_status lbm_get_populations(lbm_handle c, float *dst, void *stream) {
  if (!c || !dst) return LBM_ERR_ARG;
  if (!c->state_set) return fail(c, LBM_ERR_STATE, "init the state first");
  lbm::launch_export_pops(c->Q, c->storage, c->d, dst, (cudaStream_t)stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "get_populations");
  return LBM_OK;
}

lbm_status lbm_set_populations(lbm_handle c, const float *src, void *stream) {
  if (!c || !src) return LBM_ERR_ARG;
  if (!c->params_set) return fail(c, LBM_ERR_STATE, "set params first");
  lbm::launch_import_pops(c->Q, c->storage, c->d, src, (cudaStream_t)stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "set_populations");
  c->state_set = true;
  ++c->gen;
  return LBM_OK;
}

lbm_status lbm_debug_flags(lbm_handle c, unsigned *out_host, void *stream) {
  if (!c || !out_host) return LBM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(out_host, c->d.err, sizeof(unsigned),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "debug_flags");
  return LBM_OK;
}

lbm_status lbm_swap_inlet(lbm_handle c, int colour, void *stream) {
  if (!c) return LBM_ERR_ARG;
  if (colour != 0 && colour != 1)
    return fail(c, LBM_ERR_ARG, "colour must be 0 (r) or 1 (b)");
  if (!c->state_set) return fail(c, LBM_ERR_STATE, "init the state first");
  if (!c->p.zou_he)
    return fail(c, LBM_ERR_STATE, "the inlet plane is a Zou-He plane: zou_he = 1");
  lbm::launch_swap_inlet(c->d, colour == 1, (cudaStream_t)stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "swap_inlet");
  ++c->gen;
  return LBM_OK;
}

lbm_status lbm_get_geometry(lbm_handle c, uint8_t *cls, float *nw,
                            void *stream) {
  if (!c) return LBM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (cls)
    e = cudaMemcpyAsync(cls, c->d.cls, (size_t)c->N, cudaMemcpyDeviceToDevice, s);
  if (nw && e == cudaSuccess) {
    lbm::launch_export_nw(c->d, nw, s);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "get_geometry");
  return LBM_OK;
}

lbm_status lbm_counts(lbm_handle c, int64_t *n_nodes, int64_t *n_fluid,
                      int64_t *n_sbnd, int64_t *n_fbnd) {
  if (!c) return LBM_ERR_ARG;
  if (n_nodes) *n_nodes = c->N;
  if (n_fluid) *n_fluid = c->n_fluid;
  if (n_sbnd) *n_sbnd = c->n_sbnd;
  if (n_fbnd) *n_fbnd = c->n_fbnd;
  return LBM_OK;
}

size_t lbm_state_bytes(lbm_handle c) {
  if (!c) return 0;
  const size_t bp = c->storage == LBM_STORAGE_FP32 ? 4 : 2;
  return (size_t)c->Q * (size_t)c->d.NFp * bp + (size_t)c->d.NFp * 16;
}

lbm_status lbm_save_state(lbm_handle c, void *dst_dev, void *stream) {
  if (!c || !dst_dev) return LBM_ERR_ARG;
  if (!c->state_set) return fail(c, LBM_ERR_STATE, "no state to save");
  const size_t tb = lbm_state_bytes(c) - (size_t)c->d.NFp * 16;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(dst_dev, c->d.T_src, tb,
                                  cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((char *)dst_dev + tb, c->d.S_src,
                        (size_t)c->d.NFp * 16, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "save_state");
  return LBM_OK;
}

lbm_status lbm_load_state(lbm_handle c, const void *src_dev, void *stream) {
  if (!c || !src_dev) return LBM_ERR_ARG;
  if (!c->params_set) return fail(c, LBM_ERR_STATE, "set params first");
  const size_t tb = lbm_state_bytes(c) - (size_t)c->d.NFp * 16;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(const_cast<void *>(c->d.T_src), src_dev, tb,
                                  cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(const_cast<float4 *>(c->d.S_src),
                        (const char *)src_dev + tb, (size_t)c->d.NFp * 16,
                        cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "load_state");
  c->state_set = true;
  ++c->gen;
  return LBM_OK;
}

const char *lbm_last_error(lbm_handle c) { return c ? c->err : "null handle"; }

void lbm_destroy(lbm_handle c) { delete c; }

}  // extern "C"
