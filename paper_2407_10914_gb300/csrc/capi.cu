// The C-ABI of include/lbmgb.h: argument checks, workspace layout, launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "step.hpp"

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

size_t pop_bytes(int Q, long long Np, int storage) {
  return storage == LBM_STORAGE_FP32 ? (size_t)2 * Q * Np * sizeof(float)
                                     : (size_t)Q * Np * 4;  // half2 pairs
}

// Byte offsets of every buffer inside the caller's workspace.
struct Layout {
  size_t fA, fB, phi, nc, cls, nw, sbnd, mask, rho, u, red, out, cnt, total;
};

Layout make_layout(int Q, long long N, long long Np, int storage,
                   long long n_solid) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  const size_t pb = pop_bytes(Q, Np, storage);
  L.fA = take(pb);
  // the smoothing ping-pong buffers (2 x 8N bytes, set-up only) live in fB
  L.fB = take(pb > (size_t)16 * N ? pb : (size_t)16 * N);
  L.phi = take((size_t)N * 4);
  L.nc = take((size_t)N * 16);
  L.cls = take((size_t)N);
  L.nw = take((size_t)N * 16);
  L.sbnd = take((size_t)(n_solid > 0 ? n_solid : 1) * 4);
  L.mask = take((size_t)N);
  L.rho = take((size_t)N * 4);
  L.u = take((size_t)N * 12);
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
  return N < (1LL << 31);  // node indices are stored as int32 in lists
}

long long count_solid(const uint8_t *solid, long long N) {
  if (!solid) return N;
  long long k = 0;
  for (long long n = 0; n < N; ++n) k += solid[n] != 0;
  return k;
}

}  // namespace

extern "C" {

size_t lbm_workspace_bytes(int lattice, int nx, int ny, int nz,
                           const uint8_t *solid_host, int storage) {
  if (!valid_shape(lattice, nx, ny, nz)) return 0;
  if (storage < 0 || storage > 2) return 0;
  const long long N = (long long)nx * ny * nz;
  return make_layout(lattice, N, pad64(N), storage,
                     count_solid(solid_host, N)).total;
}

lbm_status lbm_init_geometry(lbm_handle *out, int lattice, int nx, int ny,
                             int nz, const uint8_t *solid_host,
                             unsigned periodic_mask, int storage,
                             void *ws, size_t ws_bytes, void *stream) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  if (!valid_shape(lattice, nx, ny, nz) || !solid_host || !ws ||
      storage < 0 || storage > 2 || periodic_mask > 7u)
    return LBM_ERR_ARG;
  if (((uintptr_t)ws) % ALIGN) return LBM_ERR_ARG;
  const long long N = (long long)nx * ny * nz;
  const long long Np = pad64(N);
  const long long n_solid = count_solid(solid_host, N);
  if (n_solid == N) return LBM_ERR_ARG;  // no fluid node
  const Layout L = make_layout(lattice, N, Np, storage, n_solid);
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
  c->Np = Np;
  c->periodic = periodic_mask;
  c->storage = storage;
  c->fA = base + L.fA;
  c->fB = base + L.fB;
  c->mask = (uint8_t *)(base + L.mask);
  c->g0 = (double *)(base + L.fB);
  c->g1 = (double *)(base + L.fB) + N;
  c->red = (double *)(base + L.red);
  c->red_slots = RED_SLOTS;
  c->red_out = (double *)(base + L.out);
  c->counters = (unsigned long long *)(base + L.cnt);
  Dom &d = c->d;
  d.nx = nx;
  d.ny = ny;
  d.nz = nz;
  d.N = N;
  d.Np = Np;
  d.periodic = periodic_mask;
  d.f_src = c->fA;
  d.f_dst = c->fB;
  d.phi = (float *)(base + L.phi);
  d.nc = (float4 *)(base + L.nc);
  d.cls = (const uint8_t *)(base + L.cls);
  d.nw = (const float4 *)(base + L.nw);
  d.sbnd = (const int *)(base + L.sbnd);
  d.n_sbnd = 0;
  d.rho_m = (float *)(base + L.rho);
  d.u_m = (float *)(base + L.u);
  cudaError_t e = cudaMemcpyAsync(c->mask, solid_host, (size_t)N,
                                  cudaMemcpyHostToDevice, s);
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
  k.gamma = (float)p->gamma;
  k.beta = (float)p->beta;
  k.rho0 = (float)p->rho0;
  const double th = p->theta_deg * 3.14159265358979323846 / 180.0;
  k.theta = (float)th;
  k.cos_t = (float)std::cos(th);
  k.sin_t = (float)std::sin(th);
  k.wetting = p->wetting;
  k.zou_he = p->zou_he;
  k.axis = p->flow_axis;
  k.rho_in_r = (float)(p->rho_in * p->zeta_r);
  k.rho_in_b = (float)(p->rho_in * (1.0 - p->zeta_r));
  k.rho_out = (float)p->rho_out;
  k.phi_in = (float)(p->zeta_r - (1.0 - p->zeta_r));
  for (int a = 0; a < 3; ++a) k.g[a] = (float)p->g[a];
  c->params_set = true;
  return LBM_OK;
}

lbm_status lbm_init_state(lbm_handle c, const float *phi0, void *stream) {
  if (!c || !phi0) return LBM_ERR_ARG;
  if (!c->params_set) return fail(c, LBM_ERR_STATE, "set params first");
  lbm::launch_init_state(c->Q, c->storage, c->d, phi0, (cudaStream_t)stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "init_state");
  c->state_set = true;
  return LBM_OK;
}

lbm_status lbm_step(lbm_handle c, int nsteps, void *stream) {
  if (!c || nsteps < 0) return LBM_ERR_ARG;
  if (!c->state_set) return fail(c, LBM_ERR_STATE, "init the state first");
  cudaStream_t s = (cudaStream_t)stream;
  for (int k = 0; k < nsteps; ++k) {
    lbm::launch_step(c->Q, c->storage, c->d, s, k == nsteps - 1);
    void *t = c->d.f_src;
    c->d.f_src = c->d.f_dst;
    c->d.f_dst = t;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "step");
  return LBM_OK;
}

lbm_status lbm_step_timed(lbm_handle c, int nsteps, void *stream,
                          double *pass_ms) {
  if (!c || nsteps < 0 || !pass_ms) return LBM_ERR_ARG;
  if (!c->state_set) return fail(c, LBM_ERR_STATE, "init the state first");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t ev[6];
  int made = 0;
  cudaError_t e = cudaSuccess;
  for (; made < 6 && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
  if (e != cudaSuccess) {
    for (int k = 0; k + 1 < made; ++k) cudaEventDestroy(ev[k]);
    return cuda_fail(c, e, "step_timed events");
  }
  for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
    lbm::launch_step_events(c->Q, c->storage, c->d, s, k == nsteps - 1, ev);
    void *t = c->d.f_src;
    c->d.f_src = c->d.f_dst;
    c->d.f_dst = t;
    e = cudaEventSynchronize(ev[5]);
    for (int p = 0; p < 5 && e == cudaSuccess; ++p) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[p], ev[p + 1]);
      pass_ms[p] += ms;
    }
  }
  for (int k = 0; k < 6; ++k) cudaEventDestroy(ev[k]);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "step_timed");
  return LBM_OK;
}

lbm_status lbm_macros(lbm_handle c, float *rho, float *phi, float *u,
                      void *stream) {
  if (!c) return LBM_ERR_ARG;
  if (!c->state_set) return fail(c, LBM_ERR_STATE, "init the state first");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t b = (size_t)c->N * sizeof(float);
  cudaError_t e = cudaSuccess;
  if (rho && e == cudaSuccess)
    e = cudaMemcpyAsync(rho, c->d.rho_m, b, cudaMemcpyDeviceToDevice, s);
  if (phi && e == cudaSuccess)
    e = cudaMemcpyAsync(phi, c->d.phi, b, cudaMemcpyDeviceToDevice, s);
  if (u && e == cudaSuccess)
    e = cudaMemcpyAsync(u, c->d.u_m, 3 * b, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "macros");
  return LBM_OK;
}

lbm_status lbm_reduce(lbm_handle c, int kind, double *out, void *stream) {
  if (!c || !out || kind < 0 || kind > LBM_CA_B) return LBM_ERR_ARG;
  if (!c->state_set) return fail(c, LBM_ERR_STATE, "init the state first");
  cudaStream_t s = (cudaStream_t)stream;
  double *dev_out = c->red_out;
  lbm::launch_reduce(c->Q, c->storage, c->d, kind, c->red, c->red_slots,
                     dev_out, s);
  double h[4];
  cudaError_t e = cudaMemcpyAsync(h, dev_out, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "reduce");
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

const char *lbm_last_error(lbm_handle c) { return c ? c->err : "null handle"; }

void lbm_destroy(lbm_handle c) { delete c; }

}  // extern "C"
