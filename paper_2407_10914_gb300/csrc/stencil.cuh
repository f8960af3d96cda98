// Device building blocks of the step: neighbour arithmetic, population
// storage policies, the pull of Eq. (1) with halfway bounce-back, Zou-He
// (App. B), the wetting schemes (Eqs. 28-33) and the collision (Eq. 2,
// single-rate form) with recolouring (Eqs. 20-21). All arithmetic is FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "context.hpp"
#include "lattice.cuh"

namespace lbm {

constexpr float EPS_C = 1e-8f;        // |C| at or below: no interface
constexpr float EPS_SIN = 1e-6f;      // Scheme-II: n_c parallel to n_w
constexpr float EPS_SECANT = 1e-12f;  // Scheme-I: secant denominator

__device__ __forceinline__ void node_coords(const Dom &d, long long n, int &x,
                                            int &y, int &z) {
  long long q = n / d.nx;
  x = (int)(n - q * d.nx);
  z = (int)(q / d.ny);
  y = (int)(q - (long long)z * d.ny);
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

__device__ __forceinline__ long long nb_index(const Dom &d, int x, int y,
                                              int z, int dx, int dy, int dz,
                                              bool clamp, bool &out) {
  int X = axis_step(x + dx, d.nx, d.periodic & 1u, clamp, out);
  int Y = axis_step(y + dy, d.ny, d.periodic & 2u, clamp, out);
  int Z = axis_step(z + dz, d.nz, d.periodic & 4u, clamp, out);
  return X + (long long)d.nx * (Y + (long long)d.ny * Z);
}

__device__ __forceinline__ bool is_fluid_cls(uint8_t c) { return c & 2; }

// ------------------------------------------------------------ storage
// Populations as float32: plane (s*Q + i) of stride Np.
template <int Q, int STORAGE>
struct PopIO;

template <int Q>
struct PopIO<Q, LBM_STORAGE_FP32> {
  const float *__restrict__ src;
  float *__restrict__ dst;
  long long Np;
  float rho0;
  __device__ __forceinline__ PopIO(const Dom &d)
      : src((const float *)d.f_src), dst((float *)d.f_dst), Np(d.Np),
        rho0(d.c.rho0) {}
  __device__ __forceinline__ void load(int i, long long n, float &r,
                                       float &b) const {
    r = __ldg(src + (long long)i * Np + n);
    b = __ldg(src + (long long)(Q + i) * Np + n);
  }
  __device__ __forceinline__ void store(int i, long long n, float r,
                                        float b) const {
    dst[(long long)i * Np + n] = r;
    dst[(long long)(Q + i) * Np + n] = b;
  }
};

// 16-bit offset storage: per (i, n) one pair (T'_i, D'_i) with
// T'_i = (f^r_i + f^b_i - w_i rho0)/w_i and D'_i = (f^r_i - f^b_i)/w_i,
// so that both are O(1) numbers; arithmetic stays FP32.
template <typename H2>
struct Half2Conv;
template <>
struct Half2Conv<__half2> {
  __device__ __forceinline__ static float2 to(__half2 h) {
    return __half22float2(h);
  }
  __device__ __forceinline__ static __half2 from(float a, float b) {
    return __floats2half2_rn(a, b);
  }
};
template <>
struct Half2Conv<__nv_bfloat162> {
  __device__ __forceinline__ static float2 to(__nv_bfloat162 h) {
    return __bfloat1622float2(h);
  }
  __device__ __forceinline__ static __nv_bfloat162 from(float a, float b) {
    return __floats2bfloat162_rn(a, b);
  }
};

template <int Q, typename H2>
struct PopIO16 {
  const H2 *__restrict__ src;
  H2 *__restrict__ dst;
  long long Np;
  float rho0;
  __device__ __forceinline__ PopIO16(const Dom &d)
      : src((const H2 *)d.f_src), dst((H2 *)d.f_dst), Np(d.Np),
        rho0(d.c.rho0) {}
  __device__ __forceinline__ void load(int i, long long n, float &r,
                                       float &b) const {
    const float w = Lattice<Q>::w(i);
    float2 v = Half2Conv<H2>::to(src[(long long)i * Np + n]);
    float t = w * (v.x + rho0);
    float dd = w * v.y;
    r = 0.5f * (t + dd);
    b = 0.5f * (t - dd);
  }
  __device__ __forceinline__ void store(int i, long long n, float r,
                                        float b) const {
    const float iw = 1.0f / Lattice<Q>::w(i);
    dst[(long long)i * Np + n] =
        Half2Conv<H2>::from((r + b) * iw - rho0, (r - b) * iw);
  }
};

template <int Q>
struct PopIO<Q, LBM_STORAGE_FP16> : PopIO16<Q, __half2> {
  __device__ __forceinline__ PopIO(const Dom &d) : PopIO16<Q, __half2>(d) {}
};
template <int Q>
struct PopIO<Q, LBM_STORAGE_BF16> : PopIO16<Q, __nv_bfloat162> {
  __device__ __forceinline__ PopIO(const Dom &d)
      : PopIO16<Q, __nv_bfloat162>(d) {}
};

// --------------------------------------------------------------- pull
// Eq. (1), propagation: f^s_i(x) = f^s_i*(x - e_i) when x - e_i is a fluid
// node of the box (periodic axes wrap), else the halfway bounce-back
// f^s_opp(i)*(x).
template <int Q, int STORAGE>
__device__ __forceinline__ void pull(const Dom &d, const PopIO<Q, STORAGE> &io,
                                     long long n, int x, int y, int z,
                                     float *fr, float *fb) {
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    bool out = false;
    long long src = nb_index(d, x, y, z, -Lattice<Q>::e(i, 0),
                             -Lattice<Q>::e(i, 1), -Lattice<Q>::e(i, 2),
                             false, out);
    if (i != 0 && (out || !is_fluid_cls(d.cls[src])))
      io.load(Lattice<Q>::opp(i), n, fr[i], fb[i]);
    else
      io.load(i, src, fr[i], fb[i]);
  }
}

// ------------------------------------------------------------- Zou-He
// Appendix B on a flow axis a. Inlet (coordinate 0), per colour with the
// species density rho_s = rho_in zeta^s:
//   j = rho_s - [sum_{e.a=0} f + 2 sum_{e.a=-1} f],
//   N_t = 1/2 sum_{e.a=0} (e.t) f,
//   f_i = f_opp(i) + 6 w_i j - sum_{t != a} (e_i.t) N_t      (e_i.a = +1).
template <int Q>
__device__ __forceinline__ void zou_he_inlet(float *f, float rho_s, int a) {
  float known = 0.f, Nt[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int ea = Lattice<Q>::e(i, a);
    if (ea == 0) {
      known += f[i];
#pragma unroll
      for (int t = 0; t < 3; ++t)
        if (t != a) Nt[t] += 0.5f * (float)Lattice<Q>::e(i, t) * f[i];
    } else if (ea == -1) {
      known += 2.f * f[i];
    }
  }
  const float j = rho_s - known;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (Lattice<Q>::e(i, a) != 1) continue;
    float corr = 0.f;
#pragma unroll
    for (int t = 0; t < 3; ++t)
      if (t != a) corr += (float)Lattice<Q>::e(i, t) * Nt[t];
    f[i] = f[Lattice<Q>::opp(i)] + 6.f * Lattice<Q>::w(i) * j - corr;
  }
}

// Outlet (last coordinate): total j^t = -rho_out + [sum_{e.a=0} f^t +
// 2 sum_{e.a=+1} f^t] (B.9); per colour, with chi^s of (B.12)-(B.13):
//   f_i = f_opp(i) - 6 w_i j^t chi^s - sum_{t != a} (e_i.t) N_t (e_i.a = -1).
template <int Q>
__device__ __forceinline__ void zou_he_outlet(float *fr, float *fb,
                                              float rho_out, float phi_out,
                                              int a) {
  float known = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int ea = Lattice<Q>::e(i, a);
    if (ea == 0) known += fr[i] + fb[i];
    if (ea == 1) known += 2.f * (fr[i] + fb[i]);
  }
  const float jt = known - rho_out;
  const float chi[2] = {0.5f * (1.f + phi_out), 0.5f * (1.f - phi_out)};
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    float *f = s == 0 ? fr : fb;
    float Nt[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (Lattice<Q>::e(i, a) != 0) continue;
#pragma unroll
      for (int t = 0; t < 3; ++t)
        if (t != a) Nt[t] += 0.5f * (float)Lattice<Q>::e(i, t) * f[i];
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (Lattice<Q>::e(i, a) != -1) continue;
      float corr = 0.f;
#pragma unroll
      for (int t = 0; t < 3; ++t)
        if (t != a) corr += (float)Lattice<Q>::e(i, t) * Nt[t];
      f[i] = f[Lattice<Q>::opp(i)] - 6.f * Lattice<Q>::w(i) * jt * chi[s] - corr;
    }
  }
}

__device__ __forceinline__ int axis_coord(int x, int y, int z, int a) {
  return a == 0 ? x : (a == 1 ? y : z);
}
__device__ __forceinline__ int axis_extent(const Dom &d, int a) {
  return a == 0 ? d.nx : (a == 1 ? d.ny : d.nz);
}

template <int Q>
__device__ __forceinline__ void sum_colours(const float *fr, const float *fb,
                                            float &rr, float &rb) {
  rr = 0.f;
  rb = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    rr += fr[i];
    rb += fb[i];
  }
}

// ------------------------------------------------------------ wetting
__device__ __forceinline__ float dot3(const float *a, const float *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Eq. (28): f(v) = v.n_w - |v| cos(theta)
__device__ __forceinline__ float secant_f(const float *v, const float *nw,
                                          float cth) {
  return dot3(v, nw) - sqrtf(dot3(v, v)) * cth;
}

// Scheme-I, Eqs. (29)-(31): v0 = n_c, v1 = n_c - (n_c + n_w)/2, three secant
// updates (n = 2, 3, 4), early stop on a vanishing denominator, then
// normalise; a zero-length result leaves n_c unchanged.
__device__ __forceinline__ void scheme1(float *nc, const float *nw, float cth) {
  float vm2[3], vm1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    vm2[a] = nc[a];
    vm1[a] = nc[a] - 0.5f * (nc[a] + nw[a]);
  }
#pragma unroll
  for (int it = 2; it <= 4; ++it) {
    const float f1 = secant_f(vm1, nw, cth);
    const float f2 = secant_f(vm2, nw, cth);
    const float den = f1 - f2;
    if (fabsf(den) < EPS_SECANT) break;
    const float inv = 1.f / den;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float vn = (vm2[a] * f1 - vm1[a] * f2) * inv;
      vm2[a] = vm1[a];
      vm1[a] = vn;
    }
  }
  const float m = sqrtf(dot3(vm1, vm1));
  if (m > 0.f) {
    const float im = 1.f / m;
#pragma unroll
    for (int a = 0; a < 3; ++a) nc[a] = vm1[a] * im;
  }
}

// Scheme-II, Eqs. (32)-(33): with c = n_w.n_c = cos(theta') and
// s' = sin(theta') = sqrt(1 - c^2),
//   n_+- = (cos(theta) -+ sin(theta) c/s') n_w +- (sin(theta)/s') n_c,
// keep the one nearer to n_c (n_+ on a tie); unchanged when s' < EPS_SIN.
__device__ __forceinline__ void scheme2(float *nc, const float *nw, float cth,
                                        float sth) {
  float c = fminf(1.f, fmaxf(-1.f, dot3(nw, nc)));
  const float sp = sqrtf(fmaxf(0.f, 1.f - c * c));
  if (sp < EPS_SIN) return;
  const float k = sth / sp;
  float np_[3], nm_[3], dp = 0.f, dm = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    np_[a] = (cth - k * c) * nw[a] + k * nc[a];
    nm_[a] = (cth + k * c) * nw[a] - k * nc[a];
    dp += (np_[a] - nc[a]) * (np_[a] - nc[a]);
    dm += (nm_[a] - nc[a]) * (nm_[a] - nc[a]);
  }
  const bool plus = dp <= dm;
#pragma unroll
  for (int a = 0; a < 3; ++a) nc[a] = plus ? np_[a] : nm_[a];
}

// ----------------------------------------------------------- collision
// Eqs. (13)-(14): S_nu from the harmonic-mean viscosity (phi clamped).
__device__ __forceinline__ float relaxation_rate(const StepConst &c,
                                                 float phi) {
  const float pc = fminf(1.f, fmaxf(-1.f, phi));
  const float inv_nu = (1.f + pc) / (2.f * c.nu_r) + (1.f - pc) / (2.f * c.nu_b);
  return 1.f / (3.f / inv_nu + 0.5f);
}

// Eq. (2) with one rate S for all non-conserved moments and rate 0 for rho
// and j, in velocity space:
//   f''_i = f_i - S (f_i - feq_i) + (1 - S/2) G_i + e_i . b,
//   b = S (j - rho0 u + F/2) / E2,
// feq of Eq. (A.4), G_i = w_i [3 (e_i - u) + 9 (e_i.u) e_i].F (A.5), u of
// Eq. (22); then recolouring, Eqs. (20)-(21):
//   f^r'_i = rho^r/rho f''_i + beta w_i rho^r rho^b/rho (e_i.n),
//   f^b'_i = f''_i - f^r'_i.
// fr/fb are overwritten with the post-recolouring populations; u is returned.
template <int Q>
__device__ __forceinline__ void collide_recolour(const StepConst &c, float *fr,
                                                 float *fb, float phi,
                                                 const float *F,
                                                 const float *nrm, float *u) {
  float rr, rb;
  sum_colours<Q>(fr, fb, rr, rb);
  const float rho = rr + rb;
  float j[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float ft = fr[i] + fb[i];
#pragma unroll
    for (int a = 0; a < 3; ++a) j[a] += (float)Lattice<Q>::e(i, a) * ft;
  }
  const float irho = 1.f / rho;
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5f * F[a]) * irho;
  const float S = relaxation_rate(c, phi);
  const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  float b[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    b[a] = S * (j[a] - c.rho0 * u[a] + 0.5f * F[a]) * (1.f / Lattice<Q>::E2);
  const float kf = 1.f - 0.5f * S;
  const float ratio = rr * irho;
  const float seg = c.beta * rr * rb * irho;
  const float uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float ex = (float)Lattice<Q>::e(i, 0), ey = (float)Lattice<Q>::e(i, 1),
                ez = (float)Lattice<Q>::e(i, 2);
    const float w = Lattice<Q>::w(i);
    const float eu = ex * u[0] + ey * u[1] + ez * u[2];
    const float eF = ex * F[0] + ey * F[1] + ez * F[2];
    const float feq = w * (rho + c.rho0 * (3.f * eu + 4.5f * eu * eu - 1.5f * uu));
    const float guo = w * (3.f * (eF - uF) + 9.f * eu * eF);
    const float ft = fr[i] + fb[i];
    const float out = ft - S * (ft - feq) + kf * guo +
                      (ex * b[0] + ey * b[1] + ez * b[2]);
    const float en = ex * nrm[0] + ey * nrm[1] + ez * nrm[2];
    const float r = ratio * out + seg * w * en;
    fr[i] = r;
    fb[i] = out - r;
  }
}

}  // namespace lbm
