// FP64 CPU oracle of the two-colour (colour-gradient) lattice-Boltzmann time
// step of Sedahmed & Coelho, "Wetting and pressure gradient performance in
// lattice Boltzmann color gradient model" (arXiv:2407.10914).
//
// TEST INFRASTRUCTURE ONLY. Only the test-suite, __graft_entry__.smoke() and
// the CPU-baseline leg of bench.py load this library. It shares no code,
// header or table with the CUDA path under paper_2407_10914_gb300/.
//
// It is written to be read against the paper: one function per equation,
// executed in the order of Eq. (1) and of the wetting summary at the end of
// Sec. II.B.3, over plain loops, in double precision. OpenMP only splits the
// node loops; nothing is blocked, fused or reordered.
//
// The step is templated on its scalar: double for the oracle itself, and a
// forward-mode dual number (value and derivatives with respect to the
// contact angle and the body acceleration g_x) for the tangent-linear
// reference of the adjoint (orc_tlm_*). Both run the same code.
//
// Layout (the public convention of this project, stated independently here):
//   node n = x + nx*(y + ny*z), x fastest;
//   populations f[(s*Q + i)*N + n], s = 0 red ("r"), s = 1 blue ("b");
//   vectors v[a*N + n], a = 0,1,2 for x,y,z.
//
// Readings of the paper that this file takes (each repeated at its use):
//   * collision: the single-rate (BGK) form of Eq. (2): rate S_nu (Eq. 13)
//     for every non-conserved moment, rate 0 for rho and j, equilibrium of
//     Eq. (A.4) and forcing of Eq. (A.5), written in velocity space;
//     or (collision = 1, D3Q19) the MRT form in moment space with the
//     rates of Eq. (4) read with 19 entries and Eqs. (15)-(16), m_10 and
//     m_12 of Eq. (A.4) read as -1/2 of m_9 and m_11; in both, Eq. (2) is
//     read with S^F outside the product with S;
//   * D2Q9 = the z-free subset of the D3Q19 set of Eq. (A.1), in the same
//     order, with weights 4/9, 1/9, 1/36;
//   * out-of-domain neighbours on a non-periodic axis: halfway bounce-back
//     for streaming, coordinate clamping (zero gradient) for every stencil;
//   * thresholds: |C| <= 1e-8 -> C = n_c = 0; Scheme-II leaves n_c unchanged
//     when sin(theta') < 1e-6; the Scheme-I secant stops early when the two
//     last residuals differ by less than 1e-12.
//
// parity unpinned: none of the functions here is without a pin in tests/.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

enum { CLS_SOLID = 0, CLS_SOLID_BND = 1, CLS_FLUID = 2, CLS_FLUID_BND = 3 };

const double EPS_C = 1e-8;        // |C| below this: no interface, n_c = 0
const double EPS_SIN = 1e-6;      // Scheme-II: n_c parallel to n_w
const double EPS_SECANT = 1e-12;  // Scheme-I: secant denominator
const double EPS_NW = 1e-12;      // |grad g| below this: no wall normal
const double PI = 3.14159265358979323846;

struct Lattice {
  int D = 0, Q = 0;
  int e[19][3];
  double w[19];
  int opp[19];
};

// Eq. (A.1) and Eq. (A.2): the D3Q19 velocities and weights in the order the
// paper prints them (the columns of the matrix in Eq. A.1).
const int E_D3Q19[19][3] = {
    {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
    {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, 1, 0}, {1, -1, 0},
    {-1, -1, 0}, {1, 0, 1},  {-1, 0, 1}, {1, 0, -1}, {-1, 0, -1},
    {0, 1, 1},  {0, -1, 1},  {0, 1, -1}, {0, -1, -1}};

// Eq. (3): the 19 moments of D3Q19 in the paper's order, (rho, e, eps, j_x,
// q_x, j_y, q_y, j_z, q_z, 3p_xx, 3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz, m_x,
// m_y, m_z), each written as the polynomial of the velocity e = (x, y, z)
// (s = |e|^2) whose values at the 19 velocities are one row of the
// transformation matrix of Eq. (A.3).
double moment_poly(int k, const int v[3]) {
  const double x = v[0], y = v[1], z = v[2], s = x * x + y * y + z * z;
  switch (k) {
    case 0: return 1.0;
    case 1: return 19.0 * s - 30.0;
    case 2: return (21.0 * s * s - 53.0 * s + 24.0) / 2.0;
    case 3: return x;
    case 4: return (5.0 * s - 9.0) * x;
    case 5: return y;
    case 6: return (5.0 * s - 9.0) * y;
    case 7: return z;
    case 8: return (5.0 * s - 9.0) * z;
    case 9: return 3.0 * x * x - s;
    case 10: return (3.0 * s - 5.0) * (3.0 * x * x - s);
    case 11: return y * y - z * z;
    case 12: return (3.0 * s - 5.0) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return x * (y * y - z * z);
    case 17: return y * (z * z - x * x);
    case 18: return z * (x * x - y * y);
  }
  return 0.0;
}

// M of Eq. (A.3), M[k][i] = moment k of velocity i (Eq. A.1 order), and its
// inverse by Gauss-Jordan elimination with partial pivoting.
struct MomentBasis {
  double M[19][19], Minv[19][19];
  MomentBasis() {
    double A[19][38];
    for (int k = 0; k < 19; ++k)
      for (int i = 0; i < 19; ++i) {
        M[k][i] = moment_poly(k, E_D3Q19[i]);
        A[k][i] = M[k][i];
        A[k][19 + i] = (k == i) ? 1.0 : 0.0;
      }
    for (int c = 0; c < 19; ++c) {
      int piv = c;
      for (int r = c + 1; r < 19; ++r)
        if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
      for (int j = 0; j < 38; ++j) std::swap(A[c][j], A[piv][j]);
      const double d = A[c][c];
      for (int j = 0; j < 38; ++j) A[c][j] /= d;
      for (int r = 0; r < 19; ++r) {
        if (r == c || A[r][c] == 0.0) continue;
        const double f = A[r][c];
        for (int j = 0; j < 38; ++j) A[r][j] -= f * A[c][j];
      }
    }
    for (int k = 0; k < 19; ++k)
      for (int i = 0; i < 19; ++i) Minv[k][i] = A[k][19 + i];
  }
};

const MomentBasis &moment_basis() {
  static const MomentBasis b;
  return b;
}

// Forward-mode derivatives for the tangent-linear run: a value and its
// derivatives along two directions (the contact angle in radians and the
// body acceleration g_x). Every operation applies the chain rule; a
// comparison looks at the value only, so a branch follows the value's path.
struct Dual {
  double v = 0.0;
  double d[2] = {0.0, 0.0};
  Dual() = default;
  Dual(double x) : v(x) {}  // a constant: zero derivatives
  Dual(double x, double d0, double d1) : v(x), d{d0, d1} {}
  Dual &operator+=(const Dual &b) { return *this = *this + b; }
  Dual &operator-=(const Dual &b) { return *this = *this - b; }
  Dual &operator*=(const Dual &b) { return *this = *this * b; }
  Dual &operator/=(const Dual &b) { return *this = *this / b; }
  friend Dual operator+(const Dual &a, const Dual &b) {
    return Dual(a.v + b.v, a.d[0] + b.d[0], a.d[1] + b.d[1]);
  }
  friend Dual operator-(const Dual &a, const Dual &b) {
    return Dual(a.v - b.v, a.d[0] - b.d[0], a.d[1] - b.d[1]);
  }
  friend Dual operator-(const Dual &a) { return Dual(-a.v, -a.d[0], -a.d[1]); }
  friend Dual operator*(const Dual &a, const Dual &b) {
    return Dual(a.v * b.v, a.d[0] * b.v + a.v * b.d[0],
                a.d[1] * b.v + a.v * b.d[1]);
  }
  friend Dual operator/(const Dual &a, const Dual &b) {
    const double q = a.v / b.v;
    return Dual(q, (a.d[0] - q * b.d[0]) / b.v, (a.d[1] - q * b.d[1]) / b.v);
  }
  friend bool operator<(const Dual &a, const Dual &b) { return a.v < b.v; }
  friend bool operator>(const Dual &a, const Dual &b) { return a.v > b.v; }
  friend bool operator<=(const Dual &a, const Dual &b) { return a.v <= b.v; }
  friend bool operator>=(const Dual &a, const Dual &b) { return a.v >= b.v; }
  friend bool operator==(const Dual &a, const Dual &b) { return a.v == b.v; }
  friend bool operator!=(const Dual &a, const Dual &b) { return a.v != b.v; }
};

// d/dx of sqrt, acos, sin, cos, |x|; the plain double versions alongside so
// that templated code calls one name for both.
inline Dual sqrt(const Dual &a) {
  const double r = std::sqrt(a.v);
  return Dual(r, a.d[0] / (2.0 * r), a.d[1] / (2.0 * r));
}
inline Dual acos(const Dual &a) {
  const double k = -1.0 / std::sqrt(1.0 - a.v * a.v);
  return Dual(std::acos(a.v), k * a.d[0], k * a.d[1]);
}
inline Dual sin(const Dual &a) {
  const double c = std::cos(a.v);
  return Dual(std::sin(a.v), c * a.d[0], c * a.d[1]);
}
inline Dual cos(const Dual &a) {
  const double s = -std::sin(a.v);
  return Dual(std::cos(a.v), s * a.d[0], s * a.d[1]);
}
inline Dual fabs(const Dual &a) { return a.v < 0.0 ? -a : a; }
inline double sqrt(double a) { return std::sqrt(a); }
inline double acos(double a) { return std::acos(a); }
inline double sin(double a) { return std::sin(a); }
inline double cos(double a) { return std::cos(a); }
inline double fabs(double a) { return std::fabs(a); }
inline double value_of(double x) { return x; }
inline Dual value_of(const Dual &x) { return Dual(x.v); }  // derivatives dropped
template <class R>
R clamp1(const R &x) {  // x limited to [-1, 1]
  return x < R(-1.0) ? R(-1.0) : (x > R(1.0) ? R(1.0) : x);
}

Lattice make_lattice(int q) {
  Lattice L;
  if (q == 19) {
    L.D = 3;
    L.Q = 19;
    for (int i = 0; i < 19; ++i) {
      for (int a = 0; a < 3; ++a) L.e[i][a] = E_D3Q19[i][a];
      L.w[i] = (i == 0) ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
  } else {
    // D2Q9 (not in the paper): the members of Eq. (A.1) with e_z = 0, kept
    // in the paper's order; standard D2Q9 weights.
    const int pick[9] = {0, 1, 2, 3, 4, 7, 8, 9, 10};
    L.D = 2;
    L.Q = 9;
    for (int k = 0; k < 9; ++k) {
      for (int a = 0; a < 3; ++a) L.e[k][a] = E_D3Q19[pick[k]][a];
      L.w[k] = (k == 0) ? 4.0 / 9.0 : (k <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
  }
  for (int i = 0; i < L.Q; ++i)
    for (int j = 0; j < L.Q; ++j)
      if (L.e[j][0] == -L.e[i][0] && L.e[j][1] == -L.e[i][1] &&
          L.e[j][2] == -L.e[i][2])
        L.opp[i] = j;
  return L;
}

}  // namespace

extern "C" {

// Parameters of one run. The oracle's own copy of the problem statement of
// Sec. II; the field meanings follow the paper's symbols.
typedef struct {
  double tau_r, tau_b;  // relaxation times; nu^s = (tau^s - 1/2)/3, Eq. (13)
  double gamma;         // interfacial tension, Eq. (5)
  double beta;          // segregation parameter, Eq. (20)
  double rho0;          // reference density of the equilibrium, Eq. (A.4)
  double theta_deg;     // contact angle, measured through fluid b
  int wetting;          // 0 none, 1 Scheme-I (Eqs. 28-31), 2 Scheme-II (32-33)
  int zou_he;           // 1: Zou-He pressure inlet/outlet, Appendix B
  int flow_axis;        // axis of the inlet (coordinate 0) and outlet planes
  double rho_in, rho_out;  // Zou-He densities (B.1, B.9)
  double zeta_r;        // injected red fraction zeta^r; zeta^b = 1 - zeta^r
  double g[3];          // body acceleration (Type-II), Eq. (36)
  int collision;        // 0 single-rate Eq. (2); 1 MRT (Eqs. 2, 4, 15-16)
} orc_params;

}  // extern "C"

namespace {

// R: the scalar of everything the step computes (double for the oracle,
// Dual for its tangent-linear run). The geometry stays double.
template <class R>
struct OracleT {
  Lattice L;
  int nx, ny, nz;
  long N;
  unsigned periodic;  // bit a set: axis a periodic
  orc_params p;
  std::vector<uint8_t> solid, cls;
  std::vector<double> gsm;   // smoothed indicator g^(3), Eq. (25)
  std::vector<double> nw;    // wall normal, Eq. (26), 3N
  std::vector<R> f, ftmp;  // stored post-recolouring populations, 2QN
  std::vector<R> rho_r, rho_b, phi;  // per node macros of the step
  std::vector<R> C, nc;  // colour gradient and unit normal, 3N
  std::vector<R> kappa, F;  // curvature and force (3N)
  std::vector<R> u;         // velocity of Eq. (22), 3N
  R theta;                  // contact angle (radians) of p.theta_deg
  double freeze_sin = 0.0;   // regularised Scheme-II linearisation (TLM)
  double c_min = 0.0;        // regularised normalisation linearisation
  R g[3];                   // body acceleration p.g
  long n_fluid = 0;

  int dim(int a) const { return a == 0 ? nx : (a == 1 ? ny : nz); }

  void coords(long n, int c[3]) const {
    c[0] = (int)(n % nx);
    c[1] = (int)((n / nx) % ny);
    c[2] = (int)(n / ((long)nx * ny));
  }
  long index(const int c[3]) const {
    return c[0] + (long)nx * (c[1] + (long)ny * c[2]);
  }

  // Node reached from n by the displacement d. Periodic axes wrap. On a
  // non-periodic axis a coordinate outside the box gives -1 (clamp = false)
  // or is clamped to the box (clamp = true).
  long neighbour(long n, const int d[3], bool clamp) const {
    int c[3];
    coords(n, c);
    for (int a = 0; a < 3; ++a) {
      int m = dim(a);
      int v = c[a] + d[a];
      if (v < 0 || v >= m) {
        if (periodic & (1u << a)) {
          v = ((v % m) + m) % m;
        } else if (clamp) {
          v = v < 0 ? 0 : m - 1;
        } else {
          return -1;
        }
      }
      c[a] = v;
    }
    return index(c);
  }

  bool is_fluid(long n) const { return n >= 0 && !solid[n]; }
  bool is_solid(long n) const { return n >= 0 && solid[n]; }
  R &fp(int s, int i, long n) { return f[((long)s * L.Q + i) * N + n]; }

  // Parameters; theta and g carry the derivative seeds of the tangent-linear
  // run (direction 0: theta, direction 1: g_x).
  void set_params(const orc_params &q, const R &th, const R gg[3]) {
    p = q;
    theta = th;
    for (int a = 0; a < 3; ++a) g[a] = gg[a];
  }

  // ---------------------------------------------------------------- geometry
  // Node classes from the solid image: a fluid node with a solid lattice
  // neighbour is a fluid-boundary node (where the wetting schemes act, Sec.
  // II.B); a solid node with a fluid lattice neighbour is a solid-boundary
  // node (where Eqs. 34-35 extrapolate).
  void classify() {
    cls.assign(N, CLS_SOLID);
    n_fluid = 0;
    for (long n = 0; n < N; ++n) {
      bool bnd = false;
      for (int i = 1; i < L.Q; ++i) {
        long m = neighbour(n, L.e[i], false);
        if (m < 0) continue;
        if (solid[n] ? !solid[m] : solid[m]) bnd = true;
      }
      if (solid[n]) {
        cls[n] = bnd ? CLS_SOLID_BND : CLS_SOLID;
      } else {
        cls[n] = bnd ? CLS_FLUID_BND : CLS_FLUID;
        ++n_fluid;
      }
    }
  }

  // Eq. (25): three passes of the 27-point smoothing kernel with weights
  // w_s(0) = 8/27, w_s(1) = 2/27, w_s(2) = 1/54, w_s(3) = 1/216 indexed by
  // i^2 + j^2 + k^2, applied to the fluid indicator g (1 fluid, 0 solid).
  // In 2-D the kernel is the 9-point analogue 4/9, 1/9, 1/36 (reading).
  // Off the box: wrap on periodic axes, clamp (replicate the edge) otherwise.
  void smooth_indicator() {
    const double ws3[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
    const double ws2[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
    std::vector<double> g(N), h(N);
    for (long n = 0; n < N; ++n) g[n] = solid[n] ? 0.0 : 1.0;
    const int kr = (L.D == 3) ? 1 : 0;
    for (int itr = 1; itr <= 3; ++itr) {
#pragma omp parallel for schedule(static)
      for (long n = 0; n < N; ++n) {
        double acc = 0.0;
        for (int k = -kr; k <= kr; ++k)
          for (int j = -1; j <= 1; ++j)
            for (int i = -1; i <= 1; ++i) {
              int d[3] = {i, j, k};
              int r2 = i * i + j * j + k * k;
              double wgt = (L.D == 3) ? ws3[r2] : ws2[r2];
              acc += wgt * g[neighbour(n, d, true)];
            }
        h[n] = acc;
      }
      g.swap(h);
    }
    gsm = g;
  }

  // Eq. (26): n_w = grad g^(3), the gradient taken with the isotropic
  // stencil of Eq. (6) and normalised, so that n_w points from the solid
  // into the fluid. Zero where the gradient vanishes.
  void wall_normal() {
    nw.assign(3 * N, 0.0);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
      double G[3] = {0, 0, 0};
      for (int i = 1; i < L.Q; ++i) {
        double gi = gsm[neighbour(n, L.e[i], true)];
        for (int a = 0; a < 3; ++a) G[a] += 3.0 * L.w[i] * L.e[i][a] * gi;
      }
      double m = std::sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
      if (m > EPS_NW)
        for (int a = 0; a < 3; ++a) nw[a * N + n] = G[a] / m;
    }
  }

  // ------------------------------------------------------------------ step
  // Eq. (1), propagation half: pull f^s_i(x) from x - e_i. Halfway
  // bounce-back (Sec. II.B, first sentence) when x - e_i is solid or off a
  // non-periodic axis: the population that left x along -e_i returns as i.
  void stream() {
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
      if (solid[n]) continue;
      for (int i = 0; i < L.Q; ++i) {
        int d[3] = {-L.e[i][0], -L.e[i][1], -L.e[i][2]};
        long src = neighbour(n, d, false);
        for (int s = 0; s < 2; ++s) {
          R v = is_fluid(src) ? f[((long)s * L.Q + i) * N + src]
                              : f[((long)s * L.Q + L.opp[i]) * N + n];
          ftmp[((long)s * L.Q + i) * N + n] = v;
        }
      }
    }
  }

  // Eqs. (8), (9), (7): colour densities, total density and phase field.
  void macros() {
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
      if (solid[n]) continue;
      R r = 0.0, b = 0.0;
      for (int i = 0; i < L.Q; ++i) {
        r += ftmp[(0L * L.Q + i) * N + n];
        b += ftmp[(1L * L.Q + i) * N + n];
      }
      rho_r[n] = r;
      rho_b[n] = b;
      phi[n] = (r - b) / (r + b);
    }
  }

  // Appendix B, generalised from the paper's z-axis form to a flow axis a:
  // the unknown populations are those with e_i . a = +1 at the inlet plane
  // (coordinate 0) and e_i . a = -1 at the outlet plane (last coordinate);
  // 6 w_i equals the 1/3 and 1/6 of Eqs. (B.4)-(B.8) and (B.14)-(B.18).
  //   inlet, per colour s (B.1-B.8):
  //     j^s = rho_in zeta^s - [sum_{e.a=0} f^s + 2 sum_{e.a=-1} f^s]
  //     f^s_i = f^s_opp(i) + 6 w_i j^s - sum_t (e_i.t) N^s_t
  //   outlet, total j with the weights chi^s of Eqs. (B.12)-(B.13):
  //     j^t = -rho_out + [sum_{e.a=0} f^t + 2 sum_{e.a=+1} f^t]   (B.9)
  //     f^s_i = f^s_opp(i) - 6 w_i j^t chi^s - sum_t (e_i.t) N^s_t
  //   N^s_t = 1/2 sum_{e.a=0} (e_j.t) f^s_j  (B.2-B.3, B.10-B.11).
  // The outlet phase field is phi(x_out - a), Eq. (39), from the streamed
  // populations of that node (the node's own value if that node is solid).
  // Afterwards the inlet phase field is zeta^r - zeta^b (Sec. II.D.1).
  void zou_he() {
    const int a = p.flow_axis;
    const int na = dim(a);
    const double zeta[2] = {p.zeta_r, 1.0 - p.zeta_r};
    std::vector<long> inlet, outlet;
    for (long n = 0; n < N; ++n) {
      if (solid[n]) continue;
      int c[3];
      coords(n, c);
      if (c[a] == 0) inlet.push_back(n);
      if (c[a] == na - 1) outlet.push_back(n);
    }
    auto F_ = [&](int s, int i, long n) -> R & {
      return ftmp[((long)s * L.Q + i) * N + n];
    };
    auto transverse = [&](int s, long n, R Nt[3]) {
      for (int t = 0; t < 3; ++t) Nt[t] = 0.0;
      for (int j = 0; j < L.Q; ++j) {
        if (L.e[j][a] != 0) continue;
        for (int t = 0; t < 3; ++t)
          if (t != a) Nt[t] += 0.5 * L.e[j][t] * F_(s, j, n);
      }
    };
    // phase field of the outlet nodes from the plane behind them, Eq. (39)
    std::vector<R> phi_out(outlet.size());
    for (size_t k = 0; k < outlet.size(); ++k) {
      long n = outlet[k];
      int d[3] = {0, 0, 0};
      d[a] = -1;
      long m = neighbour(n, d, false);
      phi_out[k] = is_fluid(m) ? phi[m] : phi[n];
    }
    for (long n : inlet) {
      for (int s = 0; s < 2; ++s) {
        R known = 0.0;
        for (int i = 0; i < L.Q; ++i) {
          if (L.e[i][a] == 0) known += F_(s, i, n);
          if (L.e[i][a] == -1) known += 2.0 * F_(s, i, n);
        }
        R j = p.rho_in * zeta[s] - known;
        R Nt[3];
        transverse(s, n, Nt);
        for (int i = 0; i < L.Q; ++i) {
          if (L.e[i][a] != 1) continue;
          R corr = 0.0;
          for (int t = 0; t < 3; ++t)
            if (t != a) corr += L.e[i][t] * Nt[t];
          F_(s, i, n) = F_(s, L.opp[i], n) + 6.0 * L.w[i] * j - corr;
        }
      }
    }
    for (size_t k = 0; k < outlet.size(); ++k) {
      long n = outlet[k];
      R known = 0.0;
      for (int i = 0; i < L.Q; ++i) {
        R ft = F_(0, i, n) + F_(1, i, n);
        if (L.e[i][a] == 0) known += ft;
        if (L.e[i][a] == 1) known += 2.0 * ft;
      }
      R jt = -p.rho_out + known;
      R chi[2] = {0.5 * (1.0 + phi_out[k]), 0.5 * (1.0 - phi_out[k])};
      for (int s = 0; s < 2; ++s) {
        R Nt[3];
        transverse(s, n, Nt);
        for (int i = 0; i < L.Q; ++i) {
          if (L.e[i][a] != -1) continue;
          R corr = 0.0;
          for (int t = 0; t < 3; ++t)
            if (t != a) corr += L.e[i][t] * Nt[t];
          F_(s, i, n) = F_(s, L.opp[i], n) - 6.0 * L.w[i] * jt * chi[s] - corr;
        }
      }
    }
    // densities of the rebuilt nodes, then the phase-field overrides
    auto resum = [&](long n) {
      R r = 0.0, b = 0.0;
      for (int i = 0; i < L.Q; ++i) {
        r += F_(0, i, n);
        b += F_(1, i, n);
      }
      rho_r[n] = r;
      rho_b[n] = b;
    };
    for (long n : inlet) {
      resum(n);
      phi[n] = zeta[0] - zeta[1];
    }
    for (size_t k = 0; k < outlet.size(); ++k) {
      resum(outlet[k]);
      phi[outlet[k]] = phi_out[k];
    }
  }

  // Eq. (34): phase field of a solid-boundary node, the w-weighted mean of
  // phi over its fluid lattice neighbours.
  void extrapolate_phi() {
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
      if (cls[n] != CLS_SOLID_BND) continue;
      R num = 0.0;
        double den = 0.0;
      for (int i = 1; i < L.Q; ++i) {
        long m = neighbour(n, L.e[i], false);
        if (!is_fluid(m)) continue;
        num += L.w[i] * phi[m];
        den += L.w[i];
      }
      phi[n] = num / den;
    }
  }

  // Eq. (6) with c = dt = 1, and Eq. (11)/(27): C = 3 sum_i w_i e_i
  // phi(x + e_i), n_c = C/|C|. Where |C| <= EPS_C the node holds no
  // interface: C and n_c are set to zero (reading of the threshold).
  void colour_gradient() {
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
      if (solid[n]) continue;
      R G[3] = {0.0, 0.0, 0.0};
      for (int i = 1; i < L.Q; ++i) {
        R ph = phi[neighbour(n, L.e[i], true)];
        for (int a = 0; a < 3; ++a) G[a] += 3.0 * L.w[i] * L.e[i][a] * ph;
      }
      R m = sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
      for (int a = 0; a < 3; ++a) {
        C[a * N + n] = (m > EPS_C) ? G[a] : R(0.0);
        nc[a * N + n] = (m > EPS_C) ? G[a] / m : R(0.0);
        // regularised linearisation (tangent-linear runs only): below c_min
        // the direction of n_c is held constant
        if (m > EPS_C && m < c_min) nc[a * N + n] = value_of(G[a] / m);
      }
    }
  }

  // Eq. (28): f(v) = v . n_w - |v| cos(theta)
  template <class T>
  static T secant_residual(const T v[3], const double w[3], const T &cth) {
    T vn = v[0] * w[0] + v[1] * w[1] + v[2] * w[2];
    T vv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    return vn - vv * cth;
  }

 public:
  // Scheme-I (Leclaire et al.), Eqs. (28)-(31): secant iterates
  // v0 = n_c, v1 = n_c - lambda (n_c + n_w) with lambda = 1/2, then
  // v_n = (v_{n-2} f(v_{n-1}) - v_{n-1} f(v_{n-2})) / (f(v_{n-1}) - f(v_{n-2}))
  // for n = 2, 3, 4; v4 normalised replaces n_c. If the denominator is below
  // EPS_SECANT the iteration stops and keeps v_{n-1}; if the final vector
  // has zero length n_c is left unchanged (the degenerate cases of Sec.
  // II.B.1, last paragraph).
  template <class T>
  static void scheme1(const T n_c[3], const double n_w[3], const T &theta,
                      T out[3]) {
    const double lambda = 0.5;
    const T cth = cos(theta);
    T vm2[3], vm1[3];
    for (int a = 0; a < 3; ++a) {
      vm2[a] = n_c[a];
      vm1[a] = n_c[a] - lambda * (n_c[a] + n_w[a]);
    }
    for (int it = 2; it <= 4; ++it) {
      T f1 = secant_residual(vm1, n_w, cth);
      T f2 = secant_residual(vm2, n_w, cth);
      T den = f1 - f2;
      if (fabs(den) < EPS_SECANT) break;
      T vn[3];
      for (int a = 0; a < 3; ++a) vn[a] = (vm2[a] * f1 - vm1[a] * f2) / den;
      for (int a = 0; a < 3; ++a) {
        vm2[a] = vm1[a];
        vm1[a] = vn[a];
      }
    }
    T m = sqrt(vm1[0] * vm1[0] + vm1[1] * vm1[1] + vm1[2] * vm1[2]);
    for (int a = 0; a < 3; ++a) out[a] = (m > 0.0) ? vm1[a] / m : n_c[a];
  }

  // Scheme-II (Akai et al.), Eqs. (32)-(33): theta' = arccos(n_w . n_c);
  // n_+- = (cos(+-theta) - sin(+-theta) cos(theta')/sin(theta')) n_w
  //        + sin(+-theta)/sin(theta') n_c;
  // n_c is replaced by whichever of n_+ and n_- lies nearer to n_c (n_+ on a
  // tie). Left unchanged when sin(theta') < EPS_SIN.
  template <class T>
  static void scheme2(const T n_c[3], const double n_w[3], const T &theta,
                      T out[3], double freeze_sin = 0.0) {
    T c = n_c[0] * n_w[0] + n_c[1] * n_w[1] + n_c[2] * n_w[2];
    c = clamp1(c);
    T thp = acos(c);
    T sp = sin(thp);
    if (sp < EPS_SIN) {
      for (int a = 0; a < 3; ++a) out[a] = n_c[a];
      return;
    }
    T cp = cos(thp);
    T np[3], nm[3];
    T dp = 0.0, dm = 0.0;
    for (int a = 0; a < 3; ++a) {
      T sgn_p = sin(theta), sgn_m = sin(-theta);
      np[a] = (cos(theta) - sgn_p * cp / sp) * n_w[a] + sgn_p / sp * n_c[a];
      nm[a] = (cos(-theta) - sgn_m * cp / sp) * n_w[a] + sgn_m / sp * n_c[a];
      dp += (np[a] - n_c[a]) * (np[a] - n_c[a]);
      dm += (nm[a] - n_c[a]) * (nm[a] - n_c[a]);
    }
    for (int a = 0; a < 3; ++a) out[a] = (dp <= dm) ? np[a] : nm[a];
    // Regularised linearisation (tangent-linear runs only): with n_c almost
    // along n_w the direction t = (n_c - cos(theta') n_w) / sin(theta') of
    // the result around n_w is undefined at sin(theta') = 0 and its
    // derivative grows as 1/sin(theta'). Below freeze_sin that direction is
    // held constant: out = cos(theta) n_w +- sin(theta) t with t's value.
    if (freeze_sin > 0.0 && sp < freeze_sin) {
      const T st = (dp <= dm) ? sin(theta) : sin(-theta);
      for (int a = 0; a < 3; ++a) {
        const T t = (n_c[a] - cp * n_w[a]) / sp;
        out[a] = cos(theta) * n_w[a] + st * value_of(t);
      }
    }
  }

 private:
  // Sec. II.B.3, step 3: at fluid-boundary nodes, turn n_c to the contact
  // angle with Scheme-I or Scheme-II; the magnitude |C| is kept, so the
  // colour gradient becomes |C| n_c (Sec. II.B.1).
  void wetting() {
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
      if (cls[n] != CLS_FLUID_BND) continue;
      R ncv[3], out[3];
      double nwv[3];
      R m2 = 0.0;
      double w2 = 0.0;
      for (int a = 0; a < 3; ++a) {
        ncv[a] = nc[a * N + n];
        nwv[a] = nw[a * N + n];
        m2 += ncv[a] * ncv[a];
        w2 += nwv[a] * nwv[a];
      }
      if (m2 == 0.0 || w2 == 0.0) continue;  // no interface or no wall normal
      if (p.wetting == 1)
        scheme1(ncv, nwv, theta, out);
      else
        scheme2(ncv, nwv, theta, out, freeze_sin);
      R mag = 0.0;
      for (int a = 0; a < 3; ++a) mag += C[a * N + n] * C[a * N + n];
      mag = sqrt(mag);
      for (int a = 0; a < 3; ++a) {
        nc[a * N + n] = out[a];
        C[a * N + n] = mag * out[a];
      }
    }
  }

  // Eq. (35): n_c of a solid-boundary node, the w-weighted mean of the
  // (post-wetting) n_c of its fluid lattice neighbours, not renormalised.
  void extrapolate_nc() {
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
      if (cls[n] != CLS_SOLID_BND) continue;
      R num[3] = {0.0, 0.0, 0.0};
      double den = 0.0;
      for (int i = 1; i < L.Q; ++i) {
        long m = neighbour(n, L.e[i], false);
        if (!is_fluid(m)) continue;
        for (int a = 0; a < 3; ++a) num[a] += L.w[i] * nc[a * N + m];
        den += L.w[i];
      }
      for (int a = 0; a < 3; ++a) nc[a * N + n] = num[a] / den;
    }
  }

  // Eq. (12): curvature from the derivatives d_b n_a, each taken with the
  // stencil of Eq. (6) applied to the component n_a (reading). Eq. (5):
  // F = 1/2 gamma kappa C, plus the Type-II body force rho g, Eq. (36).
  void curvature_force() {
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
      if (solid[n]) continue;
      R dn[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};  // d_b n_a
      for (int i = 1; i < L.Q; ++i) {
        long m = neighbour(n, L.e[i], true);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            dn[a][b] += 3.0 * L.w[i] * L.e[i][b] * nc[a * N + m];
      }
      R nx_ = nc[0 * N + n], ny_ = nc[1 * N + n], nz_ = nc[2 * N + n];
      R k = (nx_ * nx_ - 1.0) * dn[0][0] + (ny_ * ny_ - 1.0) * dn[1][1] +
                 (nz_ * nz_ - 1.0) * dn[2][2] +
                 (dn[0][1] + dn[1][0]) * nx_ * ny_ +
                 (dn[0][2] + dn[2][0]) * nx_ * nz_ +
                 (dn[2][1] + dn[1][2]) * nz_ * ny_;
      kappa[n] = k;
      R rho = rho_r[n] + rho_b[n];
      for (int a = 0; a < 3; ++a)
        F[a * N + n] = 0.5 * p.gamma * k * C[a * N + n] + rho * g[a];
    }
  }

 public:
  // Eqs. (34) and (35) on the current phi and n_c (for tests).
  void extrapolations_only() {
    extrapolate_phi();
    extrapolate_nc();
  }
  // Eq. (6)/(11) on the current phi, and Eq. (12) on the current n_c
  // (for tests; C, n_c and kappa are overwritten in that order).
  void gradient_only() { colour_gradient(); }
  void curvature_only() { curvature_force(); }
  // Collision and recolouring, Eqs. (2) and (20)-(21), on the current
  // streamed populations, colour densities, phase field, n_c and F (for
  // tests).
  void collide_recolour_only() { collide_recolour(); }

  // Single-node collision: Eq. (2) with one rate S for every non-conserved
  // moment and rate 0 for the conserved ones (rho, j), i.e. the relaxation
  // matrix of Eq. (4) with S_e = S_eps = S_q = S_nu = S_pi = S_m = S.
  // Eq. (2) is read as f'' = f - M^-1 S (m - m_eq) + M^-1 S^F (the print
  // multiplies S^F by S). Written in velocity space this is
  //   f''_i = f_i - S (f_i - feq_i) + (1 - S/2) G_i
  //           + S sum_a e_ia (j_a - rho0 u_a + F_a/2) / E2
  //   feq_i = w_i [rho + rho0 (3 e_i.u + 9/2 (e_i.u)^2 - 3/2 u.u)]   (A.4)
  //   G_i   = w_i [3 (e_i - u) + 9 (e_i.u) e_i] . F                  (A.5)
  // where E2 = sum_i e_ix^2 and the last term gives back the part of the
  // first two that would relax the conserved momentum: the post-collision
  // momentum is exactly j + F and the mass is unchanged. u is Eq. (22):
  // u = (sum_i e_i f_i + F/2) / rho.
  template <class T>
  static void collide(const Lattice &L, const T *ft, const T Fv[3], const T &S,
                      double rho0, T *out, T u_out[3]) {
    T rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L.Q; ++i) {
      rho += ft[i];
      for (int a = 0; a < 3; ++a) j[a] += L.e[i][a] * ft[i];
    }
    double E2 = 0.0;
    for (int i = 0; i < L.Q; ++i) E2 += L.e[i][0] * L.e[i][0];
    T u[3], back[3];
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * Fv[a]) / rho;
    for (int a = 0; a < 3; ++a)
      back[a] = S * (j[a] - rho0 * u[a] + 0.5 * Fv[a]) / E2;
    T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < L.Q; ++i) {
      T eu = L.e[i][0] * u[0] + L.e[i][1] * u[1] + L.e[i][2] * u[2];
      T feq = L.w[i] * (rho + rho0 * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu));
      T guo = 0.0, cons = 0.0;
      for (int a = 0; a < 3; ++a) {
        guo += (3.0 * (L.e[i][a] - u[a]) + 9.0 * eu * L.e[i][a]) * Fv[a];
        cons += L.e[i][a] * back[a];
      }
      guo *= L.w[i];
      out[i] = ft[i] - S * (ft[i] - feq) + (1.0 - 0.5 * S) * guo + cons;
    }
    if (u_out)
      for (int a = 0; a < 3; ++a) u_out[a] = u[a];
  }

  // Single-node MRT collision of D3Q19, Eq. (2) in moment space:
  //   m = M f,  f'' = f - M^-1 S (m - m^eq) + M^-1 S^F,
  // read with S^F outside the product with S (as in the single-rate form
  // above). S is the diagonal of Eq. (4) taken with 19 entries (the print's
  // 20 carry a spurious 0 before the first S_nu):
  //   (0, S_e, S_eps, 0, S_q, 0, S_q, 0, S_q, S_nu, S_pi, S_nu, S_pi,
  //    S_nu, S_nu, S_nu, S_m, S_m, S_m)
  // with S_e = S_eps = S_pi = S_nu (Eq. 15); S_q and S_m are passed in (the
  // step uses Eq. 16). m^eq is Eq. (A.4), m_10 read as -(1/2) m_9 and m_12
  // as -(1/2) m_11 (the print's -3/2 p_xx drops the 1/3 of p_xx = m_9 / 3);
  // S^F is Eq. (A.5), each entry with the (1 - S_k/2) of its own rate.
  // u is Eq. (22): u = (j + F/2) / rho with j = (m_3, m_5, m_7).
  template <class T>
  static void collide_mrt(const T *ft, const T Fv[3], const T &Snu,
                          const T &Sq, const T &Sm, double rho0, T *out,
                          T u_out[3]) {
    const MomentBasis &B = moment_basis();
    T m[19];
    for (int k = 0; k < 19; ++k) {
      m[k] = 0.0;
      for (int i = 0; i < 19; ++i) m[k] += B.M[k][i] * ft[i];
    }
    const T rho = m[0];
    T u[3];
    u[0] = (m[3] + 0.5 * Fv[0]) / rho;
    u[1] = (m[5] + 0.5 * Fv[1]) / rho;
    u[2] = (m[7] + 0.5 * Fv[2]) / rho;
    const T ux = u[0], uy = u[1], uz = u[2];
    const T Fx = Fv[0], Fy = Fv[1], Fz = Fv[2];
    const T u2 = ux * ux + uy * uy + uz * uz;
    const T uF = ux * Fx + uy * Fy + uz * Fz;
    const T Se = Snu, Seps = Snu, Spi = Snu;  // Eq. (15)
    const T zero = 0.0;
    const T S[19] = {zero, Se,  Seps, zero, Sq,  zero, Sq,  zero, Sq, Snu,
                     Spi,  Snu, Spi,  Snu,  Snu, Snu,  Sm,  Sm,   Sm};
    const T pxx3 = rho0 * (2.0 * ux * ux - uy * uy - uz * uz);
    const T pww = rho0 * (uy * uy - uz * uz);
    const T meq[19] = {rho,
                       -11.0 * rho + 19.0 * rho0 * u2,
                       3.0 * rho - 5.5 * rho0 * u2,
                       rho0 * ux,
                       -(2.0 / 3.0) * rho0 * ux,
                       rho0 * uy,
                       -(2.0 / 3.0) * rho0 * uy,
                       rho0 * uz,
                       -(2.0 / 3.0) * rho0 * uz,
                       pxx3,
                       -0.5 * pxx3,
                       pww,
                       -0.5 * pww,
                       rho0 * ux * uy,
                       rho0 * uy * uz,
                       rho0 * ux * uz,
                       zero,
                       zero,
                       zero};
    const T h[19] = {zero,
                     38.0 * uF,
                     -11.0 * uF,
                     Fx,
                     -(2.0 / 3.0) * Fx,
                     Fy,
                     -(2.0 / 3.0) * Fy,
                     Fz,
                     -(2.0 / 3.0) * Fz,
                     2.0 * (2.0 * ux * Fx - uy * Fy - uz * Fz),
                     -2.0 * ux * Fx + uy * Fy + uz * Fz,
                     2.0 * (uy * Fy - uz * Fz),
                     -uy * Fy + uz * Fz,
                     uy * Fx + ux * Fy,
                     uz * Fy + uy * Fz,
                     ux * Fz + uz * Fx,
                     zero,
                     zero,
                     zero};
    T dm[19];
    for (int k = 0; k < 19; ++k)
      dm[k] = -S[k] * (m[k] - meq[k]) + (1.0 - 0.5 * S[k]) * h[k];
    for (int i = 0; i < 19; ++i) {
      T acc = ft[i];
      for (int k = 0; k < 19; ++k) acc += B.Minv[i][k] * dm[k];
      out[i] = acc;
    }
    if (u_out)
      for (int a = 0; a < 3; ++a) u_out[a] = u[a];
  }

  // Eq. (16): the rate of the q and m moments from S_nu.
  template <class T>
  static T mrt_rate(const T &Snu) {
    return 8.0 * (2.0 - Snu) / (8.0 - Snu);
  }

 private:
  // Eqs. (13)-(14): harmonic-mean viscosity, S_nu = 1 / (3 nu + 1/2);
  // phi is clamped to [-1, 1] here only.
  R relaxation_rate(const R &ph) const {
    double nur = (p.tau_r - 0.5) / 3.0, nub = (p.tau_b - 0.5) / 3.0;
    R pc = clamp1(ph);
    R inv_nu = (1.0 + pc) / (2.0 * nur) + (1.0 - pc) / (2.0 * nub);
    R nu = 1.0 / inv_nu;
    return 1.0 / (3.0 * nu + 0.5);
  }

  // Collision (Eq. 2: single-rate reading, or MRT with the rates of Eqs.
  // 15-16 when collision = 1) followed by recolouring, Eqs. (20)-(21):
  //   f^r'_i = rho^r/rho f^t''_i + beta w_i rho^r rho^b / rho (e_i . n)
  //   f^b'_i = f^t''_i - f^r'_i
  // with n the post-wetting interface normal n_c (the i = 0 term vanishes
  // because e_0 = 0).
  void collide_recolour() {
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
      if (solid[n]) continue;
      R ft[19], fpp[19], Fv[3], uu[3];
      for (int i = 0; i < L.Q; ++i)
        ft[i] = ftmp[(0L * L.Q + i) * N + n] + ftmp[(1L * L.Q + i) * N + n];
      for (int a = 0; a < 3; ++a) Fv[a] = F[a * N + n];
      R S = relaxation_rate(phi[n]);
      if (p.collision == 1) {
        const R Sq = mrt_rate(S);
        collide_mrt(ft, Fv, S, Sq, Sq, p.rho0, fpp, uu);
      } else {
        collide(L, ft, Fv, S, p.rho0, fpp, uu);
      }
      for (int a = 0; a < 3; ++a) u[a * N + n] = uu[a];
      R r = rho_r[n], b = rho_b[n], rho = r + b;
      R nv[3] = {nc[0 * N + n], nc[1 * N + n], nc[2 * N + n]};
      for (int i = 0; i < L.Q; ++i) {
        R en = L.e[i][0] * nv[0] + L.e[i][1] * nv[1] + L.e[i][2] * nv[2];
        R fr = r / rho * fpp[i] + p.beta * L.w[i] * r * b / rho * en;
        f[(0L * L.Q + i) * N + n] = fr;
        f[(1L * L.Q + i) * N + n] = fpp[i] - fr;
      }
    }
  }

 public:
  void init(int q, int nx_, int ny_, int nz_, const uint8_t *mask,
            unsigned per) {
    L = make_lattice(q);
    nx = nx_;
    ny = ny_;
    nz = nz_;
    N = (long)nx * ny * nz;
    periodic = per;
    solid.assign(mask, mask + N);
    classify();
    smooth_indicator();
    wall_normal();
    f.assign(2L * L.Q * N, 0.0);
    ftmp.assign(2L * L.Q * N, 0.0);
    rho_r.assign(N, 0.0);
    rho_b.assign(N, 0.0);
    phi.assign(N, 0.0);
    C.assign(3 * N, 0.0);
    nc.assign(3 * N, 0.0);
    kappa.assign(N, 0.0);
    F.assign(3 * N, 0.0);
    u.assign(3 * N, 0.0);
    std::memset(&p, 0, sizeof(p));
    theta = 0.0;
    for (int a = 0; a < 3; ++a) g[a] = 0.0;
  }

  // Initial state: f^s_i = w_i rho^s with rho^r = rho0 (1 + phi0)/2 and
  // rho^b = rho0 (1 - phi0)/2 (a fluid at rest).
  void init_state(const double *phi0) {
    std::fill(f.begin(), f.end(), R(0.0));
    for (long n = 0; n < N; ++n) {
      if (solid[n]) continue;
      R r = p.rho0 * 0.5 * (1.0 + phi0[n]);
      R b = p.rho0 * 0.5 * (1.0 - phi0[n]);
      for (int i = 0; i < L.Q; ++i) {
        f[(0L * L.Q + i) * N + n] = L.w[i] * r;
        f[(1L * L.Q + i) * N + n] = L.w[i] * b;
      }
      rho_r[n] = r;
      rho_b[n] = b;
      phi[n] = (r - b) / (r + b);
    }
    std::fill(u.begin(), u.end(), R(0.0));
  }

  // One time step in the order of Eq. (1) and Sec. II.B.3: stream (with
  // bounce-back), macros, Zou-He (which rebuilds the macros of its two
  // planes), Eq. 34, Eqs. 6/27, wetting, Eq. 35, Eqs. 12 and 5, collision,
  // recolouring.
  void stream_part() {
    stream();
    macros();
    if (p.zou_he) zou_he();
  }

  void step() {
    stream_part();
    extrapolate_phi();
    colour_gradient();
    if (p.wetting) wetting();
    extrapolate_nc();
    curvature_force();
    collide_recolour();
  }
};

using Oracle = OracleT<double>;

}  // namespace

extern "C" {

void *orc_create(int lattice, int nx, int ny, int nz, const uint8_t *solid,
                 unsigned periodic_mask) {
  if (lattice != 9 && lattice != 19) return nullptr;
  if (lattice == 9 && nz != 1) return nullptr;
  Oracle *o = new Oracle();
  o->init(lattice, nx, ny, nz, solid, periodic_mask);
  return o;
}

void orc_destroy(void *h) { delete static_cast<Oracle *>(h); }

// Returns 0, or -1 (parameters unchanged) for a collision other than 0/1 or
// MRT (collision = 1) on D2Q9: Appendix A defines it for D3Q19 only.
int orc_set_params(void *h, const orc_params *p) {
  Oracle *o = static_cast<Oracle *>(h);
  if (p->collision != 0 && p->collision != 1) return -1;
  if (p->collision == 1 && o->L.Q != 19) return -1;
  o->set_params(*p, p->theta_deg * PI / 180.0, p->g);
  return 0;
}

void orc_init_state(void *h, const double *phi0) {
  static_cast<Oracle *>(h)->init_state(phi0);
}

void orc_set_pops(void *h, const double *src) {
  Oracle *o = static_cast<Oracle *>(h);
  std::memcpy(o->f.data(), src, sizeof(double) * o->f.size());
}

void orc_get_pops(void *h, double *dst) {
  Oracle *o = static_cast<Oracle *>(h);
  std::memcpy(dst, o->f.data(), sizeof(double) * o->f.size());
}

void orc_step(void *h, int nsteps) {
  Oracle *o = static_cast<Oracle *>(h);
  for (int s = 0; s < nsteps; ++s) o->step();
}

// Sec. II.D.1, Eqs. (37)-(38): the injected fluid is replaced by colour
// `colour` (0 = r, 1 = b) at every fluid node of the inlet plane (coordinate
// 0 of the flow axis): f^s_i += f^sbar_i, f^sbar_i = 0 for every i. The
// stored populations change; the caller sets the new zeta^s of Eq. (B.1).
// Returns the number of nodes changed, or -1 for a colour other than 0/1.
long orc_swap_inlet(void *h, int colour) {
  Oracle *o = static_cast<Oracle *>(h);
  if (colour != 0 && colour != 1) return -1;
  const int a = o->p.flow_axis;
  const long N = o->N;
  const int Q = o->L.Q;
  long changed = 0;
  for (long n = 0; n < N; ++n) {
    if (o->solid[n]) continue;
    int c[3];
    o->coords(n, c);
    if (c[a] != 0) continue;
    for (int i = 0; i < Q; ++i) {
      double &fs = o->f[((long)colour * Q + i) * N + n];
      double &fo = o->f[((long)(1 - colour) * Q + i) * N + n];
      fs = fs + fo;  // Eq. (37)
      fo = 0.0;      // Eq. (38)
    }
    ++changed;
  }
  return changed;
}

// The first half of a step only: streaming with bounce-back, the macros
// and, when enabled, Zou-He; the streamed (and rebuilt) populations go to
// dst (2QN). The stored state is not changed.
void orc_stream_only(void *h, double *dst) {
  Oracle *o = static_cast<Oracle *>(h);
  o->stream_part();
  std::memcpy(dst, o->ftmp.data(), sizeof(double) * o->ftmp.size());
}

// Test hook: the extrapolations of Eqs. (34)-(35) alone on a prescribed
// field. phi_in (N) and nc_in (3N) give the fluid nodes' phase field and
// n_c (other entries are ignored); phi_out and nc_out receive the fields
// after Eq. (34) and Eq. (35) set the solid-boundary nodes. The stored
// state is not changed.
void orc_extrapolate(void *h, const double *phi_in, const double *nc_in,
                     double *phi_out, double *nc_out) {
  Oracle *o = static_cast<Oracle *>(h);
  const long N = o->N;
  std::memcpy(o->phi.data(), phi_in, sizeof(double) * N);
  std::memcpy(o->nc.data(), nc_in, sizeof(double) * 3 * N);
  o->extrapolations_only();
  std::memcpy(phi_out, o->phi.data(), sizeof(double) * N);
  std::memcpy(nc_out, o->nc.data(), sizeof(double) * 3 * N);
}

// Test hook: the stencils alone on prescribed fields. phi_in (N): Eq. (6)
// and Eq. (11) give C and n_c (3N each, into C_out, nc_out); nc_in (3N):
// Eq. (12) gives kappa (N, into kappa_out). The stored state is not
// changed; the colour densities are taken as they are (they enter F only).
void orc_stencils(void *h, const double *phi_in, const double *nc_in,
                  double *C_out, double *nc_out, double *kappa_out) {
  Oracle *o = static_cast<Oracle *>(h);
  const long N = o->N;
  std::memcpy(o->phi.data(), phi_in, sizeof(double) * N);
  o->gradient_only();
  std::memcpy(C_out, o->C.data(), sizeof(double) * 3 * N);
  std::memcpy(nc_out, o->nc.data(), sizeof(double) * 3 * N);
  std::memcpy(o->nc.data(), nc_in, sizeof(double) * 3 * N);
  o->curvature_only();
  std::memcpy(kappa_out, o->kappa.data(), sizeof(double) * N);
}

// Test hook: collision and recolouring alone on a prescribed node state.
// ft_in (2QN) holds the streamed populations f^r, f^b (only their sum
// f^t enters the collision); rho_r, rho_b (N) the colour densities; phi
// (N) the phase field (it sets the relaxation rate, Eq. 14); nc_in and
// F_in (3N) the interface normal and the force density. f_out (2QN)
// receives the post-recolouring populations f^r', f^b' of Eqs. (20)-(21).
// The stored state is not changed apart from these inputs.
void orc_collide_recolour(void *h, const double *ft_in, const double *rho_r,
                          const double *rho_b, const double *phi_in,
                          const double *nc_in, const double *F_in,
                          double *f_out) {
  Oracle *o = static_cast<Oracle *>(h);
  const long N = o->N;
  const long QN = (long)o->L.Q * N;
  std::vector<double> keep(o->f);
  std::memcpy(o->ftmp.data(), ft_in, sizeof(double) * 2 * QN);
  std::memcpy(o->rho_r.data(), rho_r, sizeof(double) * N);
  std::memcpy(o->rho_b.data(), rho_b, sizeof(double) * N);
  std::memcpy(o->phi.data(), phi_in, sizeof(double) * N);
  std::memcpy(o->nc.data(), nc_in, sizeof(double) * 3 * N);
  std::memcpy(o->F.data(), F_in, sizeof(double) * 3 * N);
  o->collide_recolour_only();
  std::memcpy(f_out, o->f.data(), sizeof(double) * 2 * QN);
  o->f.swap(keep);
}

// Classes (0 solid, 1 solid-boundary, 2 fluid, 3 fluid-boundary), the
// smoothed indicator g^(3) and the wall normal (3N).
void orc_geometry(void *h, uint8_t *cls, double *gsm, double *nw) {
  Oracle *o = static_cast<Oracle *>(h);
  if (cls) std::memcpy(cls, o->cls.data(), o->N);
  if (gsm) std::memcpy(gsm, o->gsm.data(), sizeof(double) * o->N);
  if (nw) std::memcpy(nw, o->nw.data(), sizeof(double) * 3 * o->N);
}

// Fields of the most recent step: rho = rho^r + rho^b, phi (with the
// inlet/outlet overrides and the Eq. 34 values at solid-boundary nodes),
// u (Eq. 22, 3N), n_c (3N, post-wetting and Eq. 35), kappa, F (3N).
void orc_fields(void *h, double *rho, double *phi, double *u, double *nc,
                double *kappa, double *F) {
  Oracle *o = static_cast<Oracle *>(h);
  const long N = o->N;
  if (rho)
    for (long n = 0; n < N; ++n) rho[n] = o->rho_r[n] + o->rho_b[n];
  if (phi) std::memcpy(phi, o->phi.data(), sizeof(double) * N);
  if (u) std::memcpy(u, o->u.data(), sizeof(double) * 3 * N);
  if (nc) std::memcpy(nc, o->nc.data(), sizeof(double) * 3 * N);
  if (kappa) std::memcpy(kappa, o->kappa.data(), sizeof(double) * N);
  if (F) std::memcpy(F, o->F.data(), sizeof(double) * 3 * N);
}

// Diagnostics over the fluid nodes:
//  0: red mass sum_x sum_i f^r_i of the stored state
//  1: blue mass, likewise
//  2: S_w, the fraction of fluid nodes with phi < 0 (Sec. IV.B)
//  3: smooth S_w, mean of (1 - phi)/2
//  4: pressure drop: mean rho/3 (Eq. 23) on the inlet plane minus the same
//     on the outlet plane of the flow axis
//  5: capillary number of fluid r: rho0 nu^r <u_a>_{phi>0} / gamma
//  6: capillary number of fluid b: rho0 nu^b <u_a>_{phi<0} / gamma
// Kinds 2-6 use the fields of the most recent step (orc_fields).
double orc_reduce(void *h, int kind) {
  Oracle *o = static_cast<Oracle *>(h);
  const long N = o->N;
  const int Q = o->L.Q;
  if (kind == 0 || kind == 1) {
    double s = 0.0;
    for (long n = 0; n < N; ++n) {
      if (o->solid[n]) continue;
      for (int i = 0; i < Q; ++i) s += o->f[((long)kind * Q + i) * N + n];
    }
    return s;
  }
  if (kind == 2 || kind == 3) {
    double s = 0.0;
    for (long n = 0; n < N; ++n) {
      if (o->solid[n]) continue;
      if (kind == 2)
        s += (o->phi[n] < 0.0) ? 1.0 : 0.0;
      else
        s += 0.5 * (1.0 - o->phi[n]);
    }
    return s / (double)o->n_fluid;
  }
  if (kind == 4) {
    const int a = o->p.flow_axis, na = o->dim(a);
    double si = 0.0, so = 0.0;
    long ci = 0, co = 0;
    for (long n = 0; n < N; ++n) {
      if (o->solid[n]) continue;
      int c[3];
      o->coords(n, c);
      double P = (o->rho_r[n] + o->rho_b[n]) / 3.0;
      if (c[a] == 0) {
        si += P;
        ++ci;
      }
      if (c[a] == na - 1) {
        so += P;
        ++co;
      }
    }
    return (ci ? si / ci : 0.0) - (co ? so / co : 0.0);
  }
  if (kind == 5 || kind == 6) {
    const int a = o->p.flow_axis;
    double s = 0.0;
    long c = 0;
    for (long n = 0; n < N; ++n) {
      if (o->solid[n]) continue;
      bool red = o->phi[n] > 0.0;
      if ((kind == 5) != red) continue;
      s += o->u[a * N + n];
      ++c;
    }
    double tau = (kind == 5) ? o->p.tau_r : o->p.tau_b;
    double mu = o->p.rho0 * (tau - 0.5) / 3.0;
    return c ? mu * (s / c) / o->p.gamma : 0.0;
  }
  return NAN;
}

// ---- single-equation entry points for the tests --------------------------

// Lattice tables: e (Q x 3 ints), w (Q), opposite index (Q). Returns Q.
int orc_lattice(int lattice, int *e, double *w, int *opp) {
  Lattice L = make_lattice(lattice);
  for (int i = 0; i < L.Q; ++i) {
    for (int a = 0; a < 3; ++a) e[3 * i + a] = L.e[i][a];
    w[i] = L.w[i];
    opp[i] = L.opp[i];
  }
  return L.Q;
}

void orc_scheme1(const double *n_c, const double *n_w, double theta,
                 double *out) {
  Oracle::scheme1(n_c, n_w, theta, out);
}

void orc_scheme2(const double *n_c, const double *n_w, double theta,
                 double *out) {
  Oracle::scheme2(n_c, n_w, theta, out);
}

// One node's collision (BGK reading of Eq. 2) on total populations ft (Q).
void orc_collide(int lattice, const double *ft, const double *F, double S,
                 double rho0, double *out, double *u) {
  Lattice L = make_lattice(lattice);
  Oracle::collide(L, ft, F, S, rho0, out, u);
}

// One node's MRT collision (D3Q19, Eq. 2 in moment space) with the rates
// S_nu, S_q, S_m given; Eq. (15) fixes the others to S_nu.
void orc_collide_mrt(const double *ft, const double *F, double Snu, double Sq,
                     double Sm, double rho0, double *out, double *u) {
  Oracle::collide_mrt(ft, F, Snu, Sq, Sm, rho0, out, u);
}

// M of Eq. (A.3) as the oracle builds it (19 x 19, row = moment).
void orc_moment_matrix(double *M) {
  const MomentBasis &B = moment_basis();
  for (int k = 0; k < 19; ++k)
    for (int i = 0; i < 19; ++i) M[19 * k + i] = B.M[k][i];
}

// ---- tangent-linear run ----------------------------------------------------
// The same step on Dual numbers: every field carries its derivatives with
// respect to the contact angle theta (radians; direction 0) and one
// component of the body acceleration (direction 1), seeded in
// orc_tlm_set_params.

void *orc_tlm_create(int lattice, int nx, int ny, int nz, const uint8_t *solid,
                     unsigned periodic_mask) {
  if (lattice != 9 && lattice != 19) return nullptr;
  if (lattice == 9 && nz != 1) return nullptr;
  OracleT<Dual> *o = new OracleT<Dual>();
  o->init(lattice, nx, ny, nz, solid, periodic_mask);
  return o;
}

void orc_tlm_destroy(void *h) { delete static_cast<OracleT<Dual> *>(h); }

// Regularised linearisation of Scheme-II in the tangent-linear run: where
// sin(theta') < freeze_sin the direction of the result around n_w is held
// constant (0: exact derivatives).
void orc_tlm_set_freeze(void *h, double freeze_sin) {
  static_cast<OracleT<Dual> *>(h)->freeze_sin = freeze_sin;
}

// Regularised linearisation of n_c = C/|C|: where |C| < c_min its direction
// is held constant (0: exact derivatives).
void orc_tlm_set_cmin(void *h, double c_min) {
  static_cast<OracleT<Dual> *>(h)->c_min = c_min;
}

// Direction 1 is the component g_axis of the body acceleration.
int orc_tlm_set_params(void *h, const orc_params *p, int g_axis) {
  if (p->collision != 0 && p->collision != 1) return -1;
  if (p->collision == 1 && static_cast<OracleT<Dual> *>(h)->L.Q != 19)
    return -1;
  const Dual th(p->theta_deg * PI / 180.0, 1.0, 0.0);
  Dual gg[3] = {Dual(p->g[0]), Dual(p->g[1]), Dual(p->g[2])};
  gg[g_axis] = Dual(p->g[g_axis], 0.0, 1.0);
  static_cast<OracleT<Dual> *>(h)->set_params(*p, th, gg);
  return 0;
}

void orc_tlm_init_state(void *h, const double *phi0) {
  static_cast<OracleT<Dual> *>(h)->init_state(phi0);
}

void orc_tlm_step(void *h, int nsteps) {
  OracleT<Dual> *o = static_cast<OracleT<Dual> *>(h);
  for (int s = 0; s < nsteps; ++s) o->step();
}

// Smooth S_w of the most recent step (orc_reduce kind 3) and its
// derivatives: out = {S_w, dS_w/dtheta (per radian), dS_w/dg_axis}.
void orc_tlm_sw(void *h, double *out) {
  OracleT<Dual> *o = static_cast<OracleT<Dual> *>(h);
  Dual s = 0.0;
  for (long n = 0; n < o->N; ++n) {
    if (o->solid[n]) continue;
    s += 0.5 * (1.0 - o->phi[n]);
  }
  s = s / (double)o->n_fluid;
  out[0] = s.v;
  out[1] = s.d[0];
  out[2] = s.d[1];
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
