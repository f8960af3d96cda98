// Lattice constants for the device code: D3Q19 in the order of Eq. (A.1)
// with the weights of Eq. (A.2), and D2Q9 as the z-free members of that set
// in the same order. Everything is constexpr so that fully unrolled loops
// over i see literal velocities and weights.
#pragma once

namespace lbm {

template <int Q>
struct Lattice;

template <>
struct Lattice<19> {
  static constexpr int D = 3;
  static constexpr int E2 = 10;  // sum_i e_ix^2
  // one table per axis, so that a constant i folds to a literal and a
  // run-time axis a costs a select, never a local-memory table
  __host__ __device__ static constexpr int ex(int i) {
    constexpr int X[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1,
                           1, -1, 1, -1, 0, 0, 0, 0};
    return X[i];
  }
  __host__ __device__ static constexpr int ey(int i) {
    constexpr int Y[19] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1,
                           0, 0, 0, 0, 1, -1, 1, -1};
    return Y[i];
  }
  __host__ __device__ static constexpr int ez(int i) {
    constexpr int Z[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0,
                           1, 1, -1, -1, 1, 1, -1, -1};
    return Z[i];
  }
  __host__ __device__ static constexpr int e(int i, int a) {
    return a == 0 ? ex(i) : (a == 1 ? ey(i) : ez(i));
  }
  __host__ __device__ static constexpr float w(int i) {
    return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
  }
  __host__ __device__ static constexpr double wd(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  // opposite direction: pairs (1,2) (3,4) (5,6) (7,10) (8,9) (11,14)
  // (12,13) (15,18) (16,17)
  __host__ __device__ static constexpr int opp(int i) {
    constexpr int O[19] = {0,  2,  1,  4,  3,  6,  5,  10, 9, 8,
                           7, 14, 13, 12, 11, 18, 17, 16, 15};
    return O[i];
  }
  // the first member of the p-th opposite pair (the other is opp(pair(p)))
  __host__ __device__ static constexpr int pair(int p) {
    constexpr int P[9] = {1, 3, 5, 7, 8, 11, 12, 15, 16};
    return P[p];
  }
};

template <>
struct Lattice<9> {
  static constexpr int D = 2;
  static constexpr int E2 = 6;
  __host__ __device__ static constexpr int ex(int i) {
    constexpr int X[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
    return X[i];
  }
  __host__ __device__ static constexpr int ey(int i) {
    constexpr int Y[9] = {0, 0, 0, 1, -1, 1, 1, -1, -1};
    return Y[i];
  }
  __host__ __device__ static constexpr int ez(int) { return 0; }
  __host__ __device__ static constexpr int e(int i, int a) {
    return a == 0 ? ex(i) : (a == 1 ? ey(i) : ez(i));
  }
  __host__ __device__ static constexpr float w(int i) {
    return i == 0 ? 4.0f / 9.0f : (i <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
  }
  __host__ __device__ static constexpr double wd(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int opp(int i) {
    constexpr int O[9] = {0, 2, 1, 4, 3, 8, 7, 6, 5};
    return O[i];
  }
  __host__ __device__ static constexpr int pair(int p) {
    constexpr int P[4] = {1, 3, 5, 6};
    return P[p];
  }
};

}  // namespace lbm
