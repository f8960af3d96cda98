// FP64 diagnostics over the compact fluid list: warp-shuffle, then block,
// then a one-block pass over the per-block partials. Four accumulators per
// kind; the host combines them (a ratio or a difference).
#include <cuda_runtime.h>

#include "stencil.cuh"
#include "step.hpp"

namespace lbm {

constexpr int RBLOCK = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of four values; thread 0 gets the totals.
__device__ __forceinline__ void block_sum4(double *v) {
  __shared__ double sh[4][RBLOCK / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double s = warp_sum(v[k]);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double s = lane < RBLOCK / 32 ? sh[k][lane] : 0.0;
      v[k] = warp_sum(s);
    }
  }
}

// kind: LBM_MASS_R/B: acc0 = colour density sum_i f^s_i of the stored state
// (mu rho for the minority colour, (1 - mu) rho for the other);
// LBM_SW_COUNT: acc0 = #(phi < 0); LBM_SW_SMOOTH: acc0 = sum (1 - phi)/2;
// LBM_DP: acc0/acc1 = sum/count of rho on the inlet plane, acc2/acc3 the same
// on the outlet plane; LBM_CA_R/B: acc0/acc1 = sum/count of u_a over phi > 0
// (phi < 0).
template <int Q, int ST>
__global__ void __launch_bounds__(RBLOCK) k_reduce(Dom d, int kind,
                                                   double *__restrict__ part) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int stride = gridDim.x * RBLOCK;
  const int a = d.c.axis;
  const int na = axis_extent(d, a);
  for (int k = blockIdx.x * RBLOCK + threadIdx.x; k < d.NF; k += stride) {
    if (kind == LBM_MASS_R || kind == LBM_MASS_B) {
      double rho = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) rho += (double)TIO<Q, ST>::load(d, i, k);
      const float q = d.S_src[k].x;
      const double minor = (double)q * rho;
      const bool red_minor = m_blue(q);
      const bool want_red = kind == LBM_MASS_R;
      acc[0] += (want_red == red_minor) ? minor : rho - minor;
    } else if (kind == LBM_SW_COUNT || kind == LBM_SW_SMOOTH) {
      const float m = d.mf[k];
      if (kind == LBM_SW_COUNT)
        acc[0] += (m_blue(m) && m < 0.5f) ? 1.0 : 0.0;
      else
        acc[0] += m_blue(m) ? 1.0 - (double)m : (double)m;
    } else if (kind == LBM_DP) {
      int x, y, z;
      box_coords(d, d.fg[k], x, y, z);
      const int ca = axis_coord(x, y, z, a);
      const double rho = d.macro[k].w;
      if (ca == 0) {
        acc[0] += rho;
        acc[1] += 1.0;
      }
      if (ca == na - 1) {
        acc[2] += rho;
        acc[3] += 1.0;
      }
    } else {
      const float m = d.mf[k];
      const bool red = !m_blue(m) && m < 0.5f;  // phi > 0
      const bool blue = m_blue(m) && m < 0.5f;  // phi < 0
      if ((kind == LBM_CA_R && red) || (kind == LBM_CA_B && blue)) {
        const float4 mc = d.macro[k];
        acc[0] += a == 0 ? mc.x : (a == 1 ? mc.y : mc.z);
        acc[1] += 1.0;
      }
    }
  }
  block_sum4(acc);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) part[(long long)blockIdx.x * 4 + k] = acc[k];
}

__global__ void __launch_bounds__(RBLOCK) k_reduce_final(
    const double *__restrict__ part, int nparts, double *__restrict__ out) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nparts; b += RBLOCK)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] += part[(long long)b * 4 + k];
  block_sum4(acc);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = acc[k];
}

void launch_reduce(int Q, int st, const Dom &d, int kind, double *part,
                   int slots, double *out, cudaStream_t s) {
  const long long want = ((long long)d.NF + RBLOCK - 1) / RBLOCK;
  const int g = (int)(want < slots ? (want > 0 ? want : 1) : slots);
#define LBM_RED(QQ, SS) k_reduce<QQ, SS><<<g, RBLOCK, 0, s>>>(d, kind, part)
  if (Q == 19) {
    if (st == 0) LBM_RED(19, 0);
    if (st == 1) LBM_RED(19, 1);
    if (st == 2) LBM_RED(19, 2);
  } else {
    if (st == 0) LBM_RED(9, 0);
    if (st == 1) LBM_RED(9, 1);
    if (st == 2) LBM_RED(9, 2);
  }
#undef LBM_RED
  k_reduce_final<<<1, RBLOCK, 0, s>>>(part, g, out);
}

}  // namespace lbm
