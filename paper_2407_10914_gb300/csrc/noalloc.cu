// lbm_colour_mass_noalloc: the colour-mass reduction of lbm_reduce
// (LBM_MASS_R, LBM_MASS_B) for callers that cannot allocate device memory.
//
// Some callers run under a device-memory budget that another framework
// reserved up front (allocating would fail, or would break that budget), or
// follow a policy that forbids allocation after start-up. They cannot
// provide the workspace that a handle needs. This entry point takes a
// dense float32 population array that the caller already owns (for example
// one filled by lbm_get_populations) and returns the two colour masses using
// only a fixed scratch array that the library holds in device memory.
//
// Scratch: one file-scope __device__ array of NOALLOC_MAX_BLOCKS x 2 block
// partials plus 2 result slots (about 16 KB), present on every GPU that
// loads the library until the process exits. Every call shares it and it
// keeps the last call's contents: every block writes its own partial slot
// and the final pass overwrites the result slots, so nothing needs to start
// at zero; but calls that overlap on the GPU (two streams, or two threads)
// race on the array and may return wrong sums.
//
// The first call on a device looks up the device address of the scratch
// array (cudaGetSymbolAddress) with that device current and caches it.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/lbmgb.h"

namespace {

constexpr int NOALLOC_MAX_BLOCKS = 1024;
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_DEVICES = 64;

// [0, 2*NOALLOC_MAX_BLOCKS): per-block (red, blue) partials;
// [2*NOALLOC_MAX_BLOCKS, +2): the summed (red, blue) result.
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_BLOCKS + 2];

std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void block_sum2(double &a, double &b) {
  __shared__ double sh[2][NOALLOC_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) {
    sh[0][warp] = a;
    sh[1][warp] = b;
  }
  __syncthreads();
  if (warp == 0) {
    a = warp_sum(lane < NOALLOC_THREADS / 32 ? sh[0][lane] : 0.0);
    b = warp_sum(lane < NOALLOC_THREADS / 32 ? sh[1][lane] : 0.0);
  }
}

// sum over nodes and directions of pops[(s*Q + i)*n + node], s = 0, 1
__global__ void __launch_bounds__(NOALLOC_THREADS)
    k_mass_partials(const float *__restrict__ pops, int Q, long long n,
                    double *__restrict__ scratch) {
  double r = 0.0, b = 0.0;
  const long long stride = (long long)gridDim.x * NOALLOC_THREADS;
  for (long long node = (long long)blockIdx.x * NOALLOC_THREADS + threadIdx.x;
       node < n; node += stride) {
    for (int i = 0; i < Q; ++i) {
      r += (double)pops[(long long)i * n + node];
      b += (double)pops[(long long)(Q + i) * n + node];
    }
  }
  block_sum2(r, b);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = r;
    scratch[2 * blockIdx.x + 1] = b;
  }
}

__global__ void __launch_bounds__(NOALLOC_THREADS)
    k_mass_final(int nblocks, double *__restrict__ scratch) {
  double r = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += NOALLOC_THREADS) {
    r += scratch[2 * k];
    b += scratch[2 * k + 1];
  }
  block_sum2(r, b);
  if (threadIdx.x == 0) {
    scratch[2 * NOALLOC_MAX_BLOCKS] = r;
    scratch[2 * NOALLOC_MAX_BLOCKS + 1] = b;
  }
}

// Device address of the scratch array on the current device (set-up on the
// first call per device).
cudaError_t scratch_for_current_device(double **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    double *p = nullptr;
    e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_colour_mass_noalloc(int lattice, int64_t n_nodes,
                                              const float *pops_dev,
                                              double *mass_host,
                                              void *stream) {
  if ((lattice != 9 && lattice != 19) || !pops_dev || !mass_host)
    return LBM_ERR_ARG;
  if (n_nodes < 1 || n_nodes > LBM_NOALLOC_MAX_NODES) return LBM_ERR_ARG;
  // the kernel reads pops_dev: it must be memory of the current device (a
  // host pointer or another GPU's memory would be an illegal access)
  int dev = -1;
  cudaPointerAttributes at{};
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
  if (cudaPointerGetAttributes(&at, pops_dev) != cudaSuccess) {
    cudaGetLastError();  // clear the error of an unknown pointer
    return LBM_ERR_ARG;
  }
  if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) ||
      at.device != dev)
    return LBM_ERR_ARG;
  double *scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return LBM_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  long long want = (n_nodes + NOALLOC_THREADS - 1) / NOALLOC_THREADS;
  const int blocks = (int)(want < NOALLOC_MAX_BLOCKS ? want : NOALLOC_MAX_BLOCKS);
  k_mass_partials<<<blocks, NOALLOC_THREADS, 0, s>>>(pops_dev, lattice,
                                                     (long long)n_nodes, scratch);
  k_mass_final<<<1, NOALLOC_THREADS, 0, s>>>(blocks, scratch);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(mass_host, scratch + 2 * NOALLOC_MAX_BLOCKS,
                        2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
