// The time step as seven dependent passes. Each pass needs the previous
// one's values at lattice neighbours:
//   1 k_stream     (fluid)  pull of Eq. (1), Eqs. (7)-(9): stores f^t,
//                  (rho^r, rho^b) and the phase field; k_zh_fix then applies
//                  App. B on the Zou-He planes
//   2 k_phi_solid  (solid-boundary) Eq. (34)
//   3 k_gradient   (fluid)  Eqs. (6), (27) and wetting, Eqs. (28)-(33)
//   4 k_nc_solid   (solid-boundary) Eq. (35)
//   5 k_curvature  (fluid)  Eq. (12), stored per node
//   6 k_collide    (fluid)  Eqs. (5), (36); Eq. (2) single-rate or MRT on
//                  the stored f^t; store f'' and (q, v), i.e. the
//                  recoloured state of Eqs. (20)-(21)
// One thread per node of the compact fluid (F) or solid-boundary (S) list;
// the work of a node is in passes.cuh.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "passes.cuh"
#include "step.hpp"

namespace lbm {

constexpr int BLOCK = 256;

// Programmatic dependent launch. The passes of a step are launched with
// programmatic stream serialisation: a pass's blocks may be scheduled while
// the previous pass drains its last wave, and each waits
// (griddepcontrol.wait: the previous grid complete, its writes visible)
// before it touches global memory. A pass lets its successor launch once
// all its own blocks have started (launch_dependents), so waiting blocks
// never take the place of a block that has yet to start: no pass waits on
// one that cannot finish. Launched without the attribute (the adjoint's
// recomputation, the timed per-pass launches) both instructions do
// nothing.
__device__ __forceinline__ void pass_entry() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Blocks per SM, measured on the 256^3 rock: the gather passes are bound by
// load latency. The stream pass runs 6 blocks of 256 threads (40 registers:
// 0.205 against 0.223 ms at 7 blocks and 32 registers, with the pull's
// unconditional (q, v) load); the gradient and curvature passes 8 blocks at
// 32 registers (the gradient gains 14 % over its unbounded 34 registers; the
// curvature, a gather of the neighbours' n_c split off the collision, is 7 %
// slower at 6 blocks). The single-rate collision runs 4 blocks (64
// registers; 3 and 5 blocks are 1 % and 11 % slower); the MRT collision
// keeps 3 blocks (it would spill at 64 registers).
template <int Q, int ST>
__global__ void __launch_bounds__(BLOCK, 6) k_stream(Dom d) {
  pass_entry();
  const int k = blockIdx.x * BLOCK + threadIdx.x;
  if (k < d.NF) stream_node<Q, ST, false>(d, k);
}

template <int Q, int ST>
__global__ void __launch_bounds__(BLOCK) k_zh_fix(Dom d) {
  pass_entry();
  const int j = blockIdx.x * BLOCK + threadIdx.x;
  if (j < d.n_zh) zh_fix_node<Q, ST, false>(d, j);
}

template <int Q>
__global__ void __launch_bounds__(BLOCK) k_phi_solid(Dom d) {
  pass_entry();
  const int j = blockIdx.x * BLOCK + threadIdx.x;
  if (j < d.NS) phi_solid_node<Q, false>(d, j);
}

// MARK: the step's form, which marks the solid-boundary nodes that its
// Eq. 35 pass must compute (k_nc_solid_marked); the adjoint recomputes the
// fields with the plain form and the full Eq. 35 pass.
template <int Q, bool MARK>
__global__ void __launch_bounds__(BLOCK, 8) k_gradient(Dom d) {
  pass_entry();
  const int k = blockIdx.x * BLOCK + threadIdx.x;
  if (k < d.NF) gradient_node<Q, false, MARK>(d, k);
}

template <int Q>
__global__ void __launch_bounds__(BLOCK) k_nc_solid(Dom d) {
  pass_entry();
  const int j = blockIdx.x * BLOCK + threadIdx.x;
  if (j < d.NS) nc_solid_node<Q, false>(d, j);
}

template <int Q>
__global__ void __launch_bounds__(BLOCK) k_nc_solid_marked(Dom d) {
  pass_entry();
  const int j = blockIdx.x * BLOCK + threadIdx.x;
  if (j < d.NS) nc_solid_marked_node<Q>(d, j);
}

template <int Q>
__global__ void __launch_bounds__(BLOCK, 8) k_curvature(Dom d) {
  pass_entry();
  const int k = blockIdx.x * BLOCK + threadIdx.x;
  if (k < d.NF) curvature_node<Q, false>(d, k);
}

// MRT: the collision compiled for the single rate (0) or the MRT rates (1)
template <int Q, int ST, bool MACROS, int MRT>
__global__ void __launch_bounds__(BLOCK, MRT ? 3 : 4) k_collide(Dom d) {
  pass_entry();
  const int k = blockIdx.x * BLOCK + threadIdx.x;
  if (k < d.NF) collide_node<Q, ST, MACROS, false, MRT, true>(d, k);
}

// NVTX range around the launch of one pass (header-only NVTX: a no-op
// unless a profiler that records NVTX is attached), so that a timeline
// names every kernel by its pass of the step.
struct PassRange {
  explicit PassRange(const char *name) { nvtxRangePushA(name); }
  ~PassRange() { nvtxRangePop(); }
};

// Launch of one pass: programmatic serialisation on the stream, unless the
// per-pass events sit between the launches.
static void launch_pass(void (*kern)(Dom), unsigned grid, cudaStream_t s,
                        const Dom &d, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(BLOCK);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, d);
}

template <int Q, int ST>
static void launch_step_t(const Dom &d, cudaStream_t s, bool macros,
                          cudaEvent_t *ev) {
  PassRange step_range("lbm step");
  const unsigned g = (unsigned)((d.NF + BLOCK - 1) / BLOCK);
  const unsigned gs = (unsigned)((d.NS + BLOCK - 1) / BLOCK);
  const unsigned gz = (unsigned)((d.n_zh + BLOCK - 1) / BLOCK);
  const bool pdl = ev == nullptr;
  if (ev) cudaEventRecord(ev[0], s);
  {
    PassRange r("stream (Eq. 1, 7-9)");
    launch_pass(k_stream<Q, ST>, g, s, d, pdl);
  }
  if (ev) cudaEventRecord(ev[1], s);
  if (d.n_zh > 0) {
    PassRange r("Zou-He planes (App. B)");
    launch_pass(k_zh_fix<Q, ST>, gz, s, d, pdl);
  }
  if (ev) cudaEventRecord(ev[2], s);
  if (d.NS > 0) {
    PassRange r("phi at solid boundary (Eq. 34)");
    launch_pass(k_phi_solid<Q>, gs, s, d, pdl);
  }
  if (ev) cudaEventRecord(ev[3], s);
  {
    PassRange r("gradient, wetting (Eq. 6, 27-33)");
    launch_pass(k_gradient<Q, true>, g, s, d, pdl);
  }
  if (ev) cudaEventRecord(ev[4], s);
  if (d.NS > 0) {
    PassRange r("n_c at solid boundary (Eq. 35)");
    launch_pass(k_nc_solid_marked<Q>, gs, s, d, pdl);
  }
  if (ev) cudaEventRecord(ev[5], s);
  const bool mrt = Q == 19 && d.c.mrt;
  {
    PassRange r("curvature (Eq. 12)");
    launch_pass(k_curvature<Q>, g, s, d, pdl);
  }
  if (ev) cudaEventRecord(ev[6], s);
  PassRange r("force, collision, recolouring (Eq. 5, 2, 20-21)");
  if (macros) {
    launch_pass(mrt ? k_collide<Q, ST, true, 1> : k_collide<Q, ST, true, 0>, g, s,
                d, pdl);
  } else {
    launch_pass(mrt ? k_collide<Q, ST, false, 1> : k_collide<Q, ST, false, 0>,
                g, s, d, pdl);
  }
  if (ev) cudaEventRecord(ev[7], s);
}

template <int Q, int ST>
static void launch_fields_t(const Dom &d, cudaStream_t s) {
  const unsigned g = (unsigned)((d.NF + BLOCK - 1) / BLOCK);
  const unsigned gs = (unsigned)((d.NS + BLOCK - 1) / BLOCK);
  const unsigned gz = (unsigned)((d.n_zh + BLOCK - 1) / BLOCK);
  k_stream<Q, ST><<<g, BLOCK, 0, s>>>(d);
  if (d.n_zh > 0) k_zh_fix<Q, ST><<<gz, BLOCK, 0, s>>>(d);
  if (d.NS > 0) k_phi_solid<Q><<<gs, BLOCK, 0, s>>>(d);
  k_gradient<Q, false><<<g, BLOCK, 0, s>>>(d);
  if (d.NS > 0) k_nc_solid<Q><<<gs, BLOCK, 0, s>>>(d);
}

void launch_fields(int Q, int storage, const Dom &d, cudaStream_t s) {
  if (Q == 19) {
    if (storage == LBM_STORAGE_FP32) launch_fields_t<19, LBM_STORAGE_FP32>(d, s);
    if (storage == LBM_STORAGE_FP16) launch_fields_t<19, LBM_STORAGE_FP16>(d, s);
    if (storage == LBM_STORAGE_BF16) launch_fields_t<19, LBM_STORAGE_BF16>(d, s);
  } else {
    if (storage == LBM_STORAGE_FP32) launch_fields_t<9, LBM_STORAGE_FP32>(d, s);
    if (storage == LBM_STORAGE_FP16) launch_fields_t<9, LBM_STORAGE_FP16>(d, s);
    if (storage == LBM_STORAGE_BF16) launch_fields_t<9, LBM_STORAGE_BF16>(d, s);
  }
}

static void dispatch(int Q, int storage, const Dom &d, cudaStream_t s,
                     bool macros, cudaEvent_t *ev) {
  if (Q == 19) {
    if (storage == LBM_STORAGE_FP32) launch_step_t<19, LBM_STORAGE_FP32>(d, s, macros, ev);
    if (storage == LBM_STORAGE_FP16) launch_step_t<19, LBM_STORAGE_FP16>(d, s, macros, ev);
    if (storage == LBM_STORAGE_BF16) launch_step_t<19, LBM_STORAGE_BF16>(d, s, macros, ev);
  } else {
    if (storage == LBM_STORAGE_FP32) launch_step_t<9, LBM_STORAGE_FP32>(d, s, macros, ev);
    if (storage == LBM_STORAGE_FP16) launch_step_t<9, LBM_STORAGE_FP16>(d, s, macros, ev);
    if (storage == LBM_STORAGE_BF16) launch_step_t<9, LBM_STORAGE_BF16>(d, s, macros, ev);
  }
}

void launch_step(int Q, int storage, const Dom &d, cudaStream_t s,
                 bool macros) {
  dispatch(Q, storage, d, s, macros, nullptr);
}

void launch_step_events(int Q, int storage, const Dom &d, cudaStream_t s,
                        bool macros, cudaEvent_t *ev) {
  dispatch(Q, storage, d, s, macros, ev);
}

}  // namespace lbm
