// Many independent domains (cases) stepped together: the batched sweep.
//
// A batch holds a case table in device memory: the kernel arguments (Dom)
// of every case, with the state buffers in the orientation they had when
// the table was written; a device flag `parity` says whether they are
// swapped since. Two ways to run a step of all cases:
//
//  mode 0, level launches: one launch per pass covering every case. Block b
//    belongs to the case c with start[c] <= b < start[c + 1] (start is the
//    prefix of each case's block count for that pass). A step is five or
//    six launches whatever the number of cases.
//
//  mode 1, persistent: one launch runs all passes of nsteps steps. Work
//    items are (level, case, chunk), a chunk being `chunk` blocks' worth of
//    nodes of one pass of one case; level = 6 s + pass. Blocks take items
//    from a global counter in level-major order (every item of level L of
//    every case before any item of level L + 1). Before working on an item
//    a block waits until its case has completed every chunk of the earlier
//    levels (a per-case completion counter). The dependencies of an item
//    are items taken earlier, held by blocks that are running, so the waits
//    end whatever the grid size. Each wait is bounded by the GPU's global
//    timer: past the limit the block sets the error flag and every block
//    leaves; lbm_batch_status() reports LBM_ERR_TIMEOUT. Values written in
//    the launch are read with plain coherent loads, after the item's
//    acquire, fence and block barrier (passes.cuh, COH = true).
//
// Both modes are recorded once per (nsteps, configuration) into a CUDA
// graph on a stream the batch owns and replayed on the caller's stream.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "passes.cuh"
#include "step.hpp"

namespace lbm {

// Passes of a step in launch order and the node set each one runs over.
enum Pass { P_STREAM = 0, P_ZH = 1, P_PHI_S = 2, P_GRAD = 3, P_NC_S = 4,
            P_COLLIDE = 5, N_PASS = 6 };
enum Space { SP_F = 0, SP_Z = 1, SP_S = 2 };
__host__ __device__ constexpr int space_of(int p) {
  return p == P_ZH ? SP_Z : ((p == P_PHI_S || p == P_NC_S) ? SP_S : SP_F);
}

// Device control block of a batch (in its workspace).
struct BatchCtl {
  int parity;                // 1: every case's state buffers are swapped
  int err;                   // 1: a bounded wait ran out
  unsigned long long head;   // next work item (mode 1)
  unsigned long long spare;  // keeps done[] 16-byte aligned
};

__device__ __forceinline__ int nodes_in(const Dom &d, int space) {
  return space == SP_F ? d.NF : (space == SP_Z ? d.n_zh : d.NS);
}

// Copy the table entry of case c into shared memory, the state buffers
// swapped when `swap`.
__device__ __forceinline__ void load_case(Dom *sd, const Dom *__restrict__ table,
                                          int c, bool swap) {
  constexpr int W = sizeof(Dom) / sizeof(int);
  static_assert(sizeof(Dom) % sizeof(int) == 0, "Dom is whole words");
  const int *src = (const int *)(table + c);
  int *dst = (int *)sd;
  for (int w = threadIdx.x; w < W; w += blockDim.x) dst[w] = __ldg(src + w);
  __syncthreads();
  if (threadIdx.x == 0 && swap) {
    const void *t = sd->T_src;
    sd->T_src = sd->T_dst;
    sd->T_dst = const_cast<void *>(t);
    const float4 *u = sd->S_src;
    sd->S_src = sd->S_dst;
    sd->S_dst = const_cast<float4 *>(u);
  }
  __syncthreads();
}

// The work of one node of pass P.
template <int Q, int ST, bool COH>
__device__ __forceinline__ void run_node(const Dom &d, int pass, bool macros,
                                         int n) {
  switch (pass) {
    case P_STREAM: stream_node<Q, ST, COH>(d, n); break;
    case P_ZH: zh_fix_node<Q, ST, COH>(d, n); break;
    case P_PHI_S: phi_solid_node<Q, COH>(d, n); break;
    case P_GRAD: gradient_node<Q, COH>(d, n); break;
    case P_NC_S: nc_solid_node<Q, COH>(d, n); break;
    default:
      // the same collision instantiations as the single-domain kernels
      // (single rate or MRT fixed at compile time), so that a case stepped
      // in a batch and alone agree bit for bit
      if (d.c.mrt) {
        if (macros) collide_node<Q, ST, true, COH, 1>(d, n);
        else collide_node<Q, ST, false, COH, 1>(d, n);
      } else {
        if (macros) collide_node<Q, ST, true, COH, 0>(d, n);
        else collide_node<Q, ST, false, COH, 0>(d, n);
      }
  }
}

// Block's case: the c with start[c] <= b < start[c + 1] (binary search).
__device__ __forceinline__ int case_of(const int *__restrict__ start, int n,
                                       int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Resident 256-thread blocks per SM each pass is compiled for, as in the
// single-domain kernels (step.cu): the gather passes with few registers
// (stream 6 blocks, the stencils 8), the collision (with the curvature of
// Eq. 12 computed in it) 3 blocks; twice as many blocks of 128 threads.
template <int P, int BT>
struct PassBlocks {
  static constexpr int k256 =
      P == P_STREAM ? 6 : (P == P_COLLIDE ? 3 : 8);
  static constexpr int value = BT == 256 ? k256 : 2 * k256;
};

// Mode 0: pass P of step s for every case; start = that pass's block prefix.
template <int Q, int ST, int P, bool MACROS, int BT>
__global__ void __launch_bounds__(BT, (PassBlocks<P, BT>::value))
    k_batch_pass(const Dom *__restrict__ table,
                                                   const int *__restrict__ start,
                                                   int ncase,
                                                   const BatchCtl *__restrict__ ctl,
                                                   int s) {
  __shared__ __align__(16) Dom sd;
  const int b = blockIdx.x;
  const int c = case_of(start, ncase, b);
  load_case(&sd, table, c, (ctl->parity ^ s) & 1);
  const int n = (b - __ldg(start + c)) * BT + threadIdx.x;
  if (n < nodes_in(sd, space_of(P))) run_node<Q, ST, false>(sd, P, MACROS, n);
}

// ------------------------------------------------------------- mode 1
// Work of one launch: per space the prefix over the cases of their chunk
// counts (pre[space][c], c = 0..ncase), the chunk size in blocks, and the
// items of one step (3 fluid passes, the Zou-He fix-up, 2 solid passes).
struct Plan {
  const int *pre[3];
  int ncase;
  int chunk;
  long long tot[3];     // pre[space][ncase]
  long long per_step;   // 3 tot[F] + tot[Z] + 2 tot[S]
};

__device__ __forceinline__ unsigned long long ld_acquire(
    const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait until *cnt >= need. Gives up (returns false) after limit_ns of the
// GPU's global timer, or as soon as another block has set ctl->err.
__device__ bool wait_count(const unsigned long long *cnt,
                           unsigned long long need, const BatchCtl *ctl,
                           unsigned long long limit_ns) {
  if (ld_acquire(cnt) >= need) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    __nanosleep(200);
    if (ld_acquire(cnt) >= need) return true;
    if (*(volatile const int *)&ctl->err) return false;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// All passes in one kernel: the registers of the heaviest (the collision
// with the curvature), bounded to 4 resident blocks of 256 threads (64
// registers, 204 B of spills: 8.75-9.04 ms per step on the 96 drops,
// against 9.61-9.92 at 3 blocks and 80 registers and 11.35-11.58 at 2;
// 5 blocks would spill 848 B).
template <int Q, int ST, int BT>
__global__ void __launch_bounds__(BT, BT == 256 ? 4 : 8) k_batch_persistent(
    const Dom *__restrict__ table, Plan pl, BatchCtl *ctl,
    unsigned long long *done, int nsteps, unsigned long long limit_ns) {
  __shared__ __align__(16) Dom sd;
  __shared__ long long s_item;
  __shared__ int s_ok;
  const long long total = pl.per_step * nsteps;
  for (;;) {
    if (threadIdx.x == 0) {
      long long it = (long long)atomicAdd(&ctl->head, 1ull);
      if (*(volatile int *)&ctl->err) it = total;
      s_item = it;
    }
    __syncthreads();
    const long long item = s_item;
    if (item >= total) break;  // the same for the whole block
    // decode (step, pass, case, chunk)
    const int s = (int)(item / pl.per_step);
    long long r = item - (long long)s * pl.per_step;
    int pass = 0;
    while (r >= pl.tot[space_of(pass)]) {
      r -= pl.tot[space_of(pass)];
      ++pass;
    }
    const int sp = space_of(pass);
    const int c = case_of(pl.pre[sp], pl.ncase, (int)r);
    const int j = (int)r - __ldg(pl.pre[sp] + c);
    // chunks this case completes per step, and before this pass
    const int cf = __ldg(pl.pre[SP_F] + c + 1) - __ldg(pl.pre[SP_F] + c);
    const int cz = __ldg(pl.pre[SP_Z] + c + 1) - __ldg(pl.pre[SP_Z] + c);
    const int cs = __ldg(pl.pre[SP_S] + c + 1) - __ldg(pl.pre[SP_S] + c);
    const unsigned long long per = 3ull * cf + cz + 2ull * cs;
    const int before[N_PASS] = {0, cf, cf + cz, cf + cz + cs,
                                2 * cf + cz + cs, 2 * cf + cz + 2 * cs};
    const unsigned long long need = (unsigned long long)s * per + before[pass];
    if (threadIdx.x == 0) {
      const bool ok = wait_count(done + c, need, ctl, limit_ns);
      if (!ok) atomicExch(&ctl->err, 1);
      __threadfence();
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    load_case(&sd, table, c, (ctl->parity ^ s) & 1);
    const int cnt = nodes_in(sd, sp);
    const bool macros = s == nsteps - 1;
    for (int q = 0; q < pl.chunk; ++q) {
      const int n = (j * pl.chunk + q) * BT + threadIdx.x;
      if (n < cnt) run_node<Q, ST, true>(sd, pass, macros, n);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(done + c, 1ull);
    }
  }
}

// After every batch launch: flip the parity by the steps taken, rewind the
// queue and the completion counters.
__global__ void k_batch_finish(BatchCtl *ctl, unsigned long long *done,
                               int ncase, int nsteps) {
  for (int c = threadIdx.x; c < ncase; c += blockDim.x) done[c] = 0;
  if (threadIdx.x == 0) {
    ctl->parity ^= nsteps & 1;
    ctl->head = 0;
  }
}

// The bounded wait on a count that nothing raises: it must give up after
// limit_ns and set the error flag.
__global__ void k_batch_wait_test(BatchCtl *ctl, unsigned long long *done,
                                  unsigned long long limit_ns) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (!wait_count(done, ~0ull, ctl, limit_ns)) atomicExch(&ctl->err, 1);
  }
}

}  // namespace lbm

// ---------------------------------------------------------------- host
using lbm::BatchCtl;
using lbm::Dom;

struct lbm_batch_s {
  int n = 0, Q = 0, storage = 0;
  std::vector<lbm_ctx *> cases;
  std::vector<unsigned long long> gen;  // case generations the table holds
  int mode = 0, threads = 256, chunk = 4;
  unsigned long long limit_ns = 2000000000ull;
  // device memory inside the caller's workspace
  Dom *table = nullptr;
  BatchCtl *ctl = nullptr;
  unsigned long long *done = nullptr;
  int *start[3] = {nullptr, nullptr, nullptr};  // mode 0 block prefixes
  int *pre[3] = {nullptr, nullptr, nullptr};    // mode 1 chunk prefixes
  long long tot_blocks[3] = {0, 0, 0};
  long long tot_chunks[3] = {0, 0, 0};
  int persistent_grid = 0;
  cudaStream_t cap = nullptr;  // capture stream
  std::map<std::tuple<int, int, int, int>, cudaGraphExec_t> graphs;
  char err[256] = {0};
  ~lbm_batch_s() {
    for (auto &g : graphs) cudaGraphExecDestroy(g.second);
    if (cap) cudaStreamDestroy(cap);
  }
};

namespace {

constexpr size_t BALIGN = 256;
size_t balign(size_t v) { return (v + BALIGN - 1) / BALIGN * BALIGN; }

struct BatchLayout {
  size_t table, ctl, done, start[3], pre[3], total;
};

BatchLayout batch_layout(int n) {
  BatchLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = balign(o + bytes);
    return at;
  };
  L.table = take(sizeof(Dom) * (size_t)n);
  L.ctl = take(sizeof(BatchCtl));
  L.done = take(sizeof(unsigned long long) * (size_t)n);
  for (int s = 0; s < 3; ++s) L.start[s] = take(sizeof(int) * (size_t)(n + 1));
  for (int s = 0; s < 3; ++s) L.pre[s] = take(sizeof(int) * (size_t)(n + 1));
  L.total = o;
  return L;
}

lbm_status bfail(lbm_batch b, lbm_status st, const char *msg) {
  if (b) snprintf(b->err, sizeof(b->err), "%s", msg);
  return st;
}

int nodes_of(const Dom &d, int space) {
  return space == lbm::SP_F ? d.NF : (space == lbm::SP_Z ? d.n_zh : d.NS);
}

// Block prefixes (mode 0) and chunk prefixes (mode 1) for the configured
// block size and chunk, uploaded on `s`.
cudaError_t upload_plans(lbm_batch b, cudaStream_t s) {
  std::vector<int> st(3 * (b->n + 1)), pr(3 * (b->n + 1));
  for (int sp = 0; sp < 3; ++sp) {
    long long accb = 0, accc = 0;
    for (int c = 0; c < b->n; ++c) {
      st[sp * (b->n + 1) + c] = (int)accb;
      pr[sp * (b->n + 1) + c] = (int)accc;
      const long long nn = nodes_of(b->cases[c]->d, sp);
      accb += (nn + b->threads - 1) / b->threads;
      accc += (nn + (long long)b->threads * b->chunk - 1) /
              ((long long)b->threads * b->chunk);
    }
    st[sp * (b->n + 1) + b->n] = (int)accb;
    pr[sp * (b->n + 1) + b->n] = (int)accc;
    b->tot_blocks[sp] = accb;
    b->tot_chunks[sp] = accc;
  }
  cudaError_t e = cudaSuccess;
  for (int sp = 0; sp < 3 && e == cudaSuccess; ++sp) {
    e = cudaMemcpyAsync(b->start[sp], st.data() + sp * (b->n + 1),
                        sizeof(int) * (b->n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->pre[sp], pr.data() + sp * (b->n + 1),
                          sizeof(int) * (b->n + 1), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host vectors die
  return e;
}

// The table from the cases' current kernel arguments; parity back to 0.
cudaError_t upload_table(lbm_batch b, cudaStream_t s) {
  std::vector<Dom> h(b->n);
  for (int c = 0; c < b->n; ++c) {
    h[c] = b->cases[c]->d;
    b->gen[c] = b->cases[c]->gen;
  }
  cudaError_t e = cudaMemcpyAsync(b->table, h.data(), sizeof(Dom) * b->n,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&b->ctl->parity, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace

namespace lbm {

template <int Q, int ST, int BT>
static void launch_pass(lbm_batch b, int p, bool macros, int s,
                        cudaStream_t st) {
  const int sp = space_of(p);
  const unsigned g = (unsigned)b->tot_blocks[sp];
  if (g == 0) return;
  const int *start = b->start[sp];
#define LBM_BP(P, M) \
  k_batch_pass<Q, ST, P, M, BT><<<g, BT, 0, st>>>(b->table, start, b->n, b->ctl, s)
  switch (p) {
    case P_STREAM: LBM_BP(P_STREAM, false); break;
    case P_ZH: LBM_BP(P_ZH, false); break;
    case P_PHI_S: LBM_BP(P_PHI_S, false); break;
    case P_GRAD: LBM_BP(P_GRAD, false); break;
    case P_NC_S: LBM_BP(P_NC_S, false); break;
    default:
      if (macros) LBM_BP(P_COLLIDE, true);
      else LBM_BP(P_COLLIDE, false);
  }
#undef LBM_BP
}

template <int Q, int ST, int BT>
static void record_t(lbm_batch b, int nsteps, cudaStream_t st) {
  if (b->mode == 0) {
    for (int s = 0; s < nsteps; ++s)
      for (int p = 0; p < N_PASS; ++p)
        launch_pass<Q, ST, BT>(b, p, s == nsteps - 1, s, st);
  } else {
    Plan pl{};
    for (int sp = 0; sp < 3; ++sp) {
      pl.pre[sp] = b->pre[sp];
      pl.tot[sp] = b->tot_chunks[sp];
    }
    pl.ncase = b->n;
    pl.chunk = b->chunk;
    pl.per_step = 3 * pl.tot[SP_F] + pl.tot[SP_Z] + 2 * pl.tot[SP_S];
    k_batch_persistent<Q, ST, BT><<<b->persistent_grid, BT, 0, st>>>(
        b->table, pl, b->ctl, b->done, nsteps, b->limit_ns);
  }
  k_batch_finish<<<1, 256, 0, st>>>(b->ctl, b->done, b->n, nsteps);
}

template <int Q, int ST>
static void record_q(lbm_batch b, int nsteps, cudaStream_t st) {
  if (b->threads == 128)
    record_t<Q, ST, 128>(b, nsteps, st);
  else
    record_t<Q, ST, 256>(b, nsteps, st);
}

static void record(lbm_batch b, int nsteps, cudaStream_t st) {
  if (b->Q == 19) {
    if (b->storage == LBM_STORAGE_FP32) record_q<19, LBM_STORAGE_FP32>(b, nsteps, st);
    if (b->storage == LBM_STORAGE_FP16) record_q<19, LBM_STORAGE_FP16>(b, nsteps, st);
    if (b->storage == LBM_STORAGE_BF16) record_q<19, LBM_STORAGE_BF16>(b, nsteps, st);
  } else {
    if (b->storage == LBM_STORAGE_FP32) record_q<9, LBM_STORAGE_FP32>(b, nsteps, st);
    if (b->storage == LBM_STORAGE_FP16) record_q<9, LBM_STORAGE_FP16>(b, nsteps, st);
    if (b->storage == LBM_STORAGE_BF16) record_q<9, LBM_STORAGE_BF16>(b, nsteps, st);
  }
}

template <int Q, int ST>
static cudaError_t occupancy_q(int threads, int *per_sm) {
  if (threads == 128)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        per_sm, k_batch_persistent<Q, ST, 128>, 128, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      per_sm, k_batch_persistent<Q, ST, 256>, 256, 0);
}

// Resident blocks of the persistent kernel on this GPU.
static cudaError_t persistent_grid(lbm_batch b, int *grid) {
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = cudaSuccess;
  if (b->Q == 19) {
    if (b->storage == 0) e = occupancy_q<19, 0>(b->threads, &per_sm);
    if (b->storage == 1) e = occupancy_q<19, 1>(b->threads, &per_sm);
    if (b->storage == 2) e = occupancy_q<19, 2>(b->threads, &per_sm);
  } else {
    if (b->storage == 0) e = occupancy_q<9, 0>(b->threads, &per_sm);
    if (b->storage == 1) e = occupancy_q<9, 1>(b->threads, &per_sm);
    if (b->storage == 2) e = occupancy_q<9, 2>(b->threads, &per_sm);
  }
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *grid = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  return e;
}

}  // namespace lbm

extern "C" {

size_t lbm_batch_workspace_bytes(int ncases) {
  return ncases < 1 ? 0 : batch_layout(ncases).total;
}

lbm_status lbm_batch_create(lbm_batch *out, const lbm_handle *cases,
                            int ncases, void *dev_workspace, size_t ws_bytes,
                            void *stream) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  if (!cases || ncases < 1 || !dev_workspace) return LBM_ERR_ARG;
  if (((uintptr_t)dev_workspace) % BALIGN) return LBM_ERR_ARG;
  const BatchLayout L = batch_layout(ncases);
  if (ws_bytes < L.total) return LBM_ERR_NOMEM;
  for (int c = 0; c < ncases; ++c) {
    if (!cases[c]) return LBM_ERR_ARG;
    if (cases[c]->Q != cases[0]->Q || cases[c]->storage != cases[0]->storage)
      return LBM_ERR_ARG;
    if (!cases[c]->params_set || !cases[c]->state_set) return LBM_ERR_STATE;
    for (int k = 0; k < c; ++k)
      if (cases[k] == cases[c]) return LBM_ERR_ARG;  // stepped twice a step
  }
  lbm_batch b = new (std::nothrow) lbm_batch_s();
  if (!b) return LBM_ERR_NOMEM;
  b->n = ncases;
  b->Q = cases[0]->Q;
  b->storage = cases[0]->storage;
  b->cases.assign(cases, cases + ncases);
  b->gen.assign(ncases, 0);
  char *base = (char *)dev_workspace;
  b->table = (Dom *)(base + L.table);
  b->ctl = (BatchCtl *)(base + L.ctl);
  b->done = (unsigned long long *)(base + L.done);
  for (int s = 0; s < 3; ++s) {
    b->start[s] = (int *)(base + L.start[s]);
    b->pre[s] = (int *)(base + L.pre[s]);
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ctl, 0, sizeof(BatchCtl), s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->done, 0, sizeof(unsigned long long) * ncases, s);
  if (e == cudaSuccess) e = upload_table(b, s);
  if (e == cudaSuccess) e = upload_plans(b, s);
  if (e == cudaSuccess) e = lbm::persistent_grid(b, &b->persistent_grid);
  if (e != cudaSuccess) {
    delete b;
    return LBM_ERR_CUDA;
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_set_config(lbm_batch b, int mode, int threads, int chunk,
                                void *stream) {
  if (!b) return LBM_ERR_ARG;
  if (mode != 0 && mode != 1)
    return bfail(b, LBM_ERR_ARG, "mode must be 0 (level launches) or 1 (persistent)");
  if (threads != 128 && threads != 256)
    return bfail(b, LBM_ERR_ARG, "threads must be 128 or 256");
  if (chunk < 1 || chunk > 64)
    return bfail(b, LBM_ERR_ARG, "chunk must be in [1, 64]");
  if (mode == b->mode && threads == b->threads && chunk == b->chunk)
    return LBM_OK;
  b->mode = mode;
  b->threads = threads;
  b->chunk = chunk;
  // recorded graphs bake the previous plan's grid and chunk
  for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
  b->graphs.clear();
  cudaError_t e = upload_plans(b, (cudaStream_t)stream);
  if (e == cudaSuccess) e = lbm::persistent_grid(b, &b->persistent_grid);
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch b, int nsteps, void *stream) {
  if (!b || nsteps < 0) return LBM_ERR_ARG;
  if (nsteps == 0) return LBM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < b->n; ++c) {
    if (!b->cases[c]->state_set) return bfail(b, LBM_ERR_STATE, "case without state");
    if (b->cases[c]->gen != b->gen[c]) {
      // a case was changed or stepped on its own since the table was written
      e = upload_table(b, s);
      break;
    }
  }
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, cudaGetErrorString(e));
  const auto key = std::make_tuple(nsteps, b->mode, b->threads, b->chunk);
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      lbm::record(b, nsteps, b->cap);
      e = cudaStreamEndCapture(b->cap, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, cudaGetErrorString(e));
    it = b->graphs.emplace(key, x).first;
  }
  e = cudaGraphLaunch(it->second, s);
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, cudaGetErrorString(e));
  if (nsteps & 1)
    for (lbm_ctx *c : b->cases) lbm::swap_state(c);
  return LBM_OK;
}

lbm_status lbm_batch_status(lbm_batch b, void *stream) {
  if (!b) return LBM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, &b->ctl->err, sizeof(int),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, cudaGetErrorString(e));
  if (!err) return LBM_OK;
  e = cudaMemsetAsync(&b->ctl->err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, cudaGetErrorString(e));
  return bfail(b, LBM_ERR_TIMEOUT, "a persistent-kernel wait ran out of time");
}

lbm_status lbm_batch_check_wait(lbm_batch b, double limit_ms, double *waited_ms,
                                void *stream) {
  if (!b || !(limit_ms > 0.0) || limit_ms > 10000.0) return LBM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
  if (e == cudaSuccess) {
    lbm::k_batch_wait_test<<<1, 32, 0, s>>>(
        b->ctl, b->done, (unsigned long long)(limit_ms * 1e6));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  for (auto &x : ev)
    if (x) cudaEventDestroy(x);
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, cudaGetErrorString(e));
  if (waited_ms) *waited_ms = ms;
  const lbm_status st = lbm_batch_status(b, stream);  // reads and clears
  if (st == LBM_ERR_TIMEOUT) return LBM_OK;           // gave up, as designed
  return st == LBM_OK ? bfail(b, LBM_ERR_STATE, "the wait did not give up") : st;
}

const char *lbm_batch_last_error(lbm_batch b) { return b ? b->err : "null batch"; }

void lbm_batch_destroy(lbm_batch b) { delete b; }

}  // extern "C"
