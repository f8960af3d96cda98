/*
 * lbmgb.h - C-ABI of the GB300 two-colour lattice-Boltzmann step.
 *
 * The method is the colour-gradient model studied in Sedahmed & Coelho,
 * "Wetting and pressure gradient performance in lattice Boltzmann color
 * gradient model" (arXiv:2407.10914), Sec. II: two populations f^r, f^b on a
 * D3Q19 (Eq. A.1) or D2Q9 lattice; streaming with halfway bounce-back at
 * solid nodes (Eq. 1); Zou-He pressure ends (Type-I, Sec. II.C.1 and App. B)
 * or a uniform body force (Type-II, Eq. 36); phase field (Eq. 7), colour
 * gradient (Eq. 6), wetting by Scheme-I (Eqs. 28-31) or Scheme-II (Eqs.
 * 32-33) with the extrapolations of Eqs. 34-35, curvature (Eq. 12), CSF force
 * (Eq. 5), the collision of Eq. 2 in its single-rate (BGK) form or with the
 * MRT rates of Eqs. 4, 15-16, the viscosity of Eqs. 13-14, and recolouring
 * (Eqs. 20-21).
 *
 * Conventions shared by every call:
 *  - Layout. A field over the box has N = nx*ny*nz entries, node
 *    n = x + nx*(y + ny*z), x fastest. Populations exchanged with the caller
 *    are float32 [2][Q][N] (colour 0 = red "r", 1 = blue "b"); vector fields
 *    are [3][N]. For D2Q9, nz = 1 and the velocities are the z-free members
 *    of Eq. (A.1) in that order: (0,0) (1,0) (-1,0) (0,1) (0,-1) (1,1)
 *    (-1,1) (1,-1) (-1,-1).
 *  - Memory. The caller owns all device memory. lbm_workspace_bytes() says
 *    how much one domain needs; the caller allocates it (any allocator) and
 *    passes it to lbm_init_geometry(); the library never calls cudaMalloc.
 *    Host arrays are read during the call and not kept.
 *  - Streams. `stream` is a cudaStream_t passed as void* (0 = legacy
 *    default stream). Calls enqueue work and return, except lbm_reduce() and
 *    lbm_workspace_bytes(), which synchronise the stream.
 *  - Errors. Every call returns an lbm_status. Argument errors are found
 *    before anything is enqueued; lbm_last_error() then holds a message.
 *    A handle is used by one host thread and one stream at a time.
 */
#ifndef LBMGB_H
#define LBMGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx *lbm_handle;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,       /* invalid argument (nothing was enqueued)      */
  LBM_ERR_CUDA = -2,      /* a CUDA call failed                            */
  LBM_ERR_STATE = -3,     /* call order: params/state not set yet          */
  LBM_ERR_NONFINITE = -4, /* a reduction met NaN/Inf                       */
  LBM_ERR_TIMEOUT = -5,   /* a bounded device wait gave up                 */
  LBM_ERR_NOMEM = -6      /* workspace smaller than lbm_workspace_bytes()  */
} lbm_status;

/* Node classes returned by lbm_get_geometry(). */
enum {
  LBM_CLS_SOLID = 0,     /* solid, no fluid lattice neighbour               */
  LBM_CLS_SOLID_BND = 1, /* solid with a fluid neighbour (Eqs. 34-35 act)   */
  LBM_CLS_FLUID = 2,     /* fluid, no solid neighbour                       */
  LBM_CLS_FLUID_BND = 3  /* fluid with a solid neighbour (wetting acts)     */
};

/* Population storage (chosen at lbm_init_geometry). */
enum {
  LBM_STORAGE_FP32 = 0, /* f^r, f^b as float32                              */
  LBM_STORAGE_FP16 = 1, /* f''_i / w_i - rho0 in fp16 (f''_i = f^r + f^b
                           after recolouring); the colour split (q, v) and
                           all arithmetic stay float32                      */
  LBM_STORAGE_BF16 = 2  /* the same offsets in bfloat16                     */
};

/* Reduction kinds of lbm_reduce(). */
enum {
  LBM_MASS_R = 0,    /* sum over fluid nodes of sum_i f^r_i (stored state)  */
  LBM_MASS_B = 1,    /* the same for f^b                                    */
  LBM_SW_COUNT = 2,  /* S_w: fraction of fluid nodes with phi < 0 (Sec.IV.B)*/
  LBM_SW_SMOOTH = 3, /* mean over fluid nodes of (1 - phi)/2                */
  LBM_DP = 4,        /* mean rho/3 (Eq. 23) on the inlet plane minus the
                        same on the outlet plane of the flow axis           */
  LBM_CA_R = 5,      /* rho0 nu^r <u_a>_{phi>0} / gamma (not in the paper)  */
  LBM_CA_B = 6       /* rho0 nu^b <u_a>_{phi<0} / gamma (not in the paper)  */
};

typedef struct {
  double tau_r, tau_b; /* relaxation times, > 1/2; nu^s = (tau^s-1/2)/3 (Eq.13)*/
  double gamma;        /* interfacial tension (Eq. 5)                        */
  double beta;         /* recolouring segregation parameter, [0,1] (Eq. 20) */
  double rho0;         /* reference density of the equilibrium (Eq. A.4)    */
  double theta_deg;    /* contact angle, degrees, measured through fluid b  */
  int wetting;         /* 0 none, 1 Scheme-I (Leclaire), 2 Scheme-II (Akai) */
  int zou_he;          /* 1: Zou-He inlet (coordinate 0) and outlet (last
                          coordinate) on flow_axis, which must not be
                          periodic (Type-I; or the ends of a Type-II run)   */
  int flow_axis;       /* 0 = x, 1 = y, 2 = z                               */
  double rho_in, rho_out; /* Zou-He densities (Eqs. B.1, B.9)               */
  double zeta_r;       /* injected red fraction zeta^r in [0,1]; zeta^b =
                          1 - zeta^r; the inlet phase field is zeta^r -
                          zeta^b (Sec. II.D.1)                              */
  double g[3];         /* body acceleration; force density rho*g (Eq. 36)  */
  int collision;       /* 0: Eq. 2 with one rate S_nu for every
                          non-conserved moment (single-rate reading);
                          1: MRT, Eq. 2 with the rates of Eq. 4: S_e =
                          S_eps = S_pi = S_nu (Eq. 15), S_q = S_m =
                          8 (2 - S_nu) / (8 - S_nu) (Eq. 16). MRT is D3Q19
                          only (Appendix A); D2Q9 gives LBM_ERR_ARG       */
} lbm_params;

/* Device bytes one domain needs (populations A/B, phase field, normals,
 * classes, wall normals, lists, macros, reduction scratch). solid_host may
 * be NULL (the bound then assumes every node fluid). Returns 0 on a bad
 * argument. */
size_t lbm_workspace_bytes(int lattice, int nx, int ny, int nz,
                           const uint8_t *solid_host, int storage);

/* Create a domain. lattice = 9 (D2Q9, nz must be 1) or 19 (D3Q19).
 * solid_host: N bytes, nonzero = solid (host memory, copied).
 * periodic_mask: bit a set = axis a periodic; a non-periodic face that is
 * not a Zou-He plane acts as a halfway bounce-back wall without wetting.
 * Builds, on the device, the node classes, the three-pass smoothing of
 * Eq. (25) and the wall normal of Eq. (26) (gradient of the smoothed fluid
 * indicator by the Eq. 6 stencil, normalised; it points into the fluid).
 * dev_workspace: caller-owned device memory of ws_bytes >=
 * lbm_workspace_bytes(), 256-byte aligned, kept until lbm_destroy(). */
lbm_status lbm_init_geometry(lbm_handle *out, int lattice, int nx, int ny,
                             int nz, const uint8_t *solid_host,
                             unsigned periodic_mask, int storage,
                             void *dev_workspace, size_t ws_bytes,
                             void *stream);

/* The two calls above with a chosen tile shape (a memory-layout choice;
 * the paper has no counterpart). The fluid nodes are
 * numbered tile by tile, tiles of tile[0] x tile[1] x tile[2] nodes (x, y,
 * z; host array of 3 ints). NULL gives the default the calls above use:
 * 32 x 8 x 8 (D3Q19), 64 x 32 x 1 (D2Q9). Each extent a power of two,
 * tile[0] from 32 to 1024, at most 16384 nodes, tile[2] = 1 for D2Q9;
 * otherwise the size call returns 0 and the init call LBM_ERR_ARG. A
 * workspace must be sized with the same tile shape it is built with. The
 * shape sets only where each node's values sit in memory (so how well the
 * step's neighbour reads share cache lines): every per-node result
 * (lbm_macros, lbm_get_populations) is the same bit for bit for every
 * shape; sums over nodes (lbm_reduce) may differ in rounding order, and a
 * state saved by lbm_save_state loads only into a domain of the same
 * shape. */
size_t lbm_workspace_bytes_tiled(int lattice, int nx, int ny, int nz,
                                 const uint8_t *solid_host, int storage,
                                 const int *tile);
lbm_status lbm_init_geometry_tiled(lbm_handle *out, int lattice, int nx,
                                   int ny, int nz, const uint8_t *solid_host,
                                   unsigned periodic_mask, int storage,
                                   const int *tile, void *dev_workspace,
                                   size_t ws_bytes, void *stream);

/* Set the parameters (host struct, copied). Validates them. */
lbm_status lbm_set_params(lbm_handle h, const lbm_params *p);

/* Fluid at rest: f^s_i = w_i rho^s with rho^r = rho0 (1 + phi0)/2,
 * rho^b = rho0 (1 - phi0)/2. phi0_dev: device float32 [N] (solid entries
 * ignored). Needs lbm_set_params() first. */
lbm_status lbm_init_state(lbm_handle h, const float *phi0_dev, void *stream);

/* Advance nsteps time steps (Eq. 1), asynchronously on `stream`. All
 * steps but the last are replayed two at a time from a CUDA graph that the
 * handle records on its own stream at first use (and again after
 * lbm_set_params); the last step, which also stores the macros, and an odd
 * one are plain launches. The results equal those of nsteps single steps
 * bit for bit. If the graph cannot be recorded the steps are launched one
 * by one. */
lbm_status lbm_step(lbm_handle h, int nsteps, void *stream);

/* Kernels of a step, in launch order, as lbm_step_timed() reports them. */
#define LBM_N_PASSES 7
/* Profiling form of lbm_step(): the same nsteps steps, with CUDA events
 * recorded on `stream` around each kernel of a step: [0] streaming and the
 * phase field (Eq. 1, Eqs. 7-9); [1] App. B on the Zou-He planes; [2]
 * Eq. (34); [3] colour gradient and wetting (Eqs. 6, 27-33); [4] Eq. (35);
 * [5] curvature (Eq. 12); [6] force, collision and recolouring (Eqs. 5, 2,
 * 20-21).
 * Adds the elapsed milliseconds of each, summed over the steps, to
 * pass_ms[0..LBM_N_PASSES-1] (host array) and synchronises the stream; a
 * kernel that does not run adds about 0. The results equal lbm_step()'s. */
lbm_status lbm_step_timed(lbm_handle h, int nsteps, void *stream,
                          double *pass_ms);

/* Fields of the most recent step, each into caller device buffers (any may
 * be NULL): rho [N] (rho^r + rho^b after streaming and Zou-He), phi [N]
 * (with the inlet/outlet values and, at solid-boundary nodes, Eq. 34), u
 * [3][N] (Eq. 22). Solid nodes hold 0 (phi: Eq. 34 value at solid-boundary
 * nodes). Before the first step: the initial state, u = 0. */
lbm_status lbm_macros(lbm_handle h, float *rho, float *phi, float *u,
                      void *stream);

/* One reduction (kind LBM_MASS_R ... LBM_CA_B), accumulated in FP64,
 * written to *out_host; synchronises the stream. LBM_ERR_NONFINITE if the
 * sum is not finite. */
lbm_status lbm_reduce(lbm_handle h, int kind, double *out_host, void *stream);

/* lbm_reduce() without the wait (the same diagnostics; how they reach the
 * host has no counterpart in the paper), for a quantity read back every step
 * while the GPU runs on: enqueues the same FP64 reduction on `stream` and
 * the copy of its four raw sums to raw4_host[0..3] (host memory owned by
 * the caller; page-locked for the copy to overlap the following work), and
 * returns. Once the stream has passed that point, lbm_reduce_value() turns
 * the raw sums into the quantity lbm_reduce() would have returned. The
 * reduction's device scratch belongs to the handle, so reductions of one
 * handle must stay on one stream. */
lbm_status lbm_reduce_async(lbm_handle h, int kind, double *raw4_host,
                            void *stream);
/* The quantity of `kind` from four raw sums of lbm_reduce_async() (host
 * arithmetic only). LBM_ERR_NONFINITE if it is not finite. */
lbm_status lbm_reduce_value(lbm_handle h, int kind, const double *raw4_host,
                            double *out_host);

/* The stored (post-recolouring) populations as float32 [2][Q][N] in the
 * caller's device buffer (solid nodes 0), and back. */
lbm_status lbm_get_populations(lbm_handle h, float *dst_dev, void *stream);
lbm_status lbm_set_populations(lbm_handle h, const float *src_dev,
                               void *stream);

/* Error word of the bounds-checked build (the library compiled with
 * LBM_BOUNDS_CHECK, liblbmgb_check.so; no counterpart in the paper): bit 0
 * a pull source, bit 1 a stencil neighbour, bit 2 a Zou-He plane index,
 * bit 3 a solid-boundary link was out of range (the access was redirected
 * to index 0). Always 0 in the normal build. Synchronises the stream. */
lbm_status lbm_debug_flags(lbm_handle h, unsigned *out_host, void *stream);

/* Replace the injected fluid (Sec. II.D.1, Eqs. 37-38): at every fluid node
 * of the inlet plane (coordinate 0 of flow_axis) the stored populations of
 * the other colour are added to colour `colour` (0 = r, 1 = b) and set to
 * zero, f^s_i += f^sbar_i, f^sbar_i = 0, so those nodes hold pure fluid s.
 * For sequential injection of different fluids (e.g. forced imbibition
 * after drainage); set the matching zeta_r with lbm_set_params() as well.
 * Needs a state and zou_he = 1 (LBM_ERR_STATE), colour 0 or 1
 * (LBM_ERR_ARG). Asynchronous. */
lbm_status lbm_swap_inlet(lbm_handle h, int colour, void *stream);

/* Node classes (uint8 [N], LBM_CLS_*) and wall normals (float32 [3][N],
 * zero away from fluid-boundary nodes) into caller device buffers. */
lbm_status lbm_get_geometry(lbm_handle h, uint8_t *cls_dev, float *nw_dev,
                            void *stream);

/* Counts fixed at lbm_init_geometry: nodes, fluid nodes, solid-boundary
 * nodes and fluid-boundary nodes. */
lbm_status lbm_counts(lbm_handle h, int64_t *n_nodes, int64_t *n_fluid,
                      int64_t *n_solid_bnd, int64_t *n_fluid_bnd);

/* Largest node count lbm_colour_mass_noalloc accepts. */
#define LBM_NOALLOC_MAX_NODES ((int64_t)1 << 31)

/* Colour masses of a dense population array, for callers that cannot
 * allocate device memory (no counterpart in the paper: it is the
 * LBM_MASS_R / LBM_MASS_B reduction of lbm_reduce() without a workspace).
 * Some callers run under a device-memory budget that another framework
 * reserved up front, or under a policy that forbids allocation after
 * start-up; they cannot provide a handle's workspace. This call needs none:
 * pops_dev is the caller's device float32 array [2][Q][n_nodes] (as
 * lbm_get_populations() writes it; solid entries zero), mass_host[0..1]
 * receives the red and blue masses, summed in FP64. It allocates nothing:
 * its scratch is a fixed array of the library's own in device memory
 * (about 16 KB, present on every GPU that loads the library until exit).
 * The first call on a device looks up that array's address with the
 * device current. Every call shares the array; calls that overlap on the
 * GPU race on it. Synchronises the stream.
 * LBM_ERR_ARG for lattice not 9/19, null pointers, n_nodes outside
 * [1, LBM_NOALLOC_MAX_NODES], or a pops_dev that is not device (or
 * managed) memory of the current device; nothing is enqueued then. */
lbm_status lbm_colour_mass_noalloc(int lattice, int64_t n_nodes,
                                   const float *pops_dev, double *mass_host,
                                   void *stream);

/* Bytes of one exact copy of the stored state (the f''_i planes in the
 * storage type and the per-node colour split (q, v)): for checkpoints. */
size_t lbm_state_bytes(lbm_handle h);

/* Copy the current state to / from caller device memory of
 * lbm_state_bytes() bytes (device to device, asynchronous on `stream`).
 * A loaded state continues exactly as the saved one would have. */
lbm_status lbm_save_state(lbm_handle h, void *dst_dev, void *stream);
lbm_status lbm_load_state(lbm_handle h, const void *src_dev, void *stream);

/* Message of the last failed call on this handle ("" if none). */
const char *lbm_last_error(lbm_handle h);

/* Release the handle (host memory only; the workspace stays the caller's). */
void lbm_destroy(lbm_handle h);

/* ------------------------------------------------------------------------
 * Batches: many independent domains ("cases", e.g. a sweep of sessile drops
 * over contact angles and box sizes) stepped together. Each case is a
 * handle with its own geometry, parameters and state, all of one lattice
 * and one storage type. The paper runs one domain at a time; the batch
 * changes the scheduling only. Every case's results are those of lbm_step()
 * on that handle, bit for bit. Step a batch's cases only through the batch
 * while it exists, or expect the batch to re-read them (see lbm_batch_step).
 * The handles must outlive the batch.
 * ------------------------------------------------------------------------ */
typedef struct lbm_batch_s *lbm_batch;

/* Device workspace (bytes) of a batch of ncases cases: the case table, a
 * control block and the work plans, a few hundred bytes per case. 0 if
 * ncases < 1. */
size_t lbm_batch_workspace_bytes(int ncases);

/* Batch of ncases distinct handles (host array, copied), each with
 * parameters and state set, all with the same lattice and storage.
 * dev_workspace: caller-owned device memory of ws_bytes >=
 * lbm_batch_workspace_bytes(ncases), 256-byte aligned, kept until
 * lbm_batch_destroy(). Synchronises `stream`. Starts in mode 0 with 256
 * threads per block. */
lbm_status lbm_batch_create(lbm_batch *out, const lbm_handle *cases,
                            int ncases, void *dev_workspace, size_t ws_bytes,
                            void *stream);

/* Scheduling of lbm_batch_step():
 *   mode 0: one kernel launch per pass of a step, covering every case;
 *   mode 1: one persistent launch for all passes of all steps of a call.
 *     Blocks take (step, pass, case, chunk) work items in step-and-pass
 *     order, and each item waits until its case has finished the previous
 *     pass (a per-case completion count), so cases advance independently.
 *     Each wait is bounded by time (2 s); when one runs out, every block
 *     stops and lbm_batch_status() reports LBM_ERR_TIMEOUT.
 * threads: 128 or 256 threads per block. chunk (mode 1): blocks' worth of
 * nodes per work item, 1..64. Drops the recorded graphs; synchronises
 * `stream`. The results do not depend on the configuration. */
lbm_status lbm_batch_set_config(lbm_batch b, int mode, int threads, int chunk,
                                void *stream);

/* Advance every case by nsteps steps, asynchronously on `stream`. The
 * kernels of one call are recorded once per (nsteps, configuration) into a
 * CUDA graph on a stream the batch owns, and the graph is launched on
 * `stream`. The last step stores each case's macros, as lbm_step() does.
 * If a case was changed or stepped outside the batch since the last call,
 * the case table is written again first (synchronising `stream`). */
lbm_status lbm_batch_step(lbm_batch b, int nsteps, void *stream);

/* Synchronise `stream` and report whether a bounded wait of a mode-1
 * launch ran out since the last call: LBM_ERR_TIMEOUT (the flag is then
 * cleared; the cases' states are partly stepped and must be reset) or
 * LBM_OK. While the flag is set, further mode-1 launches stop at once. */
lbm_status lbm_batch_status(lbm_batch b, void *stream);

/* Health check of the bounded wait: runs the persistent kernel's wait on a
 * count that nothing raises, with a limit of limit_ms (0 < limit_ms <=
 * 10000). Returns LBM_OK when the wait gave up and set the error flag as
 * designed (the flag is cleared again), and the elapsed device time in
 * *waited_ms (may be NULL); LBM_ERR_STATE if it did not give up.
 * Synchronises `stream`. */
lbm_status lbm_batch_check_wait(lbm_batch b, double limit_ms,
                                double *waited_ms, void *stream);

/* Message of the last failed call on this batch ("" if none). */
const char *lbm_batch_last_error(lbm_batch b);

/* Release the batch (host side; the workspace stays the caller's). */
void lbm_batch_destroy(lbm_batch b);

/* ------------------------------------------------------------------------
 * Adjoint: the hand-written reverse of one time step, for the gradient of
 * J = LBM_SW_SMOOTH after T steps (the mean over fluid nodes of (1 - phi)/2,
 * phi from the last step's streamed populations) with respect to the
 * contact angle theta (radians) and the body acceleration g (Eq. 36).
 * The state of a fluid node is (f''_i, r = rho^r/rho, v) with the red part
 * of population i equal to r f''_i + w_i e_i.v (Eqs. 20-21); the adjoint
 * state has the same shape. Scope: float32 storage, the single-rate
 * collision (collision = 0), no wetting or Scheme-II (Eqs. 32-33), no
 * Zou-He ends (periodic axes or bounce-back walls);
 * lbm_adj_create() rejects anything else with LBM_ERR_ARG. All arithmetic
 * is float32; the parameter gradients accumulate in float64.
 *
 * Use (T steps, states x_0 .. x_T, with x_{t+1} = step(x_t)):
 *   load x_{T-1} into the handle (lbm_load_state), lbm_adj_seed_sw();
 *   for t = T-2 down to 0: load x_t, lbm_adj_step();
 *   lbm_adj_gradients().
 * The states can come from checkpoints and recomputation (the binding's
 * SwGradient keeps every K-th state and recomputes the rest, K ~ sqrt(T)).
 * Each call recomputes the forward fields of its step on the handle, which
 * changes the handle's per-step fields (macros) but not its state.
 * ------------------------------------------------------------------------ */
typedef struct lbm_adj_s *lbm_adj;

/* Device workspace (bytes) of the adjoint of handle h: about
 * (3Q + 15) x 4 bytes per fluid node. */
size_t lbm_adj_workspace_bytes(lbm_handle h);

/* Adjoint of handle h (which must have its parameters set), in caller
 * device memory of ws_bytes >= lbm_adj_workspace_bytes(h), 256-byte
 * aligned. The handle must outlive it. */
lbm_status lbm_adj_create(lbm_adj *out, lbm_handle h, void *dev_workspace,
                          size_t ws_bytes);

/* Start the reverse sweep: the handle holds x_{T-1}. Sets the adjoint state
 * to dJ/dx_{T-1} and zeroes the parameter gradients. Asynchronous. */
lbm_status lbm_adj_seed_sw(lbm_adj a, void *stream);

/* Reverse one step: the handle holds x_t, the adjoint dJ/dx_{t+1}; on
 * return (asynchronously) the adjoint is dJ/dx_t and the step's parts of
 * dJ/dtheta and dJ/dg are added. */
lbm_status lbm_adj_step(lbm_adj a, void *stream);

/* dJ/dtheta (per radian) and dJ/dg_x, dJ/dg_y, dJ/dg_z into out4 (host);
 * synchronises `stream`. */
lbm_status lbm_adj_gradients(lbm_adj a, double *out4, void *stream);

/* The current adjoint state: lt_dev float32 [Q][NFp] (fluid nodes in the
 * library's internal order) and ls_dev float32 [NF][4] (lambda r,
 * lambda v). For tests. */
lbm_status lbm_adj_get_lambda(lbm_adj a, float *lt_dev, float *ls_dev,
                              void *stream);

/* Regularised linearisation of Scheme-II: where sin(theta') (theta' the
 * angle between n_c and n_w) is below freeze_sin, the derivative of the
 * result's direction around n_w, which grows as 1/sin(theta'), is dropped
 * and only its theta dependence kept. Over long runs the exact derivative
 * of the discrete step grows without bound through such nodes; the default
 * 0.05 keeps the gradient finite and close to finite differences of the
 * forward run. 0 gives the exact derivative. Range [0, 1]. */
lbm_status lbm_adj_set_freeze(lbm_adj a, double freeze_sin);

/* Regularised linearisation of the interface normal n_c = C/|C| (Eq. 11):
 * where |C| < c_min the direction of n_c is held constant (its derivative
 * grows as 1/|C| in the tails of the interface). The default 1e-3 keeps
 * long-run gradients finite (with freeze_sin 0.05); 0 gives the exact
 * derivative. Range [0, 10]. */
lbm_status lbm_adj_set_cmin(lbm_adj a, double c_min);

/* Message of the last failed call on this adjoint ("" if none). */
const char *lbm_adj_last_error(lbm_adj a);

/* Release the adjoint (host side). */
void lbm_adj_destroy(lbm_adj a);

#ifdef __cplusplus
}
#endif

#endif /* LBMGB_H */
