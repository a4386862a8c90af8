/*
 * numa.h -- C ABI of the GB300-native CG spectral-element RHS / Runge-Kutta
 * hot path of the NUMA dynamical core (Mueller et al., "Strong scaling for
 * numerical weather prediction at petascale with the atmospheric model
 * NUMA", Sec. 2 and the main loop of code example 1 in Sec. 7).
 *
 * Ownership model
 *   - The library allocates no device memory.  The caller provides one device
 *     workspace of numa_get_mesh_info().workspace_bytes bytes and a CUDA
 *     stream (numa_bind); the library carves geometry, state and scratch out
 *     of it and enqueues every copy and kernel on that stream.
 *   - A context owns host-side mesh metadata only; numa_destroy frees it and
 *     never touches caller memory.
 *   - Pointers documented as "device" must be device-accessible for the bound
 *     device; "host" pointers are read or written before the call returns
 *     unless stated otherwise.
 *
 * Devices and threads
 *   A context works on the device that is current when numa_bind is called;
 *   calls on it must be made with that device current.  Contexts on
 *   different devices may be used from one process.  A context is not
 *   thread-safe: calls on one context must not overlap.  Calls on different
 *   contexts may come from different threads.
 *
 * Errors
 *   Every call returns an int status: NUMA_OK (0) or a negative NUMA_E* code.
 *   Nothing aborts, traps or exits.  numa_last_error() returns a message owned
 *   by the context (valid until the next call on it).
 *
 * Data layout (all calls)
 *   State q and tendency R are double[5][Ng] (structure of arrays), variable
 *   order (rho', U_x, U_y, U_z, Theta'): density perturbation, momentum
 *   U = rho u, and rho*theta minus the reference (rho theta)_0 (Eq. 1 in
 *   perturbation form about a hydrostatic reference state).
 *   Box meshes number global nodes structurally:
 *       g = ix + nx * (iy + ny * iz),  nx = nex*N + 1 (walls) or nex*N
 *       (periodic along x), likewise ny, nz; node (ix, iy, iz) lies at the
 *       LGL position of lattice index ix along x, etc.
 *   Shell meshes number global nodes internally; numa_get_coords() returns
 *   their coordinates.
 */
#ifndef NUMA_H
#define NUMA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NUMA_OK 0
#define NUMA_EINVAL (-1)     /* bad argument or configuration */
#define NUMA_ENOMEM (-2)     /* host allocation failed or workspace too small */
#define NUMA_ECUDA (-3)      /* a CUDA runtime call failed */
#define NUMA_ENONFINITE (-4) /* the state became non-finite during a step */
#define NUMA_ETIMEOUT (-5)   /* a bounded device wait gave up */
#define NUMA_EBUDGET (-6)    /* a request does not fit the HBM budget */
#define NUMA_ESTATE (-7)     /* call made in the wrong order (e.g. before numa_bind) */

enum numa_mesh_kind { NUMA_MESH_BOX = 0, NUMA_MESH_SHELL = 1 };
enum numa_ref_kind { NUMA_REF_ISENTROPIC = 0, NUMA_REF_ISOTHERMAL = 1 };
enum numa_precision {
  NUMA_FP64 = 0,      /* every step in FP64 */
  NUMA_FP32_MIXED = 1, /* fluxes, metric terms and D contractions in FP32;
                          state, EOS reference subtraction, DSS, inverse mass
                          and the RK combination in FP64 */
  NUMA_FP64_PAIRS = 2  /* FP64-accurate element kernel computed on the FP32
                          units: every value is an unevaluated sum of two
                          floats (about 48 significant bits), products by
                          error-free FMA splits, sums by TwoSum; state,
                          primitives/EOS, DSS, inverse mass and RK in FP64 */
};
enum numa_ic_kind { NUMA_IC_REST = 0, NUMA_IC_BUBBLE = 1, NUMA_IC_UNIFORM = 2, NUMA_IC_JETWAVE = 3 };

/* Mesh, physics and precision.  Sec. 2.1 (order N, Lobatto points), Sec. 3
 * (the box and the cubed-sphere shell test cases), Sec. 4 (columns of
 * radial layers). */
/* How the element kernel applies the metric terms of Eq. 5.
 * AUTO: when every element's map to the reference cube is affine (a box with
 *   warp = 0), the metric terms are constant over each element and the chain
 *   rule commutes with the derivative, sum_c (dxi_d/dx_c) dF_c/dxi_d =
 *   d/dxi_d (sum_c (dxi_d/dx_c) F_c); the kernel then differentiates the 15
 *   contravariant fluxes instead of the 13 Cartesian flux components along
 *   all three directions (15 contractions per node instead of 39, the same
 *   operator up to rounding) and reads the metric terms once per element.
 *   Any other mesh takes the per-node form.
 * NODAL: always the per-node form of Eq. 5 (metric terms read at every node,
 *   applied after the derivative). */
typedef enum { NUMA_METRIC_AUTO = 0, NUMA_METRIC_NODAL = 1 } numa_metric_form;

/* Storage of the node data (Sec. 6's comparison of CG and DG storage).
 * CG: one value per global node; element nodes that coincide share it and
 *   the element kernel gathers through the element-to-global map.
 * DG: one value per element node (Ng = Nl in numa_mesh_info): every element
 *   keeps its own copy of its nodes.  DSS still sums over all element nodes
 *   at the same point, in the same ascending order as CG storage does, so
 *   every copy holds the value CG storage holds at that point, bitwise; the
 *   state arrays, coordinates and get/set_state use the Nl storage nodes in
 *   element order.  The serving calls (numa_sched_submit) take CG only. */
typedef enum { NUMA_STORAGE_CG = 0, NUMA_STORAGE_DG = 1 } numa_storage;

typedef struct {
  int mesh_kind;           /* numa_mesh_kind */
  int N;                   /* polynomial order, 1..8 (N+1 LGL points per direction) */
  int nex, ney, nez;       /* box: elements along x, y, z */
  double Lx, Ly, Lz;       /* box: extents in m, origin at (0,0,0) */
  int periodic[3];         /* box: 1 = periodic along that axis, 0 = no-flux walls */
  double warp;             /* box: amplitude of a smooth interior warp that keeps every
                              face in place, as a fraction of the extent (0 = affine):
                              x += warp Lx sin(pi X) sin(pi Y) sin(pi Z),
                              y += warp Ly sin(2 pi X) sin(pi Y) sin(pi Z),
                              z += warp Lz sin(pi X) sin(2 pi Y) sin(pi Z), X = x/Lx ... */
  int npanel, nlayer;      /* shell: columns per cube-panel edge, radial layers */
  double r_inner, r_outer; /* shell: planet radius a and lid radius, m */
  double Rd, cp, cv, P00;  /* gas constant, heat capacities, reference pressure */
  double g;                /* box: gravity; shell: surface gravity g0, g(r) = g0 (a/r)^2 */
  double Omega;            /* shell: rotation rate about +z, 1/s */
  int ref_kind;            /* numa_ref_kind of the hydrostatic reference state */
  double theta0, T0;       /* isentropic potential temperature / isothermal temperature */
  int precision;           /* numa_precision */
  int metric_form;         /* numa_metric_form: how the element kernel applies the metric terms */
  int storage;             /* numa_storage: CG (0, default) or DG storage of the node data */
} numa_config;

typedef struct {
  long long Ne, Nl, Ng;   /* elements, element-local nodes Ne (N+1)^3, storage nodes
                             (global nodes for CG storage, Nl for DG storage) */
  size_t workspace_bytes; /* device bytes numa_bind needs */
  int N;
  long long dss_entries;  /* element residuals the DSS reads per stage: Nl for CG storage;
                             for DG storage every copy reads all residuals at its point,
                             the sum over global nodes of (element nodes there)^2 */
} numa_mesh_info;

typedef struct numa_ctx numa_ctx;

/* Build the host mesh: LGL nodes, D, coordinates, isoparametric metric terms
 * and Jacobian (Eq. 5), Jw, element-to-global map and its inverse, the
 * diagonal mass matrix M = sum_e Jw (Eq. 4) and the hydrostatic reference
 * state.  *out receives a new context or NULL on error. */
int numa_create(const numa_config* cfg, numa_ctx** out);

/* Sizes and the workspace requirement of a context. */
int numa_get_mesh_info(const numa_ctx* ctx, numa_mesh_info* info);

/* Bind a caller-owned device workspace (>= workspace_bytes, 256-byte aligned)
 * and a cudaStream_t (passed as void*; NULL = legacy default stream).  Uploads
 * the geometry into the workspace on that stream and waits for it.  May be
 * called again to move the context to another workspace or stream. */
int numa_bind(numa_ctx* ctx, void* dev_workspace, size_t bytes, void* stream);

/* Write an initial state into the context's state (Sec. 3 test cases).
 * params: REST -; BUBBLE {A, r_c, x_c, y_c, z_c} (cosine potential-
 * temperature bubble, pressure unperturbed); UNIFORM {u0, v0, w0};
 * JETWAVE {U_jet, amp, radius/a, lambda_c, phi_c} (zonal jet
 * U_jet sin^2(2 phi) plus a Gaussian zonal-wind bump). */
int numa_init_state(numa_ctx* ctx, int ic_kind, const double* params, int nparams);

/* Copy the context's state from / to a caller buffer double[5][Ng];
 * on_device = 1 for a device pointer, 0 for host memory (pinned memory
 * makes the copy asynchronous-capable; the call waits for completion).
 * From a device pointer, numa_set_state is enqueued on the bound stream
 * and returns without waiting; it copies the state and forms its
 * primitive fields in one pass (the next step's first element kernel
 * needs them). */
int numa_set_state(numa_ctx* ctx, const double* q, int on_device);
int numa_get_state(numa_ctx* ctx, double* q, int on_device);

/* R = dq/dt of Eq. 4 at state q: element volume terms, direct stiffness
 * summation, inverse mass matrix, sources and the no-normal-flow wall
 * condition.  q_dev, r_dev: device double[5][Ng] (may not alias).  Enqueued
 * on the bound stream; returns without waiting. */
int numa_rhs(numa_ctx* ctx, const double* q_dev, double* r_dev);

/* Size of the library-owned scratch used by numa_rhs_static_scratch. */
#define NUMA_STATIC_SCRATCH_BYTES (16u << 20)

/* The paper has no counterpart to this call.  It is for callers that cannot
 * allocate device memory: real-time loops that forbid allocation once they
 * run, and plug-ins whose host application owns all device memory and hands
 * them only input and output buffers.  Same result as numa_rhs, bit for bit,
 * but its scratch -- the primitive fields and the element residuals -- lives
 * in a fixed 16 MiB device array inside the library
 * (NUMA_STATIC_SCRATCH_BYTES) instead of the bound workspace, and nothing is
 * allocated: no cudaMalloc, no cudaFree, no allocating library call.
 * Scratch per global node: 72 bytes (FP64), 32 (FP32-mixed), 64 (pairs); per
 * element node: 40 (FP64, pairs) or 20 (FP32-mixed).  At N=4 the largest
 * cubic boxes that fit are 11^3 elements (FP64), 12^3 (pairs) and 15^3
 * (FP32-mixed);
 * larger meshes return NUMA_EINVAL with the bytes needed in
 * numa_last_error.  The first call in each CUDA context (normally one per
 * device) looks up the array's device address and caches it; make that first
 * call before any stream capture.  Every call shares the one array and leaves
 * its contents behind: calls whose work overlaps on the GPU (other streams,
 * other contexts) race on it.  q_dev, r_dev: device double[5][Ng] (may not
 * alias), enqueued on the bound stream. */
int numa_rhs_static_scratch(numa_ctx* ctx, const double* q_dev, double* r_dev);

/* Advance the context's state by one step of size dt of the selected
 * integrator (numa_set_time_scheme; SSP-RK3 by default; Sec. 2.2 explicit
 * stages: per stage create_rhs, DSS with the inverse mass matrix, update q).
 * Enqueued on the bound stream; returns without waiting, except that the
 * first NUMA_LEAPFROG_IMEX step with a new dt factors the column matrices on
 * the host and waits for their upload. */
int numa_rk_step(numa_ctx* ctx, double dt);

/* nsteps steps of the selected integrator (one captured CUDA graph per step,
 * replayed), then
 * waits for the stream and returns NUMA_ENONFINITE if any stage produced a
 * non-finite value. */
int numa_run(numa_ctx* ctx, double dt, int nsteps);

/* Time integrators of numa_rk_step / numa_run (Sec. 2.2).
 * SSP3: three-stage, third-order strong-stability-preserving RK (Shu-Osher):
 *   q1 = q + dt R(q); q2 = 3/4 q + 1/4 (q1 + dt R(q1));
 *   q_new = 1/3 q + 2/3 (q2 + dt R(q2)).
 * LS54: five-stage, fourth-order low-storage ("2N") RK of Carpenter and
 *   Kennedy: with dq = 0, for i = 1..5: dq <- A_i dq + dt R(q), q <- q + B_i dq.
 *   The paper's integrator has five stages and third order but is not
 *   specified further; this scheme has its stage count and exceeds its order.
 * LEAPFROG_IMEX: the 1D-IMEX scheme of Sec. 2.2 for meshes whose vertical
 *   resolution is much finer than the horizontal one: an explicit leapfrog
 *   step, then an implicit correction along each vertical column.  With L the
 *   linear vertical operator of Eq. 1 about the reference state (for rho',
 *   the vertical momentum W and Theta': (L q)_rho = -dz W,
 *   (L q)_W = -dz(c2 Theta') - g rho' (zero at the bottom and top walls),
 *   (L q)_Theta = -dz(theta0 W), c2 = gamma p0 / Theta0, theta0 = Theta0 / rho0,
 *   dz the CG derivative along the column), one step is
 *     q* = qbar^{n-1} + 2 dt R(q^n),
 *     (I - dt L) q^{n+1} = q* - dt L (2 q^n - qbar^{n-1}),
 *     qbar^n = q^n + nu (qbar^{n-1} - 2 q^n + q^{n+1})   (Robert-Asselin),
 *   i.e. the trapezoidal rule over [t^{n-1}, t^{n+1}] for L and leapfrog for
 *   the rest.  The first step after numa_set_state, numa_init_state,
 *   numa_bind or a change of scheme starts from q^0 alone:
 *     (I - dt/2 L) q^1 = q^0 + dt R(q^0) - dt/2 L q^0,  qbar^0 = q^0.
 *   Each column's system is reduced to a banded system in W and solved with
 *   LU factors (partial pivoting) made on the host for each new dt.
 *   Columns: the z-lines of a box with walls at the bottom and top and warp
 *   0, or the radial lines of the cubed-sphere shell, where W = U . r_hat,
 *   dz is the radial derivative, the divergence terms are
 *   (L q)_rho = -(dr W + 2 W / r) and (L q)_Theta = -(dr(theta0 W) + 2 theta0 W / r),
 *   g = g0 (a / r)^2, and the correction moves U along r_hat only.
 *   Needs FP64 or FP64-pairs precision, CG storage and a reference state
 *   that depends on the height only. */
typedef enum { NUMA_RK_SSP3 = 0, NUMA_RK_LS54 = 1, NUMA_LEAPFROG_IMEX = 2 } numa_rk_scheme;

/* Select the integrator (default NUMA_RK_SSP3).  NUMA_EINVAL for another
 * value, or for NUMA_LEAPFROG_IMEX on a configuration it does not support
 * (numa_last_error says why).  Takes effect at the next step. */
int numa_set_time_scheme(numa_ctx* ctx, int scheme);

/* Slab pipeline of the explicit RK step (SSP-RK3 and LS54) on boxes with CG
 * storage and walls at the bottom and top.  The elements are cut into
 * `nslabs` slabs along z and the global nodes into the matching slabs; within
 * a step the DSS/update of node slab k runs on a second, library-owned stream
 * beside the element kernel of slab k + 1 (the element kernel is bound by
 * memory or FP64 work, the update by FP64 work and latency), ordered by
 * events so that every node is computed exactly as without slabs: results are
 * identical bit for bit.  nslabs = 0 (the default) chooses 3 slabs for
 * FP32-mixed meshes of 2^18 or more global nodes (in FP64 and the pairs mode
 * both kernels compete for the same pipes and the pipeline measured no gain,
 * so it stays off there); 1 turns the pipeline off; at most 16.  Where a
 * mesh cannot be cut (shells, DG storage, periodic in z, slabs thinner than
 * two node planes, planes of fewer than 128 nodes) one slab is used.  *used
 * (may be NULL) receives the slabs in effect (before numa_bind: those that
 * numa_bind will use).  numa_time_kernels always runs unpipelined.  The
 * pipeline creates one CUDA stream and events per context at numa_bind (no
 * device memory).  NUMA_EINVAL for nslabs outside [0, 16]. */
int numa_set_slabs(numa_ctx* ctx, int nslabs, int* used);

/* Robert-Asselin filter strength nu of NUMA_LEAPFROG_IMEX, 0 <= nu < 0.5
 * (default 0.05; 0 turns it off).  NUMA_EINVAL outside that range. */
int numa_set_robert_asselin(numa_ctx* ctx, double nu);

/* Boyd-Vandeven filter (Sec. 2.3), applied as in the time loop of Sec. 7:
 * after every `every`-th step of numa_run / numa_rk_step (the count restarts
 * at numa_set_filter, numa_set_state and numa_init_state), the state becomes
 *   q <- M^-1 DSS(Jw (F x F x F) q_e),
 * the tensor product over each element of the 1D modal filter
 * F = V diag(sigma) V^-1 (V_ik = P_k(xi_i), Legendre modes k = 0..N on the
 * Lobatto points), followed by direct stiffness summation of the
 * Jw-weighted element values and the inverse mass matrix.  sigma_k = 1 for
 * k < s; for s <= k <= N Vandeven's filter of order p in Boyd's erfc-log
 * form, 1/2 erfc(2 sqrt(p) chi O), O = theta - 1/2,
 * theta = (k - s)/(N - s), chi^2 = -log(1 - 4 O^2)/(4 O^2): 1 at k = s, 0 at
 * k = N; blended with the identity by the strength mu: 1 - mu (1 - sigma_k).
 * At wall nodes the wall-normal momentum keeps its value.  The filter
 * computes in FP64 (FP32 for the element part in the FP32-mixed form; the
 * state update stays FP64).
 * every >= 0 (0: never applied by run / rk_step), 0 <= s <= N+1 (N+1: no
 * mode damped), p > 0, 0 <= mu <= 1; otherwise NUMA_EINVAL.  May be called
 * before numa_bind; a bound context uploads the matrix and waits. */
int numa_set_filter(numa_ctx* ctx, int every, int s, double p, double mu);

/* Apply the filter once to the context's state, now (enqueued on the bound
 * stream).  NUMA_ESTATE before numa_set_filter or numa_bind. */
int numa_filter(numa_ctx* ctx);

/* Measurement helper: advance the state by nsteps steps of the selected
 * integrator with plain (non-graph) launches, bracketing every kernel with
 * CUDA events on the bound stream, then wait and return the summed device
 * time in ms of the element volume kernels (*ms_volume) and of the
 * DSS/update kernels (*ms_update), (stages per step) * nsteps launches each.
 * For NUMA_LEAPFROG_IMEX a step is one stage and *ms_update covers the DSS
 * launch and the column kernel (a pending start step is the first of the
 * nsteps). */
int numa_time_kernels(numa_ctx* ctx, double dt, int nsteps, double* ms_volume, double* ms_update);

/* Non-finite flag raised by any stage update since the last call; resets it.
 * Waits for the stream. *flag = 0 or 1. */
int numa_check_finite(numa_ctx* ctx, int* flag);

/* Measurement helper, not part of the method: the arithmetic throughput of
 * one unit on the current device, from one register-only kernel of `iters`
 * loop iterations over 8 CTAs of 256 threads per SM, timed with CUDA events
 * on `stream` (cudaStream_t as void*); waits for it.
 *   kind 0: FP64 FMA (8 independent chains per thread)
 *   kind 1: FP32 FMA (8 chains per thread)
 *   kind 2: FP64 mma.sync m8n8k4 (4 accumulators per warp)
 *   kind 3: TF32 mma.sync m16n8k8 with FP32 accumulation (4 per warp)
 *   kind 4: half the warps as kind 0, half as kind 2, sized to take equal
 *           time alone: a total near the sum of the two rates means the two
 *           FP64 paths run side by side
 * dev_out: device scratch of out_bytes >= SMs * 8 * 256 * (8 bytes for kinds
 * 0, 2 and 4; 4 for kinds 1 and 3), overwritten (one value per thread).
 * *ms: kernel time; *tflops: 2 * multiply-adds / time.  NUMA_EINVAL for a bad
 * kind, iters < 1 or a short buffer. */
int numa_probe_peak(int kind, int iters, void* dev_out, size_t out_bytes, void* stream, double* ms,
                    double* tflops);

/* ---- Serving: continuous batching of ensemble members ---------------------
 * Not in the paper: many independent forecasts (members of different mesh
 * sizes, orders, precisions and step counts) share one GPU.  Members advance
 * together, one SSP-RK3 step per numa_sched_step, through ragged kernels that
 * cover the elements and nodes of all admitted members; requests that arrive
 * while others run are admitted as soon as their workspace fits. */
typedef struct numa_sched numa_sched;

enum numa_req_status {
  NUMA_REQ_QUEUED = 0,   /* waiting for its mesh or for room in the arena */
  NUMA_REQ_RUNNING = 1,  /* admitted, advancing */
  NUMA_REQ_DONE = 2,     /* finished; fetch with numa_sched_result */
  NUMA_REQ_FAILED = 3,   /* setup failed or the state became non-finite */
  NUMA_REQ_CANCELLED = 4
};

/* Create a scheduler over a caller-owned device arena (256-byte aligned) used
 * for all member workspaces and the scheduler's own tables, the compute
 * stream (cudaStream_t as void*), and build_threads host threads that build
 * meshes in the background.  The library still allocates no device memory. */
int numa_sched_create(void* dev_arena, size_t arena_bytes, void* stream, int build_threads, numa_sched** out);

/* Queue one forecast: mesh/physics/precision config, initial condition (as
 * numa_init_state), time step and number of RK3 steps.  *id receives its
 * handle.  NUMA_EBUDGET if its workspace can never fit in the arena. */
int numa_sched_submit(numa_sched* s, const numa_config* cfg, int ic_kind, const double* params, int nparams,
                      double dt, int nsteps, long long* id);

/* Admit what fits (arrival order, first fit), advance every admitted member
 * by one RK3 step (asynchronously, on the compute stream), retire members that
 * reached their step count.  *n_active: members advancing; *n_waiting:
 * requests queued, building or still copying their result out. */
int numa_sched_step(numa_sched* s, int* n_active, int* n_waiting);

/* Status (numa_req_status), steps done and global-node count of a request
 * (steps_done and Ng may be NULL). */
int numa_sched_poll(numa_sched* s, long long id, int* status, int* steps_done, long long* Ng);

/* Copy a finished request's final state, double[5][Ng] host (n = 5*Ng), and
 * forget the request.  NUMA_ENONFINITE (after copying) if it failed that way. */
int numa_sched_result(numa_sched* s, long long id, double* q_host, long long n);

/* Cancel a request that is still queued. */
int numa_sched_cancel(numa_sched* s, long long id);

const char* numa_sched_last_error(const numa_sched* s);

/* Wait for the compute stream, free all host-side state.  Never frees the
 * arena. */
int numa_sched_destroy(numa_sched* s);

/* Host copy of the global-node coordinates, double[3][Ng] (x, y, z). */
int numa_get_coords(const numa_ctx* ctx, double* xyz);

/* Last error message of this context (never NULL). */
const char* numa_last_error(const numa_ctx* ctx);

/* Free the context's host data.  Never frees the workspace. */
int numa_destroy(numa_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
