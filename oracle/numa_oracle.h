/*
 * numa_oracle.h -- plain FP64 CPU oracle for the CG spectral-element RHS and
 * Runge-Kutta stage of the NUMA dynamical core (Mueller et al., "Strong
 * scaling for numerical weather prediction at petascale with the atmospheric
 * model NUMA", Sec. 2, Eqs. 1-5).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent reference that
 * the CUDA path is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the GPU library, and the GPU library never
 * calls it.
 *
 * Everything is FP64, written for clarity rather than speed: one loop per
 * step of the method, in the order Sec. 2 states them.
 *
 * Layouts (identical meaning to the GPU library's public layout, written
 * independently):
 *   state q, tendency R : double[5][Ng], variables (rho', U_x, U_y, U_z,
 *                         Theta') with U = rho*u and Theta' = rho*theta minus
 *                         the reference (rho*theta)_0.
 *   box global node     : g = ix + nx*(iy + ny*iz), ix in [0,nx) along x, with
 *                         nx = nex*N + 1 (walls) or nex*N (periodic in x).
 *   shell global node   : oracle-internal numbering (first appearance in
 *                         ascending element-node order); compare by
 *                         coordinates.
 */
#ifndef NUMA_ORACLE_H
#define NUMA_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BOX = 0, ORC_SHELL = 1 };
enum { ORC_REF_ISENTROPIC = 0, ORC_REF_ISOTHERMAL = 1 };
enum { ORC_IC_REST = 0, ORC_IC_BUBBLE = 1, ORC_IC_UNIFORM = 2, ORC_IC_JETWAVE = 3 };

typedef struct {
  int kind;                 /* ORC_BOX or ORC_SHELL */
  int N;                    /* polynomial order (N+1 LGL points per direction), 1..8 */
  int nex, ney, nez;        /* box: elements per direction */
  double Lx, Ly, Lz;        /* box: extents, origin at (0,0,0) */
  int periodic[3];          /* box: periodic flags per axis */
  double warp;              /* box: smooth interior warp amplitude (fraction of extent) */
  int npanel, nlayer;       /* shell: elements per cube-panel edge, radial layers */
  double r_inner, r_outer;  /* shell: inner (planet) radius a, outer radius */
  double Rd, cp, cv, P00;   /* gas constant, heat capacities, reference pressure */
  double g;                 /* gravity (box) or surface gravity g0 (shell, g(r)=g0 (a/r)^2) */
  double Omega;             /* planetary rotation rate about +z (shell only) */
  int ref_kind;             /* ORC_REF_ISENTROPIC (theta0) or ORC_REF_ISOTHERMAL (T0) */
  double theta0, T0;
} orc_config;

typedef struct orc_mesh orc_mesh;

/* LGL nodes and weights on [-1,1] (Sec. 2.1: Lobatto points), N+1 of each. */
void orc_lgl(int N, double* xi, double* w);
/* Differentiation matrix D[i*(N+1)+j] = psi_j'(xi_i) (Eq. 5). */
void orc_dmatrix(int N, const double* xi, double* D);

/* Build the mesh, geometry, maps, mass matrix and reference state.
 * Returns 0 on success, -1 on a bad config, -2 on allocation failure. */
int orc_build(const orc_config* cfg, orc_mesh** out);
void orc_free(orc_mesh* m);
void orc_sizes(const orc_mesh* m, long* Ne, long* Nl, long* Ng);

/* Copies of mesh data (caller-owned buffers). */
void orc_get_coords(const orc_mesh* m, double* xyz);       /* [3][Ng] */
void orc_get_elem_coords(const orc_mesh* m, double* xyz);  /* [3][Nl] */
void orc_get_l2g(const orc_mesh* m, long* l2g);            /* [Nl] */
void orc_get_metrics(const orc_mesh* m, double* met);      /* [10][Nl]: dxi_d/dx_c (d-major), then J */
void orc_get_jw(const orc_mesh* m, double* jw);            /* [Nl] */
void orc_get_mass(const orc_mesh* m, double* M);           /* [Ng] */
void orc_get_ref(const orc_mesh* m, double* ref);          /* [3][Ng]: rho0, (rho theta)_0, p0 */
void orc_get_wall(const orc_mesh* m, unsigned char* wall); /* [Ng] bit0..2 box walls x,y,z; bit3 shell radial */

/* Pressure perturbation from the equation of state (see orc_pprime in .c). */
double orc_pprime(double Th_pert, double Th0, double p0, double gamma);
double orc_pprime_naive(double Th_pert, double Th0, double p0, const orc_config* c);

/* Initial conditions.  params:
 *   BUBBLE : {A, r_c, x_c, y_c, z_c}
 *   UNIFORM: {u0, v0, w0}
 *   JETWAVE: {U_jet, pert_amp, pert_radius_frac, lambda_c, phi_c} */
int orc_init_state(const orc_mesh* m, int kind, const double* params, double* q);

/* Element-local weighted residual r_e = -Jw (div F - S) at every element
 * node (before DSS), [5][Nl]. */
void orc_rhs_elem(const orc_mesh* m, const double* q, double* re);
/* Full tendency R = M^-1 DSS(r_e) with wall conditions applied (Eq. 4). */
void orc_rhs(const orc_mesh* m, const double* q, double* R);

/* One SSP-RK3 step on a generic right-hand side callback. */
typedef void (*orc_rhs_fn)(void* ctx, const double* q, double* r);
void orc_ssprk3_step(long n, double* q, double dt, orc_rhs_fn f, void* ctx, double* work);
/* nsteps SSP-RK3 steps of the NUMA system, in place on q. */
int orc_run(const orc_mesh* m, double* q, double dt, int nsteps);

/* The five-stage low-storage Runge-Kutta scheme (Carpenter-Kennedy, order
 * four): its coefficients A[5], B[5]; one step on a generic callback (work:
 * 2n doubles); nsteps steps of the NUMA system in place on q. */
void orc_lsrk54_coefficients(double* A, double* B);
void orc_lsrk54_step(long n, double* q, double dt, orc_rhs_fn f, void* ctx, double* work);
int orc_run_lsrk54(const orc_mesh* m, double* q, double dt, int nsteps);

/* Boyd-Vandeven filter (Sec. 2.3): weights sigma[0..N] of the Legendre modes
 * (first damped mode s, order p, strength mu), the 1D filter matrix
 * F = V diag(sigma) V^-1 (row-major, (N+1)^2), one application of the filter
 * to a global state (element-wise F x F x F, Jw-weighted DSS, division by M),
 * and an SSP-RK3 run with the filter after every `every`-th step. */
void orc_filter_weights(int N, int s, double p, double mu, double* sigma);
int orc_filter_matrix(int N, int s, double p, double mu, double* F);
int orc_filter(const orc_mesh* m, double* q, int s, double p, double mu);
int orc_run_filtered(const orc_mesh* m, double* q, double dt, int nsteps, int every, int s, double p, double mu);

#ifdef __cplusplus
}
#endif
#endif
