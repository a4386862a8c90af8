// Internal declarations of the GB300 NUMA hot-path library: host mesh data,
// the device workspace layout and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "numa.h"

namespace numa {

constexpr int kMaxN = 8;
constexpr int kEosTerms = 12;  // binomial-series terms of (1+x)^gamma - 1 for |x| <= 1/32
constexpr int kDssBlock = 128;  // threads of the update kernel; the DSS order is sorted within such blocks

// Host-side mesh and geometry (Sec. 2.1: Lobatto points, Eq. 4: Jw and M,
// Eq. 5: isoparametric metric terms).  Built once per context.
struct HostMesh {
  int N = 0, P = 0, Np = 0;
  long long Ne = 0, Nl = 0, Ng = 0;
  std::vector<double> xi, w, D;       // 1D Lobatto nodes, weights, D[i*P+j] = psi_j'(xi_i)
  std::vector<double> gxyz;           // global-node coordinates [3][Ng]
  std::vector<int32_t> l2g;           // element node -> global node [Nl]
  std::vector<int32_t> csr_off;       // global node -> first entry in csr_idx [Ng+1]
  std::vector<int32_t> csr_idx;       // element nodes of each global node, ascending [nentries]
  long long nentries = 0;             // CSR entries: Nl (CG storage) or sum of the squared counts (DG)
  std::vector<uint8_t> dss_order;     // per block of kDssBlock global nodes: local indices sorted by
                                      // their number of element nodes (stable) [ceil(Ng/kDssBlock)*kDssBlock]
  std::vector<double> met;            // [10][Nl]: dxi_d/dx_c at row 3d+c, then Jw
  std::vector<double> ref;            // [4][Ng]: rho0, (rho theta)_0, p0, 1/(rho theta)_0
  std::vector<double> Minv;           // [Ng]: 1 / sum_e Jw
  std::vector<uint8_t> wall;          // [Ng]: bit a = box wall normal to axis a; bit 3 = shell radial wall
  std::vector<double> gvec;           // shell only, [3][Ng]: g(r) r_hat
  std::vector<double> nrm;            // shell only, [3][Ng]: r_hat (wall normal)
  std::vector<double> hgt;            // shell only, [Nl] during setup: height above r_inner
};

bool build_host_mesh(const numa_config& c, HostMesh& m, std::string& err);
// Re-index a built mesh for DG storage (one storage node per element node).
void expand_to_dg_storage(HostMesh& m);
bool init_state_host(const numa_config& c, const HostMesh& m, int kind, const double* prm, int nprm,
                     double* q, std::string& err);

// Per-global-node primitive fields that the volume kernel gathers, written by
// the stage update (or the primitive pass) for the state the next create_rhs
// differentiates:
//   FP64 mode  : double [9][Ng] = the flux components U_x u_x + p', U_y u_y + p',
//                U_z u_z + p', U_x u_y, U_x u_z, U_y u_z, Theta u_x, Theta u_y,
//                Theta u_z (U comes from q), formed once per global node
//   FP32 mode  : float  [Ng][8] = (U_x, U_y, U_z, u_x), (u_y, u_z, theta, p') per node,
//                two float4 (one 32-byte sector per node for the gather)
//   pairs mode : float2 [8][Ng] = the same eight, each as a (hi, lo) pair
inline int prim_bytes_per_node(int precision) {
  return precision == NUMA_FP32_MIXED ? 32 : precision == NUMA_FP64_PAIRS ? 64 : 72;
}

// Device workspace carved from the caller's buffer.
struct DevLayout {
  double* q = nullptr;       // state q^n [5][Ng]
  double* qs = nullptr;      // stage state [5][Ng]
  void* prim = nullptr;      // primitive fields (scratch) [kPrimBytesPerNode * Ng]
  void* re = nullptr;        // element residuals -Jw div F (scratch): double or float [5][Nl]
  double* met64 = nullptr;   // [10][Nl] FP64 metric terms and Jw; for the per-node form rows 0..8
                             // hold -Jw dxi_d/dx_c (the weighted metric of volume_element_nodal64)
  float* met32 = nullptr;    // [10][Nl] FP32 copy (mixed-precision form)
  float2* met2 = nullptr;    // [10][Nl] (hi, lo) pairs (pairs mode)
  float2* D2 = nullptr;      // [P*P] (hi, lo) pairs (pairs mode)
  int32_t* l2g = nullptr;
  int32_t* csr_off = nullptr;
  int32_t* csr_idx = nullptr;
  uint8_t* dss_order = nullptr;  // [ceil(Ng/kDssBlock)*kDssBlock]
  double* ref = nullptr;     // [4][Ng]
  double* Minv = nullptr;    // [Ng]
  double* Minv_r = nullptr;  // rectilinear form (FP64, pairs): [Ng] w_i w_j w_k / M, the weight of the node's
                             // element nodes (equal at all of them) folded into the inverse mass
  uint8_t* wall = nullptr;   // [Ng]
  double* gvec = nullptr;    // [3][Ng] (shell)
  double* nrm = nullptr;     // [3][Ng] (shell)
  double* D64 = nullptr;     // [P*P]
  double* affk = nullptr;    // FP64 / pairs affine elements: [3][Ne] K_d = -J dxi_d/dx_d per element
  float* D32 = nullptr;      // [P*P]
  double* F64 = nullptr;     // [P*P] 1D filter matrix (FP64, pairs)
  float* F32 = nullptr;      // [P*P] the same in FP32 (FP32 form)
  double* imex = nullptr;    // 1D-IMEX tables (imex_table_doubles), boxes with walled columns only
  int* imex_piv = nullptr;   // [2][nz][3] pivots and row extents of the two factorisations (dt, dt/2)
  int* flags = nullptr;      // [64]: 0 = non-finite
  size_t bytes = 0;
};

size_t layout_workspace(const numa_config& c, const HostMesh& m, char* base, DevLayout* L);
size_t residual_bytes(const numa_config& c, const HostMesh& m);  // bytes of the re scratch

// ---- kernels -------------------------------------------------------------

struct PrimArgs {
  const double* q;     // state the primitives describe [5][Ng]
  const double* ref;   // [4][Ng]
  void* prim;          // output
  double* qcopy;       // prim_kernel only: where it also copies q (nullptr: no copy)
  long long Ng;
  int precision;
  double gamma;
  double eos[kEosTerms];  // binomial coefficients C(gamma, k), k = 1..kEosTerms
};

// Every element of the mesh maps affinely onto the reference cube (a box
// without warp) and the configuration lets the kernel use that.
inline bool affine_elements(const numa_config& c) {
  return c.mesh_kind == NUMA_MESH_BOX && c.warp == 0.0 && c.metric_form == NUMA_METRIC_AUTO;
}

struct VolumeArgs {
  const double* q;     // state [5][Ng] (FP64 mode reads U from it)
  const void* prim;    // primitive fields of q
  const int32_t* l2g;
  const double* met64;
  const float* met32;
  const double* D64;
  const float* D32;
  const float2* met2;  // pairs mode
  const float2* D2;    // pairs mode
  void* re;            // [5][Nl] output
  const double* affk;   // rectilinear form (FP64, pairs): [3][Ne] -J dxi_d/dx_d
  long long Ng, Nl;
  int Ne;
  int ebeg, ecnt;      // the launch covers elements [ebeg, ebeg + ecnt) (a slab, or all: 0, Ne)
  int affine;          // volume_form: 0 the per-node form; 1 every element is affine, the
                       // contravariant-flux form (FP32-mixed, pairs); 2 every element is also
                       // rectilinear (diagonal metric terms): the folded form (FP64, pairs)
};

struct UpdateArgs {
  const int32_t* off;
  const int32_t* idx;
  const uint8_t* order;  // DSS order within each block of kDssBlock nodes (single-mesh kernel)
  const void* re;
  const double* Minv;
  const uint8_t* wall;
  const double* gvec;  // shell gravity vectors or null (box)
  const double* nrm;   // shell radial unit vectors (read at wall nodes)
  const double* qk;    // state the RHS was evaluated at
  const double* qn;    // q^n (RK base), may equal qk
  double* out;         // R (mode 0) or q^{k+1} (mode 1)
  long long Ng, Nl;
  double g;            // box gravity
  double two_omega;    // shell Coriolis 2 Omega
  double a, b, dt;     // out = a qn + b (qk + dt R)
  double bdt, bdtg;    // b dt and b dt g, computed once on the host
  int first_stage;     // 1 when a = 0 and b = 1 (no q^n term); low-storage scheme: A = 0 (no dq read)
  double* dq;          // low-storage scheme (modes 4, 5): the second register; out = qk = q, a = A_i, b = B_i
  int mode;            // 0: write R, 1: SSP-RK3 stage, 3: filter DSS, 4: low-storage stage (1, 3, 4 also
                       // write the primitives of out)
  int* flag;           // non-finite flag
  PrimArgs pa;         // primitive output of mode 1 (pa.q unused)
  // the launch covers global nodes [ibeg, iend): a slab (ibeg a multiple of
  // kDssBlock), or all: 0, Ng
  long long ibeg, iend;
  // CG box meshes: the lattice of the structured global numbering (g = ix +
  // nx (iy + ny iz)), from which the DSS finds the element nodes at a global
  // node without the inverse map; box_N = 0 for any other mesh or storage
  int box_N, box_ne[3], box_per[3];
  long long box_n[3];
};

// The column part of one 1D-IMEX leapfrog step (csrc/imex.cu).  Column c,
// level k is global node c + ncol k: the z-columns of a walled box, or the
// radial columns of the shell (numbered level by level), W = U . r_hat.  The kernel
// forms q* = qprev + cR R, applies the implicit vertical correction with the
// banded LU factors of the Schur matrix, writes q^{n+1} into q, the
// Robert-Asselin filtered q^n into qs and the primitive fields of q^{n+1}.
struct ImexArgs {
  double* q;            // in: q^n, out: q^{n+1} [5][Ng]
  double* qs;           // out: filtered q^n [5][Ng]
  const double* qprev;  // filtered q^{n-1}; q itself on the start step
  double* R;            // R(q^n) [5][Ng]; overwritten (q*_rho, s_W, q*_Theta kept per node)
  const double* Dz;     // [nz][2N+1]: column derivative, entry j of row k at column k - N + j
  const double* c2;     // [nz] gamma p0 / Theta0
  const double* th0;    // [nz] Theta0 / rho0
  const double* gl;     // [nz] gravity g(r) at each level (the box: g)
  const double* r2;     // [nz] 2 / r at each level, the spherical divergence term (the box: 0)
  const double* nrm;    // shell: r_hat [3][Ng] (radial columns); box: null
  const double* Lf;     // [nz][kl]: multipliers of elimination step k (rows k+1 .. k+kl)
  const double* Uf;     // [nz][1 + ku]: 1 / U_kk, then U_{k,k+1} .. U_{k,k+ku}
  const int* piv;       // [nz][3]: row swapped with row k at step k, multipliers used (last
                        // nonzero), U entries used (last nonzero) of row k
  int N, nz, kl, ku, cols_per_block;
  long long ncol, Ng;
  double cR, tau, nu;     // q* = qprev + cR R; (I - tau L) correction; filter strength
  int* flag;              // non-finite flag
  PrimArgs pa;            // primitive fields of q^{n+1}
};

// Host tables of the vertical operator and the factors of one Schur matrix.
struct ImexTables {
  int nz = 0, N = 0, kl = 0, ku = 0;
  std::vector<double> Dz, c2, th0;  // [nz][2N+1], [nz], [nz]
  std::vector<double> gl, r2;       // [nz] g(r) and 2 / r per level (box: g and 0)
  std::vector<double> Lf, Uf;       // [nz][kl], [nz][1 + 4N] (ku <= 4N used)
  std::vector<int> piv;             // [nz][3] (see ImexArgs::piv)
};

// 1D-IMEX: whether the configuration has straight walled vertical columns
// (an unwarped box with walls at the bottom and top, FP64, CG storage), the
// column count and height, and the host tables (imex_setup.cpp).
bool imex_supported(const numa_config& c, long long* ncol, int* nz, std::string* why);
bool imex_operator(const numa_config& c, const HostMesh& m, ImexTables& t, std::string& err);
bool imex_factor(const ImexTables& t, double tau, std::vector<double>& Lf, std::vector<double>& Uf,
                 std::vector<int>& piv, int* ku, std::string& err);
size_t imex_table_doubles(int nz, int N);

// One application of the Boyd-Vandeven filter (element part).
struct FilterArgs {
  const double* q;       // state [5][Ng]
  const int32_t* l2g;
  const void* F;         // 1D filter matrix [(N+1)^2]: double (FP64, pairs) or float (FP32 form)
  const double* met64;   // Jw is row 9 of whichever metric array the precision stores
  const float* met32;
  const float2* met2;
  void* re;              // [5][Nl] Jw-weighted correction, double or float like the residuals
  long long Ng, Nl;
  int Ne;
};

cudaError_t launch_prim(const PrimArgs& a, cudaStream_t s);
// Copies D of order N (FP32, (N+1)^2 values, host memory that stays valid
// until s has run the copy) into the constant table of the FP32 line kernel.
cudaError_t upload_d32_constant(int N, const float* D, cudaStream_t s);
cudaError_t launch_volume(int N, int precision, const VolumeArgs& a, cudaStream_t s);
// the element kernels of one precision (volume_fp64.cu, volume_fp32.cu,
// volume_pairs.cu); launch_volume and launch_volume_ragged dispatch to them
cudaError_t launch_volume_fp64(int N, bool affine, const VolumeArgs& a, cudaStream_t s);
cudaError_t launch_volume_fp32(int N, bool affine, const VolumeArgs& a, cudaStream_t s);
cudaError_t launch_volume_pairs(int N, bool affine, const VolumeArgs& a, cudaStream_t s);
cudaError_t launch_update(int precision, const UpdateArgs& a, cudaStream_t s);
// the element part of the filter (filter.cu); mode 3 of launch_update does the DSS
cudaError_t launch_filter(int N, int precision, const FilterArgs& a, cudaStream_t s);
// Columns per block of the IMEX kernel for columns of nz levels (0: too tall),
// its shared memory, and its launch (imex.cu).
int imex_cols_per_block(int nz, int N);
size_t imex_smem_bytes(int nz, int N, int cols_per_block);
cudaError_t imex_kernel_setup();
cudaError_t launch_imex(const ImexArgs& a, cudaStream_t s);

// ---- serving: ragged multi-member launches --------------------------------

constexpr int kMaxMembers = 128;

// Everything the element and node kernels need for one admitted member: its
// volume arguments and its update arguments for each of the three stages.
struct MemberDesc {
  VolumeArgs va;
  UpdateArgs ua[3];
};

// One group of members that share N, precision and mesh kind: prefix sums of
// their element and global-node counts over the member slots in `member`.
struct RaggedGroup {
  int n;
  int pad;
  long long elem_prefix[kMaxMembers + 1];
  long long block_prefix[kMaxMembers + 1];  // blocks of kDssBlock global nodes (each member's padded to whole blocks)
  int member[kMaxMembers];
};

cudaError_t launch_volume_ragged(int N, int precision, bool affine, const MemberDesc* d, const RaggedGroup* g,
                                 cudaStream_t s);
cudaError_t launch_volume_ragged_fp64(int N, bool affine, const MemberDesc* d, const RaggedGroup* g, cudaStream_t s);
cudaError_t launch_volume_ragged_fp32(int N, bool affine, const MemberDesc* d, const RaggedGroup* g, cudaStream_t s);
cudaError_t launch_volume_ragged_pairs(int N, bool affine, const MemberDesc* d, const RaggedGroup* g, cudaStream_t s);
cudaError_t launch_update_ragged(int precision, bool shell, int stage, const MemberDesc* d, const RaggedGroup* g,
                                 cudaStream_t s);

}  // namespace numa

namespace numa {
// Slabs of a box along z for the pipelined RK step: element slab k is
// elements [ebeg[k], ebeg[k+1]), node slab k global nodes [ibeg[k],
// ibeg[k+1]) (ibeg a multiple of kDssBlock).  S = 1: no pipeline.
struct SlabPlan {
  int S = 1;
  std::vector<int> ebeg;
  std::vector<long long> ibeg;
};
constexpr int kMaxSlabs = 16;
}  // namespace numa

// A context: the host mesh of one configuration and, once bound, the layout of
// its device workspace.
struct numa_ctx {
  numa_config cfg;
  numa::HostMesh mesh;
  numa::DevLayout L;
  bool bound = false;
  bool prim_valid = false;  // L.prim holds the primitive fields of L.q
  bool rect = false;        // FP64, affine and every element rectilinear: the folded element kernel
  int nslab_req = 0;        // slabs asked for by numa_set_slabs (0: automatic)
  numa::SlabPlan slabs;     // the plan in use (made at bind and by numa_set_slabs)
  cudaStream_t side = nullptr;  // the second stream of the slab pipeline
  cudaEvent_t ev_fork = nullptr, ev_vol[numa::kMaxSlabs] = {}, ev_upd[numa::kMaxSlabs] = {};
  cudaStream_t stream = nullptr;
  std::string err;
  double gamma = 1.4;
  double eos[numa::kEosTerms];
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0.0;
  const double* graph_q = nullptr;
  // Boyd-Vandeven filter: parameters (set by numa_set_filter), its host
  // matrix, and the steps since it was last applied
  int rk_scheme = NUMA_RK_SSP3;
  bool filter_set = false;
  int filter_every = 0, filter_s = 0, filter_count = 0;
  double filter_p = 0.0, filter_mu = 0.0;
  std::vector<double> filter_F;
  cudaGraphExec_t fgraph = nullptr;
  const double* fgraph_q = nullptr;
  // 1D-IMEX leapfrog: Robert-Asselin strength, host tables, the dt the
  // device factors were made for, and whether q^n has a predecessor (false:
  // the next step is the start step)
  double imex_nu = 0.05;
  bool imex_tables = false;
  numa::ImexTables imex;
  long long imex_ncol = 0;
  double imex_dt = 0.0;
  int imex_ku[2] = {0, 0};  // upper bandwidths of the factors for dt and dt/2
  bool imex_factored = false;
  bool imex_started = false;
};

namespace numa {

// SSP-RK3 stage coefficients: q^{k+1} = a_k q^n + b_k (q^k + dt R(q^k))
extern const double kRkA[3];
extern const double kRkB[3];
// five-stage low-storage scheme: dq <- kLsA[i] dq + dt R(q); q <- q + kLsB[i] dq
extern const double kLsA[5];
extern const double kLsB[5];

PrimArgs prim_args(const numa_ctx* c, const double* q, void* prim);
VolumeArgs volume_args(const numa_ctx* c, const double* q, const void* prim, void* re);
int volume_form(const numa_ctx* c);
UpdateArgs update_args(const numa_ctx* c, const void* re, const double* qk, const double* qn, double* out,
                       int mode, double ra, double rb, double dt);
FilterArgs filter_args(const numa_ctx* c);
// Boyd-Vandeven weights and the 1D filter matrix F = V diag(sigma) V^-1 of
// order N on the Lobatto points xi with weights w (mesh.cpp).
void filter_matrix_host(int N, const double* xi, const double* w, int s, double p, double mu, double* F);
cudaError_t ensure_prim(numa_ctx* c);

}  // namespace numa
