// C-ABI of the GB300 NUMA hot path (declared in include/numa.h): context
// life cycle, workspace binding, state I/O and the stage loop of code
// example 1 in Sec. 7 (create_rhs, DSS with the inverse mass matrix, update
// q), with one CUDA graph per RK step for numa_run.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "numa_internal.h"

using namespace numa;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int fail(numa_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(numa_ctx* c, cudaError_t e, const char* what) {
  return fail(c, NUMA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

namespace numa {

const double kRkA[3] = {0.0, 0.75, 1.0 / 3.0};
const double kRkB[3] = {1.0, 0.25, 2.0 / 3.0};
// Carpenter and Kennedy's five-stage, fourth-order 2N-storage coefficients
const double kLsA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kLsB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};

PrimArgs prim_args(const numa_ctx* c, const double* q, void* prim) {
  PrimArgs a;
  a.q = q;
  a.ref = c->L.ref;
  a.prim = prim;
  a.qcopy = nullptr;
  a.Ng = c->mesh.Ng;
  a.precision = c->cfg.precision;
  a.gamma = c->gamma;
  for (int k = 0; k < kEosTerms; ++k) a.eos[k] = c->eos[k];
  return a;
}

VolumeArgs volume_args(const numa_ctx* c, const double* q, const void* prim, void* re) {
  VolumeArgs a;
  a.q = q;
  a.prim = prim;
  a.l2g = c->L.l2g;
  a.met64 = c->L.met64;
  a.met32 = c->L.met32;
  a.D64 = c->L.D64;
  a.D32 = c->L.D32;
  a.met2 = c->L.met2;
  a.D2 = c->L.D2;
  a.re = re;
  a.affk = c->L.affk;
  a.Ng = c->mesh.Ng;
  a.Nl = c->mesh.Nl;
  a.Ne = (int)c->mesh.Ne;
  a.ebeg = 0;
  a.ecnt = a.Ne;
  a.affine = volume_form(c);
  return a;
}

// Element-kernel form of a bound context: 2 the rectilinear form (FP64,
// pairs), 1 the general affine form (pairs, FP32-mixed), 0 the per-node form
// (any element; FP64 takes it on affine elements that are not rectilinear).
int volume_form(const numa_ctx* c) {
  if (!affine_elements(c->cfg)) return 0;
  if (c->rect) return 2;
  return c->cfg.precision == NUMA_FP64 ? 0 : 1;
}

UpdateArgs update_args(const numa_ctx* c, const void* re, const double* qk, const double* qn, double* out,
                       int mode, double ra, double rb, double dt) {
  UpdateArgs a;
  a.off = c->L.csr_off;
  a.idx = c->L.csr_idx;
  a.order = c->L.dss_order;
  a.re = re;
  // the rectilinear element kernels leave out the w_i w_j w_k weight, which
  // Minv_r carries; the filter's correction (mode 3) is Jw-weighted
  a.Minv = (mode != 3 && c->rect) ? c->L.Minv_r : c->L.Minv;
  a.wall = c->L.wall;
  a.gvec = c->L.gvec;
  a.nrm = c->L.nrm;
  a.qk = qk;
  a.qn = qn;
  a.out = out;
  a.Ng = c->mesh.Ng;
  a.Nl = c->mesh.Nl;
  a.ibeg = 0;
  a.iend = a.Ng;
  a.g = c->cfg.g;
  a.two_omega = 2.0 * c->cfg.Omega;
  a.a = ra;
  a.b = rb;
  a.dt = dt;
  a.bdt = rb * dt;
  a.bdtg = rb * dt * c->cfg.g;
  a.first_stage = (ra == 0.0 && rb == 1.0) ? 1 : 0;
  a.dq = nullptr;
  a.mode = mode;
  a.flag = c->L.flags;
  a.pa = prim_args(c, nullptr, c->L.prim);
  a.box_N = 0;
  if (c->cfg.mesh_kind == NUMA_MESH_BOX && c->cfg.storage == NUMA_STORAGE_CG && c->mesh.Nl < (1LL << 31)) {
    const int ne[3] = {c->cfg.nex, c->cfg.ney, c->cfg.nez};
    a.box_N = c->mesh.N;
    for (int d = 0; d < 3; ++d) {
      a.box_ne[d] = ne[d];
      a.box_per[d] = c->cfg.periodic[d] ? 1 : 0;
      a.box_n[d] = (long long)ne[d] * c->mesh.N + (c->cfg.periodic[d] ? 0 : 1);
    }
  }
  return a;
}

FilterArgs filter_args(const numa_ctx* c) {
  FilterArgs a;
  a.q = c->L.q;
  a.l2g = c->L.l2g;
  a.F = c->cfg.precision == NUMA_FP32_MIXED ? (const void*)c->L.F32 : (const void*)c->L.F64;
  a.met64 = c->L.met64;
  a.met32 = c->L.met32;
  a.met2 = c->L.met2;
  a.re = c->L.re;
  a.Ng = c->mesh.Ng;
  a.Nl = c->mesh.Nl;
  a.Ne = (int)c->mesh.Ne;
  return a;
}

// The filter matrix (FP64 and FP32 copies) into the bound workspace.
cudaError_t upload_filter(numa_ctx* c) {
  const size_t PP = c->filter_F.size();
  std::vector<float> f32(PP);
  for (size_t t = 0; t < PP; ++t) f32[t] = (float)c->filter_F[t];
  cudaError_t e = cudaMemcpyAsync(c->L.F64, c->filter_F.data(), PP * 8, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->L.F32, f32.data(), PP * 4, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e;
}

// One application of the filter to the state, in place on stream s; leaves
// the primitive fields of the filtered state.
cudaError_t enqueue_filter(numa_ctx* c, cudaStream_t s) {
  cudaError_t e = launch_filter(c->mesh.N, c->cfg.precision, filter_args(c), s);
  if (e == cudaSuccess)
    e = launch_update(c->cfg.precision, update_args(c, c->L.re, c->L.q, c->L.q, c->L.q, 3, 0.0, 1.0, 1.0), s);
  return e;
}

// R(q) into r_dev with the given primitive and residual scratch.
cudaError_t enqueue_rhs(numa_ctx* c, const double* q, double* r, void* prim, void* re) {
  cudaError_t e = launch_prim(prim_args(c, q, prim), c->stream);
  if (e == cudaSuccess) e = launch_volume(c->mesh.N, c->cfg.precision, volume_args(c, q, prim, re), c->stream);
  if (e == cudaSuccess) e = launch_update(c->cfg.precision, update_args(c, re, q, q, r, 0, 0.0, 1.0, 0.0), c->stream);
  return e;
}

// Primitive fields of the current state, if the state changed since they were made.
cudaError_t ensure_prim(numa_ctx* c) {
  if (c->prim_valid) return cudaSuccess;
  cudaError_t e = launch_prim(prim_args(c, c->L.q, c->L.prim), c->stream);
  if (e == cudaSuccess) c->prim_valid = true;
  return e;
}

// Stages per step of the context's integrator.
int rk_stages(const numa_ctx* c) {
  return c->rk_scheme == NUMA_RK_LS54 ? 5 : c->rk_scheme == NUMA_LEAPFROG_IMEX ? 1 : 3;
}

// Device pointers of the 1D-IMEX tables in the workspace: Dz, c2, theta0,
// g(r), 2/r, then (Lf, Uf) for tau = dt and for tau = dt/2.
struct ImexPtrs {
  double *Dz, *c2, *th0, *gl, *r2, *Lf[2], *Uf[2];
  int* piv[2];
};

ImexPtrs imex_ptrs(const numa_ctx* c) {
  const int nz = c->imex.nz, N = c->imex.N;
  ImexPtrs p;
  p.Dz = c->L.imex;
  p.c2 = p.Dz + (size_t)nz * (2 * N + 1);
  p.th0 = p.c2 + nz;
  p.gl = p.th0 + nz;
  p.r2 = p.gl + nz;
  p.Lf[0] = p.r2 + nz;
  p.Uf[0] = p.Lf[0] + (size_t)nz * 2 * N;
  p.Lf[1] = p.Uf[0] + (size_t)nz * (1 + 4 * N);
  p.Uf[1] = p.Lf[1] + (size_t)nz * 2 * N;
  p.piv[0] = c->L.imex_piv;
  p.piv[1] = c->L.imex_piv + 3 * nz;
  return p;
}

// Host factors of the column matrices for dt and dt/2 into the workspace
// (when dt changed), with the operator tables; waits for the copies.
// NUMA_EINVAL when a matrix cannot be factored, NUMA_ECUDA on a CUDA error.
int imex_prepare(numa_ctx* c, double dt) {
  cudaError_t e = imex_kernel_setup();
  if (e != cudaSuccess) return cuda_fail(c, e, "1D-IMEX kernel setup");
  if (c->imex_factored && c->imex_dt == dt) return NUMA_OK;
  std::string err;
  ImexPtrs p = imex_ptrs(c);
  const ImexTables& t = c->imex;
  std::vector<double> Lf, Uf;
  std::vector<int> piv;
  const size_t nz = (size_t)t.nz;
  e = cudaMemcpyAsync(p.Dz, t.Dz.data(), t.Dz.size() * 8, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p.c2, t.c2.data(), nz * 8, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p.th0, t.th0.data(), nz * 8, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p.gl, t.gl.data(), nz * 8, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p.r2, t.r2.data(), nz * 8, cudaMemcpyHostToDevice, c->stream);
  int ku[2] = {0, 0};
  for (int f = 0; f < 2 && e == cudaSuccess; ++f) {
    if (!imex_factor(t, f == 0 ? dt : 0.5 * dt, Lf, Uf, piv, &ku[f], err)) return fail(c, NUMA_EINVAL, err);
    e = cudaMemcpyAsync(p.Lf[f], Lf.data(), Lf.size() * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p.Uf[f], Uf.data(), Uf.size() * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p.piv[f], piv.data(), 3 * nz * sizeof(int), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // the host vectors are reused
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "1D-IMEX factor upload");
  c->imex_ku[0] = ku[0];
  c->imex_ku[1] = ku[1];
  c->imex_dt = dt;
  c->imex_factored = true;
  return NUMA_OK;
}

// One 1D-IMEX step on stream s (imex_prepare(dt) done): create_rhs on q^n,
// DSS + M^-1 into R (the primitive buffer, 40 B per node in FP64 and 64 B in
// the pairs mode, free once the element kernel has read it; R[v][g] lies
// inside node g's own primitive slots), then the column kernel, which leaves q^{n+1} in q,
// the filtered q^n in qs and the primitive fields of q^{n+1}.  The start
// step (no q^{n-1}) uses dt/2 factors, q* = q^0 + dt R and no filter.
cudaError_t enqueue_imex_step(numa_ctx* c, double dt, bool start, cudaStream_t s, cudaEvent_t* ev = nullptr) {
  double* R = static_cast<double*>(c->L.prim);
  cudaError_t e = ev ? cudaEventRecord(ev[0], s) : cudaSuccess;
  if (e == cudaSuccess) e = launch_volume(c->mesh.N, c->cfg.precision, volume_args(c, c->L.q, c->L.prim, c->L.re), s);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
  if (e == cudaSuccess)
    e = launch_update(c->cfg.precision, update_args(c, c->L.re, c->L.q, c->L.q, R, 0, 0.0, 1.0, 0.0), s);
  if (e == cudaSuccess) {
    const ImexPtrs p = imex_ptrs(c);
    const int f = start ? 1 : 0;
    ImexArgs a;
    a.q = c->L.q;
    a.qs = c->L.qs;
    a.qprev = start ? c->L.q : c->L.qs;
    a.R = R;
    a.Dz = p.Dz;
    a.c2 = p.c2;
    a.th0 = p.th0;
    a.gl = p.gl;
    a.r2 = p.r2;
    const bool shell = c->cfg.mesh_kind == NUMA_MESH_SHELL;
    a.nrm = shell ? c->L.nrm : nullptr;
    a.Lf = p.Lf[f];
    a.Uf = p.Uf[f];
    a.piv = p.piv[f];
    a.N = c->imex.N;
    a.nz = c->imex.nz;
    a.kl = c->imex.kl;
    a.ku = c->imex_ku[f];
    a.cols_per_block = imex_cols_per_block(a.nz, a.N);
    a.ncol = c->imex_ncol;
    a.Ng = c->mesh.Ng;
    a.cR = start ? dt : 2.0 * dt;
    a.tau = start ? 0.5 * dt : dt;
    a.nu = start ? 0.0 : c->imex_nu;
    a.flag = c->L.flags;
    a.pa = prim_args(c, nullptr, c->L.prim);
    e = launch_imex(a, s);
  }
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[3], s);
  return e;
}

// One step of the context's integrator on stream s: per stage create_rhs,
// then DSS + M^-1 + the stage update, which also leaves the primitive fields
// of the new stage state.  Needs the primitive fields of q^n on entry and
// leaves those of q^{n+1}.  With ev != nullptr every kernel is bracketed by
// events (4 per stage).
//   SSP-RK3: stage states q -> qs -> qs -> q.
//   low-storage: q updated in place, qs holds dq.
cudaError_t enqueue_rk_step(numa_ctx* c, double dt, cudaStream_t s, cudaEvent_t* ev = nullptr) {
  double* q = c->L.q;
  double* qs = c->L.qs;
  const bool ls = c->rk_scheme == NUMA_RK_LS54;
  const double* qin[3] = {q, qs, qs};
  double* qout[3] = {qs, qs, q};
  const int ns = rk_stages(c);
  auto stage_update = [&](int st) {
    UpdateArgs ua;
    if (ls) {
      ua = update_args(c, c->L.re, q, q, q, 4, kLsA[st], kLsB[st], dt);
      ua.first_stage = st == 0 ? 1 : 0;
      ua.dq = qs;
    } else {
      ua = update_args(c, c->L.re, qin[st], q, qout[st], 1, kRkA[st], kRkB[st], dt);
    }
    return ua;
  };
  const SlabPlan& P = c->slabs;
  if (!ev && P.S > 1) {
    // slab pipeline: element slabs on s, node slabs on the side stream; the
    // update of node slab k needs the residuals of element slabs <= k, the
    // next stage's element slab k the new state of node slabs k and k + 1
    // (every node's arithmetic is unchanged: the result is the same bit for bit)
    const int S = P.S;
    cudaStream_t side = c->side;
    cudaError_t e = cudaEventRecord(c->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, c->ev_fork, 0);
    for (int st = 0; st < ns && e == cudaSuccess; ++st) {
      const double* qi = ls ? q : qin[st];
      for (int k = 0; k < S && e == cudaSuccess; ++k) {
        if (st > 0) e = cudaStreamWaitEvent(s, c->ev_upd[k + 1 < S ? k + 1 : S - 1], 0);
        VolumeArgs va = volume_args(c, qi, c->L.prim, c->L.re);
        va.ebeg = P.ebeg[k];
        va.ecnt = P.ebeg[k + 1] - P.ebeg[k];
        if (e == cudaSuccess) e = launch_volume(c->mesh.N, c->cfg.precision, va, s);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_vol[k], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, c->ev_vol[k], 0);
        UpdateArgs ua = stage_update(st);
        ua.ibeg = P.ibeg[k];
        ua.iend = P.ibeg[k + 1];
        if (e == cudaSuccess) e = launch_update(c->cfg.precision, ua, side);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_upd[k], side);
      }
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_upd[S - 1], 0);
    return e;
  }
  for (int st = 0; st < ns; ++st) {
    const double* qi = ls ? q : qin[st];
    cudaError_t e = ev ? cudaEventRecord(ev[4 * st], s) : cudaSuccess;
    if (e == cudaSuccess) e = launch_volume(c->mesh.N, c->cfg.precision, volume_args(c, qi, c->L.prim, c->L.re), s);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[4 * st + 1], s);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[4 * st + 2], s);
    if (e == cudaSuccess) e = launch_update(c->cfg.precision, stage_update(st), s);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[4 * st + 3], s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The per-node FP64 form reads -Jw dxi_d/dx_c: rows 0..8 of the uploaded
// metric array times -Jw (row 9), in place.
__global__ void __launch_bounds__(256) weight_metric_kernel(double* met, long long Nl) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= Nl) return;
  const double mjw = -met[9 * Nl + n];
#pragma unroll
  for (int t = 0; t < 9; ++t) met[t * Nl + n] *= mjw;
}

// Slabs of a box along z for the pipelined RK step (see SlabPlan).  A plan
// needs CG storage, walls at the bottom and top (a periodic seam would tie
// the first node slab to the last element slab), element slabs at least two
// lattice planes thick and planes of at least kDssBlock nodes, so that node
// slab k (rounded down to a kDssBlock boundary) only holds nodes of element
// slabs <= k and the element slab k reads only node slabs k and k + 1.
// `want` slabs (0: three for FP32-mixed meshes of 2^18 or more global nodes,
// where the memory-bound element kernel and the FP64-bound update overlap;
// in FP64 and the pairs mode both kernels need the FP64 pipe, or the FP32
// pipe beside it, and the pipeline measured no gain, so none by default).
SlabPlan plan_slabs(const numa_config& c, const HostMesh& m, int want) {
  SlabPlan P;
  if (c.mesh_kind != NUMA_MESH_BOX || c.storage != NUMA_STORAGE_CG || c.periodic[2]) return P;
  int S = want > 0 ? want : (c.precision == NUMA_FP32_MIXED && m.Ng >= (1LL << 18) ? 3 : 1);
  if (S > kMaxSlabs) S = kMaxSlabs;
  if (S > c.nez) S = c.nez;
  if (S <= 1) return P;
  const long long N = m.N, nx = (long long)c.nex * N + (c.periodic[0] ? 0 : 1);
  const long long ny = (long long)c.ney * N + (c.periodic[1] ? 0 : 1), plane = nx * ny;
  if (plane < kDssBlock) return P;
  std::vector<int> ez(S + 1);
  for (int k = 0; k <= S; ++k) ez[k] = (int)((long long)k * c.nez / S);
  for (int k = 0; k < S; ++k)
    if ((ez[k + 1] - ez[k]) * N < 2) return P;
  P.ebeg.resize(S + 1);
  P.ibeg.resize(S + 1);
  for (int k = 0; k <= S; ++k) {
    P.ebeg[k] = (int)((long long)ez[k] * c.nex * c.ney);
    P.ibeg[k] = k == S ? m.Ng : (ez[k] * N * plane) / kDssBlock * kDssBlock;
  }
  for (int k = 0; k < S; ++k)
    if (P.ibeg[k + 1] <= P.ibeg[k] || P.ibeg[k] > ez[k] * N * plane) return SlabPlan();
  P.S = S;
  return P;
}

// The side stream and the events of the slab pipeline (once per context,
// on the device current at the call).
cudaError_t ensure_slab_streams(numa_ctx* c) {
  if (c->side) return cudaSuccess;
  // the update stream at the highest priority: its blocks take SM slots as
  // soon as element blocks finish, so that the two kernels share the SMs
  int lo = 0, hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  for (int k = 0; k < kMaxSlabs && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&c->ev_vol[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_upd[k], cudaEventDisableTiming);
  }
  return e;
}

// Whether every element has diagonal metric terms (off-diagonal entries
// exactly zero at its first node): the elements of an affine mesh are then
// rectilinear.
bool rectilinear_elements(const HostMesh& m) {
  const long long Nl = m.Nl, Np = m.Np;
  for (long long e = 0; e < m.Ne; ++e) {
    const long long n = e * Np;
    for (int t : {1, 2, 3, 5, 6, 7})
      if (m.met[t * Nl + n] != 0.0) return false;
  }
  return true;
}

}  // namespace

namespace numa {

size_t residual_bytes(const numa_config& c, const HostMesh& m) {
  return 5 * (size_t)m.Nl * (c.precision == NUMA_FP32_MIXED ? 4 : 8);
}

size_t layout_workspace(const numa_config& c, const HostMesh& m, char* base, DevLayout* L) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off = align_up(off + bytes);
    return p;
  };
  const size_t Ng = (size_t)m.Ng, Nl = (size_t)m.Nl, PP = (size_t)m.P * m.P;
  DevLayout d;
  d.flags = (int*)take(64 * sizeof(int));
  d.q = (double*)take(5 * Ng * 8);
  d.qs = (double*)take(5 * Ng * 8);
  d.prim = take(prim_bytes_per_node(c.precision) * Ng);
  d.re = take(residual_bytes(c, m));
  if (c.precision == NUMA_FP32_MIXED) d.met32 = (float*)take(10 * Nl * 4);
  else if (c.precision == NUMA_FP64_PAIRS) d.met2 = (float2*)take(10 * Nl * 8);
  else d.met64 = (double*)take(10 * Nl * 8);
  d.l2g = (int32_t*)take(Nl * 4);
  d.csr_off = (int32_t*)take((Ng + 1) * 4);
  d.csr_idx = (int32_t*)take((size_t)m.nentries * 4);
  d.dss_order = (uint8_t*)take((Ng + kDssBlock - 1) / kDssBlock * kDssBlock);
  d.ref = (double*)take(4 * Ng * 8);
  d.Minv = (double*)take(Ng * 8);
  d.wall = (uint8_t*)take(Ng);
  if (c.mesh_kind == NUMA_MESH_SHELL) {
    d.gvec = (double*)take(3 * Ng * 8);
    d.nrm = (double*)take(3 * Ng * 8);
  }
  d.D64 = (double*)take(PP * 8);
  if ((c.precision == NUMA_FP64 || c.precision == NUMA_FP64_PAIRS) && affine_elements(c)) {
    d.affk = (double*)take(3 * (size_t)m.Ne * 8);
    d.Minv_r = (double*)take(Ng * 8);
  }
  d.D32 = (float*)take(PP * 4);
  d.D2 = (float2*)take(PP * 8);
  d.F64 = (double*)take(PP * 8);
  d.F32 = (float*)take(PP * 4);
  int nz = 0;
  long long ncol = 0;
  if (imex_supported(c, &ncol, &nz, nullptr)) {
    d.imex = (double*)take(imex_table_doubles(nz, c.N) * 8);
    d.imex_piv = (int*)take(6 * (size_t)nz * sizeof(int));
  }
  d.bytes = off;
  if (L) *L = d;
  return off;
}

// RHS with caller-chosen scratch for the primitive fields and the element
// residuals (used by numa_rhs_static_scratch): the scratch holds
// kPrimBytesPerNode * Ng bytes of primitives, 256-byte aligned, then the
// residuals.
int rhs_with_scratch(numa_ctx* c, const double* q_dev, double* r_dev, double* scratch, long long scratch_doubles) {
  if (!c || !q_dev || !r_dev || !scratch) return NUMA_EINVAL;
  if (!c->bound) return fail(c, NUMA_ESTATE, "numa_rhs_static_scratch before numa_bind");
  if ((const void*)q_dev == (const void*)r_dev) return fail(c, NUMA_EINVAL, "q and r must not alias");
  const size_t prim_bytes = align_up(prim_bytes_per_node(c->cfg.precision) * (size_t)c->mesh.Ng);
  const size_t need = prim_bytes + residual_bytes(c->cfg, c->mesh);
  if (need > 8 * (size_t)scratch_doubles)
    return fail(c, NUMA_EINVAL, "mesh needs " + std::to_string(need) + " bytes of scratch; the static array holds " +
                                    std::to_string(8 * scratch_doubles));
  char* base = reinterpret_cast<char*>(scratch);
  cudaError_t e = enqueue_rhs(c, q_dev, r_dev, base, base + prim_bytes);
  if (e != cudaSuccess) return cuda_fail(c, e, "numa_rhs_static_scratch launch");
  return NUMA_OK;
}

}  // namespace numa

extern "C" {

int numa_create(const numa_config* cfg, numa_ctx** out) {
  if (!out) return NUMA_EINVAL;
  *out = nullptr;
  if (!cfg) return NUMA_EINVAL;
  if (cfg->precision != NUMA_FP64 && cfg->precision != NUMA_FP32_MIXED && cfg->precision != NUMA_FP64_PAIRS)
    return NUMA_EINVAL;
  if (cfg->metric_form != NUMA_METRIC_AUTO && cfg->metric_form != NUMA_METRIC_NODAL) return NUMA_EINVAL;
  if (cfg->storage != NUMA_STORAGE_CG && cfg->storage != NUMA_STORAGE_DG) return NUMA_EINVAL;
  if (!(cfg->cv > 0) || !(cfg->cp > cfg->cv) || !(cfg->Rd > 0) || !(cfg->P00 > 0)) return NUMA_EINVAL;
  numa_ctx* c = new (std::nothrow) numa_ctx();
  if (!c) return NUMA_ENOMEM;
  c->cfg = *cfg;
  c->gamma = cfg->cp / cfg->cv;
  // binomial coefficients C(gamma, k) of (1+x)^gamma - 1 = sum_k C(gamma,k) x^k
  double ck = 1.0;
  for (int k = 1; k <= kEosTerms; ++k) {
    ck *= (c->gamma - (k - 1)) / k;
    c->eos[k - 1] = ck;
  }
  try {
    if (!build_host_mesh(c->cfg, c->mesh, c->err)) {
      delete c;
      return NUMA_EINVAL;
    }
    if (cfg->storage == NUMA_STORAGE_DG) {
      if (c->mesh.Nl * 8 > 0x7fffffffLL) {  // DG CSR entries stay below 2^31 (at most 8 per node)
        delete c;
        return NUMA_EINVAL;
      }
      expand_to_dg_storage(c->mesh);
    }
  } catch (const std::bad_alloc&) {
    delete c;
    return NUMA_ENOMEM;
  }
  *out = c;
  return NUMA_OK;
}

int numa_get_mesh_info(const numa_ctx* c, numa_mesh_info* info) {
  if (!c || !info) return NUMA_EINVAL;
  info->Ne = c->mesh.Ne;
  info->Nl = c->mesh.Nl;
  info->Ng = c->mesh.Ng;
  info->N = c->mesh.N;
  info->dss_entries = c->mesh.nentries;
  info->workspace_bytes = layout_workspace(c->cfg, c->mesh, nullptr, nullptr);
  return NUMA_OK;
}

int numa_bind(numa_ctx* c, void* ws, size_t bytes, void* stream) {
  if (!c) return NUMA_EINVAL;
  if (!ws) return fail(c, NUMA_EINVAL, "workspace is NULL");
  if (((uintptr_t)ws) % kAlign) return fail(c, NUMA_EINVAL, "workspace must be 256-byte aligned");
  size_t need = layout_workspace(c->cfg, c->mesh, nullptr, nullptr);
  if (bytes < need) return fail(c, NUMA_ENOMEM, "workspace smaller than workspace_bytes");
  DevLayout L;
  layout_workspace(c->cfg, c->mesh, (char*)ws, &L);
  cudaStream_t s = (cudaStream_t)stream;
  const HostMesh& m = c->mesh;
  const size_t Ng = (size_t)m.Ng, Nl = (size_t)m.Nl;
  cudaError_t e = cudaSuccess;
  auto up = [&](void* dst, const void* src, size_t n) {
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s);
  };
  std::vector<float> met32, D32, D2;
  // (hi, lo) float pairs of FP64 values: hi = nearest float, lo = nearest
  // float of the remainder
  auto pairs_of = [](const std::vector<double>& v) {
    std::vector<float> out(2 * v.size());
    for (size_t t = 0; t < v.size(); ++t) {
      const float h = (float)v[t];
      out[2 * t] = h;
      out[2 * t + 1] = (float)(v[t] - (double)h);
    }
    return out;
  };
  if (c->cfg.precision == NUMA_FP32_MIXED) {
    met32.resize(m.met.size());
    for (size_t t = 0; t < m.met.size(); ++t) met32[t] = (float)m.met[t];
    up(L.met32, met32.data(), met32.size() * 4);
  } else if (c->cfg.precision == NUMA_FP64_PAIRS) {
    if (affine_elements(c->cfg)) {
      met32 = pairs_of(m.met);
    } else {
      // the per-node pairs form reads rows 0..8 as -Jw dxi_d/dx_c (row 9,
      // Jw itself, stays for the filter): weighted in FP64, then split
      std::vector<double> wm(m.met);
      for (size_t n = 0; n < Nl; ++n) {
        const double jw = m.met[9 * Nl + n];
        for (int t = 0; t < 9; ++t) wm[t * Nl + n] = -jw * m.met[t * Nl + n];
      }
      met32 = pairs_of(wm);
    }
    up(L.met2, met32.data(), met32.size() * 4);
  } else {
    up(L.met64, m.met.data(), m.met.size() * 8);
  }
  D32.resize(m.D.size());
  for (size_t t = 0; t < m.D.size(); ++t) D32[t] = (float)m.D[t];
  D2 = pairs_of(m.D);
  up(L.D64, m.D.data(), m.D.size() * 8);
  up(L.D32, D32.data(), D32.size() * 4);
  up(L.D2, D2.data(), D2.size() * 4);
  if (e == cudaSuccess) e = upload_d32_constant(m.N, D32.data(), s);
  // FP64 and pairs: the per-element constants of rectilinear elements; FP64:
  // the weighted metric of the per-node form, which it takes everywhere else
  std::vector<double> affk, w3, Minv_r;
  bool rect = false;
  if (c->cfg.precision == NUMA_FP64 || c->cfg.precision == NUMA_FP64_PAIRS) {
    if (affine_elements(c->cfg)) {
      const int P = m.P;
      rect = rectilinear_elements(m);
      affk.assign(3 * (size_t)m.Ne, 0.0);
      const double w0 = m.w[0];
      for (long long el = 0; el < m.Ne; ++el) {
        const long long n = el * m.Np;
        const double J = m.met[9 * Nl + n] / (w0 * w0 * w0);
        for (int d = 0; d < 3; ++d) affk[d * (size_t)m.Ne + el] = -J * m.met[(4 * d) * Nl + n];
      }
      w3.resize((size_t)P * P * P);
      for (int k = 0; k < P; ++k)
        for (int j = 0; j < P; ++j)
          for (int i = 0; i < P; ++i) w3[i + P * (j + P * k)] = m.w[i] * m.w[j] * m.w[k];
      // Minv_r: w_i w_j w_k of the node's first element node (its DSS list
      // is ascending), times 1/M.  Lobatto weights are symmetric, so every
      // element node of a global node of a box has that weight; a mesh
      // where they differ is not treated as rectilinear (volume_form).
      if (rect) {
        const long long Np = m.Np;
        Minv_r.resize((size_t)Ng);
        for (size_t I = 0; I < Ng && rect; ++I) {
          const double wf = w3[m.csr_idx[m.csr_off[I]] % Np];
          for (int32_t t = m.csr_off[I] + 1; t < m.csr_off[I + 1]; ++t)
            if (std::fabs(w3[m.csr_idx[t] % Np] - wf) > 1e-14 * wf) rect = false;
          Minv_r[I] = wf * m.Minv[I];
        }
      }
      up(L.affk, affk.data(), affk.size() * 8);
      if (rect) up(L.Minv_r, Minv_r.data(), Minv_r.size() * 8);
    }
    if (c->cfg.precision == NUMA_FP64 && !rect) {
      if (e == cudaSuccess && Nl)
        weight_metric_kernel<<<(unsigned)((Nl + 255) / 256), 256, 0, s>>>(L.met64, (long long)Nl);
      if (e == cudaSuccess) e = cudaGetLastError();
    }
  }
  up(L.l2g, m.l2g.data(), Nl * 4);
  up(L.csr_off, m.csr_off.data(), (Ng + 1) * 4);
  up(L.csr_idx, m.csr_idx.data(), m.csr_idx.size() * 4);
  up(L.dss_order, m.dss_order.data(), m.dss_order.size());
  up(L.ref, m.ref.data(), 4 * Ng * 8);
  up(L.Minv, m.Minv.data(), Ng * 8);
  up(L.wall, m.wall.data(), Ng);
  if (L.gvec) up(L.gvec, m.gvec.data(), 3 * Ng * 8);
  if (L.nrm) up(L.nrm, m.nrm.data(), 3 * Ng * 8);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.flags, 0, 64 * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.q, 0, 5 * Ng * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.qs, 0, 5 * Ng * 8, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "numa_bind upload");
  c->L = L;
  c->rect = rect;
  c->slabs = plan_slabs(c->cfg, m, c->nslab_req);
  if (c->slabs.S > 1) {
    e = ensure_slab_streams(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "numa_bind slab stream and events");
  }
  // kernel attributes are set outside any stream capture
  VolumeArgs probe = volume_args(c, L.q, L.prim, L.re);
  probe.ecnt = 0;
  e = launch_volume(m.N, c->cfg.precision, probe, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "numa_bind kernel setup");
  c->stream = s;
  c->bound = true;
  c->prim_valid = false;
  c->imex_started = false;
  c->imex_factored = false;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  if (c->fgraph) {
    cudaGraphExecDestroy(c->fgraph);
    c->fgraph = nullptr;
  }
  if (c->filter_set) {
    e = upload_filter(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "numa_bind filter upload");
  }
  return NUMA_OK;
}

int numa_init_state(numa_ctx* c, int kind, const double* params, int nparams) {
  if (!c) return NUMA_EINVAL;
  if (!c->bound) return fail(c, NUMA_ESTATE, "numa_init_state before numa_bind");
  if (nparams < 0 || (nparams > 0 && !params)) return fail(c, NUMA_EINVAL, "bad params");
  std::vector<double> q;
  try {
    q.resize(5 * (size_t)c->mesh.Ng);
  } catch (const std::bad_alloc&) {
    return fail(c, NUMA_ENOMEM, "host allocation");
  }
  if (!init_state_host(c->cfg, c->mesh, kind, params, nparams, q.data(), c->err)) return NUMA_EINVAL;
  c->prim_valid = false;
  c->filter_count = 0;
  c->imex_started = false;
  cudaError_t e = cudaMemcpyAsync(c->L.q, q.data(), q.size() * 8, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "numa_init_state upload");
  return NUMA_OK;
}

int numa_set_state(numa_ctx* c, const double* q, int on_device) {
  if (!c || !q) return NUMA_EINVAL;
  if (!c->bound) return fail(c, NUMA_ESTATE, "numa_set_state before numa_bind");
  c->prim_valid = false;
  c->filter_count = 0;
  c->imex_started = false;
  cudaError_t e;
  if (on_device) {
    // one pass: copy the state in and form its primitive fields (which the
    // next step's first element kernel needs)
    PrimArgs a = prim_args(c, q, c->L.prim);
    a.qcopy = c->L.q;
    e = launch_prim(a, c->stream);
    if (e == cudaSuccess) c->prim_valid = true;
  } else {
    e = cudaMemcpyAsync(c->L.q, q, 5 * (size_t)c->mesh.Ng * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "numa_set_state");
  return NUMA_OK;
}

int numa_get_state(numa_ctx* c, double* q, int on_device) {
  if (!c || !q) return NUMA_EINVAL;
  if (!c->bound) return fail(c, NUMA_ESTATE, "numa_get_state before numa_bind");
  cudaError_t e = cudaMemcpyAsync(q, c->L.q, 5 * (size_t)c->mesh.Ng * 8,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "numa_get_state");
  return NUMA_OK;
}

int numa_rhs(numa_ctx* c, const double* q_dev, double* r_dev) {
  if (!c || !q_dev || !r_dev) return NUMA_EINVAL;
  if (!c->bound) return fail(c, NUMA_ESTATE, "numa_rhs before numa_bind");
  if ((const void*)q_dev == (const void*)r_dev) return fail(c, NUMA_EINVAL, "q and r must not alias");
  c->prim_valid = false;  // the primitive scratch now describes q_dev
  cudaError_t e = enqueue_rhs(c, q_dev, r_dev, c->L.prim, c->L.re);
  if (e != cudaSuccess) return cuda_fail(c, e, "numa_rhs launch");
  return NUMA_OK;
}

int numa_rk_step(numa_ctx* c, double dt) {
  if (!c) return NUMA_EINVAL;
  if (!c->bound) return fail(c, NUMA_ESTATE, "numa_rk_step before numa_bind");
  if (!std::isfinite(dt)) return fail(c, NUMA_EINVAL, "dt must be finite");
  cudaError_t e = ensure_prim(c);
  if (c->rk_scheme == NUMA_LEAPFROG_IMEX) {
    if (e == cudaSuccess) {
      const int rc = imex_prepare(c, dt);
      if (rc != NUMA_OK) return rc;
      e = enqueue_imex_step(c, dt, !c->imex_started, c->stream);
    }
    if (e == cudaSuccess) c->imex_started = true;
  } else if (e == cudaSuccess) {
    e = enqueue_rk_step(c, dt, c->stream);
  }
  if (e == cudaSuccess && c->filter_every > 0 && ++c->filter_count == c->filter_every) {
    e = enqueue_filter(c, c->stream);
    c->filter_count = 0;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "numa_rk_step launch");
  return NUMA_OK;
}

int numa_run(numa_ctx* c, double dt, int nsteps) {
  if (!c) return NUMA_EINVAL;
  if (!c->bound) return fail(c, NUMA_ESTATE, "numa_run before numa_bind");
  if (nsteps < 0 || !std::isfinite(dt)) return fail(c, NUMA_EINVAL, "bad nsteps or dt");
  cudaError_t e = cudaSuccess;
  const bool imex = c->rk_scheme == NUMA_LEAPFROG_IMEX;
  if (imex && nsteps > 0) {
    const int rc = imex_prepare(c, dt);
    if (rc != NUMA_OK) return rc;
  }
  if (!c->graph || c->graph_dt != dt || c->graph_q != c->L.q) {
    if (c->graph) {
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
    if (!c->cap_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t el = imex ? enqueue_imex_step(c, dt, false, c->cap_stream) : enqueue_rk_step(c, dt, c->cap_stream);
      e = cudaStreamEndCapture(c->cap_stream, &g);
      if (el != cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "numa_run graph capture");
    c->graph_dt = dt;
    c->graph_q = c->L.q;
  }
  if (c->filter_every > 0 && (!c->fgraph || c->fgraph_q != c->L.q)) {
    if (c->fgraph) {
      cudaGraphExecDestroy(c->fgraph);
      c->fgraph = nullptr;
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t el = enqueue_filter(c, c->cap_stream);
      e = cudaStreamEndCapture(c->cap_stream, &g);
      if (el != cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->fgraph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "numa_run filter graph capture");
    c->fgraph_q = c->L.q;
  }
  if (nsteps > 0) e = ensure_prim(c);
  for (int t = 0; t < nsteps && e == cudaSuccess; ++t) {
    if (imex && !c->imex_started) {  // the start step, outside the graph
      e = enqueue_imex_step(c, dt, true, c->stream);
      c->imex_started = e == cudaSuccess;
    } else {
      e = cudaGraphLaunch(c->graph, c->stream);
    }
    if (e == cudaSuccess && c->filter_every > 0 && ++c->filter_count == c->filter_every) {
      e = cudaGraphLaunch(c->fgraph, c->stream);
      c->filter_count = 0;
    }
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "numa_run graph launch");
  int flag = 0;
  int rc = numa_check_finite(c, &flag);
  if (rc != NUMA_OK) return rc;
  if (flag) return fail(c, NUMA_ENONFINITE, "non-finite state");
  return NUMA_OK;
}

int numa_time_kernels(numa_ctx* c, double dt, int nsteps, double* ms_volume, double* ms_update) {
  if (!c || !ms_volume || !ms_update) return NUMA_EINVAL;
  if (!c->bound) return fail(c, NUMA_ESTATE, "numa_time_kernels before numa_bind");
  if (nsteps < 0 || !std::isfinite(dt)) return fail(c, NUMA_EINVAL, "bad nsteps or dt");
  const int ns = rk_stages(c);
  std::vector<cudaEvent_t> ev(4 * (size_t)ns * nsteps, nullptr);
  cudaError_t e = ensure_prim(c);
  for (auto& x : ev)
    if (e == cudaSuccess) e = cudaEventCreate(&x);
  if (c->rk_scheme == NUMA_LEAPFROG_IMEX && e == cudaSuccess && nsteps > 0) {
    const int rc = imex_prepare(c, dt);
    if (rc != NUMA_OK) {
      for (auto& x : ev)
        if (x) cudaEventDestroy(x);
      return rc;
    }
  }
  for (int t = 0; t < nsteps && e == cudaSuccess; ++t) {
    if (c->rk_scheme == NUMA_LEAPFROG_IMEX) {
      e = enqueue_imex_step(c, dt, !c->imex_started, c->stream, &ev[4 * (size_t)t]);
      if (e == cudaSuccess) c->imex_started = true;
    } else {
      e = enqueue_rk_step(c, dt, c->stream, &ev[4 * (size_t)ns * t]);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  double tv = 0.0, tu = 0.0;
  for (size_t t = 0; t < (size_t)ns * nsteps && e == cudaSuccess; ++t) {
    float a = 0.f, b = 0.f;
    e = cudaEventElapsedTime(&a, ev[4 * t], ev[4 * t + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[4 * t + 2], ev[4 * t + 3]);
    tv += a;
    tu += b;
  }
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  if (e != cudaSuccess) return cuda_fail(c, e, "numa_time_kernels");
  *ms_volume = tv;
  *ms_update = tu;
  return NUMA_OK;
}

int numa_check_finite(numa_ctx* c, int* flag) {
  if (!c || !flag) return NUMA_EINVAL;
  if (!c->bound) return fail(c, NUMA_ESTATE, "numa_check_finite before numa_bind");
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->L.flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess && h) e = cudaMemsetAsync(c->L.flags, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "numa_check_finite");
  *flag = h ? 1 : 0;
  return NUMA_OK;
}

int numa_get_coords(const numa_ctx* c, double* xyz) {
  if (!c || !xyz) return NUMA_EINVAL;
  std::memcpy(xyz, c->mesh.gxyz.data(), c->mesh.gxyz.size() * sizeof(double));
  return NUMA_OK;
}

const char* numa_last_error(const numa_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

int numa_set_filter(numa_ctx* c, int every, int s, double p, double mu) {
  if (!c) return NUMA_EINVAL;
  const int N = c->mesh.N;
  if (every < 0) return fail(c, NUMA_EINVAL, "filter: every must be >= 0");
  if (s < 0 || s > N + 1) return fail(c, NUMA_EINVAL, "filter: s must be in [0, N+1]");
  if (!(p > 0.0) || !std::isfinite(p)) return fail(c, NUMA_EINVAL, "filter: order p must be positive");
  if (!(mu >= 0.0 && mu <= 1.0)) return fail(c, NUMA_EINVAL, "filter: strength mu must be in [0, 1]");
  std::vector<double> F((size_t)(N + 1) * (N + 1));
  filter_matrix_host(N, c->mesh.xi.data(), c->mesh.w.data(), s, p, mu, F.data());
  c->filter_F = F;
  c->filter_set = true;
  c->filter_every = every;
  c->filter_s = s;
  c->filter_p = p;
  c->filter_mu = mu;
  c->filter_count = 0;
  if (c->bound) {
    cudaError_t e = upload_filter(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "numa_set_filter upload");
  }
  return NUMA_OK;
}

int numa_set_time_scheme(numa_ctx* c, int scheme) {
  if (!c) return NUMA_EINVAL;
  if (scheme != NUMA_RK_SSP3 && scheme != NUMA_RK_LS54 && scheme != NUMA_LEAPFROG_IMEX)
    return fail(c, NUMA_EINVAL, "unknown time scheme");
  if (scheme == NUMA_LEAPFROG_IMEX && !c->imex_tables) {
    std::string why;
    if (!imex_supported(c->cfg, &c->imex_ncol, nullptr, &why)) return fail(c, NUMA_EINVAL, why);
    if (!imex_operator(c->cfg, c->mesh, c->imex, why)) return fail(c, NUMA_EINVAL, why);
    c->imex_tables = true;
  }
  if (scheme != c->rk_scheme) c->imex_started = false;
  if (scheme != c->rk_scheme && c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->rk_scheme = scheme;
  return NUMA_OK;
}

int numa_set_slabs(numa_ctx* c, int nslabs, int* used) {
  if (!c) return NUMA_EINVAL;
  if (nslabs < 0 || nslabs > kMaxSlabs) return fail(c, NUMA_EINVAL, "slabs must be in [0, 16]");
  c->nslab_req = nslabs;
  const SlabPlan P = plan_slabs(c->cfg, c->mesh, nslabs);
  if (c->bound && P.S > 1) {
    cudaError_t e = ensure_slab_streams(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "numa_set_slabs stream and events");
  }
  if (c->bound) c->slabs = P;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  if (used) *used = c->bound ? c->slabs.S : P.S;
  return NUMA_OK;
}

int numa_set_robert_asselin(numa_ctx* c, double nu) {
  if (!c) return NUMA_EINVAL;
  if (!(nu >= 0.0 && nu < 0.5)) return fail(c, NUMA_EINVAL, "Robert-Asselin strength must be in [0, 0.5)");
  if (nu != c->imex_nu && c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->imex_nu = nu;
  return NUMA_OK;
}

int numa_filter(numa_ctx* c) {
  if (!c) return NUMA_EINVAL;
  if (!c->bound) return fail(c, NUMA_ESTATE, "numa_filter before numa_bind");
  if (!c->filter_set) return fail(c, NUMA_ESTATE, "numa_filter before numa_set_filter");
  cudaError_t e = enqueue_filter(c, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "numa_filter launch");
  c->prim_valid = true;
  return NUMA_OK;
}

int numa_destroy(numa_ctx* c) {
  if (!c) return NUMA_EINVAL;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->fgraph) cudaGraphExecDestroy(c->fgraph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  for (int k = 0; k < kMaxSlabs; ++k) {
    if (c->ev_vol[k]) cudaEventDestroy(c->ev_vol[k]);
    if (c->ev_upd[k]) cudaEventDestroy(c->ev_upd[k]);
  }
  delete c;
  return NUMA_OK;
}

}  // extern "C"
