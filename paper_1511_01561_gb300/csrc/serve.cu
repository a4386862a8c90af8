// Ensemble-forecast serving on one GPU: continuous batching of RK3
// integrations of many independent members (meshes of different sizes,
// orders and precisions) over one caller-owned device arena.
//
//  - numa_sched_submit queues a request; a pool of host threads builds its
//    mesh (numa_create) in the background.
//  - numa_sched_step admits built requests in arrival order while their
//    workspace fits in the arena (first-fit allocator, 256-byte blocks),
//    advances every admitted member by one SSP-RK3 step, and retires the
//    members that reached their step count (their final state is copied to
//    pinned host memory; the arena block is released once that copy ends).
//  - All admitted members advance together: per group of members with the
//    same order, precision and mesh kind, one persistent ragged kernel per
//    stage covers all their elements and one all their global nodes.  The
//    per-step launches are captured once in a CUDA graph that reads the
//    member and group tables from device memory, so admission and retirement
//    rewrite the tables, not the graph (the graph is recaptured only when the
//    set of groups changes).
#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "numa_internal.h"

using namespace numa;

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxGroups = 16;
constexpr size_t kMaxInflight = 3;
// Captured streams of one serving step: groups run as independent branches
// of the step graph (round-robin over this many streams, the capture stream
// included), so that one group's kernels fill the SMs another leaves idle
// (the tail of a persistent launch, a small group, an FP64-pipe-bound group
// beside a memory-bound one).
constexpr int kBranches = 4;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over [0, size) with coalescing of free blocks.
class Arena {
 public:
  void init(size_t size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
 private:
  std::map<size_t, size_t> free_;
};

struct Request {
  long long id = 0;
  numa_config cfg{};
  int ic = 0;
  double params[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int nparams = 0;
  double dt = 0.0;
  int nsteps = 0;
  int status = NUMA_REQ_QUEUED;
  int steps_done = 0;
  size_t ws_bytes = 0;
  size_t ws_off = 0;
  numa_ctx* ctx = nullptr;
  int slot = -1;
  double* result = nullptr;  // pinned, 5*Ng doubles, once retired
  int* flag = nullptr;       // pinned copy of the non-finite flag
  cudaEvent_t done = nullptr;
  std::string err;
};

using GroupKey = std::tuple<int, int, int, int>;  // N, precision, mesh kind, element-kernel form (volume_form)

// Workspace bytes of a configuration without building its mesh.
bool workspace_bytes_of(const numa_config& c, size_t* bytes, long long* Ng) {
  if (c.N < 1 || c.N > kMaxN) return false;
  HostMesh m;
  m.N = c.N;
  m.P = c.N + 1;
  m.Np = m.P * m.P * m.P;
  if (c.mesh_kind == NUMA_MESH_BOX) {
    if (c.nex < 1 || c.ney < 1 || c.nez < 1) return false;
    m.Ne = (long long)c.nex * c.ney * c.nez;
    m.Ng = ((long long)c.nex * c.N + (c.periodic[0] ? 0 : 1)) * ((long long)c.ney * c.N + (c.periodic[1] ? 0 : 1)) *
           ((long long)c.nez * c.N + (c.periodic[2] ? 0 : 1));
  } else if (c.mesh_kind == NUMA_MESH_SHELL) {
    if (c.npanel < 1 || c.nlayer < 1) return false;
    m.Ne = 6LL * c.npanel * c.npanel * c.nlayer;
    const long long K = (long long)c.npanel * c.N;
    m.Ng = (6 * K * K + 2) * ((long long)c.nlayer * c.N + 1);
  } else {
    return false;
  }
  m.Nl = m.Ne * m.Np;
  m.nentries = m.Nl;  // CG storage: one CSR entry per element node
  *bytes = layout_workspace(c, m, nullptr, nullptr);
  *Ng = m.Ng;
  return true;
}

}  // namespace

struct numa_sched {
  char* arena = nullptr;
  size_t arena_bytes = 0;
  Arena alloc;
  cudaStream_t stream = nullptr;  // compute stream (caller's)
  cudaStream_t upload = nullptr;  // geometry uploads of newly admitted members
  cudaStream_t cap = nullptr;
  cudaStream_t branch[kBranches] = {};  // [0] unused: branch 0 is the capture stream
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kBranches] = {};
  // device tables (at the start of the arena) and their pinned host mirrors
  MemberDesc* d_desc = nullptr;
  RaggedGroup* d_groups = nullptr;
  MemberDesc* h_desc = nullptr;
  RaggedGroup* h_groups = nullptr;
  cudaEvent_t tables_copied = nullptr;
  bool tables_dirty = true;
  bool need_rebuild = false;  // members retired: rebuild the tables before the next launch
  std::deque<cudaEvent_t> inflight;  // one event per launched step, at most kMaxInflight
  std::vector<cudaEvent_t> spare_events;
  std::vector<GroupKey> groups;  // group index -> key
  std::vector<GroupKey> graph_groups;
  cudaGraphExec_t graph = nullptr;
  std::vector<int> free_slots;
  // requests
  std::mutex mu;
  std::condition_variable cv;
  bool stopping = false;
  std::deque<long long> to_build;
  std::vector<long long> built;  // built, waiting for admission (arrival order)
  std::vector<long long> active;
  std::vector<long long> retiring;
  std::map<long long, std::unique_ptr<Request>> reqs;
  long long next_id = 1;
  std::vector<std::thread> workers;
  std::string err;
};

namespace {

int sfail(numa_sched* s, int code, const std::string& msg) {
  if (s) s->err = msg;
  return code;
}

void build_worker(numa_sched* s) {
  for (;;) {
    long long id;
    numa_config cfg;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stopping || !s->to_build.empty(); });
      if (s->stopping) return;
      id = s->to_build.front();
      s->to_build.pop_front();
      cfg = s->reqs[id]->cfg;
    }
    numa_ctx* ctx = nullptr;
    const int rc = numa_create(&cfg, &ctx);
    std::lock_guard<std::mutex> lk(s->mu);
    Request& r = *s->reqs[id];
    if (r.status == NUMA_REQ_CANCELLED) {
      if (ctx) numa_destroy(ctx);
      continue;
    }
    if (rc != NUMA_OK) {
      r.status = NUMA_REQ_FAILED;
      r.err = "mesh setup failed";
      continue;
    }
    r.ctx = ctx;
    s->built.push_back(id);
    std::sort(s->built.begin(), s->built.end());
  }
}

// Member table entry for RK stage `stage`: the stage's volume input (q for
// the first stage, the stage state qs afterwards) and the update arguments
// of all three stages (the same as numa_rk_step uses).
void fill_desc(const Request& r, int stage, MemberDesc* d) {
  numa_ctx* c = r.ctx;
  double* q = c->L.q;
  double* qs = c->L.qs;
  const double* qin[3] = {q, qs, qs};
  double* qout[3] = {qs, qs, q};
  d->va = volume_args(c, qin[stage], c->L.prim, c->L.re);
  for (int st = 0; st < 3; ++st)
    d->ua[st] = update_args(c, c->L.re, qin[st], q, qout[st], 1, kRkA[st], kRkB[st], r.dt);
}

// Rebuild the group tables from the active members.
void rebuild_tables(numa_sched* s) {
  s->groups.clear();
  std::map<GroupKey, int> gi;
  for (int g = 0; g < kMaxGroups; ++g) s->h_groups[g].n = 0;
  for (long long id : s->active) {
    Request& r = *s->reqs[id];
    GroupKey k{r.cfg.N, r.cfg.precision, r.cfg.mesh_kind, volume_form(r.ctx)};
    auto it = gi.find(k);
    int g;
    if (it == gi.end()) {
      g = (int)s->groups.size();
      gi[k] = g;
      s->groups.push_back(k);
      s->h_groups[g].n = 0;
      s->h_groups[g].elem_prefix[0] = 0;
      s->h_groups[g].block_prefix[0] = 0;
    } else {
      g = it->second;
    }
    RaggedGroup& G = s->h_groups[g];
    const int m = G.n++;
    G.member[m] = r.slot;
    G.elem_prefix[m + 1] = G.elem_prefix[m] + r.ctx->mesh.Ne;
    G.block_prefix[m + 1] = G.block_prefix[m] + (r.ctx->mesh.Ng + kDssBlock - 1) / kDssBlock;
  }
  s->tables_dirty = true;
}

// One RK step of every group: 3 stages x (ragged volume, ragged update), each
// stage reading its own copy of the member table (the volume kernel's input
// state differs between the first and the later stages).  Groups share no
// member, so with more than one group each takes a branch stream forked
// from st and joined back into it (st being captured, the branches become
// parallel paths of the step graph).
cudaError_t enqueue_group(numa_sched* s, size_t g, cudaStream_t st) {
  const int N = std::get<0>(s->groups[g]), prec = std::get<1>(s->groups[g]);
  const bool shell = std::get<2>(s->groups[g]) == NUMA_MESH_SHELL;
  const bool affine = std::get<3>(s->groups[g]) != 0;
  for (int stage = 0; stage < 3; ++stage) {
    const MemberDesc* d = s->d_desc + (size_t)stage * kMaxMembers;
    cudaError_t e = launch_volume_ragged(N, prec, affine, d, s->d_groups + g, st);
    if (e == cudaSuccess) e = launch_update_ragged(prec, shell, stage, d, s->d_groups + g, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t enqueue_step(numa_sched* s, cudaStream_t st) {
  const size_t ng = s->groups.size();
  const int nb = ng < (size_t)kBranches ? (int)ng : kBranches;
  if (nb <= 1) return ng ? enqueue_group(s, 0, st) : cudaSuccess;
  cudaError_t e = cudaEventRecord(s->fork, st);
  for (int b = 1; b < nb && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(s->branch[b], s->fork, 0);
  for (size_t g = 0; g < ng && e == cudaSuccess; ++g) {
    const int b = (int)(g % (size_t)nb);
    e = enqueue_group(s, g, b ? s->branch[b] : st);
  }
  // join every branch that was forked, also after an error, so that the
  // capture ends cleanly
  for (int b = 1; b < nb; ++b) {
    cudaError_t ej = cudaEventRecord(s->join[b], s->branch[b]);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(st, s->join[b], 0);
    if (e == cudaSuccess) e = ej;
  }
  return e;
}

cudaError_t upload_tables(numa_sched* s) {
  if (!s->tables_dirty) return cudaSuccess;
  cudaError_t e = cudaEventSynchronize(s->tables_copied);  // mirror no longer in use
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_desc, s->h_desc, sizeof(MemberDesc) * 3 * kMaxMembers, cudaMemcpyHostToDevice,
                        s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_groups, s->h_groups, sizeof(RaggedGroup) * kMaxGroups, cudaMemcpyHostToDevice,
                        s->stream);
  if (e == cudaSuccess) e = cudaEventRecord(s->tables_copied, s->stream);
  if (e == cudaSuccess) s->tables_dirty = false;
  return e;
}

void release_member(numa_sched* s, Request& r) {
  if (r.ctx) {
    numa_destroy(r.ctx);
    r.ctx = nullptr;
  }
  if (r.ws_bytes) s->alloc.release(r.ws_off, r.ws_bytes);
  r.ws_bytes = 0;
  if (r.slot >= 0) s->free_slots.push_back(r.slot);
  r.slot = -1;
}

}  // namespace

extern "C" {

int numa_sched_create(void* dev_arena, size_t arena_bytes, void* stream, int build_threads, numa_sched** out) {
  if (!out) return NUMA_EINVAL;
  *out = nullptr;
  if (!dev_arena || ((uintptr_t)dev_arena) % kAlign) return NUMA_EINVAL;
  const size_t tables = align_up(sizeof(MemberDesc) * 3 * kMaxMembers) + align_up(sizeof(RaggedGroup) * kMaxGroups);
  if (arena_bytes <= tables) return NUMA_ENOMEM;
  numa_sched* s = new (std::nothrow) numa_sched();
  if (!s) return NUMA_ENOMEM;
  s->arena = static_cast<char*>(dev_arena);
  s->arena_bytes = arena_bytes;
  s->stream = (cudaStream_t)stream;
  s->d_desc = reinterpret_cast<MemberDesc*>(s->arena);
  s->d_groups = reinterpret_cast<RaggedGroup*>(s->arena + align_up(sizeof(MemberDesc) * 3 * kMaxMembers));
  s->alloc.init(arena_bytes - tables);
  cudaError_t e = cudaStreamCreateWithFlags(&s->upload, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
  for (int b = 1; b < kBranches && e == cudaSuccess; ++b) {
    e = cudaStreamCreateWithFlags(&s->branch[b], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->join[b], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s->h_desc, sizeof(MemberDesc) * 3 * kMaxMembers);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s->h_groups, sizeof(RaggedGroup) * kMaxGroups);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->tables_copied, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    numa_sched_destroy(s);
    return NUMA_ECUDA;
  }
  std::memset(s->h_desc, 0, sizeof(MemberDesc) * 3 * kMaxMembers);
  std::memset(s->h_groups, 0, sizeof(RaggedGroup) * kMaxGroups);
  for (int k = kMaxMembers - 1; k >= 0; --k) s->free_slots.push_back(k);
  const int nt = build_threads > 0 ? build_threads : 1;
  for (int t = 0; t < nt; ++t) s->workers.emplace_back(build_worker, s);
  *out = s;
  return NUMA_OK;
}

int numa_sched_submit(numa_sched* s, const numa_config* cfg, int ic_kind, const double* params, int nparams,
                      double dt, int nsteps, long long* id) {
  if (!s || !cfg || !id || nparams < 0 || nparams > 8 || (nparams && !params) || nsteps < 0 || !(dt == dt))
    return NUMA_EINVAL;
  if (cfg->storage != NUMA_STORAGE_CG) return sfail(s, NUMA_EINVAL, "serving takes CG storage only");
  size_t bytes = 0;
  long long Ng = 0;
  if (!workspace_bytes_of(*cfg, &bytes, &Ng)) return sfail(s, NUMA_EINVAL, "bad mesh configuration");
  const size_t tables = align_up(sizeof(MemberDesc) * 3 * kMaxMembers) + align_up(sizeof(RaggedGroup) * kMaxGroups);
  if (align_up(bytes) > s->arena_bytes - tables)
    return sfail(s, NUMA_EBUDGET, "request needs " + std::to_string(bytes) + " bytes, more than the arena");
  auto r = std::make_unique<Request>();
  r->cfg = *cfg;
  r->ic = ic_kind;
  r->nparams = nparams;
  for (int t = 0; t < nparams; ++t) r->params[t] = params[t];
  r->dt = dt;
  r->nsteps = nsteps;
  r->ws_bytes = 0;
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  *id = r->id;
  s->to_build.push_back(r->id);
  s->reqs[r->id] = std::move(r);
  s->cv.notify_one();
  return NUMA_OK;
}

int numa_sched_step(numa_sched* s, int* n_active, int* n_waiting) {
  if (!s) return NUMA_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  // the pinned table mirrors are rewritten below: wait for their last upload
  cudaError_t e = cudaEventSynchronize(s->tables_copied);
  if (e != cudaSuccess) return sfail(s, NUMA_ECUDA, std::string("numa_sched_step: ") + cudaGetErrorString(e));
  // 1. harvest retired members whose result copies have landed
  for (size_t t = 0; t < s->retiring.size();) {
    Request& r = *s->reqs[s->retiring[t]];
    if (cudaEventQuery(r.done) == cudaSuccess) {
      r.status = (*r.flag) ? NUMA_REQ_FAILED : NUMA_REQ_DONE;
      if (*r.flag) r.err = "non-finite state";
      release_member(s, r);
      s->retiring.erase(s->retiring.begin() + t);
    } else {
      ++t;
    }
  }
  // 2. admit built requests (arrival order) whose workspace fits
  bool changed = false;
  std::vector<long long> finished;
  for (size_t t = 0; t < s->built.size();) {
    Request& r = *s->reqs[s->built[t]];
    size_t bytes = 0;
    long long Ng = 0;
    workspace_bytes_of(r.cfg, &bytes, &Ng);
    size_t off = 0;
    if (s->free_slots.empty() || !s->alloc.alloc(bytes, &off)) {
      ++t;
      continue;
    }
    const size_t tables = align_up(sizeof(MemberDesc) * 3 * kMaxMembers) + align_up(sizeof(RaggedGroup) * kMaxGroups);
    r.ws_off = off;
    r.ws_bytes = bytes;
    r.slot = s->free_slots.back();
    s->free_slots.pop_back();
    numa_ctx* c = r.ctx;
    int rc = numa_bind(c, s->arena + tables + off, bytes, s->upload);
    if (rc == NUMA_OK) rc = numa_init_state(c, r.ic, r.params, r.nparams);
    if (rc == NUMA_OK) {
      e = ensure_prim(c);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->upload);
      if (e != cudaSuccess) rc = NUMA_ECUDA;
    }
    s->built.erase(s->built.begin() + t);
    if (rc != NUMA_OK) {
      r.status = NUMA_REQ_FAILED;
      r.err = numa_last_error(c);
      release_member(s, r);
      continue;
    }
    c->stream = s->stream;  // from now on the member runs on the compute stream
    for (int st = 0; st < 3; ++st) fill_desc(r, st, s->h_desc + (size_t)st * kMaxMembers + r.slot);
    r.status = NUMA_REQ_RUNNING;
    if (r.nsteps == 0) {  // nothing to integrate: its result is the initial state
      finished.push_back(r.id);
      continue;
    }
    s->active.push_back(r.id);
    changed = true;
  }
  // 3. advance every active member by one RK step
  if (!s->active.empty()) {
    if (changed || s->need_rebuild) {
      rebuild_tables(s);
      s->need_rebuild = false;
    }
    e = upload_tables(s);
    if (e == cudaSuccess && (!s->graph || s->graph_groups != s->groups)) {
      if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
      }
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t el = enqueue_step(s, s->cap);
        e = cudaStreamEndCapture(s->cap, &g);
        if (el != cudaSuccess) e = el;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&s->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e == cudaSuccess) s->graph_groups = s->groups;
    }
    // keep at most kMaxInflight steps queued ahead of the GPU, so that results
    // are harvested (and new requests admitted) close to real time
    while (e == cudaSuccess && s->inflight.size() >= kMaxInflight) {
      e = cudaEventSynchronize(s->inflight.front());
      s->spare_events.push_back(s->inflight.front());
      s->inflight.pop_front();
    }
    // (every active member has steps left: members retire on their last step)
    if (e == cudaSuccess) e = cudaGraphLaunch(s->graph, s->stream);
    if (e == cudaSuccess) {
      cudaEvent_t ev = nullptr;
      if (!s->spare_events.empty()) {
        ev = s->spare_events.back();
        s->spare_events.pop_back();
      } else {
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      }
      if (e == cudaSuccess) e = cudaEventRecord(ev, s->stream);
      if (e == cudaSuccess) s->inflight.push_back(ev);
    }
    if (e != cudaSuccess) return sfail(s, NUMA_ECUDA, std::string("numa_sched_step: ") + cudaGetErrorString(e));
    for (long long id : s->active) {
      Request& r = *s->reqs[id];
      if (++r.steps_done >= r.nsteps) finished.push_back(id);
    }
  }
  // 4. retire finished members: copy state and flag out, drop them from the tables
  for (long long id : finished) {
    Request& r = *s->reqs[id];
    const size_t n = 5 * (size_t)r.ctx->mesh.Ng;
    e = cudaMallocHost((void**)&r.result, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&r.flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.result, r.ctx->L.q, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.flag, r.ctx->L.flags, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(r.done, s->stream);
    if (e != cudaSuccess) return sfail(s, NUMA_ECUDA, std::string("numa_sched_step retire: ") + cudaGetErrorString(e));
    auto a = std::find(s->active.begin(), s->active.end(), id);
    if (a != s->active.end()) s->active.erase(a);
    s->retiring.push_back(id);
  }
  // The pinned table mirrors may still be in flight to the device for the
  // step just launched: rebuild them at the next step, after the upload event.
  if (!finished.empty()) s->need_rebuild = true;
  if (n_active) *n_active = (int)s->active.size();
  if (n_waiting) *n_waiting = (int)(s->built.size() + s->to_build.size() + s->retiring.size());
  return NUMA_OK;
}

int numa_sched_poll(numa_sched* s, long long id, int* status, int* steps_done, long long* Ng) {
  if (!s || !status) return NUMA_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(s, NUMA_EINVAL, "unknown request");
  *status = it->second->status;
  if (steps_done) *steps_done = it->second->steps_done;
  if (Ng) {
    size_t bytes = 0;
    workspace_bytes_of(it->second->cfg, &bytes, Ng);
  }
  return NUMA_OK;
}

int numa_sched_result(numa_sched* s, long long id, double* q_host, long long n) {
  if (!s || !q_host) return NUMA_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(s, NUMA_EINVAL, "unknown request");
  Request& r = *it->second;
  if (r.status != NUMA_REQ_DONE && r.status != NUMA_REQ_FAILED) return sfail(s, NUMA_ESTATE, "request not finished");
  if (!r.result) return sfail(s, NUMA_ESTATE, "no result (" + r.err + ")");
  long long ng = 0;
  size_t bytes = 0;
  workspace_bytes_of(r.cfg, &bytes, &ng);
  if (n != 5 * ng) return sfail(s, NUMA_EINVAL, "buffer must hold 5*Ng doubles");
  std::memcpy(q_host, r.result, sizeof(double) * (size_t)n);
  const int status = r.status;
  cudaFreeHost(r.result);
  cudaFreeHost(r.flag);
  if (r.done) cudaEventDestroy(r.done);
  s->reqs.erase(it);
  return status == NUMA_REQ_DONE ? NUMA_OK : sfail(s, NUMA_ENONFINITE, "non-finite state");
}

int numa_sched_cancel(numa_sched* s, long long id) {
  if (!s) return NUMA_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(s, NUMA_EINVAL, "unknown request");
  Request& r = *it->second;
  if (r.status != NUMA_REQ_QUEUED) return sfail(s, NUMA_ESTATE, "only queued requests can be cancelled");
  r.status = NUMA_REQ_CANCELLED;
  auto b = std::find(s->built.begin(), s->built.end(), id);
  if (b != s->built.end()) {
    s->built.erase(b);
    release_member(s, r);
  }
  auto q = std::find(s->to_build.begin(), s->to_build.end(), id);
  if (q != s->to_build.end()) s->to_build.erase(q);
  return NUMA_OK;
}

const char* numa_sched_last_error(const numa_sched* s) { return s ? s->err.c_str() : "null scheduler"; }

int numa_sched_destroy(numa_sched* s) {
  if (!s) return NUMA_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv.notify_all();
  for (auto& w : s->workers) w.join();
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto& kv : s->reqs) {
    Request& r = *kv.second;
    if (r.ctx) numa_destroy(r.ctx);
    if (r.result) cudaFreeHost(r.result);
    if (r.flag) cudaFreeHost(r.flag);
    if (r.done) cudaEventDestroy(r.done);
  }
  if (s->graph) cudaGraphExecDestroy(s->graph);
  for (cudaEvent_t ev : s->inflight) cudaEventDestroy(ev);
  for (cudaEvent_t ev : s->spare_events) cudaEventDestroy(ev);
  if (s->tables_copied) cudaEventDestroy(s->tables_copied);
  if (s->h_desc) cudaFreeHost(s->h_desc);
  if (s->h_groups) cudaFreeHost(s->h_groups);
  if (s->upload) cudaStreamDestroy(s->upload);
  if (s->cap) cudaStreamDestroy(s->cap);
  for (int b = 1; b < kBranches; ++b) {
    if (s->branch[b]) cudaStreamDestroy(s->branch[b]);
    if (s->join[b]) cudaEventDestroy(s->join[b]);
  }
  if (s->fork) cudaEventDestroy(s->fork);
  delete s;
  return NUMA_OK;
}

}  // extern "C"
