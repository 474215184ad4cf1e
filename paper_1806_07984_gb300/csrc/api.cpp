// C ABI of the ADER-DG step library: context, buffers, streams, dispatch.
#include "../../include/ader.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "basis.h"
#include "dispatch.h"
#include "kernels.h"
#include "mesh.h"
#include "partition.h"

using namespace ader;

struct ader_ctx {
  ader_config cfg{};
  int n = 0, NS = 0, NF = 0, M = 0;
  Tree tree;                  // the whole mesh (every rank of a partition keeps it)
  SubDomain dd;               // this rank's sub-domain once ader_partition ran
  bool partitioned = false;
  MeshLists* L = nullptr;     // lists the device step runs over: &tree or &dd.lists
  // halo exchange lists of the partition on the device (all peers
  // concatenated; host offsets per peer, in entries)
  int32_t *halo_send = nullptr, *halo_recv = nullptr;
  int64_t halo_send_cap = 0, halo_recv_cap = 0;
  std::vector<int64_t> send_off, recv_off;
  // state migration after a partitioned remesh: the transferred cells of the
  // old base-cell range (tree cells [stage_first, stage_first + stage_count))
  double* stage = nullptr;
  int64_t stage_cap = 0, stage_first = 0, stage_count = 0;
  std::vector<int64_t> old_base_cut;
  bool migrating = false;
  BasisTables B{};
  double inv_h[kMaxLevels][3]{};
  cudaStream_t s_hi = nullptr, s_lo = nullptr;
  cudaStream_t s_copy = nullptr;          // host copies of ader_step_host (created on first use)
  std::vector<cudaEvent_t> ev_copy;       // one per copied cell range
  cudaEvent_t ev_begin = nullptr, ev_step = nullptr, ev_lo = nullptr, ev_end = nullptr;
  // device buffers (capacity in cells)
  int64_t cap = 0;
  double *u = nullptr, *ustar = nullptr, *faceQ = nullptr, *faceF = nullptr, *fstar = nullptr;
  int8_t* level = nullptr;
  int32_t *all_cells = nullptr, *skel_cells = nullptr, *encl_cells = nullptr;
  int32_t* corr_cells = nullptr;         // cells grouped by pipeline stage (Tree::corr_cells)
  std::vector<cudaEvent_t> ev_chunk;     // one per enclave chunk
  ConfFace* conf = nullptr;
  int64_t conf_cap = 0;
  ParentFace* parents = nullptr;
  int32_t* child_fine = nullptr;
  int64_t par_cap = 0;
  unsigned long long* rate = nullptr;
  uint32_t* status = nullptr;
  double* dt_scratch = nullptr;
  // subcell FV limiter (cfg.limiter): backup of u(T), subcell bounds, flags,
  // lists, neighbour table, forced cells; the candidate stage reports into
  // rate_cand / status_cand
  SubcellTables T{};
  double *u_old = nullptr, *bounds = nullptr, *fv_scratch = nullptr;
  uint32_t* lim_flags = nullptr;
  int32_t *lim_list = nullptr, *fix_list = nullptr, *nbr = nullptr;
  uint8_t* force = nullptr;
  bool force_set = false;
  int* lim_counts = nullptr;
  unsigned long long* rate_cand = nullptr;
  uint32_t* status_cand = nullptr;
  int num_sms = 0;
  cudaGraphExec_t step_exec = nullptr;  // one captured step for the current mesh
  const double* graph_dt = nullptr;
  int64_t step_graph_launches = 0;
  bool graphs_ok = true;
  bool warm = false;  // an eager step ran since the mesh lists last changed
  TransferItem* plan_dev = nullptr;  // remesh transfer plan and child lists
  int32_t* kids_dev = nullptr;
  int64_t plan_cap = 0, kids_cap = 0;
  std::string err;
  int64_t launches = 0;
};

namespace {

int64_t ipow64(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

ader_status cuda_fail(ader_ctx* c, cudaError_t e, const char* what) {
  c->err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? ADER_ERR_OOM : ADER_ERR_CUDA;
}

#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e__ = (call);                            \
    if (e__ != cudaSuccess) return cuda_fail(c, e__, what); \
  } while (0)

cudaError_t do_predict(ader_ctx* c, const PredictArgs& a, cudaStream_t s) {
  const Precision p = static_cast<Precision>(int(c->cfg.prec));
  const int N = c->cfg.order;
  c->launches += a.count > 0 ? 1 : 0;
  if (p == Precision::kTF32 || p == Precision::kTF32x3 || p == Precision::kBF16x3)
    return predict_tc_euler3d(N, p, a, s);
  if (c->cfg.predictor == ADER_PREDICTOR_CK)
    return c->cfg.dim == 2 ? predict_ck_acoustics2d(N, p, a, s) : predict_ck_acoustics3d(N, p, a, s);
  if (c->cfg.pde == ADER_EULER)
    return c->cfg.dim == 2 ? predict_euler2d(N, p, a, s) : predict_euler3d(N, p, a, s);
  return c->cfg.dim == 2 ? predict_acoustics2d(N, p, a, s) : predict_acoustics3d(N, p, a, s);
}

cudaError_t do_faces(ader_ctx* c, int which, const RiemannArgs& a, cudaStream_t s) {
  const int N = c->cfg.order;
  const int64_t items = which == 0 ? a.nconf : a.nparents;
  c->launches += items > 0 ? 1 : 0;
  if (c->cfg.pde == ADER_EULER)
    return c->cfg.dim == 2 ? faces_euler2d(N, which, a, s) : faces_euler3d(N, which, a, s);
  return c->cfg.dim == 2 ? faces_acoustics2d(N, which, a, s) : faces_acoustics3d(N, which, a, s);
}

cudaError_t do_correct(ader_ctx* c, bool update, const CorrectArgs& a, cudaStream_t s) {
  const int N = c->cfg.order;
  c->launches += a.ncells > 0 ? 1 : 0;
  if (c->cfg.pde == ADER_EULER)
    return c->cfg.dim == 2 ? correct_euler2d(N, update, a, s) : correct_euler3d(N, update, a, s);
  return c->cfg.dim == 2 ? correct_acoustics2d(N, update, a, s)
                         : correct_acoustics3d(N, update, a, s);
}

cudaError_t do_transfer(ader_ctx* c, const TransferArgs& a, cudaStream_t s) {
  const int N = c->cfg.order;
  c->launches += a.ncells_new > 0 ? 1 : 0;
  if (c->cfg.pde == ADER_EULER)
    return c->cfg.dim == 2 ? transfer_euler2d(N, a, s) : transfer_euler3d(N, a, s);
  return c->cfg.dim == 2 ? transfer_acoustics2d(N, a, s) : transfer_acoustics3d(N, a, s);
}

// Fault injection for tests (ader_debug_fail_allocations): while >= 0, the
// number of device allocations that still succeed; once it reaches 0 every
// allocation of the library fails on the host with cudaErrorMemoryAllocation,
// without reaching the driver.
std::atomic<int> g_alloc_budget{-1};

cudaError_t dev_alloc(void** p, size_t bytes) {
  int b = g_alloc_budget.load();
  while (b >= 0) {
    if (b == 0) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
    if (g_alloc_budget.compare_exchange_weak(b, b - 1)) break;
  }
  return cudaMalloc(p, bytes);
}

// Capacity for `need` elements; the old buffer is released only once the new
// one exists (contents are not kept: callers upload after growing).
template <class T>
cudaError_t grow(T** p, int64_t* cap, int64_t need) {
  if (need <= *cap && *p) return cudaSuccess;
  const int64_t nc = std::max<int64_t>(need + need / 4, 16);
  void* q = nullptr;
  const cudaError_t e = dev_alloc(&q, sizeof(T) * size_t(nc));
  if (e != cudaSuccess) return e;
  if (*p) cudaFree(*p);
  *p = static_cast<T*>(q);
  *cap = nc;
  return cudaSuccess;
}

// Cell-sized buffers for `need` cells; u keeps its contents.  Every new
// buffer is allocated before any old one is released, so a failure leaves
// the context's buffers as they were.
ader_status ensure_cells(ader_ctx* c, int64_t need) {
  if (need <= c->cap) return ADER_OK;
  const int64_t nc = need + need / 4;
  const size_t cell_bytes = size_t(c->M) * c->NS * sizeof(double);
  const size_t face_bytes = size_t(2 * c->cfg.dim) * c->M * c->NF * sizeof(double);
  const size_t N = size_t(nc);
  std::vector<std::pair<void**, size_t>> req = {
      {(void**)&c->u, cell_bytes * N},        {(void**)&c->ustar, cell_bytes * N},
      {(void**)&c->faceQ, face_bytes * N},    {(void**)&c->faceF, face_bytes * N},
      {(void**)&c->fstar, face_bytes * N},    {(void**)&c->level, N},
      {(void**)&c->all_cells, 4 * N},         {(void**)&c->skel_cells, 4 * N},
      {(void**)&c->encl_cells, 4 * N},        {(void**)&c->corr_cells, 4 * N}};
  if (c->cfg.limiter) {
    req.insert(req.end(), {{(void**)&c->u_old, cell_bytes * N},
                           {(void**)&c->bounds, sizeof(double) * 2 * c->M * N},
                           {(void**)&c->lim_flags, sizeof(uint32_t) * N},
                           {(void**)&c->lim_list, 4 * N},
                           {(void**)&c->fix_list, 4 * N},
                           {(void**)&c->nbr, 4 * size_t(2 * c->cfg.dim) * N},
                           {(void**)&c->force, N}});
  }
  std::vector<void*> fresh(req.size(), nullptr);
  auto release = [&]() {
    for (void* p : fresh)
      if (p) cudaFree(p);
  };
  for (size_t i = 0; i < req.size(); ++i) {
    const cudaError_t e = dev_alloc(&fresh[i], req[i].second);
    if (e != cudaSuccess) {
      release();
      return cuda_fail(c, e, "cudaMalloc cell buffers");
    }
  }
  cudaError_t e = cudaSuccess;
  if (c->u) e = cudaMemcpy(fresh[0], c->u, cell_bytes * size_t(c->cap), cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess && c->cfg.limiter) {
    e = cudaMemset(fresh[12], 0, sizeof(uint32_t) * N);
    if (e == cudaSuccess) e = cudaMemset(fresh[16], 0, N);
  }
  if (e != cudaSuccess) {
    release();
    return cuda_fail(c, e, "copy cell buffers");
  }
  for (size_t i = 0; i < req.size(); ++i) {
    if (*req[i].first) cudaFree(*req[i].first);
    *req[i].first = fresh[i];
  }
  if (c->cfg.limiter) c->force_set = false;
  c->cap = nc;
  return ADER_OK;
}

// The captured step bakes in the mesh lists, their sizes and pointers.
void drop_step_graph(ader_ctx* c) {
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  c->step_exec = nullptr;
  c->warm = false;
}

// Upload levels, cell lists and face lists of the current tree (synchronous).
// Default enclave pipeline (cfg.pipeline_chunks == 0): 8 chunks, fewer when
// the enclave holds less than 8 predictor CTAs per SM per chunk, down to one
// chunk (no pipeline) for small meshes, whose steps are bound by the chain of
// short launches rather than by the predictor.
void fit_chunks(ader_ctx* c) {
  if (c->partitioned || c->cfg.pipeline_chunks != 0) return;
  const int64_t ns = ipow64(c->cfg.order + 1, c->cfg.dim);
  const int64_t cpb = ns >= 128 ? 1 : 256 / ns;  // cells per predictor CTA
  const int64_t ctas = (int64_t(c->tree.encl_cells.size()) + cpb - 1) / cpb;
  const int k = int(std::max<int64_t>(1, std::min<int64_t>(8, ctas / (8 * int64_t(std::max(1, c->num_sms))))));
  if (k != c->tree.chunks) c->tree.set_chunks(k);
}

ader_status upload_mesh(ader_ctx* c) {
  drop_step_graph(c);
  fit_chunks(c);
  const MeshLists& t = *c->L;
  const int64_t C = t.nlocal;
  ader_status st = ensure_cells(c, C);
  if (st != ADER_OK) return st;
  std::vector<int32_t> all(static_cast<size_t>(C));
  for (int64_t i = 0; i < C; ++i) all[size_t(i)] = int32_t(i);
  CK(cudaMemcpy(c->level, t.levels.data(), size_t(C), cudaMemcpyHostToDevice), "upload level");
  CK(cudaMemcpy(c->all_cells, all.data(), sizeof(int32_t) * size_t(C), cudaMemcpyHostToDevice),
     "upload cells");
  if (!t.skel_cells.empty())
    CK(cudaMemcpy(c->skel_cells, t.skel_cells.data(), sizeof(int32_t) * t.skel_cells.size(),
                  cudaMemcpyHostToDevice), "upload skeleton");
  if (!t.encl_cells.empty())
    CK(cudaMemcpy(c->encl_cells, t.encl_cells.data(), sizeof(int32_t) * t.encl_cells.size(),
                  cudaMemcpyHostToDevice), "upload enclave");
  if (!t.corr_cells.empty())
    CK(cudaMemcpy(c->corr_cells, t.corr_cells.data(), sizeof(int32_t) * t.corr_cells.size(),
                  cudaMemcpyHostToDevice), "upload corrector groups");
  CK(grow(&c->conf, &c->conf_cap, int64_t(t.conf.size())), "cudaMalloc conf");
  if (!t.conf.empty())
    CK(cudaMemcpy(c->conf, t.conf.data(), sizeof(ConfFace) * t.conf.size(), cudaMemcpyHostToDevice),
       "upload conf");
  const int64_t S = c->cfg.dim == 3 ? 9 : 3;
  int64_t pc_old = c->par_cap;
  CK(grow(&c->parents, &c->par_cap, int64_t(t.parents.size())), "cudaMalloc parents");
  if (c->par_cap != pc_old || !c->child_fine) {
    void* q = nullptr;
    CK(dev_alloc(&q, sizeof(int32_t) * size_t(c->par_cap * S)), "cudaMalloc children");
    if (c->child_fine) cudaFree(c->child_fine);
    c->child_fine = static_cast<int32_t*>(q);
  }
  if (!t.parents.empty()) {
    CK(cudaMemcpy(c->parents, t.parents.data(), sizeof(ParentFace) * t.parents.size(),
                  cudaMemcpyHostToDevice), "upload parents");
    CK(cudaMemcpy(c->child_fine, t.child_fine.data(), sizeof(int32_t) * t.child_fine.size(),
                  cudaMemcpyHostToDevice), "upload children");
  }
  if (c->partitioned) {
    const SubDomain& dd = c->dd;
    std::vector<int32_t> snd, rcv;
    c->send_off.assign(size_t(dd.nranks) + 1, 0);
    c->recv_off.assign(size_t(dd.nranks) + 1, 0);
    for (int q = 0; q < dd.nranks; ++q) {
      snd.insert(snd.end(), dd.send[size_t(q)].begin(), dd.send[size_t(q)].end());
      rcv.insert(rcv.end(), dd.recv[size_t(q)].begin(), dd.recv[size_t(q)].end());
      c->send_off[size_t(q) + 1] = int64_t(snd.size());
      c->recv_off[size_t(q) + 1] = int64_t(rcv.size());
    }
    CK(grow(&c->halo_send, &c->halo_send_cap, std::max<int64_t>(int64_t(snd.size()), 1)), "cudaMalloc halo");
    CK(grow(&c->halo_recv, &c->halo_recv_cap, std::max<int64_t>(int64_t(rcv.size()), 1)), "cudaMalloc halo");
    if (!snd.empty())
      CK(cudaMemcpy(c->halo_send, snd.data(), sizeof(int32_t) * snd.size(), cudaMemcpyHostToDevice),
         "upload halo");
    if (!rcv.empty())
      CK(cudaMemcpy(c->halo_recv, rcv.data(), sizeof(int32_t) * rcv.size(), cudaMemcpyHostToDevice),
         "upload halo");
  }
  if (c->cfg.limiter) {
    // conforming neighbour across each face, -1 across a resolution transition
    const int F = 2 * c->cfg.dim;
    std::vector<int32_t> nb(static_cast<size_t>(C) * F, -1);
    for (const ConfFace& f : t.conf) {
      nb[size_t(f.left) * F + 2 * f.dir + 1] = f.right;
      nb[size_t(f.right) * F + 2 * f.dir + 0] = f.left;
    }
    CK(cudaMemcpy(c->nbr, nb.data(), sizeof(int32_t) * nb.size(), cudaMemcpyHostToDevice),
       "upload neighbours");
  }
  return ADER_OK;
}

// Status word of the predictor, Riemann and corrector stages: with the
// limiter these produce a candidate, and its failures are the limiter's input.
uint32_t* stage_status(ader_ctx* c) { return c->cfg.limiter ? c->status_cand : c->status; }

PredictArgs predict_args(ader_ctx* c, const double* dt, ader_set set) {
  PredictArgs a{};
  a.u = c->u;
  a.ustar = c->ustar;
  a.faceQ = c->faceQ;
  a.faceF = c->faceF;
  if (set == ADER_SKELETON) {
    a.cells = c->skel_cells;
    a.count = int64_t(c->L->skel_cells.size());
  } else if (set == ADER_ENCLAVE) {
    a.cells = c->encl_cells;
    a.count = int64_t(c->L->encl_cells.size());
  } else {
    a.cells = c->all_cells;
    a.count = c->L->nowned;
  }
  a.level = c->level;
  a.dt = dt;
  a.gamma = c->cfg.gamma;
  a.iters = c->cfg.picard_iters > 0 ? c->cfg.picard_iters : c->cfg.order + 1;
  a.status = stage_status(c);
  a.min_ctas = 2 * c->num_sms;
  std::memcpy(a.inv_h, c->inv_h, sizeof(a.inv_h));
  a.B = c->B;
  return a;
}

RiemannArgs riemann_args(ader_ctx* c) {
  RiemannArgs a{};
  a.faceQ = c->faceQ;
  a.faceF = c->faceF;
  a.fstar = c->fstar;
  a.parents = c->parents;
  a.child_fine = c->child_fine;
  a.nparents = int64_t(c->L->parents.size());
  a.gamma = c->cfg.gamma;
  a.status = stage_status(c);
  a.B = c->B;
  return a;
}

CorrectArgs correct_args(ader_ctx* c, const double* dt) {
  CorrectArgs a{};
  a.ustar = c->ustar;
  a.fstar = c->fstar;
  a.u = c->u;
  a.level = c->level;
  a.ncells = c->L->nowned;
  a.dt = dt;
  a.rate_max = c->rate;
  a.gamma = c->cfg.gamma;
  a.status = c->status;
  std::memcpy(a.inv_h, c->inv_h, sizeof(a.inv_h));
  a.B = c->B;
  return a;
}

ader_status enqueue_riemann(ader_ctx* c, ader_set set, cudaStream_t s) {
  RiemannArgs a = riemann_args(c);
  const MeshLists& t = *c->L;
  if (set == ADER_ALL || set == ADER_SKELETON) {
    CK(do_faces(c, 1, a, s), "riemann child faces");
    if (c->cfg.dim == 2)  // in 3D the child-face kernel also restricts
      CK(do_faces(c, 2, a, s), "restriction");
  }
  if (set == ADER_SKELETON) {
    a.conf = c->conf;
    a.nconf = t.n_conf_skeleton;
  } else if (set == ADER_ENCLAVE) {
    a.conf = c->conf + t.n_conf_skeleton;
    a.nconf = int64_t(t.conf.size()) - t.n_conf_skeleton;
  } else {
    a.conf = c->conf;
    a.nconf = int64_t(t.conf.size());
  }
  a.nparents = 0;
  CK(do_faces(c, 0, a, s), "riemann conforming faces");
  return ADER_OK;
}

LimiterArgs limiter_args(ader_ctx* c, const double* dt) {
  LimiterArgs a{};
  a.u = c->u;
  a.u_old = c->u_old;
  a.u_backup = c->u_old;
  a.ustar = c->ustar;
  a.fstar = c->fstar;
  a.bounds = c->bounds;
  a.nbr = c->nbr;
  a.force = c->force_set ? c->force : nullptr;
  a.flags = c->lim_flags;
  a.list = c->lim_list;
  a.fix_list = c->fix_list;
  a.counts = c->lim_counts;
  a.level = c->level;
  a.ncells = c->L->nowned;
  a.dt = dt;
  a.gamma = c->cfg.gamma;
  a.delta0 = c->cfg.limiter_delta0 > 0.0 ? c->cfg.limiter_delta0 : 1e-4;
  a.eps = c->cfg.limiter_eps > 0.0 ? c->cfg.limiter_eps : 1e-3;
  a.rate_max = c->rate;
  a.status = c->status;
  a.fv_scratch = c->fv_scratch;
  std::memcpy(a.inv_h, c->inv_h, sizeof(a.inv_h));
  a.B = c->B;
  a.T = c->T;
  return a;
}

cudaError_t do_limiter(ader_ctx* c, LimiterKernel which, const LimiterArgs& a, int grid,
                       cudaStream_t s) {
  const int pde = c->cfg.pde == ADER_EULER ? 0 : 1;
  c->launches += 1;
  return c->cfg.dim == 2 ? launch_limiter_2d(c->cfg.order, pde, which, a, grid, s)
                         : launch_limiter_3d(c->cfg.order, pde, which, a, grid, s);
}

// Corrector arguments for a stage: the cell list (null = all cells), and in
// limiter mode the candidate's rate and status words.
CorrectArgs stage_correct_args(ader_ctx* c, const double* dt, const int32_t* cells, int64_t count) {
  CorrectArgs a = correct_args(c, dt);
  a.cells = cells;
  if (cells) a.ncells = count;
  if (c->cfg.limiter) {
    a.rate_max = c->rate_cand;
    a.status = c->status_cand;
  }
  return a;
}

// Limiter mode, before the first corrector of a step overwrites u(T): its
// backup and the subcell bounds.
ader_status enqueue_limiter_bounds(ader_ctx* c, const double* dt, cudaStream_t s) {
  CK(do_limiter(c, LimiterKernel::kBounds, limiter_args(c, dt), 2 * c->num_sms, s), "limiter bounds");
  return ADER_OK;
}

// After all correctors of a step: in limiter mode detection, FV on the
// limited cells, the neighbours' corrector with FV face fluxes and the CFL
// rate of the final state; then dt_next.
ader_status enqueue_finish(ader_ctx* c, const double* dt, double* dt_next, cudaStream_t s) {
  if (c->cfg.limiter) {
    const LimiterArgs la = limiter_args(c, dt);
    const int grid = 2 * c->num_sms;
    CK(cudaMemsetAsync(c->lim_counts, 0, 2 * sizeof(int), s), "clear limiter counts");
    CK(do_limiter(c, LimiterKernel::kDetect, la, grid, s), "limiter detection");
    CK(do_limiter(c, LimiterKernel::kFV, la, grid, s), "limiter FV step");
    CK(do_limiter(c, LimiterKernel::kFix, la, grid, s), "limiter neighbour correction");
    CorrectArgs r = correct_args(c, dt);
    CK(do_correct(c, false, r, s), "CFL rate");
  }
  c->launches += 1;
  CK(launch_finalize_dt(c->rate, c->cfg.cfl, dt_next, c->status, s), "finalize dt");
  return ADER_OK;
}

ader_status enqueue_correct(ader_ctx* c, const double* dt, double* dt_next, cudaStream_t s) {
  if (c->cfg.limiter) {
    ader_status st = enqueue_limiter_bounds(c, dt, s);
    if (st != ADER_OK) return st;
  }
  CK(do_correct(c, true, stage_correct_args(c, dt, nullptr, 0), s), "corrector");
  return enqueue_finish(c, dt, dt_next, s);
}

// This rank's sub-domain for the tree's current mesh under base_cut, uploaded.
ader_status rebuild_subdomain(ader_ctx* c, const std::vector<int64_t>& base_cut) {
  std::vector<int64_t> starts;
  if (!base_starts(c->tree, &starts)) {
    c->err = "the cell order does not follow the base cells";
    return ADER_ERR_MESH;
  }
  build_subdomain(c->tree, starts, base_cut, c->dd.rank, &c->dd);
  c->L = &c->dd.lists;
  return upload_mesh(c);
}

bool valid_config(const ader_config* cfg, std::string* why) {
  if (cfg->dim != 2 && cfg->dim != 3) return *why = "dim must be 2 or 3", false;
  if (cfg->order < 1 || cfg->order > 7) return *why = "order must be in 1..7", false;
  if (cfg->pde != ADER_EULER && cfg->pde != ADER_ACOUSTICS) return *why = "unknown pde", false;
  const int m = cfg->pde == ADER_EULER ? cfg->dim + 2 : cfg->dim + 1;
  if (cfg->nvar != m) return *why = "nvar does not match the pde", false;
  if (cfg->max_level < 0 || cfg->max_level > kMaxLevels - 2) return *why = "max_level out of range", false;
  if (cfg->prec < ADER_FP64 || cfg->prec > ADER_DF64) return *why = "unknown precision", false;
  if (cfg->prec >= ADER_TF32 && cfg->prec <= ADER_BF16X3 &&
      !(cfg->dim == 3 && cfg->pde == ADER_EULER && cfg->order >= 5))
    return *why = "tensor-core predictor: 3D Euler, order 5..7", false;
  if (!(cfg->cfl > 0.0)) return *why = "cfl must be positive", false;
  for (int d = 0; d < cfg->dim; ++d) {
    if (cfg->base[d] < 1) return *why = "base must be >= 1", false;
    if (!(cfg->hi[d] > cfg->lo[d])) return *why = "empty domain", false;
    int64_t cells = cfg->base[d];
    for (int l = 0; l < cfg->max_level; ++l) cells *= 3;
    if (cells >= (1 << 20)) return *why = "grid too fine for the cell key", false;
  }
  if (cfg->picard_iters < 0) return *why = "picard_iters must be >= 0", false;
  if (cfg->predictor != ADER_PREDICTOR_PICARD && cfg->predictor != ADER_PREDICTOR_CK)
    return *why = "unknown predictor", false;
  if (cfg->predictor == ADER_PREDICTOR_CK && (cfg->pde != ADER_ACOUSTICS || cfg->prec > ADER_FP32))
    return *why = "Cauchy-Kowalevski predictor: linear acoustics, FP64 or FP32", false;
  if (cfg->limiter != 0 && cfg->limiter != 1) return *why = "limiter must be 0 or 1", false;
  if (cfg->pipeline_chunks < 0 || cfg->pipeline_chunks > 64)
    return *why = "pipeline_chunks must be in 0..64", false;
  if (cfg->pipeline_ctas < 0 || cfg->pipeline_ctas > 32)
    return *why = "pipeline_ctas must be in 0..32", false;

  return true;
}

}  // namespace

extern "C" {

const char* ader_error_string(ader_status s) {
  switch (s) {
    case ADER_OK: return "ok";
    case ADER_ERR_ARG: return "invalid argument";
    case ADER_ERR_CUDA: return "CUDA error";
    case ADER_ERR_OOM: return "out of device memory";
    case ADER_ERR_NONPHYSICAL: return "non-physical state";
    case ADER_ERR_PICARD: return "non-finite predictor";
    case ADER_ERR_TIMEOUT: return "device wait timed out";
    case ADER_ERR_MESH: return "mesh error";
  }
  return "unknown status";
}

const char* ader_last_error(ader_ctx* c) { return c ? c->err.c_str() : "null context"; }

ader_status ader_init(const ader_config* cfg, ader_ctx** out) {
  if (!cfg || !out) return ADER_ERR_ARG;
  *out = nullptr;
  std::string why;
  if (!valid_config(cfg, &why)) return ADER_ERR_ARG;
  ader_ctx* c = new ader_ctx();
  c->cfg = *cfg;
  for (int d = cfg->dim; d < 3; ++d) {
    c->cfg.base[d] = 1;
    c->cfg.lo[d] = 0.0;
    c->cfg.hi[d] = 1.0;
  }
  c->n = cfg->order + 1;
  c->NS = int(ipow64(c->n, cfg->dim));
  c->NF = int(ipow64(c->n, cfg->dim - 1));
  c->M = cfg->nvar;
  make_basis(c->n, &c->B);
  for (int l = 0; l < kMaxLevels; ++l)
    for (int d = 0; d < 3; ++d)
      c->inv_h[l][d] = d < cfg->dim ? double(ipow64(3, l) * c->cfg.base[d]) /
                                          (c->cfg.hi[d] - c->cfg.lo[d])
                                    : 0.0;
  c->tree = Tree(cfg->dim, c->cfg.base, cfg->max_level);
  c->L = &c->tree;
  if (!c->tree.build()) {
    delete c;
    return ADER_ERR_MESH;
  }
  c->tree.set_chunks(cfg->pipeline_chunks == 0 ? 8 : cfg->pipeline_chunks);
  ader_status st = ADER_OK;
  auto fail = [&](ader_status s) {
    ader_destroy(c);
    return s;
  };
  int lo_prio = 0, hi_prio = 0;
  if (cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) != cudaSuccess) return fail(ADER_ERR_CUDA);
  if (cudaStreamCreateWithPriority(&c->s_hi, cudaStreamNonBlocking, hi_prio) != cudaSuccess ||
      cudaStreamCreateWithPriority(&c->s_lo, cudaStreamNonBlocking, lo_prio) != cudaSuccess)
    return fail(ADER_ERR_CUDA);
  for (cudaEvent_t* e : {&c->ev_begin, &c->ev_step, &c->ev_lo, &c->ev_end})
    if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return fail(ADER_ERR_CUDA);
  if (cudaMalloc(&c->rate, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&c->status, sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&c->dt_scratch, sizeof(double)) != cudaSuccess)
    return fail(ADER_ERR_OOM);
  if (cudaMemset(c->rate, 0, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(c->status, 0, sizeof(uint32_t)) != cudaSuccess)
    return fail(ADER_ERR_CUDA);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(ADER_ERR_CUDA);
  if (cfg->limiter) {
    make_subcells(c->n, &c->T);
    const int64_t slot = cfg->dim == 3 ? limiter_fv_scratch_3d(cfg->order, cfg->pde == ADER_EULER ? 0 : 1) : 0;
    if (slot > 0 && cudaMalloc(&c->fv_scratch, sizeof(double) * size_t(slot) * 2 * c->num_sms) != cudaSuccess)
      return fail(ADER_ERR_OOM);
    if (cudaMalloc(&c->lim_counts, 2 * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->rate_cand, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->status_cand, sizeof(uint32_t)) != cudaSuccess)
      return fail(ADER_ERR_OOM);
    if (cudaMemset(c->lim_counts, 0, 2 * sizeof(int)) != cudaSuccess ||
        cudaMemset(c->rate_cand, 0, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(c->status_cand, 0, sizeof(uint32_t)) != cudaSuccess)
      return fail(ADER_ERR_CUDA);
  }
  st = upload_mesh(c);
  if (st != ADER_OK) return fail(st);
  const size_t cell_bytes = size_t(c->M) * c->NS * sizeof(double);
  if (cudaMemset(c->u, 0, cell_bytes * size_t(c->L->nlocal)) != cudaSuccess) return fail(ADER_ERR_CUDA);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(ADER_ERR_CUDA);
  *out = c;
  return ADER_OK;
}

void ader_destroy(ader_ctx* c) {
  if (!c) return;
  if (c->s_hi) cudaStreamSynchronize(c->s_hi);
  if (c->s_lo) cudaStreamSynchronize(c->s_lo);
  drop_step_graph(c);
  for (void* p : {(void*)c->u, (void*)c->ustar, (void*)c->faceQ, (void*)c->faceF, (void*)c->fstar,
                  (void*)c->level, (void*)c->all_cells, (void*)c->skel_cells, (void*)c->encl_cells,
                  (void*)c->conf, (void*)c->parents, (void*)c->child_fine, (void*)c->rate,
                  (void*)c->status, (void*)c->dt_scratch, (void*)c->u_old, (void*)c->bounds,
                  (void*)c->lim_flags, (void*)c->lim_list, (void*)c->fix_list, (void*)c->nbr,
                  (void*)c->force, (void*)c->lim_counts, (void*)c->rate_cand,
                  (void*)c->status_cand, (void*)c->corr_cells, (void*)c->plan_dev,
                  (void*)c->kids_dev, (void*)c->fv_scratch, (void*)c->halo_send,
                  (void*)c->halo_recv, (void*)c->stage})
    if (p) cudaFree(p);
  for (cudaEvent_t e : c->ev_chunk)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : {c->ev_begin, c->ev_step, c->ev_lo, c->ev_end})
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_copy)
    if (e) cudaEventDestroy(e);
  if (c->s_hi) cudaStreamDestroy(c->s_hi);
  if (c->s_lo) cudaStreamDestroy(c->s_lo);
  if (c->s_copy) cudaStreamDestroy(c->s_copy);
  delete c;
}

ader_status ader_mesh_info(ader_ctx* c, int64_t* ncells, int64_t* nskel, int64_t* nconf,
                           int64_t* nparents) {
  if (!c) return ADER_ERR_ARG;
  if (ncells) *ncells = c->L->nowned;
  if (nskel) *nskel = int64_t(c->L->skel_cells.size());
  if (nconf) *nconf = int64_t(c->L->conf.size());
  if (nparents) *nparents = int64_t(c->L->parents.size());
  return ADER_OK;
}

ader_status ader_mesh_cells(ader_ctx* c, int32_t* out) {
  if (!c || !out) return ADER_ERR_ARG;
  const size_t first = c->partitioned ? size_t(c->dd.first) : 0;
  for (size_t i = 0; i < size_t(c->L->nowned); ++i) {
    const Key& k = c->tree.cells[first + i];
    out[4 * i + 0] = k.level;
    out[4 * i + 1] = k.x[0];
    out[4 * i + 2] = k.x[1];
    out[4 * i + 3] = k.x[2];
  }
  return ADER_OK;
}

ader_status ader_mesh_skeleton(ader_ctx* c, uint8_t* out) {
  if (!c || !out) return ADER_ERR_ARG;
  std::memset(out, 0, size_t(c->L->nowned));
  for (int32_t i : c->L->skel_cells) out[i] = 1;
  return ADER_OK;
}

ader_status ader_nodes(ader_ctx* c, double* xi) {
  if (!c || !xi) return ADER_ERR_ARG;
  for (int i = 0; i < c->n; ++i) xi[i] = c->B.xi[i];
  return ADER_OK;
}

static ader_status copy_cells(ader_ctx* c, double* dst, const double* src, size_t bytes, int on_device,
                              bool to_device, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice
                                  : (to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
  CK(cudaMemcpyAsync(dst, src, bytes, kind, s), "state copy");
  if (!on_device) CK(cudaStreamSynchronize(s), "state copy sync");
  return ADER_OK;
}

ader_status ader_set_state(ader_ctx* c, const double* u, int on_device, void* stream) {
  if (!c || !u) return ADER_ERR_ARG;
  const size_t bytes = size_t(c->M) * c->NS * sizeof(double) * size_t(c->L->nowned);
  return copy_cells(c, c->u, u, bytes, on_device, true, stream);
}

ader_status ader_get_state(ader_ctx* c, double* u, int on_device, void* stream) {
  if (!c || !u) return ADER_ERR_ARG;
  const size_t bytes = size_t(c->M) * c->NS * sizeof(double) * size_t(c->L->nowned);
  return copy_cells(c, u, c->u, bytes, on_device, false, stream);
}

ader_status ader_get_field(ader_ctx* c, ader_field f, double* out, int on_device, void* stream) {
  if (!c || !out) return ADER_ERR_ARG;
  const size_t cell_bytes = size_t(c->M) * c->NS * sizeof(double) * size_t(c->L->nowned);
  const size_t face_bytes = size_t(2 * c->cfg.dim) * c->M * c->NF * sizeof(double) * size_t(c->L->nlocal);
  switch (f) {
    case ADER_FIELD_U: return copy_cells(c, out, c->u, cell_bytes, on_device, false, stream);
    case ADER_FIELD_USTAR: return copy_cells(c, out, c->ustar, cell_bytes, on_device, false, stream);
    case ADER_FIELD_FACE_Q: return copy_cells(c, out, c->faceQ, face_bytes, on_device, false, stream);
    case ADER_FIELD_FACE_F: return copy_cells(c, out, c->faceF, face_bytes, on_device, false, stream);
    case ADER_FIELD_FSTAR: return copy_cells(c, out, c->fstar, face_bytes, on_device, false, stream);
  }
  return ADER_ERR_ARG;
}

ader_status ader_compute_dt(ader_ctx* c, double* dt_dev, void* stream) {
  if (!c || !dt_dev) return ADER_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CorrectArgs a = correct_args(c, nullptr);
  CK(do_correct(c, false, a, s), "rate");
  c->launches += 1;
  CK(launch_finalize_dt(c->rate, c->cfg.cfl, dt_dev, c->status, s), "finalize dt");
  return ADER_OK;
}

ader_status ader_predict(ader_ctx* c, const double* dt_dev, ader_set set, void* stream) {
  if (!c || !dt_dev) return ADER_ERR_ARG;
  PredictArgs a = predict_args(c, dt_dev, set);
  CK(do_predict(c, a, static_cast<cudaStream_t>(stream)), "predictor");
  return ADER_OK;
}

ader_status ader_riemann(ader_ctx* c, ader_set set, void* stream) {
  if (!c) return ADER_ERR_ARG;
  return enqueue_riemann(c, set, static_cast<cudaStream_t>(stream));
}

ader_status ader_correct(ader_ctx* c, const double* dt_dev, double* dt_next_dev, void* stream) {
  if (!c || !dt_dev || !dt_next_dev) return ADER_ERR_ARG;
  return enqueue_correct(c, dt_dev, dt_next_dev, static_cast<cudaStream_t>(stream));
}

// One step with the enclave predictor in K chunks: after chunk k the
// high-priority stream solves the faces completed by it and corrects the
// cells whose faces are then all solved (Tree::set_chunks).
ader_status step_pipelined(ader_ctx* c, double* dt_dev) {
  const MeshLists& t = *c->L;
  const int K = t.chunks;
  while (int(c->ev_chunk.size()) < K) {
    cudaEvent_t e = nullptr;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    c->ev_chunk.push_back(e);
  }
  CK(cudaEventRecord(c->ev_step, c->s_hi), "event");
  CK(cudaStreamWaitEvent(c->s_lo, c->ev_step, 0), "event");
  if (c->cfg.limiter) {
    ader_status st = enqueue_limiter_bounds(c, dt_dev, c->s_hi);
    if (st != ADER_OK) return st;
  }
  PredictArgs ps = predict_args(c, dt_dev, ADER_SKELETON);
  CK(do_predict(c, ps, c->s_hi), "skeleton predictor");
  ader_status st = enqueue_riemann(c, ADER_SKELETON, c->s_hi);
  if (st != ADER_OK) return st;
  const int cap = c->num_sms * (c->cfg.pipeline_ctas > 0 ? c->cfg.pipeline_ctas : 4);
  auto correct_group = [&](int g) -> ader_status {
    const int64_t b = t.corr_off[size_t(g)], e = t.corr_off[size_t(g) + 1];
    if (e > b) {
      CorrectArgs ca = stage_correct_args(c, dt_dev, c->corr_cells + b, e - b);
      ca.max_ctas = cap;
      CK(do_correct(c, true, ca, c->s_hi), "corrector");
    }
    return ADER_OK;
  };
  st = correct_group(0);
  if (st != ADER_OK) return st;
  for (int k = 0; k < K; ++k) {
    PredictArgs pe = predict_args(c, dt_dev, ADER_ENCLAVE);
    pe.cells = c->encl_cells + t.chunk_off[size_t(k)];
    pe.count = t.chunk_off[size_t(k) + 1] - t.chunk_off[size_t(k)];
    CK(do_predict(c, pe, c->s_lo), "enclave predictor");
    CK(cudaEventRecord(c->ev_chunk[size_t(k)], c->s_lo), "event");
  }
  for (int k = 0; k < K; ++k) {
    CK(cudaStreamWaitEvent(c->s_hi, c->ev_chunk[size_t(k)], 0), "event");
    RiemannArgs a = riemann_args(c);
    a.conf = c->conf + t.n_conf_skeleton + t.face_off[size_t(k)];
    a.nconf = t.face_off[size_t(k) + 1] - t.face_off[size_t(k)];
    a.nparents = 0;
    a.max_ctas = cap;
    CK(do_faces(c, 0, a, c->s_hi), "riemann conforming faces");
    st = correct_group(k + 1);
    if (st != ADER_OK) return st;
  }
  return enqueue_finish(c, dt_dev, dt_dev, c->s_hi);
}

// One step's work on s_hi / s_lo (joined back into s_hi at the end).
ader_status enqueue_step(ader_ctx* c, double* dt_dev) {
  if (c->L->chunks > 1) return step_pipelined(c, dt_dev);
  CK(cudaEventRecord(c->ev_step, c->s_hi), "event");
  CK(cudaStreamWaitEvent(c->s_lo, c->ev_step, 0), "event");
  PredictArgs ps = predict_args(c, dt_dev, ADER_SKELETON);
  CK(do_predict(c, ps, c->s_hi), "skeleton predictor");
  ader_status st = enqueue_riemann(c, ADER_SKELETON, c->s_hi);
  if (st != ADER_OK) return st;
  PredictArgs pe = predict_args(c, dt_dev, ADER_ENCLAVE);
  CK(do_predict(c, pe, c->s_lo), "enclave predictor");
  CK(cudaEventRecord(c->ev_lo, c->s_lo), "event");
  CK(cudaStreamWaitEvent(c->s_hi, c->ev_lo, 0), "event");
  st = enqueue_riemann(c, ADER_ENCLAVE, c->s_hi);
  if (st != ADER_OK) return st;
  return enqueue_correct(c, dt_dev, dt_dev, c->s_hi);
}

// Capture one step (both streams) into a CUDA graph for this mesh and dt
// pointer.  The graph keeps each kernel's stream priority (without the
// node-priority flag a replay runs every node at the launching stream's
// priority, and the skeleton work would lose its precedence).  On any capture
// failure the context keeps launching eagerly.
void capture_step(ader_ctx* c, double* dt_dev) {
  drop_step_graph(c);
  const int64_t before = c->launches;
  if (cudaStreamBeginCapture(c->s_hi, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    c->graphs_ok = false;
    return;
  }
  const ader_status st = enqueue_step(c, dt_dev);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->s_hi, &g);
  c->step_graph_launches = c->launches - before;
  c->launches = before;
  cudaGetLastError();
  if (st != ADER_OK || e != cudaSuccess || !g ||
      cudaGraphInstantiate(&c->step_exec, g, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
    c->step_exec = nullptr;
    c->graphs_ok = false;
    cudaGetLastError();
  } else {
    c->graph_dt = dt_dev;
  }
  if (g) cudaGraphDestroy(g);
}

// One step with the state read from and written to host memory.  The state
// arrives in K contiguous cell ranges on a copy stream, range k ending where
// enclave chunk k + 1 starts, so each enclave chunk's predictor waits only
// for its own range and the copy of the next range overlaps it; the skeleton
// predictor and the transition faces follow the last range; faces and
// correctors then run as in step_pipelined, and the new state goes back in
// one copy.  The order of the predictor tasks changes no result.
ader_status step_host(ader_ctx* c, const double* u_in, double* u_out, double* dt_dev, cudaStream_t s) {
  const MeshLists& t = *c->L;
  const int K = std::max(1, t.chunks);
  const int64_t C = t.nowned;
  const size_t cell_bytes = size_t(c->M) * c->NS * sizeof(double);
  if (!c->s_copy) CK(cudaStreamCreateWithFlags(&c->s_copy, cudaStreamNonBlocking), "copy stream");
  while (int(c->ev_copy.size()) < K) {
    cudaEvent_t e = nullptr;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    c->ev_copy.push_back(e);
  }
  while (int(c->ev_chunk.size()) < K) {
    cudaEvent_t e = nullptr;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    c->ev_chunk.push_back(e);
  }
  // cell ranges of the copies: range k = [start of enclave chunk k, start of
  // enclave chunk k + 1), the first from cell 0, the last to the end
  std::vector<int64_t> lo(size_t(K) + 1, C);
  lo[0] = 0;
  const int64_t ne = int64_t(t.encl_cells.size());
  for (int k = 1; k < K; ++k) {
    const int64_t p = t.chunk_off[size_t(k)];
    lo[size_t(k)] = p < ne ? int64_t(t.encl_cells[size_t(p)]) : C;
    lo[size_t(k)] = std::max(lo[size_t(k)], lo[size_t(k) - 1]);
  }
  CK(cudaEventRecord(c->ev_begin, s), "event");
  CK(cudaStreamWaitEvent(c->s_copy, c->ev_begin, 0), "event");
  for (int k = 0; k < K; ++k) {
    const int64_t a = lo[size_t(k)], b = lo[size_t(k) + 1];
    if (b > a)
      CK(cudaMemcpyAsync(c->u + a * int64_t(c->M) * c->NS, u_in + a * int64_t(c->M) * c->NS,
                         cell_bytes * size_t(b - a), cudaMemcpyHostToDevice, c->s_copy), "state in");
    CK(cudaEventRecord(c->ev_copy[size_t(k)], c->s_copy), "event");
  }
  for (int k = 0; k < K; ++k) {
    CK(cudaStreamWaitEvent(c->s_lo, c->ev_copy[size_t(k)], 0), "event");
    PredictArgs pe = predict_args(c, dt_dev, ADER_ENCLAVE);
    pe.cells = c->encl_cells + t.chunk_off[size_t(k)];
    pe.count = t.chunk_off[size_t(k) + 1] - t.chunk_off[size_t(k)];
    CK(do_predict(c, pe, c->s_lo), "enclave predictor");
    CK(cudaEventRecord(c->ev_chunk[size_t(k)], c->s_lo), "event");
  }
  CK(cudaStreamWaitEvent(c->s_hi, c->ev_copy[size_t(K) - 1], 0), "event");
  PredictArgs ps = predict_args(c, dt_dev, ADER_SKELETON);
  CK(do_predict(c, ps, c->s_hi), "skeleton predictor");
  ader_status st = enqueue_riemann(c, ADER_SKELETON, c->s_hi);
  if (st != ADER_OK) return st;
  const int cap = c->num_sms * (c->cfg.pipeline_ctas > 0 ? c->cfg.pipeline_ctas : 4);
  auto correct_group = [&](int g) -> ader_status {
    const int64_t b = t.corr_off[size_t(g)], e = t.corr_off[size_t(g) + 1];
    if (e > b) {
      CorrectArgs ca = stage_correct_args(c, dt_dev, c->corr_cells + b, e - b);
      ca.max_ctas = cap;
      CK(do_correct(c, true, ca, c->s_hi), "corrector");
    }
    return ADER_OK;
  };
  st = correct_group(0);
  if (st != ADER_OK) return st;
  for (int k = 0; k < K; ++k) {
    CK(cudaStreamWaitEvent(c->s_hi, c->ev_chunk[size_t(k)], 0), "event");
    RiemannArgs a = riemann_args(c);
    a.conf = c->conf + t.n_conf_skeleton + t.face_off[size_t(k)];
    a.nconf = t.face_off[size_t(k) + 1] - t.face_off[size_t(k)];
    a.nparents = 0;
    a.max_ctas = cap;
    CK(do_faces(c, 0, a, c->s_hi), "riemann conforming faces");
    st = correct_group(k + 1);
    if (st != ADER_OK) return st;
  }
  st = enqueue_finish(c, dt_dev, dt_dev, c->s_hi);
  if (st != ADER_OK) return st;
  CK(cudaMemcpyAsync(u_out, c->u, cell_bytes * size_t(C), cudaMemcpyDeviceToHost, c->s_hi), "state out");
  CK(cudaEventRecord(c->ev_end, c->s_hi), "event");
  CK(cudaStreamWaitEvent(s, c->ev_end, 0), "event");
  return ADER_OK;
}

ader_status ader_step_host(ader_ctx* c, const double* u_in, double* u_out, double* dt_dev, void* stream) {
  if (!c || !u_in || !u_out || !dt_dev) return ADER_ERR_ARG;
  if (c->partitioned || c->cfg.limiter || c->L->chunks < 1) {
    c->err = "ader_step_host needs an unpartitioned context without the limiter";
    return ADER_ERR_ARG;
  }
  return step_host(c, u_in, u_out, dt_dev, static_cast<cudaStream_t>(stream));
}

ader_status ader_step(ader_ctx* c, int nsteps, double* dt_dev, void* stream) {
  if (!c || !dt_dev || nsteps < 0) return ADER_ERR_ARG;
  if (c->partitioned) {
    c->err = "a partitioned context steps by ader_predict, ader_halo_pack/unpack, ader_riemann "
             "and ader_correct, with the exchange between them";
    return ADER_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaEventRecord(c->ev_begin, s), "event");
  CK(cudaStreamWaitEvent(c->s_hi, c->ev_begin, 0), "event");
  // capture once this mesh has run one eager step (every kernel configured)
  if (nsteps > 0 && c->graphs_ok && !c->cfg.eager_steps && c->warm) {
    if (!c->step_exec || c->graph_dt != dt_dev) capture_step(c, dt_dev);
    if (c->step_exec) {
      for (int k = 0; k < nsteps; ++k) {
        CK(cudaGraphLaunch(c->step_exec, c->s_hi), "step graph launch");
        c->launches += c->step_graph_launches;
      }
      nsteps = 0;
    }
  }
  for (int k = 0; k < nsteps; ++k) {
    if (c->L->chunks > 1) {
      ader_status st = step_pipelined(c, dt_dev);
      if (st != ADER_OK) return st;
      continue;
    }
    CK(cudaEventRecord(c->ev_step, c->s_hi), "event");
    CK(cudaStreamWaitEvent(c->s_lo, c->ev_step, 0), "event");
    PredictArgs ps = predict_args(c, dt_dev, ADER_SKELETON);
    CK(do_predict(c, ps, c->s_hi), "skeleton predictor");
    ader_status st = enqueue_riemann(c, ADER_SKELETON, c->s_hi);
    if (st != ADER_OK) return st;
    PredictArgs pe = predict_args(c, dt_dev, ADER_ENCLAVE);
    CK(do_predict(c, pe, c->s_lo), "enclave predictor");
    CK(cudaEventRecord(c->ev_lo, c->s_lo), "event");
    CK(cudaStreamWaitEvent(c->s_hi, c->ev_lo, 0), "event");
    st = enqueue_riemann(c, ADER_ENCLAVE, c->s_hi);
    if (st != ADER_OK) return st;
    st = enqueue_correct(c, dt_dev, dt_dev, c->s_hi);
    if (st != ADER_OK) return st;
  }
  if (nsteps > 0) c->warm = true;
  CK(cudaEventRecord(c->ev_end, c->s_hi), "event");
  CK(cudaStreamWaitEvent(s, c->ev_end, 0), "event");
  return ADER_OK;
}

// Global time stepping with a prescribed dt (Sec. 3, the shifted task graph):
// the corrector of step k and the predictor of step k + 1 are one task per
// cell (the predictor kernel's corrector prologue), so nsteps steps take
// nsteps + 1 passes over the cells instead of 2 nsteps.  The call starts
// with a plain predictor and ends with a plain corrector, whose CFL time step
// goes to dt_next_dev; the result equals nsteps rounds of ader_predict,
// ader_riemann and ader_correct with the same dt, bit for bit.
ader_status ader_step_fixed_dt(ader_ctx* c, int nsteps, const double* dt_dev, double* dt_next_dev,
                               void* stream) {
  if (!c || !dt_dev || nsteps < 0) return ADER_ERR_ARG;
  if (c->partitioned || c->cfg.limiter) {
    c->err = "ader_step_fixed_dt needs an unpartitioned context without the limiter";
    return ADER_ERR_ARG;
  }
  if (nsteps == 0) return ADER_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaEventRecord(c->ev_begin, s), "event");
  CK(cudaStreamWaitEvent(c->s_hi, c->ev_begin, 0), "event");
  CK(do_predict(c, predict_args(c, dt_dev, ADER_ALL), c->s_hi), "predictor");
  for (int k = 0; k < nsteps; ++k) {
    ader_status st = enqueue_riemann(c, ADER_ALL, c->s_hi);
    if (st != ADER_OK) return st;
    if (k + 1 == nsteps) break;
    PredictArgs a = predict_args(c, dt_dev, ADER_ALL);
    a.corr_fstar = c->fstar;
    a.corr_u = c->u;
    CK(do_predict(c, a, c->s_hi), "corrector and next predictor");
  }
  ader_status st = enqueue_correct(c, dt_dev, dt_next_dev ? dt_next_dev : c->dt_scratch, c->s_hi);
  if (st != ADER_OK) return st;
  CK(cudaEventRecord(c->ev_end, c->s_hi), "event");
  CK(cudaStreamWaitEvent(s, c->ev_end, 0), "event");
  return ADER_OK;
}

ader_status ader_classify(ader_ctx* c, const int8_t* flags) {
  if (!c) return ADER_ERR_ARG;
  CK(cudaDeviceSynchronize(), "sync before classify");
  c->tree.classify(flags);
  if (c->partitioned) return rebuild_subdomain(c, c->dd.base_cut);
  return upload_mesh(c);
}

namespace {

// Partitioned remesh: every rank adapts its copy of the whole tree with the
// same flags; the cells of the rank's old base-cell range get their data from
// its old owned cells (no family crosses a cut), into the staging buffer;
// then the cuts are rebalanced and the overlap of the staging range with the
// new owned range is copied into u.  The rest arrives by ader_migrate_unpack.
ader_status remesh_partitioned(ader_ctx* c, const int8_t* flags) {
  const std::vector<int64_t> old_cut = c->dd.base_cut;
  const int64_t o0 = c->dd.first, nold = c->L->nowned;
  const int R = c->dd.nranks, r = c->dd.rank;
  std::vector<TransferItem> plan;
  std::vector<int32_t> kids;
  if (!c->tree.remesh(flags, &plan, &kids)) {
    c->err = c->tree.error();
    return ADER_ERR_MESH;
  }
  c->force_set = false;
  std::vector<int64_t> starts;
  if (!base_starts(c->tree, &starts)) {
    c->err = "the cell order does not follow the base cells";
    return ADER_ERR_MESH;
  }
  const int64_t n0 = starts[size_t(old_cut[size_t(r)])], n1 = starts[size_t(old_cut[size_t(r) + 1])];
  const int S = int(ipow64(3, c->cfg.dim));
  std::vector<TransferItem> lplan(size_t(n1 - n0));
  std::vector<int32_t> lkids;
  for (int64_t g = n0; g < n1; ++g) {
    TransferItem it = plan[size_t(g)];
    if (it.kind == 2) {
      const int32_t off = int32_t(lkids.size());
      for (int j = 0; j < S; ++j) {
        const int64_t k = int64_t(kids[size_t(it.src) + size_t(j)]) - o0;
        if (k < 0 || k >= nold) {
          c->err = "a coarsened family crosses a partition cut";
          return ADER_ERR_MESH;
        }
        lkids.push_back(int32_t(k));
      }
      it.src = off;
    } else {
      it.src = int32_t(int64_t(it.src) - o0);
      if (it.src < 0 || it.src >= nold) {
        c->err = "a new cell takes data from another partition";
        return ADER_ERR_MESH;
      }
    }
    lplan[size_t(g - n0)] = it;
  }
  const int64_t cell_doubles = int64_t(c->M) * c->NS;
  CK(grow(&c->stage, &c->stage_cap, std::max<int64_t>(n1 - n0, 1) * cell_doubles), "cudaMalloc staging");
  CK(grow(&c->plan_dev, &c->plan_cap, std::max<int64_t>(int64_t(lplan.size()), 1)), "cudaMalloc plan");
  CK(grow(&c->kids_dev, &c->kids_cap, std::max<int64_t>(int64_t(lkids.size()), 1)), "cudaMalloc kids");
  if (!lplan.empty())
    CK(cudaMemcpy(c->plan_dev, lplan.data(), sizeof(TransferItem) * lplan.size(), cudaMemcpyHostToDevice),
       "upload plan");
  if (!lkids.empty())
    CK(cudaMemcpy(c->kids_dev, lkids.data(), sizeof(int32_t) * lkids.size(), cudaMemcpyHostToDevice),
       "upload kids");
  TransferArgs a{};
  a.u_old = c->u;
  a.u_new = c->stage;
  a.plan = c->plan_dev;
  a.children = c->kids_dev;
  a.ncells_new = n1 - n0;
  a.ncells_old = nold;
  a.status = c->status;
  a.B = c->B;
  CK(do_transfer(c, a, nullptr), "transfer");
  CK(cudaDeviceSynchronize(), "transfer sync");
  std::vector<int64_t> base_cut;
  if (!balanced_cuts(starts, R, &base_cut)) {
    c->err = "more ranks than base cells";
    return ADER_ERR_MESH;
  }
  c->old_base_cut = old_cut;
  c->stage_first = n0;
  c->stage_count = n1 - n0;
  ader_status st = rebuild_subdomain(c, base_cut);
  if (st != ADER_OK) return st;
  const int64_t m0 = c->dd.first, m1 = m0 + c->L->nowned;
  const int64_t lo = std::max(n0, m0), hi = std::min(n1, m1);
  if (hi > lo)
    CK(cudaMemcpy(c->u + (lo - m0) * cell_doubles, c->stage + (lo - n0) * cell_doubles,
                  sizeof(double) * size_t((hi - lo) * cell_doubles), cudaMemcpyDeviceToDevice),
       "keep own cells");
  c->migrating = true;
  return ADER_OK;
}

// Tree cells [lo, hi) that this rank sends to `peer` (send) or receives from
// it (recv) after a partitioned remesh.
void migration_range(const ader_ctx* c, int peer, bool send, int64_t* lo, int64_t* hi) {
  std::vector<int64_t> starts;
  *lo = *hi = 0;
  if (!c->migrating || !base_starts(c->tree, &starts)) return;
  const std::vector<int64_t>& oc = c->old_base_cut;
  const std::vector<int64_t>& nc = c->dd.base_cut;
  const int me = c->dd.rank;
  const int src = send ? me : peer, dst = send ? peer : me;
  const int64_t a0 = starts[size_t(oc[size_t(src)])], a1 = starts[size_t(oc[size_t(src) + 1])];
  const int64_t b0 = starts[size_t(nc[size_t(dst)])], b1 = starts[size_t(nc[size_t(dst) + 1])];
  *lo = std::max(a0, b0);
  *hi = std::max(*lo, std::min(a1, b1));
}

}  // namespace

ader_status ader_remesh(ader_ctx* c, const int8_t* flags) {
  if (!c || !flags) return ADER_ERR_ARG;
  CK(cudaDeviceSynchronize(), "sync before remesh");
  if (c->partitioned) return remesh_partitioned(c, flags);
  const int64_t C_old = int64_t(c->tree.cells.size());
  std::vector<TransferItem> plan;
  std::vector<int32_t> kids;
  // The mesh before the call: restored, with its device lists, when the
  // device side cannot follow (every buffer is allocated before an old one is
  // released, so u still holds the old state then).
  Tree::State saved = c->tree.save();
  if (!c->tree.remesh(flags, &plan, &kids)) {
    c->err = c->tree.error();
    c->tree.restore(std::move(saved));
    return ADER_ERR_MESH;
  }
  const int64_t C_new = int64_t(c->tree.cells.size());
  c->force_set = false;
  double* old_u = nullptr;
  bool own_old = false;
  auto undo = [&](ader_status st) {
    const std::string why = c->err;
    if (own_old) cudaFree(old_u);
    c->tree.restore(std::move(saved));
    upload_mesh(c);  // the old mesh's lists fit the capacities already there
    c->err = why;
    return st;
  };
  // Keep the old state while the mesh lists are uploaded: in u* (free between
  // steps) when the cell buffers keep their capacity, else in a new buffer.
  const size_t cell_bytes = size_t(c->M) * c->NS * sizeof(double);
  const bool in_place = C_new <= c->cap;
  old_u = in_place ? c->ustar : nullptr;
  if (!in_place) {
    void* q = nullptr;
    const cudaError_t ea = dev_alloc(&q, cell_bytes * size_t(std::max<int64_t>(C_old, 1)));
    if (ea != cudaSuccess) return undo(cuda_fail(c, ea, "cudaMalloc remesh"));
    old_u = static_cast<double*>(q);
    own_old = true;
  }
  cudaError_t ec = cudaMemcpy(old_u, c->u, cell_bytes * size_t(C_old), cudaMemcpyDeviceToDevice);
  if (ec != cudaSuccess) return undo(cuda_fail(c, ec, "copy u"));
  ader_status st = upload_mesh(c);
  if (st != ADER_OK) return undo(st);
  ec = grow(&c->plan_dev, &c->plan_cap, int64_t(plan.size()));
  if (ec == cudaSuccess) ec = grow(&c->kids_dev, &c->kids_cap, std::max<int64_t>(int64_t(kids.size()), 1));
  if (ec != cudaSuccess) return undo(cuda_fail(c, ec, "cudaMalloc plan"));
  TransferItem* d_plan = c->plan_dev;
  int32_t* d_kids = c->kids_dev;
  CK(cudaMemcpy(d_plan, plan.data(), sizeof(TransferItem) * plan.size(), cudaMemcpyHostToDevice),
     "upload plan");
  if (!kids.empty())
    CK(cudaMemcpy(d_kids, kids.data(), sizeof(int32_t) * kids.size(), cudaMemcpyHostToDevice),
       "upload kids");
  TransferArgs a{};
  a.u_old = old_u;
  a.u_new = c->u;
  a.plan = d_plan;
  a.children = d_kids;
  a.ncells_new = C_new;
  a.ncells_old = C_old;
  a.status = c->status;
  a.B = c->B;
  cudaError_t e = do_transfer(c, a, nullptr);
  cudaError_t e2 = cudaDeviceSynchronize();
  if (own_old) cudaFree(old_u);
  if (e != cudaSuccess) return cuda_fail(c, e, "transfer");
  if (e2 != cudaSuccess) return cuda_fail(c, e2, "transfer sync");
  return ADER_OK;
}

namespace {

cudaError_t enqueue_indicator(ader_ctx* c, int var, int deriv, double* eta, cudaStream_t s) {
  IndicatorArgs a{};
  a.u = c->u;
  a.level = c->level;
  a.ncells = c->L->nowned;
  a.var = var;
  a.deriv = deriv;
  a.eta = eta;
  std::memcpy(a.inv_h, c->inv_h, sizeof(a.inv_h));
  a.B = c->B;
  const int N = c->cfg.order;
  c->launches += a.ncells > 0 ? 1 : 0;
  if (c->cfg.pde == ADER_EULER)
    return c->cfg.dim == 2 ? indicator_euler2d(N, a, s) : indicator_euler3d(N, a, s);
  return c->cfg.dim == 2 ? indicator_acoustics2d(N, a, s) : indicator_acoustics3d(N, a, s);
}

}  // namespace

ader_status ader_gradient_indicator(ader_ctx* c, int var, int deriv, double* eta_dev, void* stream) {
  if (!c || var < 0 || var >= c->M || (deriv != 1 && deriv != 2)) return ADER_ERR_ARG;
  if (!eta_dev && c->L->nowned > 0) return ADER_ERR_ARG;
  CK(enqueue_indicator(c, var, deriv, eta_dev, static_cast<cudaStream_t>(stream)), "gradient indicator");
  return ADER_OK;
}

ader_status ader_gradient_flags(ader_ctx* c, int var, int deriv, double refine_above, double coarsen_below,
                                double* eta_out, int8_t* flags) {
  if (!c || !flags || var < 0 || var >= c->M || (deriv != 1 && deriv != 2) ||
      !(refine_above >= coarsen_below))
    return ADER_ERR_ARG;
  const int64_t C = c->L->nowned;
  // the state may still be written by steps on the caller's (non-blocking) streams
  CK(cudaDeviceSynchronize(), "sync before gradient indicator");
  double* d_eta = nullptr;
  CK(cudaMalloc(&d_eta, sizeof(double) * size_t(std::max<int64_t>(C, 1))), "cudaMalloc eta");
  cudaError_t e = enqueue_indicator(c, var, deriv, d_eta, nullptr);
  std::vector<double> eta(static_cast<size_t>(C));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess && C > 0)
    e = cudaMemcpy(eta.data(), d_eta, sizeof(double) * size_t(C), cudaMemcpyDeviceToHost);
  cudaFree(d_eta);
  if (e != cudaSuccess) return cuda_fail(c, e, "gradient indicator");
  for (int64_t i = 0; i < C; ++i) {
    const int lv = c->L->levels[size_t(i)];
    int8_t f = 0;
    if (eta[size_t(i)] > refine_above && lv < c->cfg.max_level)
      f = 1;
    else if (eta[size_t(i)] < coarsen_below && lv > 0)
      f = -1;
    flags[i] = f;
    if (eta_out) eta_out[i] = eta[size_t(i)];
  }
  return ADER_OK;
}

ader_status ader_sphere_flags(ader_ctx* c, const double center[3], double radius, int8_t* flags) {
  if (!c || !center || !flags) return ADER_ERR_ARG;
  c->tree.sphere_flags(center, radius, c->cfg.lo, c->cfg.hi, flags);
  return ADER_OK;
}

ader_status ader_status_word(ader_ctx* c, uint32_t* out) {
  if (!c || !out) return ADER_ERR_ARG;
  CK(cudaDeviceSynchronize(), "sync");
  CK(cudaMemcpy(out, c->status, sizeof(uint32_t), cudaMemcpyDeviceToHost), "read status");
  CK(cudaMemset(c->status, 0, sizeof(uint32_t)), "clear status");
  return ADER_OK;
}

ader_status ader_adjoint_step(ader_ctx* c, const double* lam_in, double* lam_out,
                              const double* dt_dev, void* stream) {
  if (!c || !lam_in || !lam_out || !dt_dev || lam_in == lam_out) return ADER_ERR_ARG;
  if (c->cfg.pde != ADER_ACOUSTICS || c->cfg.prec != ADER_FP64) {
    c->err = "the adjoint step is implemented for linear acoustics in FP64";
    return ADER_ERR_ARG;
  }
  if (c->partitioned) {
    c->err = "the adjoint step needs an unpartitioned mesh";
    return ADER_ERR_ARG;
  }
  AdjointArgs a{};
  a.lam_in = lam_in;
  a.lam_out = lam_out;
  a.fstar_bar = c->fstar;
  a.faceQ_bar = c->faceQ;
  a.faceF_bar = c->faceF;
  a.conf = c->conf;
  a.nconf = int64_t(c->tree.conf.size());
  a.parents = c->parents;
  a.child_fine = c->child_fine;
  a.nparents = int64_t(c->tree.parents.size());
  a.level = c->level;
  a.ncells = int64_t(c->tree.cells.size());
  a.dt = dt_dev;
  a.iters = c->cfg.picard_iters > 0 ? c->cfg.picard_iters : c->cfg.order + 1;
  a.scheme = c->cfg.predictor;
  std::memcpy(a.inv_h, c->inv_h, sizeof(a.inv_h));
  a.B = c->B;
  c->launches += c->tree.parents.empty() ? 3 : 4;
  CK(launch_adjoint(c->cfg.dim, c->cfg.order, a, static_cast<cudaStream_t>(stream)), "adjoint step");
  return ADER_OK;
}

ader_status ader_sample(ader_ctx* c, int npts, const int32_t* cells, const double* weights, int var,
                        const double* field, double* out, void* stream) {
  if (!c || npts < 0 || (npts > 0 && (!cells || !weights || !out)) || var < 0 || var >= c->M)
    return ADER_ERR_ARG;
  c->launches += npts > 0 ? 1 : 0;
  CK(launch_sample(field ? field : c->u, c->M, c->NS, var, npts, cells, weights, out,
                   static_cast<cudaStream_t>(stream)), "sample");
  return ADER_OK;
}

ader_status ader_sample_adjoint(ader_ctx* c, int npts, const int32_t* cells, const double* weights,
                                int var, const double* values, double* field, void* stream) {
  if (!c || npts < 0 || !field || (npts > 0 && (!cells || !weights || !values)) || var < 0 ||
      var >= c->M)
    return ADER_ERR_ARG;
  c->launches += npts > 0 ? 1 : 0;
  CK(launch_sample_adjoint(field, c->M, c->NS, var, npts, cells, weights, values,
                           static_cast<cudaStream_t>(stream)), "sample adjoint");
  return ADER_OK;
}

ader_status ader_limiter_flags(ader_ctx* c, uint32_t* flags, int on_device, int64_t* nlimited,
                               void* stream) {
  if (!c || !c->cfg.limiter) return ADER_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t C = c->tree.cells.size();
  if (flags)
    CK(cudaMemcpyAsync(flags, c->lim_flags, sizeof(uint32_t) * C,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s),
       "copy limiter flags");
  if (nlimited) {
    int cnt[2] = {0, 0};
    CK(cudaMemcpyAsync(cnt, c->lim_counts, sizeof(cnt), cudaMemcpyDeviceToHost, s), "limiter count");
    CK(cudaStreamSynchronize(s), "limiter count sync");
    *nlimited = cnt[0];
  }
  if (flags && !on_device) CK(cudaStreamSynchronize(s), "limiter flags sync");
  return ADER_OK;
}

ader_status ader_limiter_force(ader_ctx* c, const uint8_t* force) {
  if (!c || !c->cfg.limiter) return ADER_ERR_ARG;
  CK(cudaDeviceSynchronize(), "sync before limiter force");
  drop_step_graph(c);
  if (!force) {
    c->force_set = false;
    return ADER_OK;
  }
  CK(cudaMemcpy(c->force, force, c->tree.cells.size(), cudaMemcpyHostToDevice), "upload force");
  c->force_set = true;
  return ADER_OK;
}

ader_status ader_step_refining(ader_ctx* c, double* dt_dev, int max_rounds, int* rounds, void* stream) {
  if (!c || !dt_dev || max_rounds < 0 || !c->cfg.limiter || c->partitioned) return ADER_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaDeviceSynchronize(), "sync before refining step");
  // status bits of a discarded attempt are dropped: the word is reset to its
  // value before the call ahead of every repeat
  uint32_t status0 = 0;
  CK(cudaMemcpy(&status0, c->status, sizeof(uint32_t), cudaMemcpyDeviceToHost), "read status");
  int r = 0;
  for (;;) {
    ader_status st = ader_step(c, 1, dt_dev, stream);
    if (st != ADER_OK) return st;
    CK(cudaStreamSynchronize(s), "refining step sync");
    CK(cudaDeviceSynchronize(), "refining step sync");
    const size_t C = c->tree.cells.size();
    std::vector<uint32_t> lf(C);
    if (C) CK(cudaMemcpy(lf.data(), c->lim_flags, sizeof(uint32_t) * C, cudaMemcpyDeviceToHost), "limiter flags");
    bool kept = false;
    for (uint32_t f : lf) kept = kept || (f & kKeptAtTransition);
    if (!kept || r == max_rounds) break;
    // back to u(T), which the limiter's first kernel of this step saved
    CK(cudaMemcpy(c->u, c->u_old, size_t(c->M) * c->NS * sizeof(double) * C, cudaMemcpyDeviceToDevice),
       "restore u(T)");
    CK(cudaMemcpy(c->status, &status0, sizeof(uint32_t), cudaMemcpyHostToDevice), "reset status");
    std::vector<uint8_t> troubled(C);
    for (size_t i = 0; i < C; ++i) troubled[i] = (lf[i] & (kLimited | kKeptAtTransition)) ? 1 : 0;
    std::vector<int8_t> fl(C);
    c->tree.refine_around(troubled.data(), fl.data());
    for (int8_t& f : fl) f = f > 0 ? 1 : 0;  // refinement only: nothing coarsens mid-step
    st = ader_remesh(c, fl.data());
    if (st != ADER_OK) return st;
    st = ader_compute_dt(c, dt_dev, stream);
    if (st != ADER_OK) return st;
    ++r;
  }
  if (rounds) *rounds = r;
  return ADER_OK;
}

ader_status ader_limiter_refine_flags(ader_ctx* c, int8_t* flags) {
  if (!c || !c->cfg.limiter || !flags) return ADER_ERR_ARG;
  const size_t C = c->tree.cells.size();
  std::vector<uint32_t> lf(C);
  CK(cudaDeviceSynchronize(), "sync before limiter flags");
  if (C) CK(cudaMemcpy(lf.data(), c->lim_flags, sizeof(uint32_t) * C, cudaMemcpyDeviceToHost), "limiter flags");
  std::vector<uint8_t> troubled(C);
  for (size_t i = 0; i < C; ++i) troubled[i] = (lf[i] & (kLimited | kKeptAtTransition)) ? 1 : 0;
  c->tree.refine_around(troubled.data(), flags);
  return ADER_OK;
}

ader_status ader_debug_fail_allocations(int after) {
  g_alloc_budget.store(after < 0 ? -1 : after);
  return ADER_OK;
}

ader_status ader_launch_count(ader_ctx* c, int64_t* out) {
  if (!c || !out) return ADER_ERR_ARG;
  *out = c->launches;
  return ADER_OK;
}

ader_status ader_partition(ader_ctx* c, int nranks, int rank) {
  if (!c || nranks < 1 || rank < 0 || rank >= nranks) return ADER_ERR_ARG;
  if (c->partitioned) {
    c->err = "the context is partitioned already";
    return ADER_ERR_ARG;
  }
  if (nranks == 1) return ADER_OK;
  if (c->cfg.limiter) {
    c->err = "the subcell limiter needs neighbour states: not available on a partition";
    return ADER_ERR_ARG;
  }
  CK(cudaDeviceSynchronize(), "sync before partition");
  std::vector<int64_t> starts, base_cut;
  if (!base_starts(c->tree, &starts)) {
    c->err = "the cell order does not follow the base cells";
    return ADER_ERR_MESH;
  }
  if (!balanced_cuts(starts, nranks, &base_cut)) {
    c->err = "more ranks than base cells";
    return ADER_ERR_ARG;
  }
  // keep the owned rows of the state, moved to the front (u* is free
  // between steps and has the same capacity)
  const int64_t g0 = starts[size_t(base_cut[size_t(rank)])];
  const int64_t g1 = starts[size_t(base_cut[size_t(rank) + 1])];
  const size_t cell_bytes = size_t(c->M) * c->NS * sizeof(double);
  if (g1 > g0)
    CK(cudaMemcpy(c->ustar, c->u + g0 * int64_t(c->M) * c->NS, cell_bytes * size_t(g1 - g0),
                  cudaMemcpyDeviceToDevice), "keep owned state");
  std::swap(c->u, c->ustar);
  c->dd.rank = rank;
  c->dd.nranks = nranks;
  c->partitioned = true;
  c->migrating = false;
  return rebuild_subdomain(c, base_cut);
}

ader_status ader_dd_info(ader_ctx* c, int* nranks, int* rank, int64_t* nglobal, int64_t* first,
                         int64_t* nowned, int64_t* nghost) {
  if (!c) return ADER_ERR_ARG;
  if (nranks) *nranks = c->partitioned ? c->dd.nranks : 1;
  if (rank) *rank = c->partitioned ? c->dd.rank : 0;
  if (nglobal) *nglobal = int64_t(c->tree.cells.size());
  if (first) *first = c->partitioned ? c->dd.first : 0;
  if (nowned) *nowned = c->L->nowned;
  if (nghost) *nghost = c->L->nlocal - c->L->nowned;
  return ADER_OK;
}

ader_status ader_dd_cuts(ader_ctx* c, int64_t* cuts) {
  if (!c || !cuts) return ADER_ERR_ARG;
  if (!c->partitioned) {
    cuts[0] = 0;
    cuts[1] = int64_t(c->tree.cells.size());
    return ADER_OK;
  }
  std::copy(c->dd.cut.begin(), c->dd.cut.end(), cuts);
  return ADER_OK;
}

ader_status ader_halo_size(ader_ctx* c, int peer, int64_t* send_doubles, int64_t* recv_doubles) {
  if (!c || !c->partitioned || peer < 0 || peer >= c->dd.nranks) return ADER_ERR_ARG;
  const int64_t blk = 2 * int64_t(c->M) * c->NF;
  if (send_doubles) *send_doubles = blk * int64_t(c->dd.send[size_t(peer)].size());
  if (recv_doubles) *recv_doubles = blk * int64_t(c->dd.recv[size_t(peer)].size());
  return ADER_OK;
}

ader_status ader_halo_pack(ader_ctx* c, int peer, double* buf_dev, void* stream) {
  if (!c || !c->partitioned || peer < 0 || peer >= c->dd.nranks) return ADER_ERR_ARG;
  const int64_t b = c->send_off[size_t(peer)], e = c->send_off[size_t(peer) + 1];
  if (e == b) return ADER_OK;
  if (!buf_dev) return ADER_ERR_ARG;
  c->launches += 1;
  CK(launch_halo_pack(c->faceQ, c->faceF, c->halo_send + b, e - b, c->M * c->NF, buf_dev,
                      static_cast<cudaStream_t>(stream)), "halo pack");
  return ADER_OK;
}

ader_status ader_halo_unpack(ader_ctx* c, int peer, const double* buf_dev, void* stream) {
  if (!c || !c->partitioned || peer < 0 || peer >= c->dd.nranks) return ADER_ERR_ARG;
  const int64_t b = c->recv_off[size_t(peer)], e = c->recv_off[size_t(peer) + 1];
  if (e == b) return ADER_OK;
  if (!buf_dev) return ADER_ERR_ARG;
  c->launches += 1;
  CK(launch_halo_unpack(c->faceQ, c->faceF, c->halo_recv + b, e - b, c->M * c->NF, buf_dev,
                        static_cast<cudaStream_t>(stream)), "halo unpack");
  return ADER_OK;
}

ader_status ader_migrate_size(ader_ctx* c, int peer, int64_t* send_doubles, int64_t* recv_doubles) {
  if (!c || !c->partitioned || peer < 0 || peer >= c->dd.nranks) return ADER_ERR_ARG;
  int64_t lo, hi;
  const int64_t cd = int64_t(c->M) * c->NS;
  migration_range(c, peer, true, &lo, &hi);
  if (send_doubles) *send_doubles = peer == c->dd.rank ? 0 : (hi - lo) * cd;
  migration_range(c, peer, false, &lo, &hi);
  if (recv_doubles) *recv_doubles = peer == c->dd.rank ? 0 : (hi - lo) * cd;
  return ADER_OK;
}

ader_status ader_migrate_pack(ader_ctx* c, int peer, double* buf_dev, void* stream) {
  if (!c || !c->partitioned || peer < 0 || peer >= c->dd.nranks) return ADER_ERR_ARG;
  int64_t lo, hi;
  migration_range(c, peer, true, &lo, &hi);
  if (hi == lo || peer == c->dd.rank) return ADER_OK;
  if (!buf_dev) return ADER_ERR_ARG;
  const int64_t cd = int64_t(c->M) * c->NS;
  CK(cudaMemcpyAsync(buf_dev, c->stage + (lo - c->stage_first) * cd, sizeof(double) * size_t((hi - lo) * cd),
                     cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)), "migrate pack");
  return ADER_OK;
}

ader_status ader_migrate_unpack(ader_ctx* c, int peer, const double* buf_dev, void* stream) {
  if (!c || !c->partitioned || peer < 0 || peer >= c->dd.nranks) return ADER_ERR_ARG;
  int64_t lo, hi;
  migration_range(c, peer, false, &lo, &hi);
  if (hi == lo || peer == c->dd.rank) return ADER_OK;
  if (!buf_dev) return ADER_ERR_ARG;
  const int64_t cd = int64_t(c->M) * c->NS;
  CK(cudaMemcpyAsync(c->u + (lo - c->dd.first) * cd, buf_dev, sizeof(double) * size_t((hi - lo) * cd),
                     cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)), "migrate unpack");
  return ADER_OK;
}

struct ader_mesh {
  Tree tree;
  SubDomain dd;
  bool has_dd = false;
};

ader_status ader_mesh_create(int dim, const int base[3], int max_level, ader_mesh** out) {
  if (!base || !out || (dim != 2 && dim != 3) || max_level < 0 || max_level > kMaxLevels - 2)
    return ADER_ERR_ARG;
  *out = nullptr;
  int b[3] = {1, 1, 1};
  for (int d = 0; d < dim; ++d) {
    if (base[d] < 1) return ADER_ERR_ARG;
    b[d] = base[d];
  }
  ader_mesh* m = new ader_mesh();
  m->tree = Tree(dim, b, max_level);
  if (!m->tree.build()) {
    delete m;
    return ADER_ERR_MESH;
  }
  *out = m;
  return ADER_OK;
}

void ader_mesh_destroy(ader_mesh* m) { delete m; }

ader_status ader_mesh_adapt(ader_mesh* m, const int8_t* flags) {
  if (!m || !flags) return ADER_ERR_ARG;
  m->has_dd = false;
  std::vector<TransferItem> plan;
  std::vector<int32_t> kids;
  return m->tree.remesh(flags, &plan, &kids) ? ADER_OK : ADER_ERR_MESH;
}

ader_status ader_mesh_sizes(ader_mesh* m, int64_t* ncells, int64_t* nskel, int64_t* nconf,
                            int64_t* nparents) {
  if (!m) return ADER_ERR_ARG;
  if (ncells) *ncells = int64_t(m->tree.cells.size());
  if (nskel) *nskel = int64_t(m->tree.skel_cells.size());
  if (nconf) *nconf = int64_t(m->tree.conf.size());
  if (nparents) *nparents = int64_t(m->tree.parents.size());
  return ADER_OK;
}

ader_status ader_mesh_leaves(ader_mesh* m, int32_t* cells_out, uint8_t* skel_out) {
  if (!m) return ADER_ERR_ARG;
  const Tree& t = m->tree;
  for (size_t i = 0; i < t.cells.size(); ++i) {
    if (cells_out) {
      cells_out[4 * i + 0] = t.cells[i].level;
      for (int d = 0; d < 3; ++d) cells_out[4 * i + 1 + d] = t.cells[i].x[d];
    }
    if (skel_out) skel_out[i] = t.skeleton[i];
  }
  return ADER_OK;
}

ader_status ader_mesh_faces(ader_mesh* m, int32_t* conf_out, int32_t* parents_out,
                            int32_t* child_out) {
  if (!m) return ADER_ERR_ARG;
  const Tree& t = m->tree;
  if (conf_out)
    for (size_t i = 0; i < t.conf.size(); ++i) {
      conf_out[3 * i + 0] = t.conf[i].left;
      conf_out[3 * i + 1] = t.conf[i].right;
      conf_out[3 * i + 2] = t.conf[i].dir;
    }
  if (parents_out)
    for (size_t i = 0; i < t.parents.size(); ++i) {
      parents_out[3 * i + 0] = t.parents[i].coarse;
      parents_out[3 * i + 1] = t.parents[i].dir;
      parents_out[3 * i + 2] = t.parents[i].coarse_side;
    }
  if (child_out) std::memcpy(child_out, t.child_fine.data(), sizeof(int32_t) * t.child_fine.size());
  return ADER_OK;
}

ader_status ader_mesh_sphere_flags(ader_mesh* m, const double center[3], double radius,
                                   const double lo[3], const double hi[3], int8_t* flags) {
  if (!m || !center || !lo || !hi || !flags) return ADER_ERR_ARG;
  m->tree.sphere_flags(center, radius, lo, hi, flags);
  return ADER_OK;
}

ader_status ader_mesh_refine_around(ader_mesh* m, const uint8_t* troubled, int8_t* flags) {
  if (!m || !troubled || !flags) return ADER_ERR_ARG;
  m->tree.refine_around(troubled, flags);
  return ADER_OK;
}

ader_status ader_mesh_partition(ader_mesh* m, int nranks, int rank, int64_t* sizes) {
  if (!m || nranks < 1 || rank < 0 || rank >= nranks || !sizes) return ADER_ERR_ARG;
  std::vector<int64_t> starts, base_cut;
  if (!base_starts(m->tree, &starts)) return ADER_ERR_MESH;
  if (!balanced_cuts(starts, nranks, &base_cut)) return ADER_ERR_ARG;
  m->dd.rank = rank;
  build_subdomain(m->tree, starts, base_cut, rank, &m->dd);
  m->has_dd = true;
  const MeshLists& L = m->dd.lists;
  int64_t ns = 0, nr = 0;
  for (int q = 0; q < nranks; ++q) {
    ns += int64_t(m->dd.send[size_t(q)].size());
    nr += int64_t(m->dd.recv[size_t(q)].size());
  }
  const int64_t v[9] = {m->dd.first, L.nowned, L.nlocal - L.nowned, int64_t(L.conf.size()),
                        L.n_conf_skeleton, int64_t(L.parents.size()), int64_t(L.skel_cells.size()), ns, nr};
  std::copy(v, v + 9, sizes);
  return ADER_OK;
}

ader_status ader_mesh_subdomain(ader_mesh* m, int64_t* cuts, int32_t* ghosts, int32_t* conf_out,
                                int32_t* parents_out, int32_t* child_out, int32_t* skel_out,
                                int64_t* send_off, int32_t* send_out, int64_t* recv_off,
                                int32_t* recv_out) {
  if (!m || !m->has_dd) return ADER_ERR_ARG;
  const SubDomain& dd = m->dd;
  const MeshLists& L = dd.lists;
  if (cuts) std::copy(dd.cut.begin(), dd.cut.end(), cuts);
  if (ghosts) std::copy(dd.ghosts.begin(), dd.ghosts.end(), ghosts);
  if (conf_out)
    for (size_t i = 0; i < L.conf.size(); ++i) {
      conf_out[3 * i + 0] = L.conf[i].left;
      conf_out[3 * i + 1] = L.conf[i].right;
      conf_out[3 * i + 2] = L.conf[i].dir;
    }
  if (parents_out)
    for (size_t i = 0; i < L.parents.size(); ++i) {
      parents_out[3 * i + 0] = L.parents[i].coarse;
      parents_out[3 * i + 1] = L.parents[i].dir;
      parents_out[3 * i + 2] = L.parents[i].coarse_side;
    }
  if (child_out) std::copy(L.child_fine.begin(), L.child_fine.end(), child_out);
  if (skel_out) std::copy(L.skel_cells.begin(), L.skel_cells.end(), skel_out);
  int64_t ps = 0, pr = 0;
  for (int q = 0; q < dd.nranks; ++q) {
    if (send_off) send_off[q] = ps;
    if (recv_off) recv_off[q] = pr;
    if (send_out) std::copy(dd.send[size_t(q)].begin(), dd.send[size_t(q)].end(), send_out + ps);
    if (recv_out) std::copy(dd.recv[size_t(q)].begin(), dd.recv[size_t(q)].end(), recv_out + pr);
    ps += int64_t(dd.send[size_t(q)].size());
    pr += int64_t(dd.recv[size_t(q)].size());
  }
  if (send_off) send_off[dd.nranks] = ps;
  if (recv_off) recv_off[dd.nranks] = pr;
  return ADER_OK;
}

ader_status ader_mesh_pipeline(ader_mesh* m, int K, int64_t* chunk_off, int64_t* face_off,
                               int64_t* corr_off, int32_t* corr_cells, int32_t* conf_out,
                               int64_t* nskel_faces) {
  if (!m || K < 1 || K > 64) return ADER_ERR_ARG;
  Tree& t = m->tree;
  t.set_chunks(K);
  if (chunk_off) std::copy(t.chunk_off.begin(), t.chunk_off.end(), chunk_off);
  if (face_off) std::copy(t.face_off.begin(), t.face_off.end(), face_off);
  if (corr_off) std::copy(t.corr_off.begin(), t.corr_off.end(), corr_off);
  if (corr_cells) std::copy(t.corr_cells.begin(), t.corr_cells.end(), corr_cells);
  if (conf_out)
    for (size_t i = 0; i < t.conf.size(); ++i) {
      conf_out[3 * i + 0] = t.conf[i].left;
      conf_out[3 * i + 1] = t.conf[i].right;
      conf_out[3 * i + 2] = t.conf[i].dir;
    }
  if (nskel_faces) *nskel_faces = t.n_conf_skeleton;
  return ADER_OK;
}

}  // extern "C"
