// C ABI of the batched step: many independent uniform periodic 2D Euler
// instances of different sizes and orders, advanced by one CUDA graph of
// persistent phase kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/ader.h"
#include "basis.h"
#include "batch_types.h"
#include "batch_launch.h"

using namespace ader;

struct ader_batch {
  ader_batch_config cfg{};
  Precision prec = Precision::kFP64;
  int ninst = 0;
  std::vector<BatchInstance> inst;
  std::vector<int64_t> u_off;  // ninst + 1
  int64_t u_total = 0, f_total = 0;
  // device
  BatchInstance* d_inst = nullptr;
  BatchItem* d_items = nullptr;
  BatchItem* d_fitems = nullptr;
  int32_t nitems = 0, nfitems = 0;
  double *u = nullptr, *ustar = nullptr, *faceQ = nullptr, *faceF = nullptr, *fstar = nullptr;
  double* dt = nullptr;
  unsigned long long* rate = nullptr;
  int32_t* counters = nullptr;
  int32_t ncounters = 0;
  BasisTables* d_B = nullptr;
  uint32_t* status = nullptr;
  // launch shape (autotuned)
  int blocks_per_sm = 1;
  int tile = 2;
  int sms = 1;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = -1;
  std::string err;
  int64_t launches = 0;
};

namespace {

#define BK(call, what)                                             \
  do {                                                             \
    cudaError_t e__ = (call);                                      \
    if (e__ != cudaSuccess) {                                      \
      b->err = std::string(what) + ": " + cudaGetErrorString(e__); \
      return e__ == cudaErrorMemoryAllocation ? ADER_ERR_OOM : ADER_ERR_CUDA; \
    }                                                              \
  } while (0)

int cpb2d(int order) {
  const int ns = (order + 1) * (order + 1);
  return ns >= 128 ? 1 : 256 / ns;
}

// Cell tiles (tile passes of cpb cells) and face tiles (tile passes of 32
// faces) of every instance, most expensive orders first.
void make_items(const ader_batch* b, int tile, std::vector<BatchItem>* items,
                std::vector<BatchItem>* fitems) {
  items->clear();
  fitems->clear();
  std::vector<int> order_idx(size_t(b->ninst));
  for (int i = 0; i < b->ninst; ++i) order_idx[size_t(i)] = i;
  std::stable_sort(order_idx.begin(), order_idx.end(), [&](int x, int y) {
    return b->inst[size_t(x)].order > b->inst[size_t(y)].order;
  });
  for (int i : order_idx) {
    const BatchInstance& in = b->inst[size_t(i)];
    const int step = cpb2d(in.order) * tile;
    for (int64_t c = 0; c < in.ncells; c += step)
      items->push_back({i, int32_t(c), int32_t(std::min<int64_t>(step, in.ncells - c)), 0});
    const int64_t nf = 2 * in.ncells;
    const int fstep = 32 * tile;
    for (int64_t f = 0; f < nf; f += fstep)
      fitems->push_back({i, int32_t(f), int32_t(std::min<int64_t>(fstep, nf - f)), 0});
  }
}

ader_status upload_items(ader_batch* b) {
  std::vector<BatchItem> items, fitems;
  make_items(b, b->tile, &items, &fitems);
  cudaFree(b->d_items);
  cudaFree(b->d_fitems);
  b->d_items = b->d_fitems = nullptr;
  BK(cudaMalloc(&b->d_items, sizeof(BatchItem) * items.size()), "cudaMalloc items");
  BK(cudaMalloc(&b->d_fitems, sizeof(BatchItem) * fitems.size()), "cudaMalloc items");
  BK(cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice),
     "upload items");
  BK(cudaMemcpy(b->d_fitems, fitems.data(), sizeof(BatchItem) * fitems.size(),
                cudaMemcpyHostToDevice), "upload items");
  b->nitems = int32_t(items.size());
  b->nfitems = int32_t(fitems.size());
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_steps = -1;
  }
  return ADER_OK;
}

BatchArgs args_of(ader_batch* b) {
  BatchArgs a{};
  a.inst = b->d_inst;
  a.ninst = b->ninst;
  a.items = b->d_items;
  a.nitems = b->nitems;
  a.fitems = b->d_fitems;
  a.nfitems = b->nfitems;
  a.u = b->u;
  a.ustar = b->ustar;
  a.faceQ = b->faceQ;
  a.faceF = b->faceF;
  a.fstar = b->fstar;
  a.dt = b->dt;
  a.rate = b->rate;
  a.counters = b->counters;
  a.B = b->d_B;
  a.gamma = b->cfg.gamma;
  a.iters = b->cfg.picard_iters;
  a.status = b->status;
  return a;
}

ader_status ensure_counters(ader_batch* b, int n) {
  if (n <= b->ncounters) return ADER_OK;
  cudaFree(b->counters);
  b->counters = nullptr;
  BK(cudaMalloc(&b->counters, sizeof(int32_t) * size_t(n)), "cudaMalloc counters");
  b->ncounters = n;
  return ADER_OK;
}

// nsteps steps on `s`: counters cleared, then per step 4 kernels.
ader_status enqueue_steps(ader_batch* b, int nsteps, cudaStream_t s) {
  ader_status st = ensure_counters(b, 3 * std::max(nsteps, 1));
  if (st != ADER_OK) return st;
  BK(cudaMemsetAsync(b->counters, 0, sizeof(int32_t) * size_t(3 * nsteps), s), "clear counters");
  const BatchArgs a = args_of(b);
  const int grid = b->sms * b->blocks_per_sm;
  for (int k = 0; k < nsteps; ++k) {
    BK(batch_launch_step(b->prec, a, grid, 3 * k, s), "batched step");
    b->launches += 4;
  }
  return ADER_OK;
}

}  // namespace

extern "C" {

ader_status ader_batch_init(const ader_batch_config* cfg, int ninst, const int* sides,
                            const int* orders, const double* cfls, ader_batch** out) {
  if (!cfg || !sides || !orders || !cfls || !out || ninst < 1) return ADER_ERR_ARG;
  *out = nullptr;
  if (cfg->dim != 2 || cfg->pde != ADER_EULER) return ADER_ERR_ARG;
  if (cfg->prec != ADER_FP64 && cfg->prec != ADER_FP32) return ADER_ERR_ARG;
  for (int i = 0; i < ninst; ++i)
    if (sides[i] < 1 || sides[i] > 4096 || orders[i] < 1 || orders[i] > 7 || !(cfls[i] > 0.0))
      return ADER_ERR_ARG;
  ader_batch* b = new ader_batch();
  b->cfg = *cfg;
  b->prec = cfg->prec == ADER_FP32 ? Precision::kFP32 : Precision::kFP64;
  b->ninst = ninst;
  const int M = 4;
  int64_t uo = 0, fo = 0;
  b->u_off.push_back(0);
  for (int i = 0; i < ninst; ++i) {
    BatchInstance in{};
    in.order = orders[i];
    in.side = sides[i];
    in.ncells = int64_t(sides[i]) * sides[i];
    in.u_off = uo;
    in.f_off = fo;
    in.inv_h = double(sides[i]);
    in.cfl = cfls[i];
    const int64_t n = orders[i] + 1;
    uo += in.ncells * M * n * n;
    fo += in.ncells * 2 * 2 * M * n;
    b->inst.push_back(in);
    b->u_off.push_back(uo);
  }
  b->u_total = uo;
  b->f_total = fo;
  auto fail = [&](ader_status s) {
    ader_batch_destroy(b);
    return s;
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(ADER_ERR_CUDA);
  if (batch_configure(b->prec) != cudaSuccess) return fail(ADER_ERR_CUDA);
  int occ = 0;
  if (batch_occupancy(b->prec, &occ) != cudaSuccess || occ < 1) return fail(ADER_ERR_CUDA);
  b->blocks_per_sm = occ;
  std::vector<BasisTables> tables(8);
  for (int N = 1; N <= 7; ++N) make_basis(N + 1, &tables[size_t(N)]);
  const size_t ub = sizeof(double) * size_t(uo), fb = sizeof(double) * size_t(fo);
  if (cudaMalloc(&b->u, ub) != cudaSuccess || cudaMalloc(&b->ustar, ub) != cudaSuccess ||
      cudaMalloc(&b->faceQ, fb) != cudaSuccess || cudaMalloc(&b->faceF, fb) != cudaSuccess ||
      cudaMalloc(&b->fstar, fb) != cudaSuccess ||
      cudaMalloc(&b->dt, sizeof(double) * size_t(ninst)) != cudaSuccess ||
      cudaMalloc(&b->rate, sizeof(unsigned long long) * size_t(ninst)) != cudaSuccess ||
      cudaMalloc(&b->d_inst, sizeof(BatchInstance) * size_t(ninst)) != cudaSuccess ||
      cudaMalloc(&b->d_B, sizeof(BasisTables) * 8) != cudaSuccess ||
      cudaMalloc(&b->status, sizeof(uint32_t)) != cudaSuccess)
    return fail(ADER_ERR_OOM);
  if (cudaMemset(b->u, 0, ub) != cudaSuccess || cudaMemset(b->rate, 0, 8 * size_t(ninst)) != cudaSuccess ||
      cudaMemset(b->dt, 0, 8 * size_t(ninst)) != cudaSuccess ||
      cudaMemset(b->status, 0, sizeof(uint32_t)) != cudaSuccess ||
      cudaMemcpy(b->d_inst, b->inst.data(), sizeof(BatchInstance) * size_t(ninst),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_B, tables.data(), sizeof(BasisTables) * 8, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(ADER_ERR_CUDA);
  ader_status st = upload_items(b);
  if (st != ADER_OK) return fail(st);
  *out = b;
  return ADER_OK;
}

void ader_batch_destroy(ader_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void* p : {(void*)b->d_inst, (void*)b->d_items, (void*)b->d_fitems, (void*)b->u,
                  (void*)b->ustar, (void*)b->faceQ, (void*)b->faceF, (void*)b->fstar, (void*)b->dt,
                  (void*)b->rate, (void*)b->counters, (void*)b->d_B, (void*)b->status})
    if (p) cudaFree(p);
  delete b;
}

const char* ader_batch_last_error(ader_batch* b) { return b ? b->err.c_str() : "null batch"; }

ader_status ader_batch_offsets(ader_batch* b, int64_t* offsets) {
  if (!b || !offsets) return ADER_ERR_ARG;
  std::memcpy(offsets, b->u_off.data(), sizeof(int64_t) * b->u_off.size());
  return ADER_OK;
}

ader_status ader_batch_set_state(ader_batch* b, const double* u, int on_device, void* stream) {
  if (!b || !u) return ADER_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BK(cudaMemcpyAsync(b->u, u, sizeof(double) * size_t(b->u_total),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s), "set state");
  if (!on_device) BK(cudaStreamSynchronize(s), "set state sync");
  return ADER_OK;
}

ader_status ader_batch_get_state(ader_batch* b, double* u, int on_device, void* stream) {
  if (!b || !u) return ADER_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BK(cudaMemcpyAsync(u, b->u, sizeof(double) * size_t(b->u_total),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s), "get state");
  if (!on_device) BK(cudaStreamSynchronize(s), "get state sync");
  return ADER_OK;
}

ader_status ader_batch_compute_dt(ader_batch* b, void* stream) {
  if (!b) return ADER_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ader_status st = ensure_counters(b, 1);
  if (st != ADER_OK) return st;
  BK(cudaMemsetAsync(b->counters, 0, sizeof(int32_t), s), "clear counter");
  BK(batch_launch_rate(args_of(b), b->sms * b->blocks_per_sm, 0, s), "rate");
  b->launches += 2;
  return ADER_OK;
}

ader_status ader_batch_get_dt(ader_batch* b, double* dt_host) {
  if (!b || !dt_host) return ADER_ERR_ARG;
  BK(cudaDeviceSynchronize(), "sync");
  BK(cudaMemcpy(dt_host, b->dt, sizeof(double) * size_t(b->ninst), cudaMemcpyDeviceToHost), "get dt");
  return ADER_OK;
}

ader_status ader_batch_set_launch(ader_batch* b, int blocks_per_sm, int tile) {
  if (!b || blocks_per_sm < 1 || tile < 1 || tile > 64) return ADER_ERR_ARG;
  int occ = 0;
  if (batch_occupancy(b->prec, &occ) != cudaSuccess) return ADER_ERR_CUDA;
  if (blocks_per_sm > occ) return ADER_ERR_ARG;
  b->blocks_per_sm = blocks_per_sm;
  b->tile = tile;
  return upload_items(b);
}

ader_status ader_batch_tune(ader_batch* b, int* blocks_per_sm_out, int* tile_out, float* ms_out) {
  if (!b) return ADER_ERR_ARG;
  int occ = 0;
  if (batch_occupancy(b->prec, &occ) != cudaSuccess) return ADER_ERR_CUDA;
  BK(cudaDeviceSynchronize(), "sync");
  // the trials advance the state: keep a copy and restore it afterwards
  double* u_save = nullptr;
  double* dt_save = nullptr;
  BK(cudaMalloc(&u_save, sizeof(double) * size_t(b->u_total)), "cudaMalloc tune");
  BK(cudaMalloc(&dt_save, sizeof(double) * size_t(b->ninst)), "cudaMalloc tune");
  BK(cudaMemcpy(u_save, b->u, sizeof(double) * size_t(b->u_total), cudaMemcpyDeviceToDevice), "save");
  BK(cudaMemcpy(dt_save, b->dt, sizeof(double) * size_t(b->ninst), cudaMemcpyDeviceToDevice), "save");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_bps = b->blocks_per_sm, best_tile = b->tile;
  const int tiles[] = {1, 2, 4, 8};
  ader_status st = ADER_OK;
  for (int bps = 1; bps <= occ && st == ADER_OK; ++bps) {
    for (int tile : tiles) {
      b->blocks_per_sm = bps;
      b->tile = tile;
      st = upload_items(b);
      if (st != ADER_OK) break;
      float t = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        BK(cudaMemcpy(b->u, u_save, sizeof(double) * size_t(b->u_total), cudaMemcpyDeviceToDevice), "restore");
        BK(cudaMemcpy(b->dt, dt_save, sizeof(double) * size_t(b->ninst), cudaMemcpyDeviceToDevice), "restore");
        cudaEventRecord(e0, nullptr);
        st = enqueue_steps(b, 1, nullptr);
        if (st != ADER_OK) break;
        cudaEventRecord(e1, nullptr);
        BK(cudaEventSynchronize(e1), "tune sync");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) t = std::min(t, ms);
      }
      if (t < best) {
        best = t;
        best_bps = bps;
        best_tile = tile;
      }
    }
  }
  BK(cudaMemcpy(b->u, u_save, sizeof(double) * size_t(b->u_total), cudaMemcpyDeviceToDevice), "restore");
  BK(cudaMemcpy(b->dt, dt_save, sizeof(double) * size_t(b->ninst), cudaMemcpyDeviceToDevice), "restore");
  cudaFree(u_save);
  cudaFree(dt_save);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != ADER_OK) return st;
  b->blocks_per_sm = best_bps;
  b->tile = best_tile;
  st = upload_items(b);
  if (st != ADER_OK) return st;
  if (blocks_per_sm_out) *blocks_per_sm_out = best_bps;
  if (tile_out) *tile_out = best_tile;
  if (ms_out) *ms_out = best;
  return ADER_OK;
}

ader_status ader_batch_run(ader_batch* b, int nsteps, void* stream) {
  if (!b || nsteps < 0) return ADER_ERR_ARG;
  if (nsteps == 0) return ADER_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!b->graph || b->graph_steps != nsteps) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    ader_status st = ensure_counters(b, 3 * nsteps);
    if (st != ADER_OK) return st;
    cudaStream_t cap;
    BK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
    BK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    const int64_t before = b->launches;
    st = enqueue_steps(b, nsteps, cap);
    b->launches = before;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (st != ADER_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    BK(e, "end capture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    BK(e, "instantiate graph");
    b->graph_steps = nsteps;
  }
  BK(cudaGraphLaunch(b->graph, s), "graph launch");
  b->launches += 4 * int64_t(nsteps);
  return ADER_OK;
}

ader_status ader_batch_status_word(ader_batch* b, uint32_t* out) {
  if (!b || !out) return ADER_ERR_ARG;
  BK(cudaDeviceSynchronize(), "sync");
  BK(cudaMemcpy(out, b->status, sizeof(uint32_t), cudaMemcpyDeviceToHost), "read status");
  BK(cudaMemset(b->status, 0, sizeof(uint32_t)), "clear status");
  return ADER_OK;
}

ader_status ader_batch_launch_count(ader_batch* b, int64_t* out) {
  if (!b || !out) return ADER_ERR_ARG;
  *out = b->launches;
  return ADER_OK;
}

}  // extern "C"
