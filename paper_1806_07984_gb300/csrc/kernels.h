// Argument blocks and launch entry points of the ADER-DG device kernels.
//
// Device data layout (all FP64, cell index c, m variables, n = N + 1 nodes
// per direction, node index x fastest, NF = n^(d-1) face nodes with the
// lowest tangential direction fastest):
//   u, ustar      [c][var][node]
//   faceQ, faceF  [c][2 * dir + side][var][fnode]   (side 0: xi_dir = 0)
//   fstar         [c][2 * dir + side][var][fnode]
#pragma once
#include <atomic>
#include <cstdint>

#include <cuda_runtime.h>

#include "basis.h"
#include "mesh.h"

namespace ader {

constexpr int kMaxLevels = 8;

enum StatusBits : uint32_t {
  kStatusNonFinitePredictor = 1u,
  kStatusNonPhysical = 2u,
  kStatusNonFiniteRate = 4u,
  kStatusBadTransfer = 8u,
  kStatusTensorTimeout = 16u,
  kStatusLimiterTransition = 32u,
};

// Per-cell limiter flags of the last step.
enum LimiterFlags : uint32_t {
  kLimited = 1u,        // step redone by FV on the subcell patch
  kFluxReplaced = 2u,   // unlimited, a face flux replaced by the FV subface fluxes
  kKeptAtTransition = 4u,  // troubled, but a face is non-conforming: DG kept
};

struct PredictArgs {
  const double* u;
  double* ustar;
  double* faceQ;
  double* faceF;
  const int32_t* cells;  // cells to process (count entries)
  int64_t count;
  const int8_t* level;   // per cell
  const double* dt;      // device scalar
  double gamma;
  int iters;             // Picard iterations
  uint32_t* status;
  double inv_h[kMaxLevels][3];
  BasisTables B;
  // Shifted task graph (Sec. 3, global time stepping with a prescribed dt):
  // when corr_fstar is set, every node is first corrected with the previous
  // step's u* (in ustar) and F* (in corr_fstar), u = u* + dt lifting(F*),
  // written to corr_u (the buffer u points to), and the predictor starts from
  // that state.
  const double* corr_fstar;
  double* corr_u;
  // 0, or a CTA count: a launch that would have fewer CTAs with CPB cells
  // each takes fewer cells per CTA (small meshes spread over more SMs).
  int32_t min_ctas;
};

struct RiemannArgs {
  const double* faceQ;
  const double* faceF;
  double* fstar;
  const ConfFace* conf;       // conforming faces to solve
  int64_t nconf;
  const ParentFace* parents;  // transitions
  const int32_t* child_fine;  // [parent * 3^(d-1) + sigma]
  int64_t nparents;
  double gamma;
  uint32_t* status;
  int max_ctas;               // conforming faces: at most this many CTAs (0 = one warp per face)
  BasisTables B;
};

struct CorrectArgs {
  const double* ustar;
  const double* fstar;
  double* u;
  const int8_t* level;
  const int32_t* cells;  // cells to process (ncells entries), or null for 0..ncells-1
  int64_t ncells;
  const double* dt;
  unsigned long long* rate_max;  // max over nodes of sum_d lambda_d / h_d (as FP64 bits)
  double gamma;
  uint32_t* status;
  int max_ctas;                  // at most this many CTAs, striding over the cells (0 = no limit)
  double inv_h[kMaxLevels][3];
  BasisTables B;
};

// Solution-based refinement indicator, h_c = max_d h_d:
//   deriv 1: eta[c] = max over the nodes of h_c |grad u_var|;
//   deriv 2: eta[c] = max over the nodes of h_c^2 |Hessian of u_var|_F
// (derivatives by D along each axis).
struct IndicatorArgs {
  const double* u;
  const int8_t* level;
  int64_t ncells;
  int var;
  int deriv;  // 1 or 2
  double* eta;
  double inv_h[kMaxLevels][3];
  BasisTables B;
};

struct TransferArgs {
  const double* u_old;
  double* u_new;
  const TransferItem* plan;
  const int32_t* children;  // coarsening: 3^d old cells per item, lexicographic s
  int64_t ncells_new;
  int64_t ncells_old;
  uint32_t* status;
  BasisTables B;
};

// A posteriori subcell FV limiter (Sec. 4, finite volumes as the limiter of
// ADER-DG on (2N+1)^d subcell patches).
struct LimiterArgs {
  double* u;               // candidate state, overwritten with the final state
  const double* u_old;     // u(T)
  double* u_backup;        // bounds kernel: copy of u(T) written here
  const double* ustar;     // u(T) + dt * volume term
  double* fstar;           // face fluxes; unlimited neighbours of limited cells get FV fluxes
  double* bounds;          // [c][var][2]: min, max of the subcell averages of u(T)
  const int32_t* nbr;      // [c][2 * dir + side]: conforming neighbour or -1
  const uint8_t* force;    // per cell, nonzero = treat as troubled (may be null)
  uint32_t* flags;         // per cell LimiterFlags
  int32_t* list;           // limited cells (counts[0] entries)
  int32_t* fix_list;       // cells with replaced face fluxes (counts[1] entries)
  int* counts;
  const int8_t* level;
  int64_t ncells;
  const double* dt;
  double gamma, delta0, eps;
  unsigned long long* rate_max;
  uint32_t* status;
  double* fv_scratch;      // 3D N >= 6: global scratch slots of the FV kernel's CTAs
  double inv_h[kMaxLevels][3];
  BasisTables B;
  SubcellTables T;
};

enum class LimiterKernel { kBounds = 0, kDetect = 1, kFV = 2, kFix = 3 };

// Limiter kernels for orders 1..7 (pde 0 Euler, 1 acoustics); `grid` is the
// CTA count of the kFV and kFix kernels, which loop over the device-side
// lists.  In 3D at orders 6 and 7 the FV kernel needs
// limiter_fv_scratch_3d(order, pde) doubles of global scratch per CTA.
cudaError_t launch_limiter_2d(int order, int pde, LimiterKernel which, const LimiterArgs& a, int grid,
                              cudaStream_t s);
cudaError_t launch_limiter_3d(int order, int pde, LimiterKernel which, const LimiterArgs& a, int grid,
                              cudaStream_t s);
int64_t limiter_fv_scratch_3d(int order, int pde);

// Opt `kernel` into `bytes` of dynamic shared memory on the current device.
// The attribute is per device, so it is set once per device; `done` is the
// caller's per-kernel set of devices already configured (one bit each).
template <class K>
inline cudaError_t smem_opt_in(std::atomic<uint64_t>& done, K kernel, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
  if (bit != 0 && (done.load(std::memory_order_acquire) & bit) != 0) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

enum class Precision { kFP64 = 0, kFP32 = 1, kTF32 = 2, kTF32x3 = 3, kBF16x3 = 4, kDF64 = 5 };

// Returns cudaErrorInvalidValue when (dim, order, pde, precision) has no
// compiled kernel.
cudaError_t launch_predict(int dim, int order, int pde, Precision prec, const PredictArgs& a,
                           cudaStream_t s);
cudaError_t launch_riemann_conf(int dim, int order, int pde, const RiemannArgs& a, cudaStream_t s);
cudaError_t launch_riemann_child(int dim, int order, int pde, const RiemannArgs& a, cudaStream_t s);
cudaError_t launch_restrict(int dim, int order, int pde, const RiemannArgs& a, cudaStream_t s);
cudaError_t launch_correct(int dim, int order, int pde, const CorrectArgs& a, cudaStream_t s);
cudaError_t launch_rate(int dim, int order, int pde, const CorrectArgs& a, cudaStream_t s);
cudaError_t launch_finalize_dt(unsigned long long* rate_max, double cfl, double* dt_next,
                               uint32_t* status, cudaStream_t s);
cudaError_t launch_transfer(int dim, int order, int nvar, const TransferArgs& a, cudaStream_t s);
// Halo exchange of a partitioned mesh: gather / scatter `count` face slots
// (local cell * 2d + slot) of Q-bar and F-bar, blk = M NF values each.
cudaError_t launch_halo_pack(const double* faceQ, const double* faceF, const int32_t* slots,
                             int64_t count, int blk, double* buf, cudaStream_t s);
cudaError_t launch_halo_unpack(double* faceQ, double* faceF, const int32_t* slots, int64_t count,
                               int blk, const double* buf, cudaStream_t s);

struct AdjointArgs {
  const double* lam_in;   // lambda for u(T+dt)      [c][var][node]
  double* lam_out;        // A^T lambda_in           [c][var][node]
  double* fstar_bar;      // [c][2d][var][fnode] scratch
  double* faceQ_bar;
  double* faceF_bar;
  const ConfFace* conf;
  int64_t nconf;
  const ParentFace* parents;  // resolution transitions
  const int32_t* child_fine;  // [parent * 3^(d-1) + sigma]
  int64_t nparents;
  const int8_t* level;
  int64_t ncells;
  const double* dt;
  int iters;
  int scheme;  // 0 Picard, 1 Cauchy-Kowalevski
  double inv_h[kMaxLevels][3];
  BasisTables B;
};

cudaError_t launch_adjoint(int dim, int order, const AdjointArgs& a, cudaStream_t s);
cudaError_t launch_sample(const double* field, int M, int NS, int var, int npts,
                          const int32_t* cells, const double* weights, double* out, cudaStream_t s);
cudaError_t launch_sample_adjoint(double* field, int M, int NS, int var, int npts,
                                  const int32_t* cells, const double* weights, const double* values,
                                  cudaStream_t s);

}  // namespace ader
