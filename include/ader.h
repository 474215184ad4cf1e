/*
 * ader.h - C ABI of the GB300 ADER-DG step library (libader.so).
 *
 * One explicit ADER-DG time step on a dynamically adaptive 3^d spacetree
 * Cartesian mesh (Charrier, Hazelwood, Weinzierl, "Enclave Tasking for DG
 * Methods on Dynamically Adaptive Meshes"):
 *   - the PDE is the first-order balance law of Eq. (1) with S = 0, delta = 0;
 *   - one step is Q(T+dT) = (C_Corr o F_R o id|dc + id|T+dT) o C_STP Q(T),
 *     Eq. (4) and Algorithm 1: a space-time predictor per cell, Riemann solves
 *     per face, a corrector per cell;
 *   - at a resolution transition (Sec. 2.3) coarse predictor data are
 *     interpolated to virtual child faces, Riemann is solved on the child
 *     faces only, and the results are restricted into the parent face;
 *   - dynamic adaptivity (Sec. 2.3) refines/coarsens cells between steps;
 *   - enclave tasking (Sec. 3) becomes a skeleton batch (cells at resolution
 *     transitions or flagged for refinement) on a high-priority CUDA stream and
 *     an enclave batch on a low-priority stream.
 *
 * Conventions for every entry point:
 *   - Returns an ader_status; never aborts or throws.  A CUDA failure returns
 *     ADER_ERR_CUDA and ader_last_error() describes it.
 *   - Device work is enqueued asynchronously.  `stream` arguments are
 *     cudaStream_t handles passed as void* (NULL = the legacy default stream);
 *     the call is ordered after earlier work on that stream and later work on
 *     it sees its results.
 *   - The context owns every device buffer (solution, face data, lists).
 *     Caller pointers are borrowed for the duration of the call (host pointers)
 *     or until the enqueued work completes (device pointers).
 *   - dt lives in device memory (a double* from the caller): kernels read it
 *     there, so a step needs no host synchronisation.
 *   - Numerical failures inside kernels (non-finite predictor output, rho <= 0
 *     or p <= 0, non-finite CFL rate) set bits of a device status word that
 *     ader_status_word() reads after synchronising.
 *   - Growing the context's buffers allocates every new buffer before it
 *     releases an old one.  ADER_ERR_OOM from ader_remesh (unpartitioned)
 *     leaves the context as it was before the call: mesh, lists and state.
 *     ADER_ERR_OOM or ADER_ERR_CUDA from ader_init, from ader_remesh on a
 *     partitioned context, or ADER_ERR_CUDA from any call may leave the
 *     context unusable: the only call it accepts afterwards is ader_destroy.
 *
 * Data layout (FP64 throughout at the boundary; c = cell, m = nvar,
 * n = order + 1 Gauss-Legendre nodes per direction, node index with x fastest,
 * NF = n^(dim-1) face nodes with the lowest tangential direction fastest):
 *   state   u[c][var][node]             c in mesh order (ader_mesh_cells)
 *   faces   X[c][2*dir + side][var][fnode]  side 0: face at xi_dir = 0
 * Euler variables: rho, rho v_1..rho v_dim, E.  Acoustics: p, v_1..v_dim.
 */
#ifndef ADER_H_
#define ADER_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ADER_OK = 0,
  ADER_ERR_ARG = -1,          /* invalid argument or unsupported configuration */
  ADER_ERR_CUDA = -2,         /* a CUDA call failed (see ader_last_error) */
  ADER_ERR_OOM = -3,          /* device allocation failed */
  ADER_ERR_NONPHYSICAL = -4,  /* status word reported a non-physical state */
  ADER_ERR_PICARD = -5,       /* status word reported a non-finite predictor */
  ADER_ERR_TIMEOUT = -6,      /* reserved: a bounded device wait expired */
  ADER_ERR_MESH = -7          /* mesh operation failed (balance, transfer) */
} ader_status;

typedef enum { ADER_EULER = 0, ADER_ACOUSTICS = 1 } ader_pde;

/* Arithmetic of the predictor (Picard, time averages, face extrapolation,
 * volume term).  Riemann, restriction, corrector, CFL reduction and the
 * stored state are FP64 in every mode.
 *   ADER_FP64    everything FP64
 *   ADER_FP32    FP32 on the CUDA cores; FP64 zero-mean correction of the
 *                volume term keeps the step conservative to FP64 rounding
 *   ADER_TF32    as FP32, with the Picard derivative contractions on the tensor
 *                cores (tcgen05, TF32 operands, FP32 accumulation in TMEM)
 *   ADER_TF32X3  tensor cores with hi/lo TF32 splits (three products),
 *                close to FP32 accuracy
 *   ADER_BF16X3  tensor cores with hi/lo BF16 splits (three products)
 *   ADER_DF64    double-float: every predictor value is a pair of FP32 numbers
 *                (about 48 significant bits) computed with error-free
 *                transformations on the FP32 pipes
 * The tensor-core modes are available for 3D Euler at orders 5..7. */
typedef enum {
  ADER_FP64 = 0,
  ADER_FP32 = 1,
  ADER_TF32 = 2,
  ADER_TF32X3 = 3,
  ADER_BF16X3 = 4,
  ADER_DF64 = 5
} ader_precision;

typedef enum { ADER_ALL = 0, ADER_SKELETON = 1, ADER_ENCLAVE = 2 } ader_set;

/* Space-time predictor: Picard iteration (Sec. 2.1; any PDE) or, for the
 * linear acoustics PDE, the Cauchy-Kowalevski Taylor expansion in time
 * (Sec. 2.4): d_0 = u, d_{k+1} = -sum_d D^(d) f_d(d_k) / h_d, time average
 * sum_{k<=N} dt^k / (k+1)! d_k. */
typedef enum { ADER_PREDICTOR_PICARD = 0, ADER_PREDICTOR_CK = 1 } ader_predictor;

typedef enum {
  ADER_FIELD_U = 0,       /* u(T) or u(T+dt) after ader_correct        [c][var][node] */
  ADER_FIELD_USTAR = 1,   /* u + dt * volume term (ader_predict)       [c][var][node] */
  ADER_FIELD_FACE_Q = 2,  /* time-averaged predictor on faces          [c][2d][var][fnode] */
  ADER_FIELD_FACE_F = 3,  /* time-averaged normal flux on faces        [c][2d][var][fnode] */
  ADER_FIELD_FSTAR = 4    /* Riemann flux F* (after restriction)       [c][2d][var][fnode] */
} ader_field;

typedef struct {
  int dim;           /* 2 or 3 */
  int order;         /* polynomial order N, 1..7 (n = N + 1 nodes per direction) */
  int nvar;          /* must be dim + 2 (Euler) or dim + 1 (acoustics) */
  ader_pde pde;
  double gamma;      /* Euler ratio of specific heats */
  double cfl;        /* dt = cfl / max_cells max_nodes sum_d lambda_d / h_d */
  int base[3];       /* base grid cells per direction (level 0), periodic */
  double lo[3];      /* domain box */
  double hi[3];
  int max_level;     /* refinement levels above the base grid, 0..6 */
  int picard_iters;  /* Picard iterations; 0 selects order + 1 */
  ader_precision prec;
  ader_predictor predictor;  /* ADER_PREDICTOR_CK: acoustics, FP64 or FP32 */
  int limiter;               /* 1: a posteriori subcell FV limiter in every corrector
                                (orders 1..7, 2D and 3D); see ader_correct, ader_limiter_flags */
  double limiter_delta0;     /* relaxed maximum principle: delta = max(delta0, eps (max - min)); */
  double limiter_eps;        /* values <= 0 select delta0 = 1e-4, eps = 1e-3 */
  int pipeline_chunks;       /* ader_step: enclave chunks K (1 disables; 0 selects 8, or fewer on
                                small meshes: at least 8 predictor CTAs per SM per chunk, recomputed
                                after every remesh); see ader_step */
  int pipeline_ctas;         /* CTAs per SM of the overlapping face/corrector kernels (0 selects 4) */
  int eager_steps;           /* 1: ader_step launches every kernel itself instead of replaying a
                                CUDA graph of one step (captured once per mesh and dt pointer) */
} ader_config;

typedef struct ader_ctx ader_ctx;

/* Create a context on the current CUDA device with the uniform base mesh
 * (every cell at level 0) and a zero state.  *out receives the context. */
ader_status ader_init(const ader_config* cfg, ader_ctx** out);

/* Release every device buffer and stream of the context (synchronises). */
void ader_destroy(ader_ctx* ctx);

/* Human-readable name of a status code. */
const char* ader_error_string(ader_status s);

/* Description of the last failure in this context ("" if none). */
const char* ader_last_error(ader_ctx* ctx);

/* Mesh sizes: cells, skeleton cells, conforming faces, parent faces of
 * resolution transitions (each split into 3^(dim-1) child faces). */
ader_status ader_mesh_info(ader_ctx* ctx, int64_t* ncells, int64_t* nskeleton, int64_t* nconf,
                           int64_t* nparents);

/* Per cell, in mesh order: level, i_x, i_y, i_z (ncells x 4 int32, host).
 * The cell covers [lo + i h, lo + (i + 1) h) with h = (hi - lo) / (base 3^level). */
ader_status ader_mesh_cells(ader_ctx* ctx, int32_t* cells_out);

/* Per cell, in mesh order: 1 if the cell is in the skeleton batch (host). */
ader_status ader_mesh_skeleton(ader_ctx* ctx, uint8_t* skel_out);

/* The library's Gauss-Legendre nodes on [0, 1] (order + 1 doubles, host). */
ader_status ader_nodes(ader_ctx* ctx, double* xi_out);

/* Copy the state u[c][var][node] in (set) or out (get).  on_device != 0 means
 * `u` is a device pointer; otherwise a host pointer (pinned or pageable). */
ader_status ader_set_state(ader_ctx* ctx, const double* u, int on_device, void* stream);
ader_status ader_get_state(ader_ctx* ctx, double* u, int on_device, void* stream);

/* Copy an intermediate field out (layouts in ader_field). */
ader_status ader_get_field(ader_ctx* ctx, ader_field f, double* out, int on_device, void* stream);

/* Global time step from the current state (global time stepping, Sec. 2.1):
 * *dt_dev = cfl / max over cells and nodes of sum_d lambda_d(u) / h_d. */
ader_status ader_compute_dt(ader_ctx* ctx, double* dt_dev, void* stream);

/* C_STP with id|T+dT and id|dc (Eq. (4), Algorithm 1 first loop) on the cells
 * of `set`: Picard iterations of the space-time predictor, then the time
 * averages of the predictor and of its fluxes, their extrapolation to the 2d
 * faces (ADER_FIELD_FACE_Q/F) and u* = u + dt * volume term (ADER_FIELD_USTAR). */
ader_status ader_predict(ader_ctx* ctx, const double* dt_dev, ader_set set, void* stream);

/* F_R (Algorithm 1 second loop) with the AMR tasks of Sec. 2.3.
 * ADER_SKELETON: Rusanov on child faces (coarse data interpolated into the
 * virtual cells' faces), restriction into the parent faces, and conforming
 * faces between two skeleton cells.  ADER_ENCLAVE: the other conforming faces.
 * ADER_ALL: both.  Needs the predictor of every cell that `set` touches. */
ader_status ader_riemann(ader_ctx* ctx, ader_set set, void* stream);

/* C_Corr (Algorithm 1 third loop) on all cells: u = u* + face lifting of F*,
 * then *dt_next_dev = cfl / max sum_d lambda_d(u) / h_d (CTA maxima by warp
 * shuffles, one atomicMax each).  dt_next_dev may equal dt_dev.
 *
 * With cfg.limiter set, the corrected state is a candidate and the a
 * posteriori subcell finite-volume limiter follows (Sec. 4, "Finite Volumes":
 * FV on (2N+1)^d subcell patches as the limiter of ADER-DG; detection after
 * Dumbser et al., J. Comput. Phys. 278 (2014)):
 *   - a cell is troubled when its candidate has a non-finite value, (Euler)
 *     rho <= 0 or p <= 0 at a node or subcell average, or a subcell average
 *     outside [min_V - delta, max_V + delta], V = the subcell averages of u(T)
 *     in the cell and its conforming face neighbours;
 *   - a troubled cell redoes its step from u(T) by one first-order Rusanov FV
 *     step on its subcells (halo: the neighbours' adjacent subcell layers) and
 *     gets its nodal values back by least squares; an unlimited neighbour
 *     lifts the L2 projection of the FV subface fluxes instead of its F*;
 *   - a troubled cell with a non-conforming face keeps its candidate and sets
 *     status bit 5;
 *   - dt_next comes from the final nodes and the limited cells' subcells.
 * Candidate-stage status bits (predictor, Riemann, corrector) go to an
 * internal word in this mode; the status word reports the final state. */
ader_status ader_correct(ader_ctx* ctx, const double* dt_dev, double* dt_next_dev, void* stream);

/* nsteps full steps.  Each step runs the skeleton predictor, transition
 * Riemann/restriction and skeleton conforming faces on the context's
 * high-priority stream, the enclave predictor on its low-priority stream, then
 * the remaining faces and the corrector after both; the step's dt is read from
 * *dt_dev and the next dt written back to it.  Ordered after earlier work on
 * `stream`; later work on `stream` sees the result.
 * With cfg.pipeline_chunks K > 1 the enclave predictor runs as K chunks of
 * contiguous cells on the low-priority stream, and after chunk k the
 * high-priority stream solves the faces whose two cells are then predicted
 * and corrects the cells whose faces are then all solved, so the face and
 * corrector work (FP64) overlaps the remaining predictor chunks.  Those face
 * and corrector kernels are capped at cfg.pipeline_ctas CTAs per SM (striding
 * over their items) so that they share the SMs with predictor CTAs instead of
 * taking them over.  The result does not depend on K or the cap.
 * Unless cfg.eager_steps is set, the first call captures one step (both
 * streams, all launches) into a CUDA graph and every step replays it; a
 * remesh, a reclassification, a change of forced limiter cells or another
 * dt pointer recaptures.  If the capture fails the steps run eagerly. */
ader_status ader_step(ader_ctx* ctx, int nsteps, double* dt_dev, void* stream);

/* Global time stepping with a prescribed time step size (Sec. 3, the shifted
 * task graph: when the admissible time step sizes are known, the pass that
 * finishes step k also issues the predictor tasks of step k + 1).  nsteps
 * steps of *dt_dev (device scalar, read only) on the whole mesh, on the
 * context's high-priority stream: one predictor pass, then per step the face
 * solves (prolongation, Rusanov, restriction) and one pass per cell that
 * corrects the cell (Eq. (4)) and immediately starts its next predictor; the
 * last step ends with the plain corrector and its CFL reduction, whose time
 * step goes to *dt_next_dev (device; NULL discards it).  nsteps + 1 cell
 * passes instead of 2 nsteps.  The state equals nsteps rounds of
 * ader_predict, ader_riemann and ader_correct with the same dt bit for bit.
 * The non-physical-state check of the corrector runs in the final corrector
 * only; the predictor's non-finite check runs every step.  Ordered after
 * earlier work on `stream`, and later work on `stream` sees the result.
 * ADER_ERR_ARG for nsteps < 0, a NULL dt_dev, a partitioned context or the
 * limiter; nsteps == 0 does nothing. */
ader_status ader_step_fixed_dt(ader_ctx* ctx, int nsteps, const double* dt_dev, double* dt_next_dev,
                               void* stream);

/* One step with the state in host memory: u_in (host, [c][var][node], mesh
 * order) is copied in and the new state copied out to u_out (host; may equal
 * u_in), with *dt_dev read and the next dt written back as in ader_step.  The
 * copy in runs on a stream of the context in contiguous cell ranges that end
 * where the enclave pipeline's chunks start, and each enclave chunk's
 * predictor waits only for its own range, so the copy overlaps the predictor;
 * the skeleton predictor follows the last range; the copy out follows the
 * corrector.  The result equals ader_set_state + ader_step + ader_get_state.
 * Host buffers should be page-locked for the copies to overlap.  Ordered
 * after earlier work on `stream`; the copy out is complete when later work on
 * `stream` runs.  Not on a partitioned context or with the limiter. */
ader_status ader_step_host(ader_ctx* ctx, const double* u_in, double* u_out, double* dt_dev,
                           void* stream);

/* Dynamic adaptivity (Sec. 2.3): flags per cell in mesh order (+1 refine,
 * -1 coarsen, 0 keep).  Refines flagged cells below max_level, restores 2:1
 * face balance by further refinement, coarsens complete families of flagged
 * leaves whose parent stays balanced, and transfers the state (interpolation
 * into children, L2 projection onto parents).  Synchronises the device. */
ader_status ader_remesh(ader_ctx* ctx, const int8_t* flags);

/* Solution-based criterion (Sec. 2.4: first or second derivatives of the
 * solution), the AMR epilogue of the corrector, computed on the device from
 * the current state, with h_c = max_d h_d:
 *   deriv 1: eta[c] = max over the nodes of h_c |grad u_var|,
 *   deriv 2: eta[c] = max over the nodes of h_c^2 |Hessian of u_var|_F
 * (Frobenius norm, mixed entries included); flags[c] = +1 if eta > refine_above
 * and the cell is below max_level, -1 if eta < coarsen_below and the cell is
 * above level 0, else 0.  eta_out (host, may be NULL) and flags (host) have
 * one entry per cell in mesh order.  Synchronises the device before and after.
 * ADER_ERR_ARG for var outside [0, nvar), deriv other than 1 or 2, or
 * refine_above < coarsen_below. */
ader_status ader_gradient_flags(ader_ctx* ctx, int var, int deriv, double refine_above,
                                double coarsen_below, double* eta_out, int8_t* flags);

/* The indicator eta of ader_gradient_flags alone, on the device: eta_dev
 * (device, caller-owned, ncells doubles, mesh order) receives eta[c] for
 * variable var and derivative order deriv (1 or 2) from the current state,
 * asynchronously on `stream` (a cudaStream_t; NULL = the legacy default
 * stream).  The caller orders it after the step that wrote the state (same
 * stream, or an event).  ADER_ERR_ARG for a bad var or deriv, or a NULL
 * eta_dev with cells present. */
ader_status ader_gradient_indicator(ader_ctx* ctx, int var, int deriv, double* eta_dev, void* stream);

/* Skeleton batch: transition cells plus cells with flags[c] > 0 (flags may be
 * NULL).  Host call; uploads the new lists (synchronous). */
ader_status ader_classify(ader_ctx* ctx, const int8_t* flags);

/* Geometric refinement criterion (host): +1 for cells below max_level whose
 * box meets the ball (center, radius) in the periodic domain, -1 for cells
 * above level 0 whose parent's box misses it, 0 otherwise. */
ader_status ader_sphere_flags(ader_ctx* ctx, const double center[3], double radius, int8_t* flags);

/* Synchronise the context's streams and return the device status word
 * (bit 0 non-finite predictor, bit 1 non-physical state, bit 2 non-finite
 * CFL rate, bit 3 bad transfer index, bit 4 a bounded wait for the tensor
 * cores expired, bit 5 a troubled cell at a resolution transition kept its
 * DG candidate); clears it. */
ader_status ader_status_word(ader_ctx* ctx, uint32_t* out);

/* Limiter outcome of the last corrector, one uint32 per cell in mesh order
 * (flags: device array when on_device, else host; the host copy
 * synchronises): bit 0 the cell's step was redone by FV on its subcell
 * patch, bit 1 an unlimited cell lifted FV subface fluxes on a face, bit 2
 * troubled at a resolution transition (DG candidate kept).  *nlimited (host,
 * may be NULL) receives the number of cells with bit 0 (synchronises).
 * ADER_ERR_ARG when the context has no limiter. */
ader_status ader_limiter_flags(ader_ctx* ctx, uint32_t* flags, int on_device, int64_t* nlimited,
                               void* stream);

/* Treat the cells with force[c] != 0 (host array, one byte per cell in mesh
 * order) as troubled in every following corrector; NULL clears.  A remesh
 * clears it too.  ADER_ERR_ARG when the context has no limiter. */
ader_status ader_limiter_force(ader_ctx* ctx, const uint8_t* force);

/* Remesh flags that follow the shocks (the paper refines the DG solution down
 * to the FV level near shocks, so that adaptivity never cuts through an FV
 * region): flags[c] = +1 for the cells that were troubled in the last
 * corrector (limited or kept at a transition) and their face neighbours, when
 * below max_level; -1 for every other cell above level 0; else 0.  Host array,
 * one entry per cell in mesh order, for ader_remesh.  Synchronises.
 * ADER_ERR_ARG when the context has no limiter. */
ader_status ader_limiter_refine_flags(ader_ctx* ctx, int8_t* flags);

/* One limited step that leaves no troubled cell at a resolution transition
 * (the paper keeps adaptivity out of FV regions by refining the DG solution
 * down to the FV level near shocks, Sec. 6).  The step runs (ader_step with
 * the limiter); when a troubled cell has a non-conforming face (kept its DG
 * candidate, limiter flag bit 2), the state goes back to u(T), the mesh is
 * refined around the troubled cells (they and their face neighbours below
 * max_level; nothing coarsens), dt is recomputed from u(T) on the refined
 * mesh into *dt_dev, and the step runs again, at most max_rounds times.
 * *rounds (may be NULL) receives the refinements made; after the last step
 * *dt_dev holds its dt_next and the status word its bits (those of discarded
 * attempts are dropped).  Needs cfg.limiter; not on a partitioned context.
 * Synchronises the device. */
ader_status ader_step_refining(ader_ctx* ctx, double* dt_dev, int max_rounds, int* rounds,
                               void* stream);

/* Discrete adjoint of one step: *lambda_out = A^T lambda_in, where A is the
 * linear map u(T) -> u(T+dt) of ader_step/ader_predict+ader_riemann+
 * ader_correct for linear acoustics (ADER_ACOUSTICS) with the dt stored at
 * dt_dev.  Each task of Eq. (4) is transposed in reverse order (corrector
 * lifting, Rusanov with s = c = 1, at resolution transitions (Sec. 2.3) the
 * restriction, child-face Rusanov and prolongation, then the predictor volume
 * term and face extrapolation, time averages, and the Picard iterations
 * unrolled with the forward count, or the Cauchy-Kowalevski sum transposed
 * by Horner's scheme).  FP64 only; any adaptive mesh, not a partitioned
 * context.  lambda arrays are device [c][var][node] and must not alias.  Uses
 * the context's face buffers as scratch. */
ader_status ader_adjoint_step(ader_ctx* ctx, const double* lambda_in, double* lambda_out,
                              const double* dt_dev, void* stream);

/* Point values of one variable: out[p] = sum_node weights[p][node]
 * field[cells[p]][var][node] (device arrays; weights npts x (order+1)^dim, the
 * Lagrange basis at each point's reference coordinates).  field NULL samples
 * the context's state.  ader_sample_adjoint adds the transpose:
 * field[cells[p]][var][node] += weights[p][node] values[p], points in order. */
ader_status ader_sample(ader_ctx* ctx, int npts, const int32_t* cells, const double* weights,
                        int var, const double* field, double* out, void* stream);
ader_status ader_sample_adjoint(ader_ctx* ctx, int npts, const int32_t* cells,
                                const double* weights, int var, const double* values,
                                double* field, void* stream);

/* Fault injection for tests (host side, no device fault): after `after`
 * more successful device allocations, every allocation the library makes
 * while growing buffers (ader_remesh, ader_classify, ader_partition) fails as
 * if the device were out of memory; after < 0 switches it off.  Process-wide;
 * the paper has no counterpart. */
ader_status ader_debug_fail_allocations(int after);

/* Number of kernel launches this context has enqueued so far. */
ader_status ader_launch_count(ader_ctx* ctx, int64_t* out);

/* ---- Domain decomposition (Sec. 3, distributed memory) -------------------
 * The paper splits the space-filling-curve order of the cells into
 * non-overlapping contiguous partitions, solves the Riemann problems on faces
 * between two partitions on both sides, and sends the predictor results of
 * the cells along a partition boundary to the neighbour once per step (those
 * cells are skeleton cells, so that their predictions come first and the
 * enclave predictions hide the exchange).  Here the depth-first cell order is
 * cut into nranks ranges on base-cell boundaries (every family of siblings in
 * one range) with cell counts as even as that allows.  Each rank's context
 * keeps the whole tree on the host (flags and remeshing need no exchange) and
 * on the device only its owned cells plus ghosts: every cell that shares a
 * conforming face or a parent face family with an owned cell.
 *
 * Partitioned context, per step (the caller moves the buffers between ranks:
 * device copies, MPI, NCCL or torch.distributed):
 *   ader_predict(SKELETON); for each peer: ader_halo_pack
 *   ader_predict(ENCLAVE)                     (overlaps the exchange)
 *   exchange the packed buffers; for each peer: ader_halo_unpack
 *   ader_riemann(ALL); ader_correct(dt, dt_local)
 *   dt_next = min over ranks of dt_local      (= cfl / max of the rates)
 * The result equals the unpartitioned step cell for cell, bit for bit.
 * In a partitioned context, state arrays (ader_set_state, ader_get_state,
 * ader_get_field of u and u*) hold the owned cells, ader_mesh_info counts and
 * ader_mesh_cells lists them, and face fields hold owned then ghost cells;
 * flags arrays (ader_remesh, ader_classify, ader_sphere_flags) have one entry
 * per cell of the whole mesh (ader_dd_info's nglobal), identical on every
 * rank.  ader_step, the limiter and the adjoint step are not available. */

/* Partition the context's current mesh into nranks ranges and keep rank
 * `rank` (0 <= rank < nranks); the owned rows of the current state are kept.
 * nranks = 1 leaves the context whole.  Synchronises the device.
 * ADER_ERR_ARG if the context is partitioned already, has the limiter, or
 * nranks exceeds the number of base cells. */
ader_status ader_partition(ader_ctx* ctx, int nranks, int rank);

/* Partition facts (any may be NULL): ranks, this rank, cells of the whole
 * mesh, first owned cell (index into the whole mesh's order), owned cells,
 * ghost cells.  An unpartitioned context reports one rank owning every cell. */
ader_status ader_dd_info(ader_ctx* ctx, int* nranks, int* rank, int64_t* nglobal, int64_t* first,
                         int64_t* nowned, int64_t* nghost);

/* The nranks + 1 cut points in the whole mesh's cell order (rank r owns
 * [cuts[r], cuts[r+1])). */
ader_status ader_dd_cuts(ader_ctx* ctx, int64_t* cuts);

/* Halo exchange with `peer`: sizes in doubles of the buffer this rank sends
 * and of the one it receives (equal to the peer's send size); 0 for a peer
 * that shares no face.  ader_halo_pack writes the predictor's face data
 * (Q-bar and F-bar of each face slot the peer needs, in an order both sides
 * derive from the mesh) into buf_dev; ader_halo_unpack copies a received
 * buffer into the ghosts' face slots.  Device buffers owned by the caller,
 * enqueued on `stream`.  ADER_ERR_ARG for an unpartitioned context or a peer
 * outside [0, nranks). */
ader_status ader_halo_size(ader_ctx* ctx, int peer, int64_t* send_doubles, int64_t* recv_doubles);
ader_status ader_halo_pack(ader_ctx* ctx, int peer, double* buf_dev, void* stream);
ader_status ader_halo_unpack(ader_ctx* ctx, int peer, const double* buf_dev, void* stream);

/* State migration after ader_remesh on a partitioned context.  The remesh
 * transfers the state of the rank's old base-cell range, rebalances the cuts
 * for the new mesh, and keeps the cells it still owns; the cells that change
 * owner go from their old to their new owner through these calls (sizes in
 * doubles; pack reads the rank's transferred cells, unpack writes owned
 * cells).  Every rank must unpack from every peer before the next step.  Valid
 * until the next remesh; sizes are 0 when no remesh has run. */
ader_status ader_migrate_size(ader_ctx* ctx, int peer, int64_t* send_doubles, int64_t* recv_doubles);
ader_status ader_migrate_pack(ader_ctx* ctx, int peer, double* buf_dev, void* stream);
ader_status ader_migrate_unpack(ader_ctx* ctx, int peer, const double* buf_dev, void* stream);

/* ---- Batched instances ---------------------------------------------------
 * Many independent problems of uneven sizes and orders advanced together
 * (Algorithm 1 per instance, each instance with its own global time step).
 * Instance i is a uniform periodic grid of sides[i]^2 cells on the unit
 * square with order orders[i] and Courant factor cfls[i].  Its state is the
 * block u[offsets[i] .. offsets[i+1]) of one concatenated FP64 array, laid
 * out like a context's state.  Every phase of a step (predictor, Riemann,
 * corrector, dt update) is one persistent kernel whose CTAs pull work items
 * (instance, tile of cells or faces) from a queue -- the consumer tasks of
 * Algorithm 2 on CTAs -- and ader_batch_run launches all steps as one CUDA
 * graph.  Currently 2D Euler. */
typedef struct {
  int dim;           /* 2 */
  ader_pde pde;      /* ADER_EULER */
  double gamma;
  int picard_iters;  /* 0 selects order + 1 per instance */
  ader_precision prec;
} ader_batch_config;

typedef struct ader_batch ader_batch;

ader_status ader_batch_init(const ader_batch_config* cfg, int ninst, const int* sides,
                            const int* orders, const double* cfls, ader_batch** out);
void ader_batch_destroy(ader_batch* b);
const char* ader_batch_last_error(ader_batch* b);

/* offsets[0..ninst] (host, int64) of each instance's state in doubles. */
ader_status ader_batch_offsets(ader_batch* b, int64_t* offsets);

/* Concatenated state in/out (on_device: device pointer, else host). */
ader_status ader_batch_set_state(ader_batch* b, const double* u, int on_device, void* stream);
ader_status ader_batch_get_state(ader_batch* b, double* u, int on_device, void* stream);

/* dt of every instance from its current state (device-resident). */
ader_status ader_batch_compute_dt(ader_batch* b, void* stream);
/* Copy the per-instance dt (of the next step) to the host (synchronises). */
ader_status ader_batch_get_dt(ader_batch* b, double* dt_host);

/* Launch shape: persistent CTAs per SM and tile factor (cells per work item =
 * tile x cells per CTA pass). */
ader_status ader_batch_set_launch(ader_batch* b, int blocks_per_sm, int tile);

/* Autotuner: times one step for every (CTAs per SM, tile in {1,2,4,8}) that
 * fits, keeps the fastest, restores the state.  Synchronises. */
ader_status ader_batch_tune(ader_batch* b, int* blocks_per_sm, int* tile, float* ms_per_step);

/* nsteps steps of every instance as one CUDA graph launch on `stream`. */
ader_status ader_batch_run(ader_batch* b, int nsteps, void* stream);

/* Status word as in ader_status_word (synchronises, clears). */
ader_status ader_batch_status_word(ader_batch* b, uint32_t* out);
ader_status ader_batch_launch_count(ader_batch* b, int64_t* out);

/* ---- Allocation-free time step ------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory: code running inside a memory pool or arena
 * it does not own (a host framework that forbids cudaMalloc once it has
 * started, or must not fragment its pool), or a path that must not fail for
 * lack of memory.  It computes the same global time step as ader_compute_dt,
 *   *dt_dev = cfl / max over cells and nodes of sum_d lambda_d(u) / h_d,
 * without a context and without allocating: it calls no cudaMalloc, cudaFree
 * or allocating library routine.  Its scratch (one FP64 partial maximum per
 * CTA) is a fixed device array inside the library, which every GPU that loads
 * the library holds until the process exits.
 *   u_dev      device state u[c][var][node] (layout as above), ncells cells
 *   level_dev  device int8 level per cell, 0 <= level < 8 (other values make
 *              the result NaN); h_d = (hi[d] - lo[d]) / (base[d] 3^level)
 *   dt_dev     device double receiving dt; NaN if a state is non-physical
 *              or if the maximum rate is zero or not finite (the cases in
 *              which the context path sets its non-finite-rate status bit)
 * Sizes: 1 <= ncells <= ADER_DT_STATIC_MAX_CELLS, else ADER_ERR_ARG.
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it for the life of the process; make that first
 * call before any stream capture.  The kept address belongs to the device's
 * primary context: after cudaDeviceReset on that device, do not call this
 * entry point again in the same process.  All calls
 * share the one array and each call overwrites the slots it reads, so calls
 * that overlap on the GPU (different streams, or several host threads) race:
 * serialise them. */
#define ADER_DT_STATIC_MAX_CELLS 1048576
ader_status ader_compute_dt_static(int dim, int order, ader_pde pde, double gamma, double cfl,
                                   const int base[3], const double lo[3], const double hi[3],
                                   int64_t ncells, const double* u_dev, const int8_t* level_dev,
                                   double* dt_dev, void* stream);

/* ---- Host-only mesh handle (no device needed) ---------------------------
 * The same spacetree logic as the context's mesh (Sec. 2.3 three-partitioning,
 * 2:1 face balance, coarsening rules, skeleton of Sec. 3), usable without a
 * GPU for planning and inspection. */
typedef struct ader_mesh ader_mesh;

/* Uniform base grid base[0..dim-1] (periodic), refinement up to max_level. */
ader_status ader_mesh_create(int dim, const int base[3], int max_level, ader_mesh** out);
void ader_mesh_destroy(ader_mesh* mesh);

/* Same flags and rules as ader_remesh, without any state transfer. */
ader_status ader_mesh_adapt(ader_mesh* mesh, const int8_t* flags);

/* Sizes as in ader_mesh_info. */
ader_status ader_mesh_sizes(ader_mesh* mesh, int64_t* ncells, int64_t* nskeleton, int64_t* nconf,
                            int64_t* nparents);

/* Leaves (ncells x 4: level, i_x, i_y, i_z) and skeleton flags in mesh order. */
ader_status ader_mesh_leaves(ader_mesh* mesh, int32_t* cells_out, uint8_t* skel_out);

/* Faces: conf_out (nconf x 3: left cell, right cell, dir; skeleton-only faces
 * first), parents_out (nparents x 3: coarse cell, dir, coarse side), and
 * child_out (nparents x 3^(dim-1): fine cell of sub-face sigma). */
ader_status ader_mesh_faces(ader_mesh* mesh, int32_t* conf_out, int32_t* parents_out,
                            int32_t* child_out);

/* Geometric criterion of ader_sphere_flags on the box [lo, hi]. */
ader_status ader_mesh_sphere_flags(ader_mesh* mesh, const double center[3], double radius,
                                   const double lo[3], const double hi[3], int8_t* flags);

/* The remesh rule of ader_limiter_refine_flags for a given troubled set
 * (troubled[c] != 0, one byte per cell in mesh order). */
ader_status ader_mesh_refine_around(ader_mesh* mesh, const uint8_t* troubled, int8_t* flags);

/* The partition of ader_partition on the host mesh: sizes[9] receives the
 * first owned cell, owned cells, ghosts, local conforming faces, those
 * between two owned skeleton cells (listed first), local parent faces,
 * skeleton cells, and the send and receive entries over all peers.
 * ader_mesh_subdomain then fills (any may be NULL): cuts[nranks + 1], ghosts
 * (index in the whole mesh of ghost g = local cell nowned + g), conf_out
 * (left, right, dir in local cells), parents_out (coarse, dir, coarse side)
 * with child_out (3^(dim-1) fine cells each), skel_out (local skeleton
 * cells), and per peer the exchange entries local_cell * 2 dim + (2 dir +
 * side) at send_out[send_off[q] .. send_off[q+1]) and recv_out likewise.
 * ader_mesh_adapt discards the partition. */
ader_status ader_mesh_partition(ader_mesh* mesh, int nranks, int rank, int64_t* sizes);
ader_status ader_mesh_subdomain(ader_mesh* mesh, int64_t* cuts, int32_t* ghosts, int32_t* conf_out,
                                int32_t* parents_out, int32_t* child_out, int32_t* skel_out,
                                int64_t* send_off, int32_t* send_out, int64_t* recv_off,
                                int32_t* recv_out);

/* The enclave pipeline of ader_step for K chunks (see ader_step) on the host
 * mesh, whose skeleton is its transition cells: fills chunk_off[K+1]
 * (enclave cell ranges in ader_mesh_leaves order), face_off[K+1]
 * (conforming faces after the skeleton ones, per chunk), corr_off[K+2] and
 * corr_cells[ncells] (cells grouped by the stage that completes their faces),
 * and conf_out[3 * nconf] (left, right, dir in pipeline order); *nskel_faces
 * receives the number of skeleton conforming faces.  Every output may be NULL. */
ader_status ader_mesh_pipeline(ader_mesh* mesh, int K, int64_t* chunk_off, int64_t* face_off,
                               int64_t* corr_off, int32_t* corr_cells, int32_t* conf_out,
                               int64_t* nskel_faces);

#ifdef __cplusplus
}
#endif

#endif /* ADER_H_ */
