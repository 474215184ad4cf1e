// Batched ADER-DG steps over many independent uniform periodic instances of
// different sizes and orders (Algorithm 1 per instance, global time stepping
// per instance).
//
// Each phase (predictor, Riemann, corrector, dt update) is one persistent
// kernel: every CTA repeatedly takes the next work item (instance, tile of
// cells or faces) from an atomic counter and runs the code path of that
// instance's order -- the consumer-task scheme of Algorithm 2 (a queue of
// logical tasks drained by a fixed set of workers) mapped to CTAs.  Items are
// ordered most expensive first so that the dynamic queue balances the tail.
// A whole multi-step run is one CUDA graph of these phase kernels; phase
// boundaries are kernel boundaries, so no CTA ever waits on another.
#pragma once
#include <type_traits>
#include "batch_types.h"
#include "faces.cuh"
#include "predict.cuh"

namespace ader {

__device__ __forceinline__ int take_item(int32_t* counter) {
  __shared__ int item;
  __syncthreads();
  if (threadIdx.x == 0) item = atomicAdd(counter, 1);
  __syncthreads();
  return item;
}

template <int DIM, class PDE, class Real, int N>
__device__ __forceinline__ void batch_predict_item(const BatchArgs& a, const BatchItem& w,
                                                   unsigned char* smem) {
  using S = PredictShape<DIM, N>;
  const BatchInstance in = a.inst[w.inst];
  const int cl = threadIdx.x < S::CPB * S::NS ? int(threadIdx.x) / S::NS : 0;
  double ihd[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) ihd[d] = in.inv_h;
  const double dt = a.dt[w.inst];
  const int iters = a.iters > 0 ? a.iters : N + 1;
  for (int p = 0; p < w.count; p += S::CPB) {
    const int64_t cell = int64_t(w.first) + p + cl;
    const bool valid = p + cl < w.count;
    predict_cells<DIM, N, PDE, Real>(a.B[N], dt, a.gamma, iters, a.status, a.u + in.u_off,
                                     a.ustar + in.u_off, a.faceQ + in.f_off, a.faceF + in.f_off,
                                     valid ? cell : 0, valid, ihd, smem);
  }
}

// FP32: registers capped for two resident CTAs per SM (the predictor is
// shared-memory bound and needs the warps); FP64 keeps one (FP64-pipe bound).
template <int DIM, class PDE, class Real>
__global__ void __launch_bounds__(256, std::is_same<Real, float>::value ? 2 : 1)
    batch_predict_kernel(const BatchArgs a, int slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (;;) {
    const int it = take_item(a.counters + slot);
    if (it >= a.nitems) break;
    const BatchItem w = a.items[it];
    switch (a.inst[w.inst].order) {
      case 1: batch_predict_item<DIM, PDE, Real, 1>(a, w, smem_raw); break;
      case 2: batch_predict_item<DIM, PDE, Real, 2>(a, w, smem_raw); break;
      case 3: batch_predict_item<DIM, PDE, Real, 3>(a, w, smem_raw); break;
      case 4: batch_predict_item<DIM, PDE, Real, 4>(a, w, smem_raw); break;
      case 5: batch_predict_item<DIM, PDE, Real, 5>(a, w, smem_raw); break;
      case 6: batch_predict_item<DIM, PDE, Real, 6>(a, w, smem_raw); break;
      case 7: batch_predict_item<DIM, PDE, Real, 7>(a, w, smem_raw); break;
      default: break;
    }
  }
}

// Riemann on the conforming faces of uniform periodic instances: face f < C
// joins cell f and its +x neighbour, face C <= f < 2C (3D: < 3C) the +y
// (+z) neighbour.  Eight lanes per face (n <= 8), 32 faces per CTA pass.
template <int DIM, class PDE, int N>
__device__ __forceinline__ void batch_face_item(const BatchArgs& a, const BatchItem& w) {
  constexpr int n = N + 1, NF = ipow(n, DIM - 1), M = PDE::M;
  static_assert(DIM == 2, "batched Riemann: 2D instances");
  const BatchInstance in = a.inst[w.inst];
  const int lane = threadIdx.x & 7;
  const int group = threadIdx.x >> 3;
  const int groups = blockDim.x >> 3;
  for (int p = 0; p < w.count; p += groups) {
    const bool valid = p + group < w.count;
    const int64_t f = int64_t(w.first) + p + group;
    const int64_t C = in.ncells;
    const int d = valid ? int(f / C) : 0;
    const int64_t c = valid ? f - int64_t(d) * C : 0;
    const int64_t x = c % in.side, y = c / in.side;
    const int64_t right = d == 0 ? ((x + 1) % in.side) + y * in.side
                                 : x + ((y + 1) % in.side) * in.side;
    const int64_t oL = in.f_off + (c * 2 * DIM + 2 * d + 1) * M * NF;
    const int64_t oR = in.f_off + (right * 2 * DIM + 2 * d + 0) * M * NF;
    const bool mine = valid && lane < NF;
    double QL[M], QR[M];
    double smax = 0.0;
    bool ok = true;
    if (mine) {
#pragma unroll
      for (int v = 0; v < M; ++v) {
        QL[v] = a.faceQ[oL + v * NF + lane];
        QR[v] = a.faceQ[oR + v * NF + lane];
      }
      bool o1, o2;
      const double l1 = PDE::max_speed(QL, d, a.gamma, &o1);
      const double l2 = PDE::max_speed(QR, d, a.gamma, &o2);
      smax = fmax(l1, l2);
      ok = o1 && o2;
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o, 8));
    if (mine && !ok) atomicOr(a.status, kStatusNonPhysical);
    if (mine) {
      double FL[M], FR[M];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        FL[v] = a.faceF[oL + v * NF + lane];
        FR[v] = a.faceF[oR + v * NF + lane];
      }
      rusanov_store<DIM, N, PDE>(QL, FL, QR, FR, smax, a.fstar + oL + lane, a.fstar + oR + lane, NF);
    }
  }
}

template <int DIM, class PDE>
__global__ void __launch_bounds__(256) batch_face_kernel(const BatchArgs a, int slot) {
  for (;;) {
    const int it = take_item(a.counters + slot);
    if (it >= a.nfitems) break;
    const BatchItem w = a.fitems[it];
    switch (a.inst[w.inst].order) {
      case 1: batch_face_item<DIM, PDE, 1>(a, w); break;
      case 2: batch_face_item<DIM, PDE, 2>(a, w); break;
      case 3: batch_face_item<DIM, PDE, 3>(a, w); break;
      case 4: batch_face_item<DIM, PDE, 4>(a, w); break;
      case 5: batch_face_item<DIM, PDE, 5>(a, w); break;
      case 6: batch_face_item<DIM, PDE, 6>(a, w); break;
      case 7: batch_face_item<DIM, PDE, 7>(a, w); break;
      default: break;
    }
  }
}

// Corrector (UPDATE) or rate only: thread per (cell, node), CPB cells per
// pass; the CTA maximum of sum_d lambda_d / h_d goes to rate[instance].
template <int DIM, class PDE, int N, bool UPDATE>
__device__ __forceinline__ void batch_correct_item(const BatchArgs& a, const BatchItem& w) {
  using SH = PredictShape<DIM, N>;
  constexpr int n = SH::n, NS = SH::NS, NF = SH::NF, CPB = SH::CPB, M = PDE::M;
  const BatchInstance in = a.inst[w.inst];
  const BasisTables& B = a.B[N];
  const int tid = threadIdx.x;
  const bool active = tid < CPB * NS;
  const int cl = active ? tid / NS : 0;
  const int node = active ? tid - cl * NS : 0;
  const int id[3] = {node % n, (node / n) % n, node / (n * n)};
  const double dt = a.dt[w.inst];
  double rate = 0.0;
  for (int p = 0; p < w.count; p += CPB) {
    const bool valid = active && p + cl < w.count;
    if (!valid) continue;
    const int64_t cell = int64_t(w.first) + p + cl;
    double q[M];
    if (UPDATE) {
      double upd[M];
#pragma unroll
      for (int v = 0; v < M; ++v) upd[v] = 0.0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        int fnode;
        if (DIM == 2)
          fnode = d == 0 ? id[1] : id[0];
        else
          fnode = d == 0 ? id[1] + n * id[2] : (d == 1 ? id[0] + n * id[2] : id[0] + n * id[1]);
        const double* F0 = a.fstar + in.f_off + (cell * 2 * DIM + 2 * d + 0) * M * NF + fnode;
        const double* F1 = a.fstar + in.f_off + (cell * 2 * DIM + 2 * d + 1) * M * NF + fnode;
        const double l0 = B.lift0[id[d]] * in.inv_h;
        const double l1 = B.lift1[id[d]] * in.inv_h;
#pragma unroll
        for (int v = 0; v < M; ++v) upd[v] = fma(l0, F0[v * NF], fma(-l1, F1[v * NF], upd[v]));
      }
#pragma unroll
      for (int v = 0; v < M; ++v) {
        const int64_t gi = in.u_off + (cell * M + v) * NS + node;
        q[v] = fma(dt, upd[v], a.ustar[gi]);
        a.u[gi] = q[v];
      }
    } else {
#pragma unroll
      for (int v = 0; v < M; ++v) q[v] = a.u[in.u_off + (cell * M + v) * NS + node];
    }
    bool ok_all = true;
    double node_rate = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      bool ok;
      node_rate += PDE::max_speed(q, d, a.gamma, &ok) * in.inv_h;
      ok_all = ok_all && ok;
    }
    if (!ok_all) {
      atomicOr(a.status, kStatusNonPhysical);
      node_rate = __longlong_as_double(0x7ff8000000000000ll);
    }
    // maximum over the passes of this item (NaN, a non-physical state, sticks)
    rate = (node_rate != node_rate || rate != rate) ? node_rate + rate : fmax(rate, node_rate);
  }
  block_max_to(rate, a.rate + w.inst);
}

template <int DIM, class PDE, bool UPDATE>
__global__ void __launch_bounds__(256) batch_correct_kernel(const BatchArgs a, int slot) {
  for (;;) {
    const int it = take_item(a.counters + slot);
    if (it >= a.nitems) break;
    const BatchItem w = a.items[it];
    switch (a.inst[w.inst].order) {
      case 1: batch_correct_item<DIM, PDE, 1, UPDATE>(a, w); break;
      case 2: batch_correct_item<DIM, PDE, 2, UPDATE>(a, w); break;
      case 3: batch_correct_item<DIM, PDE, 3, UPDATE>(a, w); break;
      case 4: batch_correct_item<DIM, PDE, 4, UPDATE>(a, w); break;
      case 5: batch_correct_item<DIM, PDE, 5, UPDATE>(a, w); break;
      case 6: batch_correct_item<DIM, PDE, 6, UPDATE>(a, w); break;
      case 7: batch_correct_item<DIM, PDE, 7, UPDATE>(a, w); break;
      default: break;
    }
  }
}

// dt[i] = cfl_i / rate[i] for every instance; resets the rate accumulators.
__global__ void batch_finalize_kernel(const BatchArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.ninst) return;
  const double r = __longlong_as_double(static_cast<long long>(a.rate[i]));
  if (!(r > 0.0) || !isfinite(r))
    atomicOr(a.status, kStatusNonFiniteRate);
  else
    a.dt[i] = a.inst[i].cfl / r;
  a.rate[i] = 0ull;
}

}  // namespace ader
