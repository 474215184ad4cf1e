// Face and cell kernels after the predictor (paper Eq. (4), Algorithm 1
// second and third loops, Sec. 2.3 interpolation/restriction):
//
// * riemann_conf  - F_R on conforming faces: Rusanov on time-averaged face
//                   data, F* = (F_L + F_R)/2 - s (Q_R - Q_L)/2, one speed s per
//                   face (max of lambda_d over the face nodes of both sides).
// * riemann_child - the same on child faces of a resolution transition; the
//                   coarse side is the virtual cell's face, obtained by
//                   tangential interpolation P_s of the coarse face data.
// * restrict      - accumulate-Riemann: parent F* = sum_sigma (R_s0 x R_s1)
//                   F*_sigma, children summed in ascending sigma (no atomics,
//                   deterministic); in 3D fused into the child-face kernel.
// * correct       - u = u* + dt sum_d h_d^-1 [lift0_{i_d} F*_{d,-} -
//                   lift1_{i_d} F*_{d,+}] with lift = phi / w, and the CFL
//                   rate max sum_d lambda_d / h_d by warp shuffles and one
//                   atomicMax per CTA.
// * transfer      - remesh volume transfer: copy, interpolate into a child,
//                   or L2-project 3^d children onto the parent.
// All in FP64.  Conforming faces: 32/G faces per warp for faces of at most 32
// nodes (G lanes each), 8 faces per CTA for 36 or 49 nodes; child faces: in
// 3D one CTA per parent face with separable prolongation, in 2D one warp per
// child face (lanes over face nodes).
#pragma once
#include "kernels.h"
#include "pde.cuh"
#include "predict.cuh"

namespace ader {

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ bool warp_all(bool b) { return __all_sync(0xffffffffu, b); }

template <int DIM, int N, class PDE>
__device__ __forceinline__ void rusanov_store(const double (&QL)[PDE::M], const double (&FL)[PDE::M],
                                              const double (&QR)[PDE::M], const double (&FR)[PDE::M],
                                              double s, double* outA, double* outB, int64_t stride) {
#pragma unroll
  for (int v = 0; v < PDE::M; ++v) {
    const double F = 0.5 * (FL[v] + FR[v]) - 0.5 * s * (QR[v] - QL[v]);
    outA[v * stride] = F;
    if (outB) outB[v * stride] = F;
  }
}

// Lanes per face: the face nodes rounded up to a power of two (at most 32),
// so that a warp solves 32 / G faces at once and small faces (2D, low order)
// keep the FP64 pipe busy with full warps.
template <int NF>
struct FaceLanes {
  static constexpr int G = NF > 16 ? 32 : (NF > 8 ? 16 : (NF > 4 ? 8 : (NF > 2 ? 4 : (NF > 1 ? 2 : 1))));
  static constexpr int FPW = 32 / G;              // faces per warp
  static constexpr int PER = (NF + G - 1) / G;    // passes (NF > 32 only)
};

template <int G>
__device__ __forceinline__ double group_max(double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Conforming face f (valid) on the G lanes of one group; gl = lane in group.
template <int DIM, int N, class PDE>
__device__ __forceinline__ void riemann_conf_face(const RiemannArgs& a, int64_t f, bool valid, int gl) {
  constexpr int n = N + 1, NF = ipow(n, DIM - 1), M = PDE::M;
  using FL_ = FaceLanes<NF>;
  constexpr int G = FL_::G, PER = FL_::PER;
  ConfFace cf{};
  if (valid) cf = a.conf[f];
  const int d = cf.dir;
  const int64_t oL = (int64_t(cf.left) * 2 * DIM + 2 * d + 1) * M * NF;
  const int64_t oR = (int64_t(cf.right) * 2 * DIM + 2 * d + 0) * M * NF;
  double QL[PER][M], QR[PER][M];
  double smax = 0.0;
  bool ok = true;
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int fn = gl + G * t;
    if (valid && fn < NF) {
#pragma unroll
      for (int v = 0; v < M; ++v) {
        QL[t][v] = a.faceQ[oL + v * NF + fn];
        QR[t][v] = a.faceQ[oR + v * NF + fn];
      }
      bool o1, o2;
      const double l1 = PDE::max_speed(QL[t], d, a.gamma, &o1);
      const double l2 = PDE::max_speed(QR[t], d, a.gamma, &o2);
      smax = fmax(smax, fmax(l1, l2));
      ok = ok && o1 && o2;
    }
  }
  smax = group_max<G>(smax);
  if (__any_sync(0xffffffffu, !ok) && (threadIdx.x & 31) == 0) atomicOr(a.status, kStatusNonPhysical);
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int fn = gl + G * t;
    if (valid && fn < NF) {
      double FL[M], FR[M];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        FL[v] = a.faceF[oL + v * NF + fn];
        FR[v] = a.faceF[oR + v * NF + fn];
      }
      rusanov_store<DIM, N, PDE>(QL[t], FL, QR[t], FR, smax, a.fstar + oL + fn, a.fstar + oR + fn,
                                 NF);
    }
  }
}

// 32 / G faces per warp; a grid smaller than the face count strides over them.
template <int DIM, int N, class PDE>
__global__ void riemann_conf_kernel(const RiemannArgs a) {
  using FL_ = FaceLanes<ipow(N + 1, DIM - 1)>;
  const int lane = threadIdx.x & 31;
  const int sub = lane / FL_::G, gl = lane % FL_::G;
  const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; w * FL_::FPW < a.nconf;
       w += warps) {
    const int64_t f = w * FL_::FPW + sub;
    riemann_conf_face<DIM, N, PDE>(a, f, f < a.nconf, gl);
  }
}

// Faces whose node count is above 32 and not a multiple of 32 (3D, N = 5, 6):
// one thread per face node, the speed of each face reduced with shared-memory
// atomics on the FP64 bit pattern (non-negative values); no lane idles
// across the two passes a warp per face would take.  8 faces per CTA (288
// threads at 36 nodes: whole warps, every lane busy; 3 faces in 128 threads,
// small enough to sit beside two FP32 predictor CTAs, measured 1.2 % slower
// on the FP32-predictor step).
template <int NF>
struct FaceBlock {
  static constexpr bool kUse = NF > 32 && NF % 32 != 0;
  static constexpr int FPC = 8;
  static constexpr int THREADS = (FPC * NF + 31) / 32 * 32;
};

template <int DIM, int N, class PDE>
__global__ void __launch_bounds__(FaceBlock<ipow(N + 1, DIM - 1)>::THREADS)
    riemann_conf_block_kernel(const RiemannArgs a) {
  constexpr int NF = ipow(N + 1, DIM - 1), M = PDE::M;
  using FB = FaceBlock<NF>;
  __shared__ unsigned long long smax[FB::FPC];
  __shared__ int bad;
  const int slot = threadIdx.x / NF, fn = threadIdx.x % NF;
  const int64_t groups = (a.nconf + FB::FPC - 1) / FB::FPC;
  for (int64_t gidx = blockIdx.x; gidx < groups; gidx += gridDim.x) {
    if (threadIdx.x < FB::FPC) smax[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    const int64_t f = gidx * FB::FPC + slot;
    const bool valid = slot < FB::FPC && f < a.nconf;
    ConfFace cf{};
    if (valid) cf = a.conf[f];
    const int d = cf.dir;
    const int64_t oL = (int64_t(cf.left) * 2 * DIM + 2 * d + 1) * M * NF;
    const int64_t oR = (int64_t(cf.right) * 2 * DIM + 2 * d + 0) * M * NF;
    double QL[M], QR[M];
    if (valid) {
#pragma unroll
      for (int v = 0; v < M; ++v) {
        QL[v] = a.faceQ[oL + v * NF + fn];
        QR[v] = a.faceQ[oR + v * NF + fn];
      }
      bool o1, o2;
      const double l = fmax(PDE::max_speed(QL, d, a.gamma, &o1), PDE::max_speed(QR, d, a.gamma, &o2));
      atomicMax(&smax[slot], static_cast<unsigned long long>(__double_as_longlong(l)));
      if (!(o1 && o2)) bad = 1;
    }
    __syncthreads();
    if (valid) {
      const double sp = __longlong_as_double(static_cast<long long>(smax[slot]));
      double FL[M], FR[M];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        FL[v] = a.faceF[oL + v * NF + fn];
        FR[v] = a.faceF[oR + v * NF + fn];
      }
      rusanov_store<DIM, N, PDE>(QL, FL, QR, FR, sp, a.fstar + oL + fn, a.fstar + oR + fn, NF);
    }
    if (threadIdx.x == 0 && bad) atomicOr(a.status, kStatusNonPhysical);
    __syncthreads();
  }
}

// Tangential interpolation of one coarse face block onto child sub-face
// (s0, s1) at face node (ia, ib): X_v = sum_j P[s1][ib][j] sum_i P[s0][ia][i] X(i + n j).
template <int DIM, int N, int M>
__device__ __forceinline__ void prolong_node(const double* X, int64_t stride, const BasisTables& B,
                                             int s0, int s1, int ia, int ib, double (&out)[M]) {
  constexpr int n = N + 1;
#pragma unroll
  for (int v = 0; v < M; ++v) out[v] = 0.0;
  if (DIM == 2) {
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const double p = B.P[s0][ia][i];
#pragma unroll
      for (int v = 0; v < M; ++v) out[v] = fma(p, X[v * stride + i], out[v]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < n; ++j) {
      double t[M];
#pragma unroll
      for (int v = 0; v < M; ++v) t[v] = 0.0;
#pragma unroll
      for (int i = 0; i < n; ++i) {
        const double p = B.P[s0][ia][i];
#pragma unroll
        for (int v = 0; v < M; ++v) t[v] = fma(p, X[v * stride + i + n * j], t[v]);
      }
      const double p1 = B.P[s1][ib][j];
#pragma unroll
      for (int v = 0; v < M; ++v) out[v] = fma(p1, t[v], out[v]);
    }
  }
}

template <int DIM, int N, class PDE>
__global__ void riemann_child_kernel(const RiemannArgs a) {
  constexpr int n = N + 1, NF = ipow(n, DIM - 1), M = PDE::M, PER = (NF + 31) / 32;
  constexpr int S = DIM == 3 ? 9 : 3;
  const int lane = threadIdx.x & 31;
  const int64_t ci = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (ci >= a.nparents * S) return;
  const int64_t p = ci / S;
  const int sigma = int(ci - p * S);
  const ParentFace pf = a.parents[p];
  const int d = pf.dir, cs = pf.coarse_side;
  const int64_t fine = a.child_fine[ci];
  const int64_t oC = (int64_t(pf.coarse) * 2 * DIM + 2 * d + cs) * M * NF;
  const int64_t oF = (fine * 2 * DIM + 2 * d + (1 - cs)) * M * NF;
  const int s0 = sigma % 3, s1 = sigma / 3;
  double Qv[PER][M], Qf[PER][M];
  double smax = 0.0;
  bool ok = true;
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int fn = lane + 32 * t;
    if (fn < NF) {
      prolong_node<DIM, N, M>(a.faceQ + oC, NF, a.B, s0, s1, fn % n, fn / n, Qv[t]);
#pragma unroll
      for (int v = 0; v < M; ++v) Qf[t][v] = a.faceQ[oF + v * NF + fn];
      bool o1, o2;
      const double l1 = PDE::max_speed(Qv[t], d, a.gamma, &o1);
      const double l2 = PDE::max_speed(Qf[t], d, a.gamma, &o2);
      smax = fmax(smax, fmax(l1, l2));
      ok = ok && o1 && o2;
    }
  }
  smax = warp_max(smax);
  if (!warp_all(ok) && lane == 0) atomicOr(a.status, kStatusNonPhysical);
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int fn = lane + 32 * t;
    if (fn < NF) {
      double Fv[M], Ff[M];
      prolong_node<DIM, N, M>(a.faceF + oC, NF, a.B, s0, s1, fn % n, fn / n, Fv);
#pragma unroll
      for (int v = 0; v < M; ++v) Ff[v] = a.faceF[oF + v * NF + fn];
      if (cs == 1)  // coarse cell on the left
        rusanov_store<DIM, N, PDE>(Qv[t], Fv, Qf[t], Ff, smax, a.fstar + oF + fn, nullptr, NF);
      else
        rusanov_store<DIM, N, PDE>(Qf[t], Ff, Qv[t], Fv, smax, a.fstar + oF + fn, nullptr, NF);
    }
  }
}

// 3D child faces and the restriction, one CTA per parent face and one thread
// per child-face node (3^2 child faces of n^2 nodes).  The coarse face's
// Q-bar and F-bar are interpolated separably: first along the lower
// tangential axis for the three sub-positions s0 (T[s0][ia][j] = sum_i
// P[s0][ia][i] X[i + n j]), then along the upper axis per child node (sum_j
// P[s1][ib][j] T[s0][ia][j]) -- the summation order of prolong_node, so the
// values are the same bit for bit, with about a fifth of its multiply-adds.
// The speed of each child face is reduced in shared memory (atomicMax on the
// FP64 bit pattern of non-negative values).  The child fluxes F*_s then stay
// in shared memory for the coarse slot's restriction sum_s R_s F*_s, taken
// separably in restrict_kernel's order (children s in turn, for each the
// lower axis first), so that it too is the same bit for bit.
template <int N, int M>
struct ChildBlock {
  static constexpr int n = N + 1, NF = n * n, S = 9;
  static constexpr int THREADS = (S * NF + 31) / 32 * 32;
  // shared doubles: phase 1 X[2][M][NF] + T[3][2][M][n][n], phase 2 Fs[S][M][NF]
  static constexpr int kPhase1 = 2 * M * NF + 6 * M * n * n, kPhase2 = S * M * NF;
  static constexpr int kBuf = kPhase1 > kPhase2 ? kPhase1 : kPhase2;
};

template <int DIM, int N, class PDE>
__global__ void __launch_bounds__(ChildBlock<N, PDE::M>::THREADS) riemann_child_block_kernel(const RiemannArgs a) {
  static_assert(DIM == 3, "3D child faces");
  using CB = ChildBlock<N, PDE::M>;
  constexpr int n = CB::n, NF = CB::NF, S = CB::S, M = PDE::M;
  __shared__ double buf[CB::kBuf];
  __shared__ double T2[S][M][n][n];  // restriction after the lower tangential axis
  __shared__ unsigned long long smax[S];
  __shared__ int bad;
  auto X = reinterpret_cast<double (*)[M][NF]>(buf);                      // [2][M][NF]
  auto T = reinterpret_cast<double (*)[2][M][n][n]>(buf + 2 * M * NF);    // [3][2][M][n][n]
  auto Fs = reinterpret_cast<double (*)[M][NF]>(buf);                     // [S][M][NF], after T
  const int tid = threadIdx.x;
  for (int64_t p = blockIdx.x; p < a.nparents; p += gridDim.x) {
    const ParentFace pf = a.parents[p];
    const int d = pf.dir, cs = pf.coarse_side;
    const int64_t oC = (int64_t(pf.coarse) * 2 * DIM + 2 * d + cs) * M * NF;
    __syncthreads();  // the previous parent face is done with the shared buffers
    for (int t = tid; t < 2 * M * NF; t += blockDim.x) {
      const int qf = t / (M * NF), r = t - qf * M * NF;
      X[qf][r / NF][r % NF] = (qf == 0 ? a.faceQ : a.faceF)[oC + r];
    }
    if (tid < S) smax[tid] = 0ull;
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int t = tid; t < 3 * 2 * M * n * n; t += blockDim.x) {
      const int j = t % n, ia = (t / n) % n, v = (t / (n * n)) % M, qf = (t / (n * n * M)) % 2,
                s0 = t / (n * n * M * 2);
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < n; ++i) acc = fma(a.B.P[s0][ia][i], X[qf][v][i + n * j], acc);
      T[s0][qf][v][ia][j] = acc;
    }
    __syncthreads();
    const int sigma = tid / NF, fn = tid - sigma * NF;
    const bool valid = sigma < S;
    double Qv[M], Fv[M], Qf[M], Ff[M];
    int64_t oF = 0;
    if (valid) {
      const int s0 = sigma % 3, s1 = sigma / 3, ia = fn % n, ib = fn / n;
#pragma unroll
      for (int v = 0; v < M; ++v) {
        double q = 0.0, f = 0.0;
#pragma unroll
        for (int j = 0; j < n; ++j) {
          const double w = a.B.P[s1][ib][j];
          q = fma(w, T[s0][0][v][ia][j], q);
          f = fma(w, T[s0][1][v][ia][j], f);
        }
        Qv[v] = q;
        Fv[v] = f;
      }
      const int64_t fine = a.child_fine[p * S + sigma];
      oF = (fine * 2 * DIM + 2 * d + (1 - cs)) * M * NF;
#pragma unroll
      for (int v = 0; v < M; ++v) {
        Qf[v] = a.faceQ[oF + v * NF + fn];
        Ff[v] = a.faceF[oF + v * NF + fn];
      }
      bool o1, o2;
      const double l = fmax(PDE::max_speed(Qv, d, a.gamma, &o1), PDE::max_speed(Qf, d, a.gamma, &o2));
      if (l > 0.0)  // a NaN speed is left out, as fmax does
        atomicMax(&smax[sigma], static_cast<unsigned long long>(__double_as_longlong(l)));
      if (!(o1 && o2)) bad = 1;
    }
    __syncthreads();  // speeds complete; T is no longer read, Fs may overwrite it
    if (valid) {
      const double sp = __longlong_as_double(static_cast<long long>(smax[sigma]));
      if (cs == 1)  // coarse cell on the left
        rusanov_store<DIM, N, PDE>(Qv, Fv, Qf, Ff, sp, a.fstar + oF + fn, &Fs[sigma][0][fn], NF);
      else
        rusanov_store<DIM, N, PDE>(Qf, Ff, Qv, Fv, sp, a.fstar + oF + fn, &Fs[sigma][0][fn], NF);
    }
    if (tid == 0 && bad) atomicOr(a.status, kStatusNonPhysical);
    __syncthreads();
    for (int t = tid; t < S * M * n * n; t += blockDim.x) {
      const int j = t % n, ia = (t / n) % n, v = (t / (n * n)) % M, sg = t / (n * n * M);
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < n; ++i) acc = fma(a.B.R[sg % 3][ia][i], Fs[sg][v][i + n * j], acc);
      T2[sg][v][ia][j] = acc;
    }
    __syncthreads();
    for (int t = tid; t < M * NF; t += blockDim.x) {
      const int v = t / NF, node = t - v * NF, ia = node % n, ib = node / n;
      double acc = 0.0;
      for (int sg = 0; sg < S; ++sg) {
#pragma unroll
        for (int j = 0; j < n; ++j) acc = fma(a.B.R[sg / 3][ib][j], T2[sg][v][ia][j], acc);
      }
      a.fstar[oC + t] = acc;
    }
  }
}

template <int DIM, int N, class PDE>
__global__ void restrict_kernel(const RiemannArgs a) {
  constexpr int n = N + 1, NF = ipow(n, DIM - 1), M = PDE::M, PER = (NF + 31) / 32;
  constexpr int S = DIM == 3 ? 9 : 3;
  const int lane = threadIdx.x & 31;
  const int64_t p = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (p >= a.nparents) return;
  const ParentFace pf = a.parents[p];
  const int d = pf.dir, cs = pf.coarse_side;
  const int64_t oC = (int64_t(pf.coarse) * 2 * DIM + 2 * d + cs) * M * NF;
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int fn = lane + 32 * t;
    if (fn >= NF) continue;
    const int ia = fn % n, ib = fn / n;
    double acc[M];
#pragma unroll
    for (int v = 0; v < M; ++v) acc[v] = 0.0;
    for (int sigma = 0; sigma < S; ++sigma) {
      const int64_t fine = a.child_fine[p * S + sigma];
      const double* X = a.fstar + (fine * 2 * DIM + 2 * d + (1 - cs)) * M * NF;
      const int s0 = sigma % 3, s1 = sigma / 3;
      if (DIM == 2) {
#pragma unroll
        for (int i = 0; i < n; ++i) {
          const double r = a.B.R[s0][ia][i];
#pragma unroll
          for (int v = 0; v < M; ++v) acc[v] = fma(r, X[v * NF + i], acc[v]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < n; ++j) {
          double tt[M];
#pragma unroll
          for (int v = 0; v < M; ++v) tt[v] = 0.0;
#pragma unroll
          for (int i = 0; i < n; ++i) {
            const double r = a.B.R[s0][ia][i];
#pragma unroll
            for (int v = 0; v < M; ++v) tt[v] = fma(r, X[v * NF + i + n * j], tt[v]);
          }
          const double r1 = a.B.R[s1][ib][j];
#pragma unroll
          for (int v = 0; v < M; ++v) acc[v] = fma(r1, tt[v], acc[v]);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < M; ++v) a.fstar[oC + v * NF + fn] = acc[v];
  }
}

// Maximum over the lanes of the calling warp that exist, valid in lane 0.
// A CTA whose size is not a multiple of 32 (216 threads at 3D N=5, 250 at
// 3D N=4, 252 at 2D N=5) ends in a partial warp; its shuffles name only the
// existing lanes and discard what a shuffle from past the last one returns.
// Every existing lane of the warp must call this (1D CTAs).
__device__ __forceinline__ double warp_max_lane0(double v) {
  const int lane = int(threadIdx.x) & 31;
  const int width = min(32, int(blockDim.x) - (int(threadIdx.x) - lane));
  const unsigned mask = width >= 32 ? 0xffffffffu : ((1u << width) - 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double x = __shfl_down_sync(mask, v, o);
    if (lane + o < width) v = fmax(v, x);
  }
  return v;
}

// CTA-wide max, one atomicMax on the FP64 bit pattern (non-negative doubles
// order like their unsigned bit patterns; NaN sorts above +inf).  Any CTA
// size from 1 to 1024 threads; every thread of the CTA must call it.
__device__ __forceinline__ void block_max_to(double v, unsigned long long* out) {
  __shared__ double red[32];
  v = warp_max_lane0(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    double x = lane < nw ? red[lane] : 0.0;
    x = warp_max_lane0(x);
    if (lane == 0) atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(x)));
  }
}

// Corrector CTAs: 128 threads over the flat (cell, node) index, grid-stride.
// A CTA (about 7k registers) fits beside two CTAs of the FP32 predictor, so
// the correctors of the enclave pipeline run on the FP64 pipe next to them.
constexpr int kCorrectThreads = 128;

template <int DIM, int N, class PDE, bool UPDATE>
__global__ void __launch_bounds__(kCorrectThreads) correct_kernel(const CorrectArgs a) {
  using SH = PredictShape<DIM, N>;
  constexpr int NS = SH::NS, M = PDE::M;
  const int64_t total = a.ncells * NS;
  double rate = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t idx = i / NS;
    const int node = int(i - idx * NS);
    const int64_t cell = a.cells ? int64_t(a.cells[idx]) : idx;
    const int lv = int(a.level[cell]);
    double q[M];
    if (UPDATE) {
      lift_node<DIM, N, M>(a.ustar, a.fstar, cell, node, a.B.lift0, a.B.lift1, a.inv_h[lv], *a.dt,
                           a.u, q);
    } else {
#pragma unroll
      for (int v = 0; v < M; ++v) q[v] = a.u[(cell * M + v) * NS + node];
    }
    bool ok_all = true;
    double r = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      bool ok;
      r += PDE::max_speed(q, d, a.gamma, &ok) * a.inv_h[lv][d];
      ok_all = ok_all && ok;
    }
    if (!ok_all) atomicOr(a.status, kStatusNonPhysical);
    rate = fmax(rate, r);
  }
  block_max_to(rate, a.rate_max);
}

// Remesh transfer: one CTA per new cell, threads over the nodes.  A kept cell
// is copied; a refined or coarsened one gets the separable per-axis
// application of P_s (refine) or R_s (coarsen) in shared memory.
template <int DIM, int N, int M>
__global__ void __launch_bounds__(PredictShape<DIM, N>::NS) transfer_kernel(const TransferArgs a) {
  constexpr int n = N + 1, NS = ipow(n, DIM);
  __shared__ double bufA[M * NS], bufB[M * NS];
  const int64_t c = blockIdx.x;
  if (c >= a.ncells_new) return;
  const TransferItem it = a.plan[c];
  const int node = threadIdx.x;
  if (it.kind == 0) {  // a kept cell (most of them): a coalesced copy, no staging
    int64_t src = int64_t(it.src);
    if (src < 0 || src >= a.ncells_old) {
      if (node == 0) atomicOr(a.status, kStatusBadTransfer);
      src = 0;
    }
#pragma unroll
    for (int v = 0; v < M; ++v) a.u_new[(c * M + v) * NS + node] = a.u_old[(src * M + v) * NS + node];
    return;  // the whole CTA (kind is uniform per cell)
  }
  const int id[3] = {node % n, (node / n) % n, node / (n * n)};
  const int stride[3] = {1, n, n * n};
  double acc[M];
#pragma unroll
  for (int v = 0; v < M; ++v) acc[v] = 0.0;
  const int nsrc = it.kind == 2 ? ipow(3, DIM) : 1;
  for (int k = 0; k < nsrc; ++k) {
    int64_t src = it.kind == 2 ? int64_t(a.children[it.src + k]) : int64_t(it.src);
    if (src < 0 || src >= a.ncells_old) {
      if (node == 0) atomicOr(a.status, kStatusBadTransfer);
      src = 0;
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < M; ++v) bufA[v * NS + node] = a.u_old[(src * M + v) * NS + node];
    __syncthreads();
    if (it.kind == 0) {
#pragma unroll
      for (int v = 0; v < M; ++v) acc[v] = bufA[v * NS + node];
      continue;
    }
    int s[3];
    const int sc = it.kind == 1 ? it.child : k;
    s[0] = sc % 3;
    s[1] = (sc / 3) % 3;
    s[2] = sc / 9;
    double* in = bufA;
    double* out = bufB;
    for (int d = 0; d < DIM; ++d) {
      const int base = node - id[d] * stride[d];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < n; ++j) {
          const double m = it.kind == 1 ? a.B.P[s[d]][id[d]][j] : a.B.R[s[d]][id[d]][j];
          t = fma(m, in[v * NS + base + j * stride[d]], t);
        }
        out[v * NS + node] = t;
      }
      __syncthreads();
      double* tmp = in;
      in = out;
      out = tmp;
    }
#pragma unroll
    for (int v = 0; v < M; ++v) acc[v] += in[v * NS + node];
  }
#pragma unroll
  for (int v = 0; v < M; ++v) a.u_new[(c * M + v) * NS + node] = acc[v];
}

// Refinement indicator (epilogue of the corrector), for one variable q:
// DERIV 1, per cell the largest h |grad q| over its nodes; DERIV 2, the
// largest h^2 |H q|_F with H the Hessian (the mixed entries from the first
// derivatives, kept in shared memory, differentiated along the other axis;
// each pair a < b counted twice).  The nodes reduce the squared norm (a tree
// maximum over the FP64 bit patterns, which order like the values for
// non-negative doubles); the square root and the power of h follow once per
// cell, which gives the same value as taking them per node (both are
// monotone and correctly rounded).
template <int DIM, int N, int M, int DERIV>
__global__ void __launch_bounds__(PredictShape<DIM, N>::THREADS) indicator_kernel(const IndicatorArgs a) {
  using SH = PredictShape<DIM, N>;
  constexpr int n = SH::n, NS = SH::NS, CPB = SH::CPB;
  constexpr int kPow2 = pow2_ceil(NS);
  constexpr int NG = DERIV == 2 ? DIM : 1;
  __shared__ double q[CPB][NS];
  __shared__ double sD[n * n];
  __shared__ double gsh[CPB][NG][NS];
  __shared__ unsigned long long r[CPB][NS];
  const int tid = threadIdx.x;
  const int cl = tid / NS;
  const int node = tid - cl * NS;
  const int64_t cell = int64_t(blockIdx.x) * CPB + cl;
  const bool valid = cell < a.ncells;
  for (int t = tid; t < n * n; t += blockDim.x) sD[t] = a.B.D[t / n][t % n];
  q[cl][node] = valid ? a.u[(cell * M + a.var) * NS + node] : 0.0;
  __syncthreads();
  const int id[3] = {node % n, (node / n) % n, node / (n * n)};
  const int stride[3] = {1, n, n * n};
  const int lv = valid ? int(a.level[cell]) : 0;
  double g2 = 0.0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int base = node - id[d] * stride[d];
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < n; ++j) s = fma(sD[id[d] * n + j], q[cl][base + j * stride[d]], s);
    s *= a.inv_h[lv][d];
    if constexpr (DERIV == 2)
      gsh[cl][d][node] = s;
    else
      g2 = fma(s, s, g2);
  }
  if constexpr (DERIV == 2) {
    __syncthreads();
#pragma unroll
    for (int da = 0; da < DIM; ++da)
#pragma unroll
      for (int db = da; db < DIM; ++db) {
        const int base = node - id[db] * stride[db];
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < n; ++j) s = fma(sD[id[db] * n + j], gsh[cl][da][base + j * stride[db]], s);
        s *= a.inv_h[lv][db];
        g2 = fma(da == db ? s : 2.0 * s, s, g2);
      }
  }
  r[cl][node] = static_cast<unsigned long long>(__double_as_longlong(g2));
  for (int st = kPow2 / 2; st > 0; st >>= 1) {
    __syncthreads();
    if (node < st && node + st < NS) r[cl][node] = r[cl][node] > r[cl][node + st] ? r[cl][node] : r[cl][node + st];
  }
  if (valid && node == 0) {
    double hmax = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) hmax = fmax(hmax, 1.0 / a.inv_h[lv][d]);
    const double w = DERIV == 2 ? hmax * hmax : hmax;
    a.eta[cell] = sqrt(__longlong_as_double(static_cast<long long>(r[cl][0]))) * w;
  }
}

template <int DIM, int N, int M>
cudaError_t launch_indicator_t(const IndicatorArgs& a, cudaStream_t s) {
  using SH = PredictShape<DIM, N>;
  if (a.ncells == 0) return cudaSuccess;
  const unsigned blocks = unsigned((a.ncells + SH::CPB - 1) / SH::CPB);
  if (a.deriv == 2)
    indicator_kernel<DIM, N, M, 2><<<blocks, SH::THREADS, 0, s>>>(a);
  else
    indicator_kernel<DIM, N, M, 1><<<blocks, SH::THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

template <int DIM, int N, class PDE>
cudaError_t launch_faces_t(int which, const RiemannArgs& a, cudaStream_t s) {
  constexpr int S = DIM == 3 ? 9 : 3;
  const int threads = 128;
  int64_t items = which == 0 ? a.nconf : (which == 1 ? a.nparents * S : a.nparents);
  if (items == 0) return cudaSuccess;
  int64_t blocks = (items * 32 + threads - 1) / threads;
  if (which == 0) {
    constexpr int FPW = FaceLanes<ipow(N + 1, DIM - 1)>::FPW;
    const int64_t warps = (items + FPW - 1) / FPW;
    blocks = (warps * 32 + threads - 1) / threads;
    if (a.max_ctas > 0 && blocks > a.max_ctas) blocks = a.max_ctas;
  }
  if (which == 0 && FaceBlock<ipow(N + 1, DIM - 1)>::kUse) {
    using FB = FaceBlock<ipow(N + 1, DIM - 1)>;
    int64_t b = (items + FB::FPC - 1) / FB::FPC;
    if (a.max_ctas > 0 && b > a.max_ctas) b = a.max_ctas;
    riemann_conf_block_kernel<DIM, N, PDE><<<unsigned(b), FB::THREADS, 0, s>>>(a);
  } else if (which == 0)
    riemann_conf_kernel<DIM, N, PDE><<<unsigned(blocks), threads, 0, s>>>(a);
  else if (which == 1) {
    if constexpr (DIM == 3)
      riemann_child_block_kernel<DIM, N, PDE><<<unsigned(a.nparents), ChildBlock<N, PDE::M>::THREADS, 0, s>>>(a);
    else
      riemann_child_kernel<DIM, N, PDE><<<unsigned(blocks), threads, 0, s>>>(a);
  } else if constexpr (DIM == 2) {
    restrict_kernel<DIM, N, PDE><<<unsigned(blocks), threads, 0, s>>>(a);
  }  // 3D: the child-face kernel has restricted already
  return cudaGetLastError();
}

template <int DIM, int N, class PDE, bool UPDATE>
cudaError_t launch_correct_t(const CorrectArgs& a, cudaStream_t s) {
  using SH = PredictShape<DIM, N>;
  if (a.ncells == 0) return cudaSuccess;
  int64_t blocks = (a.ncells * SH::NS + kCorrectThreads - 1) / kCorrectThreads;
  if (a.max_ctas > 0 && blocks > a.max_ctas) blocks = a.max_ctas;
  correct_kernel<DIM, N, PDE, UPDATE><<<unsigned(blocks), kCorrectThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <int DIM, int N, int M>
cudaError_t launch_transfer_t(const TransferArgs& a, cudaStream_t s) {
  if (a.ncells_new == 0) return cudaSuccess;
  transfer_kernel<DIM, N, M><<<unsigned(a.ncells_new), ipow(N + 1, DIM), 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ader
