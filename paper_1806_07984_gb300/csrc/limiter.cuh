// A posteriori subcell finite-volume limiter (paper Sec. 4, "Finite Volumes":
// where the ADER-DG candidate is physically wrong or oscillates, the cell's
// step is rolled back and redone by FV on a (2N+1)^d subcell patch; detection
// and the subcell operators follow Dumbser, Zanotti, Loubere and Diot,
// J. Comput. Phys. 278 (2014)).
//
// One step in limiter mode, after the unlimited predictor and Riemann solves:
//   bounds  - every cell: backup of u(T) and, per variable, min and max of
//             its subcell averages v = (A x A [x A]) u(T);
//   (corrector on all cells: the candidate)
//   detect  - every cell: non-finite or (Euler) rho <= 0 or p <= 0 at a node
//             or subcell average of the candidate, or the relaxed discrete
//             maximum principle min_V - delta <= v~ <= max_V + delta over the
//             cell and its conforming face neighbours V, delta = max(delta0,
//             eps (max_V - min_V)); troubled cells with a non-conforming face
//             keep the candidate (status bit 32), the others join the list;
//   fv      - per limited cell: subcell averages of u(T), the adjacent
//             subcell layer of each face neighbour as halo, one first-order
//             Rusanov FV step of size dt, nodes back by least squares R; the
//             subface fluxes of each face are L2-projected (Pi) onto the face
//             nodes of an unlimited neighbour, whose corrector is redone;
//   fix     - per such neighbour: u = u* + face lifting of the new F*.
// Shared-memory layouts use x fastest (subcell index sx + S sy + S^2 sz) and
// the lowest tangential direction fastest on faces, as the face data do.
#pragma once
#include <climits>
#include "faces.cuh"
#include "kernels.h"
#include "pde.cuh"

namespace ader {

template <int DIM, int N>
struct LimShape {
  static constexpr int n = N + 1;
  static constexpr int S = 2 * N + 1;
  static constexpr int NS = ipow(n, DIM);     // nodes
  static constexpr int SS = ipow(S, DIM);     // subcells
  static constexpr int SF = ipow(S, DIM - 1);  // subfaces of one face
  static constexpr int THREADS = 256;
  // bounds / detection: one CTA per cell, about one thread per subcell
  static constexpr int CELL_THREADS = SS <= 64 ? 64 : (SS <= 128 ? 128 : 256);
};

// Stage the 1D tables in shared memory (dynamic indices stay out of the
// kernel parameter space).
template <int N>
__device__ __forceinline__ void load_tables(const SubcellTables& T, double* sA, double* sR, double* sPi) {
  constexpr int n = N + 1, S = 2 * N + 1;
  for (int t = threadIdx.x; t < S * n; t += blockDim.x) {
    const int s = t / n, j = t % n;
    sA[t] = T.A[s][j];            // sA[s * n + j]
    if (sR) sR[j * S + s] = T.R[j][s];
    if (sPi) sPi[j * S + s] = T.Pi[j][s];
  }
}

// Subcell averages of M fields of one cell.  U[v][NS] nodal data (shared),
// X scratch; on return the partial contraction P (all axes but the slowest)
// is in shared memory and the last axis is contracted by `sub_value`.
//   2D: P[v][y][sx]        (M n S)
//   3D: P[v][z][sy][sx]    (M n S^2), scratch T1[v][z][y][sx] (M n^2 S)
template <int DIM, int N, int M>
__device__ __forceinline__ double* subcell_partial(const double* U, const double* sA, double* X) {
  constexpr int n = N + 1, S = 2 * N + 1;
  if constexpr (DIM == 2) {
    double* P = X;
    for (int t = threadIdx.x; t < M * n * S; t += blockDim.x) {
      const int sx = t % S, r = t / S;  // r = v * n + y
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < n; ++i) acc = fma(sA[sx * n + i], U[r * n + i], acc);
      P[t] = acc;
    }
    __syncthreads();
    return P;
  } else {
    double* T1 = X;
    double* P = X + M * n * n * S;
    for (int t = threadIdx.x; t < M * n * n * S; t += blockDim.x) {
      const int sx = t % S, r = t / S;  // r = (v * n + z) * n + y
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < n; ++i) acc = fma(sA[sx * n + i], U[r * n + i], acc);
      T1[t] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < M * n * S * S; t += blockDim.x) {
      const int sx = t % S, sy = (t / S) % S, r = t / (S * S);  // r = v * n + z
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < n; ++j) acc = fma(sA[sy * n + j], T1[(r * n + j) * S + sx], acc);
      P[t] = acc;
    }
    __syncthreads();
    return P;
  }
}

template <int DIM, int N>
constexpr int partial_scratch() {
  return DIM == 2 ? (N + 1) * (2 * N + 1) : (N + 1) * (N + 1) * (2 * N + 1) + (N + 1) * (2 * N + 1) * (2 * N + 1);
}

// Average of variable v over subcell `sub` from the partial contraction.
template <int DIM, int N, int M>
__device__ __forceinline__ double sub_value(const double* P, const double* sA, int v, int sub) {
  constexpr int n = N + 1, S = 2 * N + 1;
  constexpr int SL = ipow(S, DIM - 1);  // subcells per slab of the slowest axis
  const int slow = sub / SL, rest = sub % SL;
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < n; ++k) acc = fma(sA[slow * n + k], P[(v * n + k) * SL + rest], acc);
  return acc;
}

__device__ __forceinline__ double block_reduce(double x, bool is_max, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_xor_sync(0xffffffffu, x, o);
    x = is_max ? fmax(x, y) : fmin(x, y);
  }
  __syncthreads();
  if (lane == 0) red[warp] = x;
  __syncthreads();
  x = red[0];
  for (int w = 1; w < int(blockDim.x >> 5); ++w) x = is_max ? fmax(x, red[w]) : fmin(x, red[w]);
  return x;
}

// ---------------------------------------------------------------- bounds
// Minima and maxima on the integer pipe: a double's bit pattern, with the
// magnitude bits flipped for negative values, orders like the value (-0
// below +0), so min/max and warp reductions need no FP64 instructions (on
// GB300 the FP64 pipe is the scarce one).  A NaN is left out, as fmin/fmax
// do: it maps to the neutral key of the reduction.
__device__ __forceinline__ long long order_key(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
// The same key with -0 mapped to +0, for comparisons that must agree with
// the FP64 ones (which treat the two zeros as equal).
__device__ __forceinline__ long long compare_key(double x) {
  const long long b = __double_as_longlong(x);
  return b == LLONG_MIN ? 0 : (b ^ ((b >> 63) & 0x7fffffffffffffffLL));
}
__device__ __forceinline__ bool is_nan_bits(double x) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
}
__device__ __forceinline__ double key_value(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

template <int DIM, int N, class PDE>
__global__ void __launch_bounds__(256) limiter_bounds_kernel(const LimiterArgs a) {
  using L = LimShape<DIM, N>;
  constexpr int n = L::n, S = L::S, NS = L::NS, SS = L::SS, M = PDE::M;
  constexpr long long kNone = 0x7fffffffffffffffLL;  // neutral key of a minimum
  extern __shared__ double smem[];
  double* sA = smem;
  long long* red = reinterpret_cast<long long*>(sA + S * n);  // [warp][min M | max M]
  double* U = sA + S * n + 16 * M;
  double* X = U + M * NS;
  const int64_t cell = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  load_tables<N>(a.T, sA, nullptr, nullptr);
  for (int t = threadIdx.x; t < M * NS; t += blockDim.x) {
    const double x = a.u[cell * M * NS + t];
    U[t] = x;
    a.u_backup[cell * M * NS + t] = x;
  }
  __syncthreads();
  const double* P = subcell_partial<DIM, N, M>(U, sA, X);
  long long mn[M], mx[M];  // keys; the maximum is kept negated, so both reduce by min
#pragma unroll
  for (int v = 0; v < M; ++v) mn[v] = mx[v] = kNone;
  for (int sub = threadIdx.x; sub < SS; sub += blockDim.x)
#pragma unroll
    for (int v = 0; v < M; ++v) {
      const double x = sub_value<DIM, N, M>(P, sA, v, sub);
      if (is_nan_bits(x)) continue;
      const long long k = order_key(x);
      mn[v] = min(mn[v], k);
      mx[v] = min(mx[v], -k);  // -k: no overflow, k > LLONG_MIN for every non-NaN x
    }
#pragma unroll
  for (int v = 0; v < M; ++v)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn[v] = min(mn[v], __shfl_xor_sync(0xffffffffu, mn[v], o));
      mx[v] = min(mx[v], __shfl_xor_sync(0xffffffffu, mx[v], o));
    }
  if (lane == 0)
#pragma unroll
    for (int v = 0; v < M; ++v) {
      red[warp * 2 * M + v] = mn[v];
      red[warp * 2 * M + M + v] = mx[v];
    }
  __syncthreads();
  if (threadIdx.x < 2 * M) {
    const int v = threadIdx.x % M;
    const bool is_max = threadIdx.x >= M;
    long long k = red[threadIdx.x];
    for (int w = 1; w < int(blockDim.x >> 5); ++w) k = min(k, red[w * 2 * M + threadIdx.x]);
    // all subcell values NaN: NaN, as fmin/fmax of NaNs
    const double x = k == kNone ? __longlong_as_double(0x7ff8000000000000LL) : key_value(is_max ? -k : k);
    a.bounds[(cell * M + v) * 2 + (is_max ? 1 : 0)] = x;
  }
}

// ---------------------------------------------------------------- detect
template <int DIM, int N, class PDE>
__global__ void __launch_bounds__(256) limiter_detect_kernel(const LimiterArgs a) {
  using L = LimShape<DIM, N>;
  constexpr int n = L::n, S = L::S, NS = L::NS, SS = L::SS, M = PDE::M;
  extern __shared__ double smem[];
  double* sA = smem;
  double* lo = sA + S * n;   // [M]
  double* hi = lo + M;       // [M]
  double* U = hi + M;
  double* X = U + M * NS;
  __shared__ long long klo[M], khi[M];
  const int64_t cell = blockIdx.x;
  load_tables<N>(a.T, sA, nullptr, nullptr);
  if (threadIdx.x < M) {
    const int v = threadIdx.x;
    double l = a.bounds[(cell * M + v) * 2 + 0], h = a.bounds[(cell * M + v) * 2 + 1];
    for (int f = 0; f < 2 * DIM; ++f) {
      const int nb = a.nbr[cell * 2 * DIM + f];
      if (nb >= 0) {
        l = fmin(l, a.bounds[(int64_t(nb) * M + v) * 2 + 0]);
        h = fmax(h, a.bounds[(int64_t(nb) * M + v) * 2 + 1]);
      }
    }
    const double delta = fmax(a.delta0, a.eps * (h - l));
    lo[v] = l - delta;
    hi[v] = h + delta;
    // the same bounds as order keys for the integer-pipe comparisons below;
    // a NaN bound admits everything, as the FP64 comparisons would
    klo[v] = is_nan_bits(lo[v]) ? LLONG_MIN : compare_key(lo[v]);
    khi[v] = is_nan_bits(hi[v]) ? LLONG_MAX : compare_key(hi[v]);
  }
  bool bad = false;
  for (int node = threadIdx.x; node < NS; node += blockDim.x) {
    double q[M];
    bool fin = true;
#pragma unroll
    for (int v = 0; v < M; ++v) {
      q[v] = a.u[(cell * M + v) * NS + node];
      U[v * NS + node] = q[v];
      fin = fin && isfinite(q[v]);
    }
    bool ok = true;
    if (PDE::kPositivity) PDE::max_speed(q, 0, a.gamma, &ok);
    bad = bad || !fin || !ok;
  }
  __syncthreads();
  const double* P = subcell_partial<DIM, N, M>(U, sA, X);
  for (int sub = threadIdx.x; sub < SS; sub += blockDim.x) {
    double q[M];
    bool fin = true, dmp = false;
#pragma unroll
    for (int v = 0; v < M; ++v) {
      q[v] = sub_value<DIM, N, M>(P, sA, v, sub);
      fin = fin && isfinite(q[v]);
      const long long k = compare_key(q[v]);  // a NaN value is caught by `fin`
      dmp = dmp || k < klo[v] || k > khi[v];
    }
    bool ok = true;
    if (PDE::kPositivity) PDE::max_speed(q, 0, a.gamma, &ok);
    bad = bad || !fin || !ok || dmp;
  }
  bad = __syncthreads_or(bad) != 0;
  if (threadIdx.x == 0) {
    if (a.force && a.force[cell]) bad = true;
    uint32_t f = 0;
    if (bad) {
      bool conforming = true;
      for (int k = 0; k < 2 * DIM; ++k) conforming = conforming && a.nbr[cell * 2 * DIM + k] >= 0;
      if (conforming) {
        f = kLimited;
        a.list[atomicAdd(&a.counts[0], 1)] = int32_t(cell);
      } else {
        f = kKeptAtTransition;
        atomicOr(a.status, kStatusLimiterTransition);
      }
    }
    a.flags[cell] = f;
  }
}

// ---------------------------------------------------------------- FV step
template <int DIM, int N, int M>
struct FvSmem {
  using L = LimShape<DIM, N>;
  static constexpr int tables = 3 * L::S * L::n + 32;
  static constexpr int V = M * L::SS;
  static constexpr int H = 2 * DIM * M * L::SF;
  static constexpr int U = M * L::NS;
  // scratch: projection (nodes + partial), halo layer, reconstruction, face fluxes
  static constexpr int proj = M * L::NS + M * partial_scratch<DIM, N>();
  static constexpr int recon = DIM == 2 ? M * L::S * L::n : M * (L::S * L::S * L::n + L::S * L::n * L::n);
  static constexpr int X = (proj > recon ? proj : recon) > H ? (proj > recon ? proj : recon) : H;
  static constexpr int doubles = tables + V + H + X;
  // A patch that does not fit one CTA's shared memory (3D, N >= 6) keeps V,
  // the new averages Vn, H and X in a global scratch slot of this CTA (L2
  // resident: a few hundred KB per CTA); shared memory then holds the tables.
  static constexpr bool kBig = size_t(doubles) * 8 > 200 * 1024;
  static constexpr int slot = kBig ? 2 * V + H + X : 0;   // doubles of global scratch per CTA
  static constexpr int smem = kBig ? tables : doubles;
};

// Rusanov flux between states with a local speed.
template <class PDE>
__device__ __forceinline__ void rusanov_point(const double (&qL)[PDE::M], const double (&qR)[PDE::M],
                                              int dr, double gamma, double (&F)[PDE::M]) {
  constexpr int DIM = PDE::DIM, M = PDE::M;
  double fL[DIM][M], fR[DIM][M];
  PDE::fluxes(qL, fL, gamma);
  PDE::fluxes(qR, fR, gamma);
  bool o1, o2;
  const double s = fmax(PDE::max_speed(qL, dr, gamma, &o1), PDE::max_speed(qR, dr, gamma, &o2));
#pragma unroll
  for (int v = 0; v < M; ++v) F[v] = 0.5 * (fL[dr][v] + fR[dr][v]) - 0.5 * s * (qR[v] - qL[v]);
}

template <int DIM, int N, class PDE>
__global__ void __launch_bounds__(256) limiter_fv_kernel(const LimiterArgs a) {
  using L = LimShape<DIM, N>;
  using SM = FvSmem<DIM, N, PDE::M>;
  constexpr int n = L::n, S = L::S, NS = L::NS, SS = L::SS, SF = L::SF, M = PDE::M;
  constexpr int NF = ipow(n, DIM - 1);
  constexpr int PER = (SS + L::THREADS - 1) / L::THREADS;
  extern __shared__ double smem[];
  double* sA = smem;
  double* sR = sA + S * n;
  double* sPi = sR + S * n;
  double* red = sPi + S * n;
  double* V = SM::kBig ? a.fv_scratch + size_t(blockIdx.x) * SM::slot : smem + SM::tables;
  double* H = V + SM::V;
  double* X = H + SM::H;
  double* Vn = X + SM::X;  // kBig: new averages (else they stay in registers)
  double* G = X;  // face fluxes reuse the scratch between projection and reconstruction
  load_tables<N>(a.T, sA, sR, sPi);
  __syncthreads();
  const int count = a.counts[0];
  const double dt = *a.dt;
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    const int64_t cell = a.list[k];
    const int lv = int(a.level[cell]);
    // subcell averages of u(T)
    double* U = X;
    for (int t = threadIdx.x; t < M * NS; t += blockDim.x) U[t] = a.u_old[cell * M * NS + t];
    __syncthreads();
    const double* P = subcell_partial<DIM, N, M>(U, sA, X + M * NS);
    for (int t = threadIdx.x; t < M * SS; t += blockDim.x)
      V[t] = sub_value<DIM, N, M>(P, sA, t / SS, t % SS);
    __syncthreads();
    // halo: the adjacent subcell layer of each face neighbour at time T
    for (int f = 0; f < 2 * DIM; ++f) {
      const int dr = f >> 1, side = f & 1;
      const int64_t nb = a.nbr[cell * 2 * DIM + f];
      const int row = side == 0 ? S - 1 : 0;  // left neighbour: its last layer
      const int str = dr == 0 ? 1 : (dr == 1 ? n : n * n);
      double* Fn = X;                         // [v][tangential nodes], lowest fastest
      for (int t = threadIdx.x; t < M * NF; t += blockDim.x) {
        const int v = t / NF, tn = t % NF;
        int base;
        if (DIM == 2)
          base = dr == 0 ? tn * n : tn;
        else
          base = dr == 0 ? n * tn : (dr == 1 ? (tn % n) + n * n * (tn / n) : tn);
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < n; ++i)
          acc = fma(sA[row * n + i], a.u_old[(nb * M + v) * NS + base + i * str], acc);
        Fn[t] = acc;
      }
      __syncthreads();
      double* Hf = H + f * M * SF;
      if (DIM == 2) {
        for (int t = threadIdx.x; t < M * S; t += blockDim.x) {
          const int v = t / S, s1 = t % S;
          double acc = 0.0;
#pragma unroll
          for (int j = 0; j < n; ++j) acc = fma(sA[s1 * n + j], Fn[v * n + j], acc);
          Hf[t] = acc;
        }
      } else {
        double* T1 = X + M * NF;  // [v][j2][s1]
        for (int t = threadIdx.x; t < M * n * S; t += blockDim.x) {
          const int s1 = t % S, r = t / S;  // r = v * n + j2
          double acc = 0.0;
#pragma unroll
          for (int j = 0; j < n; ++j) acc = fma(sA[s1 * n + j], Fn[r * n + j], acc);
          T1[t] = acc;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < M * S * S; t += blockDim.x) {
          const int s1 = t % S, s2 = (t / S) % S, v = t / (S * S);
          double acc = 0.0;
#pragma unroll
          for (int j = 0; j < n; ++j) acc = fma(sA[s2 * n + j], T1[(v * n + j) * S + s1], acc);
          Hf[t] = acc;
        }
      }
      __syncthreads();
    }
    // first-order FV update of every subcell; boundary subface fluxes to G
    constexpr int PR = SM::kBig ? 1 : PER;  // register slots for the new values
    double vnew[PR][M];
    double rate = 0.0;
#pragma unroll(SM::kBig ? 1 : PER)
    for (int p = 0; p < PER; ++p) {
      const int sub = threadIdx.x + p * L::THREADS;
      const int pr = SM::kBig ? 0 : p;
      if (sub < SS) {
        const int sid[3] = {sub % S, (sub / S) % S, sub / (S * S)};
        double q[M], dv[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          q[v] = V[v * SS + sub];
          dv[v] = 0.0;
        }
#pragma unroll
        for (int dr = 0; dr < DIM; ++dr) {
          const int sstr = dr == 0 ? 1 : (dr == 1 ? S : S * S);
          int tan;
          if (DIM == 2)
            tan = dr == 0 ? sid[1] : sid[0];
          else
            tan = dr == 0 ? sid[1] + S * sid[2] : (dr == 1 ? sid[0] + S * sid[2] : sid[0] + S * sid[1]);
          double qL[M], qR[M], FL[M], FR[M];
#pragma unroll
          for (int v = 0; v < M; ++v) {
            qL[v] = sid[dr] > 0 ? V[v * SS + sub - sstr] : H[((2 * dr + 0) * M + v) * SF + tan];
            qR[v] = sid[dr] < S - 1 ? V[v * SS + sub + sstr] : H[((2 * dr + 1) * M + v) * SF + tan];
          }
          rusanov_point<PDE>(qL, q, dr, a.gamma, FL);
          rusanov_point<PDE>(q, qR, dr, a.gamma, FR);
          const double c = dt * S * a.inv_h[lv][dr];
#pragma unroll
          for (int v = 0; v < M; ++v) dv[v] -= c * (FR[v] - FL[v]);
          if (sid[dr] == 0)
#pragma unroll
            for (int v = 0; v < M; ++v) G[((2 * dr + 0) * M + v) * SF + tan] = FL[v];
          if (sid[dr] == S - 1)
#pragma unroll
            for (int v = 0; v < M; ++v) G[((2 * dr + 1) * M + v) * SF + tan] = FR[v];
        }
#pragma unroll
        for (int v = 0; v < M; ++v) vnew[pr][v] = q[v] + dv[v];
        if constexpr (SM::kBig)
#pragma unroll
          for (int v = 0; v < M; ++v) Vn[v * SS + sub] = vnew[pr][v];
        double r = 0.0;
        bool ok_all = true;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          bool ok;
          r += PDE::max_speed(vnew[pr], d, a.gamma, &ok) * a.inv_h[lv][d];
          ok_all = ok_all && ok;
        }
        if (!ok_all) atomicOr(a.status, kStatusNonPhysical);
        rate = fmax(rate, r);
      }
    }
    __syncthreads();
    if constexpr (SM::kBig) {
      for (int t = threadIdx.x; t < M * SS; t += blockDim.x) V[t] = Vn[t];
    } else {
#pragma unroll
      for (int p = 0; p < PER; ++p) {
        const int sub = threadIdx.x + p * L::THREADS;
        if (sub < SS)
#pragma unroll
          for (int v = 0; v < M; ++v) V[v * SS + sub] = vnew[p][v];
      }
    }
    rate = block_reduce(rate, true, red);
    if (threadIdx.x == 0) {
      const double r = rate;
      atomicMax(a.rate_max, static_cast<unsigned long long>(__double_as_longlong(r)));
    }
    // unlimited neighbours: lift the projected subface fluxes instead of F*
    for (int f = 0; f < 2 * DIM; ++f) {
      const int dr = f >> 1, side = f & 1;
      const int64_t nb = a.nbr[cell * 2 * DIM + f];
      if (a.flags[nb] & kLimited) continue;
      const double* Gf = G + f * M * SF;
      double* dst = a.fstar + (nb * 2 * DIM + 2 * dr + (1 - side)) * M * NF;
      for (int t = threadIdx.x; t < M * NF; t += blockDim.x) {
        const int v = t / NF, tn = t % NF;
        double acc = 0.0;
        if (DIM == 2) {
#pragma unroll
          for (int s1 = 0; s1 < S; ++s1) acc = fma(sPi[tn * S + s1], Gf[v * SF + s1], acc);
        } else {
          const int i1 = tn % n, i2 = tn / n;
          for (int s2 = 0; s2 < S; ++s2) {
            double t1 = 0.0;
#pragma unroll
            for (int s1 = 0; s1 < S; ++s1) t1 = fma(sPi[i1 * S + s1], Gf[(v * S + s2) * S + s1], t1);
            acc = fma(sPi[i2 * S + s2], t1, acc);
          }
        }
        dst[t] = acc;
      }
      if (threadIdx.x == 0) {
        const uint32_t old = atomicOr(&a.flags[nb], uint32_t(kFluxReplaced));
        if (!(old & kFluxReplaced)) a.fix_list[atomicAdd(&a.counts[1], 1)] = int32_t(nb);
      }
    }
    __syncthreads();
    // nodes from the new averages by least squares, written to u
    if (DIM == 2) {
      double* X1 = X;  // [v][sy][i]
      for (int t = threadIdx.x; t < M * S * n; t += blockDim.x) {
        const int i = t % n, r = t / n;  // r = v * S + sy
        double acc = 0.0;
#pragma unroll
        for (int s1 = 0; s1 < S; ++s1) acc = fma(sR[i * S + s1], V[r * S + s1], acc);
        X1[t] = acc;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < M * NS; t += blockDim.x) {
        const int i = t % n, j = (t / n) % n, v = t / NS;
        double acc = 0.0;
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) acc = fma(sR[j * S + s2], X1[(v * S + s2) * n + i], acc);
        a.u[cell * M * NS + t] = acc;
      }
    } else {
      double* X1 = X;                  // [v][sz][sy][i]
      double* X2 = X + M * S * S * n;  // [v][sz][j][i]
      for (int t = threadIdx.x; t < M * S * S * n; t += blockDim.x) {
        const int i = t % n, r = t / n;  // r = (v * S + sz) * S + sy
        double acc = 0.0;
#pragma unroll
        for (int s1 = 0; s1 < S; ++s1) acc = fma(sR[i * S + s1], V[r * S + s1], acc);
        X1[t] = acc;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < M * S * n * n; t += blockDim.x) {
        const int i = t % n, j = (t / n) % n, r = t / (n * n);  // r = v * S + sz
        double acc = 0.0;
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) acc = fma(sR[j * S + s2], X1[((r * S) + s2) * n + i], acc);
        X2[t] = acc;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < M * NS; t += blockDim.x) {
        const int ij = t % (n * n), kz = (t / (n * n)) % n, v = t / NS;
        double acc = 0.0;
#pragma unroll
        for (int s3 = 0; s3 < S; ++s3) acc = fma(sR[kz * S + s3], X2[(v * S + s3) * n * n + ij], acc);
        a.u[cell * M * NS + t] = acc;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- fix
template <int DIM, int N, class PDE>
__global__ void __launch_bounds__(256) limiter_fix_kernel(const LimiterArgs a) {
  constexpr int NS = ipow(N + 1, DIM), M = PDE::M;
  const int count = a.counts[1];
  const double dt = *a.dt;
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    const int64_t cell = a.fix_list[k];
    const int lv = int(a.level[cell]);
    for (int node = threadIdx.x; node < NS; node += blockDim.x) {
      double q[M];
      lift_node<DIM, N, M>(a.ustar, a.fstar, cell, node, a.B.lift0, a.B.lift1, a.inv_h[lv], dt, a.u,
                           q);
    }
  }
}

// Doubles of global scratch per CTA the FV kernel needs (0: shared memory only).
template <int DIM, int N, int M>
constexpr int fv_scratch_slot() { return FvSmem<DIM, N, M>::slot; }

template <int DIM, int N, class PDE>
cudaError_t launch_limiter_t(LimiterKernel which, const LimiterArgs& a, int grid, cudaStream_t s) {
  using L = LimShape<DIM, N>;
  constexpr int M = PDE::M, n = L::n, S = L::S;
  if (which == LimiterKernel::kBounds || which == LimiterKernel::kDetect) {
    if (a.ncells == 0) return cudaSuccess;
    const size_t bytes = sizeof(double) * size_t(S * n + 16 * M + M * L::NS +
                                                 M * partial_scratch<DIM, N>());
    static std::atomic<uint64_t> bounds_set{0}, detect_set{0};
    cudaError_t e = which == LimiterKernel::kBounds
                        ? smem_opt_in(bounds_set, limiter_bounds_kernel<DIM, N, PDE>, bytes)
                        : smem_opt_in(detect_set, limiter_detect_kernel<DIM, N, PDE>, bytes);
    if (e != cudaSuccess) return e;
    if (which == LimiterKernel::kBounds)
      limiter_bounds_kernel<DIM, N, PDE><<<unsigned(a.ncells), L::CELL_THREADS, bytes, s>>>(a);
    else
      limiter_detect_kernel<DIM, N, PDE><<<unsigned(a.ncells), L::CELL_THREADS, bytes, s>>>(a);
  } else if (which == LimiterKernel::kFV) {
    const size_t bytes = sizeof(double) * size_t(FvSmem<DIM, N, M>::smem);
    if (FvSmem<DIM, N, M>::kBig && !a.fv_scratch) return cudaErrorInvalidValue;
    static std::atomic<uint64_t> configured{0};
    cudaError_t e = smem_opt_in(configured, limiter_fv_kernel<DIM, N, PDE>, bytes);
    if (e != cudaSuccess) return e;
    limiter_fv_kernel<DIM, N, PDE><<<unsigned(grid), L::THREADS, bytes, s>>>(a);
  } else {
    limiter_fix_kernel<DIM, N, PDE><<<unsigned(grid), 128, 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace ader
