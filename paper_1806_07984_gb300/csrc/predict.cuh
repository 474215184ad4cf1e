// Space-time predictor C_STP (paper Sec. 2.1-2.2, Eq. (4), Algorithm 1 first
// loop) fused with id|T+dT, id|dc and the corrector's volume term.
//
// Per cell and spatial node i, Picard iteration on the time-weak predictor
// equation (integrated by parts in time with the upwind inflow u, strong-form
// nodal flux divergence, neighbours ignored):
//   q^(0)_k   = u
//   q^(r+1)_k = u - dt sum_l Mt[k][l] sum_d h_d^-1 (D^(d) f_d(q^(r)_l))_i,
// with Mt = K1^{-1} diag(w) (K1^{-1} theta(0) = 1 folds the inflow term).
// After I iterations:
//   Q-bar   = sum_k w_k q_k,  F-bar_d = sum_k w_k f_d(q_k)
//   u*      = u + dt sum_d h_d^-1 (V^(d) F-bar_d)_i,  V = W^-1 D^T W
//   faces   : Q-bar and F-bar_d extrapolated with phi(0), phi(1) along d.
//
// GB300 mapping: one thread per spatial node, CPB cells per CTA.  Each thread
// keeps its node's space-time column q[n][m] and the Picard accumulator in
// registers; the fluxes of one time slice are staged in shared memory so that
// the 1D derivative contractions along every axis read neighbours on chip.
// The space-time block never touches HBM: the kernel reads u once and writes
// u* and the 2d face blocks once.
#pragma once
#include <type_traits>

#include "df64.cuh"
#include "kernels.h"
#include "pde.cuh"
#include "tc.cuh"

namespace ader {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }
// Smallest power of two >= x (x >= 1).
__host__ __device__ constexpr int pow2_ceil(int x) { return x <= 1 ? 1 : 2 * pow2_ceil((x + 1) / 2); }

template <int DIM, int N>
struct PredictShape {
  static constexpr int n = N + 1;
  static constexpr int NS = ipow(n, DIM);
  static constexpr int NF = ipow(n, DIM - 1);
  static constexpr int CPB = NS >= 128 ? 1 : (256 / NS);
  static constexpr int THREADS = CPB * NS;
};

// Corrector at one node: q = u* + dt sum_d h_d^-1 [lift0_{i_d} F*_{d,-} -
// lift1_{i_d} F*_{d,+}] (face lifting of the weak form, GL mass matrix).
template <int DIM, int N, int M>
__device__ __forceinline__ void lift_node(const double* ustar, const double* fstar, int64_t cell,
                                          int node, const double* lift0, const double* lift1,
                                          const double* inv_h, double dt, double* u_out,
                                          double (&q)[M]) {
  constexpr int n = N + 1, NS = ipow(n, DIM), NF = ipow(n, DIM - 1);
  const int id[3] = {node % n, (node / n) % n, node / (n * n)};
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
    const double* F0 = fstar + (cell * 2 * DIM + 2 * d + 0) * M * NF + fnode;
    const double* F1 = fstar + (cell * 2 * DIM + 2 * d + 1) * M * NF + fnode;
    const double l0 = lift0[id[d]] * inv_h[d];
    const double l1 = lift1[id[d]] * inv_h[d];
#pragma unroll
    for (int v = 0; v < M; ++v) upd[v] = fma(l0, F0[v * NF], fma(-l1, F1[v * NF], upd[v]));
  }
#pragma unroll
  for (int v = 0; v < M; ++v) {
    const int64_t gi = (cell * M + v) * NS + node;
    q[v] = fma(dt, upd[v], ustar[gi]);
    u_out[gi] = q[v];
  }
}

// Contraction steps: a plain FMA in FP32/FP64; for double-float the
// compensated accumulation (no renormalisation per term) followed by one
// `settle` at the end of the sum.
__device__ __forceinline__ float fma_acc(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_acc(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float settle(float a) { return a; }
__device__ __forceinline__ double settle(double a) { return a; }

// Dynamic shared memory: fluxes of one slice fb[CPB][DIM][M][NS] (Real),
// Q-bar qs[CPB][M][NS] (Real), and for the FP32 variant an FP64 reduction
// buffer red[CPB][M][NS].
template <int DIM, int N, class PDE, class Real>
struct PredictSmem {
  using S = PredictShape<DIM, N>;
  static constexpr int kReal = S::CPB * (DIM + 1) * PDE::M * S::NS;
  static constexpr int kRedOffset = (kReal * int(sizeof(Real)) + 7) / 8;  // in doubles
  static constexpr int kPow2 = S::NS <= 1 ? 1 : (S::NS <= 2 ? 2 : (S::NS <= 4 ? 4 : (S::NS <= 8 ? 8 :
      (S::NS <= 16 ? 16 : (S::NS <= 32 ? 32 : (S::NS <= 64 ? 64 : (S::NS <= 128 ? 128 :
      (S::NS <= 256 ? 256 : 512))))))));
  __host__ __device__ static constexpr size_t bytes() {
    return std::is_same<Real, double>::value
               ? size_t(kReal) * sizeof(Real)
               : size_t(kRedOffset) * 8 + size_t(S::CPB) * PDE::M * S::NS * 8;
  }
};

// Tensor-core modes of the derivative contractions (FP32 predictor only):
// one TF32 product, three TF32 products of hi/lo splits (A_hi B_hi +
// A_hi B_lo + A_lo B_hi), or three BF16 products of hi/lo splits.
enum TcMode { kTcNone = 0, kTcTF32 = 1, kTcTF32x3 = 2, kTcBF16x3 = 3 };

// Shared memory and TMEM of the tensor-core path (one cell per CTA, 3D):
// per direction d the derivative along d of all m n^2 lines of CB time slices
// at once is the product A_d[rows x K] B_d[N x K]^T with A_d the slices'
// fluxes f_d laid out line by line, row (slice, variable, line) (K = the
// coordinate along d, padded to 8 TF32 / 16 BF16 values), and B_d = D / h_d
// padded to 16 x K; rows are cut into M = 128 tiles.  CB, the slices per MMA
// chain: at n^3 <= 256 nodes two CTAs per SM hide the chain's latency better
// than batching (measured at N = 5: TF32 61 ms per all-cell launch with one
// slice per chain and two CTAs, 113 ms with all six slices and one CTA), so
// CB = 1 there, the read-back in the predictor's own slice buffer; at larger
// n one CTA per SM is all the registers allow and CB is the largest count
// whose tiles fit 10 per direction (TMEM: 3 x 10 x 16 of 512 columns) and 128
// KB of operands and whose read-back buffer G[CB][DIM][M][n^3] (FP32, aliased
// onto the operand tiles once the MMAs have read them) is no larger than the
// tiles (N = 7: TF32 205 ms with CB = 4, 255 ms with CB = 1).
template <int DIM, int N, class PDE, int TC>
struct TcLayout {
  static constexpr int n = N + 1;
  static constexpr int NS = ipow(n, DIM);
  static constexpr int ROWS1 = PDE::M * n * n;       // lines per direction and slice
  static constexpr int NSPLIT = TC == kTcTF32 ? 1 : 2;
  static constexpr int EB = TC == kTcBF16x3 ? 2 : 4; // operand element bytes
  static constexpr int KPAD = 32 / EB;               // K per row (8 TF32, 16 BF16)
  static constexpr int KIND = TC == kTcBF16x3 ? 1 : 0;
  static constexpr int tiles(int cb) { return (cb * ROWS1 + 127) / 128; }
  static constexpr int a_bytes(int cb) { return NSPLIT * DIM * tiles(cb) * tc::kTileBytes; }
  static constexpr int g_bytes(int cb) { return cb * DIM * PDE::M * NS * 4; }
  static constexpr int THREADS = (ipow(n, DIM) + 31) / 32 * 32;
  static constexpr int MIN_BLOCKS = THREADS <= 256 ? 2 : 1;
  static constexpr bool fits(int cb) {
    return tiles(cb) <= 10 && a_bytes(cb) <= 128 * 1024 && g_bytes(cb) <= a_bytes(cb);
  }
  static constexpr int pick(int cb) { return cb <= 1 || fits(cb) ? cb : pick(cb - 1); }
  static constexpr int CB = MIN_BLOCKS == 2 ? 1 : pick(n);
  static constexpr int T = tiles(CB);                // M = 128 tiles per direction
  static constexpr int A_BYTES = a_bytes(CB);
  static constexpr int B_BYTES = NSPLIT * DIM * 512;  // 16 rows x 32 bytes each
  static constexpr int COLS_USED = DIM * T * 16;
  static constexpr int COLS = COLS_USED <= 32 ? 32 : COLS_USED <= 64 ? 64 : COLS_USED <= 128 ? 128
                              : COLS_USED <= 256 ? 256 : 512;
  __host__ __device__ static constexpr size_t bytes() { return size_t(A_BYTES + B_BYTES + 128); }
};

// One pass of the predictor over the cells of one CTA (CPB of them, or fewer
// when the launch spreads a small cell set over more CTAs).  Thread
// t < CPB*NS works on cell t / NS, node t % NS; further threads of the CTA
// only join the barriers.  `cell` is the cell index (relative to the field pointers) of
// this thread's cell and `valid` whether it exists; `ihd` its 1/h_d.  Every
// thread of the CTA must call this with the same dt, B and iters.
template <int DIM, int N, class PDE, class Real, int TC = kTcNone, int SCHEME = 0>
__device__ __forceinline__ void predict_cells(const BasisTables& B, double dt, double gamma_d,
                                              int iters, uint32_t* status, const double* u_in,
                                              double* ustar, double* faceQ, double* faceF,
                                              int64_t cell, bool valid, const double (&ihd)[DIM],
                                              unsigned char* smem_raw) {
  using S = PredictShape<DIM, N>;
  constexpr int n = S::n, NS = S::NS, NF = S::NF, CPB = S::CPB, M = PDE::M;
  // sDh[c][d]: D scaled by 1/h_d of cell c; sMd = -dt Mt; sRs[k] = sum_l sMd[k][l]
  __shared__ Real sDh[CPB][DIM][n * n], sMd[n * n], sRs[n], sV[n * n], sw[n], sp0[n], sp1[n];
  __shared__ Real sCk[n];  // Cauchy-Kowalevski: sCk[k] = dt^k / (k + 1)!
  // fb[CPB][DIM][M][NS] fluxes of one slice (later F-bar); qs[CPB][M][NS] Q-bar
  Real* fb = reinterpret_cast<Real*>(smem_raw);
  Real* qs = fb + CPB * DIM * M * NS;

  const int tid = threadIdx.x;
  const bool active = tid < CPB * NS;
  __syncthreads();  // a previous pass of this CTA may still read the shared tables
  for (int t = tid; t < n * n; t += blockDim.x) {
    sMd[t] = Real(-dt * B.Mt[t / n][t % n]);
    sV[t] = Real(B.V[t / n][t % n]);
  }
  if (tid < n) {
    double r = 0.0;
    for (int l = 0; l < n; ++l) r += B.Mt[tid][l];
    sRs[tid] = Real(-dt * r);
    sw[tid] = Real(B.w[tid]);
    sp0[tid] = Real(B.phi0[tid]);
    sp1[tid] = Real(B.phi1[tid]);
  }
  if (SCHEME == 1 && tid == 0) {
    // one thread forms the Taylor weights (a division each) for the CTA
    Real c = Real(1);
    sCk[0] = c;
    for (int k = 1; k <= N; ++k) {
      c = c * Real(dt) / Real(k + 1);
      sCk[k] = c;
    }
  }

  const int cl = active ? tid / NS : 0;
  const int node = active ? tid - cl * NS : 0;
  valid = valid && active;

  int id[3] = {node % n, (node / n) % n, node / (n * n)};
  const int stride[3] = {1, n, n * n};
  if (active && node < n * n) {
#pragma unroll
    for (int d = 0; d < DIM; ++d) sDh[cl][d][node] = Real(B.D[node / n][node % n] * ihd[d]);
  }
  const Real gamma = Real(gamma_d);

  Real uu[M];
#pragma unroll
  for (int v = 0; v < M; ++v)
    uu[v] = valid ? Real(u_in[(cell * M + v) * NS + node]) : Real(v == 0 ? 1 : 0);
  if (!valid && PDE::kPositivity) uu[M - 1] = Real(2.5);

  Real* my_fb = fb + cl * DIM * M * NS;
  Real* my_qs = qs + cl * M * NS;

  // FP32: this thread's rows of D/h_d live in registers for every slice
  // (shared-memory bandwidth bounds that variant).  FP64: they stay in shared
  // memory (the FP64 pipe bounds that variant and registers are scarce).
  constexpr bool kDinRegs = std::is_same<Real, float>::value;
  constexpr bool kRollSlices = std::is_same<Real, df64>::value;
  constexpr int kDr = kDinRegs ? n : 1;
  // FP32, 3D, n = 6, 7: the y and z line contractions of a thread in plane z
  // start at element z (cyclically).  Warps that straddle two z-planes then
  // read different rows/planes in the two parts at each step, which removes
  // most shared-memory bank conflicts of those contractions (n^2 = 36, 49 do
  // not divide into 32-lane warps).
  constexpr bool kRot = kDinRegs && DIM == 3 && (n == 6 || n == 7);
  const int rz = kRot ? id[2] : 0;
  __syncthreads();
  Real Dr[DIM][kDr];
  if constexpr (kDinRegs) {
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int j = 0; j < kDr; ++j) {
        int jj = j;
        if (kRot && d > 0) jj = (j + rz) % n;
        Dr[d][j] = sDh[cl][d][id[d] * n + jj];
      }
  }

  // ---- tensor-core set-up: operand tiles, B = D/h_d splits, TMEM, mbarrier
  using L = TcLayout<DIM, N, PDE, TC>;
  static_assert(TC == kTcNone || (std::is_same<Real, float>::value && DIM == 3 && CPB == 1),
                "tensor-core predictor: FP32, 3D, one cell per CTA");
  __shared__ uint64_t tc_mbar;
  __shared__ uint32_t tc_tmem;
  uint8_t* tcA = nullptr;
  uint8_t* tcB = nullptr;
  uint32_t tc_phase = 0;
  const int warp = tid >> 5, lane = tid & 31;
  if constexpr (TC != kTcNone) {
    // operand region after the predictor's own buffers, 128-byte aligned
    uint8_t* base = smem_raw + PredictSmem<DIM, N, PDE, Real>::bytes();
    const uint32_t sa = tc::smem_addr(base);
    tcA = base + ((128u - (sa & 127u)) & 127u);
    tcB = tcA + L::A_BYTES;
    for (int i = tid; i < (L::A_BYTES + L::B_BYTES) / 4; i += blockDim.x)
      reinterpret_cast<uint32_t*>(tcA)[i] = 0u;
    __syncthreads();
    // B_d[i][k] = D[i][k] / h_d for i, k < n (hi/lo split in the split modes)
    for (int t = tid; t < DIM * n * n; t += blockDim.x) {
      const int d = t / (n * n), i = (t / n) % n, k = t % n;
      const double x = B.D[i][k] * ihd[d];
      const uint32_t o = tc::canon(i, k * L::EB);
      if constexpr (TC == kTcBF16x3) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(float(x));
        const __nv_bfloat16 lo = __float2bfloat16_rn(float(x - double(__bfloat162float(hi))));
        *reinterpret_cast<__nv_bfloat16*>(tcB + d * 512 + o) = hi;
        *reinterpret_cast<__nv_bfloat16*>(tcB + (DIM + d) * 512 + o) = lo;
      } else {
        const float hi = tc::to_tf32(float(x));
        *reinterpret_cast<float*>(tcB + d * 512 + o) = hi;  // nearest TF32 (the MMA would truncate)
        if (TC == kTcTF32x3) *reinterpret_cast<float*>(tcB + (DIM + d) * 512 + o) = float(x - double(hi));
      }
    }
    if (warp == 0) tc::alloc(&tc_tmem, L::COLS);
    if (tid == 0) tc::mbar_init(&tc_mbar, 1);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }

  // ---- tensor-core contractions, up to L::CB time slices per MMA chain ----
  // tc_put(j, x): the fluxes of slice x into rows (j, variable, line) of the
  // operand tiles of every direction (hi/lo splits in the split modes); when
  // the read-back aliases the tiles (CB > 1) the thread at line position 0
  // also clears the row's K padding, which the previous chain's read-back may
  // have overwritten.
  auto tc_put = [&](int j, const Real(&x)[M]) {
    if constexpr (TC != kTcNone) {
      Real f[DIM][M];
      PDE::fluxes(x, f, gamma);
      if (active) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          // line index of this node across direction d (lowest tangential first)
          const int tl = d == 0 ? id[1] + n * id[2] : (d == 1 ? id[0] + n * id[2] : id[0] + n * id[1]);
#pragma unroll
          for (int v = 0; v < M; ++v) {
            const int r = (j * M + v) * n * n + tl;
            const uint32_t t0 = (d * L::T + (r >> 7)) * tc::kTileBytes;
            const uint32_t o = t0 + tc::canon(r & 127, id[d] * L::EB);
            const float val = float(f[d][v]);
            if constexpr (TC == kTcBF16x3) {
              const __nv_bfloat16 hi = __float2bfloat16_rn(val);
              *reinterpret_cast<__nv_bfloat16*>(tcA + o) = hi;
              *reinterpret_cast<__nv_bfloat16*>(tcA + DIM * L::T * tc::kTileBytes + o) =
                  __float2bfloat16_rn(val - __bfloat162float(hi));
            } else if constexpr (TC == kTcTF32x3) {
              const float hi = tc::to_tf32(val);
              *reinterpret_cast<float*>(tcA + o) = hi;
              *reinterpret_cast<float*>(tcA + DIM * L::T * tc::kTileBytes + o) = val - hi;
            } else {
              *reinterpret_cast<float*>(tcA + o) = tc::to_tf32(val);
            }
            if (L::CB > 1 && id[d] == 0) {
#pragma unroll
              for (int k = n; k < L::KPAD; ++k) {
                const uint32_t oz = t0 + tc::canon(r & 127, k * L::EB);
#pragma unroll
                for (int h = 0; h < L::NSPLIT; ++h) {
                  uint8_t* z = tcA + h * DIM * L::T * tc::kTileBytes + oz;
                  if constexpr (L::EB == 2)
                    *reinterpret_cast<uint16_t*>(z) = 0;
                  else
                    *reinterpret_cast<uint32_t*>(z) = 0u;
                }
              }
            }
          }
        }
      }
    }
  };
  // tc_run(cnt): the MMAs of cnt slices (one thread issues them and commits to
  // the mbarrier; bounded wait), then the accumulators back into
  // G[j][d][v][node] (FP32): the predictor's slice buffer when CB = 1, else
  // the operand tiles, which the MMAs have finished reading.
  auto tc_run = [&](int cnt) {
    if constexpr (TC != kTcNone) {
      tc::fence_proxy_async();
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      const uint32_t taddr = tc_tmem;
      const int tiles = (cnt * L::ROWS1 + 127) >> 7;
      if (tid == 0) {
        constexpr uint32_t ID = tc::idesc(L::KIND == 0 ? 2u : 1u, 128, 16);
        const uint32_t a0 = tc::smem_addr(tcA), b0 = tc::smem_addr(tcB);
#pragma unroll
        for (int d = 0; d < DIM; ++d)
          for (int t = 0; t < tiles; ++t) {
            const uint32_t dst = taddr + uint32_t((d * L::T + t) * 16);
            const uint32_t ahi = a0 + (d * L::T + t) * tc::kTileBytes;
            const uint32_t bhi = b0 + d * 512;
            tc::mma<L::KIND>(dst, tc::sdesc(ahi), tc::sdesc(bhi), ID, false);
            if constexpr (L::NSPLIT == 2) {
              const uint32_t alo = ahi + DIM * L::T * tc::kTileBytes;
              const uint32_t blo = bhi + DIM * 512;
              tc::mma<L::KIND>(dst, tc::sdesc(ahi), tc::sdesc(blo), ID, true);
              tc::mma<L::KIND>(dst, tc::sdesc(alo), tc::sdesc(bhi), ID, true);
            }
          }
        tc::commit(&tc_mbar);
      }
      if (!tc::mbar_wait(&tc_mbar, tc_phase, 1 << 22)) atomicOr(status, kStatusTensorTimeout);
      tc_phase ^= 1u;
      tc::fence_after();
      // warp w reads TMEM lane quarter w % 4
      float* G = L::CB == 1 ? reinterpret_cast<float*>(my_fb) : reinterpret_cast<float*>(tcA);
      const int q = warp & 3;
      const int nwq = (int(blockDim.x >> 5) - q + 3) >> 2;
      for (int job = warp >> 2; job < DIM * tiles; job += nwq) {
        const int d = job / tiles, t = job % tiles;
        float vals[8];
        tc::ld8(taddr + uint32_t((d * L::T + t) * 16) + (uint32_t(q * 32) << 16), vals);
        const int r = t * 128 + q * 32 + lane;
        if (r < cnt * L::ROWS1) {
          const int j = r / L::ROWS1, rr = r - j * L::ROWS1;
          const int v = rr / (n * n), tl = rr % (n * n);
#pragma unroll
          for (int i = 0; i < n; ++i) {
            const int nd = d == 0 ? i + n * tl
                                  : (d == 1 ? (tl % n) + n * i + n * n * (tl / n) : tl + n * n * i);
            G[((j * DIM + d) * M + v) * NS + nd] = vals[i];
          }
        }
      }
      tc::fence_before();
      __syncthreads();
    }
  };
  // tc_get(j, g): g = sum_d (D/h_d)^(d) f_d of slice j of the last chain at
  // this node.  The caller synchronises before the next tc_put.
  auto tc_get = [&](int j, Real(&g)[M]) {
    if constexpr (TC != kTcNone) {
      const float* G = L::CB == 1 ? reinterpret_cast<const float*>(my_fb)
                                  : reinterpret_cast<const float*>(tcA);
#pragma unroll
      for (int v = 0; v < M; ++v) {
        g[v] = Real(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) g[v] += active ? G[((j * DIM + d) * M + v) * NS + node] : Real(0);
      }
    }
  };

  // g = sum_d (D/h_d)^(d) f_d(x) at this node, for the slice held in x
  // (CUDA-core contraction over the slice's fluxes staged in shared memory).
  auto divergence = [&](const Real(&x)[M], Real(&g)[M]) {
    Real f[DIM][M];
    PDE::fluxes(x, f, gamma);
    if (active) {
#pragma unroll
      for (int d = 0; d < DIM; ++d)
#pragma unroll
        for (int v = 0; v < M; ++v)
          if (PDE::flux_nonzero(d, v)) my_fb[(d * M + v) * NS + node] = f[d][v];
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < M; ++v) g[v] = Real(0);
    if constexpr (kRollSlices) {
      // one copy of the line contraction, the direction chosen at run time
#pragma unroll 1
      for (int d = 0; d < DIM; ++d) {
        const int sd = d == 0 ? 1 : (d == 1 ? n : n * n);
        const int idd = d == 0 ? id[0] : (d == 1 ? id[1] : id[2]);
        const Real* line0 = my_fb + d * M * NS + node - idd * sd;
        const Real* drow = &sDh[cl][d][idd * n];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          if (!PDE::flux_nonzero(d, v)) continue;
          const Real* line = line0 + v * NS;
#pragma unroll
          for (int j = 0; j < n; ++j) g[v] = fma_acc(drow[j], line[j * sd], g[v]);
        }
      }
#pragma unroll
      for (int v = 0; v < M; ++v) g[v] = settle(g[v]);
    } else {
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const int base = node - id[d] * stride[d];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          if (!PDE::flux_nonzero(d, v)) continue;
          const Real* line = my_fb + (d * M + v) * NS + base;
          if constexpr (kDinRegs && n % 2 == 0) {
            // FP32 x-lines are contiguous and 8-byte aligned (they start at a
            // multiple of n): two elements per shared-memory load
            if (d == 0) {
              const float2* l2 = reinterpret_cast<const float2*>(line);
#pragma unroll
              for (int j2 = 0; j2 < n / 2; ++j2) {
                const float2 p = l2[j2];
                g[v] = fma(Dr[0][2 * j2], p.x, g[v]);
                g[v] = fma(Dr[0][2 * j2 + 1], p.y, g[v]);
              }
              continue;
            }
          }
#pragma unroll
          for (int j = 0; j < n; ++j) {
            Real dj;
            if constexpr (kDinRegs)
              dj = Dr[d][j < kDr ? j : 0];
            else
              dj = sDh[cl][d][id[d] * n + j];
            int jj = j;
            if (kRot && d > 0) {
              jj = j + rz;
              jj = jj >= n ? jj - n : jj;
            }
            g[v] = fma(dj, line[jj * stride[d]], g[v]);
          }
        }
      }
    }
    __syncthreads();
  };

  Real qb[M], Fb[DIM][M];
  if constexpr (SCHEME == 1) {
    // Cauchy-Kowalevski (linear PDEs, Sec. 2.4): d_0 = u, d_{k+1} = -sum_d
    // (D/h_d)^(d) f_d(d_k); the time average of the Taylor polynomial is
    // Q-bar = sum_k dt^k / (k+1)! d_k and F-bar_d = f_d(Q-bar).
    Real dk[M];
#pragma unroll
    for (int v = 0; v < M; ++v) {
      dk[v] = uu[v];
      qb[v] = uu[v];
    }
#pragma unroll
    for (int k = 1; k <= N; ++k) {
      Real g[M];
      divergence(dk, g);
      const Real c = sCk[k];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        dk[v] = -g[v];
        qb[v] = fma(c, dk[v], qb[v]);
      }
    }
    PDE::fluxes(qb, Fb, gamma);
  } else {
    // First Picard iteration: the initial guess u is constant in time, so one
    // slice gives every time node: q_k = u - dt (sum_l Mt[k][l]) g(u).
    Real q[n][M];
    {
      Real g[M];
      if constexpr (TC != kTcNone) {
        tc_put(0, uu);
        tc_run(1);
        tc_get(0, g);
        __syncthreads();
      } else {
        divergence(uu, g);
      }
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int v = 0; v < M; ++v) q[k][v] = fma(sRs[k], g[v], uu[v]);
    }
    if constexpr (TC != kTcNone) {
      // later iterations: the contractions of L::CB slices per MMA chain
      // (their fluxes all come from the previous iterate)
      for (int r = 1; r < iters; ++r) {
        Real acc[n][M];
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int v = 0; v < M; ++v) acc[k][v] = uu[v];
#pragma unroll
        for (int l0 = 0; l0 < n; l0 += L::CB) {
#pragma unroll
          for (int j = 0; j < L::CB; ++j)
            if (l0 + j < n) tc_put(j, q[l0 + j]);
          tc_run(l0 + L::CB <= n ? L::CB : n - l0);
#pragma unroll
          for (int j = 0; j < L::CB; ++j) {
            if (l0 + j >= n) continue;
            Real g[M];
            tc_get(j, g);
#pragma unroll
            for (int k = 0; k < n; ++k) {
              const Real c = sMd[k * n + l0 + j];
#pragma unroll
              for (int v = 0; v < M; ++v) acc[k][v] = fma(c, g[v], acc[k][v]);
            }
          }
          __syncthreads();  // G is read: the next chain may overwrite the tiles
        }
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int v = 0; v < M; ++v) q[k][v] = acc[k][v];
      }
    }
    for (int r = 1; r < iters && TC == kTcNone; ++r) {
      Real acc[n][M];
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int v = 0; v < M; ++v) acc[k][v] = uu[v];
      // one time slice of the Picard update: acc_k += -dt Mt[k][l] g(q_l)
      auto slice = [&](int l) {
        Real g[M];
        divergence(q[l], g);
#pragma unroll
        for (int k = 0; k < n; ++k) {
          const Real c = sMd[k * n + l];
#pragma unroll
          for (int v = 0; v < M; ++v) acc[k][v] = fma_acc(c, g[v], acc[k][v]);
        }
      };
      if constexpr (kRollSlices) {
        // double-float code is long: keep one copy of the slice body so the
        // kernel fits the instruction cache (q_l is then read from L1)
#pragma unroll 1
        for (int l = 0; l < n; ++l) slice(l);
      } else {
#pragma unroll
        for (int l = 0; l < n; ++l) slice(l);
      }
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int v = 0; v < M; ++v) q[k][v] = settle(acc[k][v]);
    }
    // Time averages of the final iterate and of its fluxes.
#pragma unroll
    for (int v = 0; v < M; ++v) qb[v] = Real(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int v = 0; v < M; ++v) Fb[d][v] = Real(0);
    auto average = [&](int k) {
      Real f[DIM][M];
      PDE::fluxes(q[k], f, gamma);
      const Real wk = sw[k];
#pragma unroll
      for (int v = 0; v < M; ++v) qb[v] = fma_acc(wk, q[k][v], qb[v]);
#pragma unroll
      for (int d = 0; d < DIM; ++d)
#pragma unroll
        for (int v = 0; v < M; ++v) Fb[d][v] = fma_acc(wk, f[d][v], Fb[d][v]);
    };
    if constexpr (kRollSlices) {
#pragma unroll 1
      for (int k = 0; k < n; ++k) average(k);
    } else {
#pragma unroll
      for (int k = 0; k < n; ++k) average(k);
    }
#pragma unroll
    for (int v = 0; v < M; ++v) {
      qb[v] = settle(qb[v]);
#pragma unroll
      for (int d = 0; d < DIM; ++d) Fb[d][v] = settle(Fb[d][v]);
    }
  }
  bool finite = true;
#pragma unroll
  for (int v = 0; v < M; ++v) {
    finite = finite && isfinite(qb[v]);
    if (active) my_qs[v * NS + node] = qb[v];
  }
#pragma unroll
  for (int d = 0; d < DIM; ++d)
#pragma unroll
    for (int v = 0; v < M; ++v) {
      if (!PDE::flux_nonzero(d, v)) continue;
      finite = finite && isfinite(Fb[d][v]);
      if (active) my_fb[(d * M + v) * NS + node] = Fb[d][v];
    }
  if (valid && !finite) atomicOr(status, kStatusNonFinitePredictor);
  __syncthreads();

  // Corrector volume term, contraction in Real, added to u in FP64.
  double vol[M];
#pragma unroll
  for (int v = 0; v < M; ++v) {
    vol[v] = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      if (!PDE::flux_nonzero(d, v)) continue;
      const Real* Vrow = sV + id[d] * n;
      const Real* line = my_fb + (d * M + v) * NS + node - id[d] * stride[d];
      Real s = Real(0);
#pragma unroll
      for (int j = 0; j < n; ++j) s = fma(Vrow[j], line[j * stride[d]], s);
      vol[v] = fma(ihd[d], double(s), vol[v]);
    }
  }
  if constexpr (!std::is_same<Real, double>::value) {
    // The exact volume term has zero quadrature-weighted sum over the cell
    // (sum_i w_i V_ij = w_j sum_i D_ji = 0); with V and F-bar rounded to Real it
    // does not.  Remove that weighted mean in FP64 (deterministic tree sum) so
    // that the step conserves to FP64 rounding; the change is within the
    // Real rounding error of the term itself.
    double* red = reinterpret_cast<double*>(smem_raw) + PredictSmem<DIM, N, PDE, Real>::kRedOffset;
    double* my_red = red + cl * M * NS;
    double W = 1.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) W *= B.w[id[d]];
    if (active) {
#pragma unroll
      for (int v = 0; v < M; ++v) my_red[v * NS + node] = valid ? W * vol[v] : 0.0;
    }
    for (int st = PredictSmem<DIM, N, PDE, Real>::kPow2 / 2; st > 0; st >>= 1) {
      __syncthreads();
      if (active && node < st && node + st < NS) {
#pragma unroll
        for (int v = 0; v < M; ++v) my_red[v * NS + node] += my_red[v * NS + node + st];
      }
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < M; ++v) vol[v] -= my_red[v * NS];
  }
  if constexpr (TC != kTcNone) {
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::dealloc(tc_tmem, L::COLS);
  }
  if (!valid) return;
#pragma unroll
  for (int v = 0; v < M; ++v) {
    const int64_t gi = (cell * M + v) * NS + node;
    ustar[gi] = fma(dt, vol[v], u_in[gi]);
  }

  // id|dc: extrapolate Q-bar and the normal flux F-bar_d to the 2d faces.
  // One face node per thread (2d n^(d-1) of them per cell, NS threads: all
  // lanes busy, one pass at 3D N=5), each reading its line from shared memory;
  // consecutive threads write consecutive face nodes.
  for (int t = node; t < 2 * DIM * NF; t += NS) {
    const int slot = t / NF, fnode = t - slot * NF;
    const int d = slot >> 1, side = slot & 1;
    const int ta = fnode % n, tb = fnode / n;  // tangential coordinates, lowest first
    const int base = DIM == 2 ? (d == 0 ? n * ta : ta)
                              : (d == 0 ? n * (ta + n * tb) : (d == 1 ? ta + n * n * tb : ta + n * tb));
    const int sd = d == 0 ? 1 : (d == 1 ? n : n * n);
    const Real* phi = side == 0 ? sp0 : sp1;
    const int64_t fo = ((cell * 2 * DIM + slot) * M) * NF + fnode;
#pragma unroll
    for (int v = 0; v < M; ++v) {
      const Real* lq = my_qs + v * NS + base;
      const Real* lf = my_fb + (d * M + v) * NS + base;
      const bool nz = PDE::flux_nonzero(d, v);
      Real sq = Real(0), sf = Real(0);
#pragma unroll
      for (int j = 0; j < n; ++j) {
        sq = fma(phi[j], lq[j * sd], sq);
        if (nz) sf = fma(phi[j], lf[j * sd], sf);
      }
      faceQ[fo + v * NF] = double(sq);
      faceF[fo + v * NF] = double(sf);
    }
  }
}

// Resident CTAs per SM the register allocation must allow: the double-float
// variant's long dependent chains need two CTAs to keep the FP32 pipes busy.
// The FP64 variant at 216 nodes (3D N=5) also runs two CTAs per SM, so one
// CTA's barrier waits are covered by the other's FP64 work: 128 registers
// with a few spills, measured 1 % faster per step than one CTA at 174.
template <class Real, int NS>
struct PredictMinBlocks {
  static constexpr bool kFP64 = std::is_same<Real, double>::value;
  static constexpr int value = (kFP64 ? (NS > 128 && NS <= 216) : NS <= 216) ? 2 : 1;
};

template <int DIM, int N, class PDE, class Real, int SCHEME = 0>
__global__ void __launch_bounds__(PredictShape<DIM, N>::THREADS,
                                  PredictMinBlocks<Real, PredictShape<DIM, N>::NS>::value)
    predict_kernel(const PredictArgs a) {
  using S = PredictShape<DIM, N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cl = threadIdx.x / S::NS;
  const int64_t slot = int64_t(blockIdx.x) * (blockDim.x / S::NS) + cl;  // blockDim: cpb whole cells
  const bool valid = slot < a.count;
  const int64_t cell = valid ? int64_t(a.cells[slot]) : 0;
  double ihd[DIM];
  const int lv = valid ? int(a.level[cell]) : 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) ihd[d] = a.inv_h[lv][d];
  if (a.corr_fstar && valid) {  // shifted task graph: the previous step's corrector first
    double q[PDE::M];
    lift_node<DIM, N, PDE::M>(a.ustar, a.corr_fstar, cell, int(threadIdx.x) - cl * S::NS, a.B.lift0,
                              a.B.lift1, ihd, *a.dt, a.corr_u, q);
  }
  predict_cells<DIM, N, PDE, Real, kTcNone, SCHEME>(a.B, *a.dt, a.gamma, a.iters, a.status, a.u,
                                                    a.ustar, a.faceQ, a.faceF, cell, valid, ihd,
                                                    smem_raw);
}

// Tensor-core predictor: one CTA (whole warps) per cell.
template <int N, class PDE, int TC>
__global__ void __launch_bounds__(TcLayout<3, N, PDE, TC>::THREADS, TcLayout<3, N, PDE, TC>::MIN_BLOCKS)
    predict_tc_kernel(const PredictArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t slot = blockIdx.x;
  const bool valid = slot < a.count;
  const int64_t cell = valid ? int64_t(a.cells[slot]) : 0;
  double ihd[3];
  const int lv = valid ? int(a.level[cell]) : 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) ihd[d] = a.inv_h[lv][d];
  if (a.corr_fstar && valid && int(threadIdx.x) < ipow(N + 1, 3)) {  // shifted task graph
    double q[PDE::M];
    lift_node<3, N, PDE::M>(a.ustar, a.corr_fstar, cell, int(threadIdx.x), a.B.lift0, a.B.lift1, ihd,
                            *a.dt, a.corr_u, q);
  }
  predict_cells<3, N, PDE, float, TC>(a.B, *a.dt, a.gamma, a.iters, a.status, a.u, a.ustar,
                                      a.faceQ, a.faceF, cell, valid, ihd, smem_raw);
}

template <int N, class PDE, int TC>
cudaError_t launch_predict_tc_t(const PredictArgs& a, cudaStream_t s) {
  using L = TcLayout<3, N, PDE, TC>;
  if (a.count == 0) return cudaSuccess;
  const size_t smem = PredictSmem<3, N, PDE, float>::bytes() + L::bytes();
  static std::atomic<uint64_t> configured{0};
  cudaError_t e = smem_opt_in(configured, predict_tc_kernel<N, PDE, TC>, smem);
  if (e != cudaSuccess) return e;
  predict_tc_kernel<N, PDE, TC><<<dim3(unsigned(a.count)), dim3(L::THREADS), smem, s>>>(a);
  return cudaGetLastError();
}

template <int DIM, int N, class PDE, class Real, int SCHEME = 0>
cudaError_t launch_predict_t(const PredictArgs& a, cudaStream_t s) {
  using S = PredictShape<DIM, N>;
  if (a.count == 0) return cudaSuccess;
  const size_t smem = PredictSmem<DIM, N, PDE, Real>::bytes();
  static std::atomic<uint64_t> configured{0};
  cudaError_t e = smem_opt_in(configured, predict_kernel<DIM, N, PDE, Real, SCHEME>, smem);
  if (e != cudaSuccess) return e;
  // cells per CTA: CPB, halved while the launch would have fewer than
  // a.min_ctas CTAs (every cell's work is independent of its CTA slot)
  int cpb = S::CPB;
  while (a.min_ctas > 0 && cpb > 1 && (a.count + cpb - 1) / cpb < a.min_ctas) cpb = (cpb + 1) / 2;
  const int64_t blocks = (a.count + cpb - 1) / cpb;
  predict_kernel<DIM, N, PDE, Real, SCHEME><<<dim3(unsigned(blocks)), dim3(unsigned(cpb * S::NS)), smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ader
