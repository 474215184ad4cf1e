// Discrete adjoint of one ADER-DG step for linear acoustics on adaptive
// meshes.
//
// For a linear PDE the step u -> u(T+dt) of Eq. (4) is a linear map A
// (Picard with a fixed iteration count, Rusanov with the exact speed s = c = 1,
// linear fluxes f_d = A_d q with symmetric A_d).  These kernels apply A^T to an
// adjoint state lambda by transposing each task in reverse order:
//   corrector   u+ = u* + Lift(F*)          ->  u*_bar = lambda, F*_bar = Lift^T lambda
//   Riemann     F* = (F_L + F_R)/2 - s (Q_R - Q_L)/2 on every conforming face
//                                          ->  (Q-bar, F-bar)_bar on both face slots
//   transition  virtual face = P_s (coarse face), Rusanov on each child face,
//               coarse F* = sum_s R_s F*_s (Sec. 2.3)
//                                          ->  R_s^T into each child's F*_bar,
//               Rusanov transposed, P_s^T summed into the coarse slot
//   predictor   u* = u + dt V F-bar, faces = E (Q-bar, F-bar), Q-bar/F-bar from
//               the Picard iterate          ->  lambda_out = u*_bar + (Picard,
//               time average, extrapolation and volume term transposed)
// The Picard iterations are unrolled in reverse with the same count as the
// forward kernel, so A^T is exact to rounding.
#pragma once
#include "faces.cuh"
#include "predict.cuh"

namespace ader {

// F*_bar[c][d][side][v][fn] = +-dt/h_d sum_{i_d} lift_side[i_d] lambda(node(i_d, fn)).
template <int DIM, int N, int M>
__global__ void adjoint_lift_kernel(const AdjointArgs a) {
  constexpr int n = N + 1, NS = ipow(n, DIM), NF = ipow(n, DIM - 1);
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t per_cell = 2 * DIM * NF;
  if (t >= a.ncells * per_cell) return;
  const int64_t c = t / per_cell;
  const int r = int(t - c * per_cell);
  const int slot = r / NF, fn = r % NF;
  const int d = slot / 2, side = slot % 2;
  const double dt = *a.dt;
  const double ih = a.inv_h[a.level[c]][d];
  // face node fn -> tangential indices -> base node and stride along d
  int ta, tb;  // tangential coordinates (lowest tangential direction first)
  ta = fn % n;
  tb = fn / n;
  int id[3] = {0, 0, 0};
  int k = 0;
  for (int e = 0; e < DIM; ++e) {
    if (e == d) continue;
    id[e] = (k == 0) ? ta : tb;
    ++k;
  }
  const int stride = d == 0 ? 1 : (d == 1 ? n : n * n);
  const int base = id[0] + n * id[1] + n * n * id[2];
  const double sign = side == 0 ? 1.0 : -1.0;
#pragma unroll
  for (int v = 0; v < M; ++v) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const double l = side == 0 ? a.B.lift0[i] : a.B.lift1[i];
      s = fma(l, a.lam_in[(c * M + v) * NS + base + i * stride], s);
    }
    a.fstar_bar[((c * 2 * DIM + slot) * M + v) * NF + fn] = sign * dt * ih * s;
  }
}

// Rusanov with s = 1 transposed on conforming faces; every face slot of
// every cell belongs to exactly one conforming face and is written once.
template <int DIM, int N, int M>
__global__ void adjoint_riemann_kernel(const AdjointArgs a) {
  constexpr int n = N + 1, NF = ipow(n, DIM - 1);
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= a.nconf * NF) return;
  const int64_t f = t / NF;
  const int fn = int(t - f * NF);
  const ConfFace cf = a.conf[f];
  const int d = cf.dir;
  const int64_t oL = (int64_t(cf.left) * 2 * DIM + 2 * d + 1) * M * NF + fn;
  const int64_t oR = (int64_t(cf.right) * 2 * DIM + 2 * d + 0) * M * NF + fn;
  const double s = 1.0;  // Rusanov speed of acoustics with c = 1
#pragma unroll
  for (int v = 0; v < M; ++v) {
    const double Fb = a.fstar_bar[oL + v * NF] + a.fstar_bar[oR + v * NF];
    a.faceF_bar[oL + v * NF] = 0.5 * Fb;
    a.faceQ_bar[oL + v * NF] = 0.5 * s * Fb;
    a.faceF_bar[oR + v * NF] = 0.5 * Fb;
    a.faceQ_bar[oR + v * NF] = -0.5 * s * Fb;
  }
}

// Transitions transposed, one CTA per parent face: the restriction (the
// coarse slot's F*_bar reaches each child face through R_s^T), Rusanov with
// s = 1 on the child faces, and the prolongation of the coarse face data
// (P_s^T summed over the children).  The fine cells' slots facing the coarse
// cell and the coarse cell's slot belong to this family alone, so each is
// written once, as the conforming faces' slots are.
template <int DIM, int N, int M>
__global__ void adjoint_transition_kernel(const AdjointArgs a) {
  constexpr int n = N + 1, NF = ipow(n, DIM - 1), S = DIM == 3 ? 9 : 3, nb = DIM == 3 ? n : 1;
  __shared__ double gbar[S][M][NF];  // total adjoint of F* on each child face
  const int64_t p = blockIdx.x;
  if (p >= a.nparents) return;
  const ParentFace pf = a.parents[p];
  const int d = pf.dir, cs = pf.coarse_side;
  const int64_t oC = (int64_t(pf.coarse) * 2 * DIM + 2 * d + cs) * M * NF;
  const double* GC = a.fstar_bar + oC;
  const double s = 1.0;  // Rusanov speed of acoustics with c = 1
  // Q-bar_bar factors: the fine side is right of the face when the coarse
  // cell is on the left (cs = 1), left of it otherwise
  const double qf = cs == 1 ? -0.5 * s : 0.5 * s;
  for (int t = threadIdx.x; t < S * NF; t += blockDim.x) {
    const int sigma = t / NF, fn = t - sigma * NF;
    const int s0 = sigma % 3, s1 = sigma / 3;
    const int i = fn % n, j = fn / n;
    const int64_t fine = a.child_fine[p * S + sigma];
    const int64_t oF = (fine * 2 * DIM + 2 * d + (1 - cs)) * M * NF;
#pragma unroll
    for (int v = 0; v < M; ++v) {
      double g = a.fstar_bar[oF + v * NF + fn];
      for (int ib = 0; ib < nb; ++ib) {
        const double r1 = DIM == 3 ? a.B.R[s1][ib][j] : 1.0;
        for (int ia = 0; ia < n; ++ia) g = fma(a.B.R[s0][ia][i] * r1, GC[v * NF + ia + n * ib], g);
      }
      gbar[sigma][v][fn] = g;
      a.faceF_bar[oF + v * NF + fn] = 0.5 * g;
      a.faceQ_bar[oF + v * NF + fn] = qf * g;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NF; t += blockDim.x) {
    const int i = t % n, j = t / n;
#pragma unroll
    for (int v = 0; v < M; ++v) {
      double f = 0.0;
      for (int sigma = 0; sigma < S; ++sigma) {
        const int s0 = sigma % 3, s1 = sigma / 3;
        for (int ib = 0; ib < nb; ++ib) {
          const double p1 = DIM == 3 ? a.B.P[s1][ib][j] : 1.0;
          for (int ia = 0; ia < n; ++ia)
            f = fma(a.B.P[s0][ia][i] * p1, gbar[sigma][v][ia + n * ib], f);
        }
      }
      a.faceF_bar[oC + v * NF + t] = 0.5 * f;
      a.faceQ_bar[oC + v * NF + t] = -qf * f;
    }
  }
}

// Acoustics flux Jacobian A_d (symmetric): (A_d y)[0] = y[1+d], (A_d y)[1+d] = y[0].
template <int M>
__device__ __forceinline__ void apply_Ad(int d, const double (&y)[M], double (&out)[M]) {
#pragma unroll
  for (int v = 0; v < M; ++v) out[v] = 0.0;
  out[0] = y[1 + d];
  out[1 + d] = y[0];
}

// Transposed predictor: one CTA per CPB cells, thread per node.
template <int DIM, int N, int M>
__global__ void __launch_bounds__(PredictShape<DIM, N>::THREADS) adjoint_predict_kernel(const AdjointArgs a) {
  using S = PredictShape<DIM, N>;
  constexpr int n = S::n, NS = S::NS, NF = S::NF, CPB = S::CPB;
  __shared__ double sD[n * n], sMt[n * n], sV[n * n], sw[n], sp0[n], sp1[n], sRs[n];
  __shared__ double buf[CPB][M][NS];
  const int tid = threadIdx.x;
  const double dt = *a.dt;
  for (int t = tid; t < n * n; t += blockDim.x) {
    sD[t] = a.B.D[t / n][t % n];
    sMt[t] = a.B.Mt[t / n][t % n];
    sV[t] = a.B.V[t / n][t % n];
  }
  if (tid < n) {
    double r = 0.0;
    for (int l = 0; l < n; ++l) r += a.B.Mt[tid][l];
    sRs[tid] = -dt * r;
    sw[tid] = a.B.w[tid];
    sp0[tid] = a.B.phi0[tid];
    sp1[tid] = a.B.phi1[tid];
  }
  const int cl = tid / NS;
  const int node = tid - cl * NS;
  const int64_t cell = int64_t(blockIdx.x) * CPB + cl;
  const bool valid = cell < a.ncells;
  const int64_t c = valid ? cell : 0;
  const int id[3] = {node % n, (node / n) % n, node / (n * n)};
  const int stride[3] = {1, n, n * n};
  double ih[DIM];
  const int lv = int(a.level[c]);
#pragma unroll
  for (int d = 0; d < DIM; ++d) ih[d] = a.inv_h[lv][d];
  double* my = &buf[cl][0][0];
  __syncthreads();

  auto fnode_of = [&](int d) {
    if (DIM == 2) return d == 0 ? id[1] : id[0];
    return d == 0 ? id[1] + n * id[2] : (d == 1 ? id[0] + n * id[2] : id[0] + n * id[1]);
  };
  // x -> sum_d ih_d A_d^T D^(d)^T x, with x staged in my[][node]
  auto transpose_div = [&](const double (&x)[M], double (&out)[M]) {
#pragma unroll
    for (int v = 0; v < M; ++v) my[v * NS + node] = x[v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < M; ++v) out[v] = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      double t[M];
      const int base = node - id[d] * stride[d];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < n; ++j) s = fma(sD[j * n + id[d]], my[v * NS + base + j * stride[d]], s);
        t[v] = ih[d] * s;
      }
      double At[M];
      apply_Ad<M>(d, t, At);
#pragma unroll
      for (int v = 0; v < M; ++v) out[v] += At[v];
    }
    __syncthreads();
  };

  double lam[M];
#pragma unroll
  for (int v = 0; v < M; ++v) lam[v] = valid ? a.lam_in[(c * M + v) * NS + node] : 0.0;

  // F-bar_d adjoint: volume term (dt ih_d V^T lam) + face extrapolation (phi_side[i_d] faceF_bar)
  double G[M];
#pragma unroll
  for (int v = 0; v < M; ++v) G[v] = 0.0;
#pragma unroll
  for (int v = 0; v < M; ++v) my[v * NS + node] = lam[v];
  __syncthreads();
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int base = node - id[d] * stride[d];
    const int fn = fnode_of(d);
    double Fb[M];
#pragma unroll
    for (int v = 0; v < M; ++v) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < n; ++j) s = fma(sV[j * n + id[d]], my[v * NS + base + j * stride[d]], s);
      Fb[v] = dt * ih[d] * s;
      if (valid) {
        Fb[v] += sp0[id[d]] * a.faceF_bar[((c * 2 * DIM + 2 * d + 0) * M + v) * NF + fn];
        Fb[v] += sp1[id[d]] * a.faceF_bar[((c * 2 * DIM + 2 * d + 1) * M + v) * NF + fn];
        G[v] += sp0[id[d]] * a.faceQ_bar[((c * 2 * DIM + 2 * d + 0) * M + v) * NF + fn];
        G[v] += sp1[id[d]] * a.faceQ_bar[((c * 2 * DIM + 2 * d + 1) * M + v) * NF + fn];
      }
    }
    double At[M];
    apply_Ad<M>(d, Fb, At);
#pragma unroll
    for (int v = 0; v < M; ++v) G[v] += At[v];
  }
  __syncthreads();

  if (a.scheme == 1) {
    // Cauchy-Kowalevski: Q-bar = sum_k c_k L^k u, c_k = dt^k / (k+1)!, L = -sum_d
    // ih_d D^(d) A_d, so u_bar = u*_bar + sum_k c_k (L^T)^k G by Horner's scheme.
    double ck[N + 1];
    ck[0] = 1.0;
#pragma unroll
    for (int k = 1; k <= N; ++k) ck[k] = ck[k - 1] * dt / double(k + 1);
    double z[M];
#pragma unroll
    for (int v = 0; v < M; ++v) z[v] = ck[N] * G[v];
#pragma unroll
    for (int k = N - 1; k >= 0; --k) {
      double t[M];
      transpose_div(z, t);
#pragma unroll
      for (int v = 0; v < M; ++v) z[v] = fma(ck[k], G[v], -t[v]);
    }
    if (valid) {
#pragma unroll
      for (int v = 0; v < M; ++v) a.lam_out[(c * M + v) * NS + node] = lam[v] + z[v];
    }
    return;
  }

  // Time averages: q^(I)_bar_k = w_k G.
  double qb[n][M];
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int v = 0; v < M; ++v) qb[k][v] = sw[k] * G[v];

  double acc[M];
#pragma unroll
  for (int v = 0; v < M; ++v) acc[v] = lam[v];  // u* = u + ...  ->  lambda passes through

  // Picard iterations r = I-1 .. 1 in reverse: q^(r+1)_k = u - dt sum_l Mt[k][l] g(q^(r)_l).
  for (int r = a.iters - 1; r >= 1; --r) {
    double gb[n][M];
#pragma unroll
    for (int l = 0; l < n; ++l)
#pragma unroll
      for (int v = 0; v < M; ++v) gb[l][v] = 0.0;
#pragma unroll
    for (int k = 0; k < n; ++k) {
#pragma unroll
      for (int v = 0; v < M; ++v) acc[v] += qb[k][v];
#pragma unroll
      for (int l = 0; l < n; ++l) {
        const double cmk = -dt * sMt[k * n + l];
#pragma unroll
        for (int v = 0; v < M; ++v) gb[l][v] = fma(cmk, qb[k][v], gb[l][v]);
      }
    }
#pragma unroll
    for (int l = 0; l < n; ++l) transpose_div(gb[l], qb[l]);
  }
  // First iteration: q^(1)_k = u + sRs[k] g(u).
  {
    double s[M];
#pragma unroll
    for (int v = 0; v < M; ++v) s[v] = 0.0;
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int v = 0; v < M; ++v) {
        acc[v] += qb[k][v];
        s[v] = fma(sRs[k], qb[k][v], s[v]);
      }
    double tdiv[M];
    transpose_div(s, tdiv);
#pragma unroll
    for (int v = 0; v < M; ++v) acc[v] += tdiv[v];
  }
  if (valid) {
#pragma unroll
    for (int v = 0; v < M; ++v) a.lam_out[(c * M + v) * NS + node] = acc[v];
  }
}

template <int DIM, int N, int M>
cudaError_t launch_adjoint_t(const AdjointArgs& a, cudaStream_t s) {
  using S = PredictShape<DIM, N>;
  if (a.ncells == 0) return cudaSuccess;
  constexpr int NF = ipow(N + 1, DIM - 1);
  const int64_t t1 = a.ncells * 2 * DIM * NF;
  adjoint_lift_kernel<DIM, N, M><<<unsigned((t1 + 255) / 256), 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t t2 = a.nconf * NF;
  if (t2 > 0) adjoint_riemann_kernel<DIM, N, M><<<unsigned((t2 + 255) / 256), 256, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.nparents > 0) adjoint_transition_kernel<DIM, N, M><<<unsigned(a.nparents), 128, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adjoint_predict_kernel<DIM, N, M>
      <<<unsigned((a.ncells + S::CPB - 1) / S::CPB), S::THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ader
