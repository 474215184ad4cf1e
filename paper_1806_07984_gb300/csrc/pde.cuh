// Physical fluxes of Eq. (1) (sources vanish) for the device kernels.
//
// Euler<DIM>:     q = (rho, rho v_1..rho v_DIM, E), p = (gamma-1)(E - |rho v|^2 / (2 rho)),
//                 f_d = (rho v_d, rho v v_d + p e_d, v_d (E + p)),
//                 lambda_d = |v_d| + sqrt(gamma p / rho).
// Acoustics<DIM>: q = (p, v_1..v_DIM) with c = rho = 1, f_d = (v_d, p e_d),
//                 lambda_d = 1.
#pragma once
#include <cuda_runtime.h>

namespace ader {

// 1 / x without an IEEE division: the hardware's approximate reciprocal
// (PTX rcp.approx.ftz.f64) refined by two Newton-Raphson steps
// y <- y + y (1 - x y), each of which doubles the number of correct bits
// (Markstein, IBM J. Res. Dev. 34 (1990)).  Within a few units in the last
// place for normal x; the Euler states that reach it have rho normal and
// positive, and a zero, infinite or NaN rho gives a non-finite result that
// the kernels' checks report.  FP32 keeps its division.
__device__ __forceinline__ double recip(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ float recip(float x) { return 1.0f / x; }

template <class R>
__device__ __forceinline__ R recip_of(const R& x) { return R(1) / x; }
template <>
__device__ __forceinline__ double recip_of<double>(const double& x) { return recip(x); }

template <int DIM_>
struct Euler {
  static constexpr int DIM = DIM_;
  static constexpr int M = DIM + 2;
  static constexpr bool kPositivity = true;

  // Whether component v of f_d can be nonzero (Euler: every component).
  __host__ __device__ static constexpr bool flux_nonzero(int, int) { return true; }

  // All DIM fluxes at one node.
  template <class R>
  __device__ __forceinline__ static void fluxes(const R (&q)[M], R (&f)[DIM][M], R gamma) {
    const R rinv = recip_of(q[0]);
    R v[DIM];
    R ke = R(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      v[a] = q[1 + a] * rinv;
      ke = fma(q[1 + a], v[a], ke);
    }
    const R p = (gamma - R(1)) * fma(R(-0.5), ke, q[DIM + 1]);
    const R Ep = q[DIM + 1] + p;
    // momentum flux rho v_a v_d is symmetric in (a, d): one product per pair
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      f[d][0] = q[1 + d];
      f[d][1 + d] = fma(q[1 + d], v[d], p);
#pragma unroll
      for (int a = d + 1; a < DIM; ++a) {
        f[d][1 + a] = q[1 + a] * v[d];
        f[a][1 + d] = f[d][1 + a];
      }
      f[d][DIM + 1] = v[d] * Ep;
    }
  }

  // Flux in one direction d.
  template <class R>
  __device__ __forceinline__ static void flux(const R (&q)[M], int d, R (&f)[M], R gamma) {
    const R rinv = recip_of(q[0]);
    R ke = R(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) ke = fma(q[1 + a], q[1 + a] * rinv, ke);
    const R p = (gamma - R(1)) * fma(R(-0.5), ke, q[DIM + 1]);
    const R vd = q[1 + d] * rinv;
    f[0] = q[1 + d];
#pragma unroll
    for (int a = 0; a < DIM; ++a) f[1 + a] = q[1 + a] * vd;
    f[1 + d] += p;
    f[DIM + 1] = vd * (q[DIM + 1] + p);
  }

  // Largest wave speed in direction d; also reports whether the state is
  // physical (finite, rho > 0, p > 0).
  __device__ __forceinline__ static double max_speed(const double (&q)[M], int d, double gamma,
                                                     bool* ok) {
    const double rinv = recip(q[0]);
    double ke = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) ke = fma(q[1 + a], q[1 + a] * rinv, ke);
    const double p = (gamma - 1.0) * fma(-0.5, ke, q[DIM + 1]);
    *ok = (q[0] > 0.0) && (p > 0.0) && isfinite(p) && isfinite(rinv);
    return fabs(q[1 + d] * rinv) + sqrt(fmax(gamma * p * rinv, 0.0));
  }
};

template <int DIM_>
struct Acoustics {
  static constexpr int DIM = DIM_;
  static constexpr int M = DIM + 1;
  static constexpr bool kPositivity = false;

  // f_d has two nonzero components, p-row (v_d) and v_d-row (p); the kernels
  // skip the contractions of the others (adding their zeros changes nothing).
  __host__ __device__ static constexpr bool flux_nonzero(int d, int v) { return v == 0 || v == 1 + d; }

  template <class R>
  __device__ __forceinline__ static void fluxes(const R (&q)[M], R (&f)[DIM][M], R) {
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
#pragma unroll
      for (int a = 0; a < M; ++a) f[d][a] = R(0);
      f[d][0] = q[1 + d];
      f[d][1 + d] = q[0];
    }
  }

  template <class R>
  __device__ __forceinline__ static void flux(const R (&q)[M], int d, R (&f)[M], R) {
#pragma unroll
    for (int a = 0; a < M; ++a) f[a] = R(0);
    f[0] = q[1 + d];
    f[1 + d] = q[0];
  }

  __device__ __forceinline__ static double max_speed(const double (&q)[M], int, double, bool* ok) {
    bool fin = true;
#pragma unroll
    for (int a = 0; a < M; ++a) fin = fin && isfinite(q[a]);
    *ok = fin;
    return 1.0;
  }
};

}  // namespace ader
