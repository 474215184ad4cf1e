"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds no part of the ADER-DG method: it only evaluates initial
states at node coordinates that the caller supplies, and draws seeded random
numbers.  The paper's own workloads (LOH.1, the 2D explosion) are not used; the
states below have the shapes and orders of its Euler runs (p in {3, 5, 7},
Table 1) on synthetic smooth data:

* ``isentropic_vortex`` - 2D Euler: a vortex of strength eps on rho = 1,
  v = (1, 1), p = 1, length scale R = 0.1 on the periodic unit square
  (the classic [0, 10]^2 vortex mapped to the unit square), gamma = 1.4.
* ``density_bubble``    - 3D Euler: rho = 1 + 0.2 exp(-|x - c|^2 / sigma^2),
  sigma = 0.05, uniform p = 1 and velocity v0 = (1, 1, 1): an entropy wave that
  the exact Euler flow translates with v0.
* ``acoustic_pulses``   - 3D linear acoustics: p0 = sum of 8 Gaussians of width
  0.05 with seeded amplitudes in [0.5, 1] and centres in [0, 1]^3, v = 0.
* ``random_euler``      - seeded perturbations of a uniform Euler state with
  positive density and pressure (parity inputs).
* ``circular_explosion`` - 2D/3D Euler with shocks for the subcell limiter
  (the paper's Euler-with-shocks runs use a circular explosion; its data are
  not given): rho = 1, p = 1 inside a ball of radius 0.25 around the centre,
  rho = 0.125, p = 0.1 outside, at rest (the classic Sod states), the jump
  optionally smoothed by a tanh profile.

All states are conserved variables in the layout [var, ...] of the coordinate
arrays (Euler: rho, rho v_1..rho v_d, E; acoustics: p, v_1..v_d).
"""
import numpy as np

GAMMA = 1.4

# Courant factor C per order N in dt = C / max sum_d lambda_d / h_d:
# C = 0.9 nu_N, nu_N the von Neumann limit of the ADER-DG P_N step for linear
# advection (truncated to three decimals).  Values written from the oracle's
# stability analysis and re-checked by the test suite.
ADER_CFL = {1: 0.2997, 2: 0.153, 3: 0.0927, 4: 0.0621, 5: 0.045, 6: 0.0315,
            7: 0.0225, 8: 0.0207, 9: 0.0171}


def _periodic_delta(x, c, period=1.0):
    d = np.asarray(x, dtype=np.float64) - c
    return d - period * np.round(d / period)


def _conserved(rho, vel, p, gamma=GAMMA):
    mom = [rho * v for v in vel]
    E = p / (gamma - 1.0) + 0.5 * rho * sum(v * v for v in vel)
    return np.stack(np.broadcast_arrays(rho, *mom, E))


def isentropic_vortex(x, y, t=0.0, eps=5.0, center=(0.5, 0.5), R=0.1,
                      vel=(1.0, 1.0), gamma=GAMMA):
    """Conserved 2D Euler state of the translating isentropic vortex."""
    cx = center[0] + vel[0] * t
    cy = center[1] + vel[1] * t
    dx = _periodic_delta(x, cx) / R
    dy = _periodic_delta(y, cy) / R
    r2 = dx * dx + dy * dy
    amp = eps / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    vx = vel[0] - amp * dy
    vy = vel[1] + amp * dx
    T = 1.0 - (gamma - 1.0) * eps * eps / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return _conserved(rho, [vx, vy], p, gamma)


def density_bubble(coords, t=0.0, amp=0.2, sigma=0.05, center=(0.5, 0.5, 0.5),
                   vel=(1.0, 1.0, 1.0), gamma=GAMMA):
    """Conserved Euler state of the translating Gaussian density bubble
    (any dimension: ``coords`` is a list of coordinate arrays)."""
    dim = len(coords)
    r2 = 0.0
    for a in range(dim):
        d = _periodic_delta(coords[a], center[a] + vel[a] * t)
        r2 = r2 + d * d
    rho = 1.0 + amp * np.exp(-r2 / sigma ** 2)
    vel_arr = [np.full_like(rho, vel[a]) for a in range(dim)]
    return _conserved(rho, vel_arr, np.ones_like(rho), gamma)


EXPLOSION_RADIUS = 0.25


def circular_explosion(coords, center=(0.5, 0.5, 0.5), radius=EXPLOSION_RADIUS, width=0.0,
                       gamma=GAMMA):
    """Conserved Euler state of the circular (spherical in 3D) explosion; with
    width > 0 the jump is smoothed to 0.5 (1 + tanh((radius - r) / width))."""
    dim = len(coords)
    r2 = 0.0
    for a in range(dim):
        d = _periodic_delta(coords[a], center[a])
        r2 = r2 + d * d
    if width > 0.0:
        inside = 0.5 * (1.0 + np.tanh((radius - np.sqrt(r2)) / width))
    else:
        inside = (r2 < radius * radius).astype(np.float64)
    rho = 0.125 + 0.875 * inside
    p = 0.1 + 0.9 * inside
    vel = [np.zeros_like(rho) for _ in range(dim)]
    return _conserved(rho, vel, p, gamma)


def sphere_center(t, center=(0.5, 0.5, 0.5), vel=(1.0, 1.0, 1.0)):
    """Centre of the refinement ball at time t: moves with the flow, mod 1."""
    return tuple((c + v * t) % 1.0 for c, v in zip(center, vel))


def acoustic_pulses(coords, seed=1, count=8, width=0.05):
    """Linear acoustics initial state: p = sum of seeded Gaussians, v = 0."""
    rng = np.random.default_rng(seed)
    dim = len(coords)
    amps = rng.uniform(0.5, 1.0, size=count)
    centres = rng.uniform(0.0, 1.0, size=(count, dim))
    p = np.zeros_like(np.asarray(coords[0], dtype=np.float64))
    for k in range(count):
        r2 = 0.0
        for a in range(dim):
            d = _periodic_delta(coords[a], centres[k, a])
            r2 = r2 + d * d
        p = p + amps[k] * np.exp(-r2 / width ** 2)
    return np.stack([p] + [np.zeros_like(p)] * dim)


def random_euler(rng, dim, shape, amp=0.1, gamma=GAMMA):
    """Seeded Euler state near rho = 1, v = 0.5, p = 1 (positive rho and p)."""
    rho = 1.0 + amp * rng.uniform(-1.0, 1.0, size=shape)
    vel = [0.5 + amp * rng.uniform(-1.0, 1.0, size=shape) for _ in range(dim)]
    p = 1.0 + amp * rng.uniform(-1.0, 1.0, size=shape)
    return _conserved(rho, vel, p, gamma)


def random_acoustics(rng, dim, shape, amp=1.0):
    return amp * rng.uniform(-1.0, 1.0, size=(dim + 1,) + tuple(shape))


def batch_instances(count=512, seed=0):
    """Seeded 2D instances: side in 9..81 cells, order N in 3..7, vortex
    centre in [0, 1]^2 and strength in [1, 5] on the uniform background."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        out.append(dict(side=int(rng.integers(9, 82)), order=int(rng.integers(3, 8)),
                        center=tuple(rng.uniform(0.0, 1.0, size=2)),
                        eps=float(rng.uniform(1.0, 5.0))))
    return out


def acoustic_receivers(count=64, seed=2, dim=3):
    """Seeded receiver points in [0, 1)^dim."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(count, dim))
