"""Balance laws dQ/dt + div F(Q) = 0 of Eq. (1) (oracle; test infrastructure).

Sources S and point sources delta of Eq. (1) vanish in every workload here.
Arrays carry the m variables on axis 0: ``q[var, ...]``.

* ``Euler``     - compressible Euler (the paper's Euler application, Sec. 6):
                  q = (rho, rho v_1..rho v_d, E), p = (gamma-1)(E - |rho v|^2/(2 rho)),
                  f_d = (rho v_d, rho v v_d + p e_d, v_d (E + p)),
                  lambda_d = |v_d| + sqrt(gamma p / rho).
* ``Acoustics`` - linear acoustics with c = rho = 1 (a linear PDE, for which
                  Sec. 2.4 names Cauchy-Kowalevski): q = (p, v_1..v_d),
                  f_d = (v_d, p e_d), lambda_d = 1.
"""
import numpy as np


class Euler:
    name = "euler"
    linear = False

    def __init__(self, dim, gamma=1.4):
        self.dim = dim
        self.gamma = gamma
        self.nvar = dim + 2

    def pressure(self, q):
        rho = q[0]
        kin = sum(q[1 + a] * q[1 + a] for a in range(self.dim)) / rho
        return (self.gamma - 1.0) * (q[self.dim + 1] - 0.5 * kin)

    def flux(self, q, d):
        rho = q[0]
        vd = q[1 + d] / rho
        p = self.pressure(q)
        f = np.empty_like(q)
        f[0] = q[1 + d]
        for a in range(self.dim):
            f[1 + a] = q[1 + a] * vd
        f[1 + d] = f[1 + d] + p
        f[self.dim + 1] = vd * (q[self.dim + 1] + p)
        return f

    def max_speed(self, q, d):
        rho = q[0]
        p = self.pressure(q)
        return np.abs(q[1 + d] / rho) + np.sqrt(self.gamma * p / rho)

    def primitive_to_conserved(self, rho, vel, p):
        vel = [np.asarray(v, dtype=np.float64) for v in vel]
        q = [np.asarray(rho, dtype=np.float64)]
        q += [rho * v for v in vel]
        q.append(p / (self.gamma - 1.0) + 0.5 * rho * sum(v * v for v in vel))
        return np.stack(np.broadcast_arrays(*q))


class Acoustics:
    name = "acoustics"
    linear = True

    def __init__(self, dim):
        self.dim = dim
        self.nvar = dim + 1

    def flux(self, q, d):
        f = np.zeros_like(q)
        f[0] = q[1 + d]
        f[1 + d] = q[0]
        return f

    def max_speed(self, q, d):
        return np.ones_like(q[0])

    def jacobian(self, d):
        """A_d with f_d(q) = A_d q (used by the Cauchy-Kowalevski predictor)."""
        A = np.zeros((self.nvar, self.nvar))
        A[0, 1 + d] = 1.0
        A[1 + d, 0] = 1.0
        return A


def make_pde(name, dim, gamma=1.4):
    if name == "euler":
        return Euler(dim, gamma)
    if name == "acoustics":
        return Acoustics(dim)
    raise ValueError(name)
