"""5D operators D_T(m1,m2), H_T(m1,m2) and D_odwf (oracle, FP64).

D_T(m1, m2) of Eq.(DTm1m2): D_w(-m0) on every s-slice plus P_+ M_+(m1) + P_- M_-(m2) on the
fifth dimension. H_T(m1, m2) = gamma_5 R5 D_T(m1, m2) (after Eq.(m1m2_m3m2)). The optimal
domain-wall operator itself is D_odwf = (omega D_w + 1) + (omega D_w - 1) L (see fifth.py).

5D spinor arrays have shape (Ns, Lt, Lz, Ly, Lx, 4, 3).
"""
from __future__ import annotations

import numpy as np

from . import fifth
from .wilson import GAMMA5, wilson, wilson_dag, spin_mul

UP = slice(0, 2)   # P_+ spin components in the chiral basis
DN = slice(2, 4)   # P_- spin components


def s_mul(Mat, psi):
    """(Mat psi)_s = sum_t Mat[s, t] psi_t on the fifth-dimension index (axis 0)."""
    return np.einsum("st,t...->s...", Mat, psi)


def chiral_s_mul(Mp, Mm, psi):
    """P_+ Mp psi + P_- Mm psi."""
    out = np.empty_like(psi)
    out[..., UP, :] = s_mul(Mp, psi[..., UP, :])
    out[..., DN, :] = s_mul(Mm, psi[..., DN, :])
    return out


class ODWF:
    """Gauge field, domain-wall height m0 and weights omega_s of one lattice."""

    def __init__(self, U, m0, omega):
        self.U = np.asarray(U, dtype=np.complex128)
        self.m0 = float(m0)
        self.omega = np.asarray(omega, dtype=np.float64)
        self.Ns = len(self.omega)
        Lt, Lz, Ly, Lx = self.U.shape[1:5]
        self.dims = (Lx, Ly, Lz, Lt)

    def shape5(self):
        Lx, Ly, Lz, Lt = self.dims
        return (self.Ns, Lt, Lz, Ly, Lx, 4, 3)

    def m_pair(self, m1, m2):
        return fifth.m_matrix(self.omega, m1, +1), fifth.m_matrix(self.omega, m2, -1)

    # D_T(m1, m2), Eq.(DTm1m2)
    def dt(self, psi, m1, m2):
        Mp, Mm = self.m_pair(m1, m2)
        return wilson(self.U, psi, self.m0) + chiral_s_mul(Mp, Mm, psi)

    def dt_dag(self, psi, m1, m2):
        Mp, Mm = self.m_pair(m1, m2)
        return wilson_dag(self.U, psi, self.m0) + chiral_s_mul(Mp.T, Mm.T, psi)

    # H_T(m1, m2) = gamma_5 R5 D_T(m1, m2)
    def ht(self, psi, m1, m2):
        return spin_mul(GAMMA5, self.dt(psi, m1, m2)[::-1])

    # D_odwf(m1, m2) = (omega D_w + 1) + (omega D_w - 1) L(m1, m2)
    def dodwf(self, psi, m1, m2):
        Ns = self.Ns
        Lp, Lm = fifth.l_plus(Ns, m1), fifth.l_minus(Ns, m2)
        Lpsi = chiral_s_mul(Lp, Lm, psi)
        w = self.omega.reshape((Ns,) + (1,) * 6)
        return w * wilson(self.U, psi + Lpsi, self.m0) + psi - Lpsi


def dense(apply, shape):
    """Dense matrix of a linear map on arrays of the given shape (unit-vector columns)."""
    n = int(np.prod(shape))
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        cols.append(apply(e.reshape(shape)).reshape(n))
    return np.stack(cols, axis=1)


def dt_at_sites(op: ODWF, psi, m1, m2, sites):
    """(D_T(m1, m2) psi)(x, s) for a list of (s, t, z, y, x) points, one at a time (Eq.(DTm1m2)).

    For checks at lattice sizes where a whole-lattice apply is too slow: each output is the
    site term, the eight nearest-neighbour hops of D_w and the fifth-dimension sum of M_pm.
    """
    from .wilson import GAMMA
    Mp, Mm = op.m_pair(m1, m2)
    Lx, Ly, Lz, Lt = op.dims
    L = {0: Lx, 1: Ly, 2: Lz, 3: Lt}
    out = []
    one = np.eye(4)
    for (s, t, z, y, x) in sites:
        c = [x, y, z, t]
        v = (4.0 - op.m0) * psi[s, t, z, y, x]
        for mu in range(4):
            f = list(c)
            f[mu] = (c[mu] + 1) % L[mu]
            b = list(c)
            b[mu] = (c[mu] - 1) % L[mu]
            sf = -1.0 if (mu == 3 and c[3] == Lt - 1) else 1.0
            sb = -1.0 if (mu == 3 and c[3] == 0) else 1.0
            Uf = op.U[mu, t, z, y, x]
            Ub = op.U[mu, b[3], b[2], b[1], b[0]]
            pf = sf * psi[s, f[3], f[2], f[1], f[0]]
            pb = sb * psi[s, b[3], b[2], b[1], b[0]]
            v = v - 0.5 * ((one - GAMMA[mu]) @ (pf @ Uf.T) + (one + GAMMA[mu]) @ (pb @ Ub.conj()))
        col = psi[:, t, z, y, x]  # (Ns, 4, 3)
        v = v.copy()
        v[0:2] += np.einsum("t,tic->ic", Mp[s], col[:, 0:2])
        v[2:4] += np.einsum("t,tic->ic", Mm[s], col[:, 2:4])
        out.append(v)
    return np.array(out)
