"""Dense-matrix construction of the EOFA objects on tiny lattices, for brute-force pins.

Builds D_w as a dense matrix from the oracle's matrix-free D_w (unit-vector columns) and then
assembles D_T(m1, m2) = 1_s (x) D_w + M_+(m1) (x) P_+ + M_-(m2) (x) P_- with Kronecker products,
so that the dense operator is an independent assembly of Eq.(DTm1m2).
"""
import numpy as np

from oracle import fifth
from oracle.operators import ODWF, dense
from oracle.wilson import GAMMA5, P_MINUS, P_PLUS, wilson


class DenseEOFA:
    def __init__(self, op: ODWF):
        self.op = op
        Lx, Ly, Lz, Lt = op.dims
        self.V = Lx * Ly * Lz * Lt
        self.n4 = self.V * 12
        self.Ns = op.Ns
        shape4 = (Lt, Lz, Ly, Lx, 4, 3)
        self.Dw = dense(lambda v: wilson(op.U, v, op.m0), shape4)
        iv, ic = np.eye(self.V), np.eye(3)
        self.Pp = np.kron(iv, np.kron(P_PLUS, ic))
        self.Pm = np.kron(iv, np.kron(P_MINUS, ic))
        self.G5 = np.kron(iv, np.kron(GAMMA5, ic))
        self.R5 = np.kron(fifth.r5(self.Ns), np.eye(self.n4))
        self.G5R5 = self.R5 @ np.kron(np.eye(self.Ns), self.G5)

    def dt(self, m1, m2):
        om = self.op.omega
        return (np.kron(np.eye(self.Ns), self.Dw)
                + np.kron(fifth.m_matrix(om, m1, +1), self.Pp)
                + np.kron(fifth.m_matrix(om, m2, -1), self.Pm))

    def ht(self, m1, m2):
        return self.G5R5 @ self.dt(m1, m2)

    def omega_op(self, chir):
        """4D -> 5D embedding phi -> Omega_s phi as a (Ns*n4, n4) matrix."""
        Om = fifth.omega_vector(self.op.omega, chir)
        return np.kron(Om[:, None], np.eye(self.n4))

    def chiral_index(self, chir):
        spin = (np.arange(self.n4) // 3) % 4
        return np.where(spin < 2)[0] if chir > 0 else np.where(spin >= 2)[0]

    def term_x(self, term):
        """The term's 4D operator X restricted to its chirality (square, dimension V*6)."""
        c = term.chirality
        Om = self.omega_op(c)
        Hinv = np.linalg.inv(self.ht(term.m3, term.m4))
        sgn = -1.0 if c < 0 else 1.0
        X = np.eye(self.n4) + sgn * term.k * Om.T @ Hinv @ Om
        idx = self.chiral_index(c)
        return X[np.ix_(idx, idx)]

    def logdet_dt(self, m1, m2):
        sign, ld = np.linalg.slogdet(self.dt(m1, m2))
        return ld + np.log(sign)
