"""Gauge-equivariant learned preconditioner for the Schur system (oracle, FP64).

Not in the paper: the paper solves every H_T system with CG (Section 1). This is the reading of
the learned-preconditioner requirement used by the library: a two-layer network of parallel-
transport convolutions whose only learned parameters are 4x4 complex spin matrices, placed
around the exact fifth-dimension inverse A^{-1} of the even-odd blocks. For an even-site 5D
residual r:

    u   = A^{-1} r                                   (even sites)
    h_c = sum_d W1[c, d] T_d u,   c = 0..C-1          (odd sites; layer 1, 1 -> C channels)
    v_c = A^{-1} h_c                                  (odd sites)
    y   = sum_c sum_d W2[c, d] T_d v_c                (even sites; layer 2, C -> 1 channel)
    M r = W0 u + 1/4 A^{-1} y

T_d is parallel transport along direction d: T_mu psi(x) = U_mu(x) psi(x+mu),
T_{4+mu} psi(x) = U_mu(x-mu)^dag psi(x-mu) (antiperiodic in t). W acts on the spin index only, so
M[U^g](G r) = G M[U] r for every gauge transform G. With W0 = 1, W1[0, mu] = W2[0, mu] = 1 - gamma_mu,
W1[0, 4+mu] = W2[0, 4+mu] = 1 + gamma_mu and the other channels zero, M is exactly the two-term
Neumann series A^{-1} + 1/4 A^{-1} H A^{-1} H A^{-1} of S^{-1} = (A - 1/4 H A^{-1} H)^{-1}.

Training loss over pairs (r_i, e_i = S^{-1} r_i): L = sum_i |M r_i - e_i|^2 / |e_i|^2 ("error" loss),
or, needing no solves, L = sum_i |S M r_i - r_i|^2 / |r_i|^2 ("residual" loss: how far S M is from the
identity on the training vectors). Gradients are Wirtinger derivatives dL/dconj(W) (the steepest-descent
direction for complex W); for the residual loss dL/dconj(M r) = S^dag (S M r - r) / |r|^2.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .operators import chiral_s_mul
from .solver import Schur
from .wilson import GAMMA, color_mul, dagger, link_bwd, shift_bwd, shift_fwd, spin_mul


@dataclass
class Weights:
    W0: np.ndarray   # (4, 4)
    W1: np.ndarray   # (C, 8, 4, 4)
    W2: np.ndarray   # (C, 8, 4, 4)

    @property
    def C(self):
        return self.W1.shape[0]

    def copy(self):
        return Weights(self.W0.copy(), self.W1.copy(), self.W2.copy())

    def flat(self):
        return np.concatenate([self.W0.ravel(), self.W1.ravel(), self.W2.ravel()])

    @staticmethod
    def from_flat(v, C):
        a = 16
        b = a + C * 8 * 16
        return Weights(v[:a].reshape(4, 4).copy(), v[a:b].reshape(C, 8, 4, 4).copy(),
                       v[b:].reshape(C, 8, 4, 4).copy())


def neumann_weights(C=2, noise=0.0, seed=0):
    """Weights that reproduce the two-term Neumann series; extra channels zero (or small noise)."""
    one = np.eye(4, dtype=np.complex128)
    W1 = np.zeros((C, 8, 4, 4), dtype=np.complex128)
    W2 = np.zeros((C, 8, 4, 4), dtype=np.complex128)
    for mu in range(4):
        W1[0, mu] = one - GAMMA[mu]
        W1[0, 4 + mu] = one + GAMMA[mu]
        W2[0, mu] = one - GAMMA[mu]
        W2[0, 4 + mu] = one + GAMMA[mu]
    if noise:
        rng = np.random.default_rng(seed)
        W1[1:] = noise * (rng.standard_normal(W1[1:].shape) + 1j * rng.standard_normal(W1[1:].shape))
        W2[1:] = noise * (rng.standard_normal(W2[1:].shape) + 1j * rng.standard_normal(W2[1:].shape))
    return Weights(one.copy(), W1, W2)


def transport(U, psi, d):
    """T_d psi on a 5D (or 4D) spinor field."""
    if d < 4:
        return color_mul(U[d], shift_fwd(psi, d))
    mu = d - 4
    return color_mul(dagger(link_bwd(U, mu)), shift_bwd(psi, mu))


def transport_adj(U, g, d):
    """Adjoint of T_d: T_mu^dag g(x) = U_mu(x-mu)^dag g(x-mu); T_{4+mu}^dag g(x) = U_mu(x) g(x+mu)."""
    if d < 4:
        return color_mul(dagger(link_bwd(U, d)), shift_bwd(g, d))
    mu = d - 4
    return color_mul(U[mu], shift_fwd(g, mu))


class LearnedPreconditioner:
    def __init__(self, sch: Schur, W: Weights):
        self.sch = sch
        self.U = sch.op.U
        self.W = W

    def _AinvT(self, v):
        return chiral_s_mul(self.sch.Apinv.T, self.sch.Aminv.T, v)

    def forward(self, r, keep=False):
        sch, U, W = self.sch, self.U, self.W
        even, odd = sch.even, sch.odd
        u = sch.Ainv(even * r)
        Tu = [odd * transport(U, u, d) for d in range(8)]
        h = [sum(spin_mul(W.W1[c, d], Tu[d]) for d in range(8)) for c in range(W.C)]
        v = [sch.Ainv(hc) for hc in h]
        Tv = [[even * transport(U, v[c], d) for d in range(8)] for c in range(W.C)]
        y = sum(spin_mul(W.W2[c, d], Tv[c][d]) for c in range(W.C) for d in range(8))
        out = spin_mul(W.W0, u) + 0.25 * sch.Ainv(y)
        if keep:
            return out, dict(u=u, Tu=Tu, v=v, Tv=Tv)
        return out

    def adjoint(self, g):
        """M^dag g (the adjoint network), so that <a, M b> = <M^dag a, b>."""
        sch, U, W = self.sch, self.U, self.W
        even, odd = sch.even, sch.odd
        g = even * g
        gy = 0.25 * self._AinvT(g)
        gu = spin_mul(W.W0.conj().T, g)
        for c in range(W.C):
            gv = sum(odd * transport_adj(U, spin_mul(W.W2[c, d].conj().T, gy), d) for d in range(8))
            gh = self._AinvT(gv)
            gu = gu + sum(even * transport_adj(U, spin_mul(W.W1[c, d].conj().T, gh), d) for d in range(8))
        return self._AinvT(gu)

    def _backprop(self, t, dl, G0, G1, G2):
        """Add to G the Wirtinger gradient of a loss whose derivative along conj(M r) is dl."""
        sch, U, W = self.sch, self.U, self.W
        odd = sch.odd

        def outer(a, b):  # sum over sites, s and color of a_i conj(b_j)
            return np.einsum("nic,njc->ij", a.reshape(-1, 4, 3), b.conj().reshape(-1, 4, 3))
        G0 += outer(dl, t["u"])
        gy = 0.25 * self._AinvT(dl)
        for c in range(W.C):
            for d in range(8):
                G2[c, d] += outer(gy, t["Tv"][c][d])
            gv = sum(odd * transport_adj(U, spin_mul(W.W2[c, d].conj().T, gy), d) for d in range(8))
            gh = self._AinvT(gv)
            for d in range(8):
                G1[c, d] += outer(gh, t["Tu"][d])

    def loss_and_grad(self, rs, es):
        """L = sum |M r - e|^2 / |e|^2 and its Wirtinger gradient dL/dconj(W) (as a Weights)."""
        W, even = self.W, self.sch.even
        G0, G1, G2 = np.zeros_like(W.W0), np.zeros_like(W.W1), np.zeros_like(W.W2)
        L = 0.0
        for r, e in zip(rs, es):
            out, t = self.forward(r, keep=True)
            ne = np.vdot(e, e).real
            delta = (out - e) * even
            L += np.vdot(delta, delta).real / ne
            self._backprop(t, delta / ne, G0, G1, G2)   # dL/dconj(out) = delta / ne
        return L, Weights(G0, G1, G2)

    def residual_loss_and_grad(self, rs):
        """L = sum |S M r - r|^2 / |r|^2 and its Wirtinger gradient (as a Weights)."""
        sch, W, even = self.sch, self.W, self.sch.even
        G0, G1, G2 = np.zeros_like(W.W0), np.zeros_like(W.W1), np.zeros_like(W.W2)
        L = 0.0
        for r in rs:
            r = r * even
            out, t = self.forward(r, keep=True)
            nr = np.vdot(r, r).real
            w = sch.S(out) - r
            L += np.vdot(w, w).real / nr
            self._backprop(t, sch.S_dag(w) / nr, G0, G1, G2)
        return L, Weights(G0, G1, G2)
