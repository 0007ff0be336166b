"""4D Wilson operator D_w(-m0) of the optimal domain-wall kernel (oracle, FP64).

Eq.(DTm1m2) writes D_T's diagonal blocks as W - m0 + M_pm and its off-diagonal blocks as
sigma.t, -(sigma.t)^dag: that is the Wilson operator with negative mass -m0,

    D_w(-m0) psi(x) = (4 - m0) psi(x)
                      - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
                                   + (1 + gamma_mu) U_mu^dag(x-mu) psi(x-mu) ],

written in a chiral basis where gamma_5 = diag(1,1,-1,-1), so that P_+ = (1+gamma_5)/2 is the
upper block (the phi_+ / phi_- split of Section 2 after Eq.(H)). Boundary conditions are not
stated in the paper; the reading used is periodic in x, y, z and antiperiodic in t.

Arrays: spinor (..., Lt, Lz, Ly, Lx, 4, 3); links (4, Lt, Lz, Ly, Lx, 3, 3), mu = x, y, z, t.
"""
from __future__ import annotations

import numpy as np

_SPINOR_AXIS = {0: -3, 1: -4, 2: -5, 3: -6}  # mu -> axis of a spinor array
_LINK_AXIS = {0: -3, 1: -4, 2: -5, 3: -6}    # mu -> axis of one U_mu array (3x3 trailing)


def gamma_matrices():
    """Chiral-basis Euclidean gamma matrices (gamma_x, gamma_y, gamma_z, gamma_t) and gamma_5.

    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_t = [[0, 1], [1, 0]],
    gamma_5 = gamma_x gamma_y gamma_z gamma_t = diag(1, 1, -1, -1).
    """
    s1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    s2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    s3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    z = np.zeros((2, 2), dtype=np.complex128)
    e = np.eye(2, dtype=np.complex128)
    g = [np.block([[z, -1j * s], [1j * s, z]]) for s in (s1, s2, s3)]
    g.append(np.block([[z, e], [e, z]]))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return [np.ascontiguousarray(x) for x in g], g5


GAMMA, GAMMA5 = gamma_matrices()
P_PLUS = 0.5 * (np.eye(4) + GAMMA5)
P_MINUS = 0.5 * (np.eye(4) - GAMMA5)


def spin_mul(G, psi):
    """(G psi)_i = sum_j G_ij psi_j on the spin index."""
    return np.einsum("ij,...jc->...ic", G, psi)


def color_mul(U, psi):
    """(U psi)_a = sum_b U_ab psi_b on the color index; U broadcasts over leading s axes."""
    return np.einsum("...ab,...ib->...ia", U, psi)


def _t_sign(Lt, at_index, ndim_after):
    sign = np.ones(Lt)
    sign[at_index] = -1.0
    return sign.reshape((Lt,) + (1,) * ndim_after)


def shift_fwd(psi, mu):
    """psi(x + mu), with the antiperiodic sign for the t direction."""
    ax = _SPINOR_AXIS[mu]
    out = np.roll(psi, -1, axis=ax)
    if mu == 3:
        out = out * _t_sign(psi.shape[ax], -1, 5)
    return out


def shift_bwd(psi, mu):
    """psi(x - mu), with the antiperiodic sign for the t direction."""
    ax = _SPINOR_AXIS[mu]
    out = np.roll(psi, 1, axis=ax)
    if mu == 3:
        out = out * _t_sign(psi.shape[ax], 0, 5)
    return out


def link_bwd(U, mu):
    """U_mu(x - mu) (links carry no boundary sign; the fermion shift does)."""
    return np.roll(U[mu], 1, axis=_LINK_AXIS[mu])


def dagger(U):
    return np.conj(np.swapaxes(U, -1, -2))


def hop(U, psi):
    """H psi = sum_mu [(1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu^dag(x-mu) psi(x-mu)]."""
    out = np.zeros_like(psi)
    one = np.eye(4)
    for mu in range(4):
        out += spin_mul(one - GAMMA[mu], color_mul(U[mu], shift_fwd(psi, mu)))
        out += spin_mul(one + GAMMA[mu], color_mul(dagger(link_bwd(U, mu)), shift_bwd(psi, mu)))
    return out


def hop_dag(U, psi):
    """H^dag psi written out from the definition of H (no gamma_5 trick):
    (H^dag psi)(x) = sum_mu [(1 - g_mu) U_mu^dag(x-mu) psi(x-mu) + (1 + g_mu) U_mu(x) psi(x+mu)]."""
    out = np.zeros_like(psi)
    one = np.eye(4)
    for mu in range(4):
        out += spin_mul(one - GAMMA[mu], color_mul(dagger(link_bwd(U, mu)), shift_bwd(psi, mu)))
        out += spin_mul(one + GAMMA[mu], color_mul(U[mu], shift_fwd(psi, mu)))
    return out


def wilson(U, psi, m0):
    """D_w(-m0) psi = (4 - m0) psi - 1/2 H psi."""
    return (4.0 - m0) * psi - 0.5 * hop(U, psi)


def wilson_dag(U, psi, m0):
    return (4.0 - m0) * psi - 0.5 * hop_dag(U, psi)


def parity_mask(dims):
    """1.0 on even sites (x+y+z+t even), 0.0 on odd; shape (Lt, Lz, Ly, Lx, 1, 1)."""
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    even = ((x + y + z + t) % 2 == 0).astype(np.float64)
    return even[..., None, None]


def plaquette(U):
    """Average plaquette Re tr(U_mu(x) U_nu(x+mu) U_mu^dag(x+nu) U_nu^dag(x)) / 3 (periodic links)."""
    tot = 0.0
    n = 0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            u_nu_xmu = np.roll(U[nu], -1, axis=_LINK_AXIS[mu])
            u_mu_xnu = np.roll(U[mu], -1, axis=_LINK_AXIS[nu])
            p = U[mu] @ u_nu_xmu @ dagger(u_mu_xnu) @ dagger(U[nu])
            tot += np.real(np.trace(p, axis1=-2, axis2=-1)).mean() / 3.0
            n += 1
    return tot / n
