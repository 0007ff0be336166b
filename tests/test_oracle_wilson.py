"""Pins of the oracle's 4D Wilson operator against facts the mathematics fixes."""
import numpy as np
import pytest

from oracle import wilson
from oracle.wilson import GAMMA, GAMMA5, hop, hop_dag, spin_mul, wilson as dw
from paper_1710_09621_gb300.inputs import gaussian_spinor, random_su3_links


def test_gamma_algebra():
    one = np.eye(4)
    for mu in range(4):
        assert np.allclose(GAMMA[mu], GAMMA[mu].conj().T)
        for nu in range(4):
            ac = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            assert np.allclose(ac, 2 * one * (mu == nu))
        assert np.allclose(GAMMA5 @ GAMMA[mu] + GAMMA[mu] @ GAMMA5, 0)
    # chiral basis: P_+ is the upper block (the phi_+ / phi_- split after Eq.(H))
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 2, 6, 4)])
def test_hop_adjoint_and_gamma5_hermiticity(dims):
    U = random_su3_links(dims, 0.4, 11)
    a, b = gaussian_spinor(dims, 1), gaussian_spinor(dims, 2)
    # hop_dag is written from the definition of H^dag; the inner products pin it
    assert np.isclose(np.vdot(a, hop(U, b)), np.vdot(hop_dag(U, a), b), rtol=1e-13, atol=0)
    # (gamma_5 D_w)^dag = gamma_5 D_w
    g5dw = lambda v: spin_mul(GAMMA5, dw(U, v, 1.3))
    assert np.isclose(np.vdot(a, g5dw(b)), np.vdot(g5dw(a), b), rtol=1e-13, atol=0)


def test_gauge_covariance():
    dims = (4, 4, 2, 4)
    U = random_su3_links(dims, 0.4, 3)
    G = random_su3_links(dims, 1.0, 4)[0]  # one SU(3) matrix per site
    Ug = np.empty_like(U)
    axis = {0: -3, 1: -4, 2: -5, 3: -6}
    for mu in range(4):
        G_fwd = np.roll(G, -1, axis=axis[mu])
        Ug[mu] = G @ U[mu] @ np.conj(np.swapaxes(G_fwd, -1, -2))
    psi = gaussian_spinor(dims, 9)
    Gpsi = np.einsum("...ab,...ib->...ia", G, psi)
    lhs = dw(Ug, Gpsi, 1.3)
    rhs = np.einsum("...ab,...ib->...ia", G, dw(U, psi, 1.3))
    assert np.max(np.abs(lhs - rhs)) < 1e-13 * np.max(np.abs(rhs))


def test_free_field_plane_wave():
    """U = 1: D_w(p) = i sum gamma_mu sin p_mu + sum (1 - cos p_mu) - m0, p_t antiperiodic."""
    dims = (4, 6, 4, 8)
    Lx, Ly, Lz, Lt = dims
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, Lt, Lz, Ly, Lx, 3, 3)).copy()
    m0 = 1.3
    rng = np.random.default_rng(0)
    for n in [(1, 0, 3, 0), (3, 5, 1, 6), (0, 0, 0, 7)]:
        p = np.array([2 * np.pi * n[0] / Lx, 2 * np.pi * n[1] / Ly, 2 * np.pi * n[2] / Lz,
                      (2 * n[3] + 1) * np.pi / Lt])
        t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = phase[..., None, None] * u
        Dp = sum(1j * GAMMA[mu] * np.sin(p[mu]) for mu in range(4)) + (np.sum(1 - np.cos(p)) - m0) * np.eye(4)
        expect = phase[..., None, None] * (Dp @ u)
        assert np.max(np.abs(dw(U, psi, m0) - expect)) < 1e-13


def test_plaquette_of_unit_links_is_one():
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, 2, 2, 2, 2, 3, 3)).copy()
    assert abs(wilson.plaquette(U) - 1.0) < 1e-15
