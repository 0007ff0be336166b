"""Pins of the oracle's fifth-dimension matrices and 5D operators."""
import numpy as np
import pytest

from oracle import fifth
from oracle.operators import ODWF, dense
from oracle.wilson import GAMMA5, spin_mul
from paper_1710_09621_gb300.inputs import (gaussian_spinor5, omega_shamir, omega_zolotarev,
                                           random_su3_links)

OMEGAS = {
    "shamir8": omega_shamir(8),
    "zolo16": omega_zolotarev(16, 0.05, 6.2),
    "zolo4": omega_zolotarev(4, 0.05, 6.2),
}


@pytest.mark.parametrize("name", list(OMEGAS))
@pytest.mark.parametrize("chir", [-1, +1])
def test_r5_m_is_symmetric(name, chir):
    om = OMEGAS[name]
    R5 = fifth.r5(len(om))
    for m in (0.01, 0.3, 1.0):
        X = R5 @ fifth.m_matrix(om, m, chir)
        assert np.allclose(X, X.T, atol=1e-13 * np.abs(X).max())


@pytest.mark.parametrize("name", list(OMEGAS))
@pytest.mark.parametrize("chir", [-1, +1])
def test_mass_dependence_is_rank_one(name, chir):
    """Eq.(delta_ij): R5 (M(m_j) - M(m_i)) = k(m_j, m_i) Omega Omega^T, factorised numerically."""
    om = OMEGAS[name]
    R5 = fifth.r5(len(om))
    for mj, mi in [(1.0, 0.01), (0.1, 0.05), (0.3, 0.7)]:
        D = R5 @ (fifth.m_matrix(om, mj, chir) - fifth.m_matrix(om, mi, chir))
        w, v = np.linalg.eigh(0.5 * (D + D.T))
        j = np.argmax(np.abs(w))
        assert np.all(np.abs(np.delete(w, j)) < 1e-12 * abs(w[j]))
        # the single nonzero eigenpair equals k |Omega|^2 and Omega/|Omega| (up to sign)
        Om = fifth.omega_vector(om, chir)
        k = fifth.k_eofa(mj, mi)
        assert np.isclose(w[j], k * Om @ Om, rtol=1e-11)
        assert np.isclose(abs(v[:, j] @ Om) / np.linalg.norm(Om), 1.0, rtol=1e-12)
        # and the sign convention of Omega matters only through Omega Omega^T
        assert np.allclose(D, k * np.outer(Om, Om), atol=1e-12 * np.abs(D).max())


def test_k_reduces_at_pauli_villars():
    # Eq.(Hij) -> Eq.(H) at m_j = 1: k(1, m) = (1 - m)/(1 + m) with c = 1, lambda = 0
    for m in (0.01, 0.5):
        assert np.isclose(fifth.k_eofa(1.0, m), (1 - m) / (1 + m))


def _op(dims=(2, 2, 2, 2), name="zolo4", seed=5):
    return ODWF(random_su3_links(dims, 0.4, seed), 1.3, OMEGAS[name])


def test_dodwf_factorisation_dense():
    """D_odwf = omega^{1/2} D_T omega^{1/2} (1 + L) on a 2^4 x Ns=4 lattice."""
    op = _op()
    Ns = op.Ns
    shape = op.shape5()
    m1, m2 = 0.05, 0.3
    w = op.omega.reshape((Ns,) + (1,) * 6)
    from oracle.operators import chiral_s_mul
    L = lambda v: chiral_s_mul(fifth.l_plus(Ns, m1), fifth.l_minus(Ns, m2), v)
    rhs = lambda v: np.sqrt(w) * op.dt(np.sqrt(w) * (v + L(v)), m1, m2)
    rng = np.random.default_rng(0)
    for _ in range(3):
        v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        assert np.allclose(op.dodwf(v, m1, m2), rhs(v), atol=1e-12)


def test_ht_is_hermitian():
    op = _op(dims=(2, 4, 2, 2), name="zolo4")
    a, b = gaussian_spinor5(op.dims, op.Ns, 1), gaussian_spinor5(op.dims, op.Ns, 2)
    for m1, m2 in [(0.05, 0.05), (0.01, 1.0), (1.0, 0.1)]:
        assert np.isclose(np.vdot(a, op.ht(b, m1, m2)), np.vdot(op.ht(a, m1, m2), b), rtol=1e-13)
        # D_T^dag written from the definition agrees with the adjoint
        assert np.isclose(np.vdot(a, op.dt(b, m1, m2)), np.vdot(op.dt_dag(a, m1, m2), b), rtol=1e-13)


def test_ht_dense_hermitian_2x4():
    op = _op()
    H = dense(lambda v: op.ht(v, 0.1, 0.5), op.shape5())
    assert np.max(np.abs(H - H.conj().T)) < 1e-13
