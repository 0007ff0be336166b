"""Pins of the oracle's SU(3) generators (t^a = lambda^a / 2, the reading of Section 1's U = exp(i A^a t^a)).

The Gell-Mann matrices and the structure constants are two independently written tables; the
commutation relations [lambda^a, lambda^b] = 2 i f^{abc} lambda^c tie them together, and the
normalisation, Hermiticity and tracelessness pin the rest. A wrong entry, a wrong sign or a swapped
index in either table fails at least one of these.
"""
import numpy as np
import pytest

from oracle import su3


def test_gell_mann_hermitian_traceless_normalised():
    lam = su3.gell_mann()
    for a in range(8):
        assert np.allclose(lam[a], lam[a].conj().T, atol=0)
        assert abs(np.trace(lam[a])) < 1e-15
    gram = np.einsum("aij,bji->ab", lam, lam)
    assert np.allclose(gram, 2.0 * np.eye(8), atol=1e-14)


def test_commutators_match_structure_constants():
    lam, f = su3.gell_mann(), su3.structure_constants()
    for a in range(8):
        for b in range(8):
            comm = lam[a] @ lam[b] - lam[b] @ lam[a]
            rhs = 2j * np.einsum("c,cij->ij", f[a, b], lam)
            assert np.allclose(comm, rhs, atol=1e-14), (a + 1, b + 1)


def test_structure_constants_antisymmetric_and_jacobi():
    f = su3.structure_constants()
    assert np.allclose(f, -np.swapaxes(f, 0, 1))
    assert np.allclose(f, -np.swapaxes(f, 1, 2))
    # Jacobi identity of the Lie algebra: f^{abe} f^{ecd} + f^{bce} f^{ead} + f^{cae} f^{ebd} = 0
    jac = (np.einsum("abe,ecd->abcd", f, f) + np.einsum("bce,ead->abcd", f, f) + np.einsum("cae,ebd->abcd", f, f))
    assert np.max(np.abs(jac)) < 1e-14
    # quadratic Casimir of the adjoint representation of SU(3): f^{acd} f^{bcd} = 3 delta^{ab}
    assert np.allclose(np.einsum("acd,bcd->ab", f, f), 3.0 * np.eye(8), atol=1e-14)


def test_fundamental_casimir():
    # sum_a t^a t^a = C_F 1 with C_F = 4/3 for SU(3)
    t = su3.generators()
    assert np.allclose(np.einsum("aij,ajk->ik", t, t), 4.0 / 3.0 * np.eye(3), atol=1e-14)


@pytest.mark.parametrize("seed", [0, 1])
def test_exponential_is_special_unitary_and_inverts_projection(seed):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((5, 8))
    H = su3.algebra_element(P)
    assert np.allclose(su3.project_coefficients(H), P, atol=1e-14)
    U = su3.expi(H)
    eye = np.broadcast_to(np.eye(3), U.shape)
    assert np.allclose(U @ np.conj(np.swapaxes(U, -1, -2)), eye, atol=1e-14)
    assert np.allclose(np.linalg.det(U), 1.0, atol=1e-13)
    # exp(i H) exp(-i H) = 1 and small-H expansion exp(i e H) = 1 + i e H + O(e^2)
    e = 1e-7
    Ue = su3.expi(e * H)
    assert np.allclose((Ue - eye) / e, 1j * H, atol=1e-6)
