"""The structured forms of the fifth-dimension matrices that the Ns = 16 kernels apply, pinned on the host
against the oracle's dense matrices (built from their definition in oracle/fifth.py):

* A^{-1} = W (1 + L) B^{-1} W with W = diag(omega^{1/2}) and B = (4 - m0) omega (1 + L) + (1 - L), which is
  cyclic bidiagonal (diagonal, first subdiagonal, one corner), so B^{-1} applies by one recurrence in s;
* A = (4 - m0 - 1/omega) + 2 W^{-1} (1 + L)^{-1} W^{-1}, where (1 + L)^{-1} is again a recurrence in s;
* A_-(m) = R5 A_+(m) R5 and A_+(m)^T = A_-(m) for an R5-symmetric omega: the P_- columns and the
  transposed operators run the P_+ recurrence in reversed s order.
"""
import numpy as np
import pytest

from oracle import fifth
from paper_1710_09621_gb300 import inputs

M0 = 1.3
OMEGAS = {"shamir": inputs.omega_shamir(16), "zolotarev": inputs.omega_zolotarev(16, 0.05, 6.2),
          "zolotarev8": inputs.omega_zolotarev(8, 0.05, 6.2)}


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", list(OMEGAS))
@pytest.mark.parametrize("m", [0.005, 0.01, 0.1, 1.0])
def test_ainv_factorisation(name, m):
    om = OMEGAS[name]
    Ns = len(om)
    one, W = np.eye(Ns), np.diag(np.sqrt(om))
    for chir, L in ((1, fifth.l_plus(Ns, m)), (-1, fifth.l_minus(Ns, m))):
        A = fifth.a_matrix(om, m, chir, M0)
        B = (4.0 - M0) * np.diag(om) @ (one + L) + (one - L)
        # B is cyclic bidiagonal
        mask = np.eye(Ns, dtype=bool) | np.eye(Ns, k=-1, dtype=bool) | np.eye(Ns, k=1, dtype=bool)
        mask[0, Ns - 1] = mask[Ns - 1, 0] = True
        assert np.all(B[~mask] == 0.0)
        assert _rel(W @ (one + L) @ np.linalg.inv(B) @ W, np.linalg.inv(A)) < 1e-12


@pytest.mark.parametrize("name", list(OMEGAS))
@pytest.mark.parametrize("m", [0.01, 0.3, 1.0])
def test_a_form(name, m):
    om = OMEGAS[name]
    Ns = len(om)
    one, Wi = np.eye(Ns), np.diag(om ** -0.5)
    for chir, L in ((1, fifth.l_plus(Ns, m)), (-1, fifth.l_minus(Ns, m))):
        A = fifth.a_matrix(om, m, chir, M0)
        A2 = np.diag(4.0 - M0 - 1.0 / om) + 2.0 * Wi @ np.linalg.inv(one + L) @ Wi
        assert _rel(A2, A) < 1e-13


@pytest.mark.parametrize("name", list(OMEGAS))
def test_chirality_and_transpose_are_reversals(name):
    om = OMEGAS[name]
    Ns = len(om)
    R = fifth.r5(Ns)
    assert np.allclose(om, om[::-1])  # the R5 symmetry these relations need
    for m in (0.01, 0.2, 1.0):
        Ap, Am = fifth.a_matrix(om, m, 1, M0), fifth.a_matrix(om, m, -1, M0)
        assert _rel(R @ Ap @ R, Am) < 1e-13
        assert _rel(Ap.T, Am) < 1e-13
        assert _rel(np.linalg.inv(Ap).T, np.linalg.inv(Am)) < 1e-12
