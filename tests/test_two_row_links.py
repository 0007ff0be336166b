"""The two-row link representation of the two-slice hop kernels, checked on the host (no GPU).

An SU(3) matrix V is fixed by its first two rows: V^{-1} = V^dag and det V = 1 make row 2 the complex
conjugate of the cross product of rows 0 and 1. The kernels store rows 0 and 1 of each link without the
antiperiodic boundary sign and carry the sign in the neighbour table, because for -V (det = -1) the same
construction returns +row 2. The library enables the form only when the relayout measures every link's
deviation |row 2 - conj(row 0 x row 1)| below 1e-6; a field of non-unitary links must fail that check.
"""
import numpy as np

from paper_1710_09621_gb300 import inputs


def _third_row(V):
    return np.conj(np.cross(V[..., 0, :], V[..., 1, :]))


def test_su3_links_are_fixed_by_two_rows():
    U = inputs.random_su3_links((4, 4, 2, 4), 0.4, 5)
    dev = np.max(np.abs(_third_row(U) - U[..., 2, :]))
    assert dev < 1e-13, dev
    # the backward links are stored daggered: also SU(3)
    Ud = np.conj(np.swapaxes(U, -1, -2))
    assert np.max(np.abs(_third_row(Ud) - Ud[..., 2, :])) < 1e-13


def test_boundary_sign_is_not_carried_by_two_rows():
    V = inputs.random_su3_links((2, 2, 2, 2), 0.4, 6)[0, 0, 0, 0, 0]
    W = -V
    # rows 0 and 1 of -V rebuild +row 2 of V, not -row 2: the sign has to travel separately
    assert np.allclose(_third_row(W), V[2], atol=1e-13)
    assert not np.allclose(_third_row(W), W[2], atol=1e-3)


def test_non_unitary_links_fail_the_check():
    U = 1.01 * inputs.random_su3_links((2, 2, 2, 2), 0.3, 3)
    dev = np.max(np.abs(_third_row(U) - U[..., 2, :]))
    assert dev > 1e-3  # far above the 1e-6 threshold of the relayout's check
