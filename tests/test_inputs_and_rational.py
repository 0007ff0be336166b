"""Pins of the synthetic-input generators and of the oracle's rational approximation."""
import numpy as np
import pytest

from oracle.rational import inv_sqrt_for_error, zolotarev_inv_sqrt
from paper_1710_09621_gb300.inputs import (gaussian_spinor, gell_mann, omega_zolotarev,
                                           random_su3_links)


def test_links_are_su3():
    U = random_su3_links((4, 4, 2, 6), 0.3, 1)
    eye = np.eye(3)
    assert np.max(np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - eye)) < 1e-14
    assert np.max(np.abs(np.linalg.det(U) - 1.0)) < 1e-14


def test_gell_mann_normalisation():
    l = gell_mann()
    tr = np.einsum("aij,bji->ab", l, l)
    assert np.allclose(tr, 2 * np.eye(8))
    assert np.allclose(np.einsum("aii->a", l), 0)


def test_gaussian_weight():
    eta = gaussian_spinor((8, 8, 8, 8), 3)
    # exp(-eta^dag eta): <|z|^2> = 1 per complex component
    assert abs(np.mean(np.abs(eta) ** 2) - 1.0) < 0.02


def _alternations(e, frac=1e-3):
    """Number of alternating-sign runs where |e| is within frac of its maximum."""
    big = np.abs(e) >= (1 - frac) * np.abs(e).max()
    sgn = np.sign(e[big])
    idx = np.nonzero(big)[0]
    runs = 1 + int(np.sum((np.diff(idx) > 1) | (np.diff(sgn) != 0)))
    # runs must alternate in sign
    starts = np.concatenate([[0], np.nonzero((np.diff(idx) > 1) | (np.diff(sgn) != 0))[0] + 1])
    assert np.all(np.diff(sgn[starts]) != 0)
    return runs


@pytest.mark.parametrize("Ns", [4, 6, 8, 12, 16])
def test_omega_zolotarev(Ns):
    lmin, lmax = 0.05, 6.2
    w = omega_zolotarev(Ns, lmin, lmax)
    assert np.all(w > 0) and np.array_equal(w, w[::-1])  # R5 symmetry, positive
    n = Ns // 2
    x = np.geomspace(lmin, lmax, 400001)
    T = np.prod([(1 - wi * x) / (1 + wi * x) for wi in w[:n]], axis=0)
    R = (1 - T) / (1 + T)
    e = 1 - R
    # optimal (Chebyshev) approximation: n + 1 alternation points of equal height
    assert _alternations(e) == n + 1
    # the full Ns-weight approximation is 2R/(1+R^2)
    Tf = np.prod([(1 - wi * x) / (1 + wi * x) for wi in w], axis=0)
    assert np.allclose((1 - Tf) / (1 + Tf), 2 * R / (1 + R**2), atol=1e-13)


@pytest.mark.parametrize("lo,hi", [(0.5, 1.0), (0.01, 1.0), (1.0, 1e4)])
def test_zolotarev_inv_sqrt_equioscillates(lo, hi):
    for n in (2, 4, 7):
        r = zolotarev_inv_sqrt(n, lo, hi)
        x = np.geomspace(lo, hi, 400001)
        e = 1 - np.sqrt(x) * r(x)
        # (n, n) type: 2n + 2 alternation points (until rounding dominates)
        if r.err > 1e-8:
            assert _alternations(e) == 2 * n + 2
        assert np.all(r.b > 0)


def test_inv_sqrt_target():
    r = inv_sqrt_for_error(0.49, 1.0, 1e-12)
    x = np.geomspace(0.49, 1.0, 10001)
    assert np.max(np.abs(1 - np.sqrt(x) * r(x))) <= 1e-12
    assert r.n_poles <= 6
