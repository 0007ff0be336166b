"""SU(3) generators of the force and of the link update (oracle, FP64).

The paper writes the gauge field as U = exp(i A^a t^a) and the MD equations dU/dtau = i P U
with P = P^a t^a (Section 1, Eq.(molecular_U) and Eq.(molecular_P)); it does not fix the
normalisation of t^a. The reading used throughout is t^a = lambda^a / 2 with the eight
Gell-Mann matrices lambda^a, so that tr(t^a t^b) = delta^{ab} / 2.

This module writes the Gell-Mann matrices out entry by entry and the totally antisymmetric
structure constants f^{abc} from their published non-zero values
(f^{123} = 1; f^{147} = f^{246} = f^{257} = f^{345} = 1/2; f^{156} = f^{367} = -1/2;
f^{458} = f^{678} = sqrt(3)/2). The tests pin the matrices against the commutation relations
[lambda^a, lambda^b] = 2 i f^{abc} lambda^c, so a wrong entry or a wrong sign in either table fails.
It shares nothing with the seeded input generators.
"""
from __future__ import annotations

import itertools

import numpy as np


def gell_mann() -> np.ndarray:
    """lambda^1 .. lambda^8 as an array (8, 3, 3), index a - 1."""
    s3 = np.sqrt(3.0)
    lam = [
        [[0, 1, 0], [1, 0, 0], [0, 0, 0]],
        [[0, -1j, 0], [1j, 0, 0], [0, 0, 0]],
        [[1, 0, 0], [0, -1, 0], [0, 0, 0]],
        [[0, 0, 1], [0, 0, 0], [1, 0, 0]],
        [[0, 0, -1j], [0, 0, 0], [1j, 0, 0]],
        [[0, 0, 0], [0, 0, 1], [0, 1, 0]],
        [[0, 0, 0], [0, 0, -1j], [0, 1j, 0]],
        [[1 / s3, 0, 0], [0, 1 / s3, 0], [0, 0, -2 / s3]],
    ]
    return np.array(lam, dtype=np.complex128)


def generators() -> np.ndarray:
    """t^a = lambda^a / 2, shape (8, 3, 3)."""
    return 0.5 * gell_mann()


_F_NONZERO = {(1, 2, 3): 1.0,
              (1, 4, 7): 0.5, (2, 4, 6): 0.5, (2, 5, 7): 0.5, (3, 4, 5): 0.5,
              (1, 5, 6): -0.5, (3, 6, 7): -0.5,
              (4, 5, 8): np.sqrt(3.0) / 2, (6, 7, 8): np.sqrt(3.0) / 2}


def structure_constants() -> np.ndarray:
    """f^{abc} (8, 8, 8), index a - 1, totally antisymmetric."""
    f = np.zeros((8, 8, 8))
    for (a, b, c), v in _F_NONZERO.items():
        for perm in itertools.permutations((0, 1, 2)):
            idx = tuple((a, b, c)[p] - 1 for p in perm)
            # sign of the permutation
            sgn = 1.0
            p = list(perm)
            for i in range(3):
                for j in range(i + 1, 3):
                    if p[i] > p[j]:
                        sgn = -sgn
            f[idx] = sgn * v
    return f


def algebra_element(P) -> np.ndarray:
    """P^a t^a for real coefficients P (..., 8) -> Hermitian traceless (..., 3, 3)."""
    return np.einsum("...a,aij->...ij", np.asarray(P, dtype=np.float64), generators())


def expi(H) -> np.ndarray:
    """exp(i H) of Hermitian 3x3 matrices (..., 3, 3) by the eigen-decomposition."""
    H = 0.5 * (H + np.conj(np.swapaxes(H, -1, -2)))
    w, v = np.linalg.eigh(H)
    return np.einsum("...ia,...a,...ja->...ij", v, np.exp(1j * w), v.conj())


def project_coefficients(M) -> np.ndarray:
    """Coefficients c^a = 2 Re tr(t^a M) of the Hermitian traceless part of M (..., 3, 3) -> (..., 8)."""
    return 2.0 * np.real(np.einsum("aij,...ji->...a", generators(), M))
