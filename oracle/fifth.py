"""Fifth-dimension (s-space) matrices of the optimal domain-wall operator (oracle, FP64).

The paper takes D_T, M_pm, Delta_pm, Omega_pm from its Ref. [Chen:2014hyy] (Section 1 after
Eq.(H)) and prints only the relations they satisfy: Eq.(DTm1m2), Eq.(delta_ij) and Eq.(k_ij).
The reading used here is the optimal domain-wall operator with c = 1, d = 0 (the paper's
m_PV = 2 m0 in Section 3.1 fixes d = 0, since m_PV = 2 m0 (1 - d m0) after Eq.(H)):

    D_odwf(m) = (omega D_w + 1) + (omega D_w - 1) L(m),   L = P_+ L_+ + P_- L_-,
    (L_+)_{s,s-1} = 1 (s >= 1), (L_+)_{0,Ns-1} = -m,     L_- = L_+^T        (0-based s)

which factors as D_odwf = omega^{1/2} D_T omega^{1/2} (1 + L) with
    D_T(m1, m2) = D_w + P_+ M_+(m1) + P_- M_-(m2),
    M_pm(m) = omega^{-1/2} (1 - L_pm(m)) (1 + L_pm(m))^{-1} omega^{-1/2}.

Sherman-Morrison on 1 + L_pm then gives, for even Ns, the rank-one mass dependence of
Eq.(delta_ij) with
    k(m_j, m_i) = 2 (m_j - m_i) / ((1 + m_j)(1 + m_i))     [Eq.(k_ij) at c = 1, lambda = 0]
    (Omega_-)_s = (-1)^s omega_s^{-1/2},  (Omega_+)_s = (-1)^(Ns-1-s) omega_s^{-1/2}.
These closed forms are pinned in the tests against a numerical rank-one factorisation of
R5 (M(m_j) - M(m_i)); the functions below build every matrix from its definition.
"""
from __future__ import annotations

import numpy as np


def l_plus(Ns, m):
    L = np.zeros((Ns, Ns))
    for s in range(1, Ns):
        L[s, s - 1] = 1.0
    L[0, Ns - 1] = -m
    return L


def l_minus(Ns, m):
    return l_plus(Ns, m).T.copy()


def r5(Ns):
    """Reflection in the fifth dimension, (R5 psi)_s = psi_{Ns-1-s}."""
    return np.eye(Ns)[::-1].copy()


def m_matrix(omega, m, chirality):
    """M_+(m) (chirality=+1) or M_-(m) (chirality=-1) from its definition."""
    omega = np.asarray(omega, dtype=np.float64)
    Ns = len(omega)
    L = l_plus(Ns, m) if chirality > 0 else l_minus(Ns, m)
    wm = np.diag(omega ** -0.5)
    one = np.eye(Ns)
    return wm @ (one - L) @ np.linalg.inv(one + L) @ wm


def omega_vector(omega, chirality):
    """Omega_- or Omega_+ of Eq.(delta_ij), closed form (see module docstring)."""
    omega = np.asarray(omega, dtype=np.float64)
    Ns = len(omega)
    s = np.arange(Ns)
    if chirality < 0:
        sign = (-1.0) ** s
    else:
        sign = (-1.0) ** (Ns - 1 - s)
    return sign * omega ** -0.5


def k_eofa(mj, mi):
    """k(m_j, m_i) of Eq.(k_ij) with c = 1, lambda = 0."""
    return 2.0 * (mj - mi) / ((1.0 + mj) * (1.0 + mi))


def a_matrix(omega, m, chirality, m0):
    """Site-diagonal part A_pm = (4 - m0) + M_pm(m) of D_T(m1, m2) (even-odd blocks)."""
    Ns = len(omega)
    return (4.0 - m0) * np.eye(Ns) + m_matrix(omega, m, chirality)
