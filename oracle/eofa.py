"""EOFA chiral pseudofermion terms: operator, action, force, heat-bath, term lists (oracle).

A term is the determinant ratio of Eq.(m1m2_m3m4) in one of its two chiral special cases:

  chirality -1:  (m3, m4)/(m3, m_den)   Eq.(m1m2_m1m4)
       X_- = P_- [1 - k(m_den, m4) Omega_-^T H_T(m3, m4)^{-1} Omega_-] P_-
  chirality +1:  (m3, m4)/(m_den, m4)   Eq.(m1m2_m3m2)
       X_+ = P_+ [1 + k(m_den, m3) Omega_+^T H_T(m3, m4)^{-1} Omega_+] P_+

with the action S = phi^dag X phi. Omega acts as (Omega phi)(x, s) = Omega_s phi(x) and Omega^T
contracts s. 4D fields have shape (Lt, Lz, Ly, Lx, 4, 3); only the term's chirality is used.

Force (Section 1, Eq.(molecular_P)): with U_l = exp(i A^a t^a) and dU/dtau = i P U, the force on
link (x, mu) is F^a_mu(x) = -dS/dw^a at w = 0 for U_mu(x) -> exp(i w^a t^a) U_mu(x). The paper
does not state the normalisation of t^a; the reading is t^a = lambda^a / 2.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fifth, su3
from .operators import ODWF
from .rational import InvSqrtRational, inv_sqrt_for_error
from .solver import solve_ht
from .wilson import GAMMA, GAMMA5, P_MINUS, P_PLUS, shift_fwd, spin_mul


@dataclass(frozen=True)
class Term:
    chirality: int  # -1 or +1
    m3: float
    m4: float
    m_den: float

    @property
    def k(self):
        if self.chirality < 0:
            return fifth.k_eofa(self.m_den, self.m4)
        return fifth.k_eofa(self.m_den, self.m3)

    @property
    def numerator(self):
        return (self.m3, self.m4)

    @property
    def denominator(self):
        return (self.m3, self.m_den) if self.chirality < 0 else (self.m_den, self.m4)


def term_from_ratio(num, den):
    """(m3, m4)/(m1, m2) -> Term; needs m1 == m3 (chirality -) or m2 == m4 (chirality +)."""
    (m3, m4), (m1, m2) = num, den
    if m1 == m3 and m2 != m4:
        return Term(-1, m3, m4, m2)
    if m2 == m4 and m1 != m3:
        return Term(+1, m3, m4, m1)
    raise ValueError("ratio is neither chiral special case of Eq.(m1m2_m3m4)")


def no_mp(m, M):
    """Eq.(noMP): (m,m)/(M,M) = (m,m)/(m,M) * (m,M)/(M,M); chiralities {-, +}."""
    return [term_from_ratio((m, m), (m, M)), term_from_ratio((m, M), (M, M))]


def old_mp(m, mh, M):
    """Eq.(old_MP): four factors, chiralities {-, +, -, +}."""
    return [term_from_ratio((m, m), (m, mh)), term_from_ratio((m, mh), (mh, mh)),
            term_from_ratio((mh, mh), (mh, M)), term_from_ratio((mh, M), (M, M))]


def new_mp(m, mh, M):
    """Eq.(new_MP): (m,m)/(m,mh) * (m,mh)/(M,mh) * (M,mh)/(M,M); chiralities {-, +, -}."""
    return [term_from_ratio((m, m), (m, mh)), term_from_ratio((m, mh), (M, mh)),
            term_from_ratio((M, mh), (M, M))]


def old_mp_cascade(m, mhs, M):
    """Eq.(old_MP_N): 2N+2 factors for heavy masses m < mh_1 < ... < mh_N < M."""
    ms = [m] + list(mhs) + [M]
    out = []
    for a, b in zip(ms[:-1], ms[1:]):
        out += [term_from_ratio((a, a), (a, b)), term_from_ratio((a, b), (b, b))]
    return out


def new_mp_cascade(m, mhs, M):
    """Eq.(new_MP_N): N+2 factors (m,m)/(m,h1) (m,h1)/(h2,h1) (h2,h1)/(h2,h3) ... (M,hN)/(M,M)."""
    mhs = list(mhs)
    N = len(mhs)
    ratios = []
    cur = (m, m)
    nxt = (m, mhs[0])
    ratios.append((cur, nxt))
    cur = nxt
    for i in range(1, N + 1):
        target = mhs[i] if i < N else M
        if i % 2 == 1:  # change the left mass
            nxt = (target, cur[1])
        else:           # change the right mass
            nxt = (cur[0], target)
        ratios.append((cur, nxt))
        cur = nxt
    # last factor reaches (M, M)
    ratios.append((cur, (M, M)))
    return [term_from_ratio(a, b) for a, b in ratios]


def projector(chirality):
    return P_MINUS if chirality < 0 else P_PLUS


def omega_embed(op: ODWF, chirality, phi):
    """(Omega P phi)(x, s) = Omega_s (P phi)(x) as a 5D field."""
    Om = fifth.omega_vector(op.omega, chirality)
    pphi = spin_mul(projector(chirality), phi)
    return Om.reshape((op.Ns,) + (1,) * 6) * pphi[None]


def omega_contract(op: ODWF, chirality, chi):
    """P Omega^T chi = P sum_s Omega_s chi(x, s) as a 4D field."""
    Om = fifth.omega_vector(op.omega, chirality)
    return spin_mul(projector(chirality), np.einsum("s,s...->...", Om, chi))


def term_chi(op: ODWF, term: Term, phi, tol=1e-12):
    b = omega_embed(op, term.chirality, phi)
    chi, info = solve_ht(op, b, term.m3, term.m4, tol=tol)
    return b, chi, info


def term_apply(op: ODWF, term: Term, phi, tol=1e-12):
    """X phi for the term's 4D operator."""
    sgn = -1.0 if term.chirality < 0 else 1.0
    _, chi, _ = term_chi(op, term, phi, tol)
    P = projector(term.chirality)
    return spin_mul(P, phi) + sgn * term.k * omega_contract(op, term.chirality, chi)


def action(op: ODWF, term: Term, phi, tol=1e-12):
    """S = phi^dag X phi = |P phi|^2 -/+ k <Omega P phi, H_T^{-1} Omega P phi>."""
    sgn = -1.0 if term.chirality < 0 else 1.0
    b, chi, info = term_chi(op, term, phi, tol)
    pphi = spin_mul(projector(term.chirality), phi)
    return float(np.vdot(pphi, pphi).real + sgn * term.k * np.vdot(b, chi).real), info


def _t_generators():
    return su3.generators()


def dS_dw_from_chi(op: ODWF, term: Term, chi):
    """dS/dw^a_mu(x) for U_mu(x) -> exp(i w^a t^a) U_mu(x), given chi = H_T^{-1} Omega P phi.

    S = |P phi|^2 -/+ k b^dag H_T^{-1} b with b independent of U, so
    dS = +/- k chi^dag (dH_T) chi (upper sign for chirality -1), and dH_T = gamma_5 R5 dD_w.
    The derivative of D_w's two hopping terms that contain U_mu(x):
      -1/2 (1 - g_mu) U_mu(x) psi(x+mu) at site x, -1/2 (1 + g_mu) U_mu(x)^dag psi(x) at site x+mu.
    Returns array (4, Lt, Lz, Ly, Lx, 8).
    """
    sgn = +1.0 if term.chirality < 0 else -1.0
    ta = _t_generators()
    U = op.U
    lhs = spin_mul(GAMMA5, chi[::-1])  # (gamma_5 R5 chi), hermitian-conjugated below
    one = np.eye(4)
    out = np.zeros((4,) + U.shape[1:5] + (8,))
    for mu in range(4):
        chi_f = shift_fwd(chi, mu)
        lhs_f = shift_fwd(lhs, mu)
        for a in range(8):
            dU = 1j * np.einsum("ab,...bc->...ac", ta[a], U[mu])           # d/dw of U
            dUd = np.conj(np.swapaxes(dU, -1, -2))                          # d/dw of U^dag
            t1 = spin_mul(one - GAMMA[mu], np.einsum("...ab,...ib->...ia", dU, chi_f))
            t2 = spin_mul(one + GAMMA[mu], np.einsum("...ab,...ib->...ia", dUd, chi))
            v = -0.5 * (np.einsum("s...ic,s...ic->...", np.conj(lhs), t1)
                        + np.einsum("s...ic,s...ic->...", np.conj(lhs_f), t2))
            out[mu, ..., a] = sgn * term.k * v.real
    return out


def force(op: ODWF, term: Term, phi, tol=1e-12):
    """F^a_mu(x) = -dS/dw^a_mu(x); shape (4, Lt, Lz, Ly, Lx, 8)."""
    _, chi, info = term_chi(op, term, phi, tol)
    return -dS_dw_from_chi(op, term, chi), info


def force_magnitude(F):
    """F_pm after Eq.(F_noMP): 1/(4 N_l^3 N_t) [sum_{x,mu,a} (F^a_mu(x))^2]^{1/2}, as printed."""
    V = np.prod(F.shape[1:5])
    return float(np.sqrt(np.sum(F**2)) / (4.0 * V))


def pole_mass(term: Term, kprime):
    """Mass m' with k(m', m_ref) = k', m_ref = m4 (chirality -) or m3 (chirality +)."""
    mref = term.m4 if term.chirality < 0 else term.m3
    return (kprime * (1.0 + mref) + 2.0 * mref) / (2.0 - kprime * (1.0 + mref))


def heatbath(op: ODWF, term: Term, eta, rat: InvSqrtRational, tol=1e-12):
    """phi = X^{-1/2} eta ~ a0 eta + sum_l a_l (X + b_l)^{-1} eta.

    Each pole by the Woodbury identity (derived from Eq.(delta_ij)):
      chirality -1: (X + b)^{-1} = 1/(1+b) [1 + k' Omega^T H_T(m3, m')^{-1} Omega],  k(m', m4) = k'
      chirality +1: (X + b)^{-1} = 1/(1+b) [1 - k' Omega^T H_T(m', m4)^{-1} Omega],  k(m', m3) = k'
    with k' = k / (1 + b).
    """
    c = term.chirality
    peta = spin_mul(projector(c), eta)
    phi = rat.a0 * peta
    b5 = omega_embed(op, c, eta)
    iters = 0
    for al, bl in zip(rat.a, rat.b):
        kp = term.k / (1.0 + bl)
        mp = pole_mass(term, kp)
        if c < 0:
            chi, info = solve_ht(op, b5, term.m3, mp, tol=tol)
            corr = +kp * omega_contract(op, c, chi)
        else:
            chi, info = solve_ht(op, b5, mp, term.m4, tol=tol)
            corr = -kp * omega_contract(op, c, chi)
        iters += info["iters"]
        phi = phi + (al / (1.0 + bl)) * (peta + corr)
    return phi, {"iters": iters}


def default_heatbath_rational(x_lo, x_hi, target=1e-11):
    return inv_sqrt_for_error(x_lo, x_hi, target)
