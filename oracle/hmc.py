"""HMC molecular dynamics of the gauge field (oracle, FP64).

Section 1 of the paper writes the MD Hamiltonian as H = 1/2 sum_{l,a} (P_l^a)^2 + S_g[U] + S_pf
with U_l = exp(i A_l^a t^a) and the equations of motion Eq.(molecular_U), dU_l/dtau = i P_l U_l
(P_l = P_l^a t^a), and Eq.(molecular_P), dP_l^a/dtau = -dS/dA_l^a. Section 3 runs them with the
Omelyan integrator and the multiple-time-scale (MTS) method on three levels (k0, k1, k2): the gauge
force on the finest level with k0 steps per unit trajectory, the fermion forces of the heavy terms on
k1 and those of the light terms on k2. The smallest time step, that of the link update, is 1/(2 k0):
(480, 12, 6) gives 960 link updates and (961, 25, 13) momentum updates. The paper uses the Wilson
plaquette gauge action.

Readings (the paper is silent):
  * t^a = lambda^a / 2 (oracle.su3), force F^a = -dS/dw^a for U -> exp(i w^a t^a) U.
  * S_g = beta sum_{x, mu < nu} (1 - Re tr U_{mu nu}(x) / 3) with the plaquette
    U_{mu nu}(x) = U_mu(x) U_nu(x + mu) U_mu(x + nu)^dag U_nu(x)^dag, periodic links.
  * Omelyan's second-order minimum-norm step of size e on a level with force F and the levels below
    it as the "position" part:  P += lam e F ; below(e/2) ; P += (1 - 2 lam) e F ; below(e/2) ;
    P += lam e F,  lam = 0.1931833275037836 (Omelyan, Mryglod, Folk 2002). "below(tau)" integrates the
    next finer level over time tau with its own steps; below the finest level it is the exact link
    update U <- exp(i tau P) U. The number of steps of level i per step of level i + 1 is
    k_i / (2 k_{i+1}).
Arrays: links U (4, Lt, Lz, Ly, Lx, 3, 3); momenta and forces (4, Lt, Lz, Ly, Lx, 8).
"""
from __future__ import annotations

import numpy as np

from . import su3
from .wilson import _LINK_AXIS, dagger

OMELYAN_LAMBDA = 0.1931833275037836


def shift_link(Umu, nu, k=1):
    """U(x + k nu) for one direction's link array (periodic)."""
    return np.roll(Umu, -k, axis=_LINK_AXIS[nu])


def plaquette_field(U, mu, nu):
    """U_{mu nu}(x) at every site."""
    return U[mu] @ shift_link(U[nu], mu) @ dagger(shift_link(U[mu], nu)) @ dagger(U[nu])


def gauge_action(U, beta):
    """Wilson plaquette action beta sum_{x, mu<nu} (1 - Re tr U_{mu nu}(x) / 3)."""
    S = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            tr = np.real(np.trace(plaquette_field(U, mu, nu), axis1=-2, axis2=-1))
            S += np.sum(1.0 - tr / 3.0)
    return float(beta * S)


def staple_sum(U, mu):
    """Sigma_mu(x) = sum_{nu != mu} [U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
                                    + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)],
    so that the plaquettes containing U_mu(x) contribute Re tr(U_mu(x) Sigma_mu(x))."""
    out = np.zeros_like(U[mu])
    for nu in range(4):
        if nu == mu:
            continue
        up = shift_link(U[nu], mu) @ dagger(shift_link(U[mu], nu)) @ dagger(U[nu])
        unu_m = shift_link(U[nu], nu, -1)                       # U_nu(x - nu)
        dn = dagger(shift_link(unu_m, mu)) @ dagger(shift_link(U[mu], nu, -1)) @ unu_m
        out += up + dn
    return out


def gauge_force(U, beta):
    """F^a_mu(x) = -dS_g/dw^a for U_mu(x) -> exp(i w^a t^a) U_mu(x).

    The part of S_g that holds U_mu(x) is -(beta/3) Re tr(U_mu(x) Sigma_mu(x)); its derivative at
    w = 0 is -(beta/3) Re tr(i t^a U Sigma) = (beta/3) Im tr(t^a U Sigma), hence
    F^a = -(beta/3) Im tr(t^a U_mu(x) Sigma_mu(x))."""
    t = su3.generators()
    F = np.zeros(U.shape[:5] + (8,))
    for mu in range(4):
        W = U[mu] @ staple_sum(U, mu)
        F[mu] = -(beta / 3.0) * np.imag(np.einsum("aij,...ji->...a", t, W))
    return F


def link_update(U, P, tau):
    """U <- exp(i tau P^a t^a) U on every link (Eq.(molecular_U) over a time tau at fixed P)."""
    return np.einsum("...ij,...jk->...ik", su3.expi(tau * su3.algebra_element(P)), U)


def kinetic(P):
    return float(0.5 * np.sum(P * P))


def omelyan_mts(U, P, forces, steps, lam=OMELYAN_LAMBDA, tau=1.0, counts=None):
    """Integrate Eq.(molecular_U)/(molecular_P) over time tau with nested Omelyan steps.

    forces[i](U) -> force array of level i (level 0 the finest); steps[i] = k_i, the number of steps
    of level i over the trajectory of length tau (k_i divisible by 2 k_{i+1}). Returns (U, P); counts (a dict, if
    given) receives the number of force evaluations per level and of link updates.
    """
    L = len(steps)
    if counts is not None:
        counts.setdefault("links", 0)
        for i in range(L):
            counts.setdefault(i, 0)

    def below(level, U, P, t):
        if level < 0:
            if counts is not None:
                counts["links"] += 1
            return link_update(U, P, t), P
        n = steps[level] if level == L - 1 else steps[level] // (2 * steps[level + 1])
        e = t / n
        for _ in range(n):
            for frac, sub in ((lam, True), (1.0 - 2.0 * lam, True), (lam, False)):
                if counts is not None:
                    counts[level] += 1
                P = P + frac * e * forces[level](U)
                if sub:
                    U, P = below(level - 1, U, P, 0.5 * e)
        return U, P

    return below(L - 1, U, P, tau)
