"""Pins of the oracle's HMC molecular dynamics (Section 1 HMC outline, Eq.(molecular_U)/(molecular_P);
Section 3: Omelyan integrator with multiple time scales, Wilson plaquette gauge action).

* The gauge force equals minus the derivative of the plaquette action along U -> exp(i w t^a) U
  (central differences with Richardson extrapolation), and the action vanishes on the unit field
  and is gauge invariant.
* The link update is the exact exponential: it stays in SU(3) and composes additively in time.
* The nested Omelyan integrator is reversible (forward, P -> -P, forward again returns to the
  start), conserves H up to O(e^2) (halving every step size divides Delta H by about 4), counts the
  link updates 2 k0 of the paper's (k0, k1, k2) scheme, and with the EOFA fermion force of a term
  on a tiny lattice still conserves H to O(e^2).
"""
import numpy as np
import pytest

from oracle import eofa, hmc, su3
from oracle.operators import ODWF
from paper_1710_09621_gb300.inputs import gaussian_spinor, omega_zolotarev, random_su3_links

DIMS = (2, 2, 2, 4)


def _momenta(dims, seed):
    Lx, Ly, Lz, Lt = dims
    return np.random.default_rng(seed).standard_normal((4, Lt, Lz, Ly, Lx, 8))


def test_gauge_action_unit_field_and_gauge_invariance():
    Lx, Ly, Lz, Lt = DIMS
    one = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, Lt, Lz, Ly, Lx, 3, 3)).copy()
    assert abs(hmc.gauge_action(one, 6.0)) < 1e-12
    U = random_su3_links(DIMS, 0.5, 1)
    G = random_su3_links(DIMS, 1.0, 2)[0]
    axis = {0: -3, 1: -4, 2: -5, 3: -6}
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[mu] = G @ U[mu] @ np.conj(np.swapaxes(np.roll(G, -1, axis=axis[mu]), -1, -2))
    assert abs(hmc.gauge_action(U, 5.7) - hmc.gauge_action(Ug, 5.7)) < 1e-11 * hmc.gauge_action(U, 5.7)
    # the plaquette average of the unit field is one; S_g = beta * 6 V (1 - <P>)
    V = Lx * Ly * Lz * Lt
    from oracle.wilson import plaquette
    assert abs(hmc.gauge_action(U, 2.0) - 2.0 * 6 * V * (1 - plaquette(U))) < 1e-10


def test_gauge_force_finite_difference():
    U = random_su3_links(DIMS, 0.5, 3)
    beta = 5.9
    F = hmc.gauge_force(U, beta)
    t = su3.generators()
    rng = np.random.default_rng(4)
    for _ in range(8):
        mu = int(rng.integers(4))
        site = tuple(int(rng.integers(n)) for n in U.shape[1:5])
        a = int(rng.integers(8))

        def S_at(w):
            U2 = U.copy()
            U2[(mu,) + site] = su3.expi(w * t[a]) @ U2[(mu,) + site]
            return hmc.gauge_action(U2, beta)
        h = 1e-3
        d1 = (S_at(h) - S_at(-h)) / (2 * h)
        d2 = (S_at(h / 2) - S_at(-h / 2)) / h
        deriv = (4 * d2 - d1) / 3
        assert abs(-deriv - F[(mu,) + site + (a,)]) < 1e-8 * max(1.0, np.abs(F).max())


def test_link_update_special_unitary_and_additive():
    U = random_su3_links(DIMS, 0.5, 5)
    P = _momenta(DIMS, 6)
    U1 = hmc.link_update(U, P, 0.3)
    eye = np.broadcast_to(np.eye(3), U1.shape)
    assert np.allclose(U1 @ np.conj(np.swapaxes(U1, -1, -2)), eye, atol=1e-13)
    assert np.allclose(np.linalg.det(U1), 1.0, atol=1e-12)
    U2 = hmc.link_update(hmc.link_update(U, P, 0.1), P, 0.2)
    assert np.allclose(U1, U2, atol=1e-13)


def _gauge_only(beta):
    return [lambda U: hmc.gauge_force(U, beta)]


def test_integrator_reversible_and_counts():
    U0 = random_su3_links(DIMS, 0.5, 7)
    P0 = _momenta(DIMS, 8)
    beta = 5.5
    forces = [lambda U: hmc.gauge_force(U, beta), lambda U: 0.5 * hmc.gauge_force(U, beta)]
    counts = {}
    U1, P1 = hmc.omelyan_mts(U0, P0, forces, [8, 2], tau=0.5, counts=counts)
    assert counts["links"] == 2 * 8                      # 2 k0 link updates per trajectory
    assert counts[0] == 3 * 8 and counts[1] == 3 * 2    # three momentum updates per Omelyan step
    U2, P2 = hmc.omelyan_mts(U1, -P1, forces, [8, 2], tau=0.5)
    assert np.max(np.abs(U2 - U0)) < 1e-11 and np.max(np.abs(P2 + P0)) < 1e-10


def test_integrator_second_order_energy_error():
    U0 = random_su3_links(DIMS, 0.5, 9)
    P0 = _momenta(DIMS, 10)
    beta = 5.5

    def dH(k):
        U1, P1 = hmc.omelyan_mts(U0, P0, _gauge_only(beta), [k], tau=1.0)
        return (hmc.kinetic(P1) + hmc.gauge_action(U1, beta)) - (hmc.kinetic(P0) + hmc.gauge_action(U0, beta))
    d1, d2 = dH(8), dH(16)
    assert 3.0 < abs(d1 / d2) < 5.5, (d1, d2)


def test_integrator_with_eofa_fermion_force():
    """One EOFA term (Eq.(m1m2_m1m4)) on a second, coarser time scale: Delta H = O(e^2)."""
    dims, Ns = (2, 2, 2, 2), 4
    om = omega_zolotarev(Ns, 0.05, 6.2)
    U0 = random_su3_links(dims, 0.4, 11)
    P0 = _momenta(dims, 12)
    phi = gaussian_spinor(dims, 13)
    term = eofa.Term(-1, 0.1, 0.1, 0.5)
    beta = 5.5

    def S_f(U):
        return eofa.action(ODWF(U, 1.3, om), term, phi, tol=1e-13)[0]

    def F_f(U):
        return eofa.force(ODWF(U, 1.3, om), term, phi, tol=1e-13)[0]

    def dH(k0, k1):
        U1, P1 = hmc.omelyan_mts(U0, P0, [lambda U: hmc.gauge_force(U, beta), F_f], [k0, k1], tau=0.5)
        H1 = hmc.kinetic(P1) + hmc.gauge_action(U1, beta) + S_f(U1)
        return H1 - (hmc.kinetic(P0) + hmc.gauge_action(U0, beta) + S_f(U0))
    d1, d2 = dH(8, 4), dH(16, 8)
    assert 3.0 < abs(d1 / d2) < 5.5, (d1, d2)
