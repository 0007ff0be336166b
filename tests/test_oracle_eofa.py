"""Brute-force pins of the oracle's EOFA terms on a 2^4 x Ns=4 lattice.

The determinant identities Eq.(m1m2_m1m4), Eq.(m1m2_m3m2), Eq.(det_minus), Eq.(det_plus),
Eq.(EOFA_noMP_D), Eq.(noMP), Eq.(noMP_P), Eq.(old_MP), Eq.(new_MP) and the cascades
Eq.(old_MP_N), Eq.(new_MP_N) are checked with dense log-determinants; the solver, action, force
and heat-bath of the oracle are checked against dense linear algebra and finite differences.
"""
import numpy as np
import pytest

from oracle import eofa, fifth, rational, solver, su3
from oracle.operators import ODWF
from oracle.wilson import GAMMA5, spin_mul
from paper_1710_09621_gb300.inputs import (gaussian_spinor, gaussian_spinor5, omega_shamir,
                                           omega_zolotarev, random_su3_links)

from oracle_dense import DenseEOFA

DIMS = (2, 2, 2, 2)


@pytest.fixture(scope="module", params=["one", "zolo"])
def dense_op(request):
    om = omega_shamir(4) if request.param == "one" else omega_zolotarev(4, 0.05, 6.2)
    op = ODWF(random_su3_links(DIMS, 0.4, 21), 1.3, om)
    return op, DenseEOFA(op)


def _logdet_x(d, term):
    s, ld = np.linalg.slogdet(d.term_x(term))
    return ld + np.log(s)


MASS_SETS = [(0.05, 0.1, 1.0), (0.01, 0.1, 1.0)]


@pytest.mark.parametrize("masses", MASS_SETS)
def test_chiral_term_determinants(dense_op, masses):
    """Eq.(m1m2_m1m4) and Eq.(m1m2_m3m2): the Gaussian integral of each term equals the ratio."""
    op, d = dense_op
    m, mh, M = masses
    cases = [((m, m), (m, mh)), ((m, mh), (M, mh)), ((mh, m), (mh, M)), ((m, M), (M, M))]
    for num, den in cases:
        term = eofa.term_from_ratio(num, den)
        lhs = d.logdet_dt(*num) - d.logdet_dt(*den)   # log of (m3,m4)/(m1,m2)
        rhs = -_logdet_x(d, term)                     # log of 1/det X
        assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs)), (num, den, lhs, rhs)


@pytest.mark.parametrize("masses", MASS_SETS)
def test_mp_factorisations_telescope(dense_op, masses):
    """Eq.(noMP), Eq.(noMP_P), Eq.(old_MP), Eq.(new_MP) and the cascades give det D_T(m)/det D_T(M)."""
    op, d = dense_op
    m, mh, M = masses
    target = d.logdet_dt(m, m) - d.logdet_dt(M, M)
    schemes = {
        "noMP": eofa.no_mp(m, M),
        "noMP_P": [eofa.term_from_ratio((m, m), (M, m)), eofa.term_from_ratio((M, m), (M, M))],
        "oldMP": eofa.old_mp(m, mh, M),
        "newMP": eofa.new_mp(m, mh, M),
        "oldMP_N2": eofa.old_mp_cascade(m, [mh, 0.5], M),
        "newMP_N2": eofa.new_mp_cascade(m, [mh, 0.5], M),
        "newMP_N3": eofa.new_mp_cascade(m, [mh, 0.3, 0.5], M),
    }
    chir = {"noMP": [-1, 1], "noMP_P": [1, -1], "oldMP": [-1, 1, -1, 1], "newMP": [-1, 1, -1]}
    for name, terms in schemes.items():
        total = sum(-_logdet_x(d, t) for t in terms)
        assert abs(total - target) < 1e-10 * max(1.0, abs(target)), name
        if name in chir:
            assert [t.chirality for t in terms] == chir[name]
    # term counts: N + 2 for the new cascade, 2N + 2 for the old one (concluding remarks)
    assert len(schemes["newMP_N3"]) == 5 and len(schemes["oldMP_N2"]) == 6


def test_det_minus_det_plus(dense_op):
    """Eq.(det_minus) * Eq.(det_plus) = Eq.(EOFA_noMP_D) with m_j = 1 (Eq.(H))."""
    op, d = dense_op
    m = 0.05
    t_minus = eofa.Term(-1, m, m, 1.0)
    t_plus = eofa.Term(+1, m, 1.0, 1.0)
    assert abs((d.logdet_dt(m, m) - d.logdet_dt(m, 1.0)) + _logdet_x(d, t_minus)) < 1e-10 * 100
    assert abs((d.logdet_dt(m, 1.0) - d.logdet_dt(1.0, 1.0)) + _logdet_x(d, t_plus)) < 1e-10 * 100


def test_terms_positive_definite_and_bounded(dense_op):
    """X is Hermitian positive definite (Section 1); its spectrum lies in
    [(1 + m_ref)/(1 + m_den), 1], the interval the heat-bath approximation is built on."""
    op, d = dense_op
    for terms in (eofa.new_mp(0.01, 0.1, 1.0), eofa.old_mp(0.05, 0.1, 1.0)):
        for t in terms:
            X = d.term_x(t)
            assert np.max(np.abs(X - X.conj().T)) < 1e-13
            ev = np.linalg.eigvalsh(X)
            mref = t.m4 if t.chirality < 0 else t.m3
            assert ev.min() > (1 + mref) / (1 + t.m_den) * (1 - 1e-12)
            assert ev.max() < 1.0


def test_woodbury_inverse(dense_op):
    """X_-^{-1} = 1 + k Omega^T H_T(m3, m_den)^{-1} Omega; X_+^{-1} = 1 - k Omega^T H_T(m_den, m4)^{-1} Omega."""
    op, d = dense_op
    for t in (eofa.Term(-1, 0.05, 0.05, 0.1), eofa.Term(+1, 0.05, 0.1, 1.0)):
        X = d.term_x(t)
        Om = d.omega_op(t.chirality)
        H2 = d.ht(t.m3, t.m_den) if t.chirality < 0 else d.ht(t.m_den, t.m4)
        sgn = 1.0 if t.chirality < 0 else -1.0
        Xi = np.eye(d.n4) + sgn * t.k * Om.T @ np.linalg.inv(H2) @ Om
        idx = d.chiral_index(t.chirality)
        assert np.allclose(np.linalg.inv(X), Xi[np.ix_(idx, idx)], atol=1e-12)


@pytest.mark.parametrize("m12", [(0.05, 0.05), (0.01, 1.0), (1.0, 0.1)])
def test_solver_matches_dense(dense_op, m12):
    op, d = dense_op
    b = gaussian_spinor5(op.dims, op.Ns, 3)
    x, info = solver.solve_ht(op, b, *m12, tol=1e-12)
    xd = np.linalg.solve(d.ht(*m12), b.reshape(-1)).reshape(b.shape)
    assert info["true_residual"] <= 1e-12 and info["true_residual_ht"] <= 1e-11
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9


def test_action_matches_dense(dense_op):
    op, d = dense_op
    phi = gaussian_spinor(op.dims, 4)
    for t in eofa.new_mp(0.05, 0.1, 1.0):
        S, _ = eofa.action(op, t, phi, tol=1e-13)
        idx = d.chiral_index(t.chirality)
        v = phi.reshape(-1)[idx]
        Sd = np.vdot(v, d.term_x(t) @ v).real
        assert abs(S - Sd) < 1e-11 * abs(Sd)


def test_action_gauge_invariant():
    om = omega_zolotarev(4, 0.05, 6.2)
    dims = (2, 2, 2, 4)
    U = random_su3_links(dims, 0.4, 2)
    G = random_su3_links(dims, 1.0, 8)[0]
    axis = {0: -3, 1: -4, 2: -5, 3: -6}
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[mu] = G @ U[mu] @ np.conj(np.swapaxes(np.roll(G, -1, axis=axis[mu]), -1, -2))
    phi = gaussian_spinor(dims, 1)
    Gphi = np.einsum("...ab,...ib->...ia", G, phi)
    t = eofa.Term(+1, 0.05, 0.1, 1.0)
    S1, _ = eofa.action(ODWF(U, 1.3, om), t, phi, tol=1e-13)
    S2, _ = eofa.action(ODWF(Ug, 1.3, om), t, Gphi, tol=1e-13)
    assert abs(S1 - S2) < 1e-11 * abs(S1)


@pytest.mark.parametrize("term", [eofa.Term(-1, 0.05, 0.05, 0.1), eofa.Term(+1, 0.05, 0.1, 1.0)])
def test_force_finite_difference(term):
    """F^a_mu(x) = -dS/dw^a for U_mu(x) -> exp(i w^a t^a) U_mu(x): central differences + Richardson."""
    om = omega_zolotarev(4, 0.05, 6.2)
    dims = (2, 2, 2, 4)
    U = random_su3_links(dims, 0.4, 6)
    phi = gaussian_spinor(dims, 7)
    op = ODWF(U, 1.3, om)
    F, _ = eofa.force(op, term, phi, tol=1e-14)
    ta = su3.generators()
    rng = np.random.default_rng(1)
    Lx, Ly, Lz, Lt = dims

    def S_at(mu, site, a, w):
        U2 = U.copy()
        t, z, y, x = site
        e, v = np.linalg.eigh(ta[a])
        rot = v @ np.diag(np.exp(1j * w * e)) @ v.conj().T
        U2[mu, t, z, y, x] = rot @ U2[mu, t, z, y, x]
        return eofa.action(ODWF(U2, 1.3, om), term, phi, tol=1e-14)[0]

    for _ in range(5):
        mu = int(rng.integers(4))
        site = (int(rng.integers(Lt)), int(rng.integers(Lz)), int(rng.integers(Ly)), int(rng.integers(Lx)))
        a = int(rng.integers(8))
        h = 1e-3
        d1 = (S_at(mu, site, a, h) - S_at(mu, site, a, -h)) / (2 * h)
        d2 = (S_at(mu, site, a, h / 2) - S_at(mu, site, a, -h / 2)) / h
        deriv = (4 * d2 - d1) / 3
        fa = F[(mu,) + site + (a,)]
        assert abs(-deriv - fa) < 1e-7 * max(1.0, np.abs(F).max()), (mu, site, a, -deriv, fa)


def test_force_magnitude_formula():
    F = np.ones((4, 2, 2, 2, 4, 8))
    V = 2 * 2 * 2 * 4
    assert np.isclose(eofa.force_magnitude(F), np.sqrt(4 * V * 8) / (4 * V))


@pytest.mark.parametrize("term", [eofa.Term(-1, 0.05, 0.05, 0.1), eofa.Term(+1, 0.05, 0.1, 1.0),
                                  eofa.Term(-1, 1.0, 0.1, 1.0)])
def test_heatbath(dense_op, term):
    """phi = X^{-1/2} eta: phi^dag X phi = eta^dag eta, and phi matches the dense X^{-1/2} eta."""
    op, d = dense_op
    mref = term.m4 if term.chirality < 0 else term.m3
    rat = rational.inv_sqrt_for_error(0.98 * (1 + mref) / (1 + term.m_den), 1.0, 1e-12)
    eta = gaussian_spinor(op.dims, 12)
    phi, _ = eofa.heatbath(op, term, eta, rat, tol=1e-13)
    idx = d.chiral_index(term.chirality)
    X = d.term_x(term)
    e = eta.reshape(-1)[idx]
    p = phi.reshape(-1)[idx]
    assert abs(np.vdot(p, X @ p).real / np.vdot(e, e).real - 1.0) < 1e-10
    w, v = np.linalg.eigh(X)
    pd = v @ ((v.conj().T @ e) / np.sqrt(w))
    assert np.linalg.norm(p - pd) / np.linalg.norm(pd) < 1e-10
    # the other chirality stays zero
    assert np.max(np.abs(np.delete(phi.reshape(-1), idx))) == 0.0


def test_pole_mass_inverts_k():
    t = eofa.Term(-1, 0.05, 0.05, 0.1)
    for kp in (0.01, t.k, 0.5 * t.k):
        assert np.isclose(fifth.k_eofa(eofa.pole_mass(t, kp), t.m4), kp, rtol=1e-13)


@pytest.mark.parametrize("m", [0.05, 0.3])
def test_effective_overlap_operator(dense_op, m):
    """Reading of D_T (c = 1, d = 0 optimal DWF): integrating out the fifth dimension leaves the
    overlap-type operator D_eff(m) = m + (1 - m)/2 (1 + gamma_5 S(H_w)), H_w = gamma_5 D_w(-m0),
    S(H) = (1 - prod_s T_s)/(1 + prod_s T_s), T_s = (1 - omega_s H)/(1 + omega_s H) (the rational
    sign approximation the omega_s encode), so that
        det D_T(m) / det D_T(1) = det D_eff(m) ((1 + m)/2)^{-12 V},
    the last factor being det(1 + L(m)) / det(1 + L(1)) per 4D component (even Ns), which Eq.(detDodwf)
    cancels between D_odwf and D_T. Checked on the fixture's gauge field and a second one."""
    op, d = dense_op
    fields = [d, DenseEOFA(ODWF(random_su3_links(DIMS, 0.4, 22), op.m0, op.omega))]
    for dd in fields:
        Hw = dd.G5 @ dd.Dw
        lam, V = np.linalg.eigh(0.5 * (Hw + Hw.conj().T))
        t = np.ones_like(lam)
        for w in dd.op.omega:
            t = t * (1.0 - w * lam) / (1.0 + w * lam)
        S = (V * ((1.0 - t) / (1.0 + t))) @ V.conj().T
        I4 = np.eye(dd.n4)
        Deff = m * I4 + 0.5 * (1.0 - m) * (I4 + dd.G5 @ S)
        s, ld_eff = np.linalg.slogdet(Deff)
        lhs = dd.logdet_dt(m, m) - dd.logdet_dt(1.0, 1.0)
        rhs = ld_eff + np.log(s) - dd.n4 * np.log((1.0 + m) / 2.0)
        assert abs(lhs - rhs) < 1e-10 * abs(lhs), (lhs, rhs)
