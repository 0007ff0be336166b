"""Pins of the oracle's learned preconditioner (network forward, adjoint, gradients)."""
import numpy as np
import pytest

from oracle import learned, solver
from oracle.operators import ODWF
from paper_1710_09621_gb300.inputs import gaussian_spinor5, omega_zolotarev, random_su3_links

DIMS, NS = (4, 2, 2, 4), 4


@pytest.fixture(scope="module")
def setup():
    op = ODWF(random_su3_links(DIMS, 0.4, 3), 1.3, omega_zolotarev(NS, 0.05, 6.2))
    sch = solver.Schur(op, 0.05, 0.1)
    return op, sch


def _rand_weights(C, seed):
    rng = np.random.default_rng(seed)
    z = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    return learned.Weights(z(4, 4), 0.3 * z(C, 8, 4, 4), 0.3 * z(C, 8, 4, 4))


def test_neumann_initialisation(setup):
    """Initial weights give A^{-1} r + 1/4 A^{-1} H_eo A^{-1} H_oe A^{-1} r exactly."""
    op, sch = setup
    M = learned.LearnedPreconditioner(sch, learned.neumann_weights(C=2))
    r = gaussian_spinor5(DIMS, NS, 1) * sch.even
    u = sch.Ainv(r)
    ref = u + 0.25 * sch.Ainv(sch.hop_to(sch.Ainv(sch.hop_to(u, sch.odd)), sch.even))
    assert np.linalg.norm(M.forward(r) - ref) < 1e-13 * np.linalg.norm(ref)


def test_adjoint(setup):
    op, sch = setup
    M = learned.LearnedPreconditioner(sch, _rand_weights(2, 5))
    a = gaussian_spinor5(DIMS, NS, 2) * sch.even
    b = gaussian_spinor5(DIMS, NS, 3) * sch.even
    lhs, rhs = np.vdot(a, M.forward(b)), np.vdot(M.adjoint(a), b)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_gauge_equivariance():
    om = omega_zolotarev(NS, 0.05, 6.2)
    U = random_su3_links(DIMS, 0.4, 7)
    G = random_su3_links(DIMS, 1.0, 8)[0]
    axis = {0: -3, 1: -4, 2: -5, 3: -6}
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[mu] = G @ U[mu] @ np.conj(np.swapaxes(np.roll(G, -1, axis=axis[mu]), -1, -2))
    W = _rand_weights(2, 9)
    M1 = learned.LearnedPreconditioner(solver.Schur(ODWF(U, 1.3, om), 0.05, 0.1), W)
    M2 = learned.LearnedPreconditioner(solver.Schur(ODWF(Ug, 1.3, om), 0.05, 0.1), W)
    r = gaussian_spinor5(DIMS, NS, 4) * M1.sch.even
    Gm = lambda f: np.einsum("...ab,...ib->...ia", G, f)
    assert np.linalg.norm(M2.forward(Gm(r)) - Gm(M1.forward(r))) < 1e-13 * np.linalg.norm(r)


def test_gradient_finite_difference(setup):
    """dL/dRe W = 2 Re G, dL/dIm W = 2 Im G for the Wirtinger gradient G = dL/dconj(W)."""
    op, sch = setup
    W = _rand_weights(2, 11)
    rs = [gaussian_spinor5(DIMS, NS, 20 + i) * sch.even for i in range(2)]
    es = [gaussian_spinor5(DIMS, NS, 30 + i) * sch.even for i in range(2)]
    L, G = learned.LearnedPreconditioner(sch, W).loss_and_grad(rs, es)
    flat, gflat = W.flat(), G.flat()
    rng = np.random.default_rng(0)
    h = 1e-6

    def L_at(v):
        return learned.LearnedPreconditioner(sch, learned.Weights.from_flat(v, 2)).loss_and_grad(rs, es)[0]

    for idx in rng.choice(len(flat), 8, replace=False):
        for part, unit in (("re", 1.0), ("im", 1j)):
            vp, vm = flat.copy(), flat.copy()
            vp[idx] += h * unit
            vm[idx] -= h * unit
            fd = (L_at(vp) - L_at(vm)) / (2 * h)
            an = 2 * (gflat[idx].real if part == "re" else gflat[idx].imag)
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (idx, part, fd, an)


def test_training_step_reduces_loss(setup):
    """Pairs (r, e = S^{-1} r) from the solver; gradient steps from the Neumann start lower the loss."""
    op, sch = setup
    rs, es = [], []
    for i in range(3):
        r = gaussian_spinor5(DIMS, NS, 40 + i) * sch.even
        e, _, _ = solver.cgne(sch.S, sch.S_dag, r, 1e-12 * np.linalg.norm(r), 10000)
        rs.append(r)
        es.append(e)
    W = learned.neumann_weights(C=2, noise=1e-3)
    L0, G = learned.LearnedPreconditioner(sch, W).loss_and_grad(rs, es)
    flat = W.flat()
    g = G.flat()
    # steepest descent with backtracking: the loss must drop by at least 1 %
    t = 0.5 * L0 / np.vdot(g, g).real
    best = L0
    for _ in range(30):
        L1, _ = learned.LearnedPreconditioner(sch, learned.Weights.from_flat(flat - t * g, 2)).loss_and_grad(rs, es)
        best = min(best, L1)
        if L1 < 0.99 * L0:
            break
        t *= 0.5
    assert best < 0.99 * L0, (L0, best)


def test_residual_loss_gradient_finite_difference(setup):
    """Residual loss L = sum |S M r - r|^2/|r|^2: Wirtinger gradient vs central differences, and
    with the Neumann weights L equals the closed form |(1/4 A^{-1} H A^{-1} H)^2 r'|-type remainder
    computed independently as |S M r - r|^2 from the Schur pieces."""
    op, sch = setup
    W = _rand_weights(2, 13)
    rs = [gaussian_spinor5(DIMS, NS, 50 + i) * sch.even for i in range(2)]
    L, G = learned.LearnedPreconditioner(sch, W).residual_loss_and_grad(rs)
    flat, gflat = W.flat(), G.flat()
    rng = np.random.default_rng(1)
    h = 1e-6

    def L_at(v):
        return learned.LearnedPreconditioner(sch, learned.Weights.from_flat(v, 2)).residual_loss_and_grad(rs)[0]

    for idx in rng.choice(len(flat), 8, replace=False):
        for part, unit in (("re", 1.0), ("im", 1j)):
            vp, vm = flat.copy(), flat.copy()
            vp[idx] += h * unit
            vm[idx] -= h * unit
            fd = (L_at(vp) - L_at(vm)) / (2 * h)
            an = 2 * (gflat[idx].real if part == "re" else gflat[idx].imag)
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (idx, part, fd, an)
    # Neumann weights: M = (1 + K) A^{-1} with K = 1/4 A^{-1} H A^{-1} H, S = A (1 - K), so
    # S M - 1 = A (1 - K)(1 + K) A^{-1} - 1 = -A K^2 A^{-1}
    Mn = learned.LearnedPreconditioner(sch, learned.neumann_weights(C=2))
    Ln, _ = Mn.residual_loss_and_grad(rs)
    K = lambda v: 0.25 * sch.Ainv(sch.hop_to(sch.Ainv(sch.hop_to(v, sch.odd)), sch.even))
    ref = sum(np.linalg.norm(sch.A(K(K(sch.Ainv(r))))) ** 2 / np.linalg.norm(r) ** 2 for r in rs)
    assert abs(Ln - ref) < 1e-12 * ref
