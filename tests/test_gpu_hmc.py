"""HMC molecular dynamics on the GPU against the FP64 oracle (Section 1 HMC outline,
Eq.(molecular_U)/(molecular_P); Section 3: Omelyan integrator with multiple time scales and the Wilson
plaquette gauge action).

* Gauge action, gauge force, link update and kinetic energy agree with the oracle (FP64, 1e-12).
* A whole trajectory (gauge force on level 0, EOFA terms of Eq.(Nf1_newMP) on levels 1 and 2) agrees
  with the oracle's nested Omelyan integrator run on the same U, P and pseudofermions.
* The GPU trajectory is reversible, its Delta H falls by about 4 when every step size halves, and it
  counts 2 k0 link updates and 2 k_l + 1 force evaluations per level.
"""
import numpy as np
import pytest

from oracle import eofa as oeofa
from oracle import hmc as ohmc
from oracle.operators import ODWF as OracleODWF
from paper_1710_09621_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS, NS, M0, BETA = (4, 4, 4, 4), 8, 1.3, 5.8


@pytest.fixture(scope="module")
def lib():
    from paper_1710_09621_gb300 import build
    build.build()
    from paper_1710_09621_gb300 import binding
    return binding


def _setup(lib, eps=0.4, seed=41, dims=DIMS, ns=NS):
    om = inputs.omega_zolotarev(ns, 0.05, 6.2)
    U = inputs.random_su3_links(dims, eps, seed)
    lat = lib.ODWF(dims, ns, M0, om)
    Ud = torch.from_numpy(U).cuda()
    lat.set_gauge(Ud)
    return lat, U, Ud, om


def _momenta(seed, dims=DIMS):
    Lx, Ly, Lz, Lt = dims
    return np.random.default_rng(seed).standard_normal((4, Lt, Lz, Ly, Lx, 8))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_gauge_pieces_match_oracle(lib):
    lat, U, Ud, om = _setup(lib)
    assert abs(lat.gauge_action(Ud, BETA) - ohmc.gauge_action(U, BETA)) < 1e-12 * ohmc.gauge_action(U, BETA)
    assert _rel(lat.gauge_force(Ud, BETA).cpu().numpy(), ohmc.gauge_force(U, BETA)) < 1e-12
    P = _momenta(1)
    Pd = torch.from_numpy(P).cuda()
    assert abs(lat.kinetic(Pd) - ohmc.kinetic(P)) < 1e-12 * ohmc.kinetic(P)
    U2 = Ud.clone()
    lat.link_update(U2, Pd, 0.07)
    assert np.max(np.abs(U2.cpu().numpy() - ohmc.link_update(U, P, 0.07))) < 1e-13
    F = torch.from_numpy(ohmc.gauge_force(U, BETA)).cuda()
    lat.momentum_update(Pd, F, 0.3)
    assert np.max(np.abs(Pd.cpu().numpy() - (P + 0.3 * ohmc.gauge_force(U, BETA)))) < 1e-13
    # after a link update the operator acts on the new links
    lat.close()


def _terms(lib):
    terms = oeofa.new_mp(0.1, 0.3, 1.0)   # Eq.(new_MP) with heavier masses than the paper's, for a fast test
    specs = [lib.TermSpec(t.chirality, t.m3, t.m4, t.m_den) for t in terms]
    return terms, specs


def test_trajectory_matches_oracle(lib):
    # a smaller lattice than the other tests: the oracle integrates with numpy solves
    dims, ns = (4, 2, 2, 4), 4
    lat, U, Ud, om = _setup(lib, dims=dims, ns=ns)
    P = _momenta(2, dims)
    terms, specs = _terms(lib)
    phis = [inputs.gaussian_spinor(dims, 50 + i) for i in range(len(terms))]
    # the paper's assignment (Section 3): the heaviest factor on level 1, the two lighter ones on level 2
    levels, steps, tau = [2, 2, 1], [4, 2, 1], 0.25
    Pd = torch.from_numpy(P).cuda()
    Ug = Ud.clone()
    st = lat.md(Ug, Pd, BETA, specs, [torch.from_numpy(p).cuda() for p in phis], levels, steps, tau=tau,
                opts=lib.solve_opts(tol=1e-12))
    op = lambda Ux: OracleODWF(Ux, M0, om)
    f_lvl = [lambda Ux: ohmc.gauge_force(Ux, BETA),
             lambda Ux: oeofa.force(op(Ux), terms[2], phis[2], tol=1e-13)[0],
             lambda Ux: sum(oeofa.force(op(Ux), terms[i], phis[i], tol=1e-13)[0] for i in (0, 1))]
    Uo, Po = ohmc.omelyan_mts(U, P, f_lvl, steps, tau=tau)
    assert np.max(np.abs(Ug.cpu().numpy() - Uo)) < 1e-10
    assert _rel(Pd.cpu().numpy(), Po) < 1e-9

    def H(Ux, Px):
        return (ohmc.kinetic(Px) + ohmc.gauge_action(Ux, BETA)
                + sum(oeofa.action(op(Ux), t, p, tol=1e-13)[0] for t, p in zip(terms, phis)))
    dH_o = H(Uo, Po) - H(U, P)
    assert abs(st["dH"] - dH_o) < 1e-8 * max(1.0, abs(dH_o)), (st["dH"], dH_o)
    assert st["link_updates"] == 2 * steps[0]
    assert st["force_evals"][:3] == [2 * k + 1 for k in steps]
    lat.close()


def test_trajectory_reversible_and_second_order(lib):
    lat, U, Ud, om = _setup(lib, seed=43)
    P = _momenta(3)
    terms, specs = _terms(lib)
    phis = [torch.from_numpy(inputs.gaussian_spinor(DIMS, 60 + i)).cuda() for i in range(len(terms))]
    levels, tau = [2, 2, 1], 0.5
    o = lib.solve_opts(tol=1e-12)

    def run(steps, Ustart, Pstart):
        Ux, Px = Ustart.clone(), Pstart.clone()
        st = lat.md(Ux, Px, BETA, specs, phis, levels, steps, tau=tau, opts=o)
        return Ux, Px, st

    U0, P0 = torch.from_numpy(U).cuda(), torch.from_numpy(P).cuda()
    U1, P1, st1 = run([8, 4, 2], U0, P0)
    U2, P2, _ = run([8, 4, 2], U1, -P1)
    assert torch.max(torch.abs(U2 - U0)).item() < 1e-9
    assert torch.max(torch.abs(P2 + P0)).item() < 1e-8
    _, _, st2 = run([16, 8, 4], U0, P0)
    assert 3.0 < abs(st1["dH"] / st2["dH"]) < 5.5, (st1["dH"], st2["dH"])
    lat.close()
