"""Full-size GPU checks of the larger workloads, through the C ABI.

* 24^3 x 48, Ns = 16: EOFA terms of one mass preconditioner (light pair (0.01, 0.1), heavy pair
  (0.1, 1.0), Eq.(old_MP)): heat-bath, action and force with FP32 inner solves, their error against
  FP64-accurate values, and D_T parity at sampled sites.
* 24^3 x 48, Ns = 16: 8 right-hand sides with distinct (m1, m2) on one gauge field in one batch, and
  an uneven batch of 8^4, 12^4 and 16^3 x 32 lattices in one launch per step.
* 32^3 x 64, Ns = 16, m = 0.005: the learned preconditioner trained on pairs from one gauge field and
  used on a held-out one.

At these sizes the oracle cannot solve; the checks are the properties that hold at any size (the
heat-bath identity phi^dag X phi = eta^dag eta, FP64 true residuals recomputed by the library), the
oracle's D_T at sampled sites, and the oracle's full residual where the lattice is small (8^4).
"""
import numpy as np
import pytest

from oracle import eofa as oeofa
from oracle.operators import ODWF as OracleODWF
from oracle.operators import dt_at_sites
from paper_1710_09621_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NS, M0, EPS = 16, 1.3, 0.3
D24 = (24, 24, 24, 48)


@pytest.fixture(scope="module")
def lib():
    from paper_1710_09621_gb300 import build
    build.build()
    from paper_1710_09621_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def lat24(lib):
    om = inputs.omega_zolotarev(NS, 0.05, 6.2)
    U = inputs.random_su3_links(D24, EPS, inputs.seed_for(2, 0))
    lat = lib.ODWF(D24, NS, M0, om)
    lat.set_gauge(torch.from_numpy(U).cuda())
    yield lat, U, om
    lat.close()


def _sites(rng, dims, n):
    Lx, Ly, Lz, Lt = dims
    out = [(int(rng.integers(NS)), int(rng.integers(Lt)), int(rng.integers(Lz)), int(rng.integers(Ly)),
            int(rng.integers(Lx))) for _ in range(n)]
    return out + [(0, 0, 0, 0, 0), (NS - 1, Lt - 1, Lz - 1, Ly - 1, Lx - 1)]


def test_config2_dt_sampled_parity(lib, lat24):
    lat, U, om = lat24
    op = OracleODWF(U, M0, om)
    psi = inputs.gaussian_spinor5(D24, NS, inputs.seed_for(2, 1))
    sites = _sites(np.random.default_rng(2), D24, 48)
    for prec, tol in (("double", 1e-12), ("single", 2e-6)):
        got = lat.apply(torch.from_numpy(psi).cuda(), 0.01, 0.1, op="dt", prec=prec).cpu().numpy()
        ref = dt_at_sites(op, psi, 0.01, 0.1, sites)
        g = np.array([got[s] for s in sites])
        assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < tol


def test_config2_mp_terms_mixed_precision(lib, lat24):
    """Old-MP terms with mh = 0.1: phi = X^{-1/2} eta with FP32 inner solves satisfies
    phi^dag X phi = |P eta|^2; action and force at tol 1e-10 agree with FP64-accurate values
    (tol 1e-12) to the stated bounds."""
    lat, U, om = lat24
    terms = lib.mp_terms(lib.MP_OLD, 0.01, [0.1], 1.0)
    assert [(t.chirality, t.m3, t.m4, t.m_den) for t in terms][:2] == [(-1, 0.01, 0.01, 0.1), (+1, 0.01, 0.1, 0.1)]
    eta = inputs.gaussian_spinor(D24, inputs.seed_for(2, 2))
    o10 = lib.solve_opts(tol=1e-10, prec="single", delta=0.01)
    o12 = lib.solve_opts(tol=1e-12, prec="single", delta=0.01)
    for t in terms[:2]:
        phi, hb = lat.heatbath(t, torch.from_numpy(eta).cuda(), opts=o10)
        P = oeofa.projector(t.chirality)
        peta = np.einsum("ij,...jc->...ic", P, eta)
        n2 = np.vdot(peta, peta).real
        S, st = lat.action(t, phi, opts=o10)
        S12, _ = lat.action(t, phi, opts=o12)
        assert abs(S / n2 - 1) < 1e-8, (t, S, n2)
        assert abs(S - S12) < 1e-9 * abs(S12)
        F, _ = lat.force(t, phi, opts=o10)
        F12, _ = lat.force(t, phi, opts=o12)
        # a relative residual of 1e-10 bounds the relative error of chi = H_T^{-1} Omega phi by
        # kappa(H_T) 1e-10; kappa ~ 2/m = 200 here, and the force is bilinear in chi: <= ~4e-8
        err = (torch.linalg.norm(F - F12) / torch.linalg.norm(F12)).item()
        assert err < 4e-8, err
        print(f"\nterm {t}: poles {hb['n_poles']}, |S/|P eta|^2 - 1| = {abs(S / n2 - 1):.2e}, "
              f"action error vs FP64-accurate {abs(S - S12) / abs(S12):.2e}, force error {err:.2e}")


def test_config3_eight_rhs_batch(lib, lat24):
    lat, U, om = lat24
    m12 = [(0.01, 0.01), (0.01, 0.1), (0.1, 0.1), (0.1, 1.0), (1.0, 0.1), (0.3, 0.05), (0.05, 0.3), (0.02, 0.5)]
    bs = [inputs.gaussian_spinor5(D24, NS, inputs.seed_for(3, 100 + i)) for i in range(len(m12))]
    xs, stats = lat.solve_batch([torch.from_numpy(b).cuda() for b in bs], m12,
                                opts=lib.solve_opts(tol=1e-10, prec="single", delta=0.01))
    assert all(st["true_residual"] <= 1e-10 for st in stats)
    # the oracle's residual b' - D_T x at sampled sites for two of the systems
    op = OracleODWF(U, M0, om)
    sites = _sites(np.random.default_rng(3), D24, 64)
    g5 = np.diag([1.0, 1, -1, -1])
    for i in (0, 3):
        b, x = bs[i], xs[i].cpu().numpy()
        bprime = np.einsum("ij,...jc->...ic", g5, b[::-1])
        r = np.array([bprime[s] for s in sites]) - dt_at_sites(op, x, *m12[i], sites)
        assert np.max(np.linalg.norm(r.reshape(len(sites), -1), axis=1)) <= 1e-10 * np.linalg.norm(bprime)


def test_config3_uneven_batch(lib):
    om = inputs.omega_zolotarev(NS, 0.05, 6.2)
    dims_list = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 32)]
    lats, bs, Us = [], [], []
    for k, dd in enumerate(dims_list):
        U = inputs.random_su3_links(dd, EPS, inputs.seed_for(3, k))
        lat = lib.ODWF(dd, NS, M0, om)
        lat.set_gauge(torch.from_numpy(U).cuda())
        lats.append(lat)
        Us.append(U)
        bs.append(inputs.gaussian_spinor5(dd, NS, inputs.seed_for(3, 10 + k)))
    xs, stats = lib.solve_multi(lats, [torch.from_numpy(b).cuda() for b in bs], [(0.01, 0.01)] * 3,
                                opts=lib.solve_opts(tol=1e-10, prec="single", delta=0.01))
    assert all(st["true_residual"] <= 1e-10 for st in stats)
    op = OracleODWF(Us[0], M0, om)  # 8^4: the oracle's whole-lattice residual
    res = np.linalg.norm(bs[0] - op.ht(xs[0].cpu().numpy(), 0.01, 0.01)) / np.linalg.norm(bs[0])
    assert res <= 1.05e-10
    for lat in lats:
        lat.close()


def test_config4_learned_preconditioner_held_out(lib):
    """32^3 x 64, m = 0.005: weights trained on pairs from one gauge field precondition the solve on
    a held-out gauge field; FP64 true residual 1e-10 and fewer iterations than plain CGNE."""
    D32, m = (32, 32, 32, 64), 0.005
    om = inputs.omega_zolotarev(NS, 0.05, 6.2)
    lat_tr = lib.ODWF(D32, NS, M0, om)
    lat_tr.set_gauge(torch.from_numpy(inputs.random_su3_links(D32, EPS, inputs.seed_for(4, 0))).cuda())
    net_tr = lib.Net(lat_tr, channels=2)
    rs = [torch.from_numpy(inputs.gaussian_spinor5(D32, NS, inputs.seed_for(4, 100 + i))).cuda() for i in range(2)]
    net_tr.set_pairs(rs, m, m, tol=1e-8)
    del rs
    losses = net_tr.train(20, 2e-3)
    assert losses[-1] < losses[0]
    W = net_tr.get_weights()
    net_tr.close()
    lat_tr.close()
    torch.cuda.empty_cache()

    lat = lib.ODWF(D32, NS, M0, om)
    lat.set_gauge(torch.from_numpy(inputs.random_su3_links(D32, EPS, inputs.seed_for(4, 1))).cuda())
    net = lib.Net(lat, channels=2)
    net.set_weights(W)
    b = torch.from_numpy(inputs.gaussian_spinor5(D32, NS, inputs.seed_for(4, 200))).cuda()
    _, stl = net.solve(b, m, m, opts=lib.solve_opts(tol=1e-10, prec="single", delta=1e-3))
    _, stc = lat.solve(b, m, m, opts=lib.solve_opts(tol=1e-10, prec="single", delta=0.01))
    assert stl["true_residual"] <= 1e-10 and stc["true_residual"] <= 1e-10
    assert stl["iters"] < stc["iters"]
    print(f"\n32^3x64 m=0.005 held-out field: learned {stl['iters']} iterations ({stl['seconds']:.2f} s), "
          f"plain CGNE {stc['iters']} ({stc['seconds']:.2f} s); loss {losses[0]:.3e} -> {losses[-1]:.3e}")
    net.close()
    lat.close()
