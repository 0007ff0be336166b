"""GPU learned preconditioner against the oracle: inference, adjoint, loss/gradients, training, solve.

The channel mixing runs on the tensor cores with BF16 operands and FP32 accumulation: each layer
rounds its inputs and weights to 8 significant bits (relative 2^-9), so the network output agrees
with the FP64 oracle to a few 1e-3 relative L2; the tests use 2e-2 (outputs) and 5e-2 (weight
gradients, which contract two BF16 layers). The preconditioned solve itself is exact: its FP64 true
residual must meet 1e-10 like every other solve.
"""
import numpy as np
import pytest

from oracle import learned, solver
from oracle.operators import ODWF as OracleODWF
from paper_1710_09621_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS, NS, M1, M2 = (4, 4, 4, 4), 8, 0.05, 0.1


@pytest.fixture(scope="module")
def env():
    from paper_1710_09621_gb300 import build
    build.build()
    from paper_1710_09621_gb300 import binding
    om = inputs.omega_zolotarev(NS, 0.05, 6.2)
    U = inputs.random_su3_links(DIMS, 0.4, 71)
    lat = binding.ODWF(DIMS, NS, 1.3, om)
    lat.set_gauge(torch.from_numpy(U).cuda())
    op = OracleODWF(U, 1.3, om)
    return binding, lat, op, U, om


def _rand_weights(C, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    z = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    return learned.Weights(np.eye(4) + 0.2 * z(4, 4), scale * z(C, 8, 4, 4), scale * z(C, 8, 4, 4))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("which", ["neumann", "random"])
def test_net_apply_and_adjoint(env, which):
    binding, lat, op, U, om = env
    net = binding.Net(lat, channels=2)
    W = learned.neumann_weights(C=2) if which == "neumann" else _rand_weights(2, 3)
    if which == "random":
        net.set_weights(W.flat())
    else:
        assert np.allclose(net.get_weights(), W.flat())  # the library's initial weights
    sch = solver.Schur(op, M1, M2)
    M = learned.LearnedPreconditioner(sch, W)
    r = inputs.gaussian_spinor5(DIMS, NS, 5)
    got = net.apply(torch.from_numpy(r).cuda(), M1, M2).cpu().numpy()
    ref = M.forward(r * sch.even)
    assert _rel(got, ref) < 2e-2
    assert np.max(np.abs(got * sch.odd)) == 0.0
    gad = net.apply(torch.from_numpy(r).cuda(), M1, M2, adjoint=True).cpu().numpy()
    assert _rel(gad, M.adjoint(r * sch.even)) < 2e-2
    net.close()


def test_net_equivariance(env):
    binding, lat, op, U, om = env
    G = inputs.random_su3_links(DIMS, 1.0, 9)[0]
    axis = {0: -3, 1: -4, 2: -5, 3: -6}
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[mu] = G @ U[mu] @ np.conj(np.swapaxes(np.roll(G, -1, axis=axis[mu]), -1, -2))
    lat2 = binding.ODWF(DIMS, NS, 1.3, om)
    lat2.set_gauge(torch.from_numpy(Ug).cuda())
    W = _rand_weights(2, 4).flat()
    n1, n2 = binding.Net(lat, 2), binding.Net(lat2, 2)
    n1.set_weights(W)
    n2.set_weights(W)
    r = inputs.gaussian_spinor5(DIMS, NS, 6)
    Gm = lambda f: np.einsum("...ab,...ib->...ia", G, f)
    a = n2.apply(torch.from_numpy(Gm(r)).cuda(), M1, M2).cpu().numpy()
    b = Gm(n1.apply(torch.from_numpy(r).cuda(), M1, M2).cpu().numpy())
    assert _rel(a, b) < 2e-2


def test_net_loss_and_gradient(env):
    binding, lat, op, U, om = env
    net = binding.Net(lat, 2)
    W = _rand_weights(2, 7, scale=0.2)
    net.set_weights(W.flat())
    sch = solver.Schur(op, M1, M2)
    rs = [inputs.gaussian_spinor5(DIMS, NS, 10 + i) for i in range(2)]
    es = [inputs.gaussian_spinor5(DIMS, NS, 20 + i) for i in range(2)]
    net.set_pairs([torch.from_numpy(r).cuda() for r in rs], M1, M2, es=[torch.from_numpy(e).cuda() for e in es])
    L, g = net.loss_grad()
    Lo, Go = learned.LearnedPreconditioner(sch, W).loss_and_grad([r * sch.even for r in rs], [e * sch.even for e in es])
    assert abs(L - Lo) < 2e-2 * Lo
    assert _rel(g, Go.flat()) < 5e-2


def test_net_residual_loss_and_gradient(env):
    """The residual loss |S M r - r|^2/|r|^2 (no solves) and its gradient against the oracle."""
    binding, lat, op, U, om = env
    net = binding.Net(lat, 2)
    W = _rand_weights(2, 8, scale=0.2)
    net.set_weights(W.flat())
    net.set_loss("residual")
    sch = solver.Schur(op, M1, M2)
    rs = [inputs.gaussian_spinor5(DIMS, NS, 14 + i) for i in range(2)]
    es = [inputs.gaussian_spinor5(DIMS, NS, 24 + i) for i in range(2)]  # not used by this loss
    net.set_pairs([torch.from_numpy(r).cuda() for r in rs], M1, M2, es=[torch.from_numpy(e).cuda() for e in es])
    L, g = net.loss_grad()
    Lo, Go = learned.LearnedPreconditioner(sch, W).residual_loss_and_grad([r * sch.even for r in rs])
    assert abs(L - Lo) < 2e-2 * Lo
    assert _rel(g, Go.flat()) < 5e-2
    net.close()


def test_train_and_solve(env):
    """Pairs from the library's solver; Adam lowers the loss; the preconditioned solve meets 1e-10."""
    binding, lat, op, U, om = env
    net = binding.Net(lat, 2)
    rs = [torch.from_numpy(inputs.gaussian_spinor5(DIMS, NS, 30 + i)).cuda() for i in range(4)]
    net.set_pairs(rs, M1, M2, tol=1e-9)
    losses = net.train(30, 2e-3)
    assert losses[-1] < losses[0]
    b = inputs.gaussian_spinor5(DIMS, NS, 50)
    x, st = net.solve(torch.from_numpy(b).cuda(), M1, M2,
                      opts=binding.solve_opts(tol=1e-10, prec="single", delta=1e-3))
    res = np.linalg.norm(b - op.ht(x.cpu().numpy(), M1, M2)) / np.linalg.norm(b)
    assert st["true_residual"] <= 1e-10 and res <= 1.05e-10
    # the network's starting point (Neumann weights) also converges; iteration counts are reported
    neu = binding.Net(lat, 2)
    x2, st2 = neu.solve(torch.from_numpy(b).cuda(), M1, M2,
                        opts=binding.solve_opts(tol=1e-10, prec="single", delta=1e-3))
    res2 = np.linalg.norm(b - op.ht(x2.cpu().numpy(), M1, M2)) / np.linalg.norm(b)
    assert res2 <= 1.05e-10
    _, st3 = lat.solve(torch.from_numpy(b).cuda(), M1, M2, opts=binding.solve_opts(tol=1e-10, prec="single"))
    print(f"\nloss {losses[0]:.4e} -> {losses[-1]:.4e}; iterations: trained {st['iters']}, "
          f"Neumann {st2['iters']}, plain CGNE {st3['iters']}")
    # the preconditioned solve needs fewer iterations than the method without the network, and training
    # does not make the network worse than its Neumann starting point
    assert st["iters"] < st3["iters"] and st2["iters"] < st3["iters"]
    assert st["iters"] <= 1.05 * st2["iters"]


def test_residual_loss_pairs_need_no_solves(env):
    """With the residual loss selected first, set_pairs stores the r_i without solving for e_i; training
    still lowers the loss, and switching to the error loss on those pairs is refused (ODWF_EINVAL)."""
    binding, lat, op, U, om = env
    net = binding.Net(lat, 2)
    net.set_loss("residual")
    rs = [torch.from_numpy(inputs.gaussian_spinor5(DIMS, NS, 70 + i)).cuda() for i in range(2)]
    net.set_pairs(rs, M1, M2)
    losses = net.train(10, 2e-3)
    assert losses[-1] < losses[0]
    net.set_loss("error")
    with pytest.raises(binding.OdwfError) as ei:
        net.loss_grad()
    assert ei.value.code == binding.ODWF_EINVAL
    net.close()


@pytest.mark.parametrize("which,truncate", [("none", False), ("neumann", False), ("trained", False),
                                            ("neumann", True), ("none", True)])
def test_gcr_solve(env, which, truncate):
    """Flexible GCR on S, right-preconditioned by the network (or none), restarted or with a sliding
    window of directions: FP64 true residual 1e-10."""
    binding, lat, op, U, om = env
    net = None
    if which != "none":
        net = binding.Net(lat, 2)
        if which == "trained":
            rs = [torch.from_numpy(inputs.gaussian_spinor5(DIMS, NS, 60 + i)).cuda() for i in range(3)]
            net.set_pairs(rs, M1, M2, tol=1e-9)
            net.train(20, 2e-3)
    b = inputs.gaussian_spinor5(DIMS, NS, 51)
    x, st = lat.solve_gcr(torch.from_numpy(b).cuda(), M1, M2, net=net, nvec=8, truncate=truncate,
                          opts=binding.solve_opts(tol=1e-10, prec="single", delta=1e-3))
    res = np.linalg.norm(b - op.ht(x.cpu().numpy(), M1, M2)) / np.linalg.norm(b)
    assert st["true_residual"] <= 1e-10 and res <= 1.05e-10
    print(f"\nGCR({which}, {'window' if truncate else 'restarted'}): {st['iters']} iterations, "
          f"{st['reliable_updates']} cycles")


def test_zero_rhs(env):
    """b = 0: the network-preconditioned CGNE and GCR return x = 0 with no iteration and no error."""
    binding, lat, op, U, om = env
    net = binding.Net(lat, 2)
    z = torch.zeros(lat.shape5, dtype=torch.complex128, device="cuda")
    x, st = net.solve(z, M1, M2, opts=binding.solve_opts(tol=1e-10, prec="single", delta=1e-3))
    assert torch.count_nonzero(x).item() == 0 and st["iters"] == 0 and st["true_residual"] == 0.0
    x, st = lat.solve_gcr(z, M1, M2, net=net, nvec=8, opts=binding.solve_opts(tol=1e-10, prec="single"))
    assert torch.count_nonzero(x).item() == 0 and st["iters"] == 0
    net.close()


def test_zero_training_vector_rejected(env):
    """A training vector that vanishes is refused (ODWF_EINVAL) and leaves no partial pair set; valid
    pairs set afterwards train as usual."""
    binding, lat, op, U, om = env
    net = binding.Net(lat, 2)
    net.set_loss("residual")
    good = torch.from_numpy(inputs.gaussian_spinor5(DIMS, NS, 80)).cuda()
    z = torch.zeros(lat.shape5, dtype=torch.complex128, device="cuda")
    with pytest.raises(binding.OdwfError) as ei:
        net.set_pairs([good, z], M1, M2)
    assert ei.value.code == binding.ODWF_EINVAL
    with pytest.raises(binding.OdwfError):
        net.loss_grad()  # no pairs stored
    net.set_pairs([good], M1, M2)
    losses = net.train(3, 2e-3)
    assert np.all(np.isfinite(losses))
    net.close()


def test_gcr_rejects_bad_basis_and_reports_noconv(env):
    binding, lat, op, U, om = env
    b = torch.from_numpy(inputs.gaussian_spinor5(DIMS, NS, 52)).cuda()
    for bad in (0, 17):
        with pytest.raises(binding.OdwfError):
            lat.solve_gcr(b, M1, M2, nvec=bad)
    _, st = lat.solve_gcr(b, M1, M2, nvec=4, opts=binding.solve_opts(tol=1e-10, prec="single", maxiter=3),
                          allow_noconv=True)
    assert st["status"] == binding.ODWF_ENOCONV and st["iters"] == 3 and st["true_residual"] > 1e-10


@pytest.mark.parametrize("use_tc,occ", [("1", "4:4"), ("0", "4:4"), ("1", "1:5")])
def test_net_ns16_tensor_memory_layer(use_tc, occ, monkeypatch):
    """At Ns = 16 the 1 -> 2 layer (forward, and the first adjoint layer) runs on the fifth-generation
    tensor cores: tcgen05.mma with FP32 accumulators in tensor memory; ODWF_TCGEN05=0 selects the
    mma.sync layer. Every launch form of the layers (register caps ODWF_NET_OCC) against the oracle (BF16 tolerance 2e-2 outputs, 5e-2 weight gradients), and
    the preconditioned solve meets the FP64 true residual."""
    monkeypatch.setenv("ODWF_TCGEN05", use_tc)
    monkeypatch.setenv("ODWF_NET_OCC", occ)
    from paper_1710_09621_gb300 import build
    build.build()
    from paper_1710_09621_gb300 import binding
    dims, Ns = (4, 4, 4, 8), 16
    om = inputs.omega_zolotarev(Ns, 0.05, 6.2)
    U = inputs.random_su3_links(dims, 0.4, 73)
    lat = binding.ODWF(dims, Ns, 1.3, om)
    lat.set_gauge(torch.from_numpy(U).cuda())
    op = OracleODWF(U, 1.3, om)
    sch = solver.Schur(op, M1, M2)
    net = binding.Net(lat, 2)
    W = _rand_weights(2, 11)
    net.set_weights(W.flat())
    M = learned.LearnedPreconditioner(sch, W)
    r = inputs.gaussian_spinor5(dims, Ns, 12)
    assert _rel(net.apply(torch.from_numpy(r).cuda(), M1, M2).cpu().numpy(), M.forward(r * sch.even)) < 2e-2
    assert _rel(net.apply(torch.from_numpy(r).cuda(), M1, M2, adjoint=True).cpu().numpy(),
                M.adjoint(r * sch.even)) < 2e-2
    rs = [inputs.gaussian_spinor5(dims, Ns, 13 + i) for i in range(2)]
    es = [inputs.gaussian_spinor5(dims, Ns, 23 + i) for i in range(2)]
    net.set_pairs([torch.from_numpy(x).cuda() for x in rs], M1, M2, es=[torch.from_numpy(x).cuda() for x in es])
    L, g = net.loss_grad()
    Lo, Go = M.loss_and_grad([x * sch.even for x in rs], [x * sch.even for x in es])
    assert abs(L - Lo) < 2e-2 * Lo and _rel(g, Go.flat()) < 5e-2
    neu = binding.Net(lat, 2)
    b = inputs.gaussian_spinor5(dims, Ns, 33)
    x, st = neu.solve(torch.from_numpy(b).cuda(), M1, M2, opts=binding.solve_opts(tol=1e-10, prec="single", delta=1e-3))
    assert np.linalg.norm(b - op.ht(x.cpu().numpy(), M1, M2)) / np.linalg.norm(b) <= 1.05e-10
    net.close()
    neu.close()
    lat.close()


def test_eofa_terms_with_attached_network(env):
    """With a network attached (odwf_set_preconditioner) the EOFA action and force solve with CGNE on
    S M; they still equal the oracle's (action 1e-10, force 1e-9), with fewer iterations than plain CGNE."""
    from oracle import eofa as oeofa
    binding, lat, op, U, om = env
    phi = inputs.gaussian_spinor(DIMS, 61)
    t = oeofa.Term(-1, 0.05, 0.05, 0.1)
    spec = binding.TermSpec(t.chirality, t.m3, t.m4, t.m_den)
    o = binding.solve_opts(tol=1e-12, prec="single", delta=1e-3)
    S0, st0 = lat.action(spec, torch.from_numpy(phi).cuda(), opts=o)
    net = binding.Net(lat, 2)
    lat.set_preconditioner(net)
    try:
        S1, st1 = lat.action(spec, torch.from_numpy(phi).cuda(), opts=o)
        F1, _ = lat.force(spec, torch.from_numpy(phi).cuda(), opts=o)
    finally:
        lat.set_preconditioner(None)
        net.close()
    So, _ = oeofa.action(op, t, phi, tol=1e-12)
    Fo, _ = oeofa.force(op, t, phi, tol=1e-12)
    assert abs(S1 - So) < 1e-10 * abs(So) and abs(S0 - So) < 1e-10 * abs(So)
    assert _rel(F1.cpu().numpy(), Fo) < 1e-9
    assert st1["iters"] < st0["iters"], (st1["iters"], st0["iters"])
