"""Every kernel variant the library can run, against the FP64 oracle, and its failure statuses.

* FP16 storage applies (ODWF_PREC_HALF): the input and each intermediate half field are stored as
  FP16 with one FP32 scale per (site, s), so every stored real carries a relative rounding error of
  at most 2^-11 (rms 2^-11/sqrt(3) = 2.8e-4). An apply of D_T or H_T rounds twice (input, output):
  the output's relative L2 error is about sqrt(2) x 2.8e-4 = 4e-4. The bound used is 2e-3 (D_odwf,
  which stores two more intermediates around D_T, 4e-3).
* The bulk-staged hop kernels (ODWF_STAGED=1) in FP32 (2e-6, as the plain FP32 kernels) and FP16,
  applies and solves; the solve bar is the FP64 true residual 1e-10 for every inner precision.
* The launch configuration the autotuner picks (odwf_autotune), applies and solves.
* The two-slices-per-thread kernels with two-row SU(3) links (ODWF_PAIR=1) in FP32 and FP16, applies and
  a solve, and the one-slice kernels kept for links that are not SU(3).
* Failure statuses in the allowed forms: a wall-clock budget that runs out (ODWF_ETIMEOUT), a NaN in
  the right-hand side (ODWF_EBREAKDOWN), and the bulk-staged kernels' bounded wait made to run out by a
  test-only cycle limit (ODWF_EFAULT). After each, the device and a fresh handle still work.
* The Lanczos estimate of a term operator's spectrum (eofa_term_spectrum) against the dense
  eigenvalues of the oracle's X, and the heat-bath's check that rejects an interval too narrow.
"""
import numpy as np
import pytest

from oracle import eofa as oeofa
from oracle import solver as osolver
from oracle.operators import ODWF as OracleODWF
from paper_1710_09621_gb300 import inputs

from oracle_dense import DenseEOFA

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_HALF, TOL_HALF_DODWF, TOL_SINGLE, TOL_DOUBLE = 2e-3, 4e-3, 2e-6, 1e-12

CASES = [
    ((4, 4, 4, 4), 8, "shamir", 0.4, 0),
    ((4, 2, 6, 4), 6, "zolo", 0.4, 2),     # Ns = 6: ragged CTA of 32 sites, no FP16 staging (Ns % 4)
    ((8, 8, 8, 16), 16, "zolo", 0.3, 3),   # more site groups than the grid: grid-stride path
]


@pytest.fixture(scope="module")
def lib():
    from paper_1710_09621_gb300 import build
    build.build()
    from paper_1710_09621_gb300 import binding
    return binding


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _setup(lib, dims, Ns, kind, eps, seed):
    om = inputs.omega_shamir(Ns) if kind == "shamir" else inputs.omega_zolotarev(Ns, 0.05, 6.2)
    U = inputs.random_su3_links(dims, eps, seed)
    lat = lib.ODWF(dims, Ns, 1.3, om)
    lat.set_gauge(torch.from_numpy(U).cuda())
    return lat, OracleODWF(U, 1.3, om)


def _apply_checks(lat, op, case, m12, prec):
    tol = {"half": TOL_HALF, "single": TOL_SINGLE, "double": TOL_DOUBLE}[prec]
    psi = inputs.gaussian_spinor5(case[0], case[1], 100 + case[4])
    x = torch.from_numpy(psi).cuda()
    assert _rel(lat.apply(x, *m12, op="dt", prec=prec).cpu().numpy(), op.dt(psi, *m12)) < tol
    assert _rel(lat.apply(x, *m12, op="dt", dag=True, prec=prec).cpu().numpy(), op.dt_dag(psi, *m12)) < tol
    refh = op.ht(psi, *m12)
    assert _rel(lat.apply(x, *m12, op="ht", prec=prec).cpu().numpy(), refh) < tol
    assert _rel(lat.apply(x, *m12, op="ht", dag=True, prec=prec).cpu().numpy(), refh) < tol
    tol_o = TOL_HALF_DODWF if prec == "half" else tol
    assert _rel(lat.apply(x, *m12, op="dodwf", prec=prec).cpu().numpy(), op.dodwf(psi, *m12)) < tol_o


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("m12", [(0.05, 1.0), (1.0, 0.1)])
def test_half_apply_parity(lib, case, m12):
    """FP16-storage applies element by element against the oracle (plain per-thread-gather kernels)."""
    lat, op = _setup(lib, *case)
    _apply_checks(lat, op, case, m12, "half")
    lat.close()


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["single", "half"])
def test_staged_apply_parity(lib, case, prec, monkeypatch):
    """The bulk-staged gather kernels (ODWF_STAGED=1) against the oracle."""
    monkeypatch.setenv("ODWF_STAGED", "1")
    lat, op = _setup(lib, *case)
    _apply_checks(lat, op, case, (0.05, 0.5), prec)
    lat.close()


@pytest.mark.parametrize("case", CASES[:2])
@pytest.mark.parametrize("prec", ["single", "half"])
def test_staged_solve_true_residual(lib, case, prec, monkeypatch):
    monkeypatch.setenv("ODWF_STAGED", "1")
    lat, op = _setup(lib, *case)
    b = inputs.gaussian_spinor5(case[0], case[1], 200 + case[4])
    x, st = lat.solve(torch.from_numpy(b).cuda(), 0.05, 0.1, opts=lib.solve_opts(tol=1e-10, prec=prec))
    res = np.linalg.norm(b - op.ht(x.cpu().numpy(), 0.05, 0.1)) / np.linalg.norm(b)
    assert st["true_residual"] <= 1e-10 and res <= 1.05e-10, res
    lat.close()


@pytest.mark.parametrize("prec", ["single", "half"])
def test_autotuned_variants(lib, prec):
    """After odwf_autotune has chosen grid sizes and gather kinds, the applies and a solve still agree
    with the oracle."""
    case = CASES[2]
    lat, op = _setup(lib, *case)
    report = lat.autotune(prec)
    assert "chosen key" in report
    _apply_checks(lat, op, case, (0.05, 0.5), prec)
    b = inputs.gaussian_spinor5(case[0], case[1], 250)
    x, st = lat.solve(torch.from_numpy(b).cuda(), 0.05, 0.1, opts=lib.solve_opts(tol=1e-10, prec=prec))
    res = np.linalg.norm(b - op.ht(x.cpu().numpy(), 0.05, 0.1)) / np.linalg.norm(b)
    assert res <= 1.05e-10, res
    lat.close()


@pytest.mark.parametrize("prec,form", [("single", "1"), ("single", "2"), ("single", "3"), ("half", "1"),
                                       ("half", "3")])
def test_two_slice_kernels(lib, prec, form, monkeypatch):
    """The two-slices-per-thread kernels with two-row links (ODWF_PAIR=form; Ns = 16, structured
    fifth-dimension products) against the oracle: applies, a solve to the FP64 true residual 1e-10, and
    the profile shows that they ran (kernel keys 5xxxxx above the one-slice ones; the bulk-copy forms 2
    and 3 add 1000000 and exist for FP32 storage, FP16 storage keeps the register gathers)."""
    monkeypatch.setenv("ODWF_PAIR", form)
    case = CASES[2]
    lat, op = _setup(lib, *case)
    lat.profile(True)
    _apply_checks(lat, op, case, (0.05, 0.5), prec)
    b = inputs.gaussian_spinor5(case[0], case[1], 260)
    x, st = lat.solve(torch.from_numpy(b).cuda(), 0.05, 0.1, opts=lib.solve_opts(tol=1e-10, prec=prec))
    res = np.linalg.norm(b - op.ht(x.cpu().numpy(), 0.05, 0.1)) / np.linalg.norm(b)
    assert res <= 1.05e-10, res
    stg = {"single": 1, "half": 2}[prec]
    bulk = 1000000 if (prec == "single" and form in ("2", "3")) else 0
    ran = {k for k in lat.profile_read() if (k // 100000) % 10 == stg + 5}
    # K1 (hop then A^-1), K2A / K2B (A on p plus the hop, CGNE updates) and the apply's hop + A own
    assert {bulk + stg * 100000 + 500000 + k for k in (11000, 10112, 10113, 10110)} <= ran, ran
    lat.close()


def test_two_slice_kernels_need_su3_links(lib, monkeypatch):
    """Links that are not SU(3) (here 1.01 U) are not represented by two rows: the library keeps the
    one-slice kernels, and the results still agree with the oracle."""
    monkeypatch.setenv("ODWF_PAIR", "1")
    dims, Ns = CASES[2][0], CASES[2][1]
    om = inputs.omega_zolotarev(Ns, 0.05, 6.2)
    U = 1.01 * inputs.random_su3_links(dims, 0.3, 3)
    lat = lib.ODWF(dims, Ns, 1.3, om)
    lat.set_gauge(torch.from_numpy(U).cuda())
    op = OracleODWF(U, 1.3, om)
    lat.profile(True)
    _apply_checks(lat, op, CASES[2], (0.05, 0.5), "single")
    assert not any((k // 100000) % 10 >= 5 for k in lat.profile_read() if k < 1000000)
    lat.close()


def test_timeout_status_and_recovery(lib):
    lat, op = _setup(lib, *CASES[2])
    b = torch.from_numpy(inputs.gaussian_spinor5(CASES[2][0], CASES[2][1], 31)).cuda()
    _, st = lat.solve(b, 0.01, 0.01, opts=lib.solve_opts(tol=1e-10, prec="single", max_seconds=1e-9),
                      allow_noconv=True)
    assert st["status"] == lib.ODWF_ETIMEOUT
    assert st["true_residual"] > 1e-10
    x, st2 = lat.solve(b, 0.1, 0.1, opts=lib.solve_opts(tol=1e-10, prec="single"))
    bb = b.cpu().numpy()
    assert np.linalg.norm(bb - op.ht(x.cpu().numpy(), 0.1, 0.1)) / np.linalg.norm(bb) <= 1.05e-10
    lat.close()


@pytest.mark.parametrize("prec", ["double", "single"])
def test_nan_rhs_breakdown_and_recovery(lib, prec):
    lat, op = _setup(lib, *CASES[0])
    b = inputs.gaussian_spinor5(CASES[0][0], CASES[0][1], 32)
    bad = b.copy()
    bad[3, 1, 2, 0, 1, 2, 1] = np.nan
    with pytest.raises(lib.OdwfError) as e:
        lat.solve(torch.from_numpy(bad).cuda(), 0.05, 0.1, opts=lib.solve_opts(tol=1e-10, prec=prec))
    assert e.value.code == lib.ODWF_EBREAKDOWN
    x, _ = lat.solve(torch.from_numpy(b).cuda(), 0.05, 0.1, opts=lib.solve_opts(tol=1e-10, prec=prec))
    assert np.linalg.norm(b - op.ht(x.cpu().numpy(), 0.05, 0.1)) / np.linalg.norm(b) <= 1.05e-10
    lat.close()


def test_staged_wait_timeout_status(lib, monkeypatch):
    """A one-cycle limit on the staged kernels' bounded mbarrier wait (the test-only
    ODWF_TEST_WAIT_CYCLES) makes it run out: the kernel sets its fault word, waits out its copies with
    the normal limit and returns; the call reports ODWF_EFAULT and the device stays usable."""
    case = CASES[2]
    monkeypatch.setenv("ODWF_STAGED", "1")
    monkeypatch.setenv("ODWF_TEST_WAIT_CYCLES", "1")
    lat, op = _setup(lib, *case)
    psi = inputs.gaussian_spinor5(case[0], case[1], 33)
    x = torch.from_numpy(psi).cuda()
    with pytest.raises(lib.OdwfError) as e:
        lat.apply(x, 0.05, 0.5, op="dt", prec="single")
    assert e.value.code == lib.ODWF_EFAULT
    # the fault word was cleared: with the normal limit the same handle type works again
    lat.close()
    monkeypatch.delenv("ODWF_TEST_WAIT_CYCLES")
    lat2, op2 = _setup(lib, *case)
    assert _rel(lat2.apply(x, 0.05, 0.5, op="dt", prec="single").cpu().numpy(), op2.dt(psi, 0.05, 0.5)) < TOL_SINGLE
    lat2.close()


def test_two_slice_bulk_wait_timeout_status(lib, monkeypatch):
    """The same one-cycle wait limit on the bulk-copy two-slice kernels (ODWF_PAIR=3): the waits run out,
    the kernel stops issuing, waits out the copies in flight with the normal limit and returns; the call
    reports ODWF_EFAULT and a fresh handle computes D_T correctly."""
    case = CASES[2]
    monkeypatch.setenv("ODWF_PAIR", "3")
    monkeypatch.setenv("ODWF_TEST_WAIT_CYCLES", "1")
    lat, op = _setup(lib, *case)
    psi = inputs.gaussian_spinor5(case[0], case[1], 34)
    x = torch.from_numpy(psi).cuda()
    with pytest.raises(lib.OdwfError) as e:
        lat.apply(x, 0.05, 0.5, op="dt", prec="single")
    assert e.value.code == lib.ODWF_EFAULT
    lat.close()
    monkeypatch.delenv("ODWF_TEST_WAIT_CYCLES")
    lat2, op2 = _setup(lib, *case)
    assert _rel(lat2.apply(x, 0.05, 0.5, op="dt", prec="single").cpu().numpy(), op2.dt(psi, 0.05, 0.5)) < TOL_SINGLE
    lat2.close()


TERMS = [oeofa.Term(-1, 0.05, 0.05, 0.1), oeofa.Term(+1, 0.05, 0.1, 1.0), oeofa.Term(-1, 1.0, 0.1, 1.0)]


@pytest.mark.parametrize("term", TERMS)
def test_term_spectrum_matches_dense(lib, term):
    """Lanczos extremes of X on a 2^4 x Ns = 4 lattice (96-dimensional chiral space, 80 steps) equal
    the smallest and largest eigenvalue of the oracle's dense X (to 1e-9: after 40 steps the smallest
    Ritz value was still 1.2e-7 above it)."""
    dims, Ns = (2, 2, 2, 2), 4
    om = inputs.omega_zolotarev(Ns, 0.05, 6.2)
    U = inputs.random_su3_links(dims, 0.4, 21)
    lat = lib.ODWF(dims, Ns, 1.3, om)
    lat.set_gauge(torch.from_numpy(U).cuda())
    ev = np.linalg.eigvalsh(DenseEOFA(OracleODWF(U, 1.3, om)).term_x(term))
    v0 = torch.from_numpy(inputs.gaussian_spinor(dims, 5)).cuda()
    spec = lib.TermSpec(term.chirality, term.m3, term.m4, term.m_den)
    lo, hi = lat.term_spectrum(spec, v0, n_iter=80, opts=lib.solve_opts(tol=1e-13))
    assert abs(lo - ev[0]) < 1e-9 and abs(hi - ev[-1]) < 1e-9, (lo, hi, ev[0], ev[-1])
    lat.close()


def test_heatbath_rejects_narrow_interval(lib):
    dims, Ns = (4, 4, 4, 4), 8
    lat, op = _setup(lib, dims, Ns, "zolo", 0.4, 6)
    eta = torch.from_numpy(inputs.gaussian_spinor(dims, 12)).cuda()
    spec = lib.TermSpec(-1, 0.05, 0.05, 0.5)
    o = lib.solve_opts(tol=1e-10, prec="single")
    phi, info = lat.heatbath(spec, eta, opts=o, check_iters=12)
    lo, hi = info["ritz"]
    mref, mden = 0.05, 0.5
    assert 0.98 * (1 + mref) / (1 + mden) <= lo < hi <= 1.0
    with pytest.raises(lib.OdwfError) as e:
        lat.heatbath(spec, eta, opts=o, x_lo=0.5 * (lo + hi), x_hi=1.0, check_iters=12)
    assert e.value.code == lib.ODWF_ESPECTRUM
    lat.close()


@pytest.mark.parametrize("prec", ["double", "single", "half"])
def test_dense_fifth_dimension_fallback(lib, prec, monkeypatch):
    """At Ns = 16 the kernels apply A and A^{-1} by the structured O(Ns) recurrence; ODWF_DENSE_S=1
    selects the dense Ns x Ns products instead. Both agree with the oracle, applies and a solve."""
    case = CASES[2]
    for dense in ("0", "1"):
        monkeypatch.setenv("ODWF_DENSE_S", dense)
        lat, op = _setup(lib, *case)
        _apply_checks(lat, op, case, (0.01, 0.3), prec)
        b = inputs.gaussian_spinor5(case[0], case[1], 260)
        x, st = lat.solve(torch.from_numpy(b).cuda(), 0.01, 0.3, opts=lib.solve_opts(tol=1e-10, prec=prec))
        res = np.linalg.norm(b - op.ht(x.cpu().numpy(), 0.01, 0.3)) / np.linalg.norm(b)
        assert res <= 1.05e-10, (dense, res)
        lat.close()


def test_autotune_cache_persists_and_tiles(lib, tmp_path):
    """odwf_autotune_cache: the first handle tunes and appends its choices, a second handle of the same
    lattice loads them without timing; a hand-written entry that asks for the doubled tile (twice the
    default sites per CTA) on every fused kernel, with and without bulk staging, still agrees with the oracle."""
    case = CASES[2]
    path = tmp_path / "tune.txt"
    lat, op = _setup(lib, *case)
    assert lat.autotune_cached(path, "single") is False
    assert "8x8x8x16|16|1|" in path.read_text()
    lat.close()
    lat2, op2 = _setup(lib, *case)
    assert lat2.autotune_cached(path, "single") is True
    _apply_checks(lat2, op2, case, (0.05, 0.5), "single")
    lat2.close()
    name = torch.cuda.get_device_name()
    for staged in (0, 1):
        forced = tmp_path / f"forced{staged}.txt"
        keys = [111000, 110112, 110113, 110110]   # K1, CGNE forward / adjoint halves, D_T parity block (FP32)
        forced.write_text(f"{name}|8x8x8x16|16|1|" + ",".join(f"{k}:{staged * 2}:{staged}:2" for k in keys) + "\n")
        lat3, op3 = _setup(lib, *case)
        assert lat3.autotune_cached(forced, "single") is True
        _apply_checks(lat3, op3, case, (0.05, 0.5), "single")
        b = inputs.gaussian_spinor5(case[0], case[1], 270)
        x, st = lat3.solve(torch.from_numpy(b).cuda(), 0.05, 0.1, opts=lib.solve_opts(tol=1e-10, prec="single"))
        assert np.linalg.norm(b - op3.ht(x.cpu().numpy(), 0.05, 0.1)) / np.linalg.norm(b) <= 1.05e-10
        lat3.close()


def test_fp64_fma_peak_measured(lib):
    """The FP64 roof the FP64 hop kernels are reported against is measured on the device: positive and
    below the FP32 rate (GB300 runs FP64 at a small fraction of it)."""
    lat, op = _setup(lib, *CASES[0])
    t = lat.fp64_fma_peak()
    assert 0.05 < t < 20.0, t
    lat.close()
