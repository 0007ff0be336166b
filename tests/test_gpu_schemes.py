"""Mass-preconditioning schemes on the GPU: the term lists of Eq.(noMP), Eq.(old_MP_N), Eq.(new_MP_N)
(cascades N = 1, 2) and their parity partners (Eq.(noMP_P), Section 2), each term's action and force
through the C ABI against the FP64 oracle.

Every term list is the library's own (eofa_mp_terms); the oracle builds the same lists independently,
and the counts are 2N + 2 (old) and N + 2 (new), the ratio behind the (2N + 2)/(N + 2) speed-up bound
of Section 4. A parity partner flips every chirality and swaps the masses of every factor.
"""
import numpy as np
import pytest

from oracle import eofa as oeofa
from oracle.operators import ODWF as OracleODWF
from paper_1710_09621_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS, NS, M0 = (4, 2, 2, 4), 4, 1.3   # small: the oracle solves every term with numpy
M, MPV = 0.05, 1.0


@pytest.fixture(scope="module")
def env():
    from paper_1710_09621_gb300 import build
    build.build()
    from paper_1710_09621_gb300 import binding
    om = inputs.omega_zolotarev(NS, 0.05, 6.2)
    U = inputs.random_su3_links(DIMS, 0.4, 81)
    lat = binding.ODWF(DIMS, NS, M0, om)
    lat.set_gauge(torch.from_numpy(U).cuda())
    return binding, lat, OracleODWF(U, M0, om)


def _oracle_list(scheme, mh, parity):
    if scheme == "none":
        ts = oeofa.no_mp(M, MPV)
    elif scheme == "old":
        ts = oeofa.old_mp_cascade(M, mh, MPV)
    else:
        ts = oeofa.new_mp_cascade(M, mh, MPV)
    if parity:  # P swaps the two masses of every factor (m1, m2) -> (m2, m1)
        ts = [oeofa.term_from_ratio((t.numerator[1], t.numerator[0]), (t.denominator[1], t.denominator[0])) for t in ts]
    return ts


SCHEMES = [("none", []), ("old", [0.2]), ("new", [0.2]), ("old", [0.1, 0.3]), ("new", [0.1, 0.3])]


@pytest.mark.parametrize("scheme,mh", SCHEMES)
@pytest.mark.parametrize("parity", [0, 1])
def test_scheme_terms_action_force(env, scheme, mh, parity):
    binding, lat, op = env
    code = {"none": binding.MP_NONE, "old": binding.MP_OLD, "new": binding.MP_NEW}[scheme]
    specs = binding.mp_terms(code, M, mh, MPV, parity=bool(parity))
    ref = _oracle_list(scheme, mh, parity)
    assert [(s.chirality, s.m3, s.m4, s.m_den) for s in specs] == [(t.chirality, t.m3, t.m4, t.m_den) for t in ref]
    N = len(mh)
    assert len(specs) == {"none": 2, "old": 2 * N + 2, "new": N + 2}[scheme]
    phi = inputs.gaussian_spinor(DIMS, 90 + len(specs) + parity)
    for spec, term in zip(specs, ref):
        S, _ = lat.action(spec, torch.from_numpy(phi).cuda(), opts=binding.solve_opts(tol=1e-12))
        So, _ = oeofa.action(op, term, phi, tol=1e-12)
        assert abs(S - So) < 1e-10 * abs(So)
        F, _ = lat.force(spec, torch.from_numpy(phi).cuda(), opts=binding.solve_opts(tol=1e-12, prec="single"))
        Fo, _ = oeofa.force(op, term, phi, tol=1e-12)
        assert np.linalg.norm(F.cpu().numpy() - Fo) < 1e-8 * np.linalg.norm(Fo)
