"""CPU checks of the C ABI library: it builds for sm_103a, loads, and exports every declared symbol."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "odwf.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|double|const char\*)\s+(\w+)\s*\(", src, re.M)))


def test_header_matches_binding_exports():
    from paper_1710_09621_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared()


def test_library_builds_and_exports_every_symbol():
    from paper_1710_09621_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))
    import ctypes
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    # the library on disk was built from exactly these sources, flags and host architecture
    with open(build.STAMP) as fh:
        assert fh.read().strip() == build.source_hash()


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1710_09621_gb300 import binding
    with pytest.raises(RuntimeError):
        binding._lib = None
        binding.load_library(str(tmp_path / "missing.so"))
    binding._lib = None


def test_mp_term_lists_match_oracle():
    """The library's term lists (host code) equal the oracle's Eq.(noMP)/(old_MP_N)/(new_MP_N) lists."""
    from paper_1710_09621_gb300 import binding, build
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    from oracle import eofa

    def key(ts):
        return [(t.chirality, t.m3, t.m4, t.m_den) for t in ts]

    m, M = 0.01, 1.0
    assert key(binding.mp_terms(binding.MP_NONE, m, [], M)) == key(eofa.no_mp(m, M))
    assert key(binding.mp_terms(binding.MP_OLD, m, [0.1], M)) == key(eofa.old_mp(m, 0.1, M))
    assert key(binding.mp_terms(binding.MP_NEW, m, [0.1], M)) == key(eofa.new_mp(m, 0.1, M))
    for hs in ([0.1, 0.3], [0.05, 0.1, 0.4]):
        assert key(binding.mp_terms(binding.MP_OLD, m, hs, M)) == key(eofa.old_mp_cascade(m, hs, M))
        assert key(binding.mp_terms(binding.MP_NEW, m, hs, M)) == key(eofa.new_mp_cascade(m, hs, M))
        assert len(binding.mp_terms(binding.MP_NEW, m, hs, M)) == len(hs) + 2
        assert len(binding.mp_terms(binding.MP_OLD, m, hs, M)) == 2 * len(hs) + 2
    # parity partner of Eq.(noMP) is Eq.(noMP_P): chiralities {+, -}
    pp = binding.mp_terms(binding.MP_NONE, m, [], M, parity=True)
    assert [t.chirality for t in pp] == [1, -1]
    assert key(pp) == key([eofa.term_from_ratio((m, m), (M, m)), eofa.term_from_ratio((M, m), (M, M))])
    with pytest.raises(binding.OdwfError):
        binding.mp_terms(binding.MP_NEW, m, [2.0], M)


def test_library_k_matches_the_rank_one_factor():
    """The library's k(m_j, m_i) (host code) is the coefficient of the rank-one difference
    R5 (M(m_j) - M(m_i)) = k Omega Omega^T of Eq.(delta_ij), found numerically from the oracle's
    dense fifth-dimension matrices, and reduces to (1 - m)/(1 + m) for m_j = 1."""
    import numpy as np
    from paper_1710_09621_gb300 import binding, build, inputs
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    from oracle import fifth
    om = inputs.omega_zolotarev(8, 0.05, 6.2)
    R5 = np.eye(8)[::-1]
    for mj, mi in ((0.1, 0.01), (1.0, 0.05), (0.3, 0.7)):
        D = R5 @ (fifth.m_matrix(om, mj, -1) - fifth.m_matrix(om, mi, -1))
        ev = np.linalg.eigvalsh(0.5 * (D + D.T))
        lead = ev[np.argmax(np.abs(ev))]          # the single non-zero eigenvalue = k |Omega|^2
        Om = fifth.omega_vector(om, -1)
        assert binding.eofa_k(mj, mi) == pytest.approx(lead / (Om @ Om), rel=1e-12)
    for m in (0.01, 0.1, 0.5):
        assert binding.eofa_k(1.0, m) == pytest.approx((1 - m) / (1 + m), rel=1e-15)


def test_create_rejects_bad_arguments_before_touching_the_device():
    """odwf_create validates its arguments on the host (no GPU needed): odd or too large Ns, odd
    extents, m0 outside (0, 2), non-positive or non-R5-symmetric omega give ODWF_EINVAL with a
    message; with valid arguments and no usable GPU it fails loudly (ODWF_ECUDA), never falls back."""
    import numpy as np
    from paper_1710_09621_gb300 import binding, build
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    om8 = np.ones(8)
    bad = [((4, 4, 4, 4), 7, 1.3, np.ones(7), "Ns"),
           ((4, 4, 4, 4), 34, 1.3, np.ones(34), "Ns"),
           ((4, 4, 3, 4), 8, 1.3, om8, "even"),
           ((4, 4, 4, 4), 8, 2.5, om8, "m0"),
           ((4, 4, 4, 4), 8, 1.3, np.r_[om8[:-1], -1.0], "omega"),
           ((4, 4, 4, 4), 8, 1.3, np.arange(1.0, 9.0), "R5")]
    for dims, ns, m0, om, word in bad:
        with pytest.raises(binding.OdwfError) as ei:
            binding.ODWF(dims, ns, m0, om)
        assert ei.value.code == binding.ODWF_EINVAL and word in str(ei.value), (dims, ns, m0, str(ei.value))
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        return
    with pytest.raises(binding.OdwfError) as ei:
        binding.ODWF((4, 4, 4, 4), 8, 1.3, om8)
    assert ei.value.code == binding.ODWF_ECUDA
