"""odwf_apply_noalloc: the apply for callers that cannot allocate device memory mid-run.

It is compared, through the C ABI, with odwf_apply on the same inputs (FP64 agreement to 1e-12
relative, FP32 to 2e-6 as in the other parity tests), on two calls in a row, and it must reject a
lattice that does not fit its fixed 32 MiB array. The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1710_09621_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    from paper_1710_09621_gb300 import build
    build.build()
    from paper_1710_09621_gb300 import binding as b
    return b


def _noalloc(b, lat, x, m1, m2, op, prec):
    out = torch.empty_like(x)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lat.lib.odwf_apply_noalloc(lat.h, op, float(m1), float(m2), ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), prec, stream)
    return rc, out


@pytest.mark.parametrize("dims,Ns", [((4, 4, 4, 4), 8), ((8, 8, 8, 8), 16)])
@pytest.mark.parametrize("prec", ["double", "single"])
@pytest.mark.parametrize("op", ["dt", "ht"])
def test_noalloc_matches_apply(binding, dims, Ns, prec, op):
    om = inputs.omega_zolotarev(Ns, 0.05, 6.2)
    lat = binding.ODWF(dims, Ns, 1.3, om)
    lat.set_gauge(torch.from_numpy(inputs.random_su3_links(dims, 0.4, 31)).cuda())
    tol = 1e-12 if prec == "double" else 2e-6
    for call, (m1, m2, seed) in enumerate([(0.05, 1.0, 1), (0.01, 0.01, 2)]):  # two calls in a row
        x = torch.from_numpy(inputs.gaussian_spinor5(dims, Ns, 40 + seed)).cuda()
        ref = lat.apply(x, m1, m2, op=op, prec=prec).cpu().numpy()
        rc, out = _noalloc(binding, lat, x, m1, m2, binding._OP[op], binding._PREC[prec])
        assert rc == 0, lat.lib.odwf_last_error(lat.h).decode()
        got = out.cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol, call


def test_noalloc_rejects_oversize(binding):
    dims, Ns = (16, 16, 16, 16), 16  # four FP64 half fields need 400 MiB > 32 MiB
    lat = binding.ODWF(dims, Ns, 1.3, inputs.omega_shamir(Ns))
    lat.set_gauge(torch.from_numpy(inputs.random_su3_links(dims, 0.4, 32)).cuda())
    x = torch.zeros(lat.shape5, dtype=torch.complex128, device="cuda")
    rc, _ = _noalloc(binding, lat, x, 0.1, 0.1, binding.OP_DT, binding.PREC_DOUBLE)
    assert rc == binding.ODWF_EINVAL
    assert "maximum" in lat.lib.odwf_last_error(lat.h).decode()
    # the handle and the device stay usable
    y = lat.apply(x, 0.1, 0.1)
    assert torch.count_nonzero(y).item() == 0
