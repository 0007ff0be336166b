"""The threaded driver of the oracle's Schur operator (the CPU baseline's all-core run) computes what
the serial oracle computes, and the benchmark's CPU-baseline helpers run."""
import numpy as np
import pytest

from oracle import parallel, solver
from oracle.operators import ODWF
from paper_1710_09621_gb300.inputs import gaussian_spinor5, omega_zolotarev, random_su3_links


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_threaded_schur_equals_serial(threads):
    dims, Ns = (4, 2, 4, 6), 6
    op = ODWF(random_su3_links(dims, 0.4, 3), 1.3, omega_zolotarev(Ns, 0.05, 6.2))
    ser, thr = solver.Schur(op, 0.05, 0.3), parallel.ThreadedSchur(op, 0.05, 0.3, threads=threads)
    v = gaussian_spinor5(dims, Ns, 4) * ser.even
    for f, g in ((ser.S, thr.S), (ser.S_dag, thr.S_dag)):
        a, b = f(v), g(v)
        assert np.linalg.norm(a - b) <= 1e-14 * np.linalg.norm(a)
    thr.close()


def test_bench_cpu_baseline_helpers():
    import bench
    c0 = bench.cpu_oracle_config0()
    assert c0["true_residual"] <= 1e-10 and c0["iters"] > 0 and c0["seconds"] > 0
    s = bench.cpu_oracle_sample(100, dims=(4, 4, 4, 4))
    assert s["threads"] >= 1 and s["t_iter_s"] > 0 and s["value"] == pytest.approx(100 * s["t_iter_s"])
    assert isinstance(bench.cpu_model(), str)
