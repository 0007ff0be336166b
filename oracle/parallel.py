"""The oracle's even-odd Schur operator run on every host core (test and baseline infrastructure).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: used by the CPU-baseline leg of the
benchmark to time the oracle on all cores of the host. It changes no arithmetic: the Wilson hop of
Eq.(DTm1m2) is diagonal in s, so ``ThreadedSchur`` hands contiguous ranges of s-slices to a thread
pool and concatenates the results of the same ``wilson.hop`` / ``wilson.hop_dag`` calls the serial
oracle makes; the fifth-dimension products act site by site, so they are split over ranges of t.
numpy releases the interpreter lock inside these array operations, so the threads run in parallel.
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np

from .operators import chiral_s_mul
from .solver import Schur
from .wilson import hop, hop_dag


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


class ThreadedSchur(Schur):
    """Schur complement S of D_T(m1, m2) (see solver.Schur) with its array work spread over threads."""

    def __init__(self, op, m1, m2, threads=None):
        super().__init__(op, m1, m2)
        self.threads = int(threads or host_cores())
        self.pool = cf.ThreadPoolExecutor(self.threads)

    def close(self):
        self.pool.shutdown()

    def _chunks(self, n):
        k = min(self.threads, n)
        return [slice(i * n // k, (i + 1) * n // k) for i in range(k)]

    def _over_s(self, fn, v):
        parts = list(self.pool.map(lambda sl: fn(self.op.U, v[sl]), self._chunks(v.shape[0])))
        return np.concatenate(parts, axis=0)

    def _over_t(self, Mp, Mm, v):
        out = np.empty_like(v)

        def work(sl):
            out[:, sl] = chiral_s_mul(Mp, Mm, v[:, sl])
        list(self.pool.map(work, self._chunks(v.shape[1])))
        return out

    def hop_to(self, v, target):
        return target * self._over_s(hop, v)

    def A(self, v):
        return self._over_t(self.Ap, self.Am, v)

    def Ainv(self, v):
        return self._over_t(self.Apinv, self.Aminv, v)

    def S_dag(self, ye):
        t = self._over_t(self.Apinv.T, self.Aminv.T, self.odd * self._over_s(hop_dag, ye))
        return self._over_t(self.Ap.T, self.Am.T, ye) - 0.25 * self.even * self._over_s(hop_dag, t)
