"""Rational approximation of x^{-1/2} for the pseudofermion heat-bath (oracle, FP64).

Eq.(CG_gaussian) generates phi from Gaussian noise eta by solving H^{-1/2} phi = eta, and the
paper suppresses how (Section 1). The reading used: phi = X^{-1/2} eta with X the term's 4D
operator, and X^{-1/2} ~ a0 + sum_l a_l / (X + b_l), Zolotarev's optimal (n, n) rational
approximation of 1/sqrt(x) on [x_lo, x_hi] in partial fractions. Each pole is then one
shifted-mass 5D solve (eofa.py).

Zolotarev's construction (Zolotarev 1877; Akhiezer, "Elements of the Theory of Elliptic
Functions"): on y in [1, b], k'^2 = 1 - 1/b, K' = K(k'),
    c_l = sn^2(l K'/(2n+1); k') / cn^2(l K'/(2n+1); k'),  l = 1..2n,
    r(y) = d prod_{l=1..n} (y + c_{2l}) / prod_{l=1..n} (y + c_{2l-1})  (up to constants),
with d fixed so that sqrt(y) r(y) - 1 equi-oscillates around zero.
"""
from __future__ import annotations

import numpy as np
import scipy.special as sps


class InvSqrtRational:
    def __init__(self, a0, a, b, x_lo, x_hi, err):
        self.a0 = float(a0)
        self.a = np.asarray(a, dtype=np.float64)
        self.b = np.asarray(b, dtype=np.float64)
        self.x_lo, self.x_hi, self.err = float(x_lo), float(x_hi), float(err)

    def __call__(self, x):
        x = np.asarray(x, dtype=np.float64)
        return self.a0 + np.sum(self.a[:, None] / (x[None, :] + self.b[:, None]), axis=0)

    @property
    def n_poles(self):
        return len(self.a)


def zolotarev_inv_sqrt(n, x_lo, x_hi):
    """(n, n) Zolotarev approximation of 1/sqrt(x) on [x_lo, x_hi] as a0 + sum a_l/(x + b_l)."""
    bb = x_hi / x_lo
    N = 2 * n + 1
    m = 1.0 - 1.0 / bb
    K = sps.ellipkm1(1.0 / bb)
    l = np.arange(1, N)
    sn, cn, _, _ = sps.ellipj(l * K / N, m)
    c = sn**2 / cn**2
    c_num, c_den = c[1::2], c[0::2]  # even l: zeros at -c, odd l: poles at -c

    def unscaled(y):
        y = np.asarray(y, dtype=np.float64)
        num = np.prod(y[:, None] + c_num[None, :], axis=1)
        den = np.prod(y[:, None] + c_den[None, :], axis=1)
        return num / den

    ys = np.geomspace(1.0, bb, 400001)
    f = np.sqrt(ys) * unscaled(ys)
    d = 2.0 / (f.max() + f.min())
    # partial fractions of d prod(y + c_num)/prod(y + c_den): constant d plus residues
    res = np.empty(n)
    for j in range(n):
        y0 = -c_den[j]
        num = np.prod(y0 + c_num)
        den = np.prod([y0 + c_den[i] for i in range(n) if i != j])
        res[j] = d * num / den
    # back to x = x_lo y:  x^{-1/2} = x_lo^{-1/2} r(x / x_lo)
    a0 = d / np.sqrt(x_lo)
    a = res * np.sqrt(x_lo)
    b = c_den * x_lo
    approx = InvSqrtRational(a0, a, b, x_lo, x_hi, 0.0)
    xs = np.geomspace(x_lo, x_hi, 200001)
    approx.err = float(np.max(np.abs(1.0 - np.sqrt(xs) * approx(xs))))
    return approx


def inv_sqrt_for_error(x_lo, x_hi, target=1e-11, n_max=64):
    """Smallest-n Zolotarev approximation with max relative error <= target."""
    for n in range(1, n_max + 1):
        r = zolotarev_inv_sqrt(n, x_lo, x_hi)
        if r.err <= target:
            return r
    raise RuntimeError("no Zolotarev approximation reached the target error")
