"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the CPU oracle.

This module draws random numbers and builds input data only: gauge links, Gaussian
noise vectors and the fifth-dimension weights omega_s. It contains none of the
operator, solver or EOFA arithmetic, and it imports nothing from the CUDA binding
or from the oracle.

Array layouts (complex128, C order) are the ones the C ABI takes:
  links      U[mu][t][z][y][x][a][b]          mu = 0..3 for x, y, z, t
  4D spinor  psi[t][z][y][x][spin][color]     spin 0..3, color 0..2
  5D spinor  psi[s][t][z][y][x][spin][color]  s = 0..Ns-1 outermost
"""
from __future__ import annotations

import numpy as np
import scipy.special as sps

__all__ = [
    "gell_mann",
    "random_su3_links",
    "gaussian_spinor",
    "gaussian_spinor5",
    "omega_zolotarev",
    "omega_shamir",
    "seed_for",
]


def seed_for(config: int, instance: int = 0) -> int:
    """Seed convention of the synthetic workloads: 1000 * config + instance."""
    return 1000 * int(config) + int(instance)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda^a (3x3, Hermitian, traceless, tr(l^a l^b) = 2 delta)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0, 0, 1] = l[0, 1, 0] = 1
    l[1, 0, 1], l[1, 1, 0] = -1j, 1j
    l[2, 0, 0], l[2, 1, 1] = 1, -1
    l[3, 0, 2] = l[3, 2, 0] = 1
    l[4, 0, 2], l[4, 2, 0] = -1j, 1j
    l[5, 1, 2] = l[5, 2, 1] = 1
    l[6, 1, 2], l[6, 2, 1] = -1j, 1j
    l[7, 0, 0] = l[7, 1, 1] = 1 / np.sqrt(3)
    l[7, 2, 2] = -2 / np.sqrt(3)
    return l


def random_su3_links(dims, eps: float, seed: int) -> np.ndarray:
    """U_mu(x) = exp(i eps sum_a lambda^a r^a), r^a ~ N(0,1), for every link.

    dims = (Lx, Ly, Lz, Lt). The exponential of the Hermitian traceless matrix is taken
    through its eigen-decomposition, so U is unitary with det U = 1 to rounding.
    Returns shape (4, Lt, Lz, Ly, Lx, 3, 3).
    """
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    r = rng.standard_normal((4, Lt, Lz, Ly, Lx, 8))
    h = np.einsum("...a,aij->...ij", r, gell_mann())
    w, v = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    u = np.einsum("...ia,...a,...ja->...ij", v, ph, v.conj())
    return np.ascontiguousarray(u)


def _complex_gaussian(shape, rng) -> np.ndarray:
    """Complex Gaussian with weight exp(-|z|^2): Re and Im ~ N(0, 1/2)."""
    z = rng.standard_normal(shape + (2,)) * np.sqrt(0.5)
    return np.ascontiguousarray(z[..., 0] + 1j * z[..., 1])


def gaussian_spinor(dims, seed: int) -> np.ndarray:
    """4D spinor eta(x) with weight exp(-eta^dag eta); shape (Lt, Lz, Ly, Lx, 4, 3)."""
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    return _complex_gaussian((Lt, Lz, Ly, Lx, 4, 3), np.random.default_rng(seed))


def gaussian_spinor5(dims, Ns: int, seed: int) -> np.ndarray:
    """5D spinor with weight exp(-eta^dag eta); shape (Ns, Lt, Lz, Ly, Lx, 4, 3)."""
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    return _complex_gaussian((int(Ns), Lt, Lz, Ly, Lx, 4, 3), np.random.default_rng(seed))


def omega_shamir(Ns: int) -> np.ndarray:
    """All omega_s = 1 (the unweighted kernel used by the smallest workload)."""
    return np.ones(int(Ns), dtype=np.float64)


def _zolotarev_inv_sqrt_coeffs(n_num: int, n_den: int, b: float):
    """Zolotarev's optimal rational approximation to 1/sqrt(y) on [1, b].

    Returns (c_num, c_den) with r(y) proportional to prod(1 + y/c_num) / prod(1 + y/c_den).
    Type (n-1, n): c_l = sn^2(l K'/(2n); k') / cn^2(l K'/(2n); k'), l = 1..2n-1,
    odd l in the denominator, even l in the numerator. Type (n, n): the same with 2n+1.
    k'^2 = 1 - 1/b, K' = K(k'). (Zolotarev 1877; Akhiezer, Elements of the theory of
    elliptic functions, ch. on best rational approximation.)
    """
    if n_num == n_den - 1:
        N = 2 * n_den
    elif n_num == n_den:
        N = 2 * n_den + 1
    else:
        raise ValueError("unsupported Zolotarev type")
    m = 1.0 - 1.0 / b  # parameter k'^2
    K = sps.ellipkm1(1.0 / b)
    l = np.arange(1, N)
    sn, cn, dn, _ = sps.ellipj(l * K / N, m)
    c = sn**2 / cn**2
    return c[1::2].copy(), c[0::2].copy()  # even l (numerator), odd l (denominator)


def omega_zolotarev(Ns: int, lmin: float, lmax: float) -> np.ndarray:
    """R5-symmetric fifth-dimension weights from the Zolotarev sign approximation.

    With n = Ns/2 weights w_l, R(x) = (1 - prod T_l)/(1 + prod T_l), T_l = (1 - w_l x)/(1 + w_l x),
    equals O(x)/E(x) where O, E are the odd and even parts of P(x) = prod(1 + w_l x). Choosing
    R as Zolotarev's optimal approximation of sign(x) on [lmin, lmax] fixes P, and the w_l are
    -1/roots of P. Each w_l is used twice, w_s = w_{Ns+1-s}, which makes the Ns-weight
    approximation (1 - prod_s T_s)/(1 + prod_s T_s) = 2R/(1 + R^2) and gives R5 symmetry.
    Returned order: increasing in s for s < Ns/2, mirrored after.
    """
    Ns = int(Ns)
    if Ns % 2 or Ns < 2:
        raise ValueError("Ns must be even")
    n = Ns // 2
    b = (lmax / lmin) ** 2
    if n % 2 == 0:
        c_num, c_den = _zolotarev_inv_sqrt_coeffs(n // 2 - 1, n // 2, b)
    else:
        c_num, c_den = _zolotarev_inv_sqrt_coeffs((n - 1) // 2, (n - 1) // 2, b)

    def unscaled(x):
        y = (x / lmin) ** 2
        num = np.prod(1 + y[:, None] / c_num[None, :], axis=1) if len(c_num) else np.ones_like(y)
        den = np.prod(1 + y[:, None] / c_den[None, :], axis=1)
        return (x / lmin) * num / den

    xs = np.geomspace(lmin, lmax, 200001)
    f = unscaled(xs)
    d = 2.0 / (f.max() + f.min())
    # P(x) = D(x^2) + x N(x^2) with D = prod(1 + x^2/(lmin^2 c_den)), x N = d (x/lmin) prod(...)
    poly_d = np.poly1d([1.0])
    for c in c_den:
        poly_d = poly_d * np.poly1d([1.0 / (lmin**2 * c), 0.0, 1.0])
    poly_n = np.poly1d([d / lmin, 0.0])
    for c in c_num:
        poly_n = poly_n * np.poly1d([1.0 / (lmin**2 * c), 0.0, 1.0])
    roots = (poly_d + poly_n).roots
    if np.max(np.abs(roots.imag)) > 1e-8 * np.max(np.abs(roots)) or np.any(roots.real >= 0):
        raise RuntimeError("Zolotarev polynomial has non-negative-real roots")
    w = np.sort(-1.0 / roots.real)
    # polish each root with Newton on P(-1/w) = 0 in the variable x
    p = poly_d + poly_n
    dp = p.deriv()
    x = -1.0 / w
    for _ in range(3):
        x = x - p(x) / dp(x)
    w = np.sort(-1.0 / x)
    return np.concatenate([w, w[::-1]]).astype(np.float64)
