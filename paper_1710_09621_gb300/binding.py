"""Thin ctypes binding of libodwf.so (argument marshalling only).

Every step of the hot path runs in the library's CUDA kernels; this module converts torch
tensors to device pointers and streams, checks shapes and dtypes, and turns status codes into
exceptions. There is no CPU fallback: if the library is missing or no GPU is present the calls
raise.

Field tensors are torch.complex128 CUDA tensors in the ABI layout (see include/odwf.h):
  links (4, Lt, Lz, Ly, Lx, 3, 3), 4D spinor (Lt, Lz, Ly, Lx, 4, 3),
  5D spinor (Ns, Lt, Lz, Ly, Lx, 4, 3), force (4, Lt, Lz, Ly, Lx, 8) float64.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libodwf.so")

ODWF_OK, ODWF_EINVAL, ODWF_ENOMEM, ODWF_ECUDA, ODWF_ENOCONV, ODWF_EBREAKDOWN, ODWF_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
ODWF_EFAULT, ODWF_ESPECTRUM = -7, -8
PREC_DOUBLE, PREC_SINGLE, PREC_HALF = 0, 1, 2
OP_DT, OP_HT, OP_DODWF = 0, 1, 2
_PREC = {"double": PREC_DOUBLE, "single": PREC_SINGLE, "half": PREC_HALF,
         PREC_DOUBLE: PREC_DOUBLE, PREC_SINGLE: PREC_SINGLE, PREC_HALF: PREC_HALF}
_OP = {"dt": OP_DT, "ht": OP_HT, "dodwf": OP_DODWF, OP_DT: OP_DT, OP_HT: OP_HT, OP_DODWF: OP_DODWF}

# every entry point the C ABI declares
EXPORTS = ["odwf_create", "odwf_destroy", "odwf_last_error", "odwf_set_gauge", "odwf_apply", "odwf_apply_dag",
           "eofa_solve", "eofa_solve_batch", "eofa_action", "eofa_force", "eofa_heatbath", "eofa_k",
           "odwf_omega_vector", "odwf_profile_enable", "odwf_profile_read", "eofa_mp_terms",
           "odwf_apply_noalloc", "eofa_solve_multi", "odwf_net_create", "odwf_net_destroy",
           "odwf_net_num_params", "odwf_net_weights", "odwf_net_apply", "odwf_net_set_pairs", "odwf_net_loss_grad",
           "odwf_net_train", "eofa_solve_learned", "odwf_autotune", "eofa_solve_gcr", "eofa_term_spectrum",
           "hmc_gauge_action", "hmc_gauge_force", "hmc_momentum_update", "hmc_link_update", "hmc_kinetic",
           "hmc_md", "odwf_autotune_cache", "odwf_net_set_loss", "odwf_set_preconditioner", "odwf_fp64_fma_peak"]


class OdwfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"odwf error {code}: {msg}")
        self.code = code


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("prec", ctypes.c_int),
                ("delta", ctypes.c_double), ("max_seconds", ctypes.c_double)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {"iters": self.iters, "reliable_updates": self.reliable_updates,
                "true_residual": self.true_residual, "seconds": self.seconds}


class Term(ctypes.Structure):
    _fields_ = [("chirality", ctypes.c_int), ("m3", ctypes.c_double), ("m4", ctypes.c_double),
                ("m_den", ctypes.c_double)]


class HbOpts(ctypes.Structure):
    _fields_ = [("solve", SolveOpts), ("x_lo", ctypes.c_double), ("x_hi", ctypes.c_double),
                ("rat_err", ctypes.c_double), ("n_poles_out", ctypes.c_int), ("iters_out", ctypes.c_int),
                ("check_iters", ctypes.c_int), ("ritz_lo_out", ctypes.c_double), ("ritz_hi_out", ctypes.c_double)]


HMC_MAX_LEVELS = 4
OMELYAN_LAMBDA = 0.1931833275037836


class HmcStats(ctypes.Structure):
    _fields_ = [("dH", ctypes.c_double), ("K0", ctypes.c_double), ("K1", ctypes.c_double),
                ("Sg0", ctypes.c_double), ("Sg1", ctypes.c_double), ("Sf0", ctypes.c_double), ("Sf1", ctypes.c_double),
                ("force_evals", ctypes.c_int * HMC_MAX_LEVELS), ("link_updates", ctypes.c_int),
                ("cg_iters", ctypes.c_longlong), ("seconds", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k in ("dH", "K0", "K1", "Sg0", "Sg1", "Sf0", "Sf1", "link_updates", "cg_iters",
                                           "seconds")}
        d["force_evals"] = list(self.force_evals)
        return d


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libodwf.so once; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with `python -m paper_1710_09621_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, dp, ip, d, i = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_int
    lib.odwf_create.argtypes = [ctypes.POINTER(vp), ip, i, d, dp, i]
    lib.odwf_destroy.argtypes = [vp]
    lib.odwf_last_error.argtypes = [vp]
    lib.odwf_last_error.restype = ctypes.c_char_p
    lib.odwf_set_gauge.argtypes = [vp, vp, vp]
    lib.odwf_apply.argtypes = [vp, i, d, d, vp, vp, i, vp]
    lib.odwf_apply_dag.argtypes = [vp, i, d, d, vp, vp, i, vp]
    lib.eofa_solve.argtypes = [vp, d, d, vp, vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), vp]
    lib.eofa_solve_batch.argtypes = [vp, i, dp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), vp]
    lib.eofa_action.argtypes = [vp, ctypes.POINTER(Term), vp, dp, ctypes.POINTER(SolveOpts),
                                ctypes.POINTER(SolveStats), vp]
    lib.eofa_force.argtypes = [vp, ctypes.POINTER(Term), vp, vp, ctypes.POINTER(SolveOpts),
                               ctypes.POINTER(SolveStats), vp]
    lib.eofa_heatbath.argtypes = [vp, ctypes.POINTER(Term), vp, vp, ctypes.POINTER(HbOpts), vp]
    lib.eofa_term_spectrum.argtypes = [vp, ctypes.POINTER(Term), vp, i, dp, dp, ctypes.POINTER(SolveOpts), vp]
    lib.hmc_gauge_action.argtypes = [vp, vp, d, dp, vp]
    lib.hmc_gauge_force.argtypes = [vp, vp, d, vp, vp]
    lib.hmc_momentum_update.argtypes = [vp, vp, vp, d, vp]
    lib.hmc_link_update.argtypes = [vp, vp, vp, d, vp]
    lib.hmc_kinetic.argtypes = [vp, vp, dp, vp]
    lib.hmc_md.argtypes = [vp, vp, vp, d, i, ctypes.POINTER(Term), ctypes.POINTER(vp), ip, i, ip, d, d,
                           ctypes.POINTER(SolveOpts), ctypes.POINTER(HmcStats), vp]
    lib.eofa_k.argtypes = [d, d]
    lib.eofa_k.restype = d
    lib.odwf_omega_vector.argtypes = [vp, i, dp]
    lib.odwf_fp64_fma_peak.argtypes = [vp, dp, vp]
    lib.odwf_profile_enable.argtypes = [vp, i]
    lib.odwf_profile_read.argtypes = [vp, ip, ip, dp, ip]
    lib.eofa_mp_terms.argtypes = [i, d, dp, i, d, i, ctypes.POINTER(Term), i, ip]
    lib.odwf_apply_noalloc.argtypes = [vp, i, d, d, vp, vp, i, vp]
    lib.odwf_autotune.argtypes = [vp, i, ctypes.c_char_p, i, vp]
    lib.odwf_autotune_cache.argtypes = [vp, i, ctypes.c_char_p, ip, vp]
    lib.odwf_net_create.argtypes = [vp, i, ctypes.POINTER(vp)]
    lib.odwf_net_destroy.argtypes = [vp]
    lib.odwf_net_num_params.argtypes = [vp]
    lib.odwf_net_weights.argtypes = [vp, dp, i]
    lib.odwf_net_apply.argtypes = [vp, d, d, vp, vp, i, vp]
    lib.odwf_net_set_pairs.argtypes = [vp, d, d, i, ctypes.POINTER(vp), ctypes.POINTER(vp), d, vp]
    lib.odwf_net_loss_grad.argtypes = [vp, dp, dp, vp]
    lib.odwf_net_set_loss.argtypes = [vp, i]
    lib.odwf_set_preconditioner.argtypes = [vp, vp]
    lib.odwf_net_train.argtypes = [vp, i, d, dp, vp]
    lib.eofa_solve_learned.argtypes = [vp, vp, d, d, vp, vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), vp]
    lib.eofa_solve_gcr.argtypes = [vp, vp, d, d, vp, vp, i, i, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), vp]
    lib.eofa_solve_multi.argtypes = [ctypes.POINTER(vp), i, dp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), vp]
    _lib = lib
    return lib


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def solve_opts(tol=1e-10, maxiter=100000, prec="double", delta=0.1, max_seconds=0.0):
    return SolveOpts(tol, maxiter, _PREC[prec], delta, max_seconds)


@dataclass
class TermSpec:
    chirality: int
    m3: float
    m4: float
    m_den: float

    def c(self):
        return Term(int(self.chirality), float(self.m3), float(self.m4), float(self.m_den))


class ODWF:
    """One lattice: dims (Lx, Ly, Lz, Lt), Ns, m0 and the R5-symmetric weights omega_s."""

    def __init__(self, dims, Ns, m0, omega):
        import numpy as np
        self.lib = load_library()
        self.dims = tuple(int(x) for x in dims)
        self.Ns = int(Ns)
        self.m0 = float(m0)
        om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
        if om.shape != (self.Ns,):
            raise ValueError("omega must have Ns entries")
        h = ctypes.c_void_p()
        d = (ctypes.c_int * 4)(*self.dims)
        rc = self.lib.odwf_create(ctypes.byref(h), d, self.Ns, self.m0,
                                  om.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
        if rc != 0:
            raise OdwfError(rc, self.lib.odwf_last_error(None).decode())
        self.h = h
        Lx, Ly, Lz, Lt = self.dims
        self.shape4 = (Lt, Lz, Ly, Lx, 4, 3)
        self.shape5 = (self.Ns,) + self.shape4
        self.shape_links = (4, Lt, Lz, Ly, Lx, 3, 3)
        self.shape_force = (4, Lt, Lz, Ly, Lx, 8)

    def close(self):
        if getattr(self, "h", None):
            self.lib.odwf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != 0 and rc not in allow:
            raise OdwfError(rc, self.lib.odwf_last_error(self.h).decode())
        return rc

    @staticmethod
    def _field(t, shape, dtype=None):
        import torch
        dtype = dtype or torch.complex128
        if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and tuple(t.shape) == tuple(shape)):
            raise ValueError(f"expected contiguous CUDA {dtype} tensor of shape {shape}, got "
                             f"{t.dtype} {tuple(t.shape)} on {t.device}")
        return t

    def set_gauge(self, U, stream=None):
        self._check(self.lib.odwf_set_gauge(self.h, _ptr(self._field(U, self.shape_links)), _stream_ptr(stream)))

    def apply(self, x, m1, m2, op="dt", dag=False, prec="double", out=None, stream=None):
        import torch
        self._field(x, self.shape5)
        out = torch.empty_like(x) if out is None else self._field(out, self.shape5)
        fn = self.lib.odwf_apply_dag if dag else self.lib.odwf_apply
        self._check(fn(self.h, _OP[op], float(m1), float(m2), _ptr(x), _ptr(out), _PREC[prec], _stream_ptr(stream)))
        return out

    def solve(self, b, m1, m2, x=None, opts=None, stream=None, allow_noconv=False):
        """x = H_T(m1, m2)^{-1} b; returns (x, stats dict). With allow_noconv a solve that stops above
        tol (maxiter or max_seconds) returns its last iterate with "status" instead of raising."""
        import torch
        self._field(b, self.shape5)
        x = torch.empty_like(b) if x is None else self._field(x, self.shape5)
        st = SolveStats()
        o = opts if opts is not None else solve_opts()
        rc = self.lib.eofa_solve(self.h, float(m1), float(m2), _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(st),
                                 _stream_ptr(stream))
        self._check(rc, allow=(ODWF_ENOCONV, ODWF_ETIMEOUT) if allow_noconv else ())
        d = st.as_dict()
        d["status"] = rc
        return x, d

    def solve_gcr(self, b, m1, m2, net=None, nvec=8, truncate=False, opts=None, stream=None, allow_noconv=False):
        """x = H_T(m1, m2)^{-1} b by flexible GCR on S, right-preconditioned by `net` (a Net, or None
        for plain GCR), with a basis of nvec directions (restarted, or a sliding window when
        truncate); returns (x, stats dict). With allow_noconv, a solve that ends above tol (maxiter or
        max_seconds) returns its stats with "status" instead of raising."""
        import torch
        self._field(b, self.shape5)
        x = torch.empty_like(b)
        st = SolveStats()
        o = opts if opts is not None else solve_opts(prec="single", delta=1e-3)
        rc = self.lib.eofa_solve_gcr(self.h, net.n if net is not None else None, float(m1), float(m2), _ptr(b),
                                     _ptr(x), int(nvec), int(bool(truncate)), ctypes.byref(o), ctypes.byref(st),
                                     _stream_ptr(stream))
        self._check(rc, allow=(ODWF_ENOCONV, ODWF_ETIMEOUT) if allow_noconv else ())
        d = st.as_dict()
        d["status"] = rc
        return x, d

    def solve_batch(self, bs, m12, opts=None, stream=None):
        import torch
        n = len(bs)
        xs = [torch.empty_like(b) for b in bs]
        for b in bs:
            self._field(b, self.shape5)
        arr = (ctypes.c_double * (2 * n))(*[float(v) for pair in m12 for v in pair])
        bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        st = (SolveStats * n)()
        o = opts if opts is not None else solve_opts()
        self._check(self.lib.eofa_solve_batch(self.h, n, arr, bp, xp, ctypes.byref(o), st, _stream_ptr(stream)))
        return xs, [s.as_dict() for s in st]

    def action(self, term: TermSpec, phi, opts=None, stream=None):
        self._field(phi, self.shape4)
        S = ctypes.c_double()
        st = SolveStats()
        o = opts if opts is not None else solve_opts()
        t = term.c()
        self._check(self.lib.eofa_action(self.h, ctypes.byref(t), _ptr(phi), ctypes.byref(S), ctypes.byref(o),
                                         ctypes.byref(st), _stream_ptr(stream)))
        return S.value, st.as_dict()

    def force(self, term: TermSpec, phi, opts=None, out=None, stream=None):
        import torch
        self._field(phi, self.shape4)
        F = torch.empty(self.shape_force, dtype=torch.float64, device=phi.device) if out is None else out
        self._field(F, self.shape_force, torch.float64)
        st = SolveStats()
        o = opts if opts is not None else solve_opts()
        t = term.c()
        self._check(self.lib.eofa_force(self.h, ctypes.byref(t), _ptr(phi), _ptr(F), ctypes.byref(o),
                                        ctypes.byref(st), _stream_ptr(stream)))
        return F, st.as_dict()

    def heatbath(self, term: TermSpec, eta, opts=None, x_lo=0.0, x_hi=1.0, rat_err=1e-11, check_iters=0,
                 stream=None):
        """phi = X^{-1/2} eta; with check_iters > 0 the spectrum of X is first estimated by Lanczos and
        an interval [x_lo, x_hi] that does not contain the Ritz values raises ODWF_ESPECTRUM."""
        import torch
        self._field(eta, self.shape4)
        phi = torch.empty_like(eta)
        hb = HbOpts(opts if opts is not None else solve_opts(), x_lo, x_hi, rat_err, 0, 0, int(check_iters), 0.0, 0.0)
        t = term.c()
        self._check(self.lib.eofa_heatbath(self.h, ctypes.byref(t), _ptr(eta), _ptr(phi), ctypes.byref(hb),
                                           _stream_ptr(stream)))
        info = {"n_poles": hb.n_poles_out, "iters": hb.iters_out}
        if check_iters > 0:
            info["ritz"] = (hb.ritz_lo_out, hb.ritz_hi_out)
        return phi, info

    def term_spectrum(self, term: TermSpec, v0, n_iter=12, opts=None, stream=None):
        """(smallest, largest) Ritz value of the term's operator X after n_iter Lanczos steps from P v0."""
        self._field(v0, self.shape4)
        lo, hi = ctypes.c_double(), ctypes.c_double()
        o = opts if opts is not None else solve_opts()
        t = term.c()
        self._check(self.lib.eofa_term_spectrum(self.h, ctypes.byref(t), _ptr(v0), int(n_iter), ctypes.byref(lo),
                                                ctypes.byref(hi), ctypes.byref(o), _stream_ptr(stream)))
        return lo.value, hi.value

    # ---- HMC molecular dynamics (momenta / forces: float64 tensors of shape_force) --------------
    def gauge_action(self, U, beta, stream=None):
        S = ctypes.c_double()
        self._check(self.lib.hmc_gauge_action(self.h, _ptr(self._field(U, self.shape_links)), float(beta),
                                              ctypes.byref(S), _stream_ptr(stream)))
        return S.value

    def gauge_force(self, U, beta, stream=None):
        import torch
        F = torch.empty(self.shape_force, dtype=torch.float64, device=U.device)
        self._check(self.lib.hmc_gauge_force(self.h, _ptr(self._field(U, self.shape_links)), float(beta), _ptr(F),
                                             _stream_ptr(stream)))
        return F

    def momentum_update(self, P, F, eps, stream=None):
        import torch
        self._field(P, self.shape_force, torch.float64)
        self._field(F, self.shape_force, torch.float64)
        self._check(self.lib.hmc_momentum_update(self.h, _ptr(P), _ptr(F), float(eps), _stream_ptr(stream)))

    def link_update(self, U, P, tau, stream=None):
        """U <- exp(i tau P) U in place (and the library's copies of U follow)."""
        import torch
        self._field(U, self.shape_links)
        self._field(P, self.shape_force, torch.float64)
        self._check(self.lib.hmc_link_update(self.h, _ptr(U), _ptr(P), float(tau), _stream_ptr(stream)))

    def kinetic(self, P, stream=None):
        import torch
        K = ctypes.c_double()
        self._check(self.lib.hmc_kinetic(self.h, _ptr(self._field(P, self.shape_force, torch.float64)),
                                         ctypes.byref(K), _stream_ptr(stream)))
        return K.value

    def md(self, U, P, beta, terms, phis, levels, steps, tau=1.0, lam=OMELYAN_LAMBDA, opts=None, stream=None):
        """One MD trajectory (nested Omelyan, multiple time scales): U, P updated in place; returns stats."""
        import torch
        self._field(U, self.shape_links)
        self._field(P, self.shape_force, torch.float64)
        n = len(terms)
        tarr = (Term * max(1, n))(*[t.c() for t in terms])
        parr = (ctypes.c_void_p * max(1, n))(*[self._field(p, self.shape4).data_ptr() for p in phis])
        larr = (ctypes.c_int * max(1, n))(*[int(l) for l in levels])
        sarr = (ctypes.c_int * len(steps))(*[int(k) for k in steps])
        st = HmcStats()
        o = opts if opts is not None else solve_opts()
        self._check(self.lib.hmc_md(self.h, _ptr(U), _ptr(P), float(beta), n, tarr, parr, larr, len(steps), sarr,
                                    float(tau), float(lam), ctypes.byref(o), ctypes.byref(st), _stream_ptr(stream)))
        return st.as_dict()

    def autotune(self, prec="single", stream=None):
        """Pick the fastest launch choice of each fused CGNE kernel; returns the timing report."""
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(self.lib.odwf_autotune(self.h, _PREC[prec], buf, 1 << 16, _stream_ptr(stream)))
        return buf.value.decode()

    def fp64_fma_peak(self, stream=None):
        """Measured FP64 FMA throughput of the device (TFLOP/s)."""
        t = ctypes.c_double()
        self._check(self.lib.odwf_fp64_fma_peak(self.h, ctypes.byref(t), _stream_ptr(stream)))
        return t.value

    def set_preconditioner(self, net):
        """Attach a Net (or None) for the solves of action, force and the MD trajectory."""
        self._check(self.lib.odwf_set_preconditioner(self.h, net.n if net is not None else None))
        self._net = net  # keep it alive while attached

    def autotune_cached(self, path, prec="single", stream=None):
        """Apply the choices stored in `path` for this device, lattice and precision, or tune and append
        them; returns True on a cache hit."""
        hit = ctypes.c_int(0)
        self._check(self.lib.odwf_autotune_cache(self.h, _PREC[prec], str(path).encode(), ctypes.byref(hit),
                                                 _stream_ptr(stream)))
        return bool(hit.value)

    def profile(self, enable=True):
        self._check(self.lib.odwf_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self):
        """{kernel key: (launches, total ms)} of the fused hopping kernels since profile(True)."""
        n = ctypes.c_int(64)
        keys = (ctypes.c_int * 64)()
        cnt = (ctypes.c_int * 64)()
        ms = (ctypes.c_double * 64)()
        self._check(self.lib.odwf_profile_read(self.h, keys, cnt, ms, ctypes.byref(n)))
        return {keys[i]: (cnt[i], ms[i]) for i in range(min(n.value, 64))}

    def omega_vector(self, chirality):
        out = (ctypes.c_double * self.Ns)()
        self._check(self.lib.odwf_omega_vector(self.h, int(chirality), out))
        return list(out)


MP_NONE, MP_OLD, MP_NEW = 0, 1, 2


def mp_terms(scheme, m, mh, M, parity=False):
    """Term list of a mass-preconditioning scheme (Eq.(noMP), Eq.(old_MP_N), Eq.(new_MP_N))."""
    lib = load_library()
    mh = list(mh)
    arr = (ctypes.c_double * max(1, len(mh)))(*mh)
    out = (Term * 64)()
    n = ctypes.c_int(0)
    rc = lib.eofa_mp_terms(int(scheme), float(m), arr, len(mh), float(M), 1 if parity else 0, out, 64, ctypes.byref(n))
    if rc != 0:
        raise OdwfError(rc, "eofa_mp_terms: invalid scheme or masses")
    return [TermSpec(out[i].chirality, out[i].m3, out[i].m4, out[i].m_den) for i in range(n.value)]


class Net:
    """Learned preconditioner of one lattice (see include/odwf.h); weights as complex numpy arrays."""

    def __init__(self, lat, channels=2):
        self.lat = lat
        self.lib = lat.lib
        n = ctypes.c_void_p()
        lat._check(self.lib.odwf_net_create(lat.h, int(channels), ctypes.byref(n)))
        self.n = n
        self.C = int(channels)
        self.P = self.lib.odwf_net_num_params(n)

    def close(self):
        if getattr(self, "n", None):
            self.lib.odwf_net_destroy(self.n)
            self.n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_weights(self):
        import numpy as np
        buf = np.zeros(2 * self.P, dtype=np.float64)
        self.lat._check(self.lib.odwf_net_weights(self.n, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0))
        return buf.view(np.complex128).copy()

    def set_weights(self, w):
        import numpy as np
        buf = np.ascontiguousarray(np.asarray(w, dtype=np.complex128).reshape(-1)).view(np.float64)
        if buf.size != 2 * self.P:
            raise ValueError("wrong number of parameters")
        self.lat._check(self.lib.odwf_net_weights(self.n, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1))

    def apply(self, r, m1, m2, adjoint=False, stream=None):
        import torch
        self.lat._field(r, self.lat.shape5)
        out = torch.empty_like(r)
        self.lat._check(self.lib.odwf_net_apply(self.n, float(m1), float(m2), _ptr(r), _ptr(out), 1 if adjoint else 0,
                                                _stream_ptr(stream)))
        return out

    def set_pairs(self, rs, m1, m2, es=None, tol=1e-8, stream=None):
        n = len(rs)
        rp = (ctypes.c_void_p * n)(*[r.data_ptr() for r in rs])
        ep = (ctypes.c_void_p * n)(*[e.data_ptr() for e in es]) if es is not None else None
        self.lat._check(self.lib.odwf_net_set_pairs(self.n, float(m1), float(m2), n, rp, ep, float(tol),
                                                    _stream_ptr(stream)))

    def set_loss(self, mode):
        """"error" (|M r - e|^2/|e|^2, default) or "residual" (|S M r - r|^2/|r|^2)."""
        self.lat._check(self.lib.odwf_net_set_loss(self.n, {"error": 0, "residual": 1}[mode]))

    def loss_grad(self, stream=None):
        import numpy as np
        L = ctypes.c_double()
        g = np.zeros(2 * self.P, dtype=np.float64)
        self.lat._check(self.lib.odwf_net_loss_grad(self.n, ctypes.byref(L), g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                    _stream_ptr(stream)))
        return L.value, g.view(np.complex128).copy()

    def train(self, steps, lr, stream=None):
        import numpy as np
        losses = np.zeros(steps + 1)
        self.lat._check(self.lib.odwf_net_train(self.n, int(steps), float(lr),
                                                losses.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream_ptr(stream)))
        return losses

    def solve(self, b, m1, m2, opts=None, stream=None):
        import torch
        self.lat._field(b, self.lat.shape5)
        x = torch.empty_like(b)
        st = SolveStats()
        o = opts if opts is not None else solve_opts(prec="single", delta=1e-3)
        self.lat._check(self.lib.eofa_solve_learned(self.lat.h, self.n, float(m1), float(m2), _ptr(b), _ptr(x),
                                                    ctypes.byref(o), ctypes.byref(st), _stream_ptr(stream)))
        return x, st.as_dict()


def solve_multi(lats, bs, m12, opts=None, stream=None):
    """Solve H_T on several lattices (same Ns) in lockstep; returns (xs, stats list)."""
    import torch
    lib = load_library()
    n = len(lats)
    xs = [torch.empty_like(b) for b in bs]
    for lat, b in zip(lats, bs):
        lat._field(b, lat.shape5)
    hs = (ctypes.c_void_p * n)(*[lat.h.value for lat in lats])
    arr = (ctypes.c_double * (2 * n))(*[float(v) for pair in m12 for v in pair])
    bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    st = (SolveStats * n)()
    o = opts if opts is not None else solve_opts()
    rc = lib.eofa_solve_multi(hs, n, arr, bp, xp, ctypes.byref(o), st, _stream_ptr(stream))
    if rc != 0:
        raise OdwfError(rc, lib.odwf_last_error(lats[0].h).decode())
    return xs, [s.as_dict() for s in st]


def eofa_k(mj, mi):
    return load_library().eofa_k(float(mj), float(mi))
