#!/usr/bin/env python3
"""Benchmark: EOFA CG time-to-1e-10 on one GB300 (and replicas on N GPUs).

Workload (one step = one solve H_T(m, m) x = b to an FP64 true residual of 1e-10):
  16^3 x 32 lattice, Ns = 16 optimal domain-wall weights (Zolotarev, lambda in [0.05, 6.2]),
  m0 = 1.3, normalised mass m = 0.01, seeded SU(3) links U = exp(i 0.3 sum lambda^a r^a),
  Gaussian 5D right-hand side b. Inputs are synthetic (the paper's thermalised ensembles are
  not available). The chosen method (FP32 or FP16-storage inner CGNE with FP64 reliable updates)
  is timed; the plain FP64 GPU CGNE on the same system is timed once beside it.

Output: one JSON line (rank 0). `value` = seconds per solve over the whole job (K solves per
rank, all ranks, max-over-ranks wall time / total solves). Multi-GPU runs are independent
replicas (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import resource
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EOFA CG time-to-1e-10 (chosen vs plain FP64 on GPU); dslash HBM GB/s"
WORKLOAD = {"workload": "16^3x32 Ns=16 optimal DWF (Zolotarev omega on [0.05,6.2]), m0=1.3, m=0.01, "
                        "links eps=0.3, H_T(m,m) x = b to true residual 1e-10",
            "dims": [16, 16, 16, 32], "Ns": 16, "m0": 1.3, "mass": 0.01, "tol": 1e-10}
DIMS, NS, M0, MASS, EPS, TOL = (16, 16, 16, 32), 16, 1.3, 0.01, 0.3, 1e-10
# flop conventions per 5D half-site: the spin-projected Wilson hop (8 directions x [12 projection +
# 2 x 66 SU(3) matrix-vector + 24 accumulation] - 24), the structured fifth-dimension solve, and one
# CGNE iteration (4 hops + 4 fifth-dimension solves + 5 BLAS-1 updates x, r, |r|^2, p, |p|^2 of 24
# reals at 2 flops each)
HOP_FLOPS, FIFTH_FLOPS = 1320, 240
CG_ITER_FLOPS = 4 * HOP_FLOPS + 4 * FIFTH_FLOPS + 5 * 2 * 24


def reduce_max(value, dist=None, device="cpu"):
    """Max of a per-rank float over all ranks (the slowest replica sets the job's time)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def per_solve_seconds(max_elapsed, steps, world):
    """Whole-job seconds per solve: every rank solves `steps` systems in `max_elapsed` seconds."""
    return max_elapsed / (steps * world)


def average_plaquette(U):
    """Average plaquette Re tr(U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag) / 3 of a link array
    [mu][t][z][y][x][3][3] (periodic links): the statistic that characterises a synthetic gauge field."""
    import numpy as np
    axis = {0: 3, 1: 2, 2: 1, 3: 0}  # site axis of direction mu within U[mu]
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            a = U[mu] @ np.roll(U[nu], -1, axis=axis[mu])
            b = U[nu] @ np.roll(U[mu], -1, axis=axis[nu])
            tot += np.sum(a * b.conj()).real / (3.0 * a[..., 0, 0].size)  # tr(a b^dag)
    return tot / 6.0


def dram_traffic(kernel, dims, ns):
    """ncu-measured DRAM bytes per launch of `kernel` on this lattice, or None if not captured."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    for e in json.load(open(p))["entries"]:
        if e["kernel"] == kernel and tuple(e["dims"]) == tuple(dims) and e["Ns"] == ns:
            return e["dram_read_bytes"] + e["dram_write_bytes"]
    return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.samples.append([x.strip() for x in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if len(s) > 5 + i and s[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# algorithmic bytes per launch of the fused hopping kernels (per 5D half-site: spinor reads and
# writes of 24 reals, links 8 x 18 reals per 4D half-site shared by Ns slices; 8 x 12 for the two-slice
# kernels, which store two rows of each SU(3) link)
def alg_bytes(key, Vh, Ns):
    if key >= 4000000:  # layout / vector kernels: kind, first and second storage (0 FP64, 1 FP32, 2 FP16)
        kind, s1, s2 = (key // 100) % 10, (key // 10) % 10, key % 10
        n5 = Vh * Ns
        fb = {0: 192, 1: 96, 2: 52}  # bytes per 5D half-site (FP16 with its per-site scale)
        if kind in (1, 2):           # both parities, ABI FP64 <-> internal
            return 2 * n5 * (fb[s1] + fb[s2])
        if kind == 3:
            return n5 * (fb[s1] + fb[s2])
        if kind == 4:                # read x, read and write y (FP64)
            return n5 * (fb[s1] + 2 * 192)
        return n5 * fb[s1]
    if key >= 3000000:  # GCR step kernels (FP32 half fields of Vh Ns 96 bytes)
        kind, k = (key // 100) % 10, key % 100
        fld = Vh * Ns * 96
        return {1: (k + 2) * fld, 2: 0, 3: (2 * k + 8) * fld}[kind]
    if key >= 2000000:  # learned-preconditioner layer: cin inputs, cout outputs, optional own field
        bf16, cin, cout, own = (key // 1000) % 10, (key // 100) % 10, (key // 10) % 10, key % 10
        # FP32 fields of 96 bytes per 5D half-site; with BF16 intermediates the 1 -> 2 layer writes and
        # the 2 -> 1 layer reads 48-byte BF16 rows per channel
        fin = 48 if (bf16 and cin == 2) else 96
        fout = 48 if (bf16 and cout == 2) else 96
        return Vh * Ns * (fin * cin + fout * cout + 96 * own) + Vh * 8 * 18 * 4
    st = (key // 100000) % 10
    pair = st >= 5                     # two-slice kernels: links stored as two rows (12 reals)
    st -= 5 if pair else 0
    hop, mixhop, own, mixown, epi = (key // 10000) % 10, (key // 1000) % 10, (key // 100) % 10, (key // 10) % 10, key % 10
    rb = {0: 8, 1: 4, 2: 2}[st]        # bytes per real of the spinor storage
    lb = 8 if st == 0 else 4           # link storage
    scale = 4 if st == 2 else 0        # FP16 per-site scale per field access
    n5 = Vh * Ns
    fields = 0
    if hop:
        fields += 1                    # the hopped field, read once from HBM
    if own:
        fields += 1
    fields += 1                        # output (or updated field) write
    if epi == 2:                       # CG_A: read x, r; write x, r (own = p already read)
        fields += 3
    elif epi == 3:                     # CG_B: read p (output writes p)
        fields += 1
    elif epi == 4:                     # RESID: read b
        fields += 1
    by = n5 * fields * (24 * rb + scale)
    if hop:
        by += Vh * 8 * (12 if pair else 18) * lb
    return by


def kernel_name(key):
    if key >= 4000000:
        kind, s1, s2 = (key // 100) % 10, (key // 10) % 10, key % 10
        nm = ["fp64", "fp32", "fp16"]
        return {1: f"k_pack5<{nm[s2]}>", 2: f"k_unpack5<{nm[s1]}>", 3: f"k_convert<{nm[s1]}->{nm[s2]}>",
                4: f"k_axpy_to64<{nm[s1]}>", 5: f"k_norm2<{nm[s1]}>"}[kind]
    if key >= 3000000:
        kind, k = (key // 100) % 10, key % 100
        return {1: f"k_gcr_dots<{k}>", 2: "k_gcr_sum", 3: f"k_gcr_update<{k}>"}[kind]
    if key >= 2000000:
        bf = ",bf16" if (key // 1000) % 10 else ""
        return f"k_net_layer<cin={(key // 100) % 10},cout={(key // 10) % 10}{',own' if key % 10 else ''}{bf}>"
    sd = (key // 100000) % 10
    st = ["fp64", "fp32", "fp16"][sd % 5]
    if sd >= 5:
        staged = "two-slice bulk," if key >= 1000000 else "two-slice,"
    else:
        staged = "staged," if key >= 1000000 else ""
    hop, mixhop, own, mixown, epi = (key // 10000) % 10, (key // 1000) % 10, (key // 100) % 10, (key // 10) % 10, key % 10
    kind = {(1, 1, 0, 0): "hop+A^-1", (1, 0, 1, 1): "hop+A*own", (1, 1, 1, 0): "hop+own+A^-1",
            (1, 0, 1, 0): "hop+own", (0, 0, 1, 1): "s-mix"}.get((hop, mixhop, own, mixown), "hop")
    epin = ["store", "store+norm", "cg_a", "cg_b", "resid"][epi]
    return f"k_hop<{staged}{st},{kind},{epin}>"


def cpu_model():
    """CPU model name of the host (for the CPU baseline's record)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_oracle_config0():
    """Config 0 solved to the end by the oracle: 4^4, Ns = 8, omega_s = 1, m0 = 1.3, H_T(0.05, 1.0) x = b,
    FP64 CGNE to a true residual of 1e-10 (serial numpy; the lattice is too small to split)."""
    from oracle.operators import ODWF as OO
    from oracle import solver as osol
    from paper_1710_09621_gb300 import inputs
    dims, ns = (4, 4, 4, 4), 8
    U = inputs.random_su3_links(dims, 0.4, inputs.seed_for(0, 0))
    op = OO(U, M0, inputs.omega_shamir(ns))
    b = inputs.gaussian_spinor5(dims, ns, inputs.seed_for(0, 1))
    t0 = time.perf_counter()
    _, info = osol.solve_ht(op, b, 0.05, 1.0, tol=1e-10)
    return {"seconds": time.perf_counter() - t0, "iters": info["iters"], "true_residual": info["true_residual"],
            "workload": "4^4, Ns=8, omega_s=1, m0=1.3, H_T(0.05, 1.0) x = b to 1e-10 (config 0, measured end to end)"}


def cpu_oracle_sample(n_full_iters, dims=None):
    """One oracle CGNE iteration (S then S^dag, FP64) on the full benchmark lattice, run on every host
    core (threads over s-slices for the hop, over t for the fifth-dimension products), times the
    GPU's FP64 CGNE iteration count of the same system: an estimate of the oracle's time-to-solution."""
    import numpy as np
    from oracle.operators import ODWF as OO
    from oracle import parallel as opar
    from oracle import solver as osol
    from paper_1710_09621_gb300 import inputs
    dims = tuple(dims or DIMS)
    U = inputs.random_su3_links(dims, EPS, inputs.seed_for(1, 7))
    op = OO(U, M0, inputs.omega_zolotarev(NS, 0.05, 6.2))
    sch = opar.ThreadedSchur(op, MASS, MASS)
    b = inputs.gaussian_spinor5(dims, NS, inputs.seed_for(1, 8)) * sch.even
    p = sch.S_dag(b)  # the CGNE start direction, outside the timed iteration
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    # one CGNE iteration of oracle.solver.cgne: q = S p, the x / r / p updates, p' = S^dag r + beta p
    pp = np.vdot(p, p).real
    rr = np.vdot(b, b).real
    alpha = rr / pp
    x = alpha * p
    r = b - alpha * sch.S(p)
    beta = np.vdot(r, r).real / rr
    p = sch.S_dag(r) + beta * p
    wall = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    sch.close()
    del x, r, p
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    return {"t_iter_s": wall, "cpu_s": cpu, "threads": sch.threads, "value": wall * n_full_iters,
            "dims": list(dims)}


def run_reference(args):
    """The oracle as the reference arm: each step one full-volume oracle CGNE iteration on all host
    cores, scaled by the FP64 CGNE iteration count of the workload to seconds per solve."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n_iters = args.ref_iters
    times = []
    for i in range(args.warmup + args.steps):
        s = cpu_oracle_sample(n_iters)
        if i >= args.warmup:
            times.append(s)
    v = statistics.median([t["value"] for t in times])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": WORKLOAD,
            "cpu_baseline": {"kind": "oracle", "value": v, "unit": "s", "cores": times[0]["threads"],
                             "nproc": os.cpu_count(), "cpu_model": cpu_model(),
                             "sample": f"per step one oracle CGNE iteration on the full {DIMS} lattice "
                                       f"(median {statistics.median(t['t_iter_s'] for t in times):.2f} s on "
                                       f"{times[0]['threads']} threads), times {n_iters} iterations (the FP64 "
                                       f"CGNE iteration count of this workload): estimated"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# The paper's multiple-time-scale assignment (Section 3): the last (heaviest) factor of each scheme on
# level 1 (k1 = 12 steps), the other factors on level 2 (k2 = 6); the gauge force on level 0 (k0 = 480).
PAPER_STEPS = (480, 12, 6)


def paper_levels(n_terms):
    return [2] * (n_terms - 1) + [1]


def scheme_pass(lat, binding, inputs, dims, opts, rank, timed):
    """Per term of every mass-preconditioning scheme: heat-bath, action and force with their Krylov
    iterations, and the CG iterations of one trajectory estimated with the paper's MTS schedule
    (N^cg after Eq.(old_MP): the force of a level-l term is evaluated 2 k_l + 1 times)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    schemes = [("no MP, Eq.(noMP)", binding.MP_NONE, []), ("old MP, Eq.(old_MP)", binding.MP_OLD, [0.1]),
               ("new MP, Eq.(new_MP)", binding.MP_NEW, [0.1]), ("old MP cascade N=2, Eq.(old_MP_N)", binding.MP_OLD,
                                                                [0.05, 0.2]),
               ("new MP cascade N=2, Eq.(new_MP_N)", binding.MP_NEW, [0.05, 0.2])]
    out = []
    for name, code, mh in schemes:
        terms = binding.mp_terms(code, MASS, mh, 1.0)
        lv = paper_levels(len(terms))
        rec, ncg = [], 0
        t0 = time.perf_counter()
        for i, t in enumerate(terms):
            eta = torch.from_numpy(inputs.gaussian_spinor(dims, inputs.seed_for(1, 200 + 10 * rank + i))).to(dev)
            phi, hb = lat.heatbath(t, eta, opts=opts)
            S, st_a = lat.action(t, phi, opts=opts)
            _, st_f = lat.force(t, phi, opts=opts)
            k = PAPER_STEPS[lv[i]]
            ncg += hb["iters"] + 2 * st_a["iters"] + (2 * k + 1) * st_f["iters"]
            rec.append({"chirality": t.chirality, "m3": t.m3, "m4": t.m4, "m_den": t.m_den, "level": lv[i],
                        "poles": hb["n_poles"], "hb_iters": hb["iters"], "action_iters": st_a["iters"],
                        "force_iters": st_f["iters"], "action": S})
        torch.cuda.synchronize()
        out.append({"scheme": name, "heavy_masses": mh, "n_terms": len(terms), "seconds": time.perf_counter() - t0,
                    "Ncg_trajectory_estimate": ncg, "terms": rec})
    return out


def md_step(lat, binding, inputs, dims, U, opts, opts_ref, beta, dtau, rank):
    """Config-2 MD step on one lattice with the new-MP terms (m, mh, M) = (0.01, 0.1, 1): heat-bath,
    action, force of every term, one momentum update with the gauge and fermion forces, one link
    update, the actions again and Delta H; the mixed-precision action and force are compared with the
    same solver run to a 100x tighter FP64 true residual."""
    import numpy as np
    import torch
    dev = U.device
    terms = binding.mp_terms(binding.MP_NEW, MASS, [0.1], 1.0)
    rec = []
    Ux = U.clone()
    Lx, Ly, Lz, Lt = dims
    P = torch.from_numpy(np.random.default_rng(inputs.seed_for(2, 500 + rank)).standard_normal(
        (4, Lt, Lz, Ly, Lx, 8))).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    phis, S0 = [], 0.0
    for i, t in enumerate(terms):
        eta = torch.from_numpy(inputs.gaussian_spinor(dims, inputs.seed_for(2, 600 + 10 * rank + i))).to(dev)
        th = time.perf_counter()
        phi, hb = lat.heatbath(t, eta, opts=opts)
        t_hb = time.perf_counter() - th
        ta = time.perf_counter()
        S, st_a = lat.action(t, phi, opts=opts)
        t_a = time.perf_counter() - ta
        tf = time.perf_counter()
        F, st_f = lat.force(t, phi, opts=opts)
        t_f = time.perf_counter() - tf
        Sr, _ = lat.action(t, phi, opts=opts_ref)
        Fr, _ = lat.force(t, phi, opts=opts_ref)
        lat.momentum_update(P, F, dtau)
        phis.append(phi)
        S0 += S
        rec.append({"chirality": t.chirality, "m3": t.m3, "m4": t.m4, "m_den": t.m_den,
                    "heatbath_s": t_hb, "hb_iters": hb["iters"], "action_s": t_a, "action_iters": st_a["iters"],
                    "force_s": t_f, "force_iters": st_f["iters"],
                    "action_rel_err_vs_tight": abs(S - Sr) / abs(Sr),
                    "force_rel_err_vs_tight": float(torch.linalg.vector_norm(F - Fr) / torch.linalg.vector_norm(Fr))})
    # the chosen method on the EOFA path: the same action and force solves with CGNE on S M, the network
    # (Neumann-initialised: no training cost) attached to the handle
    net = binding.Net(lat, channels=2)
    lat.set_preconditioner(net)
    lopts = binding.solve_opts(tol=opts.tol, prec="single", delta=1e-5)
    for t, phi, r in zip(terms, phis, rec):
        ta = time.perf_counter()
        S_n, st_an = lat.action(t, phi, opts=lopts)
        t_an = time.perf_counter() - ta
        tf = time.perf_counter()
        F_n, st_fn = lat.force(t, phi, opts=lopts)
        t_fn = time.perf_counter() - tf
        r.update({"net_action_s": t_an, "net_action_iters": st_an["iters"], "net_force_s": t_fn,
                  "net_force_iters": st_fn["iters"]})
    lat.set_preconditioner(None)
    net.close()
    K0 = lat.kinetic(P)  # momenta after the fermion kicks; the gauge kick and link update follow
    Sg0 = lat.gauge_action(Ux, beta)
    Fg = lat.gauge_force(Ux, beta)
    lat.momentum_update(P, Fg, dtau)
    K1 = lat.kinetic(P)
    lat.link_update(Ux, P, dtau)
    Sg1 = lat.gauge_action(Ux, beta)
    S1 = 0.0
    for t, phi in zip(terms, phis):
        S1 += lat.action(t, phi, opts=opts)[0]
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    lat.set_gauge(U)
    return {"terms": rec, "seconds": secs, "beta": beta, "dtau": dtau,
            "dS_fermion": S1 - S0, "dS_gauge": Sg1 - Sg0, "dK_gauge_kick": K1 - K0,
            "what": "per term heat-bath, action, force (mixed precision, true residual 1e-10; errors against the "
                    "same solver at 1e-12), then P += dtau (F_gauge + sum F_terms), U <- exp(i dtau P) U, actions "
                    "again"}


def hmc_trajectory(lat, binding, inputs, dims, U, opts, beta, rank, steps=PAPER_STEPS):
    """One HMC trajectory of length 1 with the new MP (m, mh, M) = (0.01, 0.1, 1): heat-bath of every
    term, then the nested Omelyan integrator on the paper's (k0, k1, k2) schedule; Delta H and the
    CG iterations of the whole trajectory."""
    import numpy as np
    import torch
    dev = U.device
    terms = binding.mp_terms(binding.MP_NEW, MASS, [0.1], 1.0)
    Lx, Ly, Lz, Lt = dims
    Ux = U.clone()
    P = torch.from_numpy(np.random.default_rng(inputs.seed_for(1, 700 + rank)).standard_normal(
        (4, Lt, Lz, Ly, Lx, 8))).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    phis, hb_iters = [], 0
    for i, t in enumerate(terms):
        eta = torch.from_numpy(inputs.gaussian_spinor(dims, inputs.seed_for(1, 800 + 10 * rank + i))).to(dev)
        phi, hb = lat.heatbath(t, eta, opts=opts)
        phis.append(phi)
        hb_iters += hb["iters"]
    t_hb = time.perf_counter() - t0
    # the force and action solves with CGNE on S M (Neumann-initialised network attached)
    net = binding.Net(lat, channels=2)
    lat.set_preconditioner(net)
    st = lat.md(Ux, P, beta, terms, phis, paper_levels(len(terms)), list(steps), tau=1.0,
                opts=binding.solve_opts(tol=opts.tol, prec="single", delta=1e-5))
    torch.cuda.synchronize()
    lat.set_preconditioner(None)
    net.close()
    lat.set_gauge(U)
    return {"dims": list(dims), "beta": beta, "steps_k0_k1_k2": list(steps),
            "solver": "heat-bath: batched mixed-precision CGNE over the poles; MD forces and actions: CGNE on S M "
                      "with the Neumann-initialised network (odwf_set_preconditioner)",
            "levels": paper_levels(len(terms)), "heatbath_seconds": t_hb, "heatbath_iters": hb_iters,
            "md_seconds": st["seconds"], "seconds": time.perf_counter() - t0, "dH": st["dH"],
            "force_evals": st["force_evals"][:3], "link_updates": st["link_updates"], "md_cg_iters": st["cg_iters"],
            "K0": st["K0"], "K1": st["K1"], "Sg0": st["Sg0"], "Sg1": st["Sg1"], "Sf0": st["Sf0"], "Sf1": st["Sf1"]}


def config4(args):
    """The learned preconditioner trained across seeded gauge configurations and evaluated on held-out ones
    (32^3 x 64, Ns = 16, m = 0.005): CGNE on S M with the trained network against plain mixed-precision CGNE
    and against the untrained (Neumann-initialised) network, every solve to an FP64 true residual of 1e-10.

    Links: U = exp(i eps sum_a lambda^a r^a) with seeded r^a ~ N(0, 1) (the generator's recipe), made on the
    device by the library's exact SU(3) exponential (hmc_link_update of the unit field with P = 2 eps r,
    tau = 1): the host generator's batched eigendecompositions take minutes at this volume. Training: for
    each training configuration in turn, `c4_pairs` seeded Gaussian vectors r_i, `c4_steps` Adam steps on
    the residual loss |S M r - r|^2 / |r|^2 (Adam's moments carry over from one configuration to the
    next). Prints one JSON line of its own."""
    import numpy as np
    import torch
    from paper_1710_09621_gb300 import build, inputs
    from paper_1710_09621_gb300.binding import ODWF, Net, solve_opts

    build.build()
    dev = torch.device("cuda", 0)
    dims = tuple(int(v) for v in args.c4_dims.split(","))
    Lx, Ly, Lz, Lt = dims
    m = 0.005
    om = inputs.omega_zolotarev(NS, 0.05, 6.2)
    lat = ODWF(dims, NS, M0, om)
    shape5 = (NS, Lt, Lz, Ly, Lx, 4, 3)

    def links(seed):
        r = np.random.default_rng(seed).standard_normal((4, Lt, Lz, Ly, Lx, 8))
        P = torch.from_numpy(r).to(dev).mul_(2.0 * EPS)
        del r
        U = torch.zeros((4, Lt, Lz, Ly, Lx, 3, 3), dtype=torch.complex128, device=dev)
        for i in range(3):
            U[..., i, i] = 1.0
        lat.link_update(U, P, 1.0)
        return U

    def gauss5(seed):
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        return torch.randn(shape5, dtype=torch.complex128, device=dev, generator=g)

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    net = neu = None
    t_start = time.perf_counter()
    train_log = []
    for c in range(args.c4_train):
        U = links(inputs.seed_for(5, c))
        lat.set_gauge(U)
        del U
        if net is None:  # a network needs the handle's gauge field; it follows later set_gauge calls
            net = Net(lat, channels=2)
            net.set_loss("residual")
            neu = Net(lat, channels=2)
        rs = [gauss5(inputs.seed_for(5, 1000 + args.c4_pairs * c + i)) for i in range(args.c4_pairs)]
        net.set_pairs(rs, m, m)
        del rs
        losses, t_tr = timed(lambda: net.train(args.c4_steps, args.lr))
        train_log.append({"config": c, "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
                          "seconds": t_tr})
    t_train = time.perf_counter() - t_start
    opts_l = solve_opts(tol=TOL, prec="single", delta=1e-5)
    opts_p = solve_opts(tol=TOL, prec="single", delta=0.01)
    evals = []
    for h in range(args.c4_heldout):
        U = links(inputs.seed_for(5, 500 + h))
        lat.set_gauge(U)
        del U
        b = gauss5(inputs.seed_for(5, 2000 + h))
        (_, sp), tp = timed(lambda: lat.solve(b, m, m, opts=opts_p))
        (_, st), tt = timed(lambda: net.solve(b, m, m, opts=opts_l))
        (_, sn), tn = timed(lambda: neu.solve(b, m, m, opts=opts_l))
        evals.append({"heldout": h, "plain_cgne": {"seconds": tp, "iters": sp["iters"], "true_residual": sp["true_residual"]},
                      "trained": {"seconds": tt, "iters": st["iters"], "true_residual": st["true_residual"]},
                      "neumann": {"seconds": tn, "iters": sn["iters"], "true_residual": sn["true_residual"]}})
        del b
    net.close()
    neu.close()
    lat.close()
    mean = lambda k, f: sum(e[k][f] for e in evals) / len(evals)
    line = {"metric": "learned-preconditioned CGNE time-to-1e-10 on held-out configurations", "value": mean("trained", "seconds"),
            "unit": "s", "n_gpus": 1, "higher_is_better": False, "dtype": "f32 + bf16 tensor-core network (FP64 residual restarts)",
            "data": "synthetic",
            "config": {"workload": f"{Lx}^3x{Lt} Ns=16 optimal DWF (Zolotarev omega on [0.05,6.2]), m0=1.3, m=0.005, links eps=0.3, "
                                   f"network trained on {args.c4_train} seeded configurations, evaluated on {args.c4_heldout} held-out ones",
                       "dims": list(dims), "Ns": NS, "mass": m, "tol": TOL},
            "plain_cgne_seconds": mean("plain_cgne", "seconds"), "neumann_seconds": mean("neumann", "seconds"),
            "iters": {"trained": mean("trained", "iters"), "neumann": mean("neumann", "iters"),
                      "plain_cgne": mean("plain_cgne", "iters")},
            "training": {"configs": args.c4_train, "pairs_per_config": args.c4_pairs, "steps_per_config": args.c4_steps,
                         "lr": args.lr, "loss": "residual", "seconds": t_train,
                         "loss_first": train_log[0]["loss_first"], "loss_last": train_log[-1]["loss_last"],
                         "per_config": train_log},
            "heldout": evals}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="single", choices=["single", "half", "double"])
    ap.add_argument("--delta", type=float, default=None,
                    help="reliable-update trigger of the inner solver (default 0.01 FP32, 0.1 FP16)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the hot-path pass, batch and learned sections")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch autotuner")
    ap.add_argument("--train-steps", type=int, default=200)
    ap.add_argument("--lr", type=float, default=5e-3, help="Adam learning rate of the network training")
    ap.add_argument("--pairs", type=int, default=8, help="training pairs (r, S^{-1} r) from the plain solver")
    ap.add_argument("--train-loss", default="residual", choices=["residual", "error"],
                    help="network training loss: |S M r - r|^2/|r|^2 (default) or |M r - e|^2/|e|^2")
    ap.add_argument("--method", default="learned", choices=["learned", "gcr", "cgne"],
                    help="timed solver: learned-preconditioned CGNE (default), flexible GCR right-preconditioned "
                         "by the learned network, or plain mixed-precision CGNE")
    ap.add_argument("--nvec", type=int, default=8, help="GCR basis size")
    ap.add_argument("--truncate", action="store_true", help="GCR keeps a sliding window of directions")
    ap.add_argument("--gcr-sweep", action="store_true",
                    help="also run flexible GCR (network / none, restarted / window) with an iteration cap")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--ref-iters", type=int, default=1103,
                    help="CGNE iterations the reference arm scales one oracle iteration by: the FP64 CGNE "
                         "iteration count of this workload (1103 on the GPU, same seeded system)")
    ap.add_argument("--dims", default=None, help="override lattice, e.g. 16,16,16,16 (profiling only)")
    ap.add_argument("--beta", type=float, default=6.2, help="Wilson plaquette coupling of the MD sections")
    ap.add_argument("--no-hmc", action="store_true", help="skip the HMC trajectory section")
    ap.add_argument("--net-delta", type=float, default=1e-5,
                    help="the learned solve's reliable-update trigger: an FP64 residual whenever the FP32 one has "
                         "dropped by this factor")
    ap.add_argument("--config4", action="store_true",
                    help="instead of the default workload: the network trained across seeded configurations and "
                         "evaluated on held-out ones (32^3 x 64, m = 0.005)")
    ap.add_argument("--c4-dims", default="32,32,32,64")
    ap.add_argument("--c4-train", type=int, default=20, help="training configurations")
    ap.add_argument("--c4-heldout", type=int, default=2, help="held-out evaluation configurations")
    ap.add_argument("--c4-pairs", type=int, default=2, help="training vectors per configuration")
    ap.add_argument("--c4-steps", type=int, default=10, help="Adam steps per configuration")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.config4:
        return config4(args)

    global DIMS
    if args.delta is None:
        args.delta = 0.01 if args.prec == "single" else 0.1
    if args.dims:
        DIMS = tuple(int(v) for v in args.dims.split(","))
    import numpy as np
    import torch
    from paper_1710_09621_gb300 import build, inputs
    from paper_1710_09621_gb300.binding import ODWF, solve_opts

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    dev = torch.device("cuda", local)
    om = inputs.omega_zolotarev(NS, 0.05, 6.2)
    U_host = inputs.random_su3_links(DIMS, EPS, inputs.seed_for(1, rank))
    plaq = average_plaquette(U_host)
    U = torch.from_numpy(U_host).to(dev)
    del U_host
    b_host = torch.from_numpy(inputs.gaussian_spinor5(DIMS, NS, inputs.seed_for(1, 100 + rank))).pin_memory()
    b = b_host.to(dev)
    lat = ODWF(DIMS, NS, M0, om)
    lat.set_gauge(U)
    opts = solve_opts(tol=TOL, prec=args.prec, delta=args.delta)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    tune_report = None
    if not args.no_tune:
        t0 = time.perf_counter()
        tune_report = lat.autotune(args.prec)
        tune_report = {"seconds": time.perf_counter() - t0,
                       "chosen": [l for l in tune_report.splitlines() if l.startswith("chosen")]}
    learned_setup = None
    net = None
    if args.method in ("learned", "gcr"):
        from paper_1710_09621_gb300.binding import Net
        net = Net(lat, channels=2)
        net.set_loss(args.train_loss)
        rs = [torch.from_numpy(inputs.gaussian_spinor5(DIMS, NS, inputs.seed_for(4, i))).to(dev)
              for i in range(args.pairs)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net.set_pairs(rs, MASS, MASS, tol=1e-8)
        t1 = time.perf_counter()
        losses = net.train(args.train_steps, args.lr)
        t2 = time.perf_counter()
        learned_setup = {"pairs": len(rs), "loss": args.train_loss, "pair_seconds": t1 - t0,
                         "train_steps": args.train_steps, "lr": args.lr,
                         "train_seconds": t2 - t1, "loss_first": float(losses[0]), "loss_last": float(losses[-1])}
        del rs
        lopts = solve_opts(tol=TOL, prec="single", delta=args.net_delta)

        if args.method == "learned":
            def do_solve(bb, xx=None):
                return net.solve(bb, MASS, MASS, opts=lopts)
        else:
            def do_solve(bb, xx=None):
                return lat.solve_gcr(bb, MASS, MASS, net=net, nvec=args.nvec, truncate=args.truncate, opts=lopts)
    else:
        def do_solve(bb, xx=None):
            return lat.solve(bb, MASS, MASS, x=xx, opts=opts)
    for _ in range(args.warmup):
        x, st = do_solve(b)
    # ---- timed region: device-resident inputs -------------------------------------------------
    lat.profile(True)
    barrier()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev0, ev1 = evs[0], evs[-1]
    stats = []
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed solves (ncu --nvtx)
        ev0.record(stream)
        for i in range(args.steps):
            x, st = do_solve(b, x)
            stats.append(st)
            evs[i + 1].record(stream)
        barrier()
        torch.cuda.nvtx.range_pop()
    prof = lat.profile_read()
    lat.profile(False)
    step_s = [evs[i].elapsed_time(evs[i + 1]) / 1e3 for i in range(args.steps)]
    elapsed = reduce_max(ev0.elapsed_time(ev1) / 1e3, dist, dev)
    value = per_solve_seconds(elapsed, args.steps, world)

    # ---- e2e: pinned host input -> device -> solve -> pinned host output ------------------------
    x_host = torch.empty_like(b_host).pin_memory()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        bd = b_host.to(dev, non_blocking=True)
        xd, _ = do_solve(bd)
        x_host.copy_(xd, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_value = per_solve_seconds(reduce_max(e0.elapsed_time(e1) / 1e3, dist, dev), args.steps, world)

    # ---- the other mixed-precision method on the same system ---------------------------------------
    other = None
    if args.method != "cgne":
        barrier()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(2):
            _, stc = lat.solve(b, MASS, MASS, opts=opts)
        c1.record(stream)
        barrier()
        other = {"method": f"CGNE, inner {args.prec}, FP64 reliable updates (no network)",
                 "seconds": c0.elapsed_time(c1) / 2e3, "iters": stc["iters"],
                 "true_residual": stc["true_residual"]}

    # ---- plain FP64 GPU CGNE on the same system ----------------------------------------------
    fp64 = None
    if not args.no_fp64:
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        lat.profile(True)
        f0.record(stream)
        _, st64 = lat.solve(b, MASS, MASS, opts=solve_opts(tol=TOL, prec="double"))
        f1.record(stream)
        barrier()
        prof64 = lat.profile_read()
        lat.profile(False)
        fp64 = {"seconds": f0.elapsed_time(f1) / 1e3, "iters": st64["iters"], "true_residual": st64["true_residual"]}
        # the FP64 hop kernels against the measured FP64 FMA roof (flop conventions of HOP_FLOPS / FIFTH_FLOPS)
        peak64 = lat.fp64_fma_peak()
        Vh = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3] // 2
        roof = []
        for key, (n, ms) in sorted(prof64.items(), key=lambda kv: -kv[1][1]):
            if key >= 1000000 or (key // 100000) % 10 != 0 or n == 0:
                continue
            hop, mixhop, mixown = (key // 10000) % 10, (key // 1000) % 10, (key // 10) % 10
            fl = Vh * NS * (HOP_FLOPS * hop + FIFTH_FLOPS * (mixhop + mixown))
            tf = fl / (ms / n * 1e-3) / 1e12
            roof.append({"kernel": kernel_name(key), "launches": n, "avg_us": ms / n * 1e3, "tflops": tf,
                         "frac_of_fp64_peak": tf / peak64})
        fp64["fp64_fma_peak_tflops"] = peak64
        fp64["fp64_kernels"] = roof

    def timed(fn):
        barrier()
        t0 = time.perf_counter()
        out = fn()
        barrier()
        return out, time.perf_counter() - t0

    # ---- the rest of the hot path on the same lattice --------------------------------------------
    extra = {}
    if not args.quick:
        from paper_1710_09621_gb300 import binding as binding_mod
        from paper_1710_09621_gb300.binding import Net

        # every mass-preconditioning scheme's terms: heat-bath, action, force and N^cg (Section 2)
        hp_opts = solve_opts(tol=TOL, prec=args.prec, delta=args.delta)
        rec, t_hp = timed(lambda: scheme_pass(lat, binding_mod, inputs, DIMS, hp_opts, rank, timed))
        extra["schemes"] = {"seconds": t_hp, "schemes": rec,
                            "what": "per term of (m,m)/(M,M), m=0.01, M=1: heat-bath (batched pole solves), action "
                                    "and force; Ncg_trajectory_estimate = sum over terms of heat-bath + 2 actions + "
                                    "(2 k + 1) forces with the paper's MTS levels (k1 = 12 for the last factor, "
                                    "k2 = 6 for the others)"}
        # one HMC trajectory on the paper's schedule (480, 12, 6) with the new-MP terms (Section 3)
        if not args.no_hmc:
            extra["hmc_trajectory"] = hmc_trajectory(lat, binding_mod, inputs, DIMS, U, hp_opts, args.beta, rank)
        # batch of 4 systems with different masses vs one after another
        m12 = [(MASS, MASS), (MASS, 0.1), (1.0, 0.1), (0.1, 0.1)]
        bsb = [torch.from_numpy(inputs.gaussian_spinor5(DIMS, NS, inputs.seed_for(1, 300 + i))).to(dev) for i in range(4)]
        _, t_batch = timed(lambda: lat.solve_batch(bsb, m12, opts=opts))
        _, t_seq = timed(lambda: [lat.solve(b_, *mm, opts=opts) for b_, mm in zip(bsb, m12)])
        extra["batch4"] = {"seconds_batched": t_batch, "seconds_sequential": t_seq, "masses": m12}
        # uneven batch: 8^4, 12^4 and the 16^3 x 32 lattice (Ns = 16) advancing in one launch per step
        from paper_1710_09621_gb300.binding import ODWF as _ODWF, solve_multi
        lats_u, bs_u = [], []
        for k, dd in enumerate([(8, 8, 8, 8), (12, 12, 12, 12)]):
            lu = _ODWF(dd, NS, M0, om)
            lu.set_gauge(torch.from_numpy(inputs.random_su3_links(dd, EPS, inputs.seed_for(3, k))).to(dev))
            lats_u.append(lu)
            bs_u.append(torch.from_numpy(inputs.gaussian_spinor5(dd, NS, inputs.seed_for(3, 10 + k))).to(dev))
        lats_u.append(lat)
        bs_u.append(b)
        mu = [(MASS, MASS)] * 3
        (_, stu), t_unb = timed(lambda: solve_multi(lats_u, bs_u, mu, opts=opts))
        _, t_uns = timed(lambda: [lz.solve(bz, MASS, MASS, opts=opts) for lz, bz in zip(lats_u, bs_u)])
        extra["uneven_batch"] = {"lattices": ["8^4", "12^4", "16^3x32"], "Ns": NS,
                                 "seconds_one_launch_per_step": t_unb, "seconds_sequential": t_uns,
                                 "iters": [s_["iters"] for s_ in stu]}
        for lz in lats_u[:2]:
            lz.close()
    if not args.quick and DIMS == (16, 16, 16, 32):
        # the paper's lattice shape, 24^3 x 48 with Ns = 16 (Section 3): every FP32 half field is
        # 510 MB, far beyond L2, so these per-kernel figures carry no cache effects
        D24 = (24, 24, 24, 48)
        l24 = ODWF(D24, NS, M0, om)
        U24 = inputs.random_su3_links(D24, EPS, inputs.seed_for(2, rank))
        plaq24 = average_plaquette(U24)
        U24d = torch.from_numpy(U24).to(dev)
        l24.set_gauge(U24d)
        del U24
        b24 = torch.from_numpy(inputs.gaussian_spinor5(D24, NS, inputs.seed_for(2, 100 + rank))).to(dev)
        tune24 = None
        if not args.no_tune:  # the launch choices of this lattice, as for the workload above
            tune24 = [l for l in l24.autotune(args.prec).splitlines() if l.startswith("chosen")]
        l24.solve(b24, MASS, MASS, opts=opts)
        l24.profile(True)
        (_, st24), t24 = timed(lambda: l24.solve(b24, MASS, MASS, opts=opts))
        p24 = l24.profile_read()
        l24.profile(False)
        # config 2: one MD step with the new-MP terms on this lattice
        extra["md_step_24"] = md_step(l24, binding_mod, inputs, D24, U24d,
                                      solve_opts(tol=TOL, prec=args.prec, delta=args.delta),
                                      solve_opts(tol=1e-12, prec=args.prec, delta=args.delta), args.beta,
                                      1.0 / (2 * PAPER_STEPS[0]), rank)
        del U24d
        Vh24 = D24[0] * D24[1] * D24[2] * D24[3] // 2
        k24 = []
        for key, (n, ms) in sorted(p24.items(), key=lambda kv: -kv[1][1]):
            avg_s = ms / 1e3 / n
            k24.append({"kernel": kernel_name(key), "launches": n, "avg_us": avg_s * 1e6,
                        "gbs": alg_bytes(key, Vh24, NS) / avg_s / 1e9, "share_ms": ms})
        extra["paper_lattice"] = {"dims": list(D24), "Ns": NS, "plaquette": plaq24, "autotune": tune24,
                                  "method": f"CGNE, inner {args.prec}, FP64 reliable updates",
                                  "seconds": t24, "iters": st24["iters"], "true_residual": st24["true_residual"],
                                  "gflops": st24["iters"] * Vh24 * NS * CG_ITER_FLOPS / t24 / 1e9,
                                  "kernels": [k for k in k24 if k["share_ms"] > 0.01 * t24 * 1e3]}
        l24.close()
        del b24
    if not args.quick:
        # preconditioned solve with the untrained (Neumann-series) network, and, when the timed method
        # is plain CGNE, with a trained one
        neu = Net(lat, channels=2)
        (xn, stn), t_n = timed(lambda: neu.solve(b, MASS, MASS, opts=solve_opts(tol=TOL, prec="single", delta=args.net_delta)))
        extra["neumann_network_solve"] = {"seconds": t_n, "iters": stn["iters"], "true_residual": stn["true_residual"]}
        if args.method == "gcr":
            (_, stp), t_p = timed(lambda: net.solve(b, MASS, MASS, opts=solve_opts(tol=TOL, prec="single", delta=args.net_delta)))
            extra["learned_pcgne"] = {"seconds": t_p, "iters": stp["iters"], "true_residual": stp["true_residual"]}
        neu.close()
    if args.gcr_sweep:
        # flexible GCR on S (right-preconditioned by the network, and without it); a run that ends above
        # the tolerance within its iteration / time cap is reported with its final true residual
        from paper_1710_09621_gb300.binding import Net
        gnet = net if net is not None else Net(lat, channels=2)
        gl = solve_opts(tol=TOL, prec="single", delta=1e-3, maxiter=3000, max_seconds=15.0)
        gcr = {"sweep": [], "weights": "trained" if net is not None else "Neumann"}
        for nv_, tr_ in ((8, False), (16, False), (4, True), (8, True)):
            (_, stg), t_g = timed(lambda: lat.solve_gcr(b, MASS, MASS, net=gnet, nvec=nv_, truncate=tr_, opts=gl,
                                                       allow_noconv=True))
            gcr["sweep"].append({"nvec": nv_, "basis": "window" if tr_ else "restarted", "seconds": t_g,
                                 "iters": stg["iters"], "true_residual": stg["true_residual"], "status": stg["status"]})
        (_, stg0), t_g0 = timed(lambda: lat.solve_gcr(b, MASS, MASS, net=None, nvec=8, truncate=True, opts=gl,
                                                     allow_noconv=True))
        gcr["no_network"] = {"nvec": 8, "basis": "window", "seconds": t_g0, "iters": stg0["iters"],
                             "true_residual": stg0["true_residual"], "status": stg0["status"]}
        extra["gcr"] = gcr
        if gnet is not net:
            gnet.close()
    if not args.quick and args.method == "cgne":
        # learned preconditioner: pairs from the solver, Adam, then preconditioned solves
        net = Net(lat, channels=2)
        rs = [torch.from_numpy(inputs.gaussian_spinor5(DIMS, NS, inputs.seed_for(4, i))).to(dev) for i in range(4)]
        _, t_pairs = timed(lambda: net.set_pairs(rs, MASS, MASS, tol=1e-8))
        losses, t_train = timed(lambda: net.train(args.train_steps, args.lr))
        lopts = solve_opts(tol=TOL, prec="single", delta=1e-3)
        (xl, stl), t_l = timed(lambda: net.solve(b, MASS, MASS, opts=lopts))
        extra["learned"] = {"pairs": len(rs), "pair_seconds": t_pairs, "train_steps": args.train_steps,
                            "train_seconds": t_train, "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
                            "trained": {"seconds": t_l, "iters": stl["iters"], "true_residual": stl["true_residual"]}}
        net.close()

    # ---- roofline of the dominant kernel -------------------------------------------------------
    Vh = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3] // 2
    peak, peak_kind = peaks()
    kern = []
    for key, (n, ms) in prof.items():
        avg_s = ms / 1e3 / n
        by = alg_bytes(key, Vh, NS)
        kern.append({"kernel": kernel_name(key), "key": key, "launches": n, "total_ms": ms,
                     "avg_us": avg_s * 1e6, "alg_bytes": by, "gbs": by / avg_s / 1e9})
    kern.sort(key=lambda k: -k["total_ms"])
    tot_ms = sum(k["total_ms"] for k in kern) or 1.0
    for k in kern:
        k["share"] = k["total_ms"] / tot_ms
    dom = kern[0] if kern else None
    roof = None
    if dom:
        roof = {"bound": "hbm", "kernel": dom["kernel"], "achieved": dom["gbs"], "peak": peak, "unit": "GB/s",
                "frac": dom["gbs"] / peak, "peak_source": f"hbm_gbs of {peak_kind}",
                "traffic": dram_traffic(dom["kernel"], DIMS, NS),
                "alg_bytes_per_launch": dom["alg_bytes"], "avg_launch_us": dom["avg_us"]}

    # the dslash proper (A3 + A4: hop over all Ns slices fused with the fifth-dimension inverse, K1)
    dsl = [k for k in kern if "hop+A^-1,store" in k["kernel"] and "fp64" not in k["kernel"]]
    dslash = None
    if dsl:
        k1 = max(dsl, key=lambda k: k["total_ms"])
        dslash = {"kernel": k1["kernel"], "avg_launch_us": k1["avg_us"], "alg_bytes_per_launch": k1["alg_bytes"],
                  "achieved_gbs": k1["gbs"], "peak_gbs": peak, "frac": k1["gbs"] / peak,
                  "traffic": dram_traffic(k1["kernel"], DIMS, NS),
                  "peak_source": f"hbm_gbs of {peak_kind}",
                  "gflops": Vh * NS * (HOP_FLOPS + FIFTH_FLOPS) / (k1["avg_us"] * 1e-6) / 1e9,
                  "gflops_convention": f"{HOP_FLOPS} hop + {FIFTH_FLOPS} fifth-dimension flops per 5D half-site"}
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("f32 + bf16 tensor-core network (FP64 residual restarts)" if args.method != "cgne" else
                  {"single": "f32 (FP64 reliable updates)", "half": "f16 storage/f32 (FP64 reliable updates)",
                   "double": "f64"}[args.prec]),
        "data": "synthetic",
        "config": dict(WORKLOAD, prec=args.prec, delta=args.delta, plaquette=plaq,
                       l2="inputs larger than L2 (each solve streams >1 GB)",
                       parallelism=f"replicas x{world}"),
        "solve": {"iters": stats[-1]["iters"], "reliable_updates": stats[-1]["reliable_updates"],
                  "true_residual": max(s["true_residual"] for s in stats),
                  "step_seconds_rank0": step_s, "median_step_seconds_rank0": statistics.median(step_s)},
        "fp64_plain": fp64,
        "speedup_vs_fp64": (fp64["seconds"] / value) if fp64 else None,
        "roofline": roof,
        "dslash": dslash,
        "kernels": kern,
        "e2e": {"value": e2e_value, "unit": "s", "h2d_bytes_per_step": b_host.numel() * 16,
                "d2h_bytes_per_step": x_host.numel() * 16},
        "gpu_launches": int(sum(k["launches"] for k in kern)),
        "clocks": clk.summary(),
        "autotune": tune_report,
        "method": {"learned": "CGNE on S M with the trained gauge-equivariant network M (BF16 tensor-core "
                              "channel mixing), FP32 inner cycles with FP64 reliable updates",
                   "gcr": f"flexible GCR ({args.nvec} directions, {'sliding window' if args.truncate else 'restarted'}) "
                          "on S right-preconditioned by the trained network, FP32 inner cycles restarted from the "
                          "FP64 residual",
                   "cgne": f"CGNE, inner {args.prec}, FP64 reliable updates"}[args.method],
        "learned_setup": learned_setup,
        "cgne_same_run": other,
    }
    # Krylov throughput in the flop convention of one CGNE iteration (CG_ITER_FLOPS per 5D half-site
    # of the even checkerboard)
    for rec in (line["cgne_same_run"], line["fp64_plain"]):
        if rec and rec.get("seconds"):
            rec["gflops"] = rec["iters"] * Vh * NS * CG_ITER_FLOPS / rec["seconds"] / 1e9
            rec["gflops_convention"] = f"{CG_ITER_FLOPS} flops per 5D half-site per CGNE iteration"
    if args.method == "cgne":
        line["solve"]["gflops"] = stats[-1]["iters"] * Vh * NS * CG_ITER_FLOPS / value / 1e9
    line.update(extra)
    if rank == 0 and not args.no_cpu and world == 1:
        n_it = fp64["iters"] if fp64 else args.ref_iters
        c0 = cpu_oracle_config0()
        s = cpu_oracle_sample(n_it)
        line["cpu_baseline"] = {"value": s["value"], "unit": "s", "cores": s["threads"], "kind": "oracle",
                                "nproc": os.cpu_count(), "cpu_model": cpu_model(),
                                "sample": f"one oracle CGNE iteration on the full {DIMS} lattice on {s['threads']} "
                                          f"threads ({s['t_iter_s']:.2f} s), times {n_it} FP64 CGNE iterations: "
                                          f"estimated",
                                "config0_measured": c0}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
