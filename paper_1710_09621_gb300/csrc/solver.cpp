// Even-odd preconditioned CGNE for D_T(m1, m2) x = b' with reliable updates.
//
// The paper computes every H_T(m3, m4)^{-1} with CG (Section 1, the paragraph after the HMC
// outline) and does not state the preconditioning or the stopping rule. Here:
//   D_T = [[A, -1/2 H_eo], [-1/2 H_oe, A]],  A = (4 - m0) + P_+ M_+(m1) + P_- M_-(m2)
//   S   = A - 1/4 H_eo A^{-1} H_oe   on even sites,  b_hat = b'_e + 1/2 H_eo A^{-1} b'_o
//   CGNE (Craig): x += alpha p, r -= alpha S p, p = S^dag r + beta p, so r = b_hat - S x_e,
//   which equals the full residual b' - D_T x once x_o = A^{-1}(b'_o + 1/2 H_oe x_e).
// The Krylov iteration runs in the inner storage precision (FP64, FP32 or FP16 with per-site
// scales); the solution accumulates in FP64 and the residual is replaced by the FP64 true
// residual b_hat - S x whenever the iterated one has dropped by `delta` (reliable updates,
// Sleijpen & van der Vorst 1996) or reached the tolerance. Each iteration is four kernel launches
// (two fused hop+fifth-dimension passes for S, two for S^dag), with the CG scalars kept on the
// device; the host only polls the solver state every few iterations.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "odwf_internal.h"

namespace odwf {

int ensure_workspace(odwf_s* h, int inner);
int apply_dt_parity(odwf_s* h, int stg, const SCoef* c, bool dag, int parity, const void* in_other,
                    const void* own, void* out, cudaStream_t st);

static inline const double* mat(const SCoef* c, int k, int Ns) { return c->dev + (size_t)k * Ns * Ns; }
enum { M_AP = 0, M_AINV = 2, M_AT = 4, M_AINVT = 6 };

struct InnerFields {
    int stg;
    void *x, *r, *p, *t;
    float *xs, *rs, *ps, *ts;
};

// t = A^{-1} H_oe in   (output parity odd); dag: t = A^{-T} H_oe gamma_5 in
static int k1(odwf_s* h, const InnerFields& f, const SCoef* c, bool dag, const void* in, const float* in_s,
              CGState* state, cudaStream_t st) {
    HopArgs a{};
    a.in = in;
    a.in_scale = in_s;
    a.out = f.t;
    a.out_scale = f.ts;
    a.mhop = mat(c, dag ? M_AINVT : M_AINV, h->Ns);
    a.c_hop = 1.0;
    a.g5 = dag ? G5_HOP_IN : 0;
    a.state = state;
    return launch_hop(h, f.stg, 1, true, false, false, EPI_STORE, a, st);
}

// CGNE forward half step: q = A p - 1/4 H_eo t ; x += alpha p ; r -= alpha q ; rr = |r|^2
static int k2a(odwf_s* h, const InnerFields& f, const SCoef* c, cudaStream_t st) {
    HopArgs a{};
    a.in = f.t;
    a.in_scale = f.ts;
    a.own = f.p;
    a.own_scale = f.ps;
    a.mown = mat(c, M_AP, h->Ns);
    a.c_hop = -0.25;
    a.x = f.x;
    a.x_scale = f.xs;
    a.r = f.r;
    a.r_scale = f.rs;
    a.state = h->state;
    return launch_hop(h, f.stg, 0, false, true, true, EPI_CG_A, a, st);
}

// CGNE adjoint half step: z = g5 (A^T g5 r - 1/4 H_eo t) = S^dag r ; p = z + beta p ; pp = |p|^2
static int k2b(odwf_s* h, const InnerFields& f, const SCoef* c, cudaStream_t st) {
    HopArgs a{};
    a.in = f.t;
    a.in_scale = f.ts;
    a.own = f.r;
    a.own_scale = f.rs;
    a.mown = mat(c, M_AT, h->Ns);
    a.c_hop = -0.25;
    a.g5 = G5_OWN_IN | G5_OUT;
    a.r = f.p;
    a.r_scale = f.ps;
    a.state = h->state;
    return launch_hop(h, f.stg, 0, false, true, true, EPI_CG_B, a, st);
}

// FP64: out = bh - S x (even parity), result[slot] = |out|^2 ; uses tmp as the odd intermediate
static int schur_residual64(odwf_s* h, const SCoef* c, const void* bh, const void* x, void* tmp, void* out,
                            int slot, cudaStream_t st) {
    InnerFields f{ST_DOUBLE, nullptr, nullptr, nullptr, tmp, nullptr, nullptr, nullptr, nullptr};
    int rc = k1(h, f, c, false, x, nullptr, nullptr, st);
    if (rc) return rc;
    HopArgs a{};
    a.in = tmp;
    a.own = x;
    a.out = out;
    a.mown = mat(c, M_AP, h->Ns);
    a.c_hop = -0.25;
    a.x = const_cast<void*>(bh);
    a.slot = slot;
    return launch_hop(h, ST_DOUBLE, 0, false, true, true, EPI_RESID, a, st);
}

static int read_state(odwf_s* h, cudaStream_t st) {
    int rc = cuda_check(h, cudaMemcpyAsync(h->state_host, h->state, sizeof(CGState), cudaMemcpyDeviceToHost, st),
                        "state D2H");
    if (rc) return rc;
    return cuda_check(h, cudaStreamSynchronize(st), "stream sync");
}

static int write_state(odwf_s* h, cudaStream_t st) {
    int rc = cuda_check(h, cudaMemcpyAsync(h->state, h->state_host, sizeof(CGState), cudaMemcpyHostToDevice, st),
                        "state H2D");
    if (rc) return rc;
    // the pinned mirror is reused right away: wait for the copy
    return cuda_check(h, cudaStreamSynchronize(st), "stream sync");
}

// Solve D_T(m1, m2) x = b' with b' already packed in ws.b_e / ws.b_o (FP64); the solution is left
// in ws.x_e / ws.x_o (FP64).
int solve_core(odwf_s* h, double m1, double m2, const odwf_solve_opts* opts_in, odwf_solve_stats* stats,
               cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    const bool debug = std::getenv("ODWF_DEBUG") != nullptr;
    odwf_solve_opts o{1e-10, 100000, ODWF_PREC_DOUBLE, 0.1, 0.0};
    if (opts_in) o = *opts_in;
    if (!(o.tol > 0.0) || o.maxiter < 1) return set_err(h, ODWF_EINVAL, "bad solve options");
    if (o.prec != ODWF_PREC_DOUBLE && o.prec != ODWF_PREC_SINGLE && o.prec != ODWF_PREC_HALF)
        return set_err(h, ODWF_EINVAL, "bad precision");
    const int stg = o.prec == ODWF_PREC_DOUBLE ? ST_DOUBLE : (o.prec == ODWF_PREC_SINGLE ? ST_FLOAT : ST_HALF);
    int rc = ensure_workspace(h, stg);
    if (rc) return rc;
    const SCoef* c = get_coef(h, m1, m2);
    if (!c) return ODWF_EINVAL;
    Workspace& w = h->ws;
    const size_t b64 = half_elems_bytes(h, ST_DOUBLE);
    InnerFields f{stg, w.xi, w.ri, w.pi, w.ti, nullptr, nullptr, nullptr, nullptr};
    if (stg == ST_HALF) {
        f.xs = w.xi_s; f.rs = w.ri_s; f.ps = w.pi_s; f.ts = w.ti_s;
    }
    const size_t bi = half_elems_bytes(h, stg);

    // |b'|^2 and b_hat = b'_e + 1/2 H_eo A^{-1} b'_o
    if ((rc = launch_norm2(h, w.b_e, ST_DOUBLE, nullptr, 0, st))) return rc;
    if ((rc = launch_norm2(h, w.b_o, ST_DOUBLE, nullptr, 1, st))) return rc;
    if ((rc = launch_smix(h, ST_DOUBLE, w.b_o, w.t64, mat(c, M_AINV, h->Ns), 1.0, st))) return rc;
    {
        HopArgs a{};
        a.in = w.t64;
        a.own = w.b_e;
        a.out = w.bh;
        a.a_own = 1.0;
        a.c_hop = 0.5;
        if ((rc = launch_hop(h, ST_DOUBLE, 0, false, true, false, EPI_STORE, a, st))) return rc;
    }
    if ((rc = launch_norm2(h, w.bh, ST_DOUBLE, nullptr, 2, st))) return rc;
    if ((rc = read_state(h, st))) return rc;
    const double bnorm2 = h->state_host->result[0] + h->state_host->result[1];
    double rr64 = h->state_host->result[2];
    odwf_solve_stats sres{0, 0, 0.0, 0.0};
    if (bnorm2 == 0.0) {
        cudaMemsetAsync(w.x_e, 0, b64, st);
        cudaMemsetAsync(w.x_o, 0, b64, st);
        if (stats) *stats = sres;
        return cuda_check(h, cudaStreamSynchronize(st), "sync");
    }
    const double tol2 = o.tol * o.tol * bnorm2;

    // x = 0, r = b_hat, p = S^dag r
    if ((rc = cuda_check(h, cudaMemsetAsync(w.x_e, 0, b64, st), "memset"))) return rc;
    if ((rc = cuda_check(h, cudaMemcpyAsync(w.r64, w.bh, b64, cudaMemcpyDeviceToDevice, st), "copy"))) return rc;
    int iters = 0, updates = 0;
    double beta_keep = 0.0;
    bool converged = rr64 <= tol2;
    while (!converged) {
        // restart the inner iteration from the FP64 residual in r64
        if ((rc = cuda_check(h, cudaMemsetAsync(f.x, 0, bi, st), "memset"))) return rc;
        if (stg == ST_HALF && (rc = cuda_check(h, cudaMemsetAsync(f.xs, 0, sizeof(float) * h->Vh * h->Ns, st), "memset")))
            return rc;
        if ((rc = launch_convert(h, w.r64, ST_DOUBLE, nullptr, f.r, stg, f.rs, st))) return rc;
        CGState& hs = *h->state_host;
        std::memset(&hs, 0, sizeof(CGState));
        hs.rr = rr64;
        hs.rr_max = rr64;
        hs.tol2 = (stg == ST_DOUBLE ? 0.81 : 0.25) * tol2;
        hs.delta2 = (stg == ST_DOUBLE) ? 0.0 : o.delta * o.delta;
        hs.maxiter = o.maxiter - iters;
        // The cycle that stopped on a residual check had updated x and r with the last direction but
        // not yet formed the next one. Form it from the replaced residual: p = S^dag r + beta' p with
        // beta' = |r_true|^2 / |r_prev|^2 (Sleijpen & van der Vorst). First cycle: p = S^dag r.
        hs.beta = (updates == 0) ? 0.0 : beta_keep;
        if ((rc = write_state(h, st))) return rc;
        if (updates == 0) {
            if ((rc = cuda_check(h, cudaMemsetAsync(f.p, 0, bi, st), "memset"))) return rc;
            if (stg == ST_HALF && (rc = cuda_check(h, cudaMemsetAsync(f.ps, 0, sizeof(float) * h->Vh * h->Ns, st), "memset")))
                return rc;
        }
        if ((rc = k1(h, f, c, true, f.r, f.rs, h->state, st))) return rc;
        if ((rc = k2b(h, f, c, st))) return rc;
        // iterate until the device flags convergence, an update, a breakdown or maxiter
        int flag = FLAG_RUN;
        int chunk = 8;
        long queued = 0;
        while (flag == FLAG_RUN) {
            // host-side guard: the device counts iterations and stops at maxiter; never queue far past it
            if (queued > (long)hs.maxiter + 256) return set_err(h, ODWF_ENOCONV, "solver state stopped advancing");
            queued += chunk;
            for (int i = 0; i < chunk; ++i) {
                if ((rc = k1(h, f, c, false, f.p, f.ps, h->state, st))) return rc;
                if ((rc = k2a(h, f, c, st))) return rc;
                if ((rc = k1(h, f, c, true, f.r, f.rs, h->state, st))) return rc;
                if ((rc = k2b(h, f, c, st))) return rc;
            }
            if ((rc = read_state(h, st))) return rc;
            flag = h->state_host->flag;
            if (debug) {
                const CGState& d = *h->state_host;
                std::fprintf(stderr, "[odwf] cycle %d iter %d flag %d rr %.6e pp %.6e alpha %.6e beta %.6e rr_max %.6e\n",
                             updates, d.iter, d.flag, d.rr, d.pp, d.alpha, d.beta, d.rr_max);
            }
            if (chunk < 64) chunk *= 2;
            if (o.max_seconds > 0) {
                const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                if (el > o.max_seconds && flag == FLAG_RUN) {
                    iters += h->state_host->iter;
                    if (stats) {
                        sres.iters = iters;
                        sres.reliable_updates = updates;
                        sres.seconds = el;
                        *stats = sres;
                    }
                    return set_err(h, ODWF_ETIMEOUT, "solver exceeded max_seconds");
                }
            }
        }
        iters += h->state_host->iter;
        // previous iterated |r|^2 = rr / beta (the device set beta = rr_new / rr_old)
        const double rr_prev = h->state_host->beta > 0.0 ? h->state_host->rr / h->state_host->beta : 0.0;
        if (flag == FLAG_BREAKDOWN) {
            if (stats) {
                sres.iters = iters;
                *stats = sres;
            }
            return set_err(h, ODWF_EBREAKDOWN, "CGNE breakdown (<p,p> <= 0 or non-finite reduction)");
        }
        // reliable update: x64 += x_inner ; r64 = b_hat - S x64 in FP64
        if ((rc = launch_axpy_to64(h, 1.0, f.x, stg, f.xs, (double*)w.x_e, st))) return rc;
        if ((rc = schur_residual64(h, c, w.bh, w.x_e, w.t64, w.r64, 3, st))) return rc;
        if ((rc = read_state(h, st))) return rc;
        rr64 = h->state_host->result[3];
        beta_keep = rr_prev > 0.0 ? rr64 / rr_prev : 0.0;
        if (debug) std::fprintf(stderr, "[odwf] update %d: true |r|^2 %.6e (tol2 %.6e), beta' %.6e\n", updates, rr64, tol2, beta_keep);
        ++updates;
        if (!std::isfinite(rr64)) return set_err(h, ODWF_EBREAKDOWN, "non-finite true residual");
        converged = rr64 <= tol2;
        if (!converged && iters >= o.maxiter) break;
    }

    // x_o = A^{-1} (b'_o + 1/2 H_oe x_e)
    {
        HopArgs a{};
        a.in = w.x_e;
        a.own = w.b_o;
        a.out = w.x_o;
        a.a_own = 1.0;
        a.c_hop = 0.5;
        a.mhop = mat(c, M_AINV, h->Ns);
        if ((rc = launch_hop(h, ST_DOUBLE, 1, true, true, false, EPI_STORE, a, st))) return rc;
    }
    // FP64 true residual of the full system: ||b' - D_T x|| / ||b'||
    {
        HopArgs a{};
        a.mown = mat(c, M_AP, h->Ns);
        a.c_hop = -0.5;
        a.in = w.x_o;
        a.own = w.x_e;
        a.x = w.b_e;
        a.out = w.r64;
        a.slot = 0;
        if ((rc = launch_hop(h, ST_DOUBLE, 0, false, true, true, EPI_RESID, a, st))) return rc;
        a.in = w.x_e;
        a.own = w.x_o;
        a.x = w.b_o;
        a.out = w.t64;
        a.slot = 1;
        if ((rc = launch_hop(h, ST_DOUBLE, 1, false, true, true, EPI_RESID, a, st))) return rc;
    }
    if ((rc = read_state(h, st))) return rc;
    const double res = std::sqrt((h->state_host->result[0] + h->state_host->result[1]) / bnorm2);
    sres.iters = iters;
    sres.reliable_updates = updates;
    sres.true_residual = res;
    sres.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = sres;
    if (!(res <= o.tol)) {
        return set_err(h, ODWF_ENOCONV, "true residual " + std::to_string(res) + " above tol after " +
                                            std::to_string(iters) + " iterations");
    }
    return ODWF_OK;
}

}  // namespace odwf

extern "C" int eofa_solve(odwf_t* h, double m1, double m2, const void* b, void* x, const odwf_solve_opts* opts,
                          odwf_solve_stats* stats, void* stream) {
    using namespace odwf;
    if (!h || !b || !x) return set_err(h, ODWF_EINVAL, "null argument");
    if (!h->have_gauge) return set_err(h, ODWF_EINVAL, "odwf_set_gauge has not been called");
    if (!(m1 > 0.0 && m1 <= 1.0) || !(m2 > 0.0 && m2 <= 1.0)) return set_err(h, ODWF_EINVAL, "masses must lie in (0, 1]");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_workspace(h, ST_DOUBLE);
    if (rc) return rc;
    // H_T x = b  <=>  D_T x = R5 gamma_5 b
    if ((rc = launch_pack5(h, (const double*)b, h->ws.b_e, h->ws.b_o, ST_DOUBLE, 1, st))) return rc;
    const int src = solve_core(h, m1, m2, opts, stats, st);
    if (src != ODWF_OK && src != ODWF_ENOCONV) return src;
    if ((rc = launch_unpack5(h, h->ws.x_e, h->ws.x_o, (double*)x, ST_DOUBLE, 0, st))) return rc;
    return src;
}

extern "C" int eofa_solve_batch(odwf_t* h, int n, const double* m12, const void* const* b, void* const* x,
                                const odwf_solve_opts* opts, odwf_solve_stats* stats, void* stream) {
    using namespace odwf;
    if (!h || n < 0 || (n > 0 && (!m12 || !b || !x))) return set_err(h, ODWF_EINVAL, "null argument");
    int worst = ODWF_OK;
    for (int i = 0; i < n; ++i) {
        const int rc = eofa_solve(h, m12[2 * i], m12[2 * i + 1], b[i], x[i], opts, stats ? stats + i : nullptr, stream);
        if (rc != ODWF_OK && rc != ODWF_ENOCONV) return rc;
        if (rc != ODWF_OK) worst = rc;
    }
    return worst;
}
