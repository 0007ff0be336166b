// Even-odd preconditioned CGNE for D_T(m1, m2) x = b' with reliable updates, for one system or
// a batch of independent systems.
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
// (two fused hop + fifth-dimension passes for S, two for S^dag), with the CG scalars kept on the
// device. A batch of systems (same Ns; any masses, any lattices) runs in lockstep: each launch
// covers every system (blockIdx.y), systems that stop early return at once, and the host handles
// each system's reliable updates separately. The chunk of iterations between two host polls is
// captured once into a CUDA graph and replayed.
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "odwf_internal.h"

namespace odwf {

static inline const double* mat(const SCoef* c, int k, int Ns) { return c->dev + (size_t)k * Ns * Ns; }
enum { M_AP = 0, M_AINV = 2, M_AT = 4, M_AINVT = 6 };

struct InnerFields {
    int stg;
    void *x, *r, *p, *t;
    float *xs, *rs, *ps, *ts;
};

// One system of a solve.
struct Slot {
    odwf_s* h = nullptr;
    Workspace* ws = nullptr;
    int ws_index = -1;
    CGState* state = nullptr;    // device
    CGState* hstate = nullptr;   // pinned mirror
    double* partials = nullptr;
    const SCoef* c = nullptr;
    double m1 = 0, m2 = 0;
    InnerFields f{};
    double bnorm2 = 0, tol2 = 0, rr64 = 0, beta_keep = 0;
    int iters = 0, updates = 0, status = ODWF_OK;
    bool done = false;
    odwf_solve_stats stats{0, 0, 0.0, 0.0};
};

static HopArgs k1_args(const Slot& s, bool dag) {
    HopArgs a{};
    a.in = dag ? s.f.r : s.f.p;
    a.in_scale = dag ? s.f.rs : s.f.ps;
    a.out = s.f.t;
    a.out_scale = s.f.ts;
    a.mhop = mat(s.c, dag ? M_AINVT : M_AINV, s.h->Ns);
    set_sop(a, s.c, dag ? (SOP_AINV | SOP_T) : SOP_AINV);
    a.c_hop = 1.0;
    a.g5 = dag ? G5_HOP_IN : 0;
    a.state = s.state;
    a.partials = s.partials;
    return a;
}

// CGNE forward half step: q = A p - 1/4 H_eo t ; x += alpha p ; r -= alpha q ; rr = |r|^2
static HopArgs k2a_args(const Slot& s) {
    HopArgs a{};
    a.in = s.f.t;
    a.in_scale = s.f.ts;
    a.own = s.f.p;
    a.own_scale = s.f.ps;
    a.mown = mat(s.c, M_AP, s.h->Ns);
    set_sop(a, s.c, SOP_A);
    a.c_hop = -0.25;
    a.x = s.f.x;
    a.x_scale = s.f.xs;
    a.r = s.f.r;
    a.r_scale = s.f.rs;
    a.state = s.state;
    a.partials = s.partials;
    return a;
}

// CGNE adjoint half step: z = g5 (A^T g5 r - 1/4 H_eo t) = S^dag r ; p = z + beta p ; pp = |p|^2
static HopArgs k2b_args(const Slot& s) {
    HopArgs a{};
    a.in = s.f.t;
    a.in_scale = s.f.ts;
    a.own = s.f.r;
    a.own_scale = s.f.rs;
    a.mown = mat(s.c, M_AT, s.h->Ns);
    set_sop(a, s.c, SOP_A | SOP_T);
    a.c_hop = -0.25;
    a.g5 = G5_OWN_IN | G5_OUT;
    a.r = s.f.p;
    a.r_scale = s.f.ps;
    a.state = s.state;
    a.partials = s.partials;
    return a;
}

static int k1(const Slot& s, bool dag, cudaStream_t st) {
    return launch_hop(s.h, s.f.stg, 1, true, false, false, EPI_STORE, k1_args(s, dag), st);
}
static int k2a(const Slot& s, cudaStream_t st) {
    return launch_hop(s.h, s.f.stg, 0, false, true, true, EPI_CG_A, k2a_args(s), st);
}
static int k2b(const Slot& s, cudaStream_t st) {
    return launch_hop(s.h, s.f.stg, 0, false, true, true, EPI_CG_B, k2b_args(s), st);
}

// FP64: out = bh - S x (even parity), result[rslot] = |out|^2 ; tmp holds the odd intermediate
static int schur_residual64(const Slot& s, const void* x, void* tmp, void* out, int rslot, cudaStream_t st) {
    odwf_s* h = s.h;
    HopArgs a{};
    a.in = x;
    a.out = tmp;
    a.mhop = mat(s.c, M_AINV, h->Ns);
    set_sop(a, s.c, SOP_AINV);
    a.c_hop = 1.0;
    int rc = launch_hop(h, ST_DOUBLE, 1, true, false, false, EPI_STORE, a, st);
    if (rc) return rc;
    HopArgs b{};
    b.in = tmp;
    b.own = x;
    b.out = out;
    b.mown = mat(s.c, M_AP, h->Ns);
    set_sop(b, s.c, SOP_A);
    b.c_hop = -0.25;
    b.x = s.ws->bh;
    b.slot = rslot;
    b.state = s.state;
    b.partials = s.partials;
    return launch_hop(h, ST_DOUBLE, 0, false, true, true, EPI_RESID, b, st);
}

static int read_slot(Slot& s, cudaStream_t st) {
    return cuda_check(s.h, cudaMemcpyAsync(s.hstate, s.state, sizeof(CGState), cudaMemcpyDeviceToHost, st), "state D2H");
}

static int sync(odwf_s* h, cudaStream_t st) { return cuda_check(h, cudaStreamSynchronize(st), "stream sync"); }

// Phase 1: |b'|^2, b_hat = b'_e + 1/2 H_eo A^{-1} b'_o, |b_hat|^2 (b' already packed in ws->b_e/b_o)
static int prepare(Slot& s, cudaStream_t st) {
    odwf_s* h = s.h;
    Workspace& w = *s.ws;
    int rc;
    if ((rc = launch_norm2(h, w.b_e, ST_DOUBLE, nullptr, 0, st, s.state, s.partials))) return rc;
    if ((rc = launch_norm2(h, w.b_o, ST_DOUBLE, nullptr, 1, st, s.state, s.partials))) return rc;
    if ((rc = launch_smix(h, ST_DOUBLE, w.b_o, w.t64, mat(s.c, M_AINV, h->Ns), 1.0, st, nullptr, nullptr, s.c,
                          SOP_AINV)))
        return rc;
    HopArgs a{};
    a.in = w.t64;
    a.own = w.b_e;
    a.out = w.bh;
    a.a_own = 1.0;
    a.c_hop = 0.5;
    if ((rc = launch_hop(h, ST_DOUBLE, 0, false, true, false, EPI_STORE, a, st))) return rc;
    if ((rc = launch_norm2(h, w.bh, ST_DOUBLE, nullptr, 2, st, s.state, s.partials))) return rc;
    const size_t b64 = half_elems_bytes(h, ST_DOUBLE);
    if ((rc = cuda_check(h, cudaMemsetAsync(w.x_e, 0, b64, st), "memset"))) return rc;
    return cuda_check(h, cudaMemcpyAsync(w.r64, w.bh, b64, cudaMemcpyDeviceToDevice, st), "copy");
}

// Start a Krylov cycle from the FP64 residual in r64: x_inner = 0, r_inner = r64, and the next
// search direction p = S^dag r + beta' p (beta' = 0 with p = 0 on the first cycle; after a
// residual replacement beta' = |r_true|^2 / |r_prev|^2, the last step having consumed p).
static int start_cycle(Slot& s, const odwf_solve_opts& o, cudaStream_t st) {
    odwf_s* h = s.h;
    const size_t bi = half_elems_bytes(h, s.f.stg);
    const size_t bs = sizeof(float) * (size_t)h->Vh * h->Ns;
    int rc;
    if ((rc = cuda_check(h, cudaMemsetAsync(s.f.x, 0, bi, st), "memset"))) return rc;
    if (s.f.stg == ST_HALF && (rc = cuda_check(h, cudaMemsetAsync(s.f.xs, 0, bs, st), "memset"))) return rc;
    if ((rc = launch_convert(h, s.ws->r64, ST_DOUBLE, nullptr, s.f.r, s.f.stg, s.f.rs, st))) return rc;
    // the pinned mirror may still be the target of an earlier read: let it land first
    if ((rc = sync(h, st))) return rc;
    CGState& hs = *s.hstate;
    std::memset(&hs, 0, sizeof(CGState));
    hs.rr = s.rr64;
    hs.rr_max = s.rr64;
    hs.tol2 = (s.f.stg == ST_DOUBLE ? 0.81 : 0.25) * s.tol2;
    hs.delta2 = (s.f.stg == ST_DOUBLE) ? 0.0 : o.delta * o.delta;
    hs.maxiter = o.maxiter - s.iters;
    hs.beta = (s.updates == 0) ? 0.0 : s.beta_keep;
    if ((rc = cuda_check(h, cudaMemcpyAsync(s.state, s.hstate, sizeof(CGState), cudaMemcpyHostToDevice, st), "state H2D")))
        return rc;
    if ((rc = sync(h, st))) return rc;
    if (s.updates == 0) {
        if ((rc = cuda_check(h, cudaMemsetAsync(s.f.p, 0, bi, st), "memset"))) return rc;
        if (s.f.stg == ST_HALF && (rc = cuda_check(h, cudaMemsetAsync(s.f.ps, 0, bs, st), "memset"))) return rc;
    }
    if ((rc = k1(s, true, st))) return rc;
    return k2b(s, st);
}

// Reliable update after a cycle stopped: x64 += x_inner ; r64 = b_hat - S x64 (FP64). The new
// |r64|^2 is read after the next synchronisation.
static int begin_update(Slot& s, cudaStream_t st) {
    int rc = launch_axpy_to64(s.h, 1.0, s.f.x, s.f.stg, s.f.xs, (double*)s.ws->x_e, st);
    if (rc) return rc;
    return schur_residual64(s, s.ws->x_e, s.ws->t64, s.ws->r64, 3, st);
}

// x_o = A^{-1}(b'_o + 1/2 H_oe x_e), then the FP64 true residual of the full system
static int finish(Slot& s, cudaStream_t st) {
    odwf_s* h = s.h;
    Workspace& w = *s.ws;
    int rc;
    HopArgs a{};
    a.in = w.x_e;
    a.own = w.b_o;
    a.out = w.x_o;
    a.a_own = 1.0;
    a.c_hop = 0.5;
    a.mhop = mat(s.c, M_AINV, h->Ns);
    set_sop(a, s.c, SOP_AINV);
    if ((rc = launch_hop(h, ST_DOUBLE, 1, true, true, false, EPI_STORE, a, st))) return rc;
    HopArgs b{};
    b.mown = mat(s.c, M_AP, h->Ns);
    set_sop(b, s.c, SOP_A);
    b.c_hop = -0.5;
    b.in = w.x_o;
    b.own = w.x_e;
    b.x = w.b_e;
    b.out = w.r64;
    b.slot = 0;
    b.state = s.state;
    b.partials = s.partials;
    if ((rc = launch_hop(h, ST_DOUBLE, 0, false, true, true, EPI_RESID, b, st))) return rc;
    b.in = w.x_e;
    b.own = w.x_o;
    b.x = w.b_o;
    b.out = w.t64;
    b.slot = 1;
    return launch_hop(h, ST_DOUBLE, 1, false, true, true, EPI_RESID, b, st);
}

static bool use_graphs() {
    const char* e = std::getenv("ODWF_NO_GRAPH");
    return !(e && e[0] == '1');
}

// A chunk of `iters` CGNE iterations for every system: four launches per iteration.
static int enqueue_chunk(std::vector<Slot>& S, const HopArgs* dargs, int iters, int max_vh, cudaStream_t st) {
    const int n = (int)S.size();
    odwf_s* h0 = S[0].h;
    const int stg = S[0].f.stg;
    bool sn = h0->Ns == kStructNs;
    for (const Slot& s : S) sn = sn && s.c->has_st;
    int rc;
    for (int i = 0; i < iters; ++i) {
        if (n == 1) {
            if ((rc = k1(S[0], false, st)) || (rc = k2a(S[0], st)) || (rc = k1(S[0], true, st)) || (rc = k2b(S[0], st)))
                return rc;
        } else {
            if ((rc = launch_hop_multi(h0, stg, true, false, false, EPI_STORE, dargs + 0 * n, n, max_vh, st, sn))) return rc;
            if ((rc = launch_hop_multi(h0, stg, false, true, true, EPI_CG_A, dargs + 1 * n, n, max_vh, st, sn))) return rc;
            if ((rc = launch_hop_multi(h0, stg, true, false, false, EPI_STORE, dargs + 2 * n, n, max_vh, st, sn))) return rc;
            if ((rc = launch_hop_multi(h0, stg, false, true, true, EPI_CG_B, dargs + 3 * n, n, max_vh, st, sn))) return rc;
        }
    }
    return ODWF_OK;
}

// Solve every slot (b' already packed into each slot's ws->b_e / b_o); solutions in ws->x_e / x_o.
int solve_slots(std::vector<Slot>& S, const odwf_solve_opts* opts_in, cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    const bool debug = std::getenv("ODWF_DEBUG") != nullptr;
    odwf_solve_opts o{1e-10, 100000, ODWF_PREC_DOUBLE, 0.1, 0.0};
    if (opts_in) o = *opts_in;
    odwf_s* h0 = S[0].h;
    if (!(o.tol > 0.0) || o.maxiter < 1) return set_err(h0, ODWF_EINVAL, "bad solve options");
    if (o.prec != ODWF_PREC_DOUBLE && o.prec != ODWF_PREC_SINGLE && o.prec != ODWF_PREC_HALF)
        return set_err(h0, ODWF_EINVAL, "bad precision");
    const int stg = o.prec == ODWF_PREC_DOUBLE ? ST_DOUBLE : (o.prec == ODWF_PREC_SINGLE ? ST_FLOAT : ST_HALF);
    const int n = (int)S.size();
    int rc;
    int max_vh = 0;
    for (Slot& s : S) {
        if ((rc = ensure_ws(s.h, *s.ws, stg))) return rc;
        s.c = get_coef(s.h, s.m1, s.m2);
        if (!s.c) return ODWF_EINVAL;
        Workspace& w = *s.ws;
        s.f = InnerFields{stg, w.xi, w.ri, w.pi, w.ti, nullptr, nullptr, nullptr, nullptr};
        if (stg == ST_HALF) {
            s.f.xs = w.xi_s; s.f.rs = w.ri_s; s.f.ps = w.pi_s; s.f.ts = w.ti_s;
        }
        if (s.h->Vh > max_vh) max_vh = s.h->Vh;
        if ((rc = prepare(s, st))) return rc;
    }
    for (Slot& s : S)
        if ((rc = read_slot(s, st))) return rc;
    if ((rc = sync(h0, st))) return rc;
    int active = 0;
    for (Slot& s : S) {
        s.bnorm2 = s.hstate->result[0] + s.hstate->result[1];
        s.rr64 = s.hstate->result[2];
        s.tol2 = o.tol * o.tol * s.bnorm2;
        if (!std::isfinite(s.bnorm2) || !std::isfinite(s.rr64)) {
            s.status = set_err(s.h, ODWF_EBREAKDOWN, "non-finite right-hand side (|b|^2 is not finite)");
            s.done = true;
            continue;
        }
        if (s.bnorm2 == 0.0 || s.rr64 <= s.tol2) {
            s.done = true;
            continue;
        }
        if ((rc = start_cycle(s, o, st))) return rc;
        ++active;
    }

    // kernel arguments of the multi-system launches, uploaded once per call
    HopArgs* dargs = nullptr;
    if (n > 1) {
        std::vector<HopArgs> args(4 * (size_t)n);
        for (int i = 0; i < n; ++i) {
            args[0 * n + i] = k1_args(S[i], false);
            args[1 * n + i] = k2a_args(S[i]);
            args[2 * n + i] = k1_args(S[i], true);
            args[3 * n + i] = k2b_args(S[i]);
            hop_fill(S[i].h, stg, 1, args[0 * n + i], false);
            hop_fill(S[i].h, stg, 0, args[1 * n + i], true);
            hop_fill(S[i].h, stg, 1, args[2 * n + i], false);
            hop_fill(S[i].h, stg, 0, args[3 * n + i], true);
        }
        if (h0->bargs_cap < 4 * n) {
            cudaFree(h0->bargs);
            h0->bargs = nullptr;
            h0->bargs_cap = 0;
            if (cudaMalloc((void**)&h0->bargs, sizeof(HopArgs) * 4 * n) != cudaSuccess)
                return set_err(h0, ODWF_ENOMEM, "cudaMalloc batch arguments");
            h0->bargs_cap = 4 * n;
        }
        if ((rc = cuda_check(h0, cudaMemcpyAsync(h0->bargs, args.data(), sizeof(HopArgs) * 4 * n,
                                                 cudaMemcpyHostToDevice, st), "args H2D")))
            return rc;
        if ((rc = sync(h0, st))) return rc;
        dargs = h0->bargs;
    }

    // chunk graph (captured on a private non-default stream, launched on the caller's stream)
    const int kChunk = 16;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    bool prof_any = false;
    for (Slot& s : S) prof_any |= s.h->prof;
    if (use_graphs() && !prof_any && active > 0) {
        // one real iteration first, so every kernel's attributes and occupancy are set up outside
        // the capture
        if ((rc = enqueue_chunk(S, dargs, 1, max_vh, st))) return rc;
        if (!h0->cap_stream && cudaStreamCreateWithFlags(&h0->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            return set_err(h0, ODWF_ECUDA, "cudaStreamCreate");
        if ((rc = cuda_check(h0, cudaStreamBeginCapture(h0->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture")))
            return rc;
        const int erc = enqueue_chunk(S, dargs, kChunk, max_vh, h0->cap_stream);
        const cudaError_t ce = cudaStreamEndCapture(h0->cap_stream, &graph);
        if (erc) {
            if (graph) cudaGraphDestroy(graph);
            return erc;
        }
        if ((rc = cuda_check(h0, ce, "end capture"))) return rc;
        if ((rc = cuda_check(h0, cudaGraphInstantiate(&gexec, graph, 0), "graph instantiate"))) {
            cudaGraphDestroy(graph);
            return rc;
        }
    }
    struct GraphGuard {
        cudaGraphExec_t& e;
        cudaGraph_t& g;
        ~GraphGuard() {
            if (e) cudaGraphExecDestroy(e);
            if (g) cudaGraphDestroy(g);
        }
    } guard{gexec, graph};

    int chunk = 8;
    long queued = 0;
    while (active > 0) {
        if (gexec) {
            if ((rc = cuda_check(h0, cudaGraphLaunch(gexec, st), "graph launch"))) return rc;
            queued += kChunk;
        } else {
            if ((rc = enqueue_chunk(S, dargs, chunk, max_vh, st))) return rc;
            queued += chunk;
            if (chunk < 64) chunk *= 2;
        }
        for (Slot& s : S)
            if (!s.done && (rc = read_slot(s, st))) return rc;
        if ((rc = sync(h0, st))) return rc;
        if (debug) {
            for (int i = 0; i < n; ++i) {
                const CGState& d = *S[i].hstate;
                if (!S[i].done)
                    std::fprintf(stderr, "[odwf] sys %d cycle %d iter %d flag %d rr %.6e pp %.6e\n", i, S[i].updates,
                                 d.iter, d.flag, d.rr, d.pp);
            }
        }
        // systems that stopped: breakdown, or a reliable update / convergence check
        std::vector<Slot*> upd;
        for (Slot& s : S) {
            if (s.done) continue;
            const CGState& d = *s.hstate;
            if (d.flag == FLAG_RUN) {
                // host-side guard: the device stops at maxiter; never queue far past it
                if (queued > (long)o.maxiter + 4096) {
                    s.status = set_err(s.h, ODWF_ENOCONV, "solver state stopped advancing");
                    s.iters += d.iter;
                    s.done = true;
                    --active;
                }
                continue;
            }
            s.iters += d.iter;
            if (d.flag == FLAG_BREAKDOWN) {
                s.status = set_err(s.h, ODWF_EBREAKDOWN, "CGNE breakdown (<p,p> <= 0 or non-finite reduction)");
                s.done = true;
                --active;
                continue;
            }
            // previous iterated |r|^2 = rr / beta (the device set beta = rr_new / rr_old)
            s.beta_keep = d.beta > 0.0 ? d.rr / d.beta : 0.0;  // holds rr_prev until the update lands
            if ((rc = begin_update(s, st))) return rc;
            upd.push_back(&s);
        }
        if (!upd.empty()) {
            for (Slot* s : upd)
                if ((rc = read_slot(*s, st))) return rc;
            if ((rc = sync(h0, st))) return rc;
            for (Slot* s : upd) {
                const double rr_prev = s->beta_keep;
                s->rr64 = s->hstate->result[3];
                s->beta_keep = rr_prev > 0.0 ? s->rr64 / rr_prev : 0.0;
                ++s->updates;
                if (debug)
                    std::fprintf(stderr, "[odwf] update %d: true |r|^2 %.6e (tol2 %.6e), beta' %.6e\n", s->updates,
                                 s->rr64, s->tol2, s->beta_keep);
                if (!std::isfinite(s->rr64)) {
                    s->status = set_err(s->h, ODWF_EBREAKDOWN, "non-finite true residual");
                    s->done = true;
                    --active;
                } else if (s->rr64 <= s->tol2 || s->iters >= o.maxiter) {
                    s->done = true;  // its device flag stays set, so later launches skip it
                    --active;
                } else if ((rc = start_cycle(*s, o, st))) {
                    return rc;
                }
            }
        }
        if (active > 0 && o.max_seconds > 0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > o.max_seconds) {
            for (Slot& s : S)
                if (!s.done) {
                    s.status = set_err(s.h, ODWF_ETIMEOUT, "solver exceeded max_seconds");
                    s.iters += s.hstate->iter;
                    s.done = true;
                }
            active = 0;
        }
    }

    for (Slot& s : S) {
        if (s.bnorm2 == 0.0) {
            const size_t b64 = half_elems_bytes(s.h, ST_DOUBLE);
            cudaMemsetAsync(s.ws->x_e, 0, b64, st);
            cudaMemsetAsync(s.ws->x_o, 0, b64, st);
            continue;
        }
        if (s.status == ODWF_EBREAKDOWN) continue;
        if ((rc = finish(s, st))) return rc;
    }
    for (Slot& s : S)
        if ((rc = read_slot(s, st))) return rc;
    if ((rc = sync(h0, st))) return rc;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int worst = ODWF_OK;
    // a bulk-staged kernel whose bounded wait ran out left part of its outputs unwritten
    for (Slot& s : S)
        if ((rc = check_fault(s.h, st))) {
            if (rc != ODWF_EFAULT) return rc;
            s.status = rc;
        }
    for (Slot& s : S) {
        s.stats.iters = s.iters;
        s.stats.reliable_updates = s.updates;
        s.stats.seconds = secs;
        if (s.bnorm2 > 0.0 && s.status != ODWF_EBREAKDOWN) {
            const double res = std::sqrt((s.hstate->result[0] + s.hstate->result[1]) / s.bnorm2);
            s.stats.true_residual = res;
            if (s.status == ODWF_OK && !(res <= o.tol))
                s.status = set_err(s.h, ODWF_ENOCONV, "true residual " + std::to_string(res) + " above tol after " +
                                                          std::to_string(s.iters) + " iterations");
        }
        if (s.status != ODWF_OK && (worst == ODWF_OK || worst == ODWF_ENOCONV)) worst = s.status;
        if (s.status == ODWF_EFAULT) worst = ODWF_EFAULT;
    }
    return worst;
}

// Single system on the handle's own workspace and state.
int solve_core(odwf_s* h, double m1, double m2, const odwf_solve_opts* opts, odwf_solve_stats* stats, cudaStream_t st) {
    std::vector<Slot> S(1);
    Slot& s = S[0];
    s.h = h;
    s.ws = &h->ws;
    s.state = h->state;
    s.hstate = h->state_host;
    s.partials = h->partials;
    s.m1 = m1;
    s.m2 = m2;
    const int rc = solve_slots(S, opts, st);
    if (stats) *stats = s.stats;
    return rc;
}

// Batch pools of a handle: k systems' workspaces, states and reduction buffers.
static int ensure_batch(odwf_s* h, int k) {
    if ((int)h->bws.size() < k) h->bws.resize(k);
    if (h->bcap >= k) return ODWF_OK;
    cudaFree(h->bstate);
    cudaFree(h->bpartials);
    if (h->bstate_host) cudaFreeHost(h->bstate_host);
    h->bstate = nullptr;
    h->bpartials = nullptr;
    h->bstate_host = nullptr;
    h->bcap = 0;
    if (cudaMalloc((void**)&h->bstate, sizeof(CGState) * k) != cudaSuccess ||
        cudaMalloc((void**)&h->bpartials, sizeof(double) * h->partials_n * (size_t)k) != cudaSuccess ||
        cudaMallocHost((void**)&h->bstate_host, sizeof(CGState) * k) != cudaSuccess)
        return set_err(h, ODWF_ENOMEM, "batch pools");
    if (cudaMemset(h->bstate, 0, sizeof(CGState) * k) != cudaSuccess) return set_err(h, ODWF_ECUDA, "memset");
    h->bcap = k;
    return ODWF_OK;
}

// Systems on possibly different handles (same Ns): H_T(m12[2i], m12[2i+1]) x[i] = b[i] on hs[i].
int solve_multi(odwf_s* const* hs, int n, const double* m12, const void* const* b, void* const* x,
                const odwf_solve_opts* opts, odwf_solve_stats* stats, cudaStream_t st) {
    std::vector<Slot> S(n);
    std::vector<std::pair<odwf_s*, int>> counts;  // handle, systems so far
    int rc;
    for (int i = 0; i < n; ++i) {
        odwf_s* h = hs[i];
        if (!h || !b[i] || !x[i]) return set_err(hs[0], ODWF_EINVAL, "null argument");
        if (!h->have_gauge) return set_err(h, ODWF_EINVAL, "odwf_set_gauge has not been called");
        if (h->Ns != hs[0]->Ns) return set_err(hs[0], ODWF_EINVAL, "a batch must share Ns");
        const double m1 = m12[2 * i], m2 = m12[2 * i + 1];
        if (!(m1 > 0.0 && m1 <= 1.0) || !(m2 > 0.0 && m2 <= 1.0)) return set_err(h, ODWF_EINVAL, "masses must lie in (0, 1]");
        int k = -1;
        for (auto& c : counts)
            if (c.first == h) k = c.second++;
        if (k < 0) {
            counts.push_back({h, 1});
            k = 0;
        }
        S[i].h = h;
        S[i].m1 = m1;
        S[i].m2 = m2;
        S[i].ws_index = k;
    }
    for (auto& c : counts)
        if ((rc = ensure_batch(c.first, c.second))) return rc;
    for (int i = 0; i < n; ++i) {
        odwf_s* h = S[i].h;
        const int k = S[i].ws_index;
        S[i].ws = &h->bws[k];
        S[i].state = h->bstate + k;
        S[i].hstate = h->bstate_host + k;
        S[i].partials = h->bpartials + (size_t)k * h->partials_n;
        if ((rc = ensure_ws(h, *S[i].ws, ST_DOUBLE))) return rc;
        // H_T x = b  <=>  D_T x = R5 gamma_5 b
        if ((rc = launch_pack5(h, (const double*)b[i], S[i].ws->b_e, S[i].ws->b_o, ST_DOUBLE, 1, st))) return rc;
    }
    const int src = solve_slots(S, opts, st);
    if (src != ODWF_OK && src != ODWF_ENOCONV && src != ODWF_ETIMEOUT && src != ODWF_EBREAKDOWN) return src;
    for (int i = 0; i < n; ++i) {
        if (stats) stats[i] = S[i].stats;
        if ((rc = launch_unpack5(S[i].h, S[i].ws->x_e, S[i].ws->x_o, (double*)x[i], ST_DOUBLE, 0, st))) return rc;
    }
    if ((rc = sync(hs[0], st))) return rc;
    return src;
}

// n systems on handle h sharing one right-hand side b' given in the internal FP64 layout (be, bo):
// D_T(m12[2i], m12[2i+1]) x_i = b'. On return ws_out[i] holds x_i in x_e / x_o.
int solve_shared_rhs(odwf_s* h, int n, const double* m12, const void* be, const void* bo, const odwf_solve_opts* opts,
                     odwf_solve_stats* stats, std::vector<Workspace*>& ws_out, cudaStream_t st) {
    int rc = ensure_batch(h, n);
    if (rc) return rc;
    std::vector<Slot> S(n);
    const size_t b64 = half_elems_bytes(h, ST_DOUBLE);
    ws_out.assign(n, nullptr);
    for (int i = 0; i < n; ++i) {
        S[i].h = h;
        S[i].m1 = m12[2 * i];
        S[i].m2 = m12[2 * i + 1];
        S[i].ws = &h->bws[i];
        S[i].state = h->bstate + i;
        S[i].hstate = h->bstate_host + i;
        S[i].partials = h->bpartials + (size_t)i * h->partials_n;
        if ((rc = ensure_ws(h, *S[i].ws, ST_DOUBLE))) return rc;
        if ((rc = cuda_check(h, cudaMemcpyAsync(S[i].ws->b_e, be, b64, cudaMemcpyDeviceToDevice, st), "copy"))) return rc;
        if ((rc = cuda_check(h, cudaMemcpyAsync(S[i].ws->b_o, bo, b64, cudaMemcpyDeviceToDevice, st), "copy"))) return rc;
        ws_out[i] = S[i].ws;
    }
    const int src = solve_slots(S, opts, st);
    for (int i = 0; i < n; ++i)
        if (stats) stats[i] = S[i].stats;
    return src;
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
    if (src != ODWF_OK && src != ODWF_ENOCONV && src != ODWF_ETIMEOUT) return src;
    if ((rc = launch_unpack5(h, h->ws.x_e, h->ws.x_o, (double*)x, ST_DOUBLE, 0, st))) return rc;
    return src;
}

extern "C" int eofa_solve_batch(odwf_t* h, int n, const double* m12, const void* const* b, void* const* x,
                                const odwf_solve_opts* opts, odwf_solve_stats* stats, void* stream) {
    using namespace odwf;
    if (!h || n < 0 || (n > 0 && (!m12 || !b || !x))) return set_err(h, ODWF_EINVAL, "null argument");
    if (n == 0) return ODWF_OK;
    std::vector<odwf_s*> hs(n, h);
    return solve_multi(hs.data(), n, m12, b, x, opts, stats, (cudaStream_t)stream);
}

extern "C" int eofa_solve_multi(odwf_t* const* hs, int n, const double* m12, const void* const* b, void* const* x,
                                const odwf_solve_opts* opts, odwf_solve_stats* stats, void* stream) {
    using namespace odwf;
    if (!hs || n < 1 || !hs[0] || !m12 || !b || !x) return set_err(hs ? hs[0] : nullptr, ODWF_EINVAL, "null argument");
    return solve_multi(hs, n, m12, b, x, opts, stats, (cudaStream_t)stream);
}
