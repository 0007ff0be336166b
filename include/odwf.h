/*
 * odwf.h -- C ABI of the GB300 library for the exact one-flavor action (EOFA) of optimal
 * domain-wall fermions with mass preconditioning.
 *
 * Paper: Y.-C. Chen and T.-W. Chiu, "Mass Preconditioning for the Exact One-Flavor Action in
 * Lattice QCD with Domain-Wall Fermion", arXiv:1710.09621. Citations below are to its sections
 * and equation labels, written Eq.(label).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Status: every call returns int; ODWF_OK (0) on success, a negative ODWF_E* code otherwise.
 *    Nothing is thrown across the ABI. odwf_last_error(h) returns a message for the last failure
 *    on that handle (odwf_last_error(NULL) for failures of odwf_create).
 *  - Device pointers: every field argument is a CUDA device pointer owned by the caller, and must
 *    stay valid until the work queued on `stream` has finished. `stream` is a cudaStream_t passed
 *    as void* (NULL = the legacy default stream). All library work on a call is queued on that
 *    stream; calls that return host scalars (action, statistics) synchronise it.
 *  - Field layout at the ABI: complex128 (interleaved re, im doubles), C order,
 *      4D spinor   [t][z][y][x][spin 4][color 3]
 *      5D spinor   [s][t][z][y][x][spin 4][color 3]      s = 0..Ns-1 outermost
 *      gauge links [mu 4][t][z][y][x][a 3][b 3]          mu = 0..3 for x, y, z, t
 *    Gamma matrices are in the chiral basis gamma_5 = diag(1, 1, -1, -1): spins 0,1 are P_+,
 *    spins 2,3 are P_- (the phi_+ / phi_- split after Eq.(H)). Boundary conditions: periodic in
 *    x, y, z, antiperiodic in t for the fermion fields.
 *  - Masses are normalised masses m = m_q / m_PV with m_PV = 2 m0 (after Eq.(H), Section 3.1);
 *    1.0 is the Pauli-Villars mass. Every mass must lie in (0, 1].
 *  - The library owns its internal workspaces (even-odd copies of the fields in FP64, FP32 and
 *    FP16, the reordered gauge field, reduction buffers). A handle is not thread-safe.
 */
#ifndef ODWF_H
#define ODWF_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define ODWF_OK          0
#define ODWF_EINVAL     -1   /* bad argument: dims, Ns, masses, omega, null pointer, option   */
#define ODWF_ENOMEM     -2   /* device or host allocation failed                              */
#define ODWF_ECUDA      -3   /* a CUDA runtime call or kernel launch failed                   */
#define ODWF_ENOCONV    -4   /* the solver reached maxiter without meeting the tolerance      */
#define ODWF_EBREAKDOWN -5   /* Krylov breakdown: <p,p> <= 0 or a NaN/Inf in a reduction      */
#define ODWF_ETIMEOUT   -6   /* the solver exceeded its wall-clock budget                     */
#define ODWF_EFAULT     -7   /* a kernel's bounded wait for its bulk copies ran out: its outputs
                                are incomplete; the device and the handle stay usable           */
#define ODWF_ESPECTRUM  -8   /* heat-bath: the spectrum of X estimated by Lanczos lies outside
                                the interval of the rational approximation                      */

/* arithmetic of a call */
#define ODWF_PREC_DOUBLE 0   /* FP64 storage and arithmetic                                    */
#define ODWF_PREC_SINGLE 1   /* FP32 storage and arithmetic; solves add FP64 reliable updates  */
#define ODWF_PREC_HALF   2   /* FP16 storage with a per-site scale, FP32 arithmetic            */

/* operator selector of odwf_apply / odwf_apply_dag */
#define ODWF_OP_DT    0      /* D_T(m1, m2) of Eq.(DTm1m2)                                     */
#define ODWF_OP_HT    1      /* H_T(m1, m2) = gamma_5 R5 D_T(m1, m2) (after Eq.(m1m2_m3m2))    */
#define ODWF_OP_DODWF 2      /* D_odwf(m1, m2) = (omega D_w + 1) + (omega D_w - 1) L(m1, m2)   */

typedef struct odwf_s odwf_t;

typedef struct {
    double tol;          /* stop when ||b' - D_T x|| <= tol ||b'|| (FP64 true residual); e.g. 1e-10 */
    int    maxiter;      /* Krylov iterations, summed over reliable-update cycles                   */
    int    prec;         /* ODWF_PREC_*: inner-solver storage precision                             */
    double delta;        /* reliable-update trigger: |r_inner| < delta * max |r| since last update  */
    double max_seconds;  /* wall-clock budget; <= 0 means none                                      */
} odwf_solve_opts;

typedef struct {
    int    iters;            /* Krylov iterations (each: one Schur apply and one adjoint apply)  */
    int    reliable_updates; /* FP64 residual replacements                                        */
    double true_residual;    /* ||b' - D_T x|| / ||b'|| recomputed in FP64 after the solve        */
    double seconds;          /* host wall time of the call                                        */
} odwf_solve_stats;

/* One EOFA pseudofermion term, Eq.(m1m2_m3m4) in its two chiral special cases:
 *   chirality -1: (m3, m4)/(m3, m_den), Eq.(m1m2_m1m4), k = k(m_den, m4)
 *   chirality +1: (m3, m4)/(m_den, m4), Eq.(m1m2_m3m2), k = k(m_den, m3)
 * Its 4D operator is X = P [1 -/+ k Omega^T H_T(m3, m4)^{-1} Omega] P and its action phi^dag X phi. */
typedef struct {
    int    chirality;
    double m3, m4, m_den;
} eofa_term;

typedef struct {
    odwf_solve_opts solve;   /* options of every pole solve                                       */
    double x_lo, x_hi;       /* spectral interval of X for the rational approximation of X^{-1/2};
                                x_lo <= 0 selects [0.98 (1+m_ref)/(1+m_den), 1]                    */
    double rat_err;          /* target max relative error of the rational approximation (1e-11)   */
    int    n_poles_out;      /* written: number of poles used                                      */
    int    iters_out;        /* written: Krylov iterations summed over poles                       */
    int    check_iters;      /* > 0: first estimate the extreme eigenvalues of X with this many
                                Lanczos steps from eta (eofa_term_spectrum) and return
                                ODWF_ESPECTRUM if they fall outside [x_lo, x_hi]                   */
    double ritz_lo_out;      /* written when check_iters > 0: smallest / largest Ritz value        */
    double ritz_hi_out;
} odwf_hb_opts;

/* Create a handle for an Lx x Ly x Lz x Lt lattice (all even, each >= 2) with Ns slices
 * (even, 2..32), domain-wall height m0 (0 < m0 < 2) and weights omega[Ns] (host, each > 0,
 * R5-symmetric: omega_s == omega_{Ns-1-s}, which makes H_T Hermitian). The operator is the
 * optimal domain-wall fermion read with c = 1, d = 0 (m_PV = 2 m0, Section 3.1). flags: 0.
 * Returns ODWF_EINVAL for bad arguments, ODWF_ECUDA/ENOMEM on device failures. */
int odwf_create(odwf_t** h, const int dims[4], int Ns, double m0, const double* omega, int flags);
int odwf_destroy(odwf_t* h);
const char* odwf_last_error(const odwf_t* h);

/* Load the gauge field U (device, [4][V][3][3] complex128, unitary). The library keeps even-odd
 * reordered FP64, FP32 and FP16 copies with the antiperiodic sign folded in; U may be freed after
 * the stream reaches this point. Must be called before any operator, solve or EOFA call. */
int odwf_set_gauge(odwf_t* h, const void* U, void* stream);

/* out = Op(m1, m2) in, or its adjoint, on full 5D fields (device, complex128, ABI layout): D_T of
 * Eq.(DTm1m2), H_T = gamma_5 R5 D_T (after Eq.(m1m2_m3m2)) or D_odwf (Eq.(detDodwf)), see ODWF_OP_*.
 * prec: storage and arithmetic of the hopping and fifth-dimension kernels, in/out staying FP64:
 * ODWF_PREC_DOUBLE, ODWF_PREC_SINGLE, or ODWF_PREC_HALF (the input and every intermediate stored as
 * FP16 with one FP32 scale per (site, s), FP32 arithmetic: relative error a few 1e-4). in and out
 * must not overlap. Returns ODWF_EFAULT (after synchronising `stream`) if a bulk-staged kernel's
 * bounded wait ran out during the call. */
int odwf_apply(odwf_t* h, int op, double m1, double m2, const void* in, void* out, int prec, void* stream);
int odwf_apply_dag(odwf_t* h, int op, double m1, double m2, const void* in, void* out, int prec, void* stream);

/* Allocation-free variant of odwf_apply (forward D_T or H_T only; prec DOUBLE or SINGLE), for
 * callers that cannot allocate device memory while they run (a fixed memory budget set at start-up,
 * all memory handed to the caller's own pool, or a region where the allocator must not be touched).
 * The paper has no counterpart. It uses a 32 MiB file-scope device array instead of the handle's
 * work fields and allocates nothing; lattices whose four even-odd half fields plus coefficients
 * exceed 32 MiB (Vh * Ns above ~43,000 in FP64, ~87,000 in FP32) are rejected with ODWF_EINVAL.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current. Each call copies its fifth-dimension coefficients from pageable host memory,
 * so do not call it while `stream` is being captured into a CUDA graph. Every call shares the
 * array: calls whose GPU work overlaps race on it. The handle itself is created by odwf_create. */
int odwf_apply_noalloc(odwf_t* h, int op, double m1, double m2, const void* in, void* out, int prec, void* stream);

/* Solve H_T(m1, m2) x = b (5D, device, complex128), the system behind every EOFA heat-bath,
 * action and force (Eq.(m1m2_m1m4), Eq.(m1m2_m3m2)); CG is the paper's solver (Section 1).
 * Method: D_T x = R5 gamma_5 b, even-odd Schur complement S = A - 1/4 H_eo A^{-1} H_oe, CGNE on S,
 * inner precision opts->prec with FP64 reliable updates, FP64 true residual at the end.
 * opts may be NULL (tol 1e-10, maxiter 100000, FP64, delta 0.1). stats may be NULL.
 * Returns ODWF_ENOCONV / EBREAKDOWN / ETIMEOUT when the tolerance is not met (x holds the last
 * iterate). Synchronises `stream`. */
int eofa_solve(odwf_t* h, double m1, double m2, const void* b, void* x,
               const odwf_solve_opts* opts, odwf_solve_stats* stats, void* stream);

/* n independent solves H_T(m12[2i], m12[2i+1]) x[i] = b[i] on the same gauge field (e.g. the
 * terms of a mass-preconditioning scheme, Eq.(new_MP), or the poles of a heat-bath). The Krylov
 * iterations of all systems advance in lockstep on one stream: each kernel launch covers every
 * active system, and the chunk of iterations between host polls is one replayed CUDA graph.
 * stats: array of n (may be NULL). */
int eofa_solve_batch(odwf_t* h, int n, const double* m12, const void* const* b, void* const* x,
                     const odwf_solve_opts* opts, odwf_solve_stats* stats, void* stream);

/* Like eofa_solve_batch, but system i lives on its own handle hs[i] (lattices of different sizes,
 * one shared Ns): H_T(m12[2i], m12[2i+1]) x[i] = b[i] on hs[i]. All systems advance together, one
 * kernel launch per step covering every system. stats: array of n (may be NULL). */
int eofa_solve_multi(odwf_t* const* hs, int n, const double* m12, const void* const* b, void* const* x,
                     const odwf_solve_opts* opts, odwf_solve_stats* stats, void* stream);

/* S = phi^dag X phi for one term, X the 4D operator of Eq.(m1m2_m1m4) (chirality -) or
 * Eq.(m1m2_m3m2) (chirality +): X = 1 -/+ k Omega^T H_T(m3, m4)^{-1} Omega on the term's chirality,
 * one H_T solve. phi: 4D device field (only the term's chirality is read). Written to *S_host.
 * stats (may be NULL) receives the solve's statistics. Synchronises `stream`. */
int eofa_action(odwf_t* h, const eofa_term* term, const void* phi, double* S_host,
                const odwf_solve_opts* opts, odwf_solve_stats* stats, void* stream);

/* F^a_mu(x) = -dS/dw^a for U_mu(x) -> exp(i w^a t^a) U_mu(x), t^a = lambda^a / 2 (Section 1,
 * Eq.(molecular_U), Eq.(molecular_P)). F: device, double [4][V][8] (mu, lexicographic site, a). */
int eofa_force(odwf_t* h, const eofa_term* term, const void* phi, double* F,
               const odwf_solve_opts* opts, odwf_solve_stats* stats, void* stream);

/* Heat-bath phi = X^{-1/2} eta (Eq.(CG_gaussian)) with Zolotarev's optimal rational approximation
 * of x^{-1/2} on [x_lo, x_hi]; each pole is one shifted-mass H_T solve (Woodbury on Eq.(delta_ij)),
 * all poles solved as one batch. eta, phi: 4D device fields; phi gets only the term's chirality. */
int eofa_heatbath(odwf_t* h, const eofa_term* term, const void* eta, void* phi,
                  odwf_hb_opts* opts, void* stream);

/* Extreme eigenvalues of a term's 4D operator X (the operator of eofa_action) estimated by n_iter
 * (1..1000) steps of the Lanczos recurrence in FP64, started from P v0 (v0: 4D device field, only the
 * term's chirality is used; it must not vanish there). Each step applies X once, i.e. one H_T(m3, m4)
 * solve with `opts` (NULL: FP64 defaults). Writes the smallest and largest Ritz values, which lie
 * inside the spectrum of X and approach its ends as n_iter grows. The paper states X > 0 (Section 1)
 * and leaves the heat-bath's spectral interval to the implementer (Eq.(CG_gaussian)); this call lets
 * a caller check or choose that interval. Synchronises `stream`. */
int eofa_term_spectrum(odwf_t* h, const eofa_term* term, const void* v0, int n_iter, double* lo, double* hi,
                       const odwf_solve_opts* opts, void* stream);

/* ---- HMC molecular dynamics (Section 1: HMC outline, Eq.(molecular_U), Eq.(molecular_P);
 * Section 3: Omelyan integrator, multiple time scales, Wilson plaquette gauge action) -------------
 * U_l = exp(i A_l^a t^a), t^a = lambda^a / 2; momenta P_l = P_l^a t^a with H = 1/2 sum (P_l^a)^2 + S_g +
 * sum of the EOFA terms' actions; forces F^a = -dS/dw^a for U -> exp(i w^a t^a) U (as eofa_force).
 * Fields: U the ABI gauge layout (device, complex128, updated in place where stated), P and F device
 * double [4][V][8] (mu, lexicographic site, a). All of it is FP64. Every call synchronises `stream`
 * when it returns a host scalar. */

/* S_g = beta sum_{x, mu < nu} (1 - Re tr U_{mu nu}(x) / 3), U_{mu nu}(x) = U_mu(x) U_nu(x+mu)
 * U_mu(x+nu)^dag U_nu(x)^dag (periodic links), written to *S. */
int hmc_gauge_action(odwf_t* h, const void* U, double beta, double* S, void* stream);
/* F^a_mu(x) = -dS_g/dw^a = -(beta/3) Im tr(t^a U_mu(x) Sigma_mu(x)), Sigma_mu the sum of the six staples. */
int hmc_gauge_force(odwf_t* h, const void* U, double beta, double* F, void* stream);
/* P += eps F (a momentum update of Eq.(molecular_P) with a fixed force). */
int hmc_momentum_update(odwf_t* h, double* P, const double* F, double eps, void* stream);
/* U <- exp(i tau P^a t^a) U on every link (Eq.(molecular_U) over time tau at fixed P), in place, with the
 * exact SU(3) exponential (scaling and squaring of the Taylor series); also reloads the library's
 * reordered copies of U, so the operator, solve and EOFA calls act on the new links at once. */
int hmc_link_update(odwf_t* h, void* U, const double* P, double tau, void* stream);
/* K = 1/2 sum (P^a)^2, written to *K. */
int hmc_kinetic(odwf_t* h, const double* P, double* K, void* stream);

#define ODWF_HMC_MAX_LEVELS 4
typedef struct {
    double dH;              /* H(end) - H(start)                                                    */
    double K0, K1;          /* kinetic energy at the start and the end                               */
    double Sg0, Sg1;        /* gauge action                                                          */
    double Sf0, Sf1;        /* sum of the EOFA terms' actions                                        */
    int    force_evals[ODWF_HMC_MAX_LEVELS]; /* momentum updates (force evaluations) per level        */
    int    link_updates;
    long long cg_iters;     /* Krylov iterations of every solve of the trajectory                    */
    double seconds;
} hmc_md_stats;

/* One molecular-dynamics trajectory of length tau (step 5 of the HMC outline in Section 1): the
 * Omelyan integrator with nlevels time scales (Section 3). Level 0 carries the gauge force with
 * steps[0] steps per trajectory; EOFA term i (pseudofermion phis[i], fixed, e.g. from eofa_heatbath)
 * carries its force on level term_level[i] (0 <= level < nlevels), and level l has steps[l] steps
 * (steps[l] a multiple of 2 steps[l + 1]). One Omelyan step of size e on level l is
 *   P += lambda e F_l ; levels below over e/2 ; P += (1 - 2 lambda) e F_l ; levels below over e/2 ;
 *   P += lambda e F_l
 * and below level 0 is the link update over the half step; the smallest time step is tau/(2 steps[0])
 * ((k0, k1, k2) = (480, 12, 6) gives 960 link updates). Momentum updates of one level that meet at
 * the same links are applied as one (so level l evaluates its force 2 steps[l] + 1 times).
 * lambda: Omelyan's parameter (0.1931833275037836 for the minimum-norm scheme). U and P are
 * updated in place; stats (may be NULL) receives Delta H = H(end) - H(start) and its parts (each term's
 * action is one H_T solve at each end), the force evaluations per level and the Krylov iterations.
 * The accept / reject step and the momentum refresh are the caller's (it draws P). */
int hmc_md(odwf_t* h, void* U, double* P, double beta, int nterms, const eofa_term* terms,
           const void* const* phis, const int* term_level, int nlevels, const int* steps, double tau,
           double lambda, const odwf_solve_opts* opts, hmc_md_stats* stats, void* stream);

/* ---- learned preconditioner (not in the paper) ----------------------------------------------
 * A gauge-equivariant two-layer network of parallel-transport convolutions approximating S^{-1}
 * for the even-odd Schur complement S of D_T(m1, m2) (the system eofa_solve iterates on):
 *   u = A^{-1} r, v_c = A^{-1} sum_d W1[c,d] T_d u, M r = W0 u + 1/4 A^{-1} sum_{c,d} W2[c,d] T_d v_c,
 * T_d = parallel transport by one link along d (4 forward, 4 backward), W = 4x4 complex spin
 * matrices, c = 0..channels-1. Channel mixing runs on the tensor cores in BF16 with FP32
 * accumulation; everything else in FP32. Weights (complex128, host): W0 [4][4], then W1
 * [channels][8][4][4], then W2 [channels][8][4][4], each matrix [out spin][in spin]; the initial
 * weights make M the two-term Neumann series A^{-1} + 1/4 A^{-1} H A^{-1} H A^{-1} of S^{-1}. */
typedef struct odwf_net_s odwf_net_t;
int odwf_net_create(odwf_t* h, int channels, odwf_net_t** net);      /* channels 1 or 2 */
int odwf_net_destroy(odwf_net_t* net);
int odwf_net_num_params(const odwf_net_t* net);                       /* complex parameters */
int odwf_net_weights(odwf_net_t* net, double* host, int set);         /* set = 1 upload, 0 download */
/* M r (adjoint = 0) or M^dag r (adjoint = 1); r, out: 5D ABI fields, only even sites read, odd
 * sites of out set to zero. */
int odwf_net_apply(odwf_net_t* net, double m1, double m2, const void* r, void* out, int adjoint, void* stream);
/* Training pairs (r_i, e_i = S^{-1} r_i): r_i are 5D ABI fields (even sites used); if e is NULL the
 * library solves for e_i itself (FP32 CGNE with FP64 reliable updates to tol), except when the loss
 * selected beforehand is ODWF_NET_LOSS_RESIDUAL, which never reads e_i: then no solve runs, and a later
 * switch to ODWF_NET_LOSS_ERROR makes odwf_net_loss_grad / odwf_net_train return ODWF_EINVAL. An r_i that
 * vanishes (or is not finite) on the even sites is rejected with ODWF_EINVAL. */
int odwf_net_set_pairs(odwf_net_t* net, double m1, double m2, int npairs, const void* const* r,
                       const void* const* e, double tol, void* stream);
/* Training loss of odwf_net_loss_grad / odwf_net_train: ODWF_NET_LOSS_ERROR (default),
 * L = sum_i |M r_i - e_i|^2 / |e_i|^2, or ODWF_NET_LOSS_RESIDUAL, L = sum_i |S M r_i - r_i|^2 / |r_i|^2
 * (how far S M is from the identity on the training vectors; the e_i are not used). */
#define ODWF_NET_LOSS_ERROR    0
#define ODWF_NET_LOSS_RESIDUAL 1
int odwf_net_set_loss(odwf_net_t* net, int mode);
/* L (the selected loss) and dL/dconj(W) (host complex128, may be NULL). */
int odwf_net_loss_grad(odwf_net_t* net, double* loss, double* grad, void* stream);
/* steps Adam updates with learning rate lr on the stored pairs; losses[steps + 1] may be NULL. */
int odwf_net_train(odwf_net_t* net, int steps, double lr, double* losses, void* stream);
/* Attach net (created on h) so that the single-system solves of eofa_action, eofa_force and hmc_md use
 * the network-preconditioned CGNE of eofa_solve_learned (FP32 inner cycles with FP64 reliable updates
 * whenever the residual has dropped by opts->delta; opts->prec is not used) instead of plain CGNE; the
 * network applies the fifth-dimension inverse of each solve's own masses, its weights are shared. NULL
 * detaches. The heat-bath keeps the batched plain solver for its poles. Not in the paper. */
int odwf_set_preconditioner(odwf_t* h, odwf_net_t* net);
/* H_T(m1, m2) x = b like eofa_solve, with CGNE on S M (right preconditioning by the network, the
 * iterate accumulating x = M y directly), FP32 inner cycles whose residual is replaced by the FP64 one
 * whenever it has dropped by opts->delta (reliable updates: the search direction and the last beta carry
 * over into the next cycle). */
int eofa_solve_learned(odwf_t* h, odwf_net_t* net, double m1, double m2, const void* b, void* x,
                       const odwf_solve_opts* opts, odwf_solve_stats* stats, void* stream);
/* H_T(m1, m2) x = b like eofa_solve, with flexible GCR on the even-odd Schur system S (Sec. 2, the
 * even-odd preconditioned D_T), right-preconditioned by the network (net may be NULL: plain GCR).
 * Not in the paper, which solves with CG. Each step applies the network and S once and
 * orthonormalises the new direction S z (classical Gram-Schmidt) against a basis of up to nvec - 1
 * earlier ones (1 <= nvec <= 16): truncate = 0 restarts with an empty basis every nvec steps,
 * truncate = 1 keeps the last nvec - 1 directions (sliding window). FP32 inner iteration whose
 * residual is replaced by the FP64 true residual whenever it has dropped by opts->delta;
 * stats->reliable_updates counts those replacements. Allocates 2 nvec + 3 FP32 half fields on the
 * handle (kept until odwf_destroy). Returns ODWF_EINVAL for nvec outside 1..16 or masses outside
 * (0, 1], ODWF_ENOCONV if opts->maxiter steps end above tol, ODWF_ETIMEOUT if opts->max_seconds
 * (> 0, checked every nvec steps) ran out; x and stats then hold the last iterate and its true
 * residual. */
int eofa_solve_gcr(odwf_t* h, odwf_net_t* net, double m1, double m2, const void* b, void* x, int nvec, int truncate,
                   const odwf_solve_opts* opts, odwf_solve_stats* stats, void* stream);

/* Autotuner: times the launch choices (fifth-dimension form at Ns = 16: the structured recurrence or the
 * dense Ns x Ns product; at Ns = 16 with SU(3) links the two-slices-per-thread kernels with two-row links,
 * their neighbours gathered into registers or by bulk copies through 2 or 3 shared-memory stages; tile:
 * the default number of sites per CTA or twice it, as long as the CTA stays within 256 threads; grid
 * size: one resident wave, one CTA per site group, two or four waves; per-thread neighbour gathers or
 * bulk-staged gathers) of the four fused kernels of the
 * CGNE iteration in precision prec on this handle's lattice and keeps the fastest for later calls.
 * report (may be NULL) receives the timings as text. Overwrites the handle's inner work fields and
 * solver state; call it between solves. The paper has no counterpart (a tuning aid). */
int odwf_autotune(odwf_t* h, int prec, char* report, int report_len, void* stream);

/* Persisted autotuner choices: if the text file `path` holds an entry for this device name, lattice,
 * Ns and precision, its choices are applied (*hit = 1, no timing); otherwise odwf_autotune runs and
 * its choices are appended to the file as one line (*hit = 0). Returns ODWF_EINVAL if the file cannot
 * be appended to. Entries are plain text: device|LxxLyxLzxLt|Ns|prec|key:grid-mode:staged:tile:dense:two-slice,...
 * (two-slice: 0 none, 1 register gathers, 2 / 3 bulk-copy stages; older 5-field entries read it as 0) */
int odwf_autotune_cache(odwf_t* h, int prec, const char* path, int* hit, void* stream);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (independent FMA chains on every SM,
 * CUDA-event timed): the roof of the FP64 hop kernels, which the double-precision pipe bounds rather
 * than HBM. A measurement aid with no counterpart in the paper; allocates and frees a small buffer. */
int odwf_fp64_fma_peak(odwf_t* h, double* tflops, void* stream);

/* Kernel timing for measurement: while enabled, every launch of the library's kernels on this
 * handle (hopping, network, GCR, layout and vector kernels) is bracketed by CUDA events on its
 * stream. odwf_profile_read synchronises the device and returns, per kernel variant seen since the
 * last enable, its key, the number of launches and the summed event time in milliseconds; n_io is
 * the capacity of the arrays on entry and the number of variants on exit. Keys: hopping kernels
 * storage*100000 + hop*10000 + mixhop*1000 + own*100 + mixown*10 + epilogue (+1000000 for the
 * bulk-staged gathers); network layers 2000000 + bf16*1000 + cin*100 + cout*10 + own; GCR kernels
 * 3000000 + kind*100 + basis size; layout / vector kernels 4000000 + kind*100 + storage*10 +
 * storage (kind 1 pack, 2 unpack, 3 convert, 4 axpy to FP64, 5 norm).
 * The paper has no counterpart: this is instrumentation. */
int odwf_profile_enable(odwf_t* h, int enable);
int odwf_profile_read(odwf_t* h, int* keys, int* launches, double* total_ms, int* n_io);

/* Mass-preconditioning term lists for (m, m)/(M, M), M <= 1 (host only, no GPU work):
 *   ODWF_MP_NONE: Eq.(noMP)    2 terms {-, +}            (n_mh = 0)
 *   ODWF_MP_OLD : Eq.(old_MP_N) 2N + 2 terms {-, +, ...}  (N = n_mh heavy masses, Eq.(old_MP) at N = 1)
 *   ODWF_MP_NEW : Eq.(new_MP_N) N + 2 terms               (Eq.(new_MP) at N = 1)
 * mh[] must increase strictly within (m, M). parity = 1 applies the parity operation P (swap the
 * two mass columns of every factor: Eq.(noMP_P) and the parity partners of Section 2), which flips
 * every chirality. Writes at most cap terms to out and the count to *n_out. */
#define ODWF_MP_NONE 0
#define ODWF_MP_OLD  1
#define ODWF_MP_NEW  2
int eofa_mp_terms(int scheme, double m, const double* mh, int n_mh, double M, int parity,
                  eofa_term* out, int cap, int* n_out);

/* k(m_j, m_i) of Eq.(k_ij) (c = 1, lambda = 0) and Omega_pm of Eq.(delta_ij) (host, out[Ns]). */
double eofa_k(double mj, double mi);
int    odwf_omega_vector(const odwf_t* h, int chirality, double* out);

#ifdef __cplusplus
}
#endif
#endif /* ODWF_H */
