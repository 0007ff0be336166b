// Internal declarations of the optimal domain-wall / EOFA library (not part of the ABI).
//
// Internal field layout ("even-odd chunked"): a 5D half-lattice field of one parity holds, for
// every checkerboard site cb (lexicographic index / 2) and slice s, the 12 complex spinor
// components (spin-major, then color). They are stored as 16-byte chunks,
//     chunk(cb, j, s) at ((cb * NCH + j) * Ns + s),
// NCH = 12 (FP64: one complex per chunk), 6 (FP32: two complex per chunk) or 3 (FP16: four
// complex per chunk, plus one float scale per (cb, s)). The Ns slices of one chunk of one site are
// contiguous, so the Ns threads of a site read 16*Ns contiguous bytes per chunk.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "odwf.h"

namespace odwf {

constexpr int kMaxNs = 32;
constexpr int kNumCoef = 14;  // s-matrices per mass pair (see SCoef)

// ---- Krylov solver state in device memory ------------------------------------------------------
enum : int { FLAG_RUN = 0, FLAG_CONVERGED = 1, FLAG_UPDATE = 2, FLAG_BREAKDOWN = 3, FLAG_MAXITER = 4 };

struct CGState {
    double rr;        // |r|^2 of the iterated residual
    double pp;        // |p|^2
    double alpha, beta;
    double tol2;      // stop when rr <= tol2
    double rr_max;    // max rr since the last reliable update
    double delta2;    // request a reliable update when rr < delta2 * rr_max (0: never)
    double result[4]; // reductions of the RESID / NORM epilogues
    int flag;         // FLAG_*; every solver kernel returns at once when flag != 0
    int iter;
    int maxiter;
    unsigned int ticket;
};

// ---- kernel epilogues --------------------------------------------------------------------------
enum : int {
    EPI_STORE = 0,       // out = v
    EPI_STORE_NORM = 1,  // out = v, result[slot] = |v|^2
    EPI_CG_A = 2,        // CGNE: x += alpha own, r -= alpha v, rr = |r|^2 (then beta)
    EPI_CG_B = 3,        // CGNE: p = v + beta p, pp = |p|^2 (then alpha)
    EPI_RESID = 4,       // out = b - v, result[slot] = |out|^2
};

// gamma_5 flags of the generic hopping kernel
enum : int { G5_HOP_IN = 1, G5_OWN_IN = 2, G5_OUT = 4 };

// ---- structured fifth-dimension operators -------------------------------------------------------
// With B = (4 - m0) omega (1 + L) + (1 - L), a cyclic bidiagonal matrix, and W = omega^{1/2}:
//   A      = (4 - m0) + M = (4 - m0 - 1/omega) + 2 W^{-1} (1 + L)^{-1} W^{-1}
//   A^{-1} = W (1 + L) B^{-1} W
// (M = W^{-1} (1 - L)(1 + L)^{-1} W^{-1}). Both apply in O(Ns) per spinor component by one forward
// recurrence in s plus the cyclic corner term. For chirality P_+ the recurrence runs forward in s
// (L_+ is lower bidiagonal with the corner -m1); A_-(m2) = R5 A_+(m2) R5 and A_+(m)^T = A_-(m), so
// P_- components and transposed operators run the same recurrence on the reversed s index. Since
// omega is R5-symmetric, the coefficients below, indexed by the step sigma of the recurrence, are
// the same in both orientations; only the mass terms depend on the chirality.
constexpr int kStructNs = 16;  // Ns of the structured kernels (other Ns use the dense Ns x Ns mixing)
enum : int { SOP_DENSE = 0, SOP_A = 1, SOP_AINV = 2, SOP_T = 4 };
template <typename R>
struct SStructT {
    R w[kStructNs];      // omega^{1/2}
    R rw[kStructNs];     // omega^{1/2} / d,  d = (4 - m0) omega + 1 (diagonal of B)
    R f[kStructNs];      // e / d,  e = (4 - m0) omega - 1 (sub-diagonal of B)
    R q[kStructNs];      // prod_{i = 1..sigma} (-e_i / d_i) (homogeneous solution of B y = 0 rows 1..)
    R wi[kStructNs];     // omega^{-1/2}
    R adiag[kStructNs];  // 4 - m0 - 1/omega
    R wi2s[kStructNs];   // 2 (-1)^sigma omega^{-1/2}
    R m[2];              // mass of chirality P_+ (m1) and P_- (m2)
    R me0[2];            // m e_0
    R cu[2];             // 1 / (d_0 - m e_0 q_{Ns-1})
    R au[2];             // 1 / (1 + m)
};
struct SStruct {
    SStructT<double> d;
    SStructT<float> f;
};

enum StorageKind : int { ST_DOUBLE = 0, ST_FLOAT = 1, ST_HALF = 2 };

// Arguments of the generic 5D hopping kernel (one output parity). Field pointers are to the
// storage type of the instantiation; links/nbr are those of the output parity.
struct HopArgs {
    const void* in;      // hopped field (opposite parity)
    const void* own;     // field at the output sites (same parity), used by OWN kernels
    void* out;
    const void* links;   // [Vh][8][LINK_STRIDE] : 4 forward U_mu(x), 4 backward U_mu(x-mu)^dag
    const int* nbr;      // [Vh][8] checkerboard index of x+mu (0..3), x-mu (4..7)
    const double* mhop;  // 2*Ns*Ns, transposed s-matrices (P_+ then P_-) applied to the hop sum
    const double* mown;  // 2*Ns*Ns, transposed s-matrices applied to the own field
    const float* in_scale;   // FP16 per-(cb,s) scales of `in`, `own`, `out` (else null)
    const float* own_scale;
    float* out_scale;
    void* x;             // CG_A: solution; RESID: b
    void* r;             // CG_A: residual; CG_B: search direction p
    float* x_scale;
    float* r_scale;
    CGState* state;      // may be null for plain applies
    double* partials;    // [gridDim.x] block partial sums
    double c_hop;        // coefficient of the hop sum
    double a_own;        // coefficient of `own` added before the hop-mix (OWN && !MIXOWN)
    int g5;              // G5_* flags
    int Vh, Ns;
    int slot;            // result slot of NORM / RESID
    int parity;          // output parity (bulk-staged kernels derive in-block neighbours from it)
    unsigned int* fault; // set to 1 if a bulk-copy wait ran out of time (never expected)
    long long wait_cycles;  // limit of the bulk-copy wait in SM clock cycles (0: the default, ~1 s)
    int sop;             // SOP_*: structured form of the Mhop / Mown matrix (SOP_DENSE: use the matrix)
    SStruct sc;          // its coefficients (used when sop != SOP_DENSE and Ns == kStructNs)
    const float* links12;  // two-slice kernels: [Vh][8][12] first two rows of each (unsigned) SU(3) link
    const int* nbrs;       // two-slice kernels: nbr with ~index where the link carries the sign -1
};

// ---- host-side handle --------------------------------------------------------------------------
// Launch choice of a fused hop kernel: grid mode (0 one resident wave, 1 one CTA per site group, 2 / 3
// two / four waves), bulk-staged gathers or not, and the tile: spbm x the default sites per CTA.
struct TuneChoice {
    int mode = 0;
    int staged = 0;
    int spbm = 1;
    int dense = 0;  // 1: the dense Ns x Ns fifth-dimension product even where the structured one applies
    int pair = 0;   // two-slices-per-thread kernel (hop_pair.cu) where it applies: 1 register gathers,
                    // 2 / 3 bulk-copy gathers through 2 / 3 shared-memory stages
};

struct SCoef {
    // kNumCoef transposed Ns x Ns matrices, in this order:
    //  0 A_+(m1), 1 A_-(m2), 2 A_+^{-1}, 3 A_-^{-1}, 4 A_+^T, 5 A_-^T, 6 A_+^{-T}, 7 A_-^{-T},
    //  8 N_+ = omega^{1/2}(1 + L_+(m1)), 9 N_-, 10/11 omega^{1/2} (diagonal), 12 N_+^T, 13 N_-^T
    // "transposed" means stored as Mt[s'][s] = M[s][s'] so thread s reads consecutive words.
    double* dev = nullptr;
    SStruct st{};        // structured coefficients of A_pm and A_pm^{-1} (Ns == kStructNs only)
    bool has_st = false;
};

struct Workspace {
    // FP64 half fields
    void* b_e = nullptr; void* b_o = nullptr;   // b' = R5 g5 b by parity
    void* x_e = nullptr; void* x_o = nullptr;
    void* r64 = nullptr; void* t64 = nullptr; void* bh = nullptr;
    // inner-precision half fields (storage of the inner solver)
    void* xi = nullptr; void* ri = nullptr; void* pi = nullptr; void* ti = nullptr;
    float* xi_s = nullptr; float* ri_s = nullptr; float* pi_s = nullptr; float* ti_s = nullptr;
    size_t inner_bytes = 0;
};

}  // namespace odwf

struct odwf_s {
    int L[4] = {0, 0, 0, 0};
    int V = 0, Vh = 0, Ns = 0;
    double m0 = 0;
    std::vector<double> omega;
    std::string err;
    int num_sms = 0;
    // geometry tables, per output parity
    int* nbr[2] = {nullptr, nullptr};
    int* lexof[2] = {nullptr, nullptr};   // lexicographic site of (parity, cb)
    // links, per output parity: FP64 [Vh][8][18], FP32 [Vh][8][20], FP16 [Vh][8][24 halves]
    double* U64[2] = {nullptr, nullptr};
    float* U32[2] = {nullptr, nullptr};
    // two-row links of the two-slice kernels, [Vh][8][12] FP32, and the signed neighbour table
    float* U12[2] = {nullptr, nullptr};
    int* nbrs[2] = {nullptr, nullptr};
    unsigned int* u12_dev = nullptr;       // device: max |row 2 - conj(row 0 x row 1)| over the links (float bits)
    unsigned int* u12_dev_host = nullptr;  // pinned mirror
    bool links12_ok = false;               // the links are SU(3) to FP32 accuracy: two rows determine them
    int pair = -1;                         // two-slice kernels (ODWF_PAIR): -1 the tuned choice, 0 never, 1 / 2 / 3 that
                                           // form wherever it applies
    bool have_gauge = false;
    std::map<std::pair<double, double>, odwf::SCoef> coefs;
    // reductions
    double* partials = nullptr;
    int partials_n = 0;
    odwf::CGState* state = nullptr;        // device
    odwf::CGState* state_host = nullptr;   // pinned mirror
    odwf::Workspace ws;
    // scratch full-lattice FP64 fields for apply / EOFA
    void* f64[4] = {nullptr, nullptr, nullptr, nullptr};
    // 4D scratch
    double* acc4 = nullptr;
    double* lz[3] = {nullptr, nullptr, nullptr};  // Lanczos vectors of eofa_term_spectrum (4D FP64)
    unsigned int* fault = nullptr;        // device word, see HopArgs::fault
    unsigned int* fault_host = nullptr;   // pinned mirror of the fault word
    bool staged_used = false;             // a bulk-staged kernel ran since the fault word was last read
    long long wait_cycles = 0;            // HopArgs::wait_cycles (ODWF_TEST_WAIT_CYCLES, tests only)
    int staged = 0;                       // use the bulk-staged hop kernels where they apply (ODWF_STAGED=1)
    bool dense_s = false;                 // dense Ns x Ns fifth-dimension products everywhere (ODWF_DENSE_S=1)
    // autotuned launch choice per kernel variant (key without the staged flag)
    std::map<int, odwf::TuneChoice> tune;
    // batch-solve pools: per-system workspaces, solver states, reduction buffers, kernel arguments
    std::vector<odwf::Workspace> bws;
    odwf::CGState* bstate = nullptr;
    odwf::CGState* bstate_host = nullptr;
    double* bpartials = nullptr;
    int bcap = 0;
    odwf::HopArgs* bargs = nullptr;
    int bargs_cap = 0;
    cudaStream_t cap_stream = nullptr;   // non-default stream used only to capture CUDA graphs
    // network whose preconditioned CGNE replaces plain CGNE in the single-system solves of the EOFA
    // term calls (odwf_set_preconditioner); not owned
    struct odwf_net_s* net = nullptr;
    // flexible-GCR basis and work fields, kept between calls; released by gcr_free at destroy
    void* gcr = nullptr;
    void (*gcr_free)(void*) = nullptr;
    // kernel timing (odwf_profile_*)
    bool prof = false;
    struct ProfRec { int key; cudaEvent_t a, b; };
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
};

struct odwf_net_s;

namespace odwf {

// sizes
inline size_t half_elems_bytes(const odwf_s* h, int st) {
    size_t n = (size_t)h->Vh * h->Ns;
    switch (st) {
        case ST_DOUBLE: return n * 24 * sizeof(double);
        case ST_FLOAT: return n * 24 * sizeof(float);
        default: return n * 24 * sizeof(__half);
    }
}

int set_err(odwf_s* h, int code, const std::string& msg);
// After work that may have run bulk-staged kernels: synchronise `st`, read and clear the fault word,
// and return ODWF_EFAULT if a bounded wait ran out (ODWF_OK otherwise, at once if no staged kernel ran).
int check_fault(odwf_s* h, cudaStream_t st);
int ensure_ws(odwf_s* h, Workspace& w, int inner);
int ensure_workspace(odwf_s* h, int inner);
int cuda_check(odwf_s* h, cudaError_t e, const char* what);
const SCoef* get_coef(odwf_s* h, double m1, double m2);
bool coef_host(const odwf_s* h, double m1, double m2, std::vector<double>& host, std::string& err);
// structured coefficients of the mass pair (false if Ns != kStructNs)
bool struct_host(const odwf_s* h, double m1, double m2, SStruct* out);
// the kernel arguments' structured operator: A (SOP_A) or A^{-1} (SOP_AINV), optionally transposed
void set_sop(HopArgs& a, const SCoef* c, int sop);
// FP16 storage passes the per-(cb, s) scales of the three fields (ignored for FP64 / FP32)
int apply_dt_parity(odwf_s* h, int stg, const SCoef* c, bool dag, int parity, const void* in_other,
                    const void* own, void* out, cudaStream_t st, const float* in_scale = nullptr,
                    const float* own_scale = nullptr, float* out_scale = nullptr);

// launch helpers (kernels.cu)
// Generic hop: out_p = epi( [MIXOWN ? Mown own : 0] + Mhop?( c_hop H in + a_own own ) )
int launch_hop(odwf_s* h, int storage, int parity, bool mixhop, bool own, bool mixown, int epi,
               HopArgs a, cudaStream_t st);
int launch_smix(odwf_s* h, int storage, const void* in, void* out, const double* mt, double scale,
                cudaStream_t st, const float* in_scale = nullptr, float* out_scale = nullptr,
                const SCoef* c = nullptr, int sop = SOP_DENSE);
int launch_pack5(odwf_s* h, const double* lex5, void* e, void* o, int storage, int r5g5, cudaStream_t st,
                 float* e_scale = nullptr, float* o_scale = nullptr);
int launch_unpack5(odwf_s* h, const void* e, const void* o, double* lex5, int storage, int r5g5,
                   cudaStream_t st, const float* e_scale = nullptr, const float* o_scale = nullptr);
int launch_convert(odwf_s* h, const void* in, int st_in, const float* in_scale, void* out, int st_out,
                   float* out_scale, cudaStream_t st);
int launch_axpy_to64(odwf_s* h, double a, const void* xin, int st_in, const float* xin_scale, double* y,
                     cudaStream_t st);
int launch_norm2(odwf_s* h, const void* v, int storage, const float* scale, int slot, cudaStream_t st,
                 CGState* state = nullptr, double* partials = nullptr);
void hop_fill(odwf_s* h, int storage, int parity, HopArgs& a, bool reduces);
int launch_hop_own_cgb(odwf_s* h, int storage, HopArgs a, cudaStream_t st);
// several systems (blockIdx.y), one launch; structured: every system's arguments carry the structured
// fifth-dimension products (set_sop with coefficients that have them) and Ns = kStructNs
int launch_hop_multi(odwf_s* h, int storage, bool mixhop, bool own, bool mixown, int epi, const HopArgs* dev_args,
                     int n, int max_vh, cudaStream_t st, bool structured = false);
int launch_gauge(odwf_s* h, const double* U, cudaStream_t st);
// grid of a fused kernel for grid mode `mode` (0 one resident wave, 1 one CTA per site group, 2 / 3
// two / four waves), occupancy occ CTAs per SM, `groups` site groups
int grid_for_mode(const odwf_s* h, int mode, int occ, int groups, bool reduces);
// two-slices-per-thread hop kernels (hop_pair.cu): whether a variant has one, and its launch (a filled
// by hop_fill; spbm the tile multiplier of 16 sites per CTA); key = the profiling key of the launch
bool pair_variant(int storage, bool mixhop, bool own, bool mixown, int epi);
bool pair_applies(const odwf_s* h, int storage, const HopArgs& a);
// form 1: neighbours gathered into registers; 2 / 3: gathered by bulk copies through 2 / 3 shared-memory
// stages (FP32 storage with 16-byte aligned fields, else form 1)
int launch_hop_pair(odwf_s* h, int storage, bool mixhop, bool own, bool mixown, int epi, const HopArgs& a,
                    int mode, int spbm, cudaStream_t st, int form = 1);
bool pair_tma_applies(int storage, const HopArgs& a);
int launch_init_state(odwf_s* h, cudaStream_t st);
void prof_begin(odwf_s* h, int key, cudaStream_t st, cudaEvent_t* a);
void prof_end(odwf_s* h, int key, cudaStream_t st, cudaEvent_t a);

// network-preconditioned CGNE (learned.cu): b / x are ABI fields, or null for b' packed in ws.b_e / b_o
// and x left in ws.x_e / x_o
int learned_solve(odwf_s* h, odwf_net_s* n, double m1, double m2, const void* b, void* x,
                  const odwf_solve_opts* opts, odwf_solve_stats* stats, cudaStream_t st);

// field helpers for EOFA (eofa.cu)
// F (accumulate = 0) or F += coef F_term (accumulate = 1), F^a_mu(x) = -dS/dw^a of one EOFA term
int term_force(odwf_s* h, const eofa_term* t, const void* phi, double* F, double coef, int accumulate,
               const odwf_solve_opts* opts, odwf_solve_stats* stats, cudaStream_t st);
}  // namespace odwf
