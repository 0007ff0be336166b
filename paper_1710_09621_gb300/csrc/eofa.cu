// EOFA pseudofermion terms on the GPU: action, force and heat-bath.
//
// A term (Eq.(m1m2_m1m4) / Eq.(m1m2_m3m2)) has the 4D operator
//   chirality -1:  X = P_- [1 - k Omega_-^T H_T(m3, m4)^{-1} Omega_-] P_-,  k = k(m_den, m4)
//   chirality +1:  X = P_+ [1 + k Omega_+^T H_T(m3, m4)^{-1} Omega_+] P_+,  k = k(m_den, m3)
// with k(m_j, m_i) = 2 (m_j - m_i) / ((1 + m_j)(1 + m_i)) (Eq.(k_ij) at c = 1, lambda = 0) and
// (Omega_-)_s = (-1)^s omega_s^{-1/2}, (Omega_+)_s = (-1)^(Ns-1-s) omega_s^{-1/2} (Eq.(delta_ij)).
// Every call needs chi = H_T(m3, m4)^{-1} Omega P phi, i.e. D_T chi = R5 g5 Omega P phi.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "field_access.cuh"

namespace odwf {

int ensure_workspace(odwf_s* h, int inner);
int solve_core(odwf_s* h, double m1, double m2, const odwf_solve_opts* opts, odwf_solve_stats* stats,
               cudaStream_t st);
int solve_shared_rhs(odwf_s* h, int n, const double* m12, const void* be, const void* bo, const odwf_solve_opts* opts,
                     odwf_solve_stats* stats, std::vector<Workspace*>& ws_out, cudaStream_t st);

struct SWeights {
    double w[kMaxNs];
};

// b'(x, s) = R5 g5 (Omega P phi)(x, s) = c * Omega_{Ns-1-s} (P_c phi)(x)  into FP64 internal e/o fields
__global__ void k_embed(const double2* __restrict__ phi, double* e, double* o, const int* __restrict__ lex_e,
                        const int* __restrict__ lex_o, int Vh, int Ns, int chir, SWeights coef) {
    const size_t total = (size_t)2 * Vh * Ns;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % Ns);
        const size_t rest = i / Ns;
        const int cb = (int)(rest % Vh);
        const int par = (int)(rest / Vh);
        const int lex = par ? lex_o[cb] : lex_e[cb];
        const double cf = coef.w[s];
        double v[24];
        for (int k = 0; k < 12; ++k) {
            const bool keep = (chir > 0) ? (k < 6) : (k >= 6);
            const double2 z = phi[(size_t)lex * 12 + k];
            v[2 * k] = keep ? cf * z.x : 0.0;
            v[2 * k + 1] = keep ? cf * z.y : 0.0;
        }
        Store<ST_DOUBLE>::store(par ? o : e, nullptr, cb, s, Ns, v);
    }
}

// acc(x) = P_c sum_s w_s chi(x, s);  out4(x) += acc(x) (if out4);
// result[slot] = Re sum_x phi(x)^dag acc(x) (if phi), result[slot+1] = |P_c phi|^2 (if phi)
__global__ void k_contract(const double* e, const double* o, const int* __restrict__ lex_e,
                           const int* __restrict__ lex_o, int Vh, int Ns, int chir, SWeights w,
                           const double2* __restrict__ phi, double2* out4, CGState* state, double* partials,
                           int slot) {
    __shared__ double wsum[32];
    __shared__ int is_last;
    double dot = 0.0, nrm = 0.0;
    const int total = 2 * Vh;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int cb = i % Vh;
        const int par = i / Vh;
        const int lex = par ? lex_o[cb] : lex_e[cb];
        double acc[24];
        for (int k = 0; k < 24; ++k) acc[k] = 0.0;
        for (int s = 0; s < Ns; ++s) {
            double v[24];
            Store<ST_DOUBLE>::load(par ? o : e, nullptr, cb, s, Ns, v);
            for (int k = 0; k < 24; ++k) acc[k] = fma(w.w[s], v[k], acc[k]);
        }
        const int k0 = chir > 0 ? 0 : 12;
        for (int k = 0; k < 24; ++k)
            if (k < k0 || k >= k0 + 12) acc[k] = 0.0;
        if (phi) {
            for (int k = 0; k < 12; ++k) {
                const bool keep = (chir > 0) ? (k < 6) : (k >= 6);
                if (!keep) continue;
                const double2 z = phi[(size_t)lex * 12 + k];
                dot += z.x * acc[2 * k] + z.y * acc[2 * k + 1];
                nrm += z.x * z.x + z.y * z.y;
            }
        }
        if (out4) {
            for (int k = 0; k < 12; ++k) {
                double2 z = out4[(size_t)lex * 12 + k];
                z.x += acc[2 * k];
                z.y += acc[2 * k + 1];
                out4[(size_t)lex * 12 + k] = z;
            }
        }
    }
    if (!phi) return;
    // two deterministic grid reductions (dot, norm) through the shared state
    for (int which = 0; which < 2; ++which) {
        double v = which == 0 ? dot : nrm;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        __syncthreads();
        if (lane == 0) wsum[warp] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) b += wsum[q];
            partials[which * gridDim.x + blockIdx.x] = b;
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&state->ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < (int)gridDim.x; ++q) {
            a += ((volatile double*)partials)[q];
            b += ((volatile double*)partials)[gridDim.x + q];
        }
        state->result[slot] = a;
        state->result[slot + 1] = b;
        state->ticket = 0;
    }
}

// Force: for each link (x, mu) of output parity p, with chi the 5D solution and psi = g5 R5 chi,
//   Z = sum_s sum_spin [ (U chi(x+mu,s)) (x) conj((1 - g_mu) psi(x,s)) - chi(x,s) (x) conj(U (1 + g_mu) psi(x+mu,s)) ]
//   F^a_mu(x) = -(sgnk / 4) Im tr(lambda^a Z),  sgnk = +k (chirality -1), -k (chirality +1).
// U is the stored forward link (antiperiodic sign folded in, which multiplies both terms alike).
template <int MU>
__device__ void gamma_mul(const double* p, double* o) {
    // o = gamma_mu p in the chiral basis: upper = B p_dn, lower = C p_up
    for (int c = 0; c < 3; ++c) {
        const double *u0 = p + (0 * 3 + c) * 2, *u1 = p + (1 * 3 + c) * 2;
        const double *d0 = p + (2 * 3 + c) * 2, *d1 = p + (3 * 3 + c) * 2;
        double *o0 = o + (0 * 3 + c) * 2, *o1 = o + (1 * 3 + c) * 2;
        double *o2 = o + (2 * 3 + c) * 2, *o3 = o + (3 * 3 + c) * 2;
        if (MU == 0) {  // B = -i s1, C = i s1
            o0[0] = d1[1]; o0[1] = -d1[0];  // -i d1
            o1[0] = d0[1]; o1[1] = -d0[0];  // -i d0
            o2[0] = -u1[1]; o2[1] = u1[0];  // i u1
            o3[0] = -u0[1]; o3[1] = u0[0];  // i u0
        } else if (MU == 1) {  // B = [[0,-1],[1,0]], C = [[0,1],[-1,0]]
            o0[0] = -d1[0]; o0[1] = -d1[1];
            o1[0] = d0[0]; o1[1] = d0[1];
            o2[0] = u1[0]; o2[1] = u1[1];
            o3[0] = -u0[0]; o3[1] = -u0[1];
        } else if (MU == 2) {  // B = diag(-i, i), C = diag(i, -i)
            o0[0] = d0[1]; o0[1] = -d0[0];
            o1[0] = -d1[1]; o1[1] = d1[0];
            o2[0] = -u0[1]; o2[1] = u0[0];
            o3[0] = u1[1]; o3[1] = -u1[0];
        } else {
            o0[0] = d0[0]; o0[1] = d0[1];
            o1[0] = d1[0]; o1[1] = d1[1];
            o2[0] = u0[0]; o2[1] = u0[1];
            o3[0] = u1[0]; o3[1] = u1[1];
        }
    }
}

__device__ void su3_mul4(const double* u, const double* v, double* w) {
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) {
            double re = 0, im = 0;
            for (int j = 0; j < 3; ++j) {
                const double ur = u[(i * 3 + j) * 2], ui = u[(i * 3 + j) * 2 + 1];
                const double vr = v[(a * 3 + j) * 2], vi = v[(a * 3 + j) * 2 + 1];
                re += ur * vr - ui * vi;
                im += ur * vi + ui * vr;
            }
            w[(a * 3 + i) * 2] = re;
            w[(a * 3 + i) * 2 + 1] = im;
        }
}

template <int MU>
__device__ void force_link(const double* chi_self, const double* chi_nb, const int* nbr, const double* links,
                           const int* lexof, int par, int cb, int Ns, double sgnk, double* F, int V, double coef,
                           int accumulate) {
    const int n = nbr[(size_t)cb * 8 + MU];
    double u[18];
    {
        const double* lp = links + ((size_t)cb * 8 + MU) * 18;
        for (int k = 0; k < 18; ++k) u[k] = lp[k];
    }
    double Zr[9], Zi[9];
    for (int k = 0; k < 9; ++k) Zr[k] = Zi[k] = 0.0;
    for (int s = 0; s < Ns; ++s) {
        double cx[24], cn[24], px[24], pn[24], t[24], a[24], b[24];
        Store<ST_DOUBLE>::load(chi_self, nullptr, cb, s, Ns, cx);
        Store<ST_DOUBLE>::load(chi_nb, nullptr, n, s, Ns, cn);
        Store<ST_DOUBLE>::load(chi_self, nullptr, cb, Ns - 1 - s, Ns, px);
        Store<ST_DOUBLE>::load(chi_nb, nullptr, n, Ns - 1 - s, Ns, pn);
        for (int k = 12; k < 24; ++k) {  // psi = g5 R5 chi
            px[k] = -px[k];
            pn[k] = -pn[k];
        }
        // term 1: A1 = U chi(x+mu), B1 = (1 - g_mu) psi(x)
        su3_mul4(u, cn, a);
        gamma_mul<MU>(px, t);
        for (int k = 0; k < 24; ++k) b[k] = px[k] - t[k];
        for (int al = 0; al < 4; ++al)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    const double ar = a[(al * 3 + i) * 2], ai = a[(al * 3 + i) * 2 + 1];
                    const double br = b[(al * 3 + j) * 2], bi = b[(al * 3 + j) * 2 + 1];
                    Zr[i * 3 + j] += ar * br + ai * bi;  // a * conj(b)
                    Zi[i * 3 + j] += ai * br - ar * bi;
                }
        // term 2: A2 = chi(x), B2 = U (1 + g_mu) psi(x+mu)
        gamma_mul<MU>(pn, t);
        for (int k = 0; k < 24; ++k) t[k] = pn[k] + t[k];
        su3_mul4(u, t, b);
        for (int al = 0; al < 4; ++al)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    const double ar = cx[(al * 3 + i) * 2], ai = cx[(al * 3 + i) * 2 + 1];
                    const double br = b[(al * 3 + j) * 2], bi = b[(al * 3 + j) * 2 + 1];
                    Zr[i * 3 + j] -= ar * br + ai * bi;
                    Zi[i * 3 + j] -= ai * br - ar * bi;
                }
    }
    // Im tr(lambda^a Z) = Im sum_{c,b} lambda^a_{cb} Z_{bc}
    auto zr = [&](int i, int j) { return Zr[i * 3 + j]; };
    auto zi = [&](int i, int j) { return Zi[i * 3 + j]; };
    double im[8];
    im[0] = zi(1, 0) + zi(0, 1);                          // lambda1: Z10 + Z01
    im[1] = -zr(1, 0) + zr(0, 1);                         // lambda2: -i Z10 + i Z01
    im[2] = zi(0, 0) - zi(1, 1);                          // lambda3
    im[3] = zi(2, 0) + zi(0, 2);                          // lambda4
    im[4] = -zr(2, 0) + zr(0, 2);                         // lambda5
    im[5] = zi(2, 1) + zi(1, 2);                          // lambda6
    im[6] = -zr(2, 1) + zr(1, 2);                         // lambda7
    im[7] = (zi(0, 0) + zi(1, 1) - 2.0 * zi(2, 2)) / sqrt(3.0);  // lambda8
    const int lex = lexof[cb];
    double* out = F + ((size_t)MU * V + lex) * 8;
    for (int a8 = 0; a8 < 8; ++a8) {
        const double f = -0.25 * sgnk * im[a8];
        out[a8] = accumulate ? fma(coef, f, out[a8]) : f;
    }
}

// F^a_mu(x) written (accumulate = 0) or added as F += coef * F^a_mu(x) (accumulate = 1: a momentum update)
__global__ void k_force(const double* e, const double* o, const int* nbr_e, const int* nbr_o, const double* lk_e,
                        const double* lk_o, const int* lex_e, const int* lex_o, int Vh, int Ns, double sgnk,
                        double* F, double coef, int accumulate) {
    const int total = 2 * Vh * 4;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int mu = i % 4;
        const int rest = i / 4;
        const int cb = rest % Vh;
        const int par = rest / Vh;
        const double* self = par ? o : e;
        const double* nb = par ? e : o;
        const int* nbr = par ? nbr_o : nbr_e;
        const double* lk = par ? lk_o : lk_e;
        const int* lx = par ? lex_o : lex_e;
        switch (mu) {
            case 0: force_link<0>(self, nb, nbr, lk, lx, par, cb, Ns, sgnk, F, 2 * Vh, coef, accumulate); break;
            case 1: force_link<1>(self, nb, nbr, lk, lx, par, cb, Ns, sgnk, F, 2 * Vh, coef, accumulate); break;
            case 2: force_link<2>(self, nb, nbr, lk, lx, par, cb, Ns, sgnk, F, 2 * Vh, coef, accumulate); break;
            default: force_link<3>(self, nb, nbr, lk, lx, par, cb, Ns, sgnk, F, 2 * Vh, coef, accumulate); break;
        }
    }
}

__global__ void k_scale4(const double2* in, double2* out, int V, int chir, double c) {
    const int total = V * 12;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int k = i % 12;
        const bool keep = (chir > 0) ? (k < 6) : (k >= 6);
        const double2 z = in[i];
        out[i] = keep ? make_double2(c * z.x, c * z.y) : make_double2(0.0, 0.0);
    }
}

// ---- 4D FP64 vector algebra of the Lanczos estimate (n doubles) -----------------------------------
// out = ca A + cb B + cc C (any of B, C may be null)
__global__ void k_lincomb4(double* out, double ca, const double* A, double cb, const double* B, double cc,
                           const double* C, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double v = ca * A[i];
        if (B) v = fma(cb, B[i], v);
        if (C) v = fma(cc, C[i], v);
        out[i] = v;
    }
}

// per-block partial sums of sum_i A[i] B[i] (the real part of <A, B> for interleaved complex data)
__global__ void k_dot4(const double* A, const double* B, size_t n, double* partials) {
    __shared__ double wsum[32];
    double v = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        v = fma(A[i], B[i], v);
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) b += wsum[q];
        partials[blockIdx.x] = b;
    }
}

// ---- host helpers ------------------------------------------------------------------------------
static int grid_for(odwf_s* h, size_t n, int block) {
    size_t g = (n + block - 1) / block;
    const size_t cap = (size_t)h->num_sms * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

static int check_term(odwf_s* h, const eofa_term* t) {
    if (!t) return set_err(h, ODWF_EINVAL, "null term");
    if (t->chirality != 1 && t->chirality != -1) return set_err(h, ODWF_EINVAL, "term chirality must be +1 or -1");
    const double ms[3] = {t->m3, t->m4, t->m_den};
    for (double m : ms)
        if (!(m > 0.0 && m <= 1.0)) return set_err(h, ODWF_EINVAL, "term masses must lie in (0, 1]");
    if ((t->chirality < 0 && t->m_den == t->m4) || (t->chirality > 0 && t->m_den == t->m3))
        return set_err(h, ODWF_EINVAL, "term with k = 0 (m_den equals the reference mass)");
    return ODWF_OK;
}

static double term_k(const eofa_term* t) {
    return t->chirality < 0 ? eofa_k(t->m_den, t->m4) : eofa_k(t->m_den, t->m3);
}

static void omega_vec(const odwf_s* h, int chir, double* out) { odwf_omega_vector(h, chir, out); }

// pack b' = R5 g5 Omega P phi into ws.b_e / ws.b_o
static int embed(odwf_s* h, const eofa_term* t, const void* phi, cudaStream_t st) {
    double om[kMaxNs];
    omega_vec(h, t->chirality, om);
    SWeights c{};
    for (int s = 0; s < h->Ns; ++s) c.w[s] = t->chirality * om[h->Ns - 1 - s];
    const size_t n = (size_t)2 * h->Vh * h->Ns;
    k_embed<<<grid_for(h, n, 256), 256, 0, st>>>((const double2*)phi, (double*)h->ws.b_e, (double*)h->ws.b_o,
                                                   h->lexof[0], h->lexof[1], h->Vh, h->Ns, t->chirality, c);
    return cuda_check(h, cudaGetLastError(), "k_embed");
}

static int contract(odwf_s* h, int chir, const double* w, const void* phi, void* out4, int slot, cudaStream_t st,
                    const Workspace* ws = nullptr) {
    if (!ws) ws = &h->ws;
    SWeights c{};
    for (int s = 0; s < h->Ns; ++s) c.w[s] = w[s];
    int g = grid_for(h, (size_t)2 * h->Vh, 256);
    if (2 * g > h->partials_n) g = h->partials_n / 2;
    k_contract<<<g, 256, 0, st>>>((const double*)ws->x_e, (const double*)ws->x_o, h->lexof[0], h->lexof[1], h->Vh,
                                  h->Ns, chir, c, (const double2*)phi, (double2*)out4, h->state, h->partials, slot);
    return cuda_check(h, cudaGetLastError(), "k_contract");
}

// chi = H_T(m1, m2)^{-1} Omega P phi into ws.x_e / ws.x_o: plain mixed-precision CGNE, or, with a
// network attached to the handle (odwf_set_preconditioner), CGNE on S M
static int term_solve(odwf_s* h, const eofa_term* t, double m1, double m2, const void* phi,
                      const odwf_solve_opts* opts, odwf_solve_stats* stats, cudaStream_t st) {
    int rc = ensure_workspace(h, ST_DOUBLE);
    if (rc) return rc;
    if ((rc = embed(h, t, phi, st))) return rc;
    if (h->net) return learned_solve(h, h->net, m1, m2, nullptr, nullptr, opts, stats, st);
    return solve_core(h, m1, m2, opts, stats, st);
}

// ---- Zolotarev rational approximation of x^{-1/2} on [x_lo, x_hi] (host, FP64) ------------------
// sn, cn of modulus k by the arithmetic-geometric mean (Abramowitz & Stegun 16.4); kc = sqrt(1 - k^2).
static void sncn_agm(double u, double k, double kc, double& sn, double& cn, double& K) {
    double a[64], c[64];
    double an = 1.0, bn = kc;
    a[0] = 1.0;
    c[0] = k;
    int N = 0;
    while (std::fabs(c[N]) > 1e-17 && N < 60) {
        const double a1 = 0.5 * (an + bn), b1 = std::sqrt(an * bn), c1 = 0.5 * (an - bn);
        ++N;
        a[N] = a1;
        c[N] = c1;
        an = a1;
        bn = b1;
    }
    K = M_PI / (2.0 * a[N]);
    double phi = std::ldexp(a[N] * u, N);
    for (int n = N; n > 0; --n) phi = 0.5 * (phi + std::asin(c[n] * std::sin(phi) / a[n]));
    sn = std::sin(phi);
    cn = std::cos(phi);
}

struct Rational {
    double a0;
    std::vector<double> a, b;
    double err;
};

static Rational zolotarev_inv_sqrt(int n, double x_lo, double x_hi) {
    const double bb = x_hi / x_lo;
    const int N = 2 * n + 1;
    const double k = std::sqrt(1.0 - 1.0 / bb), kc = 1.0 / std::sqrt(bb);
    double sn, cn, K;
    sncn_agm(0.0, k, kc, sn, cn, K);
    std::vector<double> cnum, cden;
    for (int l = 1; l < N; ++l) {
        sncn_agm(l * K / N, k, kc, sn, cn, K);
        const double cl = (sn * sn) / (cn * cn);
        if (l % 2) cden.push_back(cl);
        else cnum.push_back(cl);
    }
    auto unscaled = [&](double y) {
        double r = 1.0;
        for (int i = 0; i < n; ++i) r *= (y + cnum[i]) / (y + cden[i]);
        return r;
    };
    const int G = 20000;
    double fmax = -1e300, fmin = 1e300;
    for (int i = 0; i <= G; ++i) {
        const double y = std::exp(std::log(bb) * i / G);
        const double f = std::sqrt(y) * unscaled(y);
        fmax = std::max(fmax, f);
        fmin = std::min(fmin, f);
    }
    const double d = 2.0 / (fmax + fmin);
    Rational r;
    r.a0 = d / std::sqrt(x_lo);
    for (int j = 0; j < n; ++j) {
        const double y0 = -cden[j];
        double num = 1.0, den = 1.0;
        for (int i = 0; i < n; ++i) num *= (y0 + cnum[i]);
        for (int i = 0; i < n; ++i)
            if (i != j) den *= (y0 + cden[i]);
        r.a.push_back(d * num / den * std::sqrt(x_lo));
        r.b.push_back(cden[j] * x_lo);
    }
    double err = 0.0;
    for (int i = 0; i <= G; ++i) {
        const double x = x_lo * std::exp(std::log(bb) * i / G);
        double v = r.a0;
        for (int j = 0; j < n; ++j) v += r.a[j] / (x + r.b[j]);
        err = std::max(err, std::fabs(1.0 - std::sqrt(x) * v));
    }
    r.err = err;
    return r;
}

static int ensure_acc4(odwf_s* h) {
    if (h->acc4) return ODWF_OK;
    if (cudaMalloc((void**)&h->acc4, sizeof(double) * 24 * (size_t)h->V) != cudaSuccess)
        return set_err(h, ODWF_ENOMEM, "cudaMalloc acc4");
    return ODWF_OK;
}

// X v = P v -/+ k P Omega^T H_T(m3, m4)^{-1} Omega P v (chirality -1 / +1) for a 4D FP64 field
static int term_apply(odwf_s* h, const eofa_term* t, const double* v, double* out, const odwf_solve_opts* opts,
                      int* iters, cudaStream_t st) {
    odwf_solve_stats ss{};
    int rc = term_solve(h, t, t->m3, t->m4, v, opts, &ss, st);
    if (rc != ODWF_OK) return rc;
    *iters += ss.iters;
    k_scale4<<<grid_for(h, (size_t)h->V * 12, 256), 256, 0, st>>>((const double2*)v, (double2*)out, h->V,
                                                                    t->chirality, 1.0);
    if ((rc = cuda_check(h, cudaGetLastError(), "k_scale4"))) return rc;
    double om[kMaxNs], w[kMaxNs];
    omega_vec(h, t->chirality, om);
    const double sgn = t->chirality < 0 ? -1.0 : 1.0;
    for (int q = 0; q < h->Ns; ++q) w[q] = sgn * term_k(t) * om[q];
    return contract(h, t->chirality, w, nullptr, out, 0, st);
}

// Re <A, B> of two 4D FP64 fields (n doubles), summed on the host in block order (deterministic)
static int dot4(odwf_s* h, const double* A, const double* B, size_t n, double* out, cudaStream_t st) {
    int g = grid_for(h, n, 256);
    if (g > h->partials_n) g = h->partials_n;
    k_dot4<<<g, 256, 0, st>>>(A, B, n, h->partials);
    int rc = cuda_check(h, cudaGetLastError(), "k_dot4");
    if (rc) return rc;
    std::vector<double> part(g);
    if ((rc = cuda_check(h, cudaMemcpyAsync(part.data(), h->partials, sizeof(double) * g, cudaMemcpyDeviceToHost, st),
                         "dot D2H")))
        return rc;
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "sync"))) return rc;
    double sum = 0.0;
    for (double p : part) sum += p;
    *out = sum;
    return ODWF_OK;
}

static int lincomb4(odwf_s* h, double* out, double ca, const double* A, double cb, const double* B, double cc,
                    const double* C, size_t n, cudaStream_t st) {
    k_lincomb4<<<grid_for(h, n, 256), 256, 0, st>>>(out, ca, A, cb, B, cc, C, n);
    return cuda_check(h, cudaGetLastError(), "k_lincomb4");
}

// Smallest or largest eigenvalue of the symmetric tridiagonal matrix (diagonal a[0..n-1], off-diagonal
// b[1..n-1]) by bisection on the Sturm sequence count (the number of eigenvalues below x).
static double tridiag_extreme(const std::vector<double>& a, const std::vector<double>& b, bool largest) {
    const int n = (int)a.size();
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {  // Gershgorin interval
        const double r = (i > 0 ? std::fabs(b[i]) : 0.0) + (i + 1 < n ? std::fabs(b[i + 1]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    auto count_below = [&](double x) {
        int c = 0;
        double d = 1.0;
        for (int i = 0; i < n; ++i) {
            d = a[i] - x - (i > 0 ? b[i] * b[i] / d : 0.0);
            if (d == 0.0) d = -1e-300;
            if (d < 0.0) ++c;
        }
        return c;
    };
    const int target = largest ? n - 1 : 0;  // find x with count_below(x) == target .. target + 1
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (count_below(mid) > target) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// n_iter steps of Lanczos on X from P v0 (FP64, the last two directions re-orthogonalised once more
// each step); writes the extreme Ritz values.
static int term_spectrum(odwf_s* h, const eofa_term* t, const void* v0, int n_iter, double* lo, double* hi,
                         const odwf_solve_opts* opts, int* iters, cudaStream_t st) {
    const size_t n = (size_t)h->V * 24;
    int rc = ensure_acc4(h);
    if (rc) return rc;
    for (int i = 0; i < 3 && !rc; ++i)
        if (!h->lz[i] && cudaMalloc((void**)&h->lz[i], sizeof(double) * n) != cudaSuccess)
            rc = set_err(h, ODWF_ENOMEM, "cudaMalloc Lanczos vectors");
    if (rc) return rc;
    double *vp = h->lz[0], *v = h->lz[1], *w = h->lz[2];
    k_scale4<<<grid_for(h, (size_t)h->V * 12, 256), 256, 0, st>>>((const double2*)v0, (double2*)v, h->V,
                                                                    t->chirality, 1.0);
    if ((rc = cuda_check(h, cudaGetLastError(), "k_scale4"))) return rc;
    double nrm2 = 0.0;
    if ((rc = dot4(h, v, v, n, &nrm2, st))) return rc;
    if (!(nrm2 > 0.0) || !std::isfinite(nrm2)) return set_err(h, ODWF_EINVAL, "Lanczos start vector is zero on the term's chirality");
    if ((rc = lincomb4(h, v, 1.0 / std::sqrt(nrm2), v, 0.0, nullptr, 0.0, nullptr, n, st))) return rc;
    if ((rc = cuda_check(h, cudaMemsetAsync(vp, 0, sizeof(double) * n, st), "memset"))) return rc;
    std::vector<double> al, be(1, 0.0);
    for (int j = 0; j < n_iter; ++j) {
        if ((rc = term_apply(h, t, v, w, opts, iters, st))) return rc;
        double a = 0.0;
        if ((rc = dot4(h, v, w, n, &a, st))) return rc;
        // w -= a v + b_j v_prev, then once more against v and v_prev (local re-orthogonalisation)
        if ((rc = lincomb4(h, w, 1.0, w, -a, v, -be[j], vp, n, st))) return rc;
        double c1 = 0.0, c2 = 0.0;
        if ((rc = dot4(h, v, w, n, &c1, st)) || (rc = dot4(h, vp, w, n, &c2, st))) return rc;
        if ((rc = lincomb4(h, w, 1.0, w, -c1, v, -c2, vp, n, st))) return rc;
        al.push_back(a + c1);
        double b2 = 0.0;
        if ((rc = dot4(h, w, w, n, &b2, st))) return rc;
        const double b = std::sqrt(std::max(b2, 0.0));
        if (j + 1 == n_iter || !(b > 1e-12 * std::fabs(a))) break;  // invariant subspace found
        be.push_back(b);
        // v_prev <- v, v <- w / b
        std::swap(vp, v);
        if ((rc = lincomb4(h, v, 1.0 / b, w, 0.0, nullptr, 0.0, nullptr, n, st))) return rc;
    }
    be.resize(al.size());
    *lo = tridiag_extreme(al, be, false);
    *hi = tridiag_extreme(al, be, true);
    return ODWF_OK;
}

}  // namespace odwf

using namespace odwf;

extern "C" int eofa_action(odwf_t* h, const eofa_term* t, const void* phi, double* S_host,
                           const odwf_solve_opts* opts, odwf_solve_stats* stats, void* stream) {
    if (!h || !phi || !S_host) return set_err(h, ODWF_EINVAL, "null argument");
    if (!h->have_gauge) return set_err(h, ODWF_EINVAL, "odwf_set_gauge has not been called");
    int rc = check_term(h, t);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int src = term_solve(h, t, t->m3, t->m4, phi, opts, stats, st);
    if (src != ODWF_OK && src != ODWF_ENOCONV) return src;
    double om[kMaxNs];
    omega_vec(h, t->chirality, om);
    if ((rc = contract(h, t->chirality, om, phi, nullptr, 0, st))) return rc;
    CGState hs;
    if ((rc = cuda_check(h, cudaMemcpyAsync(h->state_host, h->state, sizeof(CGState), cudaMemcpyDeviceToHost, st), "D2H")))
        return rc;
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "sync"))) return rc;
    hs = *h->state_host;
    const double sgn = t->chirality < 0 ? -1.0 : 1.0;
    *S_host = hs.result[1] + sgn * term_k(t) * hs.result[0];
    return src;
}

namespace odwf {
// F (accumulate = 0) or F += coef * F_term (accumulate = 1) for one term; one H_T(m3, m4) solve
int term_force(odwf_s* h, const eofa_term* t, const void* phi, double* F, double coef, int accumulate,
               const odwf_solve_opts* opts, odwf_solve_stats* stats, cudaStream_t st) {
    int rc = check_term(h, t);
    if (rc) return rc;
    const int src = term_solve(h, t, t->m3, t->m4, phi, opts, stats, st);
    if (src != ODWF_OK && src != ODWF_ENOCONV) return src;
    const double sgnk = (t->chirality < 0 ? 1.0 : -1.0) * term_k(t);
    const int total = 2 * h->Vh * 4;
    k_force<<<grid_for(h, total, 128), 128, 0, st>>>((const double*)h->ws.x_e, (const double*)h->ws.x_o, h->nbr[0],
                                                     h->nbr[1], h->U64[0], h->U64[1], h->lexof[0], h->lexof[1], h->Vh,
                                                     h->Ns, sgnk, F, coef, accumulate);
    if ((rc = cuda_check(h, cudaGetLastError(), "k_force"))) return rc;
    return src;
}
}  // namespace odwf

extern "C" int eofa_force(odwf_t* h, const eofa_term* t, const void* phi, double* F, const odwf_solve_opts* opts,
                          odwf_solve_stats* stats, void* stream) {
    if (!h || !phi || !F) return set_err(h, ODWF_EINVAL, "null argument");
    if (!h->have_gauge) return set_err(h, ODWF_EINVAL, "odwf_set_gauge has not been called");
    return term_force(h, t, phi, F, 1.0, 0, opts, stats, (cudaStream_t)stream);
}

extern "C" int eofa_term_spectrum(odwf_t* h, const eofa_term* t, const void* v0, int n_iter, double* lo, double* hi,
                                  const odwf_solve_opts* opts, void* stream) {
    if (!h || !v0 || !lo || !hi) return set_err(h, ODWF_EINVAL, "null argument");
    if (!h->have_gauge) return set_err(h, ODWF_EINVAL, "odwf_set_gauge has not been called");
    if (n_iter < 1 || n_iter > 1000) return set_err(h, ODWF_EINVAL, "n_iter must lie in 1..1000");
    int rc = check_term(h, t);
    if (rc) return rc;
    int iters = 0;
    return term_spectrum(h, t, v0, n_iter, lo, hi, opts, &iters, (cudaStream_t)stream);
}

extern "C" int eofa_heatbath(odwf_t* h, const eofa_term* t, const void* eta, void* phi, odwf_hb_opts* hb,
                             void* stream) {
    if (!h || !eta || !phi) return set_err(h, ODWF_EINVAL, "null argument");
    if (!h->have_gauge) return set_err(h, ODWF_EINVAL, "odwf_set_gauge has not been called");
    int rc = check_term(h, t);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const double mref = t->chirality < 0 ? t->m4 : t->m3;
    double x_lo = 0.98 * (1.0 + mref) / (1.0 + t->m_den), x_hi = 1.0, target = 1e-11;
    odwf_solve_opts so{1e-10, 100000, ODWF_PREC_DOUBLE, 0.1, 0.0};
    if (hb) {
        so = hb->solve;
        if (hb->x_lo > 0.0) {
            x_lo = hb->x_lo;
            x_hi = hb->x_hi;
        }
        if (hb->rat_err > 0.0) target = hb->rat_err;
    }
    if (!(x_lo > 0.0 && x_hi > x_lo)) return set_err(h, ODWF_EINVAL, "bad spectral interval");
    if (hb && hb->check_iters > 0) {
        // Lanczos on X from eta: its extreme Ritz values lie inside the spectrum of X and approach its
        // ends; an interval that does not contain them cannot contain the spectrum
        double rlo = 0.0, rhi = 0.0;
        int it = 0;
        odwf_solve_opts co = so;
        if (co.tol < 1e-8) co.tol = 1e-8;
        if ((rc = term_spectrum(h, t, eta, hb->check_iters, &rlo, &rhi, &co, &it, st))) return rc;
        hb->ritz_lo_out = rlo;
        hb->ritz_hi_out = rhi;
        if (rlo < x_lo || rhi > x_hi) {
            char buf[200];
            std::snprintf(buf, sizeof buf, "spectrum of X estimated as [%.6g, %.6g] by Lanczos, outside the interval "
                          "[%.6g, %.6g] of the rational approximation", rlo, rhi, x_lo, x_hi);
            return set_err(h, ODWF_ESPECTRUM, buf);
        }
    }
    Rational r;
    int n = 1;
    for (; n <= 64; ++n) {
        r = zolotarev_inv_sqrt(n, x_lo, x_hi);
        if (r.err <= target) break;
    }
    if (n > 64) return set_err(h, ODWF_EINVAL, "rational approximation did not reach the target error");
    const double k = term_k(t);
    double c0 = r.a0;
    for (int l = 0; l < n; ++l) c0 += r.a[l] / (1.0 + r.b[l]);
    // phi = c0 P eta + sum_l w_l P Omega^T chi_l
    k_scale4<<<grid_for(h, (size_t)h->V * 12, 256), 256, 0, st>>>((const double2*)eta, (double2*)phi, h->V,
                                                                    t->chirality, c0);
    if ((rc = cuda_check(h, cudaGetLastError(), "k_scale4"))) return rc;
    if ((rc = ensure_workspace(h, ST_DOUBLE))) return rc;
    if ((rc = embed(h, t, eta, st))) return rc;
    double om[kMaxNs];
    omega_vec(h, t->chirality, om);
    // every pole is one shifted-mass system with the same source: solve them as one batch
    std::vector<double> m12(2 * (size_t)n), wl(n);
    for (int l = 0; l < n; ++l) {
        const double kp = k / (1.0 + r.b[l]);
        const double mp = (kp * (1.0 + mref) + 2.0 * mref) / (2.0 - kp * (1.0 + mref));
        m12[2 * l] = t->chirality < 0 ? t->m3 : mp;
        m12[2 * l + 1] = t->chirality < 0 ? mp : t->m4;
        wl[l] = (t->chirality < 0 ? 1.0 : -1.0) * (r.a[l] / (1.0 + r.b[l])) * kp;
    }
    std::vector<odwf_solve_stats> ss(n);
    std::vector<Workspace*> wsx;
    const int src = solve_shared_rhs(h, n, m12.data(), h->ws.b_e, h->ws.b_o, &so, ss.data(), wsx, st);
    if (src != ODWF_OK && src != ODWF_ENOCONV) return src;
    const int worst = src;
    int iters = 0;
    for (int l = 0; l < n; ++l) {
        iters += ss[l].iters;
        double w[kMaxNs];
        for (int q = 0; q < h->Ns; ++q) w[q] = wl[l] * om[q];
        if ((rc = contract(h, t->chirality, w, nullptr, phi, 0, st, wsx[l]))) return rc;
    }
    if (hb) {
        hb->n_poles_out = n;
        hb->iters_out = iters;
    }
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "sync"))) return rc;
    return worst;
}
