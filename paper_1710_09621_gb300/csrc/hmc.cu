// HMC molecular dynamics on the GPU: the Wilson plaquette gauge action and its force, the momentum
// and link updates, and the Omelyan integrator with multiple time scales around the EOFA fermion
// forces (Section 1: HMC outline, Eq.(molecular_U), Eq.(molecular_P); Section 3: Omelyan integrator,
// MTS levels (k0, k1, k2), Wilson plaquette action).
//
// Conventions (the paper leaves them open): U_l = exp(i A_l^a t^a) with t^a = lambda^a / 2, momenta
// P_l = P_l^a t^a with H = 1/2 sum (P_l^a)^2 + S_g + S_pf, forces F^a = -dS/dw^a for
// U -> exp(i w^a t^a) U; S_g = beta sum_{x, mu < nu} (1 - Re tr U_{mu nu}(x) / 3). Everything here is FP64.
// Fields: U [4][V][3][3] complex128 (the ABI gauge layout), P and F [4][V][8] double.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>
#include <string>
#include <vector>

#include "field_access.cuh"

namespace odwf {
namespace {

struct Geo {
    int L[4];
    int V;
};

__device__ __forceinline__ int site_shift(int lex, int mu, int d, const Geo& g) {
    int c[4] = {lex % g.L[0], (lex / g.L[0]) % g.L[1], (lex / (g.L[0] * g.L[1])) % g.L[2],
                lex / (g.L[0] * g.L[1] * g.L[2])};
    c[mu] = (c[mu] + d + g.L[mu]) % g.L[mu];
    return c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}

struct M3 {
    double2 m[9];
};

__device__ __forceinline__ M3 m3_load(const double2* U, int mu, int lex, int V) {
    M3 r;
    const double2* p = U + ((size_t)mu * V + lex) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) r.m[k] = p[k];
    return r;
}

// c = a b (tb = 0) or a b^dag (tb = 1); ta = 1 takes a^dag
template <bool TA, bool TB>
__device__ __forceinline__ M3 m3_mul(const M3& a, const M3& b) {
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                double2 x = TA ? a.m[k * 3 + i] : a.m[i * 3 + k];
                double2 y = TB ? b.m[j * 3 + k] : b.m[k * 3 + j];
                if (TA) x.y = -x.y;
                if (TB) y.y = -y.y;
                re = fma(x.x, y.x, fma(-x.y, y.y, re));
                im = fma(x.x, y.y, fma(x.y, y.x, im));
            }
            c.m[i * 3 + j] = make_double2(re, im);
        }
    return c;
}

// Im tr(lambda^a Z) for the eight Gell-Mann matrices: tr(lambda Z) = sum_{ij} lambda_{ij} Z_{ji}
__device__ __forceinline__ void im_tr_lambda(const M3& Z, double* im) {
    auto zr = [&](int i, int j) { return Z.m[i * 3 + j].x; };
    auto zi = [&](int i, int j) { return Z.m[i * 3 + j].y; };
    im[0] = zi(1, 0) + zi(0, 1);
    im[1] = -zr(1, 0) + zr(0, 1);
    im[2] = zi(0, 0) - zi(1, 1);
    im[3] = zi(2, 0) + zi(0, 2);
    im[4] = -zr(2, 0) + zr(0, 2);
    im[5] = zi(2, 1) + zi(1, 2);
    im[6] = -zr(2, 1) + zr(1, 2);
    im[7] = (zi(0, 0) + zi(1, 1) - 2.0 * zi(2, 2)) * 0.57735026918962576451;
}

// Gauge force of link (mu, x): Sigma = sum_{nu != mu} [U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
//   + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)] holds every plaquette through U_mu(x), and
//   F^a = -(beta/3) Im tr(t^a U Sigma) = -(beta/6) Im tr(lambda^a U Sigma).
// out = F (accumulate = 0) or P += coef F (accumulate = 1).
__global__ void k_gauge_force(const double2* __restrict__ U, Geo g, double beta, double* out, double coef,
                              int accumulate) {
    const int total = 4 * g.V;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int mu = i / g.V, x = i % g.V;
        M3 S;
#pragma unroll
        for (int k = 0; k < 9; ++k) S.m[k] = make_double2(0.0, 0.0);
        const int xpmu = site_shift(x, mu, 1, g);
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == mu) continue;
            const int xpnu = site_shift(x, nu, 1, g), xmnu = site_shift(x, nu, -1, g);
            const int xpmu_mnu = site_shift(xpmu, nu, -1, g);
            const M3 up = m3_mul<false, true>(m3_mul<false, true>(m3_load(U, nu, xpmu, g.V), m3_load(U, mu, xpnu, g.V)),
                                              m3_load(U, nu, x, g.V));
            const M3 dn = m3_mul<false, false>(m3_mul<true, true>(m3_load(U, nu, xpmu_mnu, g.V), m3_load(U, mu, xmnu, g.V)),
                                               m3_load(U, nu, xmnu, g.V));
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                S.m[k].x += up.m[k].x + dn.m[k].x;
                S.m[k].y += up.m[k].y + dn.m[k].y;
            }
        }
        const M3 W = m3_mul<false, false>(m3_load(U, mu, x, g.V), S);
        double im[8];
        im_tr_lambda(W, im);
        double* o = out + (size_t)i * 8;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const double f = -(beta / 6.0) * im[a];
            o[a] = accumulate ? fma(coef, f, o[a]) : f;
        }
    }
}

// per-block partial sums of sum_x sum_{mu < nu} Re tr U_{mu nu}(x)
__global__ void k_plaquette_sum(const double2* __restrict__ U, Geo g, double* partials) {
    __shared__ double wsum[32];
    double acc = 0.0;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.V; x += gridDim.x * blockDim.x) {
        for (int mu = 0; mu < 4; ++mu) {
            const int xpmu = site_shift(x, mu, 1, g);
            for (int nu = mu + 1; nu < 4; ++nu) {
                const int xpnu = site_shift(x, nu, 1, g);
                const M3 a = m3_mul<false, false>(m3_load(U, mu, x, g.V), m3_load(U, nu, xpmu, g.V));
                const M3 b = m3_mul<false, false>(m3_load(U, nu, x, g.V), m3_load(U, mu, xpnu, g.V));
                // Re tr(a b^dag) = sum_{ij} Re(a_ij conj(b_ij))
#pragma unroll
                for (int k = 0; k < 9; ++k) acc += a.m[k].x * b.m[k].x + a.m[k].y * b.m[k].y;
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) b += wsum[q];
        partials[blockIdx.x] = b;
    }
}

// U <- exp(i tau P^a t^a) U on every link. exp(i Q) of the Hermitian traceless Q = tau P^a lambda^a / 2 by
// scaling and squaring: Q / 2^k with Frobenius norm <= 1/4, then the Taylor series to order 14 in Horner
// form (truncation below 1e-20 relative), then k squarings.
__global__ void k_link_update(double2* __restrict__ U, const double* __restrict__ P, double tau, int nlinks) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nlinks; i += gridDim.x * blockDim.x) {
        const double* p = P + (size_t)i * 8;
        const double h = 0.5 * tau, r3 = 0.57735026918962576451;
        // Q = tau sum_a P^a lambda^a / 2
        M3 Q;
        Q.m[0] = make_double2(h * (p[2] + r3 * p[7]), 0.0);
        Q.m[4] = make_double2(h * (-p[2] + r3 * p[7]), 0.0);
        Q.m[8] = make_double2(-2.0 * h * r3 * p[7], 0.0);
        Q.m[1] = make_double2(h * p[0], -h * p[1]);
        Q.m[3] = make_double2(h * p[0], h * p[1]);
        Q.m[2] = make_double2(h * p[3], -h * p[4]);
        Q.m[6] = make_double2(h * p[3], h * p[4]);
        Q.m[5] = make_double2(h * p[5], -h * p[6]);
        Q.m[7] = make_double2(h * p[5], h * p[6]);
        double n2 = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) n2 += Q.m[k].x * Q.m[k].x + Q.m[k].y * Q.m[k].y;
        int sq = 0;
        double sc = 1.0;
        while (n2 * sc * sc > 0.0625 && sq < 60) {
            sc *= 0.5;
            ++sq;
        }
        // A = i sc Q
        M3 A;
#pragma unroll
        for (int k = 0; k < 9; ++k) A.m[k] = make_double2(-sc * Q.m[k].y, sc * Q.m[k].x);
        // E = I + A/1 (I + A/2 (I + ... (I + A/14)))
        M3 E;
#pragma unroll
        for (int k = 0; k < 9; ++k) E.m[k] = make_double2((k % 4 == 0) ? 1.0 : 0.0, 0.0);
        for (int n = 14; n >= 1; --n) {
            M3 T = m3_mul<false, false>(A, E);
            const double inv = 1.0 / n;
#pragma unroll
            for (int k = 0; k < 9; ++k)
                E.m[k] = make_double2(((k % 4 == 0) ? 1.0 : 0.0) + inv * T.m[k].x, inv * T.m[k].y);
        }
        for (int s = 0; s < sq; ++s) E = m3_mul<false, false>(E, E);
        M3 u;  // link i = mu V + x
#pragma unroll
        for (int k = 0; k < 9; ++k) u.m[k] = U[(size_t)i * 9 + k];
        const M3 w = m3_mul<false, false>(E, u);
#pragma unroll
        for (int k = 0; k < 9; ++k) U[(size_t)i * 9 + k] = w.m[k];
    }
}

__global__ void k_axpy_d(double* y, const double* x, double c, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = fma(c, x[i], y[i]);
}

__global__ void k_sumsq_d(const double* x, size_t n, double* partials) {
    __shared__ double wsum[32];
    double v = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        v = fma(x[i], x[i], v);
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

Geo geo_of(const odwf_s* h) {
    Geo g;
    for (int i = 0; i < 4; ++i) g.L[i] = h->L[i];
    g.V = h->V;
    return g;
}

int grid_n(const odwf_s* h, size_t n, int block) {
    size_t g = (n + block - 1) / block;
    const size_t cap = (size_t)h->num_sms * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

// deterministic host sum of the first g block partials
int sum_partials(odwf_s* h, int g, double* out, cudaStream_t st) {
    std::vector<double> part(g);
    int rc = cuda_check(h, cudaMemcpyAsync(part.data(), h->partials, sizeof(double) * g, cudaMemcpyDeviceToHost, st),
                        "partials D2H");
    if (!rc) rc = cuda_check(h, cudaStreamSynchronize(st), "sync");
    if (rc) return rc;
    double s = 0.0;
    for (double p : part) s += p;
    *out = s;
    return ODWF_OK;
}

int gauge_action(odwf_s* h, const void* U, double beta, double* S, cudaStream_t st) {
    int g = grid_n(h, h->V, 256);
    if (g > h->partials_n) g = h->partials_n;
    k_plaquette_sum<<<g, 256, 0, st>>>((const double2*)U, geo_of(h), h->partials);
    int rc = cuda_check(h, cudaGetLastError(), "k_plaquette_sum");
    if (rc) return rc;
    double tr = 0.0;
    if ((rc = sum_partials(h, g, &tr, st))) return rc;
    *S = beta * (6.0 * (double)h->V - tr / 3.0);
    return ODWF_OK;
}

int gauge_force(odwf_s* h, const void* U, double beta, double* out, double coef, int accumulate, cudaStream_t st) {
    k_gauge_force<<<grid_n(h, 4 * (size_t)h->V, 128), 128, 0, st>>>((const double2*)U, geo_of(h), beta, out, coef,
                                                                     accumulate);
    return cuda_check(h, cudaGetLastError(), "k_gauge_force");
}

int link_update(odwf_s* h, void* U, const double* P, double tau, cudaStream_t st) {
    k_link_update<<<grid_n(h, 4 * (size_t)h->V, 128), 128, 0, st>>>((double2*)U, P, tau, 4 * h->V);
    return cuda_check(h, cudaGetLastError(), "k_link_update");
}

int kinetic(odwf_s* h, const double* P, double* K, cudaStream_t st) {
    const size_t n = (size_t)h->V * 32;
    int g = grid_n(h, n, 256);
    if (g > h->partials_n) g = h->partials_n;
    k_sumsq_d<<<g, 256, 0, st>>>(P, n, h->partials);
    int rc = cuda_check(h, cudaGetLastError(), "k_sumsq_d");
    if (rc) return rc;
    double s = 0.0;
    if ((rc = sum_partials(h, g, &s, st))) return rc;
    *K = 0.5 * s;
    return ODWF_OK;
}

}  // namespace
}  // namespace odwf

using namespace odwf;

extern "C" int hmc_gauge_action(odwf_t* h, const void* U, double beta, double* S, void* stream) {
    if (!h || !U || !S) return set_err(h, ODWF_EINVAL, "null argument");
    return gauge_action(h, U, beta, S, (cudaStream_t)stream);
}

extern "C" int hmc_gauge_force(odwf_t* h, const void* U, double beta, double* F, void* stream) {
    if (!h || !U || !F) return set_err(h, ODWF_EINVAL, "null argument");
    return gauge_force(h, U, beta, F, 1.0, 0, (cudaStream_t)stream);
}

extern "C" int hmc_momentum_update(odwf_t* h, double* P, const double* F, double eps, void* stream) {
    if (!h || !P || !F) return set_err(h, ODWF_EINVAL, "null argument");
    const size_t n = (size_t)h->V * 32;
    k_axpy_d<<<grid_n(h, n, 256), 256, 0, (cudaStream_t)stream>>>(P, F, eps, n);
    return cuda_check(h, cudaGetLastError(), "k_axpy_d");
}

extern "C" int hmc_link_update(odwf_t* h, void* U, const double* P, double tau, void* stream) {
    if (!h || !U || !P) return set_err(h, ODWF_EINVAL, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = link_update(h, U, P, tau, st);
    if (rc) return rc;
    // the operator calls read the library's reordered copies: refresh them from the new links
    if ((rc = launch_gauge(h, (const double*)U, st))) return rc;
    h->have_gauge = true;
    return ODWF_OK;
}

extern "C" int hmc_kinetic(odwf_t* h, const double* P, double* K, void* stream) {
    if (!h || !P || !K) return set_err(h, ODWF_EINVAL, "null argument");
    return kinetic(h, P, K, (cudaStream_t)stream);
}

extern "C" int hmc_md(odwf_t* h, void* U, double* P, double beta, int nterms, const eofa_term* terms,
                      const void* const* phis, const int* term_level, int nlevels, const int* steps, double tau,
                      double lambda, const odwf_solve_opts* opts, hmc_md_stats* stats, void* stream) {
    using namespace odwf;
    if (!h || !U || !P || (nterms > 0 && (!terms || !phis || !term_level)) || !steps || nterms < 0)
        return set_err(h, ODWF_EINVAL, "null argument");
    if (nlevels < 1 || nlevels > ODWF_HMC_MAX_LEVELS) return set_err(h, ODWF_EINVAL, "nlevels must lie in 1..4");
    for (int l = 0; l < nlevels; ++l) {
        if (steps[l] < 1) return set_err(h, ODWF_EINVAL, "steps must be positive");
        if (l + 1 < nlevels && steps[l] % (2 * steps[l + 1]))
            return set_err(h, ODWF_EINVAL, "steps[l] must be a multiple of 2 steps[l + 1]");
    }
    for (int i = 0; i < nterms; ++i)
        if (term_level[i] < 0 || term_level[i] >= nlevels || !phis[i])
            return set_err(h, ODWF_EINVAL, "term level outside 0..nlevels-1 or null pseudofermion");
    if (!(tau > 0.0)) return set_err(h, ODWF_EINVAL, "tau must be positive");
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)stream;
    hmc_md_stats s{};
    int rc = launch_gauge(h, (const double*)U, st);
    if (rc) return rc;
    h->have_gauge = true;
    bool gauge_dirty = false;
    auto refresh = [&]() -> int {
        if (!gauge_dirty) return ODWF_OK;
        gauge_dirty = false;
        return launch_gauge(h, (const double*)U, st);
    };
    // H = K + S_g + sum of the terms' actions (one solve each)
    auto energy = [&](double* K, double* Sg, double* Sf) -> int {
        int r = kinetic(h, P, K, st);
        if (!r) r = gauge_action(h, U, beta, Sg, st);
        if (r) return r;
        if ((r = refresh())) return r;
        *Sf = 0.0;
        for (int i = 0; i < nterms; ++i) {
            double S = 0.0;
            odwf_solve_stats ss{};
            r = eofa_action(h, &terms[i], phis[i], &S, opts, &ss, st);
            s.cg_iters += ss.iters;
            if (r) return r;
            *Sf += S;
        }
        return ODWF_OK;
    };
    if ((rc = energy(&s.K0, &s.Sg0, &s.Sf0))) return rc;
    // momentum updates are pending per level and applied at the current links before the next link
    // update (updates at the same links add: P += a F(U) + b F(U) = P += (a + b) F(U))
    std::vector<double> pend(nlevels, 0.0);
    auto flush = [&]() -> int {
        for (int l = 0; l < nlevels; ++l) {
            if (pend[l] == 0.0) continue;
            int r;
            if (l == 0 && (r = gauge_force(h, U, beta, P, pend[l], 1, st))) return r;
            for (int i = 0; i < nterms; ++i) {
                if (term_level[i] != l) continue;
                if ((r = refresh())) return r;
                odwf_solve_stats ss{};
                r = term_force(h, &terms[i], phis[i], P, pend[l], 1, opts, &ss, st);
                s.cg_iters += ss.iters;
                if (r) return r;
            }
            ++s.force_evals[l];
            pend[l] = 0.0;
        }
        return ODWF_OK;
    };
    std::function<int(int, double)> below = [&](int level, double t) -> int {
        int r;
        if (level < 0) {
            if ((r = flush())) return r;
            if ((r = link_update(h, U, P, t, st))) return r;
            gauge_dirty = true;
            ++s.link_updates;
            return ODWF_OK;
        }
        const int n = (level == nlevels - 1) ? steps[level] : steps[level] / (2 * steps[level + 1]);
        const double e = t / n;
        for (int j = 0; j < n; ++j) {
            pend[level] += lambda * e;
            if ((r = below(level - 1, 0.5 * e))) return r;
            pend[level] += (1.0 - 2.0 * lambda) * e;
            if ((r = below(level - 1, 0.5 * e))) return r;
            pend[level] += lambda * e;
        }
        return ODWF_OK;
    };
    if ((rc = below(nlevels - 1, tau))) return rc;
    if ((rc = flush())) return rc;
    if ((rc = energy(&s.K1, &s.Sg1, &s.Sf1))) return rc;
    if ((rc = refresh())) return rc;
    s.dH = (s.K1 - s.K0) + (s.Sg1 - s.Sg0) + (s.Sf1 - s.Sf0);
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "sync"))) return rc;
    s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = s;
    return ODWF_OK;
}
