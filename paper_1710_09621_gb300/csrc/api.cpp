// Handle management, fifth-dimension coefficient setup and the operator applies of the C ABI.
//
// The fifth-dimension matrices are the optimal domain-wall ones read with c = 1, d = 0:
//   M_pm(m) = omega^{-1/2} (1 - L_pm(m)) (1 + L_pm(m))^{-1} omega^{-1/2}      (Eq.(DTm1m2) blocks)
//   (L_+)_{s,s-1} = 1 (s >= 1), (L_+)_{0,Ns-1} = -m, L_- = L_+^T
// and the even-odd diagonal block is A_pm = (4 - m0) + M_pm. They are computed once per mass pair
// on the host in FP64 (Ns x Ns, negligible work) and uploaded transposed for the kernels.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "odwf_internal.h"

using namespace odwf;

namespace odwf {

int spb_for(int Ns);
int solve_core(odwf_s* h, double m1, double m2, const odwf_solve_opts* opts, odwf_solve_stats* stats,
               cudaStream_t st);

static std::string g_create_err;
int ensure_ws(odwf_s* h, Workspace& w, int inner);

int set_err(odwf_s* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_err = msg;
    return code;
}

int cuda_check(odwf_s* h, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return ODWF_OK;
    return set_err(h, ODWF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int check_fault(odwf_s* h, cudaStream_t st) {
    if (!h->staged_used) return ODWF_OK;
    int rc = cuda_check(h, cudaMemcpyAsync(h->fault_host, h->fault, sizeof(unsigned int), cudaMemcpyDeviceToHost, st),
                        "fault word D2H");
    if (!rc) rc = cuda_check(h, cudaStreamSynchronize(st), "stream sync");
    if (rc) return rc;
    h->staged_used = false;
    if (*h->fault_host == 0u) return ODWF_OK;
    *h->fault_host = 0u;
    if ((rc = cuda_check(h, cudaMemsetAsync(h->fault, 0, sizeof(unsigned int), st), "fault word reset"))) return rc;
    return set_err(h, ODWF_EFAULT, "a bulk-staged hop kernel's wait for its neighbour copies ran out; its outputs "
                                   "are incomplete");
}

// ---- small dense FP64 linear algebra on the host (Ns <= 32) ------------------------------------
using Mat = std::vector<double>;  // row-major Ns x Ns

static Mat mat_eye(int n) {
    Mat m(n * n, 0.0);
    for (int i = 0; i < n; ++i) m[i * n + i] = 1.0;
    return m;
}

static Mat mat_mul(const Mat& a, const Mat& b, int n) {
    Mat c(n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const double aik = a[i * n + k];
            if (aik == 0.0) continue;
            for (int j = 0; j < n; ++j) c[i * n + j] += aik * b[k * n + j];
        }
    return c;
}

// Gauss-Jordan elimination with partial pivoting; returns false if singular.
static bool mat_inv(const Mat& a, Mat& inv, int n) {
    Mat w = a;
    inv = mat_eye(n);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(w[r * n + col]) > std::fabs(w[piv * n + col])) piv = r;
        if (w[piv * n + col] == 0.0) return false;
        if (piv != col)
            for (int j = 0; j < n; ++j) {
                std::swap(w[piv * n + j], w[col * n + j]);
                std::swap(inv[piv * n + j], inv[col * n + j]);
            }
        const double d = 1.0 / w[col * n + col];
        for (int j = 0; j < n; ++j) {
            w[col * n + j] *= d;
            inv[col * n + j] *= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const double f = w[r * n + col];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                w[r * n + j] -= f * w[col * n + j];
                inv[r * n + j] -= f * inv[col * n + j];
            }
        }
    }
    return true;
}

static Mat transpose(const Mat& a, int n) {
    Mat t(n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) t[j * n + i] = a[i * n + j];
    return t;
}

// M_pm(m) for chirality c = +1 (L_+) or -1 (L_- = L_+^T)
static bool m_matrix(const std::vector<double>& omega, double m, int c, Mat& M) {
    const int n = (int)omega.size();
    Mat L(n * n, 0.0);
    for (int s = 1; s < n; ++s) L[s * n + (s - 1)] = 1.0;
    L[0 * n + (n - 1)] = -m;
    if (c < 0) L = transpose(L, n);
    Mat onepl = mat_eye(n), oneml = mat_eye(n);
    for (int i = 0; i < n * n; ++i) {
        onepl[i] += L[i];
        oneml[i] -= L[i];
    }
    Mat inv;
    if (!mat_inv(onepl, inv, n)) return false;
    Mat core = mat_mul(oneml, inv, n);
    M.assign(n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) M[i * n + j] = core[i * n + j] / std::sqrt(omega[i] * omega[j]);
    return true;
}

// The kNumCoef fifth-dimension matrices of a mass pair, each stored transposed (Mt[s'][s]), in
// the order documented at SCoef. Host FP64; returns false (with a message) if a block is singular.
bool coef_host(const odwf_s* h, double m1, double m2, std::vector<double>& host, std::string& err) {
    const int n = h->Ns;
    Mat Mp, Mm;
    if (!m_matrix(h->omega, m1, +1, Mp) || !m_matrix(h->omega, m2, -1, Mm)) {
        err = "singular 1 + L in the fifth-dimension setup";
        return false;
    }
    Mat Ap = Mp, Am = Mm;
    for (int i = 0; i < n; ++i) {
        Ap[i * n + i] += 4.0 - h->m0;
        Am[i * n + i] += 4.0 - h->m0;
    }
    Mat Api, Ami;
    if (!mat_inv(Ap, Api, n) || !mat_inv(Am, Ami, n)) {
        err = "singular even-odd diagonal block A";
        return false;
    }
    // D_odwf = omega^{1/2} D_T omega^{1/2} (1 + L): N_pm = omega^{1/2} (1 + L_pm), W = omega^{1/2}
    Mat Np(n * n, 0.0), Nm(n * n, 0.0), W(n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        const double sq = std::sqrt(h->omega[i]);
        W[i * n + i] = sq;
        Np[i * n + i] = sq;
        Nm[i * n + i] = sq;
        if (i >= 1) Np[i * n + (i - 1)] = sq;       // (L_+)_{i,i-1} = 1
        if (i + 1 < n) Nm[i * n + (i + 1)] = sq;    // (L_-)_{i,i+1} = 1
    }
    Np[0 * n + (n - 1)] = -m1 * std::sqrt(h->omega[0]);
    Nm[(n - 1) * n + 0] = -m2 * std::sqrt(h->omega[n - 1]);
    // order: A+, A-, A+^-1, A-^-1, A+^T, A-^T, A+^-T, A-^-T, N+, N-, W, W, N+^T, N-^T
    const Mat* mats[kNumCoef];
    Mat ApT = transpose(Ap, n), AmT = transpose(Am, n), ApiT = transpose(Api, n), AmiT = transpose(Ami, n);
    Mat NpT = transpose(Np, n), NmT = transpose(Nm, n);
    mats[0] = &Ap; mats[1] = &Am; mats[2] = &Api; mats[3] = &Ami;
    mats[4] = &ApT; mats[5] = &AmT; mats[6] = &ApiT; mats[7] = &AmiT;
    mats[8] = &Np; mats[9] = &Nm; mats[10] = &W; mats[11] = &W; mats[12] = &NpT; mats[13] = &NmT;
    host.assign((size_t)kNumCoef * n * n, 0.0);
    for (int k = 0; k < kNumCoef; ++k) {
        Mat t = transpose(*mats[k], n);
        std::memcpy(host.data() + (size_t)k * n * n, t.data(), sizeof(double) * n * n);
    }
    return true;
}

bool struct_host(const odwf_s* h, double m1, double m2, SStruct* out) {
    const int n = h->Ns;
    if (n != kStructNs) return false;
    SStructT<double>& d = out->d;
    const double a4 = 4.0 - h->m0;
    double q = 1.0;
    for (int s = 0; s < n; ++s) {
        const double om = h->omega[s], dd = a4 * om + 1.0, ee = a4 * om - 1.0;
        d.w[s] = std::sqrt(om);
        d.rw[s] = std::sqrt(om) / dd;
        d.f[s] = ee / dd;
        if (s > 0) q *= -ee / dd;
        d.q[s] = q;
        d.wi[s] = 1.0 / std::sqrt(om);
        d.adiag[s] = a4 - 1.0 / om;
        d.wi2s[s] = ((s & 1) ? -2.0 : 2.0) / std::sqrt(om);
    }
    const double d0 = a4 * h->omega[0] + 1.0, e0 = a4 * h->omega[0] - 1.0;
    const double ms[2] = {m1, m2};
    for (int c = 0; c < 2; ++c) {
        d.m[c] = ms[c];
        d.me0[c] = ms[c] * e0;
        d.cu[c] = 1.0 / (d0 - ms[c] * e0 * d.q[n - 1]);
        d.au[c] = 1.0 / (1.0 + ms[c]);
    }
    SStructT<float>& f = out->f;
    for (int s = 0; s < n; ++s) {
        f.w[s] = (float)d.w[s], f.rw[s] = (float)d.rw[s], f.f[s] = (float)d.f[s], f.q[s] = (float)d.q[s];
        f.wi[s] = (float)d.wi[s], f.adiag[s] = (float)d.adiag[s], f.wi2s[s] = (float)d.wi2s[s];
    }
    for (int c = 0; c < 2; ++c) {
        f.m[c] = (float)d.m[c], f.me0[c] = (float)d.me0[c], f.cu[c] = (float)d.cu[c], f.au[c] = (float)d.au[c];
    }
    return true;
}

void set_sop(HopArgs& a, const SCoef* c, int sop) {
    if (!c->has_st) {
        a.sop = SOP_DENSE;
        return;
    }
    a.sop = sop;
    a.sc = c->st;
}

const SCoef* get_coef(odwf_s* h, double m1, double m2) {
    auto key = std::make_pair(m1, m2);
    auto it = h->coefs.find(key);
    if (it != h->coefs.end()) return &it->second;
    std::vector<double> host;
    std::string err;
    if (!coef_host(h, m1, m2, host, err)) {
        set_err(h, ODWF_EINVAL, err);
        return nullptr;
    }
    SCoef c;
    c.has_st = !h->dense_s && struct_host(h, m1, m2, &c.st);
    if (cudaMalloc(&c.dev, sizeof(double) * host.size()) != cudaSuccess) {
        set_err(h, ODWF_ENOMEM, "cudaMalloc coefficients");
        return nullptr;
    }
    if (cudaMemcpy(c.dev, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(c.dev);
        set_err(h, ODWF_ECUDA, "cudaMemcpy coefficients");
        return nullptr;
    }
    auto res = h->coefs.emplace(key, c);
    return &res.first->second;
}

static int alloc(odwf_s* h, void** p, size_t bytes) {
    if (*p) return ODWF_OK;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        *p = nullptr;
        return set_err(h, ODWF_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    return ODWF_OK;
}

int ensure_workspace(odwf_s* h, int inner) { return ensure_ws(h, h->ws, inner); }

int ensure_ws(odwf_s* h, Workspace& w, int inner) {
    const size_t b64 = half_elems_bytes(h, ST_DOUBLE);
    int rc;
    void** f64s[] = {&w.b_e, &w.b_o, &w.x_e, &w.x_o, &w.r64, &w.t64, &w.bh};
    for (void** p : f64s)
        if ((rc = alloc(h, p, b64))) return rc;
    // inner-solver fields, sized for the widest storage requested so far
    const size_t bi = half_elems_bytes(h, inner == ST_HALF ? ST_FLOAT : inner);
    if (bi > w.inner_bytes) {
        void** fis[] = {&w.xi, &w.ri, &w.pi, &w.ti};
        for (void** p : fis) {
            cudaFree(*p);
            *p = nullptr;
            if ((rc = alloc(h, p, bi))) return rc;
        }
        w.inner_bytes = bi;
    }
    if (inner == ST_HALF) {
        const size_t bs = (size_t)h->Vh * h->Ns * sizeof(float);
        void** scs[] = {(void**)&w.xi_s, (void**)&w.ri_s, (void**)&w.pi_s, (void**)&w.ti_s};
        for (void** p : scs)
            if ((rc = alloc(h, p, bs))) return rc;
    }
    return ODWF_OK;
}

}  // namespace odwf

// ================================================================================================
extern "C" {

const char* odwf_last_error(const odwf_t* h) { return h ? h->err.c_str() : odwf::g_create_err.c_str(); }

double eofa_k(double mj, double mi) { return 2.0 * (mj - mi) / ((1.0 + mj) * (1.0 + mi)); }

int odwf_create(odwf_t** out, const int dims[4], int Ns, double m0, const double* omega, int flags) {
    if (!out || !dims || !omega) return set_err(nullptr, ODWF_EINVAL, "null argument");
    *out = nullptr;
    (void)flags;
    for (int i = 0; i < 4; ++i)
        if (dims[i] < 2 || dims[i] % 2) return set_err(nullptr, ODWF_EINVAL, "every lattice extent must be even and >= 2");
    if (Ns < 2 || Ns % 2 || Ns > kMaxNs || spb_for(Ns) * Ns > 256)
        return set_err(nullptr, ODWF_EINVAL, "Ns must be even, <= 32 and not 18, 22, 26 or 30");
    if (!(m0 > 0.0 && m0 < 2.0)) return set_err(nullptr, ODWF_EINVAL, "m0 must lie in (0, 2)");
    for (int s = 0; s < Ns; ++s) {
        if (!(omega[s] > 0.0) || !std::isfinite(omega[s])) return set_err(nullptr, ODWF_EINVAL, "omega_s must be > 0");
        if (omega[s] != omega[Ns - 1 - s])
            return set_err(nullptr, ODWF_EINVAL, "omega must be R5-symmetric (omega_s == omega_{Ns-1-s})");
    }
    const long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
    if (V * Ns * 12 > (1LL << 40) || V > (1LL << 30)) return set_err(nullptr, ODWF_EINVAL, "lattice too large");
    odwf_s* h = new odwf_s();
    for (int i = 0; i < 4; ++i) h->L[i] = dims[i];
    h->V = (int)V;
    h->Vh = (int)(V / 2);
    h->Ns = Ns;
    h->m0 = m0;
    h->omega.assign(omega, omega + Ns);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        std::string msg = std::string("no CUDA device: ") + cudaGetErrorString(e);
        delete h;
        return set_err(nullptr, ODWF_ECUDA, msg);
    }
    // geometry tables (host-built, uploaded once)
    const int Lx = dims[0], Ly = dims[1], Lz = dims[2], Lt = dims[3];
    std::vector<int> lexof[2], cbof(V), nbr[2], nbrs[2];
    for (int p = 0; p < 2; ++p) {
        lexof[p].resize(h->Vh);
        nbr[p].resize((size_t)h->Vh * 8);
        nbrs[p].resize((size_t)h->Vh * 8);
    }
    // Checkerboard order: the lattice is tiled by 2^4 blocks (all extents are even); block b holds
    // the checkerboard indices 8b .. 8b+7 of each parity, lexicographic inside the block. A CTA of
    // 8 (or 16) consecutive sites therefore covers one (two) whole blocks, and half of the
    // neighbours it reads belong to its own block, which raises L1 reuse of the hopped field.
    const int nbx = Lx / 2, nby = Ly / 2, nbz = Lz / 2;
    for (int lex = 0; lex < V; ++lex) {
        const int x = lex % Lx, y = (lex / Lx) % Ly, z = (lex / (Lx * Ly)) % Lz, t = lex / (Lx * Ly * Lz);
        const int p = (x + y + z + t) & 1;
        const int b = (x / 2) + nbx * ((y / 2) + nby * ((z / 2) + nbz * (t / 2)));
        const int inner = (x & 1) + 2 * ((y & 1) + 2 * ((z & 1) + 2 * (t & 1)));  // 0..15
        const int cb = 8 * b + (inner >> 1);  // each parity takes every other inner index
        lexof[p][cb] = lex;
        cbof[lex] = cb;
    }
    for (int p = 0; p < 2; ++p)
        for (int cb = 0; cb < h->Vh; ++cb) {
            const int lex = lexof[p][cb];
            int c[4] = {lex % Lx, (lex / Lx) % Ly, (lex / (Lx * Ly)) % Lz, lex / (Lx * Ly * Lz)};
            const int L[4] = {Lx, Ly, Lz, Lt};
            for (int mu = 0; mu < 4; ++mu) {
                int f[4] = {c[0], c[1], c[2], c[3]}, b[4] = {c[0], c[1], c[2], c[3]};
                f[mu] = (f[mu] + 1) % L[mu];
                b[mu] = (b[mu] + L[mu] - 1) % L[mu];
                const int lf = f[0] + Lx * (f[1] + Ly * (f[2] + Lz * f[3]));
                const int lb = b[0] + Lx * (b[1] + Ly * (b[2] + Lz * b[3]));
                nbr[p][(size_t)cb * 8 + mu] = cbof[lf];
                nbr[p][(size_t)cb * 8 + 4 + mu] = cbof[lb];
                // signed table of the two-slice kernels: ~index where the link crosses the antiperiodic
                // t boundary (U_t(x) at x_t = Lt - 1, U_t(x - t)^dag at x_t = 0)
                const bool fneg = mu == 3 && c[3] == Lt - 1, bneg = mu == 3 && c[3] == 0;
                nbrs[p][(size_t)cb * 8 + mu] = fneg ? ~cbof[lf] : cbof[lf];
                nbrs[p][(size_t)cb * 8 + 4 + mu] = bneg ? ~cbof[lb] : cbof[lb];
            }
        }
    int rc = ODWF_OK;
    for (int p = 0; p < 2 && !rc; ++p) {
        rc = alloc(h, (void**)&h->lexof[p], sizeof(int) * h->Vh);
        if (!rc) rc = alloc(h, (void**)&h->nbr[p], sizeof(int) * 8 * (size_t)h->Vh);
        if (!rc) rc = alloc(h, (void**)&h->U64[p], sizeof(double) * 8 * 18 * (size_t)h->Vh);
        if (!rc) rc = alloc(h, (void**)&h->U32[p], sizeof(float) * 8 * 20 * (size_t)h->Vh);
        if (!rc) rc = alloc(h, (void**)&h->U12[p], sizeof(float) * 8 * 12 * (size_t)h->Vh);
        if (!rc) rc = alloc(h, (void**)&h->nbrs[p], sizeof(int) * 8 * (size_t)h->Vh);
        if (!rc) rc = cuda_check(h, cudaMemcpy(h->nbrs[p], nbrs[p].data(), sizeof(int) * 8 * (size_t)h->Vh, cudaMemcpyHostToDevice), "upload nbrs");
        if (!rc) rc = cuda_check(h, cudaMemcpy(h->lexof[p], lexof[p].data(), sizeof(int) * h->Vh, cudaMemcpyHostToDevice), "upload lexof");
        if (!rc) rc = cuda_check(h, cudaMemcpy(h->nbr[p], nbr[p].data(), sizeof(int) * 8 * (size_t)h->Vh, cudaMemcpyHostToDevice), "upload nbr");
    }
    h->partials_n = h->num_sms * 32;
    if (!rc) rc = alloc(h, (void**)&h->partials, sizeof(double) * h->partials_n);
    if (!rc) rc = alloc(h, (void**)&h->state, sizeof(CGState));
    if (!rc) rc = alloc(h, (void**)&h->fault, sizeof(unsigned int));
    if (!rc) rc = alloc(h, (void**)&h->u12_dev, sizeof(unsigned int));
    if (!rc) rc = cuda_check(h, cudaMallocHost((void**)&h->u12_dev_host, sizeof(unsigned int)), "cudaMallocHost link check");
    if (!rc) rc = cuda_check(h, cudaMemset(h->fault, 0, sizeof(unsigned int)), "memset fault");
    if (const char* e = std::getenv("ODWF_STAGED")) h->staged = (e[0] == '1') ? 1 : 0;
    if (const char* e = std::getenv("ODWF_TEST_WAIT_CYCLES")) h->wait_cycles = std::atoll(e);
    if (const char* e = std::getenv("ODWF_DENSE_S")) h->dense_s = (e[0] == '1');
    if (const char* e = std::getenv("ODWF_PAIR")) h->pair = (e[0] >= '0' && e[0] <= '3') ? e[0] - '0' : -1;
    if (!rc) rc = cuda_check(h, cudaMallocHost((void**)&h->fault_host, sizeof(unsigned int)), "cudaMallocHost fault");
    if (!rc) *h->fault_host = 0u;
    if (!rc) rc = cuda_check(h, cudaMemset(h->state, 0, sizeof(CGState)), "memset state");
    if (!rc) rc = cuda_check(h, cudaMallocHost((void**)&h->state_host, sizeof(CGState)), "cudaMallocHost state");
    if (rc) {
        std::string msg = h->err;
        odwf_destroy(h);
        return set_err(nullptr, rc, msg);
    }
    *out = h;
    return ODWF_OK;
}

int odwf_destroy(odwf_t* h) {
    if (!h) return ODWF_OK;
    for (int p = 0; p < 2; ++p) {
        cudaFree(h->nbr[p]);
        cudaFree(h->lexof[p]);
        cudaFree(h->U64[p]);
        cudaFree(h->U32[p]);
        cudaFree(h->U12[p]);
        cudaFree(h->nbrs[p]);
    }
    cudaFree(h->u12_dev);
    if (h->u12_dev_host) cudaFreeHost(h->u12_dev_host);
    for (auto& kv : h->coefs) cudaFree(kv.second.dev);
    for (auto& r : h->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : h->prof_pool) cudaEventDestroy(e);
    cudaFree(h->partials);
    cudaFree(h->state);
    cudaFree(h->fault);
    if (h->state_host) cudaFreeHost(h->state_host);
    if (h->fault_host) cudaFreeHost(h->fault_host);
    Workspace& w = h->ws;
    void* ps[] = {w.b_e, w.b_o, w.x_e, w.x_o, w.r64, w.t64, w.bh, w.xi, w.ri, w.pi, w.ti,
                  w.xi_s, w.ri_s, w.pi_s, w.ti_s, h->f64[0], h->f64[1], h->f64[2], h->f64[3], h->acc4,
                  h->lz[0], h->lz[1], h->lz[2]};
    for (void* p : ps) cudaFree(p);
    for (Workspace& b : h->bws) {
        void* qs[] = {b.b_e, b.b_o, b.x_e, b.x_o, b.r64, b.t64, b.bh, b.xi, b.ri, b.pi, b.ti, b.xi_s, b.ri_s, b.pi_s, b.ti_s};
        for (void* q : qs) cudaFree(q);
    }
    cudaFree(h->bstate);
    cudaFree(h->bpartials);
    cudaFree(h->bargs);
    if (h->bstate_host) cudaFreeHost(h->bstate_host);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->gcr_free) h->gcr_free(h->gcr);
    delete h;
    return ODWF_OK;
}

int odwf_set_gauge(odwf_t* h, const void* U, void* stream) {
    if (!h || !U) return set_err(h, ODWF_EINVAL, "null argument");
    int rc = launch_gauge(h, (const double*)U, (cudaStream_t)stream);
    if (!rc) h->have_gauge = true;
    return rc;
}

int odwf_omega_vector(const odwf_t* h, int chirality, double* out) {
    if (!h || !out || (chirality != 1 && chirality != -1)) return ODWF_EINVAL;
    const int n = h->Ns;
    for (int s = 0; s < n; ++s) {
        const int e = chirality < 0 ? s : (n - 1 - s);
        out[s] = ((e & 1) ? -1.0 : 1.0) / std::sqrt(h->omega[s]);
    }
    return ODWF_OK;
}

}  // extern "C"

// ---- operator applies --------------------------------------------------------------------------
namespace odwf {

static int check_mass(odwf_s* h, double m) {
    if (!(m > 0.0 && m <= 1.0)) return set_err(h, ODWF_EINVAL, "masses must lie in (0, 1]");
    return ODWF_OK;
}

// out_p = A_p-block(own) - 1/2 H in_{1-p}, i.e. D_T (dagger: with transposed s-matrices and
// gamma_5 on both sides) for one output parity; storage of the fields: `stg`.
int apply_dt_parity(odwf_s* h, int stg, const SCoef* c, bool dag, int parity, const void* in_other,
                    const void* own, void* out, cudaStream_t st, const float* in_scale, const float* own_scale,
                    float* out_scale) {
    HopArgs a{};
    a.in = in_other;
    a.own = own;
    a.out = out;
    a.in_scale = in_scale;
    a.own_scale = own_scale;
    a.out_scale = out_scale;
    a.mown = c->dev + (size_t)(dag ? 4 : 0) * h->Ns * h->Ns;
    set_sop(a, c, dag ? (SOP_A | SOP_T) : SOP_A);
    a.c_hop = -0.5;
    a.g5 = dag ? (G5_HOP_IN | G5_OWN_IN | G5_OUT) : 0;
    return launch_hop(h, stg, parity, false, true, true, EPI_STORE, a, st);
}

static int apply_common(odwf_s* h, int op, double m1, double m2, const void* in, void* out, int prec, bool dag,
                        cudaStream_t st) {
    if (!h || !in || !out) return set_err(h, ODWF_EINVAL, "null argument");
    if (!h->have_gauge) return set_err(h, ODWF_EINVAL, "odwf_set_gauge has not been called");
    if (op != ODWF_OP_DT && op != ODWF_OP_HT && op != ODWF_OP_DODWF) return set_err(h, ODWF_EINVAL, "bad op");
    if (prec != ODWF_PREC_DOUBLE && prec != ODWF_PREC_SINGLE && prec != ODWF_PREC_HALF)
        return set_err(h, ODWF_EINVAL, "apply: prec must be DOUBLE, SINGLE or HALF");
    int rc;
    if ((rc = check_mass(h, m1)) || (rc = check_mass(h, m2))) return rc;
    const int stg = prec == ODWF_PREC_DOUBLE ? ST_DOUBLE : (prec == ODWF_PREC_SINGLE ? ST_FLOAT : ST_HALF);
    if ((rc = ensure_workspace(h, stg))) return rc;
    const SCoef* c = get_coef(h, m1, m2);
    if (!c) return ODWF_EINVAL;
    Workspace& w = h->ws;
    // FP64 / FP32 applies use the FP64-sized fields; FP16 storage uses the inner-solver fields, which
    // carry the per-(cb, s) scales
    void *ie = w.b_e, *io = w.b_o, *oe = w.x_e, *oo = w.x_o;
    float *ies = nullptr, *ios = nullptr, *oes = nullptr, *oos = nullptr;
    if (stg == ST_HALF) {
        ie = w.pi, io = w.ti, oe = w.xi, oo = w.ri;
        ies = w.pi_s, ios = w.ti_s, oes = w.xi_s, oos = w.ri_s;
    }
    if (op == ODWF_OP_DODWF) {
        // D_odwf = W D_T W N (N = omega^{1/2}(1 + L), W = omega^{1/2});  D_odwf^dag = N^T W D_T^dag W
        const double* pre = c->dev + (size_t)(dag ? 10 : 8) * h->Ns * h->Ns;
        const double* post = c->dev + (size_t)(dag ? 12 : 10) * h->Ns * h->Ns;
        if ((rc = launch_pack5(h, (const double*)in, oe, oo, stg, 0, st, oes, oos))) return rc;
        if ((rc = launch_smix(h, stg, oe, ie, pre, 1.0, st, oes, ies))) return rc;
        if ((rc = launch_smix(h, stg, oo, io, pre, 1.0, st, oos, ios))) return rc;
        if ((rc = apply_dt_parity(h, stg, c, dag, 0, io, ie, oe, st, ios, ies, oes))) return rc;
        if ((rc = apply_dt_parity(h, stg, c, dag, 1, ie, io, oo, st, ies, ios, oos))) return rc;
        if ((rc = launch_smix(h, stg, oe, ie, post, 1.0, st, oes, ies))) return rc;
        if ((rc = launch_smix(h, stg, oo, io, post, 1.0, st, oos, ios))) return rc;
        if ((rc = launch_unpack5(h, ie, io, (double*)out, stg, 0, st, ies, ios))) return rc;
        return check_fault(h, st);
    }
    // H_T = g5 R5 D_T ; H_T^dag = H_T. D_T^dag = g5 (D_T with transposed M) g5.
    // For H_T: out = g5 R5 D_T in  -> pack in plainly, unpack with R5 g5.
    // For H_T^dag = D_T^dag R5 g5: pack with R5 g5, apply D_T^dag, unpack plainly.
    const bool ht = (op == ODWF_OP_HT);
    const int pack_flag = (ht && dag) ? 1 : 0;
    const int unpack_flag = (ht && !dag) ? 1 : 0;
    if ((rc = launch_pack5(h, (const double*)in, ie, io, stg, pack_flag, st, ies, ios))) return rc;
    if ((rc = apply_dt_parity(h, stg, c, dag, 0, io, ie, oe, st, ios, ies, oes))) return rc;
    if ((rc = apply_dt_parity(h, stg, c, dag, 1, ie, io, oo, st, ies, ios, oos))) return rc;
    if ((rc = launch_unpack5(h, oe, oo, (double*)out, stg, unpack_flag, st, oes, oos))) return rc;
    return check_fault(h, st);
}

}  // namespace odwf

extern "C" {

int odwf_apply(odwf_t* h, int op, double m1, double m2, const void* in, void* out, int prec, void* stream) {
    return odwf::apply_common(h, op, m1, m2, in, out, prec, false, (cudaStream_t)stream);
}

int odwf_apply_dag(odwf_t* h, int op, double m1, double m2, const void* in, void* out, int prec, void* stream) {
    return odwf::apply_common(h, op, m1, m2, in, out, prec, true, (cudaStream_t)stream);
}

}  // extern "C"

// ---- kernel timing -----------------------------------------------------------------------------
namespace odwf {

static cudaEvent_t prof_event(odwf_s* h) {
    if (!h->prof_pool.empty()) {
        cudaEvent_t e = h->prof_pool.back();
        h->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(odwf_s* h, int, cudaStream_t st, cudaEvent_t* a) {
    *a = prof_event(h);
    cudaEventRecord(*a, st);
}

void prof_end(odwf_s* h, int key, cudaStream_t st, cudaEvent_t a) {
    cudaEvent_t b = prof_event(h);
    cudaEventRecord(b, st);
    h->prof_recs.push_back({key, a, b});
}

}  // namespace odwf

extern "C" int odwf_profile_enable(odwf_t* h, int enable) {
    if (!h) return ODWF_EINVAL;
    for (auto& r : h->prof_recs) {
        h->prof_pool.push_back(r.a);
        h->prof_pool.push_back(r.b);
    }
    h->prof_recs.clear();
    h->prof = enable != 0;
    return ODWF_OK;
}

extern "C" int odwf_profile_read(odwf_t* h, int* keys, int* launches, double* total_ms, int* n_io) {
    if (!h || !n_io) return ODWF_EINVAL;
    int rc = cuda_check(h, cudaDeviceSynchronize(), "profile sync");
    if (rc) return rc;
    std::map<int, std::pair<int, double>> acc;
    for (auto& r : h->prof_recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto& e = acc[r.key];
        e.first += 1;
        e.second += ms;
    }
    int i = 0;
    for (auto& kv : acc) {
        if (i < *n_io && keys && launches && total_ms) {
            keys[i] = kv.first;
            launches[i] = kv.second.first;
            total_ms[i] = kv.second.second;
        }
        ++i;
    }
    *n_io = i;
    return ODWF_OK;
}

// ---- mass-preconditioning term lists (Section 2) ----------------------------------------------
namespace {

// (m3, m4)/(m1, m2) with m1 == m3 (chirality -) or m2 == m4 (chirality +), Eq.(m1m2_m3m4)
bool make_term(double m3, double m4, double m1, double m2, eofa_term* t) {
    if (m1 == m3 && m2 != m4) {
        *t = eofa_term{-1, m3, m4, m2};
        return true;
    }
    if (m2 == m4 && m1 != m3) {
        *t = eofa_term{+1, m3, m4, m1};
        return true;
    }
    return false;
}

}  // namespace

extern "C" int eofa_mp_terms(int scheme, double m, const double* mh, int n_mh, double M, int parity,
                             eofa_term* out, int cap, int* n_out) {
    if (!n_out || (n_mh > 0 && !mh) || n_mh < 0) return ODWF_EINVAL;
    if (!(m > 0.0 && m < M && M <= 1.0)) return ODWF_EINVAL;
    std::vector<double> h(mh, mh + n_mh);
    for (int i = 0; i < n_mh; ++i) {
        if (!(h[i] > m && h[i] < M)) return ODWF_EINVAL;
        if (i > 0 && !(h[i] > h[i - 1])) return ODWF_EINVAL;
    }
    // factors as (numerator pair, denominator pair)
    std::vector<std::pair<std::pair<double, double>, std::pair<double, double>>> f;
    if (scheme == ODWF_MP_NONE) {
        if (n_mh != 0) return ODWF_EINVAL;
        f.push_back({{m, m}, {m, M}});
        f.push_back({{m, M}, {M, M}});
    } else if (scheme == ODWF_MP_OLD) {
        std::vector<double> ms;
        ms.push_back(m);
        for (double x : h) ms.push_back(x);
        ms.push_back(M);
        for (size_t i = 0; i + 1 < ms.size(); ++i) {
            const double a = ms[i], b = ms[i + 1];
            f.push_back({{a, a}, {a, b}});
            f.push_back({{a, b}, {b, b}});
        }
    } else if (scheme == ODWF_MP_NEW) {
        if (n_mh < 1) return ODWF_EINVAL;
        std::pair<double, double> cur{m, m}, nxt{m, h[0]};
        f.push_back({cur, nxt});
        cur = nxt;
        for (int i = 1; i <= n_mh; ++i) {
            const double target = i < n_mh ? h[i] : M;
            nxt = (i % 2 == 1) ? std::make_pair(target, cur.second) : std::make_pair(cur.first, target);
            f.push_back({cur, nxt});
            cur = nxt;
        }
        f.push_back({cur, {M, M}});
    } else {
        return ODWF_EINVAL;
    }
    int n = 0;
    for (auto& fr : f) {
        double m3 = fr.first.first, m4 = fr.first.second, m1 = fr.second.first, m2 = fr.second.second;
        if (parity) {
            std::swap(m3, m4);
            std::swap(m1, m2);
        }
        eofa_term t;
        if (!make_term(m3, m4, m1, m2, &t)) return ODWF_EINVAL;
        if (out && n < cap) out[n] = t;
        ++n;
    }
    *n_out = n;
    return ODWF_OK;
}

// ---- autotuning --------------------------------------------------------------------------------
namespace odwf {
int autotune_storage(odwf_s* h, int stg, const SCoef* c, cudaStream_t st, std::vector<std::string>& log);
}

extern "C" int odwf_autotune(odwf_t* h, int prec, char* report, int report_len, void* stream) {
    if (!h) return ODWF_EINVAL;
    if (prec != ODWF_PREC_DOUBLE && prec != ODWF_PREC_SINGLE && prec != ODWF_PREC_HALF)
        return set_err(h, ODWF_EINVAL, "autotune: bad precision");
    const int stg = prec == ODWF_PREC_DOUBLE ? ST_DOUBLE : (prec == ODWF_PREC_SINGLE ? ST_FLOAT : ST_HALF);
    int rc = ensure_workspace(h, stg);
    if (rc) return rc;
    const SCoef* c = get_coef(h, 0.5, 0.5);
    if (!c) return ODWF_EINVAL;
    std::vector<std::string> log;
    rc = autotune_storage(h, stg, c, (cudaStream_t)stream, log);
    if (report && report_len > 0) {
        // the chosen launches first: a short buffer keeps them and loses only timing lines
        std::string all, timings;
        for (auto& l : log) timings += l + "\n";
        for (auto& kv : h->tune) {
            char buf[128];
            std::snprintf(buf, sizeof buf, "chosen key %d: grid-mode %d staged %d tile x%d %s%s\n", kv.first,
                          kv.second.mode, kv.second.staged, kv.second.spbm, kv.second.dense ? "dense" : "structured",
                          kv.second.pair == 1 ? " two-slice" : (kv.second.pair >= 2 ? " two-slice bulk" : ""));
            all += buf;
        }
        all += timings;
        std::strncpy(report, all.c_str(), report_len - 1);
        report[report_len - 1] = 0;
    }
    return rc;
}

// ---- persisted autotuner choices ---------------------------------------------------------------
// One text line per (device, lattice, Ns, precision):
//   <device name>|<Lx>x<Ly>x<Lz>x<Lt>|<Ns>|<prec>|<kernel key>:<grid mode>:<staged>:<tile>:<dense>:<two-slice>,...
// (entries written before the last two fields existed read them as 0)
namespace {

std::string tune_key(const odwf_s* h, int prec) {
    int dev = 0;
    cudaDeviceProp prop{};
    std::string name = "unknown";
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char& ch : name)
        if (ch == '|' || ch == '\n') ch = '_';
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s|%dx%dx%dx%d|%d|%d", name.c_str(), h->L[0], h->L[1], h->L[2], h->L[3], h->Ns,
                  prec);
    return buf;
}

int tune_storage_of(int prec) { return prec == ODWF_PREC_DOUBLE ? ST_DOUBLE : (prec == ODWF_PREC_SINGLE ? ST_FLOAT : ST_HALF); }

}  // namespace

extern "C" int odwf_autotune_cache(odwf_t* h, int prec, const char* path, int* hit, void* stream) {
    if (!h || !path || !hit) return set_err(h, ODWF_EINVAL, "null argument");
    if (prec != ODWF_PREC_DOUBLE && prec != ODWF_PREC_SINGLE && prec != ODWF_PREC_HALF)
        return set_err(h, ODWF_EINVAL, "autotune: bad precision");
    *hit = 0;
    const std::string key = tune_key(h, prec);
    const int stg = tune_storage_of(prec);
    if (FILE* f = std::fopen(path, "r")) {
        char line[4096];
        std::string found;
        while (std::fgets(line, sizeof line, f)) {
            std::string l(line);
            while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
            if (l.size() > key.size() && l.compare(0, key.size(), key) == 0 && l[key.size()] == '|')
                found = l.substr(key.size() + 1);  // the last entry for the key wins
        }
        std::fclose(f);
        if (!found.empty()) {
            std::map<int, TuneChoice> parsed;
            size_t pos = 0;
            bool bad = false;
            while (pos < found.size()) {
                size_t end = found.find(',', pos);
                if (end == std::string::npos) end = found.size();
                int k = 0;
                TuneChoice tc;
                const int nf = std::sscanf(found.substr(pos, end - pos).c_str(), "%d:%d:%d:%d:%d:%d", &k, &tc.mode, &tc.staged,
                                           &tc.spbm, &tc.dense, &tc.pair);
                if (nf < 4 || tc.mode < 0 || tc.mode > 3 || tc.staged < 0 || tc.staged > 1 || tc.spbm < 1 ||
                    tc.spbm > 2 || tc.dense < 0 || tc.dense > 1 || tc.pair < 0 || tc.pair > 3 ||
                    (k / 100000) % 10 != stg) {
                    bad = true;
                    break;
                }
                parsed[k] = tc;
                pos = end + 1;
            }
            if (!bad && !parsed.empty()) {
                for (auto& kv : parsed) h->tune[kv.first] = kv.second;
                *hit = 1;
                return ODWF_OK;
            }
        }
    }
    int rc = odwf_autotune(h, prec, nullptr, 0, stream);
    if (rc) return rc;
    std::string entry = key + "|";
    bool first = true;
    for (auto& kv : h->tune) {
        if ((kv.first / 100000) % 10 != stg) continue;
        char buf[64];
        std::snprintf(buf, sizeof buf, "%s%d:%d:%d:%d:%d:%d", first ? "" : ",", kv.first, kv.second.mode,
                      kv.second.staged, kv.second.spbm, kv.second.dense, kv.second.pair);
        entry += buf;
        first = false;
    }
    FILE* f = std::fopen(path, "a");
    if (!f) return set_err(h, ODWF_EINVAL, std::string("cannot append to the autotuner cache ") + path);
    std::fprintf(f, "%s\n", entry.c_str());
    std::fclose(f);
    return ODWF_OK;
}
