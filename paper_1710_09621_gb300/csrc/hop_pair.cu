// Fused hopping kernels with two fifth-dimension slices per thread: FP32 and FP16 storage, Ns = 16, the
// structured fifth-dimension products (A or A^{-1} of Eq.(DTm1m2)'s s-local part by their O(Ns) recurrences).
//
// The Wilson hop is diagonal in s, so the Ns slices of a site multiply the same eight links. In the
// one-slice kernels (kernels.cu) each of a site's 16 threads loads every link: a broadcast load still
// writes the link into every lane's registers, so the data pipe of L1 moves 16 copies of each link per
// site. Here a site has 8 threads, thread k holding slices k and k + 8 (one load instruction then still
// reads 8 consecutive 16-byte vectors per site), and each link is stored as its first two rows, 12 floats
// in three 16-byte vectors: for V in SU(3) the third row is the complex conjugate of the cross product of
// the first two (V^{-1} = V^dag and det V = 1 make row 2 the conjugated cofactors of rows 0 and 1). The
// stored matrix is the link without the antiperiodic boundary sign, which the neighbour table carries
// instead (the complemented index). Per slice the link writebacks fall from 5 vectors x 16 lanes to
// 3 x 8 per site and direction.
//
// The fifth-dimension pass keeps the layout of the one-slice structured kernels: after the hop each thread
// stages its two rows in shared memory, then thread k takes three real columns of all 16 rows (reals
// 3k .. 3k + 2: k < 4 the P_+ components, k >= 4 the P_- ones; the coefficients are real, so real and
// imaginary parts follow one recurrence), and every thread reads its rows back. All 32 lanes take part in
// the column pass (12 of 16 in the one-slice kernels).
#include <type_traits>

#include "hop_common.cuh"

namespace odwf {

constexpr int kPairLanes = kStructNs / 2;            // threads per site
constexpr int kPRow = 28;                            // floats per staged row (16-byte row stores of 8 lanes
                                                     // on 8 distinct 4-bank groups)
constexpr int kPSite = kStructNs * kPRow + 8;        // site stride 456 = 8 (mod 32) words: the column loads
                                                     // of the 4 sites of a warp (lanes at 3k) hit 32 banks
constexpr int kPairSites = 16;                       // sites per CTA at tile x1 (128 threads)

// one direction mu (forward and backward) of the hop for the thread's two slices
template <int ST, int MU>
__device__ __forceinline__ void pair_dir(const HopArgs& a, const int* n, int cb, int s0, float* v0, float* v1,
                                         bool g5in) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        int nb = n[b * 4 + MU];
        float sg = 1.f;
        if (MU == 3) {  // only t links cross the antiperiodic boundary
            sg = nb < 0 ? -1.f : 1.f;
            nb = nb < 0 ? ~nb : nb;
        }
        float p0[24], p1[24], h[12], w[12], u[18];
        Store<ST>::load(a.in, a.in_scale, (size_t)nb, s0, a.Ns, p0);
        Store<ST>::load(a.in, a.in_scale, (size_t)nb, s0 + kPairLanes, a.Ns, p1);
        link12_load(a.links12, cb, b * 4 + MU, u);
        if (MU == 3) {
#pragma unroll
            for (int i = 0; i < 18; ++i) u[i] *= sg;
        }
        if (g5in) {
            g5_flip(p0);
            g5_flip(p1);
        }
        // forward (b = 0): (1 - gamma_mu) U_mu(x) psi(x + mu); backward: (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu)
        if (b == 0) {
            project<MU, -1>(p0, h);
            su3_mul_half(u, h, w);
            reconstruct<MU, -1>(v0, w);
            project<MU, -1>(p1, h);
            su3_mul_half(u, h, w);
            reconstruct<MU, -1>(v1, w);
        } else {
            project<MU, +1>(p0, h);
            su3_mul_half(u, h, w);
            reconstruct<MU, +1>(v0, w);
            project<MU, +1>(p1, h);
            su3_mul_half(u, h, w);
            reconstruct<MU, +1>(v1, w);
        }
    }
}

// A^{-1} = W (1 + L) B^{-1} W and A = (4 - m0 - 1/omega) + 2 W^{-1} (1 + L)^{-1} W^{-1} on NC real columns
// in recurrence order: the same steps as s_ainv_col / s_a_col (field_access.cuh), column by column.
template <int N, int NC>
__device__ __forceinline__ void s_ainv_cols(const SStructT<float>& k, int c, float (&x)[NC][N]) {
    const float me0 = c ? k.me0[1] : k.me0[0], cu = c ? k.cu[1] : k.cu[0], m = c ? k.m[1] : k.m[0];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const float z0 = k.w[0] * x[j][0];
        x[j][0] = 0.f;
#pragma unroll
        for (int s = 1; s < N; ++s) x[j][s] = fmaf(-k.f[s], x[j][s - 1], k.rw[s] * x[j][s]);
        const float u = cu * fmaf(me0, x[j][N - 1], z0);
#pragma unroll
        for (int s = 0; s < N; ++s) x[j][s] = fmaf(k.q[s], u, x[j][s]);
        const float yl = x[j][N - 1];
#pragma unroll
        for (int s = N - 1; s >= 1; --s) x[j][s] = k.w[s] * (x[j][s] + x[j][s - 1]);
        x[j][0] = k.w[0] * fmaf(-m, yl, x[j][0]);
    }
}

template <int N, int NC>
__device__ __forceinline__ void s_a_cols(const SStructT<float>& k, int c, float (&x)[NC][N]) {
    const float m = c ? k.m[1] : k.m[0], au = c ? k.au[1] : k.au[0];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const float z0 = k.wi[0] * x[j][0];
        float p = 0.f;
        x[j][0] = k.adiag[0] * x[j][0];
#pragma unroll
        for (int s = 1; s < N; ++s) {
            p = fmaf(k.wi[s], x[j][s], -p);
            x[j][s] = fmaf(k.wi[s], p + p, k.adiag[s] * x[j][s]);
        }
        const float u = au * fmaf(m, p, z0);
#pragma unroll
        for (int s = 0; s < N; ++s) x[j][s] = fmaf(k.wi2s[s], u, x[j][s]);
    }
}

// column pass of thread k over its site's 16 staged rows (reals 3k .. 3k + 2 of every row), from the rows
// at src to those at dst (the same rows, or a second copy that leaves the input rows in place)
__device__ __forceinline__ void pair_col(const SStruct& sc, int sop, const float* src, float* dst, int k) {
    constexpr int N = kStructNs;
    const int c = k < kPairLanes / 2 ? 0 : 1;
    const bool rev = (c == 1) != ((sop & SOP_T) != 0);
    const float* p0 = src + 3 * k;
    float* d0 = dst + 3 * k;
    float x[3][N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
#pragma unroll
        for (int j = 0; j < 3; ++j) x[j][q] = p0[q * kPRow + j];
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) col_reverse<float, N>(rev, x[j]);
    if ((sop & 3) == SOP_AINV) s_ainv_cols<N, 3>(sc.f, c, x);
    else s_a_cols<N, 3>(sc.f, c, x);
#pragma unroll
    for (int j = 0; j < 3; ++j) col_reverse<float, N>(rev, x[j]);
#pragma unroll
    for (int q = 0; q < N; ++q) {
#pragma unroll
        for (int j = 0; j < 3; ++j) d0[q * kPRow + j] = x[j][q];
    }
}

// The operator of hop_body (kernels.cu) for one output parity, two slices per thread:
//   v = c_hop H(in); [v += a_own own]; v = Mhop v (MIXHOP) or v += Mown own (MIXOWN); [gamma_5]; epilogue.
// A site's 8 threads are consecutive lanes of one warp and only they touch its staged rows, so warp
// barriers order the row and column accesses. With MIXOWN the own rows stay staged (the column pass
// writes a second set of rows) and the epilogue reads its own-field rows from there instead of keeping
// them in registers through the hop and the column pass.
template <int ST, bool MIXHOP, bool OWN, bool MIXOWN, int EPI>
__device__ __forceinline__ void pair_body(const HopArgs& a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* sh = reinterpret_cast<float*>(smem_raw);
    const int k = threadIdx.x, ls = threadIdx.y, spb = blockDim.y;
    const int s0 = k, s1 = k + kPairLanes;
    if (a.state != nullptr && EPI != EPI_STORE_NORM && EPI != EPI_RESID) {
        if (((volatile CGState*)a.state)->flag != FLAG_RUN) return;
    }
    double alpha = 0.0, beta = 0.0;
    if (EPI == EPI_CG_A) alpha = a.state->alpha;
    if (EPI == EPI_CG_B) beta = a.state->beta;
    const bool g5h = (a.g5 & G5_HOP_IN) != 0, g5o = (a.g5 & G5_OWN_IN) != 0, g5out = (a.g5 & G5_OUT) != 0;
    const float chop = (float)a.c_hop, aown = (float)a.a_own;
    double part = 0.0;
    constexpr int NSET = MIXOWN ? 2 : 1;  // row sets per site
    float* site = sh + ls * NSET * kPSite;
    float* mixed = site + (NSET - 1) * kPSite;  // MIXOWN: the column pass's output rows
    float* row0 = site + s0 * kPRow;
    float* row1 = site + s1 * kPRow;

    for (int g = blockIdx.x; g * spb < a.Vh; g += gridDim.x) {
        __syncwarp();
        const int cb = g * spb + ls;
        const bool valid = cb < a.Vh;
        float v0[24], v1[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) v0[i] = v1[i] = 0.f;
        if (valid) {
            int n[8];
            const int4* nb = reinterpret_cast<const int4*>(a.nbrs + (size_t)cb * 8);
            const int4 n0 = __ldg(nb), n1 = __ldg(nb + 1);
            n[0] = n0.x; n[1] = n0.y; n[2] = n0.z; n[3] = n0.w;
            n[4] = n1.x; n[5] = n1.y; n[6] = n1.z; n[7] = n1.w;
            pair_dir<ST, 0>(a, n, cb, s0, v0, v1, g5h);
            pair_dir<ST, 1>(a, n, cb, s0, v0, v1, g5h);
            pair_dir<ST, 2>(a, n, cb, s0, v0, v1, g5h);
            pair_dir<ST, 3>(a, n, cb, s0, v0, v1, g5h);
#pragma unroll
            for (int i = 0; i < 24; ++i) {
                v0[i] *= chop;
                v1[i] *= chop;
            }
        }
        float ow0[24], ow1[24];
        if (OWN) {
            if (valid) {
                Store<ST>::load(a.own, a.own_scale, (size_t)cb, s0, a.Ns, ow0);
                Store<ST>::load(a.own, a.own_scale, (size_t)cb, s1, a.Ns, ow1);
                if (g5o) {
                    g5_flip(ow0);
                    g5_flip(ow1);
                }
            } else {
#pragma unroll
                for (int i = 0; i < 24; ++i) ow0[i] = ow1[i] = 0.f;
            }
            if (!MIXOWN) {
#pragma unroll
                for (int i = 0; i < 24; ++i) {
                    v0[i] = fmaf(aown, ow0[i], v0[i]);
                    v1[i] = fmaf(aown, ow1[i], v1[i]);
                }
            }
        }
        if (MIXHOP) {
            row24_store(row0, v0);
            row24_store(row1, v1);
            __syncwarp();
            pair_col(a.sc, a.sop, site, site, k);
            __syncwarp();
            row24_load(row0, v0, false);
            row24_load(row1, v1, false);
        }
        if (MIXOWN) {
            row24_store(row0, ow0);
            row24_store(row1, ow1);
            __syncwarp();
            pair_col(a.sc, a.sop, site, mixed, k);
            __syncwarp();
            row24_load(mixed + s0 * kPRow, v0, true);
            row24_load(mixed + s1 * kPRow, v1, true);
        }
        if (g5out) {
            g5_flip(v0);
            g5_flip(v1);
        }
        if (!valid) continue;
        if (MIXOWN) {  // the own field's rows, as loaded (after gamma_5 where asked)
            float ow[24];
            row24_load(row0, ow, false);
            epilogue<ST, EPI>(a, cb, s0, v0, ow, alpha, beta, part);
            row24_load(row1, ow, false);
            epilogue<ST, EPI>(a, cb, s1, v1, ow, alpha, beta, part);
        } else {
            epilogue<ST, EPI>(a, cb, s0, v0, ow0, alpha, beta, part);
            epilogue<ST, EPI>(a, cb, s1, v1, ow1, alpha, beta, part);
        }
    }
    if (EPI != EPI_STORE) grid_finalize<EPI>(a, part);
}

template <int ST, bool MIXHOP, bool OWN, bool MIXOWN, int EPI>
__global__ void __launch_bounds__(256, 2) k_hop_pair(HopArgs a) {
    pair_body<ST, MIXHOP, OWN, MIXOWN, EPI>(a);
}

// ---- two-slice kernels with the neighbour gathers pipelined through bulk copies (FP32 storage) ------
// A neighbour site's 16 slices are one contiguous run of the FP32 field (chunk-major, slice-minor: 1536
// bytes) and its two-row link 48 contiguous bytes. Thread 0 of each site requests both for one leg (a
// direction and orientation) with two bulk copies into a stage buffer, completed on the site's mbarrier of
// that stage, NST - 1 legs ahead of the leg that the site's 8 threads compute from shared memory. The
// copies run on the tensor memory accelerator and hold no registers, so NST - 1 legs of every site stay in
// flight while a third is computed; in the register-gather kernels a thread has one leg in flight and then
// waits. Every wait is bounded: a wait that runs out sets the fault word and a CTA flag after which no
// thread waits or issues again, and the issuing threads wait (bounded) for their copies still in flight
// before the CTA exits. The column-pass rows alias the stage buffers once all sites of the CTA have
// finished their legs (CTA barrier).
constexpr int kSiteBytes = 6 * kStructNs * 16;   // one site's 16 slices, FP32
constexpr int kLinkBytes = 48;                   // one two-row link

__host__ __device__ constexpr int pair_tma_region(int nst, int nset) {
    return nst * kPairSites * (kSiteBytes + kLinkBytes) > nset * kPairSites * kPSite * 4
               ? nst * kPairSites * (kSiteBytes + kLinkBytes)
               : nset * kPairSites * kPSite * 4;
}
__host__ __device__ constexpr int pair_tma_smem(int nst, int nset) {
    return pair_tma_region(nst, nset) + nst * kPairSites * 8 + 16;
}

// one leg from the staged neighbour (sp: the site's 1536 bytes) and link (lk: 48 bytes)
template <int MU, int B>
__device__ __forceinline__ void pair_leg_smem(const float4* sp, const float4* lk, float sg, int s0, bool g5in,
                                              float* v0, float* v1) {
    float u[18], p[24], h[12], w[12];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float4 c = lk[q];
        u[4 * q] = c.x, u[4 * q + 1] = c.y, u[4 * q + 2] = c.z, u[4 * q + 3] = c.w;
    }
    link12_complete(u);
    if (MU == 3) {
#pragma unroll
        for (int i = 0; i < 18; ++i) u[i] *= sg;
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int s = s0 + t * kPairLanes;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const float4 c = sp[j * kStructNs + s];
            p[4 * j] = c.x, p[4 * j + 1] = c.y, p[4 * j + 2] = c.z, p[4 * j + 3] = c.w;
        }
        if (g5in) g5_flip(p);
        project<MU, B ? +1 : -1>(p, h);
        su3_mul_half(u, h, w);
        reconstruct<MU, B ? +1 : -1>(t ? v1 : v0, w);
    }
}

template <bool MIXHOP, bool OWN, bool MIXOWN, int EPI, int NST>
__device__ __forceinline__ void pair_tma_body(const HopArgs& a) {
    constexpr int ST = ST_FLOAT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int k = threadIdx.x, ls = threadIdx.y;  // blockDim.y == kPairSites
    constexpr int spb = kPairSites;
    const int s0 = k, s1 = k + kPairLanes;
    constexpr int NSET = MIXOWN ? 2 : 1;
    unsigned char* sbuf = smem_raw;
    unsigned char* lbuf = sbuf + (size_t)NST * spb * kSiteBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + pair_tma_region(NST, NSET));
    volatile int* fail_s = reinterpret_cast<volatile int*>(bars + NST * spb);
    float* sh = reinterpret_cast<float*>(smem_raw);
    if (a.state != nullptr && EPI != EPI_STORE_NORM && EPI != EPI_RESID) {
        if (((volatile CGState*)a.state)->flag != FLAG_RUN) return;
    }
    if (k == 0) {
#pragma unroll
        for (int st = 0; st < NST; ++st) mbar_init(&bars[st * spb + ls]);
    }
    if (k == 0 && ls == 0) *fail_s = 0;
    __syncthreads();
    double alpha = 0.0, beta = 0.0;
    if (EPI == EPI_CG_A) alpha = a.state->alpha;
    if (EPI == EPI_CG_B) beta = a.state->beta;
    const bool g5h = (a.g5 & G5_HOP_IN) != 0, g5o = (a.g5 & G5_OWN_IN) != 0, g5out = (a.g5 & G5_OUT) != 0;
    const float chop = (float)a.c_hop, aown = (float)a.a_own;
    double part = 0.0;
    float* site = sh + ls * NSET * kPSite;
    float* mixed = site + (NSET - 1) * kPSite;
    float* row0 = site + s0 * kPRow;
    float* row1 = site + s1 * kPRow;
    const char* inb = reinterpret_cast<const char*>(a.in);
    const char* lkb = reinterpret_cast<const char*>(a.links12);
    uint32_t phase = 0;        // bit st: parity of the next completion of this site slot's stage st
    uint32_t outstanding = 0;  // issuing thread: stages whose last copy it has not seen complete
    uint32_t out_par = 0;      // issuing thread: the parity those copies complete with

    for (int g = blockIdx.x; g * spb < a.Vh; g += gridDim.x) {
        __syncthreads();  // the previous group's rows (aliasing the stage buffers) have been read
        const int cb = g * spb + ls;
        const bool valid = cb < a.Vh;
        int n[8];
        if (valid) {
            const int4* nb = reinterpret_cast<const int4*>(a.nbrs + (size_t)cb * 8);
            const int4 n0 = __ldg(nb), n1 = __ldg(nb + 1);
            n[0] = n0.x; n[1] = n0.y; n[2] = n0.z; n[3] = n0.w;
            n[4] = n1.x; n[5] = n1.y; n[6] = n1.z; n[7] = n1.w;
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) n[i] = 0;
        }
        auto issue = [&](int L) {
            const int st = L % NST, mu = L >> 1, b = L & 1;
            int nb = n[b * 4 + mu];
            nb = nb < 0 ? ~nb : nb;
            uint64_t* bar = &bars[st * spb + ls];
            fence_proxy_async_cta();
            mbar_expect(bar, kSiteBytes + kLinkBytes);
            bulk_copy(sbuf + (size_t)(st * spb + ls) * kSiteBytes, inb + (size_t)nb * kSiteBytes, kSiteBytes, bar);
            bulk_copy(lbuf + (size_t)(st * spb + ls) * kLinkBytes, lkb + ((size_t)cb * 8 + b * 4 + mu) * kLinkBytes,
                      kLinkBytes, bar);
            outstanding |= 1u << st;
            out_par = (out_par & ~(1u << st)) | (phase & (1u << st));
        };
        if (k == 0 && valid && !*fail_s) {
#pragma unroll
            for (int L = 0; L < NST - 1; ++L) issue(L);
        }
        float v0[24], v1[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) v0[i] = v1[i] = 0.f;
        // leg L: wait for its stage, compute from shared memory; first hand the stage freed by leg L - 1
        // to leg L + NST - 1 (after the site's threads have all read it)
        auto leg = [&](auto mu_c, auto b_c, int L) {
            constexpr int MU = decltype(mu_c)::value, B = decltype(b_c)::value;
            if (L + NST - 1 < 8) {
                __syncwarp();
                if (k == 0 && valid && !*fail_s) issue(L + NST - 1);
            }
            const int st = L % NST;
            if (valid) {
                bool ok = false;
                if (!*fail_s) {
                    ok = mbar_wait_bounded(&bars[st * spb + ls], (phase >> st) & 1u, a.wait_cycles);
                    if (!ok) {
                        *fail_s = 1;
                        if (a.fault) atomicOr(a.fault, 1u);
                    }
                }
                phase ^= 1u << st;
                if (ok && k == 0) outstanding &= ~(1u << st);
                const float sg = (MU == 3 && n[B * 4 + MU] < 0) ? -1.f : 1.f;
                pair_leg_smem<MU, B>(reinterpret_cast<const float4*>(sbuf + (size_t)(st * spb + ls) * kSiteBytes),
                                     reinterpret_cast<const float4*>(lbuf + (size_t)(st * spb + ls) * kLinkBytes), sg,
                                     s0, g5h, v0, v1);
            }
        };
        leg(std::integral_constant<int, 0>{}, std::integral_constant<int, 0>{}, 0);
        leg(std::integral_constant<int, 0>{}, std::integral_constant<int, 1>{}, 1);
        leg(std::integral_constant<int, 1>{}, std::integral_constant<int, 0>{}, 2);
        leg(std::integral_constant<int, 1>{}, std::integral_constant<int, 1>{}, 3);
        leg(std::integral_constant<int, 2>{}, std::integral_constant<int, 0>{}, 4);
        leg(std::integral_constant<int, 2>{}, std::integral_constant<int, 1>{}, 5);
        leg(std::integral_constant<int, 3>{}, std::integral_constant<int, 0>{}, 6);
        leg(std::integral_constant<int, 3>{}, std::integral_constant<int, 1>{}, 7);
#pragma unroll
        for (int i = 0; i < 24; ++i) {
            v0[i] *= chop;
            v1[i] *= chop;
        }
        __syncthreads();  // every site of the CTA is done with the stage buffers: the rows may alias them
        float ow0[24], ow1[24];
        if (OWN) {
            if (valid) {
                Store<ST>::load(a.own, a.own_scale, (size_t)cb, s0, a.Ns, ow0);
                Store<ST>::load(a.own, a.own_scale, (size_t)cb, s1, a.Ns, ow1);
                if (g5o) {
                    g5_flip(ow0);
                    g5_flip(ow1);
                }
            } else {
#pragma unroll
                for (int i = 0; i < 24; ++i) ow0[i] = ow1[i] = 0.f;
            }
            if (!MIXOWN) {
#pragma unroll
                for (int i = 0; i < 24; ++i) {
                    v0[i] = fmaf(aown, ow0[i], v0[i]);
                    v1[i] = fmaf(aown, ow1[i], v1[i]);
                }
            }
        }
        if (MIXHOP) {
            row24_store(row0, v0);
            row24_store(row1, v1);
            __syncwarp();
            pair_col(a.sc, a.sop, site, site, k);
            __syncwarp();
            row24_load(row0, v0, false);
            row24_load(row1, v1, false);
        }
        if (MIXOWN) {
            row24_store(row0, ow0);
            row24_store(row1, ow1);
            __syncwarp();
            pair_col(a.sc, a.sop, site, mixed, k);
            __syncwarp();
            row24_load(mixed + s0 * kPRow, v0, true);
            row24_load(mixed + s1 * kPRow, v1, true);
        }
        if (g5out) {
            g5_flip(v0);
            g5_flip(v1);
        }
        if (!valid) continue;
        if (MIXOWN) {
            float ow[24];
            row24_load(row0, ow, false);
            epilogue<ST, EPI>(a, cb, s0, v0, ow, alpha, beta, part);
            row24_load(row1, ow, false);
            epilogue<ST, EPI>(a, cb, s1, v1, ow, alpha, beta, part);
        } else {
            epilogue<ST, EPI>(a, cb, s0, v0, ow0, alpha, beta, part);
            epilogue<ST, EPI>(a, cb, s1, v1, ow1, alpha, beta, part);
        }
    }
    // copies whose completion a timed-out wait did not see must land before the CTA's shared memory is
    // released
    if (k == 0 && outstanding) {
#pragma unroll
        for (int st = 0; st < NST; ++st)
            if (outstanding & (1u << st)) mbar_wait_bounded(&bars[st * spb + ls], (out_par >> st) & 1u, 0);
    }
    if (EPI != EPI_STORE) grid_finalize<EPI>(a, part);
}

template <bool MIXHOP, bool OWN, bool MIXOWN, int EPI, int NST>
__global__ void __launch_bounds__(128, 3) k_hop_pair_tma(HopArgs a) {
    pair_tma_body<MIXHOP, OWN, MIXOWN, EPI, NST>(a);
}

// variants with a two-slice kernel: the fused kernels of the CGNE iteration (K1 = A^{-1} after the hop,
// K2A / K2B / K2 = A on the own field plus the hop)
bool pair_variant(int storage, bool mixhop, bool own, bool mixown, int epi) {
    if (storage != ST_FLOAT && storage != ST_HALF) return false;
    if (mixhop && !own && !mixown && epi == EPI_STORE) return true;
    if (!mixhop && own && mixown && (epi == EPI_STORE || epi == EPI_CG_A || epi == EPI_CG_B)) return true;
    return false;
}

bool pair_applies(const odwf_s* h, int storage, const HopArgs& a) {
    return h->Ns == kStructNs && h->links12_ok && a.sop != SOP_DENSE && (storage == ST_FLOAT || storage == ST_HALF);
}

template <int ST, bool MIXHOP, bool OWN, bool MIXOWN, int EPI>
static int launch_pair_t(odwf_s* h, const HopArgs& a, int mode, int spbm, cudaStream_t st) {
    const void* fn = (const void*)k_hop_pair<ST, MIXHOP, OWN, MIXOWN, EPI>;
    const int spb = kPairSites * (spbm > 1 ? 2 : 1);
    const size_t smem = sizeof(float) * (size_t)spb * kPSite * (MIXOWN ? 2 : 1);
    static int occ_cache[2] = {0, 0};
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    int& occ = occ_cache[spb == kPairSites ? 0 : 1];
    if (occ == 0) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, kPairLanes * spb, smem) != cudaSuccess || o < 1) o = 1;
        occ = o;
    }
    const int groups = (a.Vh + spb - 1) / spb;
    const int grid = grid_for_mode(h, mode, occ, groups, EPI != EPI_STORE);
    k_hop_pair<ST, MIXHOP, OWN, MIXOWN, EPI><<<grid, dim3(kPairLanes, spb), smem, st>>>(a);
    return cuda_check(h, cudaGetLastError(), "k_hop_pair launch");
}

template <bool MIXHOP, bool OWN, bool MIXOWN, int EPI, int NST>
static int launch_pair_tma_t(odwf_s* h, const HopArgs& a, int mode, cudaStream_t st) {
    const void* fn = (const void*)k_hop_pair_tma<MIXHOP, OWN, MIXOWN, EPI, NST>;
    constexpr int smem = pair_tma_smem(NST, MIXOWN ? 2 : 1);
    static int occ = 0;
    if (occ == 0) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, kPairLanes * kPairSites, smem) != cudaSuccess || o < 1)
            o = 1;
        occ = o;
    }
    const int groups = (a.Vh + kPairSites - 1) / kPairSites;
    const int grid = grid_for_mode(h, mode, occ, groups, EPI != EPI_STORE);
    h->staged_used = true;  // its waits are bounded and report through the fault word
    k_hop_pair_tma<MIXHOP, OWN, MIXOWN, EPI, NST><<<grid, dim3(kPairLanes, kPairSites), smem, st>>>(a);
    return cuda_check(h, cudaGetLastError(), "k_hop_pair_tma launch");
}

template <int NST>
static int launch_pair_tma(odwf_s* h, bool mixhop, bool own, bool mixown, int epi, const HopArgs& a, int mode,
                           cudaStream_t st) {
    if (mixhop && !own && !mixown && epi == EPI_STORE)
        return launch_pair_tma_t<true, false, false, EPI_STORE, NST>(h, a, mode, st);
    if (!mixhop && own && mixown) {
        if (epi == EPI_STORE) return launch_pair_tma_t<false, true, true, EPI_STORE, NST>(h, a, mode, st);
        if (epi == EPI_CG_A) return launch_pair_tma_t<false, true, true, EPI_CG_A, NST>(h, a, mode, st);
        if (epi == EPI_CG_B) return launch_pair_tma_t<false, true, true, EPI_CG_B, NST>(h, a, mode, st);
    }
    return set_err(h, ODWF_EINVAL, "no two-slice kernel for this hop variant");
}

template <int ST>
static int launch_pair_st(odwf_s* h, bool mixhop, bool own, bool mixown, int epi, const HopArgs& a, int mode,
                          int spbm, cudaStream_t st) {
    if (mixhop && !own && !mixown && epi == EPI_STORE)
        return launch_pair_t<ST, true, false, false, EPI_STORE>(h, a, mode, spbm, st);
    if (!mixhop && own && mixown) {
        if (epi == EPI_STORE) return launch_pair_t<ST, false, true, true, EPI_STORE>(h, a, mode, spbm, st);
        if (epi == EPI_CG_A) return launch_pair_t<ST, false, true, true, EPI_CG_A>(h, a, mode, spbm, st);
        if (epi == EPI_CG_B) return launch_pair_t<ST, false, true, true, EPI_CG_B>(h, a, mode, spbm, st);
    }
    return set_err(h, ODWF_EINVAL, "no two-slice kernel for this hop variant");
}

// the bulk-copy pipeline needs FP32 storage and 16-byte aligned fields and links (bulk copies move whole
// 16-byte units between 16-byte aligned addresses)
bool pair_tma_applies(int storage, const HopArgs& a) {
    return storage == ST_FLOAT && ((uintptr_t)a.in % 16) == 0 && ((uintptr_t)a.links12 % 16) == 0;
}

int launch_hop_pair(odwf_s* h, int storage, bool mixhop, bool own, bool mixown, int epi, const HopArgs& a,
                    int mode, int spbm, cudaStream_t st, int form) {
    if (form >= 2 && pair_tma_applies(storage, a)) {
        if (form == 2) return launch_pair_tma<2>(h, mixhop, own, mixown, epi, a, mode, st);
        return launch_pair_tma<3>(h, mixhop, own, mixown, epi, a, mode, st);
    }
    if (storage == ST_FLOAT) return launch_pair_st<ST_FLOAT>(h, mixhop, own, mixown, epi, a, mode, spbm, st);
    if (storage == ST_HALF) return launch_pair_st<ST_HALF>(h, mixhop, own, mixown, epi, a, mode, spbm, st);
    return set_err(h, ODWF_EINVAL, "no two-slice kernel for FP64 storage");
}

}  // namespace odwf
