// Hopping (dslash) kernels of D_T(m1, m2) and the even-odd Schur complement, plus layout and
// BLAS-1 kernels.
//
// Operator (Eq.(DTm1m2), read with c = 1, d = 0):
//   D_T(m1, m2) = D_w(-m0) + P_+ M_+(m1) + P_- M_-(m2),
//   D_w(-m0)    = (4 - m0) - 1/2 H,
//   H psi(x)    = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu^dag(x-mu) psi(x-mu).
// The hop H is diagonal in s, so one gauge link serves all Ns slices of a site. Each CTA owns all
// Ns slices of `spb` checkerboard sites (threadIdx.x = s, threadIdx.y = site), which lets the
// fifth-dimension part (a dense Ns x Ns matrix per chirality, applied to the hop sum or to the
// own-site field) be fused into the same pass through shared memory.
//
// Spin projection in the chiral basis gamma_5 = diag(1,1,-1,-1), gamma_mu = [[0, B_mu],[C_mu, 0]]
// with C_mu = B_mu^dag unitary: (1 -/+ gamma_mu) psi = [h; -/+ C h], h = psi_up -/+ B psi_dn, so each
// direction multiplies one 2-spin half spinor by U.
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "hop_common.cuh"

namespace odwf {

int spb_for(int Ns);

template <int ST, int MU>
__device__ __forceinline__ void hop_dir(const HopArgs& a, const int* n, int cb, int s,
                                        typename Store<ST>::R* v, bool g5in) {
    using R = typename Store<ST>::R;
    R psi[24], h[12], w[12], u[18];
    // forward: (1 - gamma_mu) U_mu(x) psi(x + mu)
    Store<ST>::load(a.in, a.in_scale, (size_t)n[MU], s, a.Ns, psi);
    if (g5in) g5_flip(psi);
    project<MU, -1>(psi, h);
    Links<ST>::load(a.links, cb, MU, u);
    su3_mul_half(u, h, w);
    reconstruct<MU, -1>(v, w);
    // backward: (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu); the stored link is already daggered
    Store<ST>::load(a.in, a.in_scale, (size_t)n[4 + MU], s, a.Ns, psi);
    if (g5in) g5_flip(psi);
    project<MU, +1>(psi, h);
    Links<ST>::load(a.links, cb, 4 + MU, u);
    su3_mul_half(u, h, w);
    reconstruct<MU, +1>(v, w);
}


// Barrier over the threads that share staged rows: the whole CTA, or just the warp when every site
// lies inside one warp (WS: Ns divides 32, so a site's Ns threads are consecutive lanes of one warp
// and only they write and read its rows).
template <bool WS>
__device__ __forceinline__ void site_barrier() {
    if constexpr (WS) __syncwarp();
    else __syncthreads();
}

// FP32 K1 (hop then mix, no own field): register-capped FMA variant (true) or the uncapped variant
// with the tensor-core s-mixing (false)
constexpr bool kLeanK1 = true;
template <int ST, bool HOP, bool MIXHOP, bool OWN, bool MIXOWN>
constexpr bool kLeanHop = kLeanK1 && ST == ST_FLOAT && HOP && MIXHOP && !OWN && !MIXOWN;

// Generic kernel for one output parity:
//   v = c_hop * H(in)                              (HOP; in gets gamma_5 if G5_HOP_IN)
//   v += a_own * own                               (OWN && !MIXOWN; own gets gamma_5 if G5_OWN_IN)
//   v = Mhop v                                     (MIXHOP)
//   v += Mown own                                  (MIXOWN)
//   v = gamma_5 v                                  (G5_OUT)
//   epilogue EPI
// SN > 0 (= kStructNs = Ns): the fifth-dimension product is the structured O(Ns) recurrence of
// a.sop (s_struct_col) instead of the dense Ns x Ns matrix.
template <int ST, bool HOP, bool MIXHOP, bool OWN, bool MIXOWN, int EPI, bool WS, int SN>
__device__ __forceinline__ void hop_body(const HopArgs& a) {
    using S = Store<ST>;
    using R = typename S::R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ns = a.Ns;
    const int s = threadIdx.x, ls = threadIdx.y, spb = blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    constexpr bool STRUCT = SN > 0;
    // FP32 arithmetic at Ns = 16 (dense form): warp-local tensor-core s-mixing, with its A-fragment
    // tables first in shared memory; otherwise FMA s-mixing from the matrices mh / mo
    constexpr bool kTC = !STRUCT && std::is_same<R, float>::value && (MIXHOP || MIXOWN) &&
                         !kLeanHop<ST, HOP, MIXHOP, OWN, MIXOWN>;
    const bool tc = kTC && Ns == 16;
    // staging row stride: 24 reals for the tensor-core mixing (its fragment loads are laid out for
    // it), the padded stride for the FMA mixing, the structured geometry for the column pass
    const int rst = STRUCT ? kSRow<R> : (tc ? 24 : kRowStride<R>);
    const int sst = STRUCT ? kSSite<R> : Ns * rst;
    constexpr int NMAT = STRUCT ? 0 : 1;
    uint32_t* afr_h = reinterpret_cast<uint32_t*>(smem_raw);
    uint32_t* afr_o = afr_h + (tc && MIXHOP ? kAfrag16Words : 0);
    R* mh = reinterpret_cast<R*>(afr_o + (tc && MIXOWN ? kAfrag16Words : 0));
    R* mo = mh + (MIXHOP ? NMAT * 2 * Ns * Ns : 0);
    R* sh = mo + (MIXOWN ? NMAT * 2 * Ns * Ns : 0);
    const int lane = tid & 31, warp = tid >> 5;
    constexpr bool REDUCE = (EPI != EPI_STORE);

    if (a.state != nullptr && EPI != EPI_STORE_NORM && EPI != EPI_RESID) {
        if (((volatile CGState*)a.state)->flag != FLAG_RUN) return;
    }
    if constexpr (!STRUCT) {
        for (int i = tid; i < 2 * Ns * Ns; i += nth) {
            // interleaved chirality pairs: (M_+, M_-)[s' Ns + s] side by side, one load per s'
            const int j = i < Ns * Ns ? 2 * i : 2 * (i - Ns * Ns) + 1;
            if (MIXHOP) mh[j] = (R)a.mhop[i];
            if (MIXOWN) mo[j] = (R)a.mown[i];
        }
    }
    if constexpr (kTC) {
        if (tc) {
            if (MIXHOP) s_mix16_afrag(a.mhop, afr_h, tid, nth);
            if (MIXOWN) s_mix16_afrag(a.mown, afr_o, tid, nth);
        }
    }
    double alpha = 0.0, beta = 0.0;
    if (EPI == EPI_CG_A) alpha = a.state->alpha;
    if (EPI == EPI_CG_B) beta = a.state->beta;
    const bool g5h = (a.g5 & G5_HOP_IN) != 0, g5o = (a.g5 & G5_OWN_IN) != 0, g5out = (a.g5 & G5_OUT) != 0;
    const R chop = (R)a.c_hop, aown = (R)a.a_own;
    double part = 0.0;
    __syncthreads();  // the matrices (and fragment tables) staged above are visible to every warp

    for (int g = blockIdx.x; g * spb < a.Vh; g += gridDim.x) {
        site_barrier<WS>();
        const int cb = g * spb + ls;
        const bool valid = cb < a.Vh;
        R v[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) v[k] = 0;
        if (HOP && valid) {
            int n[8];
            const int4* nb = reinterpret_cast<const int4*>(a.nbr + (size_t)cb * 8);
            int4 n0 = __ldg(nb), n1 = __ldg(nb + 1);
            n[0] = n0.x; n[1] = n0.y; n[2] = n0.z; n[3] = n0.w;
            n[4] = n1.x; n[5] = n1.y; n[6] = n1.z; n[7] = n1.w;
            hop_dir<ST, 0>(a, n, cb, s, v, g5h);
            hop_dir<ST, 1>(a, n, cb, s, v, g5h);
            hop_dir<ST, 2>(a, n, cb, s, v, g5h);
            hop_dir<ST, 3>(a, n, cb, s, v, g5h);
#pragma unroll
            for (int k = 0; k < 24; ++k) v[k] *= chop;
        }
        R ow[24];
        if (OWN) {
            if (valid) {
                S::load(a.own, a.own_scale, (size_t)cb, s, Ns, ow);
                if (g5o) g5_flip(ow);
            } else {
#pragma unroll
                for (int k = 0; k < 24; ++k) ow[k] = 0;
            }
            if (!MIXOWN) {
#pragma unroll
                for (int k = 0; k < 24; ++k) v[k] = fma(aown, ow[k], v[k]);
            }
        }
        if (MIXHOP && STRUCT) {
            R* row = sh + ls * sst + s * rst;
            row24_store(row, v);
            site_barrier<WS>();
            if constexpr (STRUCT) s_struct_col<R, (STRUCT ? SN : 1)>(a.sc, a.sop, sh + ls * sst, rst, s);
            site_barrier<WS>();
            row24_load(row, v, false);
        } else if (MIXHOP) {
            row24_store(sh + ls * sst + s * rst, v);
            if constexpr (kTC) {
                if (tc) {
                    __syncwarp();
                    s_mix16_tc(afr_h, sh, lane, warp, ls * Ns + s, v, false);
                } else {
                    site_barrier<WS>();
                    s_mix2(mh, sh + ls * sst, s, Ns, v, false, rst);
                }
            } else {
                site_barrier<WS>();
                s_mix2(mh, sh + ls * sst, s, Ns, v, false, rst);
            }
        }
        if (MIXOWN && STRUCT) {
            if (MIXHOP) site_barrier<WS>();
            R* row = sh + ls * sst + s * rst;
            row24_store(row, ow);
            site_barrier<WS>();
            if constexpr (STRUCT) s_struct_col<R, (STRUCT ? SN : 1)>(a.sc, a.sop, sh + ls * sst, rst, s);
            site_barrier<WS>();
            row24_load(row, v, true);
        } else if (MIXOWN) {
            if (MIXHOP) {
                if (tc) __syncwarp();
                else site_barrier<WS>();
            }
            row24_store(sh + ls * sst + s * rst, ow);
            if constexpr (kTC) {
                if (tc) {
                    __syncwarp();
                    s_mix16_tc(afr_o, sh, lane, warp, ls * Ns + s, v, true);
                } else {
                    site_barrier<WS>();
                    s_mix2(mo, sh + ls * sst, s, Ns, v, true, rst);
                }
            } else {
                site_barrier<WS>();
                s_mix2(mo, sh + ls * sst, s, Ns, v, true, rst);
            }
        }
        if (g5out) g5_flip(v);
        if (!valid) continue;

        epilogue<ST, EPI>(a, cb, s, v, ow, alpha, beta, part);
    }
    if (REDUCE) grid_finalize<EPI>(a, part);
}

// The system's arguments are copied once into shared memory, so field accesses in the body are
// shared-memory broadcasts rather than repeated global loads.
__device__ __forceinline__ const HopArgs& stage_args(const HopArgs* __restrict__ args, HopArgs* sa) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    constexpr int nw = (int)(sizeof(HopArgs) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(args + blockIdx.y);
    int* dst = reinterpret_cast<int*>(sa);
    for (int i = tid; i < nw; i += blockDim.x * blockDim.y) dst[i] = __ldg(src + i);
    __syncthreads();
    return *sa;
}

// ---- bulk-staged variant ------------------------------------------------------------------------
// The same operator as hop_body, but the CTA first requests all the neighbour spinors it needs
// with asynchronous bulk copies (cp.async.bulk, completion on one shared-memory mbarrier), so the
// whole gather of a CTA is in flight at once instead of one dependent load per thread. A CTA owns
// spb = 8k checkerboard sites = k whole 2^4 blocks (see the site order in odwf_create). Inside a
// block every site has one neighbour per axis in the same block (the site with that coordinate
// bit flipped: the whole other-parity half of the block, one contiguous run of 8 sites) and one
// outside it (fetched individually through the neighbour table). Shared memory per CTA:
//   slots [k*8 inside + 4*spb outside][NCH][Ns] 16-byte chunks (+ FP16 scales), the CTA's links
//   [spb][8][20] floats, and the fifth-dimension matrices; the s-mixing buffer aliases the slots.
template <int ST>
struct StagedGeom {
    static constexpr int NCH = Store<ST>::NCH;
    static __host__ __device__ int slot_bytes(int Ns) { return NCH * Ns * 16; }
    static __host__ __device__ int scale_bytes(int Ns) { return ST == ST_HALF ? Ns * 4 : 0; }
    static __host__ __device__ int nslots(int spb) { return spb + 4 * spb; }
};

// Spinor of slot `slot`, slice s, from shared memory (FP32 or FP16 chunks).
template <int ST>
__device__ __forceinline__ void slot_load(const unsigned char* slots, const float* scales, int slot, int s, int Ns,
                                          float v[24]) {
    if (ST == ST_FLOAT) {
        const float4* p = reinterpret_cast<const float4*>(slots + (size_t)slot * StagedGeom<ST>::slot_bytes(Ns)) + s;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            float4 c = p[j * Ns];
            v[4 * j] = c.x;
            v[4 * j + 1] = c.y;
            v[4 * j + 2] = c.z;
            v[4 * j + 3] = c.w;
        }
    } else {
        const uint4* p = reinterpret_cast<const uint4*>(slots + (size_t)slot * StagedGeom<ST>::slot_bytes(Ns)) + s;
        const float sc = scales[slot * Ns + s];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            uint4 c = p[j * Ns];
            const __half2* hh = reinterpret_cast<const __half2*>(&c);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2 f = __half22float2(hh[q]);
                v[8 * j + 2 * q] = f.x * sc;
                v[8 * j + 2 * q + 1] = f.y * sc;
            }
        }
    }
}

template <int ST, int MU>
__device__ __forceinline__ void hop_dir_staged(const unsigned char* slots, const float* scales, const float* lk,
                                               int spb, int ls, int s, int Ns, const int bits[4], bool g5in,
                                               float* v) {
    float psi[24], h[12], w[12], u[18];
    const int blk = ls >> 3, i = ls & 7;
    const int partner = blk * 8 + (MU == 0 ? i : (i ^ (1 << (MU - 1))));
    const int outside = spb + ls * 4 + MU;
    // forward neighbour is in the block iff the site's MU coordinate bit is 0
    const int sf = bits[MU] == 0 ? partner : outside;
    const int sb = bits[MU] == 1 ? partner : outside;
    slot_load<ST>(slots, scales, sf, s, Ns, psi);
    if (g5in) g5_flip(psi);
    project<MU, -1>(psi, h);
#pragma unroll
    for (int k = 0; k < 18; ++k) u[k] = lk[(ls * 8 + MU) * 20 + k];
    su3_mul_half(u, h, w);
    reconstruct<MU, -1>(v, w);
    slot_load<ST>(slots, scales, sb, s, Ns, psi);
    if (g5in) g5_flip(psi);
    project<MU, +1>(psi, h);
#pragma unroll
    for (int k = 0; k < 18; ++k) u[k] = lk[(ls * 8 + 4 + MU) * 20 + k];
    su3_mul_half(u, h, w);
    reconstruct<MU, +1>(v, w);
}

template <int ST, bool MIXHOP, bool OWN, bool MIXOWN, int EPI>
__device__ __forceinline__ void hop_body_staged(const HopArgs& a) {
    static_assert(ST == ST_FLOAT || ST == ST_HALF, "staged kernels are FP32 / FP16 storage");
    using S = Store<ST>;
    using G = StagedGeom<ST>;
    extern __shared__ __align__(16) unsigned char smem_st[];
    unsigned char* smem_raw = smem_st;
    const int Ns = a.Ns;
    const int s = threadIdx.x, ls = threadIdx.y, spb = blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    const int SB = G::slot_bytes(Ns), SCB = G::scale_bytes(Ns), NSL = G::nslots(spb);
    // layout: [mbarrier 16][matrices][links][slots][scales]
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    float* mh = reinterpret_cast<float*>(smem_raw + 16);
    float* mo = mh + (MIXHOP ? 2 * Ns * Ns : 0);
    float* lk = mo + (MIXOWN ? 2 * Ns * Ns : 0);
    unsigned char* slots = reinterpret_cast<unsigned char*>(lk + spb * 8 * 20);
    float* scales = reinterpret_cast<float*>(slots + (size_t)NSL * SB);
    float* sh = reinterpret_cast<float*>(slots);  // s-mixing buffer, reused after the hop
    __shared__ int ok_s;
    constexpr bool REDUCE = (EPI != EPI_STORE);

    if (a.state != nullptr && EPI != EPI_STORE_NORM && EPI != EPI_RESID) {
        if (((volatile CGState*)a.state)->flag != FLAG_RUN) return;
    }
    if (tid == 0) mbar_init(bar);
    for (int i = tid; i < 2 * Ns * Ns; i += nth) {
        if (MIXHOP) mh[i] = (float)a.mhop[i];
        if (MIXOWN) mo[i] = (float)a.mown[i];
    }
    __syncthreads();
    double alpha = 0.0, beta = 0.0;
    if (EPI == EPI_CG_A) alpha = a.state->alpha;
    if (EPI == EPI_CG_B) beta = a.state->beta;
    const bool g5h = (a.g5 & G5_HOP_IN) != 0, g5o = (a.g5 & G5_OWN_IN) != 0, g5out = (a.g5 & G5_OUT) != 0;
    const float chop = (float)a.c_hop, aown = (float)a.a_own;
    double part = 0.0;
    // site coordinate bits inside its 2^4 block (block-local index i = cb & 7: y, z, t bits; x from parity)
    int bits[4];
    {
        const int i = ls & 7;
        bits[1] = i & 1;
        bits[2] = (i >> 1) & 1;
        bits[3] = (i >> 2) & 1;
        bits[0] = (a.parity ^ bits[1] ^ bits[2] ^ bits[3]) & 1;
    }
    uint32_t phase = 0;
    const char* in_base = reinterpret_cast<const char*>(a.in);
    const char* in_scale = reinterpret_cast<const char*>(a.in_scale);
    const char* lk_base = reinterpret_cast<const char*>(a.links);

    for (int g = blockIdx.x; g * spb < a.Vh; g += gridDim.x) {
        // order this thread's generic shared-memory accesses before the next bulk copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();  // every thread is done with the previous group's shared memory
        const int cb0 = g * spb;
        const int nv = min(spb, a.Vh - cb0);  // a multiple of 8
        const int nblk = nv >> 3;
        const int cb = cb0 + ls;
        const bool valid = ls < nv;
        if (tid < 32) {
            // warp 0 issues the gather: inside runs, outside singles, links (+ FP16 scales)
            const int n_in = nblk, n_out = 4 * nv;
            const int ncopy = (n_in + n_out) * (ST == ST_HALF ? 2 : 1) + 1;
            if (tid == 0) {
                const uint32_t total = (uint32_t)((size_t)(nblk * 8 + n_out) * (SB + SCB) + (size_t)nv * 8 * 80);
                mbar_expect(bar, total);
            }
            __syncwarp();
            for (int k = tid; k < ncopy; k += 32) {
                int kk = k;
                const bool sc = (ST == ST_HALF) && kk >= n_in + n_out + 1;
                if (sc) kk -= n_in + n_out + 1;
                if (!sc && kk == n_in + n_out) {
                    bulk_copy(lk, lk_base + (size_t)cb0 * 8 * 80, (uint32_t)(nv * 8 * 80), bar);
                    continue;
                }
                int src_cb, slot, count;
                if (kk < n_in) {
                    src_cb = cb0 + kk * 8;
                    slot = kk * 8;
                    count = 8;
                } else {
                    const int q = kk - n_in, site = q >> 2, mu = q & 3;
                    const int i = site & 7;
                    int b[4];
                    b[1] = i & 1;
                    b[2] = (i >> 1) & 1;
                    b[3] = (i >> 2) & 1;
                    b[0] = (a.parity ^ b[1] ^ b[2] ^ b[3]) & 1;
                    const int dir = b[mu] ? mu : 4 + mu;  // the neighbour outside the block
                    src_cb = __ldg(a.nbr + (size_t)(cb0 + site) * 8 + dir);
                    slot = spb + site * 4 + mu;
                    count = 1;
                }
                if (!sc)
                    bulk_copy(slots + (size_t)slot * SB, in_base + (size_t)src_cb * SB, (uint32_t)(count * SB), bar);
                else
                    bulk_copy(scales + (size_t)slot * Ns, in_scale + (size_t)src_cb * SCB, (uint32_t)(count * SCB), bar);
            }
        }
        // own field (streamed) while the gather is in flight
        float ow[24];
        if (OWN) {
            if (valid) {
                S::load(a.own, a.own_scale, (size_t)cb, s, Ns, ow);
                if (g5o) g5_flip(ow);
            } else {
#pragma unroll
                for (int k = 0; k < 24; ++k) ow[k] = 0;
            }
        }
        if (tid == 0) {
            bool ok = mbar_wait_bounded(bar, phase, a.wait_cycles);
            if (!ok) {
                if (a.fault) atomicOr(a.fault, 1u);
                // the copies of this phase still target this CTA's shared memory: wait for them with
                // the full limit before the CTA leaves its groups
                mbar_wait_bounded(bar, phase);
            }
            ok_s = ok;
        }
        __syncthreads();
        // on a time-out the CTA skips its remaining groups but still joins the grid reduction, so
        // the reduction ticket of the solver state stays consistent
        if (!ok_s) break;
        phase ^= 1u;
        float v[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) v[k] = 0;
        if (valid) {
            hop_dir_staged<ST, 0>(slots, scales, lk, spb, ls, s, Ns, bits, g5h, v);
            hop_dir_staged<ST, 1>(slots, scales, lk, spb, ls, s, Ns, bits, g5h, v);
            hop_dir_staged<ST, 2>(slots, scales, lk, spb, ls, s, Ns, bits, g5h, v);
            hop_dir_staged<ST, 3>(slots, scales, lk, spb, ls, s, Ns, bits, g5h, v);
#pragma unroll
            for (int k = 0; k < 24; ++k) v[k] *= chop;
        }
        if (OWN && !MIXOWN) {
#pragma unroll
            for (int k = 0; k < 24; ++k) v[k] = fma(aown, ow[k], v[k]);
        }
        __syncthreads();  // slots are read; the mixing buffer may overwrite them
        if (MIXHOP) {
            row24_store(sh + (ls * Ns + s) * 24, v);
            __syncthreads();
            s_mix(mh, sh + ls * Ns * 24, s, Ns, v, false);
        }
        if (MIXOWN) {
            if (MIXHOP) __syncthreads();
            row24_store(sh + (ls * Ns + s) * 24, ow);
            __syncthreads();
            s_mix(mo, sh + ls * Ns * 24, s, Ns, v, true);
        }
        if (g5out) g5_flip(v);
        if (!valid) continue;
        epilogue<ST, EPI>(a, cb, s, v, ow, alpha, beta, part);
    }
    if (REDUCE) grid_finalize<EPI>(a, part);
}

template <int ST, bool MIXHOP, bool OWN, bool MIXOWN, int EPI>
__global__ void __launch_bounds__(256) k_hop_staged(HopArgs a) {
    hop_body_staged<ST, MIXHOP, OWN, MIXOWN, EPI>(a);
}

template <int ST, bool MIXHOP, bool OWN, bool MIXOWN, int EPI>
__global__ void __launch_bounds__(256) k_hop_staged_multi(const HopArgs* __restrict__ args) {
    __shared__ HopArgs sa;
    hop_body_staged<ST, MIXHOP, OWN, MIXOWN, EPI>(stage_args(args, &sa));
}

template <int ST>
size_t staged_smem(int Ns, int spb, bool mixhop, bool mixown) {
    using G = StagedGeom<ST>;
    return 16 + sizeof(float) * (size_t)(mixhop + mixown) * 2 * Ns * Ns + (size_t)spb * 8 * 80 +
           (size_t)G::nslots(spb) * (G::slot_bytes(Ns) + G::scale_bytes(Ns));
}

template <int ST, bool HOP, bool MIXHOP, bool OWN, bool MIXOWN, int EPI, bool WS, int SN = 0>
__global__ void __launch_bounds__(256) k_hop(HopArgs a) {
    hop_body<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, WS, SN>(a);
}

// Register-capped copy for the FP32 hop-then-mix variant (K1, K1^dag): at most 64 registers (4 CTAs
// of 256 or 8 of 128 threads per SM) costs it 8 bytes of spill and buys resident warps for its
// latency-bound neighbour gathers; the other variants (which would spill more) keep k_hop.
template <int ST, bool HOP, bool MIXHOP, bool OWN, bool MIXOWN, int EPI, bool WS, int SN = 0>
__global__ void __launch_bounds__(256, 4) k_hop_lean(HopArgs a) {
    hop_body<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, WS, SN>(a);
}



// Several independent systems in one launch: blockIdx.y selects the system's arguments (its own
// fields, lattice tables, solver state and reduction buffer); blockIdx.x strides over its sites.
// Systems that are converged or waiting for a host-side update return at once.
template <int ST, bool HOP, bool MIXHOP, bool OWN, bool MIXOWN, int EPI, bool WS, int SN = 0>
__global__ void __launch_bounds__(256) k_hop_multi(const HopArgs* __restrict__ args) {
    __shared__ HopArgs sa;
    hop_body<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, WS, SN>(stage_args(args, &sa));
}

template <int ST, bool HOP, bool MIXHOP, bool OWN, bool MIXOWN, int EPI, bool WS, int SN = 0>
__global__ void __launch_bounds__(256, 4) k_hop_multi_lean(const HopArgs* __restrict__ args) {
    __shared__ HopArgs sa;
    hop_body<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, WS, SN>(stage_args(args, &sa));
}

// the per-thread-gather kernel of a variant, single system and several systems; WS (Ns divides
// 32) selects warp-level instead of CTA-wide synchronisation of the staged rows; SN the
// structured fifth-dimension product (single-system kernels, Ns = kStructNs)
template <int ST, bool HOP, bool MIXHOP, bool OWN, bool MIXOWN, int EPI, bool WS, int SN = 0>
constexpr auto hop_kernel() {
    if constexpr (kLeanHop<ST, HOP, MIXHOP, OWN, MIXOWN>) return k_hop_lean<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, WS, SN>;
    else return k_hop<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, WS, SN>;
}
template <int ST, bool HOP, bool MIXHOP, bool OWN, bool MIXOWN, int EPI, bool WS, int SN = 0>
constexpr auto hop_multi_kernel() {
    if constexpr (kLeanHop<ST, HOP, MIXHOP, OWN, MIXOWN>) return k_hop_multi_lean<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, WS, SN>;
    else return k_hop_multi<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, WS, SN>;
}

static bool warp_sites(int Ns) { return 32 % Ns == 0; }

// ---- launch ------------------------------------------------------------------------------------
// Sites per CTA: the CTA holds spb * Ns threads, a multiple of 32 and at least 128.
int spb_for(int Ns) {
    int g = 32, n = Ns;
    while (n) { int t = g % n; g = n; n = t; }  // gcd(32, Ns)
    const int base = 32 / g;
    int spb = base;
    while (spb * Ns < 128) spb += base;
    return spb;
}

// Lattice tables of handle h for output parity `parity`; reducing epilogues default to the
// handle's own state and reduction buffer. A plain store keeps a.state as given (null: no
// early-exit check on the solver flag).
void hop_fill(odwf_s* h, int storage, int parity, HopArgs& a, bool reduces) {
    a.links = (storage == ST_DOUBLE) ? (const void*)h->U64[parity] : (const void*)h->U32[parity];
    a.nbr = h->nbr[parity];
    a.links12 = h->U12[parity];
    a.nbrs = h->nbrs[parity];
    a.Vh = h->Vh;
    a.Ns = h->Ns;
    a.parity = parity;
    a.fault = h->fault;
    a.wait_cycles = h->wait_cycles;
    if (a.partials == nullptr) a.partials = h->partials;
    if (reduces && a.state == nullptr) a.state = h->state;
}

// The bulk-staged kernels need CTAs of whole 2^4 blocks (spb a multiple of 8) and, for FP16,
// 16-byte scale rows (Ns a multiple of 4).
static bool staged_geom_ok(const odwf_s* h, int st) {
    if (st == ST_DOUBLE) return false;
    if (spb_for(h->Ns) % 8) return false;
    if (st == ST_HALF && h->Ns % 4) return false;
    return true;
}

static bool staged_ok(const odwf_s* h, int st) { return h->staged && staged_geom_ok(h, st); }

// Grid of a fused kernel: mode 0 one resident wave (SMs x occupancy), 1 one CTA per site group,
// 2 / 3 two / four resident waves; reducing kernels are capped by the partial-sum buffer.
int grid_for_mode(const odwf_s* h, int mode, int occ, int groups, bool reduces) {
    long g;
    switch (mode) {
        case 1: g = groups; break;
        case 2: g = 2L * h->num_sms * occ; break;
        case 3: g = 4L * h->num_sms * occ; break;
        default: g = (long)h->num_sms * occ; break;
    }
    if (g > groups) g = groups;
    if (reduces && g > h->partials_n) g = h->partials_n;
    return g < 1 ? 1 : (int)g;
}

template <int ST, bool HOP, bool MIXHOP, bool OWN, bool MIXOWN, int EPI>
struct KernelPick {
    static constexpr bool CAN_STAGE = HOP && ST != ST_DOUBLE;
    static constexpr bool CAN_STRUCT = MIXHOP || MIXOWN;
    // kind: 0 plain single, 1 plain multi, 2 staged single, 3 staged multi, 4 structured single,
    // 5 structured multi
    static const void* fn(int kind, bool ws) {
        if constexpr (CAN_STAGE) {
            if (kind == 2) return (const void*)k_hop_staged<ST, MIXHOP, OWN, MIXOWN, EPI>;
            if (kind == 3) return (const void*)k_hop_staged_multi<ST, MIXHOP, OWN, MIXOWN, EPI>;
        }
        if constexpr (CAN_STRUCT) {
            if (kind == 4) return (const void*)hop_kernel<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, true, kStructNs>();
            if (kind == 5) return (const void*)hop_multi_kernel<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, true, kStructNs>();
        }
        if (ws)
            return kind == 1 ? (const void*)hop_multi_kernel<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, true>()
                             : (const void*)hop_kernel<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, true>();
        return kind == 1 ? (const void*)hop_multi_kernel<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, false>()
                         : (const void*)hop_kernel<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, false>();
    }
};

template <int ST, bool HOP, bool MIXHOP, bool OWN, bool MIXOWN, int EPI>
static int occupancy(odwf_s* h, int kind, size_t* smem_out, int spb = 0) {
    using R = typename Store<ST>::R;
    const int Ns = h->Ns;
    if (spb <= 0) spb = spb_for(Ns);
    size_t smem = sizeof(R) * ((size_t)(MIXHOP + MIXOWN) * 2 * Ns * Ns + (size_t)spb * Ns * kRowStride<R>);
    // A-fragment tables of the tensor-core s-mixing (FP32 arithmetic, Ns = 16)
    if (std::is_same<R, float>::value && Ns == 16 && !kLeanHop<ST, HOP, MIXHOP, OWN, MIXOWN>)
        smem += sizeof(uint32_t) * kAfrag16Words * (MIXHOP + MIXOWN);
    if constexpr (ST != ST_DOUBLE) {
        if (kind == 2 || kind == 3) smem = staged_smem<ST>(Ns, spb, MIXHOP, MIXOWN);
    }
    if (kind == 4 || kind == 5) smem = sizeof(R) * (size_t)spb * kSSite<R>;
    *smem_out = smem;
    static std::map<long, int> occ_cache;  // (kind, Ns, sites per CTA) -> resident CTAs per SM
    static bool attr_set[6][2] = {{false, false}, {false, false}, {false, false},
                                  {false, false}, {false, false}, {false, false}};
    const bool ws = warp_sites(Ns);
    const void* fn = KernelPick<ST, HOP, MIXHOP, OWN, MIXOWN, EPI>::fn(kind, ws);
    if (!attr_set[kind][ws]) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set[kind][ws] = true;
    }
    int& occ = occ_cache[((long)kind * 64 + Ns) * 1024 + spb];
    if (occ == 0) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, Ns * spb, smem) != cudaSuccess || o < 1) o = 1;
        occ = o;
    }
    return occ;
}

template <int ST, bool HOP, bool MIXHOP, bool OWN, bool MIXOWN, int EPI>
static int launch_multi_one(odwf_s* h, const HopArgs* dev_args, int n, int max_vh, bool structured, cudaStream_t st) {
    size_t smem = 0;
    const bool stg = KernelPick<ST, HOP, MIXHOP, OWN, MIXOWN, EPI>::CAN_STAGE && staged_ok(h, ST);
    // structured fifth-dimension products: every system's arguments carry them (Ns = kStructNs)
    const bool sn = KernelPick<ST, HOP, MIXHOP, OWN, MIXOWN, EPI>::CAN_STRUCT && !stg && structured &&
                    h->Ns == kStructNs;
    const int kind = stg ? 3 : (sn ? 5 : 1);
    const int occ = occupancy<ST, HOP, MIXHOP, OWN, MIXOWN, EPI>(h, kind, &smem);
    const int spb = spb_for(h->Ns);
    const int groups = (max_vh + spb - 1) / spb;
    // one full resident wave per system: while several systems run their CTAs queue behind one
    // another, and once the others have stopped (their CTAs return at once) the last running
    // system still has the whole GPU rather than a 1/n share of it
    int gx = h->num_sms * occ;
    if (gx > groups) gx = groups;
    if (EPI != EPI_STORE && gx > h->partials_n) gx = h->partials_n;
    if (gx < 1) gx = 1;
    if constexpr (KernelPick<ST, HOP, MIXHOP, OWN, MIXOWN, EPI>::CAN_STAGE) {
        if (stg) {
            h->staged_used = true;
            k_hop_staged_multi<ST, MIXHOP, OWN, MIXOWN, EPI><<<dim3(gx, n), dim3(h->Ns, spb), smem, st>>>(dev_args);
            return cuda_check(h, cudaGetLastError(), "k_hop_staged_multi launch");
        }
    }
    if constexpr (KernelPick<ST, HOP, MIXHOP, OWN, MIXOWN, EPI>::CAN_STRUCT) {
        if (sn) {
            hop_multi_kernel<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, true, kStructNs>()<<<dim3(gx, n), dim3(h->Ns, spb), smem, st>>>(
                dev_args);
            return cuda_check(h, cudaGetLastError(), "k_hop_multi launch");
        }
    }
    if (warp_sites(h->Ns))
        hop_multi_kernel<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, true>()<<<dim3(gx, n), dim3(h->Ns, spb), smem, st>>>(dev_args);
    else
        hop_multi_kernel<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, false>()<<<dim3(gx, n), dim3(h->Ns, spb), smem, st>>>(dev_args);
    return cuda_check(h, cudaGetLastError(), "k_hop_multi launch");
}

template <int ST, bool HOP, bool MIXHOP, bool OWN, bool MIXOWN, int EPI>
static int launch_one(odwf_s* h, int parity, HopArgs a, cudaStream_t st) {
    const int Ns = h->Ns;
    int spb = spb_for(Ns);
    size_t smem = 0;
    const int base_key = ST * 100000 + HOP * 10000 + MIXHOP * 1000 + OWN * 100 + MIXOWN * 10 + EPI;
    bool stg = KernelPick<ST, HOP, MIXHOP, OWN, MIXOWN, EPI>::CAN_STAGE && staged_ok(h, ST);
    int mode = 0;
    bool force_dense = false;
    auto tuned = h->tune.find(base_key);
    if (tuned != h->tune.end()) {
        mode = tuned->second.mode;
        force_dense = tuned->second.dense != 0;
        stg = KernelPick<ST, HOP, MIXHOP, OWN, MIXOWN, EPI>::CAN_STAGE && staged_geom_ok(h, ST) && tuned->second.staged;
        // tile: a multiple of the default sites per CTA while the CTA stays within 256 threads
        if (tuned->second.spbm > 1 && spb * tuned->second.spbm * Ns <= 256) spb *= tuned->second.spbm;
    }
    // the structured fifth-dimension product: single-system per-thread-gather kernels at Ns = kStructNs
    const bool sn = KernelPick<ST, HOP, MIXHOP, OWN, MIXOWN, EPI>::CAN_STRUCT && !stg && Ns == kStructNs &&
                    a.sop != SOP_DENSE && !force_dense;
    // two slices per thread (hop_pair.cu): ODWF_PAIR=1 wherever it applies, else the tuned choice
    int pair = 0;
    int pair_tile = 1;
    if (sn && HOP && pair_variant(ST, MIXHOP, OWN, MIXOWN, EPI) && pair_applies(h, ST, a) && h->pair != 0) {
        if (h->pair > 0) pair = h->pair;
        else if (tuned != h->tune.end()) pair = tuned->second.pair;
        if (tuned != h->tune.end()) pair_tile = tuned->second.spbm;
    }
    if (pair) {
        hop_fill(h, ST, parity, a, EPI != EPI_STORE);
        const int pkey = base_key + 500000 + (pair >= 2 && pair_tma_applies(ST, a) ? 1000000 : 0);
        cudaEvent_t ev = nullptr;
        if (h->prof) prof_begin(h, pkey, st, &ev);
        const int rc = launch_hop_pair(h, ST, MIXHOP, OWN, MIXOWN, EPI, a, mode, pair_tile, st, pair);
        if (h->prof) prof_end(h, pkey, st, ev);
        return rc;
    }
    const int occ = occupancy<ST, HOP, MIXHOP, OWN, MIXOWN, EPI>(h, stg ? 2 : (sn ? 4 : 0), &smem, spb);
    const int groups = (h->Vh + spb - 1) / spb;
    const int grid = grid_for_mode(h, mode, occ, groups, EPI != EPI_STORE);
    hop_fill(h, ST, parity, a, EPI != EPI_STORE);
    const int key = (stg ? 1000000 : 0) + base_key;
    cudaEvent_t ev0 = nullptr;
    if (h->prof) prof_begin(h, key, st, &ev0);
    bool plain = true;
    if constexpr (KernelPick<ST, HOP, MIXHOP, OWN, MIXOWN, EPI>::CAN_STAGE) {
        if (stg) {
            h->staged_used = true;
            k_hop_staged<ST, MIXHOP, OWN, MIXOWN, EPI><<<grid, dim3(Ns, spb), smem, st>>>(a);
            plain = false;
        }
    }
    if constexpr (KernelPick<ST, HOP, MIXHOP, OWN, MIXOWN, EPI>::CAN_STRUCT) {
        if (sn) {
            hop_kernel<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, true, kStructNs>()<<<grid, dim3(Ns, spb), smem, st>>>(a);
            plain = false;
        }
    }
    if (plain) {
        if (warp_sites(Ns)) hop_kernel<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, true>()<<<grid, dim3(Ns, spb), smem, st>>>(a);
        else hop_kernel<ST, HOP, MIXHOP, OWN, MIXOWN, EPI, false>()<<<grid, dim3(Ns, spb), smem, st>>>(a);
    }
    if (h->prof) prof_end(h, key, st, ev0);
    return cuda_check(h, cudaGetLastError(), "k_hop launch");
}

template <int ST>
static int launch_st(odwf_s* h, int parity, bool hop, bool mixhop, bool own, bool mixown, int epi, HopArgs a,
                     cudaStream_t st) {
#define ODWF_CASE(HOPV, MH, OW, MO, E)                                                          \
    if (hop == HOPV && mixhop == MH && own == OW && mixown == MO && epi == E)                     \
        return launch_one<ST, HOPV, MH, OW, MO, E>(h, parity, a, st);
    ODWF_CASE(true, true, false, false, EPI_STORE)      // K1: t = Mhop c H in
    ODWF_CASE(true, true, true, false, EPI_STORE)       // t = Mhop (c H in + a own)
    ODWF_CASE(true, false, true, true, EPI_STORE)       // out = Mown own + c H in
    ODWF_CASE(true, false, true, true, EPI_STORE_NORM)  // same, |out|^2
    ODWF_CASE(true, false, true, true, EPI_RESID)       // out = b - (Mown own + c H in)
    ODWF_CASE(true, false, true, true, EPI_CG_A)        // CGNE forward half step
    ODWF_CASE(true, false, true, true, EPI_CG_B)        // CGNE adjoint half step
    ODWF_CASE(true, false, true, false, EPI_STORE)      // out = a own + c H in
    ODWF_CASE(false, false, true, true, EPI_STORE)      // out = Mown own (s-local)
#undef ODWF_CASE
    return set_err(h, ODWF_EINVAL, "unsupported hop kernel variant");
}

template <int ST>
static int launch_multi_st(odwf_s* h, bool mixhop, bool own, bool mixown, int epi, const HopArgs* dev_args, int n,
                           int max_vh, bool structured, cudaStream_t st) {
#define ODWF_MCASE(MH, OW, MO, E)                                                                  \
    if (mixhop == MH && own == OW && mixown == MO && epi == E)                                     \
        return launch_multi_one<ST, true, MH, OW, MO, E>(h, dev_args, n, max_vh, structured, st);
    ODWF_MCASE(true, false, false, EPI_STORE)
    ODWF_MCASE(false, true, true, EPI_CG_A)
    ODWF_MCASE(false, true, true, EPI_CG_B)
#undef ODWF_MCASE
    return set_err(h, ODWF_EINVAL, "unsupported multi-system hop kernel variant");
}

int launch_hop_multi(odwf_s* h, int storage, bool mixhop, bool own, bool mixown, int epi, const HopArgs* dev_args,
                     int n, int max_vh, cudaStream_t st, bool structured) {
    switch (storage) {
        case ST_DOUBLE: return launch_multi_st<ST_DOUBLE>(h, mixhop, own, mixown, epi, dev_args, n, max_vh, structured, st);
        case ST_FLOAT: return launch_multi_st<ST_FLOAT>(h, mixhop, own, mixown, epi, dev_args, n, max_vh, structured, st);
        case ST_HALF: return launch_multi_st<ST_HALF>(h, mixhop, own, mixown, epi, dev_args, n, max_vh, structured, st);
    }
    return set_err(h, ODWF_EINVAL, "bad storage");
}

int launch_hop(odwf_s* h, int storage, int parity, bool mixhop, bool own, bool mixown, int epi, HopArgs a,
               cudaStream_t st) {
    switch (storage) {
        case ST_DOUBLE: return launch_st<ST_DOUBLE>(h, parity, true, mixhop, own, mixown, epi, a, st);
        case ST_FLOAT: return launch_st<ST_FLOAT>(h, parity, true, mixhop, own, mixown, epi, a, st);
        case ST_HALF: return launch_st<ST_HALF>(h, parity, true, mixhop, own, mixown, epi, a, st);
    }
    return set_err(h, ODWF_EINVAL, "bad storage");
}

// p = a_own * own + beta p with |p|^2 and the CGNE alpha update (no hop, no s-mixing)
int launch_hop_own_cgb(odwf_s* h, int storage, HopArgs a, cudaStream_t st) {
    switch (storage) {
        case ST_DOUBLE: return launch_one<ST_DOUBLE, false, false, true, false, EPI_CG_B>(h, 0, a, st);
        case ST_FLOAT: return launch_one<ST_FLOAT, false, false, true, false, EPI_CG_B>(h, 0, a, st);
    }
    return set_err(h, ODWF_EINVAL, "bad storage");
}

int launch_smix(odwf_s* h, int storage, const void* in, void* out, const double* mt, double, cudaStream_t st,
                const float* in_scale, float* out_scale, const SCoef* c, int sop) {
    HopArgs a{};
    a.own = in;
    a.out = out;
    a.mown = mt;
    if (c && sop != SOP_DENSE) set_sop(a, c, sop);
    a.own_scale = in_scale;
    a.out_scale = out_scale;
    switch (storage) {
        case ST_DOUBLE: return launch_st<ST_DOUBLE>(h, 0, false, false, true, true, EPI_STORE, a, st);
        case ST_FLOAT: return launch_st<ST_FLOAT>(h, 0, false, false, true, true, EPI_STORE, a, st);
        case ST_HALF: return launch_st<ST_HALF>(h, 0, false, false, true, true, EPI_STORE, a, st);
    }
    return set_err(h, ODWF_EINVAL, "bad storage for smix");
}

// ---- layout kernels ----------------------------------------------------------------------------
// ABI 5D lexicographic complex128 [s][lex][12] <-> internal even-odd chunked storage.
template <int ST>
__global__ void k_pack5(const double2* __restrict__ lex5, void* e, void* o, float* es, float* os,
                        const int* __restrict__ lex_e, const int* __restrict__ lex_o, int Vh, int V, int Ns,
                        int r5g5) {
    using R = typename Store<ST>::R;
    const size_t total = (size_t)2 * Vh * Ns;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % Ns);
        const size_t rest = i / Ns;
        const int cb = (int)(rest % Vh);
        const int par = (int)(rest / Vh);
        const int lex = par ? lex_o[cb] : lex_e[cb];
        const int sin = r5g5 ? (Ns - 1 - s) : s;
        const double2* src = lex5 + ((size_t)sin * V + lex) * 12;
        R v[24];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 c = src[k];
            const double sg = (r5g5 && k >= 6) ? -1.0 : 1.0;
            v[2 * k] = (R)(sg * c.x);
            v[2 * k + 1] = (R)(sg * c.y);
        }
        Store<ST>::store(par ? o : e, par ? os : es, cb, s, Ns, v);
    }
}

template <int ST>
__global__ void k_unpack5(const void* e, const void* o, const float* es, const float* os, double2* __restrict__ lex5,
                          const int* __restrict__ lex_e, const int* __restrict__ lex_o, int Vh, int V, int Ns,
                          int r5g5) {
    using R = typename Store<ST>::R;
    const size_t total = (size_t)2 * Vh * Ns;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % Ns);
        const size_t rest = i / Ns;
        const int cb = (int)(rest % Vh);
        const int par = (int)(rest / Vh);
        const int lex = par ? lex_o[cb] : lex_e[cb];
        R v[24];
        Store<ST>::load(par ? o : e, par ? os : es, cb, s, Ns, v);
        const int sout = r5g5 ? (Ns - 1 - s) : s;
        double2* dst = lex5 + ((size_t)sout * V + lex) * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double sg = (r5g5 && k >= 6) ? -1.0 : 1.0;
            dst[k] = make_double2(sg * (double)v[2 * k], sg * (double)v[2 * k + 1]);
        }
    }
}

static int grid_1d(odwf_s* h, size_t n) {
    size_t g = (n + 255) / 256;
    const size_t cap = (size_t)h->num_sms * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

// Kernel timing of the layout and vector launches (odwf_profile_*): key 4000000 + kind * 100 +
// first storage * 10 + second storage; kind 1 pack5, 2 unpack5, 3 convert, 4 axpy to FP64, 5 norm.
struct ProfScope {
    odwf_s* h;
    int key;
    cudaStream_t st;
    cudaEvent_t ev = nullptr;
    ProfScope(odwf_s* h_, int kind, int s1, int s2, cudaStream_t st_) : h(h_), key(4000000 + kind * 100 + s1 * 10 + s2), st(st_) {
        if (h->prof) prof_begin(h, key, st, &ev);
    }
    ~ProfScope() {
        if (h->prof) prof_end(h, key, st, ev);
    }
};

int launch_pack5(odwf_s* h, const double* lex5, void* e, void* o, int storage, int r5g5, cudaStream_t st,
                 float* es, float* os) {
    ProfScope ps(h, 1, ST_DOUBLE, storage, st);
    const size_t n = (size_t)2 * h->Vh * h->Ns;
    const int g = grid_1d(h, n);
    if (storage == ST_DOUBLE)
        k_pack5<ST_DOUBLE><<<g, 256, 0, st>>>((const double2*)lex5, e, o, nullptr, nullptr, h->lexof[0], h->lexof[1],
                                              h->Vh, h->V, h->Ns, r5g5);
    else if (storage == ST_FLOAT)
        k_pack5<ST_FLOAT><<<g, 256, 0, st>>>((const double2*)lex5, e, o, nullptr, nullptr, h->lexof[0], h->lexof[1],
                                             h->Vh, h->V, h->Ns, r5g5);
    else if (storage == ST_HALF && es && os)
        k_pack5<ST_HALF><<<g, 256, 0, st>>>((const double2*)lex5, e, o, es, os, h->lexof[0], h->lexof[1], h->Vh,
                                            h->V, h->Ns, r5g5);
    else
        return set_err(h, ODWF_EINVAL, "pack5: storage");
    return cuda_check(h, cudaGetLastError(), "k_pack5");
}

int launch_unpack5(odwf_s* h, const void* e, const void* o, double* lex5, int storage, int r5g5, cudaStream_t st,
                   const float* es, const float* os) {
    ProfScope ps(h, 2, storage, ST_DOUBLE, st);
    const size_t n = (size_t)2 * h->Vh * h->Ns;
    const int g = grid_1d(h, n);
    if (storage == ST_DOUBLE)
        k_unpack5<ST_DOUBLE><<<g, 256, 0, st>>>(e, o, nullptr, nullptr, (double2*)lex5, h->lexof[0], h->lexof[1],
                                                h->Vh, h->V, h->Ns, r5g5);
    else if (storage == ST_FLOAT)
        k_unpack5<ST_FLOAT><<<g, 256, 0, st>>>(e, o, nullptr, nullptr, (double2*)lex5, h->lexof[0], h->lexof[1],
                                               h->Vh, h->V, h->Ns, r5g5);
    else if (storage == ST_HALF && es && os)
        k_unpack5<ST_HALF><<<g, 256, 0, st>>>(e, o, es, os, (double2*)lex5, h->lexof[0], h->lexof[1], h->Vh, h->V,
                                              h->Ns, r5g5);
    else
        return set_err(h, ODWF_EINVAL, "unpack5: storage");
    return cuda_check(h, cudaGetLastError(), "k_unpack5");
}

// ---- elementwise kernels over one half field (Vh * Ns spinors) ---------------------------------
template <int STI, int STO>
__global__ void k_convert(const void* in, const float* isc, void* out, float* osc, int Vh, int Ns) {
    using RI = typename Store<STI>::R;
    using RO = typename Store<STO>::R;
    const size_t total = (size_t)Vh * Ns;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % Ns);
        const size_t cb = i / Ns;
        RI v[24];
        RO w[24];
        Store<STI>::load(in, isc, cb, s, Ns, v);
#pragma unroll
        for (int k = 0; k < 24; ++k) w[k] = (RO)v[k];
        Store<STO>::store(out, osc, cb, s, Ns, w);
    }
}

template <int STI>
__global__ void k_axpy_to64(double a, const void* x, const float* xsc, double* y, int Vh, int Ns) {
    using RI = typename Store<STI>::R;
    const size_t total = (size_t)Vh * Ns;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % Ns);
        const size_t cb = i / Ns;
        RI v[24];
        double w[24];
        Store<STI>::load(x, xsc, cb, s, Ns, v);
        Store<ST_DOUBLE>::load(y, nullptr, cb, s, Ns, w);
#pragma unroll
        for (int k = 0; k < 24; ++k) w[k] = fma(a, (double)v[k], w[k]);
        Store<ST_DOUBLE>::store(y, nullptr, cb, s, Ns, w);
    }
}

template <int ST>
__global__ void k_norm2(const void* v, const float* sc, CGState* state, double* partials, int slot, int Vh, int Ns) {
    using R = typename Store<ST>::R;
    const size_t total = (size_t)Vh * Ns;
    double part = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % Ns);
        const size_t cb = i / Ns;
        R w[24];
        Store<ST>::load(v, sc, cb, s, Ns, w);
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < 24; ++k) t += (double)w[k] * (double)w[k];
        part += t;
    }
    HopArgs a{};
    a.state = state;
    a.partials = partials;
    a.slot = slot;
    grid_finalize<EPI_STORE_NORM>(a, part);
}

static int convert_dispatch(odwf_s* h, const void* in, int sti, const float* isc, void* out, int sto, float* osc,
                            cudaStream_t st) {
    const int g = grid_1d(h, (size_t)h->Vh * h->Ns);
#define ODWF_CV(A, B)                                                                              \
    if (sti == A && sto == B) {                                                                    \
        k_convert<A, B><<<g, 256, 0, st>>>(in, isc, out, osc, h->Vh, h->Ns);                       \
        return cuda_check(h, cudaGetLastError(), "k_convert");                                     \
    }
    ODWF_CV(ST_DOUBLE, ST_FLOAT)
    ODWF_CV(ST_DOUBLE, ST_HALF)
    ODWF_CV(ST_FLOAT, ST_DOUBLE)
    ODWF_CV(ST_HALF, ST_DOUBLE)
    ODWF_CV(ST_DOUBLE, ST_DOUBLE)
    ODWF_CV(ST_FLOAT, ST_FLOAT)
#undef ODWF_CV
    return set_err(h, ODWF_EINVAL, "convert: unsupported pair");
}

int launch_convert(odwf_s* h, const void* in, int st_in, const float* in_scale, void* out, int st_out,
                   float* out_scale, cudaStream_t st) {
    ProfScope ps(h, 3, st_in, st_out, st);
    return convert_dispatch(h, in, st_in, in_scale, out, st_out, out_scale, st);
}

int launch_axpy_to64(odwf_s* h, double a, const void* x, int st_in, const float* xsc, double* y, cudaStream_t st) {
    ProfScope ps(h, 4, st_in, ST_DOUBLE, st);
    const int g = grid_1d(h, (size_t)h->Vh * h->Ns);
    if (st_in == ST_FLOAT) k_axpy_to64<ST_FLOAT><<<g, 256, 0, st>>>(a, x, xsc, y, h->Vh, h->Ns);
    else if (st_in == ST_HALF) k_axpy_to64<ST_HALF><<<g, 256, 0, st>>>(a, x, xsc, y, h->Vh, h->Ns);
    else k_axpy_to64<ST_DOUBLE><<<g, 256, 0, st>>>(a, x, xsc, y, h->Vh, h->Ns);
    return cuda_check(h, cudaGetLastError(), "k_axpy_to64");
}

int launch_norm2(odwf_s* h, const void* v, int storage, const float* sc, int slot, cudaStream_t st,
                 CGState* state, double* partials) {
    ProfScope ps(h, 5, storage, storage, st);
    int g = grid_1d(h, (size_t)h->Vh * h->Ns);
    if (g > h->partials_n) g = h->partials_n;
    if (!state) state = h->state;
    if (!partials) partials = h->partials;
    if (storage == ST_DOUBLE) k_norm2<ST_DOUBLE><<<g, 256, 0, st>>>(v, sc, state, partials, slot, h->Vh, h->Ns);
    else if (storage == ST_FLOAT) k_norm2<ST_FLOAT><<<g, 256, 0, st>>>(v, sc, state, partials, slot, h->Vh, h->Ns);
    else k_norm2<ST_HALF><<<g, 256, 0, st>>>(v, sc, state, partials, slot, h->Vh, h->Ns);
    return cuda_check(h, cudaGetLastError(), "k_norm2");
}

// ---- gauge field -------------------------------------------------------------------------------
// U (ABI): [mu][lex][3][3] complex128. Output per parity p and checkerboard site cb:
//   dir mu     : U_mu(x), times -1 when mu = t and x_t = Lt - 1 (antiperiodic fermion boundary)
//   dir 4 + mu : U_mu(x - mu)^dag, times -1 when mu = t and x_t = 0
// Also written: U12 (two-slice kernels), rows 0 and 1 of the link without the boundary sign, and in
// *dev the largest deviation |row 2 - conj(row 0 x row 1)| over all links (as float bits; the
// two-row links stand for the links only when it is at rounding level).
__global__ void k_gauge(const double2* __restrict__ U, double* __restrict__ U64e, double* __restrict__ U64o,
                        float* __restrict__ U32e, float* __restrict__ U32o, float* __restrict__ U12e,
                        float* __restrict__ U12o, unsigned int* __restrict__ dev, const int* __restrict__ lex_e,
                        const int* __restrict__ lex_o, int Lx, int Ly, int Lz, int Lt, int Vh) {
    const int V = 2 * Vh;
    const int total = 2 * Vh * 8;
    float dmax = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int dir = i % 8;
        const int rest = i / 8;
        const int cb = rest % Vh;
        const int par = rest / Vh;
        const int lex = par ? lex_o[cb] : lex_e[cb];
        int c[4];
        c[0] = lex % Lx;
        c[1] = (lex / Lx) % Ly;
        c[2] = (lex / (Lx * Ly)) % Lz;
        c[3] = lex / (Lx * Ly * Lz);
        const int L[4] = {Lx, Ly, Lz, Lt};
        const int mu = dir & 3;
        double m[18];
        if (dir < 4) {
            const double sg = (mu == 3 && c[3] == Lt - 1) ? -1.0 : 1.0;
            const double2* src = U + ((size_t)mu * V + lex) * 9;
            for (int k = 0; k < 9; ++k) {
                m[2 * k] = sg * src[k].x;
                m[2 * k + 1] = sg * src[k].y;
            }
        } else {
            int d[4] = {c[0], c[1], c[2], c[3]};
            d[mu] = (d[mu] + L[mu] - 1) % L[mu];
            const int lexn = d[0] + Lx * (d[1] + Ly * (d[2] + Lz * d[3]));
            const double sg = (mu == 3 && c[3] == 0) ? -1.0 : 1.0;
            const double2* src = U + ((size_t)mu * V + lexn) * 9;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {  // (U^dag)_{ab} = conj(U_{ba})
                    m[(a * 3 + b) * 2] = sg * src[b * 3 + a].x;
                    m[(a * 3 + b) * 2 + 1] = -sg * src[b * 3 + a].y;
                }
        }
        double* d64 = (par ? U64o : U64e) + ((size_t)cb * 8 + dir) * 18;
        float* d32 = (par ? U32o : U32e) + ((size_t)cb * 8 + dir) * 20;
        for (int k = 0; k < 18; ++k) {
            d64[k] = m[k];
            d32[k] = (float)m[k];
        }
        d32[18] = 0.f;
        d32[19] = 0.f;
        // the unsigned link sg m: its first two rows, and how far its third row is from conj(row 0 x row 1)
        const double sg = (mu == 3 && c[3] == (dir < 4 ? Lt - 1 : 0)) ? -1.0 : 1.0;
        float* d12 = (par ? U12o : U12e) + ((size_t)cb * 8 + dir) * 12;
        for (int k = 0; k < 12; ++k) d12[k] = (float)(sg * m[k]);
        for (int k = 0; k < 3; ++k) {
            const int a = (k + 1) % 3, b = (k + 2) % 3;
            const double ar = m[2 * a], ai = m[2 * a + 1], br = m[6 + 2 * b], bi = m[6 + 2 * b + 1];
            const double cr = m[2 * b], ci = m[2 * b + 1], dr = m[6 + 2 * a], di = m[6 + 2 * a + 1];
            const double re = (ar * br - ai * bi) - (cr * dr - ci * di);
            const double im = (ar * bi + ai * br) - (cr * di + ci * dr);
            // sg^2 = 1: the cross product of the signed rows is that of the unsigned ones
            const double er = fabs(sg * m[12 + 2 * k] - re), ei = fabs(sg * m[13 + 2 * k] + im);
            dmax = fmaxf(dmax, (float)fmax(er, ei));
        }
    }
    if (!(dmax == dmax)) dmax = 3.0e38f;  // NaN links never qualify
    unsigned int bits = __float_as_uint(dmax);
    bits = __reduce_max_sync(0xffffffffu, bits);
    if ((threadIdx.x & 31) == 0) atomicMax(dev, bits);
}

int launch_gauge(odwf_s* h, const double* U, cudaStream_t st) {
    const int total = 2 * h->Vh * 8;
    int g = (total + 255) / 256;
    if (g > h->num_sms * 16) g = h->num_sms * 16;
    int rc = cuda_check(h, cudaMemsetAsync(h->u12_dev, 0, sizeof(unsigned int), st), "memset");
    if (rc) return rc;
    k_gauge<<<g, 256, 0, st>>>((const double2*)U, h->U64[0], h->U64[1], h->U32[0], h->U32[1], h->U12[0], h->U12[1],
                               h->u12_dev, h->lexof[0], h->lexof[1], h->L[0], h->L[1], h->L[2], h->L[3], h->Vh);
    if ((rc = cuda_check(h, cudaGetLastError(), "k_gauge"))) return rc;
    // the two-slice kernels take the two-row links only for SU(3) links (to well below FP32 rounding)
    if ((rc = cuda_check(h, cudaMemcpyAsync(h->u12_dev_host, h->u12_dev, sizeof(unsigned int), cudaMemcpyDeviceToHost, st),
                         "read link check")))
        return rc;
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "link check sync"))) return rc;
    float d;
    std::memcpy(&d, h->u12_dev_host, sizeof d);
    h->links12_ok = d < 1e-6f;
    return ODWF_OK;
}


// ---- autotuner ------------------------------------------------------------------------------------
// Times every launch choice (grid mode 0..3, bulk-staged or per-thread gather) of the four fused
// kernels of the CGNE iteration in one storage precision, on the handle's own lattice, and keeps
// the fastest per kernel. Inputs are the inner work fields filled with a constant byte pattern
// (finite, positive values), and a private solver state that never stops the kernels.
int autotune_storage(odwf_s* h, int stg, const SCoef* c, cudaStream_t st, std::vector<std::string>& log) {
    Workspace& w = h->ws;
    const size_t bi = half_elems_bytes(h, stg == ST_HALF ? ST_FLOAT : stg);
    const size_t bs = sizeof(float) * (size_t)h->Vh * h->Ns;
    void* fields[4] = {w.xi, w.ri, w.pi, w.ti};
    float* scales[4] = {w.xi_s, w.ri_s, w.pi_s, w.ti_s};
    auto fill = [&]() -> int {
        for (int i = 0; i < 4; ++i) {
            if (cudaMemsetAsync(fields[i], 0x3c, bi, st) != cudaSuccess) return ODWF_ECUDA;
            if (stg == ST_HALF && cudaMemsetAsync(scales[i], 0x3c, bs, st) != cudaSuccess) return ODWF_ECUDA;
        }
        CGState hs{};
        hs.rr = 1.0;
        hs.pp = 1.0;
        hs.alpha = 0.01;
        hs.beta = 0.5;
        hs.tol2 = -1.0;
        hs.rr_max = 1.0;
        hs.maxiter = 1 << 30;
        if (cudaMemcpyAsync(h->state, &hs, sizeof(CGState), cudaMemcpyHostToDevice, st) != cudaSuccess) return ODWF_ECUDA;
        return cudaStreamSynchronize(st) == cudaSuccess ? ODWF_OK : ODWF_ECUDA;
    };
    const int NN = h->Ns * h->Ns;
    struct V {
        const char* name;
        bool mixhop, own, mixown;
        int epi, parity;
    } vars[4] = {{"K1", true, false, false, EPI_STORE, 1},
                 {"K2A", false, true, true, EPI_CG_A, 0},
                 {"K2B", false, true, true, EPI_CG_B, 0},
                 {"K2", false, true, true, EPI_STORE, 0}};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool can_stage = staged_geom_ok(h, stg);
    const int saved_prof = h->prof;
    h->prof = false;
    for (const V& v : vars) {
        const int base_key = stg * 100000 + 1 * 10000 + v.mixhop * 1000 + v.own * 100 + v.mixown * 10 + v.epi;
        HopArgs a{};
        a.in = w.ti;
        a.in_scale = w.ti_s;
        a.own = w.pi;
        a.own_scale = w.pi_s;
        a.out = v.epi == EPI_STORE ? w.ti : nullptr;
        a.out_scale = w.ti_s;
        if (v.mixhop) {
            a.in = w.pi;
            a.in_scale = w.pi_s;
        }
        a.mhop = c->dev + (size_t)2 * NN;
        a.mown = c->dev;
        set_sop(a, c, v.mixhop ? SOP_AINV : SOP_A);
        a.c_hop = v.mixhop ? 1.0 : -0.25;
        a.x = w.xi;
        a.x_scale = w.xi_s;
        a.r = v.epi == EPI_CG_B ? w.pi : w.ri;
        a.r_scale = v.epi == EPI_CG_B ? w.pi_s : w.ri_s;
        if (v.epi == EPI_STORE && !v.mixhop) {
            a.out = w.ri;  // plain store variant writes r (a throw-away field here)
            a.out_scale = w.ri_s;
        }
        a.state = (v.epi == EPI_STORE) ? nullptr : h->state;
        float best = 1e30f;
        TuneChoice best_choice{};
        const int max_spbm = spb_for(h->Ns) * 2 * h->Ns <= 256 ? 2 : 1;
        // the structured and the dense fifth-dimension product where both exist (Ns = kStructNs), and
        // the two-slice kernel for the structured one
        const int max_dense = (h->Ns == kStructNs && a.sop != SOP_DENSE) ? 1 : 0;
        hop_fill(h, stg, v.parity, a, false);
        int max_pair = (max_dense && h->pair != 0 && pair_variant(stg, v.mixhop, v.own, v.mixown, v.epi) &&
                        pair_applies(h, stg, a)) ? 1 : 0;
        if (max_pair && pair_tma_applies(stg, a)) max_pair = 3;  // the bulk-copy forms with 2 and 3 stages
        for (int dense = 0; dense <= max_dense; ++dense)
        for (int pair = 0; pair <= (dense ? 0 : max_pair); ++pair)
        for (int spbm = 1; spbm <= (pair >= 2 ? 1 : max_spbm); ++spbm)
        for (int staged = 0; staged <= (can_stage && !dense && !pair ? 1 : 0); ++staged)
            for (int mode = 0; mode < 4; ++mode) {
                TuneChoice tc;
                tc.mode = mode;
                tc.staged = staged;
                tc.spbm = spbm;
                tc.dense = dense;
                tc.pair = pair;
                h->tune[base_key] = tc;
                int rc = fill();
                if (rc) return set_err(h, rc, "autotune: fill");
                for (int k = 0; k < 2; ++k)
                    if ((rc = launch_hop(h, stg, v.parity, v.mixhop, v.own, v.mixown, v.epi, a, st))) return rc;
                cudaEventRecord(e0, st);
                const int reps = 10;
                for (int k = 0; k < reps; ++k)
                    if ((rc = launch_hop(h, stg, v.parity, v.mixhop, v.own, v.mixown, v.epi, a, st))) return rc;
                cudaEventRecord(e1, st);
                if ((rc = cuda_check(h, cudaEventSynchronize(e1), "autotune sync"))) return rc;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= reps;
                char buf[160];
                std::snprintf(buf, sizeof buf, "%s storage %d %s%s tile x%d staged %d grid-mode %d: %.1f us", v.name,
                              stg, dense ? "dense" : "structured",
                              pair == 1 ? " two-slice" : (pair == 2 ? " two-slice bulk x2" : (pair == 3 ? " two-slice bulk x3" : "")),
                              spbm, staged, mode, 1e3 * ms);
                log.push_back(buf);
                if (ms < best) {
                    best = ms;
                    best_choice = tc;
                }
            }
        h->tune[base_key] = best_choice;
    }
    h->prof = saved_prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ODWF_OK;
}
}  // namespace odwf
